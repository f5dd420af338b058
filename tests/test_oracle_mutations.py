"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each.

Every case monkeypatches one oracle function with a subtly wrong variant (a
dropped normalisation, transposed fractions, a flipped sign, a missing
conjugate) and re-runs a pin from test_oracle_pins; the pin must fail.
"""
import inspect
import textwrap

import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from tests import test_oracle_pins as pins


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def _rewritten(fn, old, new):
    """`fn` recompiled with the source fragment `old` replaced by `new` (exactly
    one occurrence), resolving names in a copy of the oracle module's globals."""
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, old
    ns = dict(fn.__globals__)
    exec(compile(src.replace(old, new), "<planted mistake>", "exec"), ns)
    return ns[fn.__name__]


def test_missing_fft_normalisation_is_caught(monkeypatch):
    monkeypatch.setattr(orc, "dft2", lambda x: np.fft.fft2(np.asarray(x, complex)))
    _fails(pins.test_dft2_parseval_and_inverse)
    _fails(pins.test_dft2_matches_bruteforce_definition, 8)


def test_transposed_bilinear_fractions_are_caught(monkeypatch):
    real = orc.tile_origin

    def swapped(r, N):
        t, f = real(r, N)
        return t, f[::-1]

    monkeypatch.setattr(orc, "tile_origin", swapped)
    _fails(pins.test_bilinear_reproduces_affine_functions_exactly)


def test_flipped_exit_wave_change_is_caught(monkeypatch):
    real = orc.modulus_ratio
    monkeypatch.setattr(orc, "modulus_ratio", lambda I, Im, n, e: 2.0 - real(I, Im, n, e))
    _fails(pins.test_eq2_object_gradient_is_minus_twice_conj_probe_times_exit_wave_change)


def test_wrong_cross_term_sign_in_step_solve_is_caught(monkeypatch):
    real = orc.step_solve
    monkeypatch.setattr(orc, "step_solve", lambda a, c, d, b1, b2, lam: real(a, -c, d, b1, b2, lam))
    _fails(pins.test_step_sizes_solve_the_least_squares_problem)


def test_missing_probe_conjugate_in_gradient_is_caught(monkeypatch):
    real_vjp = orc.vjp

    def wrong(O, P, pos, G):
        gO, gP, gr = real_vjp(O, P, pos, G)
        # recompute the object gradient with P instead of conj(P)
        H, W = O.shape
        N = P.shape[-1]
        gO = np.zeros((H, W), complex)
        for j in range(pos.shape[0]):
            o = orc.extract(O, pos[j], N)
            gpsi = orc.idft2(2.0 * G[j][None] * orc.dft2(P * o[None]))
            gO += orc.scatter(np.sum(P * gpsi, axis=0), pos[j], H, W)
        return gO, gP, gr

    monkeypatch.setattr(orc, "vjp", wrong)
    _fails(pins.test_gradients_match_central_finite_differences, orc.GAUSSIAN)


def test_eigenmodes_paired_with_the_wrong_weights_are_caught(monkeypatch):
    real = orc.opr_primary
    monkeypatch.setattr(orc, "opr_primary", lambda U, w_j: real(U, np.asarray(w_j)[::-1]))
    _fails(pins.test_opr_unit_weights_select_one_eigenmode)


def test_weight_update_of_the_wrong_sign_is_caught(monkeypatch):
    real = orc.weight_solve
    monkeypatch.setattr(orc, "weight_solve", lambda A, b, lam: -real(A, b, lam))
    _fails(pins.test_lsqml_opr_truth_is_a_fixed_point_and_weights_converge)


def test_position_step_with_swapped_derivatives_is_caught(monkeypatch):
    real = orc.extract_dr
    monkeypatch.setattr(orc, "extract_dr", lambda O, r, N: real(O, r, N)[::-1])
    _fails(pins.test_position_correction_converges_to_the_true_positions)


def test_per_epoch_update_applied_per_batch_is_caught(monkeypatch):
    real = orc.lsqml_batch

    def per_batch(O, P, pos, I_m, idx, opts, record=None):
        import dataclasses
        return real(O, P, pos, I_m, idx, dataclasses.replace(opts, object_per_epoch=False), record)

    monkeypatch.setattr(orc, "lsqml_batch", per_batch)
    _fails(pins.test_per_epoch_object_update_does_not_depend_on_the_batch_order)


def test_propagator_of_the_wrong_handedness_is_caught(monkeypatch):
    real = orc.asm_propagator
    monkeypatch.setattr(orc, "asm_propagator", lambda *a: np.conj(real(*a)))
    _fails(pins.test_asm_propagator_properties)


def test_poisson_full_likelihood_step_is_caught(monkeypatch):
    real = orc.modulus_ratio

    def full_step(I, Im, n, e):
        if n == orc.POISSON:
            return Im / (I + e)
        return real(I, Im, n, e)

    monkeypatch.setattr(orc, "modulus_ratio", full_step)
    _fails(pins.test_lsqml_accumulators_are_fixed_multiples_of_the_finite_difference_gradients,
           orc.POISSON, -0.25)


def test_probe_direction_without_the_object_conjugate_is_caught(monkeypatch):
    wrong = _rewritten(orc.lsqml_batch, "dP_acc += np.conj(o)[None] * chi", "dP_acc += o[None] * chi")
    monkeypatch.setattr(orc, "lsqml_batch", wrong)
    _fails(pins.test_lsqml_accumulators_are_fixed_multiples_of_the_finite_difference_gradients,
           orc.GAUSSIAN, -0.5)
    _fails(pins.test_probe_only_update_has_the_closed_form_of_a_known_object, 1)


def test_probe_step_summed_instead_of_averaged_is_caught(monkeypatch):
    wrong = _rewritten(orc.lsqml_batch, "float(np.mean(alpha[:, 1]))", "float(np.sum(alpha[:, 1]))")
    monkeypatch.setattr(orc, "lsqml_batch", wrong)
    _fails(pins.test_probe_only_update_has_the_closed_form_of_a_known_object, 2)


def test_probe_damping_from_the_illumination_is_caught(monkeypatch):
    wrong = _rewritten(orc.lsqml_batch, "opts.delta_p * float(np.max(Dp))", "opts.delta_p * float(np.max(illum))")
    monkeypatch.setattr(orc, "lsqml_batch", wrong)
    _fails(pins.test_probe_only_update_has_the_closed_form_of_a_known_object, 1)


def test_multislice_lsqml_backpropagation_with_the_forward_propagator_is_caught(monkeypatch):
    wrong = _rewritten(orc.lsqml_batch_ms, "chi = propagate(chi, Hc)", "chi = propagate(chi, Hf)")
    monkeypatch.setattr(orc, "lsqml_batch_ms", wrong)
    _fails(pins.test_multislice_lsqml_accumulators_are_multiples_of_the_finite_difference_gradients,
           orc.GAUSSIAN, -0.5)


def test_multislice_lsqml_backpropagation_without_the_slice_conjugate_is_caught(monkeypatch):
    wrong = _rewritten(orc.lsqml_batch_ms, "chi = np.conj(o[s])[None] * chi", "chi = o[s][None] * chi")
    monkeypatch.setattr(orc, "lsqml_batch_ms", wrong)
    _fails(pins.test_multislice_lsqml_accumulators_are_multiples_of_the_finite_difference_gradients,
           orc.GAUSSIAN, -0.5)


def test_multislice_lsqml_probe_damping_from_the_last_slice_is_caught(monkeypatch):
    wrong = _rewritten(orc.lsqml_batch_ms, "Dp += np.abs(o[0]) ** 2", "Dp += np.abs(o[-1]) ** 2")
    monkeypatch.setattr(orc, "lsqml_batch_ms", wrong)
    _fails(pins.test_multislice_probe_only_update_has_the_closed_form_of_a_known_object)


def test_multislice_lsqml_tangent_without_the_slice_sources_is_caught(monkeypatch):
    wrong = _rewritten(orc.lsqml_batch_ms,
                       "u = propagate(u, Hf) * o[s][None] + inc[s] * extract(dO_hat[s], pos[j], N)[None]",
                       "u = propagate(u, Hf) * o[s][None]")
    monkeypatch.setattr(orc, "lsqml_batch_ms", wrong)
    _fails(pins.test_multislice_lsqml_step_sizes_fit_the_exit_plane_change_by_finite_difference_tangents)
