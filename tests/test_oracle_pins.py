"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

Each test checks the oracle against something other than itself: a brute-force
DFT, Parseval's identity, exact reproduction of affine functions by bilinear
interpolation, adjoint dot products, closed-form far fields, central finite
differences, a library least-squares solve of the step-size problem, the
single-position reduction to plain CDI, and convergence on noiseless data.
"""
import math

import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2510_20929_gb300 import synth


def crandn(g, *shape):
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


# --------------------------------------------------------------------------- DFT
@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_dft2_matches_bruteforce_definition(N):
    g = np.random.default_rng(N)
    x = crandn(g, N, N)
    X = orc.dft2(x)
    a = np.arange(N)
    ref = np.zeros((N, N), complex)
    for u in range(N):
        for v in range(N):
            ph = np.exp(-2j * math.pi * (u * a[:, None] + v * a[None, :]) / N)
            ref[u, v] = np.sum(x * ph) / N
    assert np.max(np.abs(X - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_dft2_parseval_and_inverse():
    g = np.random.default_rng(1)
    x = crandn(g, 3, 32, 32)
    X = orc.dft2(x)
    assert abs(np.sum(np.abs(X) ** 2) - np.sum(np.abs(x) ** 2)) < 1e-10 * np.sum(np.abs(x) ** 2)
    assert np.max(np.abs(orc.idft2(X) - x)) < 1e-12


# --------------------------------------------------------------------------- S_j
def test_integer_position_is_a_crop():
    g = np.random.default_rng(2)
    O = crandn(g, 30, 37)
    N = 8
    r = np.array([13.0, 21.0])            # t = (9, 17), f = 0
    o = orc.extract(O, r, N)
    assert np.array_equal(o, O[9:17, 17:25])


def test_bilinear_reproduces_affine_functions_exactly():
    H, W, N = 33, 41, 8
    yy, xx = np.meshgrid(np.arange(H, dtype=float), np.arange(W, dtype=float), indexing="ij")
    c0, cy, cx = 0.3 - 0.2j, 1.7 + 0.4j, -0.9 + 2.1j
    O = c0 + cy * yy + cx * xx
    r = np.array([15.37, 19.81])
    o = orc.extract(O, r, N)
    a = np.arange(N, dtype=float)
    ey = r[0] - N / 2 + a[:, None]        # exact sample coordinates t + f + a
    ex = r[1] - N / 2 + a[None, :]
    assert np.max(np.abs(o - (c0 + cy * ey + cx * ex))) < 1e-12
    d_dy, d_dx = orc.extract_dr(O, r, N)
    assert np.max(np.abs(d_dy - cy)) < 1e-12 and np.max(np.abs(d_dx - cx)) < 1e-12


def test_scatter_is_the_adjoint_of_extract():
    g = np.random.default_rng(3)
    H, W, N = 29, 34, 8
    O = crandn(g, H, W)
    y = crandn(g, N, N)
    r = np.array([12.61, 17.29])
    lhs = np.vdot(y, orc.extract(O, r, N))
    rhs = np.vdot(orc.scatter(y, r, H, W), O)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    # partition of unity: the weights of each patch pixel sum to one
    assert abs(np.sum(orc.scatter(np.ones((N, N)), r, H, W)) - N * N) < 1e-11


def test_extract_dr_matches_central_differences():
    g = np.random.default_rng(4)
    O = crandn(g, 30, 30)
    N, r, h = 8, np.array([14.3, 13.6]), 1e-6
    d_dy, d_dx = orc.extract_dr(O, r, N)
    fy = (orc.extract(O, r + [h, 0], N) - orc.extract(O, r - [h, 0], N)) / (2 * h)
    fx = (orc.extract(O, r + [0, h], N) - orc.extract(O, r - [0, h], N)) / (2 * h)
    assert np.max(np.abs(fy - d_dy)) < 1e-8 and np.max(np.abs(fx - d_dx)) < 1e-8


def test_bounds_rule():
    assert orc.in_bounds([4.0, 4.0], 8, 9, 9)         # t = 0, t + N + 1 = 9
    assert not orc.in_bounds([3.9, 4.0], 8, 9, 9)     # t = -1
    assert not orc.in_bounds([5.0, 4.0], 8, 9, 9)     # t + N + 1 = 10 > 9


# --------------------------------------------------------------------------- forward model
def test_forward_parseval_over_modes():
    w = synth.workload_small(N=16, M=3, J=5)
    I = orc.forward(w["object"], w["probe"], w["pos"])
    for j in range(5):
        o = orc.extract(w["object"], w["pos"][j], 16)
        ref = np.sum(np.abs(w["probe"] * o[None]) ** 2)
        assert abs(I[j].sum() - ref) < 1e-11 * ref


def test_forward_plane_wave_closed_form():
    # probe = plane wave with frequency (u0, v0), object constant c -> a single
    # bright pixel of intensity N^2 |c|^2 at (u0, v0), zero elsewhere
    N, u0, v0, c = 16, 3, 11, 0.7 - 0.4j
    a = np.arange(N)
    P = np.exp(2j * math.pi * (u0 * a[:, None] + v0 * a[None, :]) / N)[None]
    O = np.full((40, 40), c)
    I = orc.forward(O, P, np.array([[20.3, 19.6]]))[0]
    ref = np.zeros((N, N))
    ref[u0, v0] = N * N * abs(c) ** 2
    assert np.max(np.abs(I - ref)) < 1e-10


def test_forward_delta_probe_closed_form():
    # probe = delta at (a0, b0) -> flat pattern |o(a0, b0)|^2 / N^2
    N, a0, b0 = 8, 2, 5
    P = np.zeros((1, N, N), complex)
    P[0, a0, b0] = 1.0
    g = np.random.default_rng(5)
    O = crandn(g, 20, 20)
    r = np.array([9.25, 10.5])
    o = orc.extract(O, r, N)
    I = orc.forward(O, P, r[None])[0]
    assert np.max(np.abs(I - abs(o[a0, b0]) ** 2 / N ** 2)) < 1e-13


# --------------------------------------------------------------------------- gradients
def _fd_problem(noise, seed=6):
    g = np.random.default_rng(seed)
    w = synth.workload_small(N=8, M=2, H=24, W=24, J=4, seed=seed, step=3.0)
    O_true, P, pos = w["object"], w["probe"], w["pos"]
    I_m = synth.poisson_counts(50.0 * orc.forward(O_true, P, pos) / orc.forward(O_true, P, pos).mean(), seed)
    P = P * math.sqrt(50.0 / orc.forward(O_true, P, pos).mean())
    O = O_true * (1 + 0.1 * crandn(g, *O_true.shape))
    return O, P, pos, I_m


@pytest.mark.parametrize("noise", [orc.GAUSSIAN, orc.POISSON])
def test_gradients_match_central_finite_differences(noise):
    O, P, pos, I_m = _fd_problem(noise)
    eps = 1e-3
    L, gO, gP, gr = orc.loss_and_gradients(O, P, pos, I_m, noise, eps)
    g = np.random.default_rng(7)
    h = 1e-6

    def L_at(O_, P_, pos_):
        return orc.loss_and_gradients(O_, P_, pos_, I_m, noise, eps)[0]

    dO = crandn(g, *O.shape)
    fd = (L_at(O + h * dO, P, pos) - L_at(O - h * dO, P, pos)) / (2 * h)
    assert abs(fd - np.real(np.vdot(gO, dO))) < 1e-6 * abs(fd)
    dP = crandn(g, *P.shape)
    fd = (L_at(O, P + h * dP, pos) - L_at(O, P - h * dP, pos)) / (2 * h)
    assert abs(fd - np.real(np.vdot(gP, dP))) < 1e-6 * abs(fd)
    dr = g.standard_normal(pos.shape)
    fd = (L_at(O, P, pos + h * dr) - L_at(O, P, pos - h * dr)) / (2 * h)
    assert abs(fd - np.sum(gr * dr)) < 1e-5 * abs(fd)


def test_eq2_object_gradient_is_minus_twice_conj_probe_times_exit_wave_change():
    # Eq. 2: dL/do* = -p* (psi' - psi) per patch (unnormalised), i.e. the
    # PyTorch-convention gradient is -2 sum_k P_k* chi_k, and the LSQML object
    # accumulator is minus half the object gradient.
    O, P, pos, I_m = _fd_problem(orc.GAUSSIAN, seed=8)
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=4, eps=1e-3)
    rec = {}
    orc.lsqml_batch(O, P, pos, I_m, range(4), opts, rec)
    _, gO, _, _ = orc.loss_and_gradients(O, P, pos, I_m, orc.GAUSSIAN, 1e-3)
    assert np.max(np.abs(rec["dO_acc"] + 0.5 * gO)) < 1e-10 * np.max(np.abs(gO))
    # psi' - psi computed the long way round: back-propagate the replaced modulus
    o = orc.extract(O, pos[0], 8)
    psi = P * o[None]
    Psi = orc.dft2(psi)
    I = np.sum(np.abs(Psi) ** 2, axis=0)
    psi_new = orc.idft2(Psi * np.sqrt(I_m[0]) / np.sqrt(I + 1e-3))
    assert np.max(np.abs(rec["chi"][0] - (psi_new - psi))) < 1e-12


def test_loss_and_gradient_vanish_at_the_truth():
    w = synth.workload_small(N=8, M=2, H=24, W=24, J=4, step=3.0)
    I = orc.forward(w["object"], w["probe"], w["pos"])
    L, gO, gP, gr = orc.loss_and_gradients(w["object"], w["probe"], w["pos"], I, orc.GAUSSIAN, 0.0)
    assert L < 1e-20 and np.max(np.abs(gO)) < 1e-10 and np.max(np.abs(gr)) < 1e-9


def test_gradient_is_sum_over_position_subsets():
    # Sec. 2.3: summing per-worker gradients equals the full-batch gradient.
    O, P, pos, I_m = _fd_problem(orc.GAUSSIAN, seed=9)
    _, gO, gP, gr = orc.loss_and_gradients(O, P, pos, I_m, orc.GAUSSIAN, 1e-3)
    parts = [orc.loss_and_gradients(O, P, pos[s], I_m[s], orc.GAUSSIAN, 1e-3) for s in ([0, 3], [1, 2])]
    assert np.max(np.abs(parts[0][1] + parts[1][1] - gO)) < 1e-12 * np.max(np.abs(gO))
    assert np.max(np.abs(parts[0][2] + parts[1][2] - gP)) < 1e-12 * np.max(np.abs(gP))


# --------------------------------------------------------------------------- LSQML step sizes
def test_step_sizes_solve_the_least_squares_problem():
    # alpha_j minimises sum_k ||chi_jk - a_O u_jk - a_P v_jk||^2; compare every
    # position of a batch with numpy's least-squares on the stacked real system.
    O, P, pos, I_m = _fd_problem(orc.GAUSSIAN, seed=10)
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=4, eps=1e-3, lam=0.0)
    rec = {}
    _, _, _, alpha = orc.lsqml_batch(O, P, pos, I_m, range(4), opts, rec)
    for j in range(4):
        u = (orc.extract(rec["dO_hat"], pos[j], 8)[None] * P).ravel()
        v = (orc.extract(O, pos[j], 8)[None] * rec["dP"]).ravel()
        chi = rec["chi"][j].ravel()
        Amat = np.concatenate([np.stack([u.real, v.real], 1), np.stack([u.imag, v.imag], 1)])
        bvec = np.concatenate([chi.real, chi.imag])
        ref = np.linalg.lstsq(Amat, bvec, rcond=None)[0]
        assert np.max(np.abs(alpha[j] - ref)) < 1e-8 * np.max(np.abs(ref))


def test_step_solve_grid_search_and_fallbacks():
    g = np.random.default_rng(11)
    u, v, chi = crandn(g, 50), crandn(g, 50), crandn(g, 50)
    A11, A22 = np.sum(abs(u) ** 2), np.sum(abs(v) ** 2)
    A12 = np.real(np.vdot(u, v))
    b1, b2 = np.real(np.vdot(u, chi)), np.real(np.vdot(v, chi))
    a = np.array(orc.step_solve(A11, A12, A22, b1, b2, 0.0))
    q = lambda x: np.sum(np.abs(chi - x[0] * u - x[1] * v) ** 2)
    grid = np.linspace(-0.05, 0.05, 101)
    best = min(q(a + [dy, dx]) for dy in grid for dx in grid)
    assert q(a) <= best + 1e-12
    # a zero second direction reduces to the 1x1 solve b1 / A11 (lam = 0: det = 0)
    assert orc.step_solve(A11, 0.0, 0.0, b1, 0.0, 0.0) == (b1 / A11, 0.0)
    assert orc.step_solve(0.0, 0.0, 0.0, 0.0, 0.0, 1e-6) == (0.0, 0.0)


def test_single_position_reduces_to_plain_cdi():
    # One position at an integer offset, probe known: the LSQML object update
    # is alpha * conj(P) chi / (|P|^2 + delta) on the patch, with the 1x1 step
    # alpha = Re<u, chi> / ||u||^2 (lam = 0, probe not updated).
    g = np.random.default_rng(12)
    N, H, W = 16, 24, 26
    P = synth.gaussian_probe(N, sigma=4.0, quad_phase=0.05) * 3.0
    O_true = synth.make_object(H, W, 3, phase_sigma=1.0)
    r = np.array([12.0, 13.0])                           # t = (4, 5), f = 0
    I_m = orc.forward(O_true, P, r[None])
    O = O_true * (1 + 0.2 * crandn(g, H, W))
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=1, delta_o=1e-2, lam=0.0,
                            update_probe=False)
    O_new, P_new, loss, alpha = orc.lsqml_batch(O, P, r[None], I_m, [0], opts)
    # plain single-view CDI on the crop, written without S_j or the batch sums
    p = P[0]
    o = O[4:20, 5:21]
    Psi = np.fft.fft2(p * o) / N
    Psi_new = np.sqrt(I_m[0]) * np.exp(1j * np.angle(Psi))
    chi = np.fft.ifft2(Psi_new) * N - p * o
    w = np.abs(p) ** 2 + 1e-2 * np.max(np.abs(p) ** 2)
    d = np.conj(p) * chi / w
    u = d * p
    a = np.real(np.vdot(u, chi)) / np.vdot(u, u).real
    ref = O.copy()
    ref[4:20, 5:21] += a * d
    assert abs(alpha[0, 0] - a) < 1e-10 * abs(a) and alpha[0, 1] == 0.0
    assert np.max(np.abs(O_new - ref)) < 1e-12
    assert np.array_equal(P_new, P)


# --------------------------------------------------------------------------- whole iteration
def _noiseless_problem(probe_error):
    N, H, W = 32, 80, 80
    O_true = synth.make_object(H, W, 21, phase_sigma=2.0, amp_sigma=2.0)
    P_true = synth.gaussian_probe(N, sigma=5.0, quad_phase=0.02) * 4.0
    pos = synth.raster_positions(7, 7, 5.0, (H / 2, W / 2), 0.5, 22)
    I_m = orc.forward(O_true, P_true, pos)
    O0 = np.ones((H, W), complex)
    ramp = 1 + probe_error * (np.arange(N)[None, :, None] / N)
    return O_true, P_true, pos, I_m, O0, P_true * ramp


def test_lsqml_converges_to_the_truth_on_noiseless_data():
    # known probe, flat start, random minibatches of 16: the object converges to
    # the truth up to the global phase, and the loss falls by three decades
    O_true, P, pos, I_m, O, _ = _noiseless_problem(0.0)
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=16, eps=1e-12, delta_o=0.1,
                            update_probe=False)
    order = synth.random_order(pos.shape[0], 5)
    illum = sum(orc.scatter(np.abs(P[0]) ** 2, r, *O.shape) for r in pos)
    mask = illum > 0.5 * illum.max()

    def err(O_):
        A = orc.align_global_phase(O_, O_true, mask)
        return np.linalg.norm((A - O_true)[mask]) / np.linalg.norm(O_true[mask])

    e0 = err(O)
    losses = []
    for _ in range(40):
        O, _, L, _ = orc.lsqml_epoch(O, P, pos, I_m, order, opts)
        losses.append(L)
    assert err(O) < 0.02 * e0
    assert losses[-1] < 1e-3 * losses[0]


def test_lsqml_joint_probe_update_reduces_the_loss():
    O_true, P_true, pos, I_m, O, P = _noiseless_problem(0.1)
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=16, eps=1e-12, delta_o=0.1, delta_p=0.1)
    order = synth.random_order(pos.shape[0], 6)
    losses = []
    for _ in range(10):
        O, P, L, _ = orc.lsqml_epoch(O, P, pos, I_m, order, opts)
        losses.append(L)
    assert losses[-1] < 0.02 * losses[0]


def test_poisson_lsqml_reduces_the_loss():
    O_true, P, pos, I_m, O, _ = _noiseless_problem(0.0)
    I_m = synth.poisson_counts(I_m, 3)
    opts = orc.LsqmlOptions(noise=orc.POISSON, batch=16, eps=1e-6, delta_o=0.1,
                            update_probe=False)
    order = synth.random_order(pos.shape[0], 7)
    losses = []
    for _ in range(6):
        O, _, L, _ = orc.lsqml_epoch(O, P, pos, I_m, order, opts)
        losses.append(L)
    assert losses[-1] < losses[0]


# --------------------------------------------------------------------------- orthogonal probe relaxation
def _opr_problem(seed=13):
    g = np.random.default_rng(seed)
    w = synth.workload_small(N=8, M=3, H=24, W=24, J=4, seed=seed, step=3.0)
    P = w["probe"] * 3.0
    U = np.stack([P[0], 0.3 * P[1] * np.exp(0.4j)])             # two eigenmodes of the primary mode
    wts = 1.0 + 0.1 * g.standard_normal((4, 2))
    I_m = synth.poisson_counts(orc.forward_opr(w["object"], U, wts, P[1:], w["pos"]), seed)
    O = w["object"] * (1 + 0.1 * crandn(g, 24, 24))
    return O, U, wts, P[1:], w["pos"], I_m


def test_opr_with_one_unit_weight_mode_is_the_shared_probe_model():
    O, U, wts, P_rest, pos, I_m = _opr_problem()
    U1, w1 = U[:1], np.ones((4, 1))
    P = np.concatenate([U1, P_rest])
    assert np.max(np.abs(orc.forward_opr(O, U1, w1, P_rest, pos) - orc.forward(O, P, pos))) < 1e-12
    G = np.random.default_rng(2).standard_normal(I_m.shape)
    gO, gU, gw, gP, gr = orc.vjp_opr(O, U1, w1, P_rest, pos, G)
    gO_ref, gP_ref, gr_ref = orc.vjp(O, P, pos, G)
    assert np.max(np.abs(gO - gO_ref)) < 1e-10 and np.max(np.abs(gr - gr_ref)) < 1e-10
    assert np.max(np.abs(gU[0] - gP_ref[0])) < 1e-10 and np.max(np.abs(gP - gP_ref[1:])) < 1e-10


def test_opr_unit_weights_select_one_eigenmode():
    # w_j = e_m makes U_m the primary mode of every position (the plain model)
    O, U, wts, P_rest, pos, I_m = _opr_problem()
    for m in range(U.shape[0]):
        e = np.zeros((4, U.shape[0]))
        e[:, m] = 1.0
        ref = orc.forward(O, np.concatenate([U[m:m + 1], P_rest]), pos)
        assert np.max(np.abs(orc.forward_opr(O, U, e, P_rest, pos) - ref)) < 1e-12 * np.max(ref)


def test_opr_gradients_match_central_finite_differences():
    O, U, wts, P_rest, pos, I_m = _opr_problem()
    L, gO, gU, gw, gP, gr = orc.loss_and_gradients_opr(O, U, wts, P_rest, pos, I_m, orc.GAUSSIAN, 1e-3)
    g = np.random.default_rng(3)
    h = 1e-6

    def L_at(U_, w_):
        return orc.loss_and_gradients_opr(O, U_, w_, P_rest, pos, I_m, orc.GAUSSIAN, 1e-3)[0]

    dU = crandn(g, *U.shape)
    fd = (L_at(U + h * dU, wts) - L_at(U - h * dU, wts)) / (2 * h)
    assert abs(fd - np.real(np.vdot(gU, dU))) < 1e-6 * abs(fd)
    dw = g.standard_normal(wts.shape)
    fd = (L_at(U, wts + h * dw) - L_at(U, wts - h * dw)) / (2 * h)
    assert abs(fd - np.sum(gw * dw)) < 1e-6 * abs(fd)


def test_lsqml_opr_with_one_unit_weight_mode_is_plain_lsqml():
    O, U, wts, P_rest, pos, I_m = _opr_problem()
    P = np.concatenate([U[:1], P_rest])
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=4, eps=1e-3, delta_o=0.1, delta_p=0.1)
    idx = [2, 0, 3, 1]
    O1, P1, L1, a1 = orc.lsqml_batch(O, P, pos, I_m, idx, opts)
    O2, U2, w2, Pr2, L2, a2 = orc.lsqml_batch_opr(O, U[:1], np.ones((4, 1)), P_rest, pos, I_m, idx, opts,
                                                  orc.OprOptions(update_weights=False))
    assert abs(L1 - L2) < 1e-12 * abs(L1)
    assert np.max(np.abs(a1 - a2)) < 1e-10 * np.max(np.abs(a1))
    assert np.max(np.abs(O1 - O2)) < 1e-12
    assert np.max(np.abs(P1 - np.concatenate([U2, Pr2]))) < 1e-12
    assert np.all(w2 == 1.0)


def test_lsqml_opr_is_equivariant_under_weight_rescaling():
    # (s w, U / s) is the same probe family: with no probe damping and no
    # regularisation (whose trace term mixes the modes' scales) the batch
    # update maps to the rescaled update of (w, U)
    O, U, wts, P_rest, pos, I_m = _opr_problem()
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=4, eps=1e-3, delta_o=0.1, delta_p=0.0, lam=0.0)
    opr = orc.OprOptions(update_weights=True, weight_step=0.7)
    idx = [1, 3, 0, 2]
    s = np.array([2.5, 0.4])
    O1, U1, w1, Pr1, L1, a1 = orc.lsqml_batch_opr(O, U, wts, P_rest, pos, I_m, idx, opts, opr)
    O2, U2, w2, Pr2, L2, a2 = orc.lsqml_batch_opr(O, U / s[:, None, None], wts * s[None], P_rest, pos, I_m,
                                                  idx, opts, opr)
    assert abs(L1 - L2) < 1e-11 * abs(L1)
    assert np.max(np.abs(a1 - a2)) < 1e-9 * np.max(np.abs(a1))
    assert np.max(np.abs(O1 - O2)) < 1e-11
    assert np.max(np.abs(U1 - U2 * s[:, None, None])) < 1e-11 * np.max(np.abs(U1))
    assert np.max(np.abs(w1 - w2 / s[None])) < 1e-11
    assert np.max(np.abs(Pr1 - Pr2)) < 1e-12


def _opr_noiseless(seed=17):
    g = np.random.default_rng(seed)
    N, H, W, J = 16, 48, 48, 25
    O = synth.make_object(H, W, seed, phase_sigma=2.0, amp_sigma=2.0)
    modes = synth.hg_probe(N, [0.6, 0.2, 0.15, 0.05], waist=3.5, quad_phase=0.02) * 6.0
    U, P_rest = modes[:3], modes[3:]
    pos = synth.raster_positions(5, 5, 4.0, (H / 2, W / 2), 0.5, seed)
    w_true = 1.0 + 0.1 * g.standard_normal((J, 3))
    I_m = orc.forward_opr(O, U, w_true, P_rest, pos)
    return O, U, w_true, P_rest, pos, I_m, g


def test_lsqml_opr_truth_is_a_fixed_point_and_weights_converge():
    O, U, w_true, P_rest, pos, I_m, g = _opr_noiseless()
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=5, eps=0.0, delta_o=0.1, delta_p=0.1,
                            update_object=False, update_probe=False)
    opr = orc.OprOptions(update_weights=True)
    order = synth.random_order(pos.shape[0], 3)
    O1, U1, w1, Pr1, L, _ = orc.lsqml_epoch_opr(O, U, w_true, P_rest, pos, I_m, order, opts, opr)
    assert L < 1e-20 and np.max(np.abs(w1 - w_true)) < 1e-12 and np.max(np.abs(O1 - O)) == 0.0
    w = w_true + 0.05 * g.standard_normal(w_true.shape)
    e0 = np.linalg.norm(w - w_true)
    for _ in range(12):   # linear convergence, about 0.77 per epoch
        _, _, w, _, L, _ = orc.lsqml_epoch_opr(O, U, w, P_rest, pos, I_m, order, opts, opr)
    assert np.linalg.norm(w - w_true) < 0.05 * e0


# --------------------------------------------------------------------------- position correction, per-epoch object update
def test_position_step_solves_the_least_squares_problem():
    # the closed-form 2x2 system equals numpy's least squares on the stacked
    # real system sum_k ||chi_k - P_k (d_y dr_y + d_x dr_x)||^2
    g = np.random.default_rng(21)
    O = synth.make_object(40, 40, 4, phase_sigma=1.5)
    P = crandn(g, 2, 12, 12)
    r = np.array([19.3, 20.6])
    chi = crandn(g, 2, 12, 12)
    d_y, d_x = orc.extract_dr(O, r, 12)
    cols = [np.concatenate([np.real(P * d[None]).ravel(), np.imag(P * d[None]).ravel()]) for d in (d_y, d_x)]
    rhs = np.concatenate([np.real(chi).ravel(), np.imag(chi).ravel()])
    ref = np.linalg.lstsq(np.stack(cols, axis=1), rhs, rcond=None)[0]
    got = orc.position_step(O, P, r, np.sum(np.conj(P) * chi, axis=0), 0.0)
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))


def _position_problem(seed=31):
    N, H, W = 16, 64, 64
    O = synth.make_object(H, W, seed, phase_sigma=2.0, amp_sigma=2.0)
    P = synth.gaussian_probe(N, sigma=3.0, quad_phase=0.05) * 5.0
    pos_true = synth.raster_positions(6, 6, 5.0, (H / 2, W / 2), 0.4, seed)
    I_m = orc.forward(O, P, pos_true)
    g = np.random.default_rng(seed)
    pos0 = pos_true + g.uniform(-1.0, 1.0, pos_true.shape)
    return O, P, pos_true, pos0, I_m


def test_position_correction_converges_to_the_true_positions():
    O, P, pos_true, pos, I_m = _position_problem()
    opts = orc.LsqmlOptions(batch=6, eps=0.0, update_object=False, update_probe=False, update_positions=True,
                            pos_step=1.0, pos_max_shift=1.0)
    order = synth.random_order(pos.shape[0], 2)
    e0 = np.sqrt(np.mean((pos - pos_true) ** 2))
    for _ in range(15):   # linear convergence, about 0.75 per epoch
        _, _, pos, _, _ = orc.lsqml_epoch_state(O, P, pos, I_m, order, opts)
    e = np.sqrt(np.mean((pos - pos_true) ** 2))
    assert e < 0.05 * e0
    # the truth is a fixed point
    _, _, p1, _, _ = orc.lsqml_epoch_state(O, P, pos_true, I_m, order, opts)
    assert np.max(np.abs(p1 - pos_true)) < 1e-9


def test_per_epoch_object_update_with_one_batch_is_the_per_batch_update():
    O_true, P, pos, I_m, O, _ = _noiseless_problem(0.0)
    order = synth.random_order(pos.shape[0], 8)
    a = orc.LsqmlOptions(batch=pos.shape[0], eps=1e-12, delta_o=0.1, delta_p=0.1)
    b = orc.LsqmlOptions(batch=pos.shape[0], eps=1e-12, delta_o=0.1, delta_p=0.1, object_per_epoch=True)
    Oa, Pa, La, _ = orc.lsqml_epoch(O, P, pos, I_m, order, a)
    Ob, Pb, Lb, _ = orc.lsqml_epoch(O, P, pos, I_m, order, b)
    assert np.max(np.abs(Oa - Ob)) < 1e-12 and np.max(np.abs(Pa - Pb)) < 1e-12 and La == Lb


def test_per_epoch_object_update_does_not_depend_on_the_batch_order():
    # every minibatch sees the epoch's starting object and (without probe
    # updates) the same probe, so the summed update ignores the batch order;
    # the per-batch update does not
    O_true, P, pos, I_m, O, _ = _noiseless_problem(0.0)
    order = synth.random_order(pos.shape[0], 9)
    B = 7
    batches = [order[i:i + B] for i in range(0, len(order), B)]
    # the full groups in reverse order; the ragged last group stays last so that
    # the grouping is unchanged
    reordered = np.concatenate([b for b in batches if len(b) == B][::-1] + [b for b in batches if len(b) < B])
    for per_epoch in (True, False):
        o = orc.LsqmlOptions(batch=B, eps=1e-12, delta_o=0.1, update_probe=False, object_per_epoch=per_epoch)
        diff = np.max(np.abs(orc.lsqml_epoch(O, P, pos, I_m, order, o)[0]
                             - orc.lsqml_epoch(O, P, pos, I_m, reordered, o)[0]))
        assert (diff < 1e-12) if per_epoch else (diff > 1e-6)


# --------------------------------------------------------------------------- multislice
def test_asm_propagator_properties():
    N, px, lam = 32, 10e-9, 0.1e-9
    H1 = orc.asm_propagator(N, px, lam, 1e-6)
    H2 = orc.asm_propagator(N, px, lam, 2.5e-6)
    H3 = orc.asm_propagator(N, px, lam, 3.5e-6)
    assert np.max(np.abs(H1 * H2 - H3)) < 1e-12                      # propagation composes
    assert np.max(np.abs(orc.asm_propagator(N, px, lam, 0.0) - 1.0)) == 0.0
    assert np.max(np.abs(np.abs(H1) - 1.0)) < 1e-14                   # no evanescent waves here
    # paraxial (Fresnel) limit: phase -> -pi lambda dz |f|^2, relative error ~ (lambda f)^2 / 4
    f = np.fft.fftfreq(N, d=px)
    f2 = f[:, None] ** 2 + f[None, :] ** 2
    fres = -np.pi * lam * 1e-6 * f2
    assert np.max(np.abs(np.angle(H1) - fres)) < 1e-4 * np.max(np.abs(fres))
    # frequencies beyond 1/lambda are evanescent and removed
    Hc = orc.asm_propagator(8, 0.4, 1.0, 1.0)
    f = np.fft.fftfreq(8, d=0.4)
    ev = (f[:, None] ** 2 + f[None, :] ** 2) >= 1.0
    assert ev.any() and np.all(Hc[ev] == 0) and np.all(np.abs(Hc[~ev]) > 0.99)


def _ms_problem(S=3, seed=19, M=2):
    g = np.random.default_rng(seed)
    w = synth.workload_small(N=8, M=M, H=24, W=24, J=4, seed=seed, step=3.0)
    Os = np.stack([w["object"] ** (1.0 / S) * np.exp(0.2j * g.standard_normal((24, 24))) for _ in range(S)])
    Hf = orc.asm_propagator(8, 10e-9, 0.1e-9, 40e-6)   # a strong propagator for an 8-px window
    I_m = synth.poisson_counts(orc.forward_ms(Os, w["probe"] * 3.0, w["pos"], Hf), seed)
    return Os, w["probe"] * 3.0, w["pos"], Hf, I_m


def test_multislice_with_one_slice_is_the_single_slice_model():
    Os, P, pos, Hf, I_m = _ms_problem(S=1)
    assert np.max(np.abs(orc.forward_ms(Os, P, pos, Hf) - orc.forward(Os[0], P, pos))) < 1e-12
    G = np.random.default_rng(1).standard_normal(I_m.shape)
    gO, gP, gr = orc.vjp_ms(Os, P, pos, Hf, G)
    gO1, gP1, gr1 = orc.vjp(Os[0], P, pos, G)
    assert np.max(np.abs(gO[0] - gO1)) < 1e-10 and np.max(np.abs(gP - gP1)) < 1e-10
    assert np.max(np.abs(gr - gr1)) < 1e-10


def test_multislice_without_propagation_is_the_product_object():
    # integer positions: the patches are crops, so the patch of a product is
    # the product of the patches
    Os, P, pos, _, _ = _ms_problem(S=3)
    pos = np.round(pos)
    one = orc.asm_propagator(8, 10e-9, 0.1e-9, 0.0)
    ref = orc.forward(Os[0] * Os[1] * Os[2], P, pos)
    assert np.max(np.abs(orc.forward_ms(Os, P, pos, one) - ref)) < 1e-11 * np.max(ref)


def test_multislice_conserves_energy_through_pure_phase_slices():
    Os, P, pos, Hf, _ = _ms_problem(S=4)
    Os = np.exp(1j * np.angle(Os))
    I = orc.forward_ms(Os, P, np.round(pos), Hf)   # crops of pure-phase slices are pure phase
    assert np.max(np.abs(I.sum(axis=(1, 2)) - np.sum(np.abs(P) ** 2))) < 1e-10 * np.sum(np.abs(P) ** 2)


def test_multislice_gradients_match_central_finite_differences():
    Os, P, pos, Hf, I_m = _ms_problem(S=3)
    L, gO, gP, gr = orc.loss_and_gradients_ms(Os, P, pos, Hf, I_m, orc.GAUSSIAN, 1e-3)
    g = np.random.default_rng(5)
    h = 1e-6

    def L_at(Os_, P_, pos_):
        return orc.loss_and_gradients_ms(Os_, P_, pos_, Hf, I_m, orc.GAUSSIAN, 1e-3)[0]

    dO = crandn(g, *Os.shape)
    fd = (L_at(Os + h * dO, P, pos) - L_at(Os - h * dO, P, pos)) / (2 * h)
    assert abs(fd - np.real(np.vdot(gO, dO))) < 1e-6 * abs(fd)
    dP = crandn(g, *P.shape)
    fd = (L_at(Os, P + h * dP, pos) - L_at(Os, P - h * dP, pos)) / (2 * h)
    assert abs(fd - np.real(np.vdot(gP, dP))) < 1e-6 * abs(fd)
    dr = g.standard_normal(pos.shape) * 0.1
    fd = (L_at(Os, P, pos + h * dr) - L_at(Os, P, pos - h * dr)) / (2 * h)
    assert abs(fd - np.sum(gr * dr)) < 1e-5 * abs(fd)


# --------------------------------------------------------------------------- exit-wave step and probe direction
@pytest.mark.parametrize("noise,factor", [(orc.GAUSSIAN, -0.5), (orc.POISSON, -0.25)])
def test_lsqml_accumulators_are_fixed_multiples_of_the_finite_difference_gradients(noise, factor):
    # The LSQML accumulators are the exit-wave changes back-projected onto the
    # object (sum_k conj(P_k) chi_k) and onto the probe (conj(o) chi_k); their
    # ratio to the loss gradient is fixed by the data term (Sec. 2.2):
    #   Gaussian (Eq. 2): psi' - psi = F^-1[(rho - 1) Psi] with rho = sqrt(I_m)/sqrt(I + eps),
    #     and 2 dL/dpsi* = F^-1[2 (1 - rho) Psi]: chi = -1/2 grad;
    #   Poisson, half a likelihood step (rho - 1 = (I_m/(I + eps) - 1)/2) against
    #     2 dL/dpsi* = F^-1[2 (1 - I_m/(I + eps)) Psi]: chi = -1/4 grad.
    # The gradients are pinned by central finite differences, so a wrong step
    # length or a missing conjugate in either accumulator fails here.
    O, P, pos, I_m = _fd_problem(noise, seed=14)
    opts = orc.LsqmlOptions(noise=noise, batch=4, eps=1e-3)
    rec = {}
    orc.lsqml_batch(O, P, pos, I_m, range(4), opts, rec)
    _, gO, gP, _ = orc.loss_and_gradients(O, P, pos, I_m, noise, 1e-3)
    assert np.max(np.abs(rec["dO_acc"] - factor * gO)) < 1e-10 * np.max(np.abs(gO))
    assert np.max(np.abs(rec["dP_acc"] - factor * gP)) < 1e-10 * np.max(np.abs(gP))


def _probe_step_problem(n_pos):
    g = np.random.default_rng(15)
    N, H, W = 16, 40, 40
    P_true = synth.hg_probe(N, np.array([1.0, 0.5]), waist=N / 5.0, quad_phase=0.03) * 3.0
    O = synth.make_object(H, W, 4, phase_sigma=1.0)
    pos = np.array([[12.0, 13.0], [27.0, 26.0]])[:n_pos]     # integer, non-overlapping tiles
    I_m = orc.forward(O, P_true, pos)
    P = P_true * (1 + 0.2 * crandn(g, *P_true.shape))
    return N, O, P, pos, I_m


@pytest.mark.parametrize("n_pos", [1, 2])
def test_probe_only_update_has_the_closed_form_of_a_known_object(n_pos):
    # Object known and held (update_object False), lam = 0: the object step
    # vanishes and each alpha_P,j is the 1x1 solve Re<v_j, chi_j> / ||v_j||^2
    # with v_jk = o_j dP_k; the probe moves by mean_j(alpha_P,j) dP_k with
    # dP_k = sum_j conj(o_j) chi_jk / (sum_j |o_j|^2 + delta_p max(...)).
    # Written out on the crops with numpy's FFT, without S_j or the batch code.
    N, O, P, pos, I_m = _probe_step_problem(n_pos)
    dp = 5e-2
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=n_pos, delta_p=dp, lam=0.0, eps=0.0,
                            update_object=False)
    O_new, P_new, _, alpha = orc.lsqml_batch(O, P, pos, I_m, range(n_pos), opts)
    crops, chis = [], []
    for j in range(n_pos):
        ty, tx = int(pos[j, 0]) - N // 2, int(pos[j, 1]) - N // 2
        o = O[ty:ty + N, tx:tx + N]
        Psi = np.fft.fft2(P * o[None]) / N
        I = np.sum(np.abs(Psi) ** 2, axis=0)
        chi = np.fft.ifft2(Psi * np.sqrt(I_m[j] / I)[None]) * N - P * o[None]
        crops.append(o)
        chis.append(chi)
    Dp = sum(np.abs(o) ** 2 for o in crops)
    d = sum(np.conj(o)[None] * c for o, c in zip(crops, chis)) / (Dp + dp * Dp.max())[None]
    a = []
    for o, c in zip(crops, chis):
        v = o[None] * d
        a.append(np.real(np.vdot(v, c)) / np.real(np.vdot(v, v)))
    ref = P + np.mean(a) * d
    assert np.allclose(alpha[:, 1], a, rtol=1e-10, atol=0) and np.all(alpha[:, 0] == 0.0)
    assert np.max(np.abs(P_new - ref)) < 1e-12 * np.max(np.abs(P))
    assert np.array_equal(O_new, O)


# --------------------------------------------------------------------------- multislice LSQML
def test_multislice_lsqml_with_one_slice_is_the_single_slice_minibatch():
    Os, P, pos, Hf, I_m = _ms_problem(S=1)
    g = np.random.default_rng(23)
    Os = Os * (1 + 0.1 * crandn(g, *Os.shape))
    for noise in (orc.GAUSSIAN, orc.POISSON):
        opts = orc.LsqmlOptions(noise=noise, batch=4, eps=1e-3, delta_o=0.1, delta_p=0.1)
        O1, P1, L1, a1 = orc.lsqml_batch_ms(Os, P, pos, I_m, range(4), Hf, opts)
        O0, P0, L0, a0 = orc.lsqml_batch(Os[0], P, pos, I_m, range(4), opts)
        assert np.max(np.abs(O1[0] - O0)) < 1e-13 and np.max(np.abs(P1 - P0)) < 1e-13
        assert abs(L1 - L0) <= 1e-12 * abs(L0) and np.max(np.abs(a1 - a0)) <= 1e-12 * np.max(np.abs(a0))


@pytest.mark.parametrize("noise,factor", [(orc.GAUSSIAN, -0.5), (orc.POISSON, -0.25)])
def test_multislice_lsqml_accumulators_are_multiples_of_the_finite_difference_gradients(noise, factor):
    # every slice's accumulator is its exit-plane change back-projected through
    # the slices after it; against the finite-difference-pinned multislice
    # gradients it is -1/2 (amplitude term) or -1/4 (Poisson half step) of the
    # slice's gradient, and the probe accumulator likewise
    Os, P, pos, Hf, I_m = _ms_problem(S=3)
    opts = orc.LsqmlOptions(noise=noise, batch=4, eps=1e-3)
    rec = {}
    orc.lsqml_batch_ms(Os, P, pos, I_m, range(4), Hf, opts, rec)
    _, gO, gP, _ = orc.loss_and_gradients_ms(Os, P, pos, Hf, I_m, noise, 1e-3)
    for s in range(3):
        assert np.max(np.abs(rec["dO_acc"][s] - factor * gO[s])) < 1e-10 * np.max(np.abs(gO[s]))
    assert np.max(np.abs(rec["dP_acc"] - factor * gP)) < 1e-10 * np.max(np.abs(gP))


def test_multislice_lsqml_step_sizes_fit_the_exit_plane_change_by_finite_difference_tangents():
    # u and v are the first-order changes of the exit waves when all slices move
    # along their directions and when the probe moves along dP; taken here by
    # central differences of the forward model itself, the step sizes are
    # numpy's least squares of the exit-plane change by them (lam = 0)
    Os, P, pos, Hf, I_m = _ms_problem(S=3)
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=4, eps=1e-3, lam=0.0, delta_o=0.1, delta_p=0.1)
    rec = {}
    _, _, _, alpha = orc.lsqml_batch_ms(Os, P, pos, I_m, range(4), Hf, opts, rec)
    h = 1e-5
    for j in range(4):
        def exit_wave(Os_, P_):
            return orc.exit_waves_ms(Os_, P_, pos[j], Hf)[0]
        u = (exit_wave(Os + h * rec["dO_hat"], P) - exit_wave(Os - h * rec["dO_hat"], P)) / (2 * h)
        v = (exit_wave(Os, P + h * rec["dP"]) - exit_wave(Os, P - h * rec["dP"])) / (2 * h)
        assert np.max(np.abs(u - rec["u"][j])) < 1e-7 * np.max(np.abs(u))
        assert np.max(np.abs(v - rec["v"][j])) < 1e-7 * np.max(np.abs(v))
        u, v, chi = u.ravel(), v.ravel(), rec["chi"][j][-1].ravel()
        A = np.concatenate([np.stack([u.real, v.real], 1), np.stack([u.imag, v.imag], 1)])
        b = np.concatenate([chi.real, chi.imag])
        ref = np.linalg.lstsq(A, b, rcond=None)[0]
        assert np.max(np.abs(alpha[j] - ref)) < 1e-6 * np.max(np.abs(ref))


def test_multislice_lsqml_object_term_of_the_step_equals_the_slices_numerators():
    # adjoint identity: Re<u, chi_exit> = sum_s Re<dO_s(r_j), g_js>, the form the
    # GPU evaluates (no exit-plane change is stored)
    Os, P, pos, Hf, I_m = _ms_problem(S=3)
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=4, eps=1e-3, delta_o=0.1, delta_p=0.1)
    rec = {}
    orc.lsqml_batch_ms(Os, P, pos, I_m, range(4), Hf, opts, rec)
    for j in range(4):
        lhs = np.real(np.vdot(rec["u"][j], rec["chi"][j][-1]))
        rhs = sum(np.real(np.vdot(orc.extract(rec["dO_hat"][s], pos[j], 8), rec["g"][j][s])) for s in range(3))
        assert abs(lhs - rhs) < 1e-10 * abs(lhs)
        lhs = np.real(np.vdot(rec["v"][j], rec["chi"][j][-1]))
        _, _, o = orc.exit_waves_ms(Os, P, pos[j], Hf)
        rhs = np.real(np.vdot(rec["dP"], np.conj(o[0])[None] * rec["chi"][j][0]))
        assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_multislice_lsqml_exit_plane_changes_are_the_propagated_differences():
    # the last slice's change is psi' - psi of the exit wave; each earlier
    # slice's is the adjoint propagation of conj(o_s) times the later one,
    # written out with numpy's FFT
    Os, P, pos, Hf, I_m = _ms_problem(S=2, M=1)
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=4, eps=1e-3)
    rec = {}
    orc.lsqml_batch_ms(Os, P, pos, I_m, range(4), Hf, opts, rec)
    psi, inc, o = orc.exit_waves_ms(Os, P, pos[0], Hf)
    Psi = np.fft.fft2(psi[0]) / 8
    new = np.fft.ifft2(Psi * np.sqrt(I_m[0]) / np.sqrt(np.abs(Psi) ** 2 + 1e-3)) * 8
    assert np.max(np.abs(rec["chi"][0][1][0] - (new - psi[0]))) < 1e-12
    back = np.fft.ifft2(np.conj(Hf) * np.fft.fft2(np.conj(o[1]) * (new - psi[0])))
    assert np.max(np.abs(rec["chi"][0][0][0] - back)) < 1e-12


def test_multislice_lsqml_truth_is_fixed_and_noiseless_loss_falls():
    Os, P, pos, Hf, _ = _ms_problem(S=2, seed=29)
    I_t = orc.forward_ms(Os, P, pos, Hf)
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=2, eps=1e-12, delta_o=0.1, delta_p=0.1)
    O1, P1, L1, _ = orc.lsqml_epoch_ms(Os, P, pos, I_t, np.arange(4), Hf, opts)
    assert L1 < 1e-18 and np.max(np.abs(O1 - Os)) < 1e-9 and np.max(np.abs(P1 - P)) < 1e-9
    g = np.random.default_rng(31)
    O = Os * (1 + 0.05 * crandn(g, *Os.shape))
    losses = []
    for _ in range(8):
        O, _, L, _ = orc.lsqml_epoch_ms(O, P, pos, I_t, np.arange(4), Hf,
                                        orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=2, eps=1e-12, delta_o=0.1,
                                                         update_probe=False))
        losses.append(L)
    assert losses[-1] < 0.1 * losses[0]


def test_multislice_lsqml_from_flat_slices_is_stable_and_reduces_the_loss():
    # four slices, all flat at the start, Poisson counts: the joint step keeps the
    # iteration stable (step sizes of order one) while the loss falls
    N, S, H = 16, 4, 48
    Os_true = np.stack([synth.make_object(H, H, 40 + s, phase_sigma=1.5) ** (1.0 / S) for s in range(S)])
    P = synth.hg_probe(N, np.array([0.7, 0.3]), waist=N / 5.0, quad_phase=0.02)
    pos = synth.raster_positions(5, 5, 5.0, (H / 2, H / 2), 0.5, 3)
    Hf = orc.asm_propagator(N, 10e-9, 0.1e-9, 0.1e-6)
    I = orc.forward_ms(Os_true, P, pos, Hf)
    P = P * np.sqrt(1e5 / I.sum(axis=(1, 2)).mean())
    I_m = synth.poisson_counts(orc.forward_ms(Os_true, P, pos, Hf), 5)
    Os = np.ones_like(Os_true)
    opts = orc.LsqmlOptions(batch=5, delta_o=0.1, delta_p=0.1, eps=1.0)
    losses = []
    for _ in range(6):
        Os, P, L, alpha = orc.lsqml_epoch_ms(Os, P, pos, I_m, synth.random_order(25, 4), Hf, opts)
        losses.append(L)
        assert np.all(np.isfinite(alpha)) and np.max(np.abs(alpha)) < 10
    assert losses[-1] < 0.5 * losses[0] and all(np.isfinite(losses))


def test_multislice_probe_only_update_has_the_closed_form_of_a_known_object():
    # one position at an integer offset, two slices held fixed: the probe moves
    # by alpha_P dP with dP = conj(o_0) chi_0 / (|o_0|^2 + delta_p max|o_0|^2),
    # chi_0 the exit-plane change carried back through slice 1 and the
    # propagator, alpha_P the 1x1 fit of the exit-plane change by the probe
    # direction carried forward through the slices; written out on the crops
    g = np.random.default_rng(37)
    N, H, W = 16, 30, 30
    P_true = synth.hg_probe(N, np.array([1.0, 0.4]), waist=N / 5.0, quad_phase=0.03) * 3.0
    Os = np.stack([synth.make_object(H, W, 5, phase_sigma=1.0), synth.make_object(H, W, 6, phase_sigma=1.0)])
    Hf = orc.asm_propagator(N, 10e-9, 0.1e-9, 2e-6)
    r = np.array([[15.0, 14.0]])
    I_m = orc.forward_ms(Os, P_true, r, Hf)
    P = P_true * (1 + 0.2 * crandn(g, *P_true.shape))
    dp = 5e-2
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=1, delta_p=dp, lam=0.0, eps=0.0, update_object=False)
    O_new, P_new, _, alpha = orc.lsqml_batch_ms(Os, P, r, I_m, [0], Hf, opts)
    o0, o1 = Os[0, 7:23, 6:22], Os[1, 7:23, 6:22]
    prop = lambda x, H_: np.fft.ifft2(H_ * np.fft.fft2(x))
    inc1 = prop(P * o0[None], Hf)
    psi = inc1 * o1[None]
    Psi = np.fft.fft2(psi) / N
    I = np.sum(np.abs(Psi) ** 2, axis=0)
    chi1 = np.fft.ifft2(Psi * np.sqrt(I_m[0] / I)[None]) * N - psi
    chi0 = prop(np.conj(o1)[None] * chi1, np.conj(Hf))
    Dp = np.abs(o0) ** 2
    d = np.conj(o0)[None] * chi0 / (Dp + dp * Dp.max())[None]
    v = prop(o0[None] * d, Hf) * o1[None]
    a = np.real(np.vdot(v, chi1)) / np.real(np.vdot(v, v))
    assert abs(alpha[0, 1] - a) < 1e-10 * abs(a) and alpha[0, 0] == 0.0
    assert np.max(np.abs(P_new - (P + a * d))) < 1e-12 * np.max(np.abs(P))
    assert np.array_equal(O_new, Os)
