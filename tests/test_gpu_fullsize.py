"""Parity at the paper-shaped workloads' full sizes, in the launch configuration
bench.py times (minibatch, window, modes and object size), against the FP64
oracle: the raster64 workload in full, and the spiral128 workload on one full
minibatch of 256 positions, one whole epoch of all 4096 positions, sampled
forward outputs and epoch-level properties."""
import math

import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2510_20929_gb300 import synth
from tests.parity_util import TOL_EPOCH, TOL_FWD, err, to_dev

pytestmark = pytest.mark.gpu

# The amplitude data term at a tiny eps is ill-conditioned where the
# prediction is dark but counts were measured (a flat starting object): the
# phase of a near-zero far-field pixel, and with it the projected wave, moves
# by the input's relative rounding divided by the pixel's relative amplitude.
# In FP64 the oracle's own minibatch moves by up to 6.7e-4 element-wise (and a
# whole spiral128 epoch by 1.7e-3 norm-wise) when the probe is perturbed by
# one FP32 rounding unit, against 1e-7 at eps = 1 count. The workload's
# configuration therefore uses eps = 1 count (one photon, the scale of the
# Poisson data); parity at eps = 1e-9 is held to a few times the oracle's
# measured response to an FP32-sized perturbation instead of a fixed bar.
U32 = 2.0 ** -24


def _measured(w, O_true, P, pos, seed):
    """Oracle intensities of the true object, scaled to the workload's counts, Poisson-sampled."""
    I = orc.forward(O_true, P, pos)
    per = w["total_counts"] / (I.sum() if w["counts_per"] == "all" else I.sum(axis=(1, 2)).mean())
    return P * math.sqrt(per), synth.poisson_counts(I * per, seed)


def _f32(x, complex_=False):
    return np.asarray(x, np.complex64 if complex_ else np.float32).astype(np.complex128 if complex_ else np.float64)


@pytest.mark.parametrize("noise", ["gaussian", "poisson"])
def test_raster64_full_workload(noise):
    import torch
    from paper_2510_20929_gb300 import api
    w = synth.workload_raster64()
    O_true = _f32(w["object"], True)
    pos = _f32(w["pos"])
    P, I_m = _measured(w, O_true, _f32(w["probe"], True), pos, 11)
    P, I_m = _f32(P, True), _f32(I_m)
    O0 = np.ones_like(O_true)
    dO, dP = to_dev(O0, torch.complex64), to_dev(P, torch.complex64)
    dpos, dI = to_dev(pos, torch.float32), to_dev(I_m, torch.float32)
    # forward
    e = err(api.forward(dO, dP, dpos).cpu().numpy(), orc.forward(O0, P, pos))
    assert e < TOL_FWD, e
    # one epoch, one minibatch of all 100 positions (the workload's batch). From the flat
    # start many pixels are predicted near zero yet hold counts; the Poisson factor
    # I_m / (I + eps) then amplifies the FP32 rounding of I (about 1e-7 of the peak) by
    # I_m / eps^2, so the Poisson case takes eps = 1 count (the Gaussian factor is bounded).
    nz = orc.GAUSSIAN if noise == "gaussian" else orc.POISSON
    eps = 1e-9 if noise == "gaussian" else 1.0
    order = synth.random_order(w["J"], 3)
    opts = orc.LsqmlOptions(noise=nz, batch=w["batch"], delta_o=0.1, delta_p=0.1, lam=1e-6, eps=eps)
    O_ref, P_ref, L_ref, a_ref = orc.lsqml_epoch(O0, P, pos, I_m, order, opts)
    loss, alpha = api.lsqml_epoch(dO, dP, dpos, dI, to_dev(order, torch.int32), noise=noise, batch=w["batch"],
                                  delta_o=0.1, delta_p=0.1, lam=1e-6, eps=eps, want_alpha=True)
    e = (err(dO.cpu().numpy(), O_ref), err(dP.cpu().numpy(), P_ref, axis=0), err(alpha.cpu().numpy(), a_ref, axis=1),
         abs(loss.item() - L_ref) / abs(L_ref))
    print(f"raster64 {noise}: O {e[0]:.2e} P {e[1]:.2e} alpha {e[2]:.2e} loss {e[3]:.2e}")
    assert max(e) < TOL_EPOCH


def test_raster64_full_workload_gradients():
    import torch
    from paper_2510_20929_gb300 import api
    w = synth.workload_raster64()
    O_true = _f32(w["object"], True)
    pos = _f32(w["pos"])
    P, I_m = _measured(w, O_true, _f32(w["probe"], True), pos, 12)
    P, I_m = _f32(P, True), _f32(I_m)
    g = np.random.default_rng(5)
    O = _f32(O_true * np.exp(0.3j * g.standard_normal(O_true.shape)), True)
    L_ref, gO_ref, gP_ref, gr_ref = orc.loss_and_gradients(O, P, pos, I_m, orc.GAUSSIAN, 1e-9)
    loss, gO, gP, gr = api.adjoint(to_dev(O, torch.complex64), to_dev(P, torch.complex64),
                                   to_dev(pos, torch.float32), to_dev(I_m, torch.float32), "gaussian", eps=1e-9,
                                   batch=100)
    e = (abs(loss.item() - L_ref) / L_ref, err(gO.cpu().numpy(), gO_ref), err(gP.cpu().numpy(), gP_ref, axis=0),
         err(gr.cpu().numpy(), gr_ref, axis=1))
    print("raster64 gradients:", e)
    assert e[0] < TOL_FWD and max(e[1:]) < TOL_EPOCH


@pytest.fixture(scope="module")
def spiral():
    w = synth.workload_spiral128()
    O_true = _f32(w["object"], True)
    pos = _f32(w["pos"])
    order = synth.random_order(w["J"], 5)
    idx = order[:256]                                   # the first minibatch of the bench's order
    P, I_sub = _measured(w, O_true, _f32(w["probe"], True), pos[idx], 21)
    return w, O_true, _f32(P, True), pos, order, idx, _f32(I_sub)


def _oracle_response(fn, P, seed=3):
    """How far the oracle's outputs move when the probe is perturbed by one FP32
    rounding unit (random complex, relative): the outputs of fn(P) and fn(P')."""
    g = np.random.default_rng(seed)
    Pp = P * (1 + U32 * (g.standard_normal(P.shape) + 1j * g.standard_normal(P.shape)))
    return fn(P), fn(Pp)


@pytest.mark.parametrize("eps", [1.0, 1e-9])
def test_spiral128_first_minibatch(spiral, eps):
    import torch
    from paper_2510_20929_gb300 import api
    w, O_true, P, pos, order, idx, I_sub = spiral
    O0 = np.ones_like(O_true)
    sub_pos = pos[idx]
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=256, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=eps)
    ref, ref_p = _oracle_response(lambda P_: orc.lsqml_batch(O0, P_, sub_pos, I_sub, range(256), opts), P)
    O_ref, P_ref, L_ref, a_ref = ref
    dO, dP = to_dev(O0, torch.complex64), to_dev(P, torch.complex64)
    loss, alpha = api.lsqml_epoch(dO, dP, to_dev(sub_pos, torch.float32), to_dev(I_sub, torch.float32),
                                  None, batch=256, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=eps, want_alpha=True)
    e = (err(dO.cpu().numpy(), O_ref), err(dP.cpu().numpy(), P_ref, axis=0), err(alpha.cpu().numpy(), a_ref, axis=1),
         abs(loss.item() - L_ref) / abs(L_ref))
    s = (err(ref_p[0], O_ref), err(ref_p[1], P_ref, axis=0), err(ref_p[3], a_ref, axis=1))
    print(f"spiral128 first minibatch, eps {eps:g}: O {e[0]:.2e} P {e[1]:.2e} alpha {e[2]:.2e} loss {e[3]:.2e}; "
          f"oracle response to one rounding unit: O {s[0]:.2e} P {s[1]:.2e} alpha {s[2]:.2e}")
    assert e[3] < TOL_FWD
    for ei, si in zip(e[:3], s):
        assert ei < max(TOL_EPOCH, 4.0 * si)
    if eps >= 1.0:
        assert max(s) < 0.1 * TOL_EPOCH   # well conditioned: the fixed bar applies


def test_spiral128_sampled_forward_and_epoch_properties(spiral):
    import torch
    from paper_2510_20929_gb300 import api
    w, O_true, P, pos, order, idx, _ = spiral
    dO_true, dP = to_dev(O_true, torch.complex64), to_dev(P, torch.complex64)
    dpos = to_dev(pos, torch.float32)
    I = api.forward(dO_true, dP, dpos)
    sample = np.random.default_rng(9).choice(w["J"], 12, replace=False)
    ref = orc.forward(O_true, P, pos[sample])
    e = err(I[torch.as_tensor(sample, device=I.device)].cpu().numpy(), ref)
    assert e < TOL_FWD, e
    # epochs over all 4096 positions: finite, decreasing loss from a flat start (noiseless data)
    O = torch.ones_like(dO_true)
    P_est = dP.clone()
    dorder = to_dev(order, torch.int32)
    losses = []
    for _ in range(3):
        loss, alpha = api.lsqml_epoch(O, P_est, dpos, I, dorder, batch=256, delta_o=0.1, delta_p=0.1,
                                      eps=1e-9, want_alpha=True)
        losses.append(loss.item())
        assert torch.isfinite(alpha).all()
    print("spiral128 losses:", losses)
    assert losses[2] < losses[1] < losses[0]


def test_spiral128_full_epoch_matches_oracle():
    # The epoch the bench times, in full: all 4096 positions in 16 minibatches of
    # 256 in the bench's order, from the flat object and the true probe, on
    # Poisson-sampled counts (1e6 per pattern) with the amplitude data term at
    # eps = 1 count; every minibatch updates the object and the probe, so the
    # comparison covers the compounding of 16 updates.
    import torch
    from paper_2510_20929_gb300 import api
    w = synth.workload_spiral128()
    O_true = _f32(w["object"], True)
    pos = _f32(w["pos"])
    P, I_m = _measured(w, O_true, _f32(w["probe"], True), pos, 31)
    P, I_m = _f32(P, True), _f32(I_m)
    order = synth.random_order(w["J"], 5)
    O0 = np.ones_like(O_true)
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=256, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1.0)
    O_ref, P_ref, L_ref, a_ref = orc.lsqml_epoch(O0, P, pos, I_m, order, opts)
    dO, dP = to_dev(O0, torch.complex64), to_dev(P, torch.complex64)
    loss, alpha = api.lsqml_epoch(dO, dP, to_dev(pos, torch.float32), to_dev(I_m, torch.float32),
                                  to_dev(order, torch.int32), batch=256, delta_o=0.1, delta_p=0.1, lam=1e-6,
                                  eps=1.0, want_alpha=True)
    e = (err(dO.cpu().numpy(), O_ref), err(dP.cpu().numpy(), P_ref, axis=0), err(alpha.cpu().numpy(), a_ref, axis=1),
         abs(loss.item() - L_ref) / abs(L_ref))
    print(f"spiral128 full epoch: O {e[0]:.2e} P {e[1]:.2e} alpha {e[2]:.2e} loss {e[3]:.2e}")
    assert max(e) < TOL_EPOCH


def test_spiral128_first_minibatch_split_bf16(spiral):
    # The split-BF16 DFT-GEMM form on the same full minibatch, in the workload's
    # configuration (eps = 1 count), every output held to the split-BF16 bound
    # of 1e-3. (At eps = 1e-9 the FP64 oracle itself moves by 6.7e-4 under an
    # FP32-sized perturbation of its input, see the note at the top: no fixed
    # bound of that size can hold there.)
    import torch
    from paper_2510_20929_gb300 import api
    w, O_true, P, pos, order, idx, I_sub = spiral
    O0 = np.ones_like(O_true)
    sub_pos = pos[idx]
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=256, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1.0)
    O_ref, P_ref, L_ref, a_ref = orc.lsqml_batch(O0, P, sub_pos, I_sub, range(256), opts)
    dO, dP = to_dev(O0, torch.complex64), to_dev(P, torch.complex64)
    loss, alpha = api.lsqml_epoch(dO, dP, to_dev(sub_pos, torch.float32), to_dev(I_sub, torch.float32),
                                  None, batch=256, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1.0, want_alpha=True,
                                  precision="bf16x3")
    e = (err(dO.cpu().numpy(), O_ref), err(dP.cpu().numpy(), P_ref, axis=0), abs(loss.item() - L_ref) / abs(L_ref),
         err(alpha.cpu().numpy(), a_ref, axis=1))
    print(f"spiral128 first minibatch, split BF16, eps 1: O {e[0]:.2e} P {e[1]:.2e} loss {e[2]:.2e} "
          f"alpha {e[3]:.2e}")
    assert max(e) < 1e-3


@pytest.fixture(scope="module")
def spiral256():
    w = synth.workload_spiral256()
    return w


def test_spiral256_sampled_gradients_match_oracle(spiral256):
    # the full 2048^2 object and 8-mode 256^2 probe; the data term over four
    # sampled positions of the perturbed scan, against the oracle on the same four
    import torch
    from paper_2510_20929_gb300.autograd import data_term
    w = spiral256
    idx = np.array([17, 2500, 6001, 9876])
    O = _f32(w["object"] * np.exp(0.2j), True)
    P = _f32(w["probe"] * 4.0, True)
    pos_true, pos0 = _f32(w["pos"][idx]), _f32(w["pos_init"][idx])
    I_m = _f32(synth.poisson_counts(orc.forward(_f32(w["object"], True), P, pos_true), 5))
    L, gO, gP, gr = orc.loss_and_gradients(O, P, pos0, I_m, orc.GAUSSIAN, 1e-6)
    dO, dP, dpos = to_dev(O, torch.complex64), to_dev(P, torch.complex64), to_dev(pos0, torch.float32)
    for t in (dO, dP, dpos):
        t.requires_grad_(True)
    loss = data_term(dO, dP, dpos, to_dev(I_m, torch.float32), "gaussian", 1e-6)
    loss.backward()
    e = (abs(loss.item() - L) / L, err(dO.grad.cpu().numpy(), gO), err(dP.grad.cpu().numpy(), gP, axis=0),
         err(dpos.grad.cpu().numpy(), gr, axis=1))
    print("spiral256 sampled gradients:", e)
    assert e[0] < TOL_FWD and max(e[1:]) < TOL_EPOCH


def test_spiral256_adam_on_all_three_reduces_loss_and_position_error(spiral256):
    # Adam on object, probe and positions over all 10,000 positions from
    # N(0, 1.5 px) position errors (data: the forward model at the true positions)
    import torch
    from paper_2510_20929_gb300 import api
    from paper_2510_20929_gb300.autograd import reconstruct_adam
    w = spiral256
    O_true = to_dev(_f32(w["object"], True), torch.complex64)
    P = to_dev(_f32(w["probe"] * 4.0, True), torch.complex64)
    pos_true = to_dev(_f32(w["pos"]), torch.float32)
    I_m = api.forward(O_true, P, pos_true)
    pos = to_dev(_f32(w["pos_init"]), torch.float32)
    O = O_true.clone()
    rmse0 = (pos - pos_true).pow(2).mean().sqrt().item()
    hist = reconstruct_adam(O, P.clone(), pos, I_m, epochs=20, lr_object=1e-3, lr_probe=1e-3, lr_pos=0.1)
    rmse = (pos - pos_true).pow(2).mean().sqrt().item()
    print("spiral256 Adam: loss", hist[0], "->", hist[-1], "position rmse", rmse0, "->", rmse)
    assert hist[-1] < 0.7 * hist[0] and rmse < 0.95 * rmse0


# --------------------------------------------------------------------------- multislice (4 slices of 2048^2)
@pytest.fixture(scope="module")
def multislice256():
    return synth.workload_multislice256()


def test_multislice256_sampled_forward_and_gradients_match_oracle(multislice256):
    # the full 4 x 2048^2 slices and the 4-mode 256^2 probe with the workload's
    # propagator; forward and gradients over four sampled positions, in the
    # launch configuration of the bench (minibatch 512)
    import torch
    from paper_2510_20929_gb300 import api
    w = multislice256
    idx = np.array([3, 2100, 5555, 7999])
    Os = _f32(w["slices"], True)
    P = _f32(w["probe"] * 4.0, True)
    pos = _f32(w["pos"][idx])
    Hf = orc.asm_propagator(256, w["pixel_size"], w["wavelength"], w["dz"])
    ms = api.make_multislice(w["S"], w["dz"], w["wavelength"], w["pixel_size"])
    dOs, dP, dpos = to_dev(Os, torch.complex64), to_dev(P, torch.complex64), to_dev(pos, torch.float32)
    I = api.forward_ms(dOs, dP, dpos, ms, batch=w["batch"]).cpu().numpy()
    ref = orc.forward_ms(Os, P, pos, Hf)
    e_fwd = err(I, ref)
    I_m = _f32(synth.poisson_counts(ref * 1.05, 9))
    L, gO, gP, gr = orc.loss_and_gradients_ms(Os, P, pos, Hf, I_m, orc.GAUSSIAN, 1e-6)
    loss, dgO, dgP, dgr = api.adjoint_ms(dOs, dP, dpos, to_dev(I_m, torch.float32), ms, "gaussian", eps=1e-6,
                                         batch=w["batch"])
    e = (e_fwd, abs(loss.item() - L) / L, err(dgO.cpu().numpy(), gO), err(dgP.cpu().numpy(), gP, axis=0),
         err(dgr.cpu().numpy(), gr, axis=1))
    print("multislice256 sampled:", e)
    assert e[0] < 10 * TOL_FWD and e[1] < TOL_FWD and max(e[2:]) < TOL_EPOCH


def test_multislice256_adam_over_all_positions_reduces_the_loss(multislice256):
    import torch
    from paper_2510_20929_gb300 import api
    from paper_2510_20929_gb300.autograd import reconstruct_adam_ms
    w = multislice256
    ms = api.make_multislice(w["S"], w["dz"], w["wavelength"], w["pixel_size"])
    Os_true = to_dev(_f32(w["slices"], True), torch.complex64)
    P = to_dev(_f32(w["probe"] * 4.0, True), torch.complex64)
    pos = to_dev(_f32(w["pos"]), torch.float32)
    I_m = api.forward_ms(Os_true, P, pos, ms, batch=w["batch"])
    Os = torch.ones_like(Os_true)
    hist = reconstruct_adam_ms(Os, P.clone(), pos, I_m, ms, epochs=6, lr_object=1e-2, update=("object",))
    print("multislice256 Adam:", hist)
    assert all(math.isfinite(h) for h in hist) and hist[-1] < 0.8 * hist[0]


# --------------------------------------------------------------------------- uneven serving with OPR (16 reconstructions)
def test_uneven16_opr_batched_epoch_matches_oracle_on_sampled_minibatches():
    # three reconstructions of the serving mix (windows 64, 128 and 192 with
    # their full objects and 8 eigenmodes), one batched graph-replayed epoch
    # over the first positions of each (the oracle's scatter is O(H W) per
    # position, so it takes the reconstructions with the smallest objects),
    # against the oracle's minibatch
    import torch
    from paper_2510_20929_gb300 import api
    ws = synth.workload_uneven(16, seed=1005, opr_K=8)
    recons, opts, oprs, refs = [], [], [], []
    for i, n in ((12, 64), (0, 64), (1, 16)):
        w = ws[i]
        O_true = _f32(w["object"], True)
        pos = _f32(w["pos"][:n])
        wt = _f32(w["opr_w"][:n])
        I0 = orc.forward_opr(O_true, _f32(w["opr_U"], True), wt, None, pos)
        sc = math.sqrt(w["total_counts"] / w["J"] / I0.sum(axis=(1, 2)).mean())
        U = _f32(w["opr_U"] * sc, True)
        Im = _f32(synth.poisson_counts(I0 * sc * sc, 100 + i))
        O0, w0 = np.ones_like(O_true), np.ones((n, 8))
        refs.append(orc.lsqml_batch_opr(O0, U, w0, None, pos, Im, np.arange(n),
                                        orc.LsqmlOptions(batch=n, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6),
                                        orc.OprOptions()))
        recons.append([to_dev(O0, torch.complex64), to_dev(U, torch.complex64), to_dev(w0, torch.float32), None,
                       to_dev(pos, torch.float32), to_dev(Im, torch.float32), None])
        opts.append(api.make_opts(batch=n, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6, graph=True))
        oprs.append(api.make_opr_opts(8))
    losses = api.lsqml_epoch_opr_batched(recons, opts, oprs).cpu().numpy()
    for (dO, dU, dw, _, _, _, _), (O1, U1, w1, _, L1, _), L in zip(recons, refs, losses):
        e = (err(dO.cpu().numpy(), O1), err(dU.cpu().numpy(), U1, axis=0), err(dw.cpu().numpy(), w1, axis=1), abs(L - L1) / L1)
        print("uneven16opr first positions:", " ".join(f"{x:.2e}" for x in e))
        assert max(e) < TOL_EPOCH


def test_uneven16_opr_full_epochs_are_finite_and_lower_every_data_term():
    # all 16 reconstructions at full size (194,169 positions), data from the
    # GPU forward model with the true weights, three batched epochs from unit weights
    import torch
    from paper_2510_20929_gb300 import api
    dev = torch.device("cuda", 0)
    ws = synth.workload_uneven(16, seed=1005, opr_K=8)
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    recons = []
    for w in ws:
        Ot = torch.tensor(w["object"], dtype=torch.complex64, device=dev)
        pos = torch.tensor(w["pos"], dtype=torch.float32, device=dev)
        U = torch.tensor(w["opr_U"], dtype=torch.complex64, device=dev)
        wt = torch.tensor(w["opr_w"], dtype=torch.float32, device=dev)
        I0 = api.forward_opr(Ot, U, wt, None, pos)
        s = w["total_counts"] / I0.sum().item()
        U *= math.sqrt(s)
        recons.append([torch.ones_like(Ot), U, torch.ones_like(wt), None, pos, torch.poisson(I0 * s, generator=gen),
                       torch.tensor(synth.random_order(w["J"], 3), dtype=torch.int32, device=dev)])
        del Ot, I0
    opts = [api.make_opts(batch=w["batch"], graph=True) for w in ws]
    hist = [api.lsqml_epoch_opr_batched(recons, opts, api.make_opr_opts(8)).cpu().numpy() for _ in range(3)]
    print("uneven16opr losses per epoch:", [h.sum() for h in hist])
    assert all(np.isfinite(h).all() for h in hist)
    assert np.all(hist[2] < hist[0])
