"""GPU parity: the CUDA library through its C ABI against the FP64 oracle on the
same seeded inputs."""
import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from tests.parity_util import TOL_EPOCH, TOL_FWD, TOL_GRAD, c64, err, f32pos, problem, rel, to_dev

pytestmark = pytest.mark.gpu



def _dev(p):
    import torch
    O, P, pos, I_m = c64(p["O"]), c64(p["P"]), f32pos(p["pos"]), np.float32(p["I_m"]).astype(np.float64)
    return (O, P, pos, I_m), (to_dev(O, torch.complex64), to_dev(P, torch.complex64),
                              to_dev(pos, torch.float32), to_dev(I_m, torch.float32))


CASES = [  # N, M, H, W, J, step
    (16, 1, 40, 44, 12, 4.0),
    (16, 3, 41, 37, 9, 3.0),
    (32, 2, 72, 76, 16, 6.0),
    (64, 1, 160, 150, 25, 12.0),
    (64, 3, 150, 160, 20, 12.0),
    (128, 2, 300, 310, 12, 24.0),
    (128, 5, 290, 300, 9, 30.0),
]


@pytest.mark.parametrize("N,M,H,W,J,step", CASES)
def test_forward_matches_oracle(N, M, H, W, J, step):
    from paper_2510_20929_gb300 import api
    p = problem(N=N, M=M, H=H, W=W, J=J, step=step)
    (O, P, pos, _), (dO, dP, dpos, _) = _dev(p)
    I = api.forward(dO, dP, dpos).cpu().numpy()
    ref = orc.forward(O, P, pos)
    e = err(I, ref)
    print(f"forward N={N} M={M}: rel {e:.3e}")
    assert e < TOL_FWD
    for j in range(J):
        assert rel(I[j], ref[j]) < 10 * TOL_FWD


@pytest.mark.parametrize("noise", ["gaussian", "poisson"])
@pytest.mark.parametrize("N,M,H,W,J,step", [CASES[1], CASES[2], CASES[4], CASES[6]])
def test_gradients_match_oracle(noise, N, M, H, W, J, step):
    from paper_2510_20929_gb300 import api
    p = problem(N=N, M=M, H=H, W=W, J=J, step=step)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    eps = 1e-6
    nz = orc.GAUSSIAN if noise == "gaussian" else orc.POISSON
    L_ref, gO_ref, gP_ref, gr_ref = orc.loss_and_gradients(O, P, pos, I_m, nz, eps)
    loss, gO, gP, gr = api.adjoint(dO, dP, dpos, dI, noise, eps=eps, batch=5)
    e = (abs(loss.item() - L_ref) / abs(L_ref), err(gO.cpu().numpy(), gO_ref),
         err(gP.cpu().numpy(), gP_ref, axis=0), err(gr.cpu().numpy(), gr_ref, axis=1))
    print(f"grad {noise} N={N} M={M}: loss {e[0]:.2e} gO {e[1]:.2e} gP {e[2]:.2e} gr {e[3]:.2e}")
    assert e[0] < TOL_FWD
    assert max(e[1:]) < TOL_GRAD


def test_vjp_matches_oracle():
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=32, M=3, H=72, W=76, J=16, step=6.0)
    (O, P, pos, _), (dO, dP, dpos, _) = _dev(p)
    G = np.float32(np.random.default_rng(4).standard_normal((16, 32, 32))).astype(np.float64)
    gO_ref, gP_ref, gr_ref = orc.vjp(O, P, pos, G)
    loss, gO, gP, gr = api.adjoint(dO, dP, dpos, to_dev(G, torch.float32), "vjp", batch=7)
    assert loss is None
    e = (err(gO.cpu().numpy(), gO_ref), err(gP.cpu().numpy(), gP_ref, axis=0), err(gr.cpu().numpy(), gr_ref, axis=1))
    print(f"vjp: {e}")
    assert max(e) < TOL_GRAD


def _epoch_case(N, M, H, W, J, step, batch, noise, update_probe=True, seed=7):
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=N, M=M, H=H, W=W, J=J, step=step, seed=seed)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    order = np.random.default_rng(seed).permutation(J).astype(np.int32)
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN if noise == "gaussian" else orc.POISSON, batch=batch,
                            delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6, update_probe=update_probe)
    O_ref, P_ref, L_ref, a_ref = orc.lsqml_epoch(O, P, pos, I_m, order, opts)
    loss, alpha = api.lsqml_epoch(dO, dP, dpos, dI, to_dev(order, torch.int32), noise=noise, batch=batch,
                                  delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6, update_probe=update_probe,
                                  want_alpha=True)
    e = dict(O=err(dO.cpu().numpy(), O_ref), P=err(dP.cpu().numpy(), P_ref, axis=0),
             alpha=err(alpha.cpu().numpy(), a_ref, axis=1), loss=abs(loss.item() - L_ref) / abs(L_ref))
    print(f"epoch N={N} M={M} J={J} B={batch} {noise}: " + " ".join(f"{k} {v:.2e}" for k, v in e.items()))
    return e


@pytest.mark.parametrize("N,M,H,W,J,step,batch", [
    (16, 2, 40, 44, 12, 4.0, 12),       # one batch
    (16, 2, 40, 44, 12, 4.0, 5),        # ragged last batch (5, 5, 2)
    (32, 3, 72, 76, 16, 6.0, 6),
    (64, 1, 160, 150, 25, 12.0, 8),
    (128, 5, 290, 300, 9, 30.0, 4),
])
@pytest.mark.parametrize("noise", ["gaussian", "poisson"])
def test_lsqml_epoch_matches_oracle(N, M, H, W, J, step, batch, noise):
    e = _epoch_case(N, M, H, W, J, step, batch, noise)
    assert e["loss"] < TOL_FWD
    assert e["alpha"] < TOL_EPOCH
    assert e["O"] < TOL_EPOCH and e["P"] < TOL_EPOCH


@pytest.mark.parametrize("N,M,H,W,J,step,batch", [
    (16, 2, 200, 180, 12, 4.0, 4),
    (64, 1, 600, 620, 10, 12.0, 3),
    (256, 1, 600, 620, 4, 10.0, 2),
])
def test_lsqml_epoch_on_a_large_object_matches_oracle(N, M, H, W, J, step, batch):
    # the batch's tiles cover a small part of the object: the illumination
    # maximum and the accumulator clear visit only those tiles
    e = _epoch_case(N, M, H, W, J, step, batch, "gaussian")
    assert e["loss"] < TOL_FWD and e["alpha"] < TOL_EPOCH and e["O"] < TOL_EPOCH and e["P"] < TOL_EPOCH


def test_lsqml_epoch_object_only_matches_oracle():
    e = _epoch_case(32, 2, 72, 76, 16, 6.0, 16, "gaussian", update_probe=False)
    assert e["O"] < TOL_EPOCH and e["P"] == 0.0 and e["alpha"] < TOL_EPOCH


def _state_case(N, M, H, W, J, step, batch, update_positions, object_per_epoch, seed=11, shift=0.8):
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=N, M=M, H=H, W=W, J=J, step=step, seed=seed)
    g = np.random.default_rng(seed + 3)
    p["pos"] = p["pos"] + (g.uniform(-shift, shift, p["pos"].shape) if update_positions else 0.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    order = np.random.default_rng(seed).permutation(J).astype(np.int32)
    kw = dict(batch=batch, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    opts = orc.LsqmlOptions(**kw, update_positions=update_positions, pos_step=0.9, pos_max_shift=0.5,
                            object_per_epoch=object_per_epoch)
    O_ref, P_ref, pos_ref, L_ref, a_ref = orc.lsqml_epoch_state(O, P, pos, I_m, order, opts)
    loss, alpha = api.lsqml_epoch(dO, dP, dpos, dI, to_dev(order, torch.int32), want_alpha=True, **kw,
                                  update_positions=update_positions, pos_step=0.9, pos_max_shift=0.5,
                                  object_per_epoch=object_per_epoch)
    e = dict(O=err(dO.cpu().numpy(), O_ref), P=err(dP.cpu().numpy(), P_ref, axis=0),
             alpha=err(alpha.cpu().numpy(), a_ref, axis=1), loss=abs(loss.item() - L_ref) / abs(L_ref))
    dpos_err = float(np.max(np.abs(dpos.cpu().numpy().astype(np.float64) - pos_ref)))
    moved = float(np.max(np.abs(pos_ref - pos)))
    print(f"epoch N={N} M={M} pos={update_positions} per_epoch={object_per_epoch}: "
          + " ".join(f"{k} {v:.2e}" for k, v in e.items()) + f" pos {dpos_err:.2e} px (moved {moved:.2e})")
    return e, dpos_err, moved


@pytest.mark.parametrize("N,M,H,W,J,step,batch", [
    (16, 2, 44, 48, 12, 4.0, 5),
    (64, 3, 160, 150, 14, 12.0, 6),
    (128, 2, 300, 310, 9, 24.0, 4),
    (256, 1, 320, 330, 4, 20.0, 3),
])
def test_lsqml_epoch_with_position_correction_matches_oracle(N, M, H, W, J, step, batch):
    e, dpos_err, moved = _state_case(N, M, H, W, J, step, batch, True, False)
    assert max(e.values()) < TOL_EPOCH
    assert moved > 1e-3 and dpos_err < 1e-3   # px; positions are float32 values near 100 px


@pytest.mark.parametrize("N,M,H,W,J,step,batch", [
    (16, 2, 44, 48, 12, 4.0, 5),
    (64, 1, 160, 150, 25, 12.0, 8),
    (192, 1, 256, 266, 6, 20.0, 4),
])
def test_lsqml_epoch_with_per_epoch_object_update_matches_oracle(N, M, H, W, J, step, batch):
    e, _, _ = _state_case(N, M, H, W, J, step, batch, False, True)
    assert max(e.values()) < TOL_EPOCH


def test_lsqml_epoch_with_both_modes_on_host_buffers_matches_oracle():
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=32, M=2, H=72, W=76, J=16, step=6.0, seed=13)
    p["pos"] = p["pos"] + np.random.default_rng(4).uniform(-0.5, 0.5, p["pos"].shape)
    O, P, pos, I_m = c64(p["O"]), c64(p["P"]), f32pos(p["pos"]), np.float32(p["I_m"]).astype(np.float64)
    order = np.random.default_rng(2).permutation(16).astype(np.int32)
    kw = dict(batch=6, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    opts = orc.LsqmlOptions(**kw, update_positions=True, object_per_epoch=True)
    O_ref, P_ref, pos_ref, L_ref, _ = orc.lsqml_epoch_state(O, P, pos, I_m, order, opts)
    hO = torch.tensor(O, dtype=torch.complex64).pin_memory()
    hP = torch.tensor(P, dtype=torch.complex64).pin_memory()
    hpos = torch.tensor(pos, dtype=torch.float32).pin_memory()
    hI = torch.tensor(I_m, dtype=torch.float32).pin_memory()
    L = api.lsqml_epoch_host(hO, hP, hpos, hI, torch.tensor(order), api.make_opts(**kw, update_positions=True,
                                                                                   object_per_epoch=True))
    e = (err(hO.numpy(), O_ref), err(hP.numpy(), P_ref, axis=0), abs(L - L_ref) / L_ref,
         float(np.max(np.abs(hpos.numpy() - pos_ref))))
    print("host epoch, both modes:", e)
    assert max(e[:3]) < TOL_EPOCH and e[3] < 1e-3


@pytest.mark.parametrize("batch", [8, 3])
def test_host_epoch_with_pinned_and_with_pageable_intensities_match_oracle(batch):
    # pinned (mapped) intensities are read in place by the passes, pageable ones
    # staged first; with four minibatches or more (batch 3: seven) the later
    # ones read the copy a worker stream makes during the first ones
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=64, M=2, H=150, W=160, J=20, step=12.0, seed=17)
    O, P, pos, I_m = c64(p["O"]), c64(p["P"]), f32pos(p["pos"]), np.float32(p["I_m"]).astype(np.float64)
    order = np.random.default_rng(6).permutation(20).astype(np.int32)
    kw = dict(batch=batch, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    O_ref, P_ref, L_ref, _ = orc.lsqml_epoch(O, P, pos, I_m, order, orc.LsqmlOptions(**kw))
    out = []
    for pinned in (True, False):
        hI = torch.tensor(I_m, dtype=torch.float32)
        if pinned:
            hI = hI.pin_memory()
        hO = torch.tensor(O, dtype=torch.complex64).pin_memory()
        hP = torch.tensor(P, dtype=torch.complex64).pin_memory()
        L = api.lsqml_epoch_host(hO, hP, torch.tensor(pos, dtype=torch.float32), hI, torch.tensor(order),
                                 api.make_opts(**kw))
        e = (err(hO.numpy(), O_ref), err(hP.numpy(), P_ref, axis=0), abs(L - L_ref) / L_ref)
        print(f"host epoch, {'pinned' if pinned else 'pageable'} intensities:", e)
        assert max(e) < TOL_EPOCH
        out.append(hO.numpy())
    assert err(out[0], out[1]) < 1e-5


def test_compact_sampler_with_per_epoch_object_update_matches_oracle():
    # the compact sampler's order and the accumulate-once object update, as
    # LSQML pairs them, over an epoch of several minibatches
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=32, M=2, H=120, W=124, J=64, step=6.0, seed=17)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    order = api.sampler_order(torch.tensor(pos, dtype=torch.float32), 16, "compact").numpy()
    assert np.array_equal(order, orc.sampler_order(pos, 16, orc.SAMPLER_COMPACT))
    kw = dict(batch=16, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    O_ref, P_ref, _, L_ref, a_ref = orc.lsqml_epoch_state(O, P, pos, I_m, order,
                                                          orc.LsqmlOptions(**kw, object_per_epoch=True))
    loss, alpha = api.lsqml_epoch(dO, dP, dpos, dI, to_dev(order, torch.int32), want_alpha=True, **kw,
                                  object_per_epoch=True)
    e = (err(dO.cpu().numpy(), O_ref), err(dP.cpu().numpy(), P_ref, axis=0), err(alpha.cpu().numpy(), a_ref, axis=1),
         abs(loss.item() - L_ref) / L_ref)
    print("compact + per-epoch:", e)
    assert max(e) < TOL_EPOCH


@pytest.mark.parametrize("pass1,pass2,reduce", [(0, 0, 0), (1, 1, 1), (2, 0, 2), (2, 1, 0), (0, 2, 1), (1, 3, 3)])
def test_every_tuned_variant_matches_oracle(pass1, pass2, reduce):
    # the autotuner's candidates pinned one combination at a time (window 128:
    # 1024 threads, 512 threads, the pair of CTAs; single, split or cluster
    # step-size pass at 4 or 3 CTAs per SM; 16, 8 or 32 positions in flight
    # in the probe reduction, or the batch split over 4 threads)
    import torch
    from paper_2510_20929_gb300 import api
    N, M, H, W, J, step, batch = 128, 3, 300, 310, 10, 24.0, 4
    p = problem(N=N, M=M, H=H, W=W, J=J, step=step, seed=19)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    order = np.random.default_rng(19).permutation(J).astype(np.int32)
    api.set_tuning(api.dims_of(dO, dP, dpos), batch, pass1, pass2, reduce)
    kw = dict(batch=batch, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    O_ref, P_ref, L_ref, a_ref = orc.lsqml_epoch(O, P, pos, I_m, order, orc.LsqmlOptions(**kw))
    loss, alpha = api.lsqml_epoch(dO, dP, dpos, dI, to_dev(order, torch.int32), want_alpha=True, autotune=True, **kw)
    assert api.tuning(api.dims_of(dO, dP, dpos), batch)["pass1"] == pass1     # pinned, not retuned
    e = (err(dO.cpu().numpy(), O_ref), err(dP.cpu().numpy(), P_ref, axis=0), err(alpha.cpu().numpy(), a_ref, axis=1),
         abs(loss.item() - L_ref) / abs(L_ref))
    print(f"variants {pass1}/{pass2}/{reduce}:", e)
    assert max(e[:3]) < TOL_EPOCH and e[3] < TOL_FWD
