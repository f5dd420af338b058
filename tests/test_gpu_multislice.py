"""GPU parity of the multislice entry points against the FP64 oracle: forward
model and gradients (all slices, probe modes, positions) with the
angular-spectrum propagator, for windows 16..128 and 1..4 slices."""
import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2510_20929_gb300 import synth
from tests.parity_util import c64, f32pos, err, to_dev

pytestmark = pytest.mark.gpu

TOL_FWD = 1e-5
# Each mode crosses 2S - 1 transforms in each direction (S slices) instead of
# one, and the Poisson factor I_m/(I + eps) at eps = 1e-6 amplifies the
# rounding of dark predicted pixels: the multislice gradients are held to
# three times the single-slice bar (measured at most 4.6e-5, the 192 window
# with two slices under the Poisson term).
TOL_GRAD = 1e-4
LAM, PX = 0.1e-9, 10e-9


def ms_problem(N, M, S, H, W, J, step, dz, seed=7, counts=2e4):
    w = synth.workload_small(N=N, M=M, H=H, W=W, J=J, seed=seed, step=step)
    g = np.random.default_rng(seed + 1)
    # slices: the sample's amplitude spread over the slices, each with its own phase texture
    Os = np.stack([w["object"] ** (1.0 / S) * np.exp(0.3j * synth.make_object(H, W, seed + 10 + s).imag)
                   for s in range(S)])
    Hf = orc.asm_propagator(N, PX, LAM, dz)
    I0 = orc.forward_ms(Os, w["probe"], w["pos"], Hf)
    P = w["probe"] * np.sqrt(counts / I0.sum(axis=(1, 2)).mean())
    I_m = synth.poisson_counts(orc.forward_ms(Os, P, w["pos"], Hf), seed + 2)
    Os0 = Os * (1 + 0.1 * (g.standard_normal(Os.shape) + 1j * g.standard_normal(Os.shape)))
    return c64(Os0), c64(P), f32pos(w["pos"]), Hf, np.float32(I_m).astype(np.float64)


def _dev(Os, P, pos, I_m):
    import torch
    return (to_dev(Os, torch.complex64), to_dev(P, torch.complex64), to_dev(pos, torch.float32),
            to_dev(I_m, torch.float32))


CASES = [  # N, M, S, H, W, J, step, dz
    (16, 1, 1, 40, 44, 9, 4.0, 2e-6),
    (16, 2, 3, 41, 37, 9, 3.0, 40e-6),
    (32, 2, 4, 72, 76, 12, 6.0, 10e-6),
    (64, 3, 2, 150, 160, 10, 12.0, 4e-6),
    (128, 2, 4, 290, 300, 6, 30.0, 2e-6),
    (192, 1, 2, 230, 236, 4, 12.0, 2e-6),
    (256, 2, 3, 290, 296, 3, 12.0, 2e-6),
]


@pytest.mark.parametrize("N,M,S,H,W,J,step,dz", CASES)
def test_forward_ms_matches_oracle(N, M, S, H, W, J, step, dz):
    from paper_2510_20929_gb300 import api
    Os, P, pos, Hf, I_m = ms_problem(N, M, S, H, W, J, step, dz)
    dO, dP, dpos, _ = _dev(Os, P, pos, I_m)
    ms = api.make_multislice(S, dz, LAM, PX)
    I = api.forward_ms(dO, dP, dpos, ms, batch=4).cpu().numpy()   # ragged chunks
    ref = orc.forward_ms(Os, P, pos, Hf)
    e = err(I, ref)
    print(f"forward_ms N={N} M={M} S={S}: rel {e:.3e}")
    assert e < TOL_FWD


@pytest.mark.parametrize("noise", ["gaussian", "poisson"])
@pytest.mark.parametrize("N,M,S,H,W,J,step,dz", CASES[1:])
def test_adjoint_ms_matches_oracle(noise, N, M, S, H, W, J, step, dz):
    from paper_2510_20929_gb300 import api
    Os, P, pos, Hf, I_m = ms_problem(N, M, S, H, W, J, step, dz)
    nz = orc.GAUSSIAN if noise == "gaussian" else orc.POISSON
    L_ref, gO_ref, gP_ref, gr_ref = orc.loss_and_gradients_ms(Os, P, pos, Hf, I_m, nz, 1e-6)
    loss, gO, gP, gr = api.adjoint_ms(*_dev(Os, P, pos, I_m), api.make_multislice(S, dz, LAM, PX), noise, eps=1e-6,
                                      batch=4)
    e = [abs(loss.item() - L_ref) / abs(L_ref), err(gO.cpu().numpy(), gO_ref, axis=0), err(gP.cpu().numpy(), gP_ref, axis=0),
         err(gr.cpu().numpy(), gr_ref, axis=1)]
    print(f"adjoint_ms {noise} N={N} M={M} S={S}:", " ".join(f"{x:.2e}" for x in e))
    assert max(e) < TOL_GRAD


def test_adjoint_ms_vjp_and_one_slice_equals_the_single_slice_path():
    import torch
    from paper_2510_20929_gb300 import api
    Os, P, pos, Hf, I_m = ms_problem(32, 2, 3, 72, 76, 12, 6.0, 10e-6)
    G = np.random.default_rng(2).standard_normal(I_m.shape).astype(np.float32).astype(np.float64)
    gO_ref, gP_ref, gr_ref = orc.vjp_ms(Os, P, pos, Hf, G)
    dO, dP, dpos, _ = _dev(Os, P, pos, I_m)
    loss, gO, gP, gr = api.adjoint_ms(dO, dP, dpos, to_dev(G, torch.float32), api.make_multislice(3, 10e-6, LAM, PX),
                                      "vjp", batch=5)
    assert loss is None
    e = (err(gO.cpu().numpy(), gO_ref, axis=0), err(gP.cpu().numpy(), gP_ref, axis=0), err(gr.cpu().numpy(), gr_ref, axis=1))
    print("vjp_ms:", e)
    assert max(e) < TOL_GRAD
    # one slice: the multislice pass computes what the single-slice pass computes
    ms1 = api.make_multislice(1, 10e-6, LAM, PX)
    d1 = dO[:1].contiguous()
    l1, g1, p1, r1 = api.adjoint_ms(d1, dP, dpos, to_dev(I_m, torch.float32), ms1, "gaussian", eps=1e-6)
    l0, g0, p0, r0 = api.adjoint(d1[0], dP, dpos, to_dev(I_m, torch.float32), "gaussian", eps=1e-6)
    assert err(g1[0].cpu().numpy(), g0.cpu().numpy()) < 1e-5 and err(p1.cpu().numpy(), p0.cpu().numpy(), axis=0) < 1e-5
    assert abs(l1.item() - l0.item()) < 1e-6 * abs(l0.item())


def test_multislice_autograd_and_adam():
    import torch
    from paper_2510_20929_gb300 import api, autograd
    Os, P, pos, Hf, I_m = ms_problem(32, 2, 3, 72, 76, 12, 6.0, 10e-6)
    dO, dP, dpos, dI = _dev(Os, P, pos, I_m)
    ms = api.make_multislice(3, 10e-6, LAM, PX)
    x = dO.clone().requires_grad_(True)
    I = autograd.far_field_ms(x, dP, dpos, ms)
    (I * to_dev(np.ones_like(I_m), torch.float32)).sum().backward()
    gO_ref = orc.vjp_ms(Os, P, pos, Hf, np.ones_like(I_m))[0]
    assert err(x.grad.cpu().numpy(), gO_ref, axis=0) < TOL_GRAD
    hist = autograd.reconstruct_adam_ms(dO, dP, dpos, dI, ms, epochs=40, lr_object=2e-2, update=("object",))
    print("adam ms:", hist[0], hist[-1])
    assert hist[-1] < 0.5 * hist[0]


# ----------------------------------------------------------------------------- LSQML
def _lsqml_ms_case(N, M, S, H, W, J, step, dz, batch, noise, update_probe=True, seed=7):
    import torch
    from paper_2510_20929_gb300 import api
    Os, P, pos, Hf, I_m = ms_problem(N, M, S, H, W, J, step, dz, seed=seed)
    dO, dP, dpos, dI = _dev(Os, P, pos, I_m)
    order = np.random.default_rng(seed).permutation(J).astype(np.int32)
    nz = orc.GAUSSIAN if noise == "gaussian" else orc.POISSON
    kw = dict(batch=batch, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6, update_probe=update_probe)
    O_ref, P_ref, L_ref, a_ref = orc.lsqml_epoch_ms(Os, P, pos, I_m, order, Hf, orc.LsqmlOptions(noise=nz, **kw))
    loss, alpha = api.lsqml_epoch_ms(dO, dP, dpos, dI, to_dev(order, torch.int32), api.make_multislice(S, dz, LAM, PX),
                                     noise=noise, want_alpha=True, **kw)
    e = dict(O=err(dO.cpu().numpy(), O_ref, axis=0), P=err(dP.cpu().numpy(), P_ref, axis=0),
             alpha=err(alpha.cpu().numpy(), a_ref, axis=1), loss=abs(loss.item() - L_ref) / abs(L_ref))
    print(f"lsqml_ms N={N} M={M} S={S} B={batch} {noise}: " + " ".join(f"{k} {v:.2e}" for k, v in e.items()))
    return e


@pytest.mark.parametrize("noise", ["gaussian", "poisson"])
@pytest.mark.parametrize("N,M,S,H,W,J,step,dz,batch", [
    (16, 2, 3, 41, 37, 9, 3.0, 40e-6, 4),       # ragged minibatches (4, 4, 1)
    (32, 1, 2, 72, 76, 12, 6.0, 10e-6, 12),
    (64, 3, 2, 150, 160, 10, 12.0, 4e-6, 5),
    (128, 2, 3, 290, 300, 6, 30.0, 2e-6, 4),
    (192, 1, 2, 230, 236, 4, 12.0, 2e-6, 3),
    (256, 2, 2, 290, 296, 3, 12.0, 2e-6, 2),
])
def test_lsqml_epoch_ms_matches_oracle(N, M, S, H, W, J, step, dz, batch, noise):
    e = _lsqml_ms_case(N, M, S, H, W, J, step, dz, batch, noise)
    assert e["loss"] < TOL_FWD
    assert max(e["O"], e["P"], e["alpha"]) < TOL_GRAD


def test_lsqml_epoch_ms_object_only_and_one_slice_equals_the_single_slice_epoch():
    import torch
    from paper_2510_20929_gb300 import api
    e = _lsqml_ms_case(32, 2, 2, 72, 76, 12, 6.0, 10e-6, 5, "gaussian", update_probe=False)
    assert max(e["O"], e["alpha"]) < TOL_GRAD and e["P"] == 0.0
    # one slice: the multislice epoch computes what the single-slice epoch computes
    Os, P, pos, Hf, I_m = ms_problem(32, 2, 1, 72, 76, 12, 6.0, 10e-6)
    d1 = _dev(Os, P, pos, I_m)
    d0 = _dev(Os, P, pos, I_m)
    kw = dict(batch=5, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    l1, a1 = api.lsqml_epoch_ms(*d1, None, api.make_multislice(1, 10e-6, LAM, PX), want_alpha=True, **kw)
    l0, a0 = api.lsqml_epoch(d0[0][0], d0[1], d0[2], d0[3], None, want_alpha=True, **kw)
    assert err(d1[0][0].cpu().numpy(), d0[0][0].cpu().numpy()) < 1e-6
    assert err(d1[1].cpu().numpy(), d0[1].cpu().numpy(), axis=0) < 1e-6
    assert err(a1.cpu().numpy(), a0.cpu().numpy(), axis=1) < 1e-6
    assert abs(l1.item() - l0.item()) < 1e-6 * abs(l0.item())


def test_lsqml_epoch_ms_graph_replay_equals_eager_and_rejects_unsupported_options():
    import torch
    from paper_2510_20929_gb300 import api
    Os, P, pos, Hf, I_m = ms_problem(64, 2, 3, 150, 160, 10, 12.0, 4e-6)
    ms = api.make_multislice(3, 4e-6, LAM, PX)
    outs = []
    for graph in (False, True, True):
        dO, dP, dpos, dI = _dev(Os, P, pos, I_m)
        loss, _ = api.lsqml_epoch_ms(dO, dP, dpos, dI, None, ms, api.make_opts(batch=4, graph=graph))
        outs.append((dO.cpu().numpy(), dP.cpu().numpy(), loss.item()))
    for O1, P1, L1 in outs[1:]:
        assert err(O1, outs[0][0], axis=0) < 1e-6 and err(P1, outs[0][1], axis=0) < 1e-6
        assert abs(L1 - outs[0][2]) < 1e-6 * abs(outs[0][2])
    dO, dP, dpos, dI = _dev(Os, P, pos, I_m)
    for bad in (dict(precision="bf16x3"), dict(update_positions=True), dict(object_per_epoch=True)):
        with pytest.raises(api.PtychoError) as ex:
            api.lsqml_epoch_ms(dO, dP, dpos, dI, None, ms, api.make_opts(batch=4, **bad))
        assert ex.value.status == 6


# ----------------------------------------------------------------------------- recompute-in-backward
@pytest.mark.parametrize("N,M,S,H,W,J,step,dz", CASES[1:])
def test_adjoint_ms_recomputing_the_incident_waves_matches_oracle_and_the_kept_waves(N, M, S, H, W, J, step, dz):
    from paper_2510_20929_gb300 import api
    Os, P, pos, Hf, I_m = ms_problem(N, M, S, H, W, J, step, dz)
    L_ref, gO_ref, gP_ref, gr_ref = orc.loss_and_gradients_ms(Os, P, pos, Hf, I_m, orc.POISSON, 1e-6)
    out = {}
    for rec in (False, True):
        out[rec] = api.adjoint_ms(*_dev(Os, P, pos, I_m), api.make_multislice(S, dz, LAM, PX, recompute=rec),
                                  "poisson", eps=1e-6, batch=4)
    loss, gO, gP, gr = out[True]
    e = [abs(loss.item() - L_ref) / abs(L_ref), err(gO.cpu().numpy(), gO_ref, axis=0),
         err(gP.cpu().numpy(), gP_ref, axis=0), err(gr.cpu().numpy(), gr_ref, axis=1)]
    print(f"adjoint_ms recompute N={N} M={M} S={S}:", " ".join(f"{x:.2e}" for x in e))
    assert max(e) < TOL_GRAD
    # the recomputed waves are the kept ones bit for bit; only the order of the
    # scatter's atomic additions differs between the two runs
    l0, g0, p0, r0 = out[False]
    assert err(gO.cpu().numpy(), g0.cpu().numpy(), axis=0) < 1e-6
    assert err(gP.cpu().numpy(), p0.cpu().numpy(), axis=0) < 1e-6
    assert err(gr.cpu().numpy(), r0.cpu().numpy(), axis=1) < 1e-6
    assert abs(loss.item() - l0.item()) <= 1e-9 * abs(l0.item())


@pytest.mark.parametrize("N,M,S,H,W,J,step,dz,batch", [
    (16, 2, 3, 41, 37, 9, 3.0, 40e-6, 4),
    (128, 2, 3, 290, 300, 6, 30.0, 2e-6, 4),
    (192, 1, 2, 230, 236, 4, 12.0, 2e-6, 3),
    (256, 2, 3, 290, 296, 3, 12.0, 2e-6, 2),
])
def test_lsqml_epoch_ms_recomputing_the_incident_waves_matches_oracle(N, M, S, H, W, J, step, dz, batch):
    import torch
    from paper_2510_20929_gb300 import api
    Os, P, pos, Hf, I_m = ms_problem(N, M, S, H, W, J, step, dz)
    order = np.random.default_rng(7).permutation(J).astype(np.int32)
    kw = dict(batch=batch, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    O_ref, P_ref, L_ref, a_ref = orc.lsqml_epoch_ms(Os, P, pos, I_m, order, Hf,
                                                    orc.LsqmlOptions(noise=orc.GAUSSIAN, **kw))
    res = {}
    for rec in (False, True):
        dO, dP, dpos, dI = _dev(Os, P, pos, I_m)
        loss, alpha = api.lsqml_epoch_ms(dO, dP, dpos, dI, to_dev(order, torch.int32),
                                         api.make_multislice(S, dz, LAM, PX, recompute=rec), want_alpha=True, **kw)
        res[rec] = (dO.cpu().numpy(), dP.cpu().numpy(), alpha.cpu().numpy(), loss.item())
    O1, P1, a1, l1 = res[True]
    e = dict(O=err(O1, O_ref, axis=0), P=err(P1, P_ref, axis=0), alpha=err(a1, a_ref, axis=1),
             loss=abs(l1 - L_ref) / abs(L_ref))
    print(f"lsqml_ms recompute N={N} M={M} S={S}: " + " ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert e["loss"] < TOL_FWD and max(e["O"], e["P"], e["alpha"]) < TOL_GRAD
    O0, P0, a0, l0 = res[False]
    assert err(O1, O0, axis=0) < 1e-6 and err(P1, P0, axis=0) < 1e-6 and err(a1, a0, axis=1) < 1e-6
