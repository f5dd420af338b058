"""GPU parity of the orthogonal-probe-relaxation entry points against the FP64
oracle: forward model, gradients (object, eigenmodes, weights, shared modes,
positions) and the LSQML epoch with eigenmode and weight updates, for the
shared-memory windows and the cluster windows (192, 256)."""
import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from tests.parity_util import TOL_EPOCH, TOL_FWD, TOL_GRAD, c64, err, f32pos, opr_problem, rel, to_dev

pytestmark = pytest.mark.gpu



def _host(p):
    O, U, pos = c64(p["O"]), c64(p["U"]), f32pos(p["pos"])
    w = np.float32(p["w"]).astype(np.float64)
    Pr = c64(p["P_rest"]) if p["P_rest"] is not None else None
    I_m = np.float32(p["I_m"]).astype(np.float64)
    return O, U, w, Pr, pos, I_m


def _dev(h):
    import torch
    O, U, w, Pr, pos, I_m = h
    return (to_dev(O, torch.complex64), to_dev(U, torch.complex64), to_dev(w, torch.float32),
            to_dev(Pr, torch.complex64) if Pr is not None else None, to_dev(pos, torch.float32),
            to_dev(I_m, torch.float32))


CASES = [  # N, K, M, H, W, J, step
    (16, 1, 1, 40, 44, 12, 4.0),
    (16, 3, 2, 41, 37, 9, 3.0),
    (32, 4, 1, 72, 76, 16, 6.0),
    (64, 2, 3, 150, 160, 14, 12.0),
    (128, 8, 2, 290, 300, 9, 30.0),
]
CLUSTER_CASES = [
    (192, 3, 2, 230, 236, 4, 12.0),
    (256, 2, 1, 290, 296, 4, 12.0),
]


@pytest.mark.parametrize("N,K,M,H,W,J,step", CASES + CLUSTER_CASES)
def test_forward_opr_matches_oracle(N, K, M, H, W, J, step):
    from paper_2510_20929_gb300 import api
    h = _host(opr_problem(N=N, K=K, M=M, H=H, W=W, J=J, step=step))
    d = _dev(h)
    I = api.forward_opr(*d[:5]).cpu().numpy()
    ref = orc.forward_opr(*h[:5])
    e = err(I, ref)
    print(f"forward_opr N={N} K={K} M={M}: rel {e:.3e}")
    assert e < TOL_FWD
    for j in range(J):
        assert rel(I[j], ref[j]) < 10 * TOL_FWD


@pytest.mark.parametrize("noise", ["gaussian", "poisson"])
@pytest.mark.parametrize("N,K,M,H,W,J,step", [CASES[1], CASES[2], CASES[3], CASES[4], CLUSTER_CASES[0]])
def test_adjoint_opr_matches_oracle(noise, N, K, M, H, W, J, step):
    from paper_2510_20929_gb300 import api
    h = _host(opr_problem(N=N, K=K, M=M, H=H, W=W, J=J, step=step))
    O, U, w, Pr, pos, I_m = h
    eps = 1e-6
    nz = orc.GAUSSIAN if noise == "gaussian" else orc.POISSON
    L_ref, gO_ref, gU_ref, gw_ref, gP_ref, gr_ref = orc.loss_and_gradients_opr(O, U, w, Pr, pos, I_m, nz, eps)
    loss, gO, gU, gw, gP, gr = api.adjoint_opr(*_dev(h), noise, eps=eps, batch=4)   # ragged chunks
    e = [abs(loss.item() - L_ref) / abs(L_ref), err(gO.cpu().numpy(), gO_ref), err(gU.cpu().numpy(), gU_ref, axis=0),
         err(gw.cpu().numpy(), gw_ref, axis=1), err(gr.cpu().numpy(), gr_ref, axis=1)]
    if Pr is not None:
        e.append(err(gP.cpu().numpy(), gP_ref, axis=0))
    print(f"adjoint_opr {noise} N={N} K={K} M={M}:", " ".join(f"{x:.2e}" for x in e))
    assert max(e) < TOL_GRAD


def test_adjoint_opr_vjp_mode_is_the_chain_rule_of_the_forward():
    # dL/dI = G given directly: the gradients equal the oracle's vjp
    import torch
    from paper_2510_20929_gb300 import api
    h = _host(opr_problem(N=32, K=3, M=2, H=72, W=76, J=10, step=6.0))
    O, U, w, Pr, pos, _ = h
    G = np.random.default_rng(3).standard_normal((10, 32, 32)).astype(np.float32).astype(np.float64)
    gO_ref, gU_ref, gw_ref, gP_ref, gr_ref = orc.vjp_opr(O, U, w, Pr, pos, G)
    d = _dev(h)
    loss, gO, gU, gw, gP, gr = api.adjoint_opr(*d[:5], to_dev(G, torch.float32), "vjp", batch=3)
    assert loss is None
    e = [err(gO.cpu().numpy(), gO_ref), err(gU.cpu().numpy(), gU_ref, axis=0), err(gw.cpu().numpy(), gw_ref, axis=1),
         err(gP.cpu().numpy(), gP_ref, axis=0), err(gr.cpu().numpy(), gr_ref, axis=1)]
    print("vjp_opr:", " ".join(f"{x:.2e}" for x in e))
    assert max(e) < TOL_GRAD


def _epoch_case(N, K, M, H, W, J, step, batch, update_weights, noise="gaussian", seed=7):
    import torch
    from paper_2510_20929_gb300 import api
    h = _host(opr_problem(N=N, K=K, M=M, H=H, W=W, J=J, step=step, seed=seed))
    O, U, w, Pr, pos, I_m = h
    order = np.random.default_rng(seed + 1).permutation(J).astype(np.int32)
    opts_o = orc.LsqmlOptions(noise=orc.GAUSSIAN if noise == "gaussian" else orc.POISSON, batch=batch,
                              delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    opr_o = orc.OprOptions(update_weights=update_weights, weight_step=0.8)
    ref = orc.lsqml_epoch_opr(O, U, w, Pr, pos, I_m, order, opts_o, opr_o)
    dO, dU, dw, dPr, dpos, dI = _dev(h)
    opts = api.make_opts(noise=noise, batch=batch, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    opr = api.make_opr_opts(K, update_weights=update_weights, weight_step=0.8)
    loss, alpha = api.lsqml_epoch_opr(dO, dU, dw, dPr, dpos, dI, to_dev(order, torch.int32), opts, opr,
                                      want_alpha=True)
    O1, U1, w1, Pr1, L1, a1 = ref
    e = {"O": err(dO.cpu().numpy(), O1), "U": err(dU.cpu().numpy(), U1, axis=0), "w": err(dw.cpu().numpy(), w1, axis=1),
         "alpha": err(alpha.cpu().numpy(), a1, axis=1), "loss": abs(loss.item() - L1) / abs(L1)}
    if Pr is not None:
        e["P_rest"] = err(dPr.cpu().numpy(), Pr1, axis=0)
    # the weights moved (when updated), so the comparison is not vacuous
    dw_ref = rel(w1, w)
    return e, dw_ref


@pytest.mark.parametrize("update_weights", [False, True])
@pytest.mark.parametrize("N,K,M,H,W,J,step", [CASES[1], CASES[2], CASES[3], CASES[4]])
def test_lsqml_epoch_opr_matches_oracle(update_weights, N, K, M, H, W, J, step):
    batch = 4 if J > 4 else J
    e, moved = _epoch_case(N, K, M, H, W, J, step, batch, update_weights)
    print(f"lsqml_opr N={N} K={K} M={M} weights={update_weights}:",
          " ".join(f"{k} {v:.2e}" for k, v in e.items()), f"(weights moved {moved:.2e})")
    assert max(e.values()) < TOL_EPOCH
    if update_weights:
        assert moved > 1e-4


def test_lsqml_epoch_opr_poisson_matches_oracle():
    e, _ = _epoch_case(32, 3, 2, 72, 76, 16, 6.0, 6, True, noise="poisson")
    print("lsqml_opr poisson:", " ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert max(e.values()) < TOL_EPOCH


@pytest.mark.parametrize("N,K,M,H,W,J,step", CLUSTER_CASES + [(32, 3, 2, 300, 280, 12, 6.0)])
def test_lsqml_epoch_opr_cluster_windows_match_oracle(N, K, M, H, W, J, step):
    e, moved = _epoch_case(N, K, M, H, W, J, step, 3, True)
    print(f"lsqml_opr N={N} K={K} M={M}:", " ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert max(e.values()) < TOL_EPOCH and moved > 1e-4


def test_lsqml_epoch_opr_graph_replay_matches_direct():
    import torch
    from paper_2510_20929_gb300 import api
    h = _host(opr_problem(N=32, K=3, M=2, H=72, W=76, J=16, step=6.0))
    outs = []
    for graph in (False, True):
        dO, dU, dw, dPr, dpos, dI = _dev(h)
        opts = api.make_opts(batch=6, delta_o=0.1, delta_p=0.1, eps=1e-6, graph=graph)
        opr = api.make_opr_opts(3, weight_step=0.8)
        for _ in range(3):   # capture once, then replay
            loss, _ = api.lsqml_epoch_opr(dO, dU, dw, dPr, dpos, dI, None, opts, opr)
        outs.append((dO.cpu().numpy(), dU.cpu().numpy(), dw.cpu().numpy(), loss.item()))
    (O0, U0, w0, L0), (O1, U1, w1, L1) = outs
    assert err(O1, O0) < 1e-5 and err(U1, U0) < 1e-5 and err(w1, w0) < 1e-5 and abs(L1 - L0) < 1e-5 * abs(L0)


def test_opr_rejects_bad_arguments():
    import ctypes
    from paper_2510_20929_gb300 import api
    L = api.lib()
    d = api.Dims(72, 76, 32, 2, 16)
    assert L.ptycho_workspace_bytes_opr(ctypes.byref(d), 0, 4) == 0
    assert L.ptycho_workspace_bytes_opr(ctypes.byref(d), 9, 4) == 0
    h = _host(opr_problem(N=32, K=3, M=2, H=72, W=76, J=16, step=6.0))
    dO, dU, dw, dPr, dpos, dI = _dev(h)
    opts = api.make_opts(batch=4)
    opr = api.make_opr_opts(3)
    ws = api.workspace(d, 4, dO.device, opr_K=3)
    # shared modes missing while M = 2: rejected on the host, nothing launched
    st = L.ptycho_lsqml_epoch_opr(ctypes.byref(d), ctypes.byref(opr), api._ptr(dO), api._ptr(dU), api._ptr(dw),
                                  None, api._ptr(dpos), api._ptr(dI), None, ctypes.byref(opts), None, None,
                                  api._P(ws.ptr), ws.nbytes, api._stream())
    assert st == 1
    opr.K = 2   # K disagrees with nothing the library can see, but the reserved words must be zero
    opr.reserved[0] = 1
    st = L.ptycho_lsqml_epoch_opr(ctypes.byref(d), ctypes.byref(opr), api._ptr(dO), api._ptr(dU), api._ptr(dw),
                                  api._ptr(dPr), api._ptr(dpos), api._ptr(dI), None, ctypes.byref(opts), None,
                                  None, api._P(ws.ptr), ws.nbytes, api._stream())
    assert st == 1


def test_data_term_opr_autograd_and_adam():
    # the autograd Function returns the library's gradients; Adam on object,
    # eigenmodes and weights lowers the data term
    import torch
    from paper_2510_20929_gb300 import api, autograd
    h = _host(opr_problem(N=32, K=3, M=2, H=72, W=76, J=16, step=6.0, perturb=0.3, w_perturb=0.1))
    dO, dU, dw, dPr, dpos, dI = _dev(h)
    O, U, w, Pr, pos, I_m = h
    L_ref, gO_ref, gU_ref, gw_ref, _, _ = orc.loss_and_gradients_opr(O, U, w, Pr, pos, I_m, orc.GAUSSIAN, 1e-6)
    x = [t.clone().requires_grad_(True) for t in (dO, dU, dw)]
    loss = autograd.data_term_opr(x[0], x[1], x[2], dPr, dpos, dI, "gaussian", 1e-6)
    (2.0 * loss).backward()
    e = [abs(loss.item() - L_ref) / L_ref, err(x[0].grad.cpu().numpy(), 2 * gO_ref),
         err(x[1].grad.cpu().numpy(), 2 * gU_ref, axis=0), err(x[2].grad.cpu().numpy(), 2 * gw_ref, axis=1)]
    print("autograd opr:", " ".join(f"{v:.2e}" for v in e))
    assert max(e) < TOL_GRAD
    hist = autograd.reconstruct_adam_opr(dO, dU, dw, dPr, dpos, dI, epochs=40, lr_object=2e-2, lr_probe=2e-2,
                                         lr_weights=1e-2, update=("object", "eigenmodes", "weights"))
    print("adam opr loss:", hist[0], hist[-1])
    assert hist[-1] < 0.5 * hist[0]


OPR_SHAPES = [  # N, K, M, H, W, J, step, batch
    (32, 3, 2, 72, 76, 16, 6.0, 6), (64, 8, 1, 150, 160, 14, 12.0, 5), (16, 2, 3, 41, 37, 9, 3.0, 9),
    (128, 4, 1, 290, 300, 9, 30.0, 4), (192, 2, 2, 230, 236, 4, 12.0, 3), (256, 8, 1, 290, 296, 3, 12.0, 2)]


@pytest.mark.parametrize("graph", [False, True])
def test_opr_batched_matches_oracle_per_reconstruction(graph):
    import torch
    from paper_2510_20929_gb300 import api
    recons, refs, opts, oprs = [], [], [], []
    for i, (N, K, M, H, W, J, step, B) in enumerate(OPR_SHAPES):
        h = _host(opr_problem(N=N, K=K, M=M, H=H, W=W, J=J, step=step, seed=60 + i))
        O, U, w, Pr, pos, I_m = h
        order = np.random.default_rng(i).permutation(J).astype(np.int32)
        refs.append(orc.lsqml_epoch_opr(O, U, w, Pr, pos, I_m, order,
                                        orc.LsqmlOptions(batch=B, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6),
                                        orc.OprOptions(update_weights=True, weight_step=0.8)))
        recons.append(list(_dev(h)) + [to_dev(order, torch.int32)])
        opts.append(api.make_opts(batch=B, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6, graph=graph))
        oprs.append(api.make_opr_opts(K, weight_step=0.8))
    losses = api.lsqml_epoch_opr_batched(recons, opts, oprs).cpu().numpy()
    for i, ((dO, dU, dw, dPr, _, _, _), (O1, U1, w1, Pr1, L1, _)) in enumerate(zip(recons, refs)):
        e = [err(dO.cpu().numpy(), O1), err(dU.cpu().numpy(), U1, axis=0), err(dw.cpu().numpy(), w1, axis=1),
             abs(losses[i] - L1) / abs(L1)]
        if Pr1 is not None:
            e.append(err(dPr.cpu().numpy(), Pr1, axis=0))
        print(f"opr batched[{i}] N={OPR_SHAPES[i][0]}:", " ".join(f"{x:.2e}" for x in e))
        assert max(e) < TOL_EPOCH
