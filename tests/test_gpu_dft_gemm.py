"""GPU parity of the split-BF16 DFT-GEMM precision (the far field on the
tcgen05 tensor cores) through the C ABI against the FP64 oracle, on the same
seeded inputs as the FP32 parity tests.

Tolerance: each operand is carried as hi + lo BF16 parts, so an element is
represented to within 2^-16 of its magnitude (about 2^-17 typically) and the
dropped lo*lo product is of the same order; with FP32 accumulation over the N terms of each of the two
passes the transform's norm-wise error stays near 1e-5. TOL_BF16 = 1e-3 is
the bound the path is specified to (split BF16 on exit waves and gradients);
the measured errors are printed."""
import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from tests.parity_util import c64, f32pos, problem, err, rel, to_dev

pytestmark = pytest.mark.gpu

TOL_BF16 = 1e-3


def _dev(p):
    import torch
    O, P, pos, I_m = c64(p["O"]), c64(p["P"]), f32pos(p["pos"]), np.float32(p["I_m"]).astype(np.float64)
    return (O, P, pos, I_m), (to_dev(O, torch.complex64), to_dev(P, torch.complex64),
                              to_dev(pos, torch.float32), to_dev(I_m, torch.float32))


CASES = [  # N, M, H, W, J, step
    (32, 2, 72, 76, 16, 6.0),
    (64, 1, 160, 150, 25, 12.0),
    (64, 3, 150, 160, 20, 12.0),
    (128, 2, 300, 310, 12, 24.0),
    (128, 5, 290, 300, 9, 30.0),
]


@pytest.mark.parametrize("N,M,H,W,J,step", CASES)
def test_forward_bf16x3_matches_oracle(N, M, H, W, J, step):
    from paper_2510_20929_gb300 import api
    p = problem(N=N, M=M, H=H, W=W, J=J, step=step)
    (O, P, pos, _), (dO, dP, dpos, _) = _dev(p)
    ref = orc.forward(O, P, pos)
    I = api.forward(dO, dP, dpos, precision="bf16x3", batch=5).cpu().numpy()   # ragged chunks of 5
    I32 = api.forward(dO, dP, dpos).cpu().numpy()
    e, e32 = err(I, ref), err(I32, ref)
    print(f"forward bf16x3 N={N} M={M}: rel {e:.3e} (fp32 path {e32:.3e})")
    assert e < TOL_BF16
    for j in range(J):
        assert rel(I[j], ref[j]) < TOL_BF16


@pytest.mark.parametrize("W", [151, 152])
def test_bf16x3_exit_waves_on_odd_and_even_object_widths(W):
    # even widths stage the object tile with one tensor copy; odd widths (a row
    # pitch that is not a multiple of 16 bytes) take the per-pixel gather
    from paper_2510_20929_gb300 import api
    p = problem(N=64, M=2, H=160, W=W, J=20, step=12.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    e_fwd = err(api.forward(dO, dP, dpos, precision="bf16x3", batch=7).cpu().numpy(), orc.forward(O, P, pos))
    L, gO, gP, gr = orc.loss_and_gradients(O, P, pos, I_m, orc.GAUSSIAN, 1e-6)
    loss, dgO, dgP, dgr = api.adjoint(dO, dP, dpos, dI, "gaussian", eps=1e-6, batch=7, precision="bf16x3")
    e = (e_fwd, abs(loss.item() - L) / L, err(dgO.cpu().numpy(), gO), err(dgP.cpu().numpy(), gP, axis=0),
         err(dgr.cpu().numpy(), gr, axis=1))
    print(f"bf16x3 W={W}:", " ".join(f"{x:.2e}" for x in e))
    assert max(e) < TOL_BF16


@pytest.mark.parametrize("noise", ["gaussian", "poisson"])
@pytest.mark.parametrize("N,M,H,W,J,step", [CASES[0], CASES[2], CASES[4]])
def test_gradients_bf16x3_match_oracle(noise, N, M, H, W, J, step):
    from paper_2510_20929_gb300 import api
    p = problem(N=N, M=M, H=H, W=W, J=J, step=step)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    eps = 1e-6
    nz = orc.GAUSSIAN if noise == "gaussian" else orc.POISSON
    L_ref, gO_ref, gP_ref, gr_ref = orc.loss_and_gradients(O, P, pos, I_m, nz, eps)
    loss, gO, gP, gr = api.adjoint(dO, dP, dpos, dI, noise, eps=eps, batch=4, precision="bf16x3")
    e = (abs(loss.item() - L_ref) / abs(L_ref), err(gO.cpu().numpy(), gO_ref),
         err(gP.cpu().numpy(), gP_ref, axis=0), err(gr.cpu().numpy(), gr_ref, axis=1))
    print(f"grad bf16x3 {noise} N={N} M={M}: loss {e[0]:.2e} gO {e[1]:.2e} gP {e[2]:.2e} gr {e[3]:.2e}")
    assert max(e) < TOL_BF16


def test_vjp_bf16x3_matches_oracle():
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=32, M=3, H=72, W=76, J=16, step=6.0)
    (O, P, pos, _), (dO, dP, dpos, _) = _dev(p)
    G = np.float32(np.random.default_rng(4).standard_normal((16, 32, 32))).astype(np.float64)
    gO_ref, gP_ref, gr_ref = orc.vjp(O, P, pos, G)
    loss, gO, gP, gr = api.adjoint(dO, dP, dpos, to_dev(G, torch.float32), "vjp", batch=7, precision="bf16x3")
    assert loss is None
    e = (err(gO.cpu().numpy(), gO_ref), err(gP.cpu().numpy(), gP_ref, axis=0), err(gr.cpu().numpy(), gr_ref, axis=1))
    print(f"vjp bf16x3: {e}")
    assert max(e) < TOL_BF16


@pytest.mark.parametrize("N,M,H,W,J,step,batch", [
    (32, 3, 72, 76, 16, 6.0, 6),          # ragged last batch (6, 6, 4)
    (64, 1, 160, 150, 25, 12.0, 8),
    (128, 5, 290, 300, 9, 30.0, 4),
])
@pytest.mark.parametrize("noise", ["gaussian", "poisson"])
def test_lsqml_epoch_bf16x3_matches_oracle(N, M, H, W, J, step, batch, noise):
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=N, M=M, H=H, W=W, J=J, step=step)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    order = np.random.default_rng(7).permutation(J).astype(np.int32)
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN if noise == "gaussian" else orc.POISSON, batch=batch,
                            delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    O_ref, P_ref, L_ref, a_ref = orc.lsqml_epoch(O, P, pos, I_m, order, opts)
    loss, alpha = api.lsqml_epoch(dO, dP, dpos, dI, to_dev(order, torch.int32), noise=noise, batch=batch,
                                  delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6, want_alpha=True,
                                  precision="bf16x3")
    e = dict(O=err(dO.cpu().numpy(), O_ref), P=err(dP.cpu().numpy(), P_ref, axis=0),
             alpha=err(alpha.cpu().numpy(), a_ref, axis=1), loss=abs(loss.item() - L_ref) / abs(L_ref))
    print(f"epoch bf16x3 N={N} M={M} B={batch} {noise}: " + " ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert max(e.values()) < TOL_BF16


def test_bf16x3_skips_and_reports_out_of_bounds_positions():
    # two positions moved off the object: flagged, skipped (their blocks left
    # untouched), the rest equal the oracle's
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=64, M=2, H=150, W=160, J=10, step=12.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    bad = pos.copy()
    bad[3] = (-50.0, 20.0)
    bad[7] = (40.0, 1e4)
    keep = [j for j in range(10) if j not in (3, 7)]
    dbad = to_dev(bad, torch.float32)
    d = api.dims_of(dO, dP, dbad)
    I = torch.full((10, 64, 64), -7.0, dtype=torch.float32, device=dO.device)
    ws = api.workspace(d, 4, dO.device)
    assert api.lib().ptycho_forward_ex(api.ctypes.byref(d), 1, 4, api._ptr(dO), api._ptr(dP), api._ptr(dbad),
                                       api._ptr(I), api._P(ws.ptr), ws.nbytes, api._stream()) == 0
    assert ws.status() == 2
    I = I.cpu().numpy()
    assert np.all(I[[3, 7]] == -7.0)
    assert err(I[keep], orc.forward(O, P, pos[keep])) < TOL_BF16
    loss, gO, gP, gr = api.adjoint(dO, dP, dbad, dI, "gaussian", eps=1e-6, batch=4, precision="bf16x3",
                                   check=False)
    assert api.workspace(d, 4, dO.device).status() == 2
    L, gO_ref, gP_ref, gr_ref = orc.loss_and_gradients(O, P, pos[keep], I_m[keep], orc.GAUSSIAN, 1e-6)
    assert abs(loss.item() - L) / L < TOL_BF16
    assert err(gO.cpu().numpy(), gO_ref) < TOL_BF16 and err(gP.cpu().numpy(), gP_ref, axis=0) < TOL_BF16
    assert err(gr.cpu().numpy()[keep], gr_ref, axis=1) < TOL_BF16 and np.all(gr.cpu().numpy()[[3, 7]] == 0)


def test_bf16x3_graph_replay_and_host_epoch_match_the_device_epoch():
    # the captured-graph replay and the host-buffer entry run the same launches
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=128, M=2, H=300, W=310, J=12, step=24.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    order = np.random.default_rng(9).permutation(12).astype(np.int32)
    dorder = to_dev(order, torch.int32)
    res = []
    for graph in (False, True):
        o, pr = dO.clone(), dP.clone()
        for _ in range(2):
            api.lsqml_epoch(o, pr, dpos, dI, dorder, batch=5, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6,
                            graph=graph, precision="bf16x3")
        res.append((o.cpu().numpy(), pr.cpu().numpy()))
    # (the overlap-add atomics may sum in another order: equal to rounding)
    assert err(res[1][0], res[0][0]) < 1e-5 and err(res[1][1], res[0][1], axis=0) < 1e-5
    hO, hP = O.astype(np.complex64), P.astype(np.complex64)
    opts = api.make_opts(batch=5, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6, precision="bf16x3")
    hO_t, hP_t = torch.from_numpy(hO.copy()), torch.from_numpy(hP.copy())
    for _ in range(2):
        api.lsqml_epoch_host(hO_t, hP_t, torch.from_numpy(np.float32(pos)), torch.from_numpy(np.float32(I_m)),
                             torch.from_numpy(order), opts, device=dO.device)
    assert err(hO_t.numpy(), res[0][0]) < 1e-5 and err(hP_t.numpy(), res[0][1], axis=0) < 1e-5


def test_bf16x3_batched_reconstructions_equal_their_single_epochs():
    # two reconstructions of different window and mode count in one batched call
    import torch
    from paper_2510_20929_gb300 import api
    recs = []
    for (N, M, H, W, J, step) in ((64, 3, 150, 160, 20, 12.0), (128, 2, 300, 310, 12, 24.0)):
        p = problem(N=N, M=M, H=H, W=W, J=J, step=step)
        (_, _, _, _), (dO, dP, dpos, dI) = _dev(p)
        recs.append((dO, dP, dpos, dI, to_dev(np.random.default_rng(N).permutation(J).astype(np.int32),
                                                torch.int32)))
    single = []
    for dO, dP, dpos, dI, order in recs:
        o, pr = dO.clone(), dP.clone()
        L, _ = api.lsqml_epoch(o, pr, dpos, dI, order, batch=5, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6,
                               precision="bf16x3")
        single.append((o.cpu().numpy(), pr.cpu().numpy(), L.item()))
    batch = [[dO.clone(), dP.clone(), dpos, dI, order] for dO, dP, dpos, dI, order in recs]
    opts = [api.make_opts(batch=5, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6, precision="bf16x3")] * 2
    losses = api.lsqml_epoch_batched(batch, opts).cpu().numpy()
    for (o, pr, *_), (O1, P1, L1), L in zip(batch, single, losses):
        assert err(o.cpu().numpy(), O1) < 1e-5 and err(pr.cpu().numpy(), P1, axis=0) < 1e-5
        assert abs(L - L1) <= 1e-5 * abs(L1)


def test_bf16x3_empty_inputs_leave_everything_untouched():
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=32, M=2, H=72, W=76, J=4, step=6.0)
    _, (dO, dP, dpos, dI) = _dev(p)
    pos0 = dpos[:0].contiguous()
    assert api.forward(dO, dP, pos0, precision="bf16x3").shape == (0, 32, 32)
    loss, gO, gP, gr = api.adjoint(dO, dP, pos0, dI[:0].contiguous(), "gaussian", precision="bf16x3")
    assert loss.item() == 0.0 and gO.abs().max().item() == 0.0 and gP.abs().max().item() == 0.0
    O0, P0 = dO.clone(), dP.clone()
    loss, _ = api.lsqml_epoch(dO, dP, pos0, dI[:0].contiguous(), None, batch=4, precision="bf16x3")
    assert loss.item() == 0.0 and torch.equal(dO, O0) and torch.equal(dP, P0)


@pytest.mark.parametrize("batch", [1, 100])
def test_bf16x3_one_position_and_whole_set_minibatches(batch):
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=32, M=2, H=72, W=76, J=9, step=6.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    order = np.random.default_rng(5).permutation(9).astype(np.int32)
    kw = dict(batch=batch, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    O1, P1, L1, a1 = orc.lsqml_epoch(O, P, pos, I_m, order, orc.LsqmlOptions(**kw))
    loss, alpha = api.lsqml_epoch(dO, dP, dpos, dI, to_dev(order, torch.int32), want_alpha=True,
                                  precision="bf16x3", **kw)
    e = (err(dO.cpu().numpy(), O1), err(dP.cpu().numpy(), P1, axis=0), err(alpha.cpu().numpy(), a1, axis=1))
    print(f"bf16x3 batch {batch}:", e)
    assert max(e) < TOL_BF16


def test_bf16x3_sixteen_modes():
    # the largest mode count: intensities summed over 16 modes, gradients of every mode
    from paper_2510_20929_gb300 import api
    p = problem(N=32, M=16, H=72, W=76, J=8, step=6.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    e_fwd = err(api.forward(dO, dP, dpos, precision="bf16x3").cpu().numpy(), orc.forward(O, P, pos))
    L, gO, gP, gr = orc.loss_and_gradients(O, P, pos, I_m, orc.POISSON, 1e-6)
    loss, dgO, dgP, dgr = api.adjoint(dO, dP, dpos, dI, "poisson", eps=1e-6, batch=3, precision="bf16x3")
    e = (e_fwd, abs(loss.item() - L) / abs(L), err(dgO.cpu().numpy(), gO), err(dgP.cpu().numpy(), gP, axis=0),
         err(dgr.cpu().numpy(), gr, axis=1))
    print("bf16x3 16 modes:", " ".join(f"{x:.2e}" for x in e))
    assert max(e) < TOL_BF16


def test_bounded_wait_reports_timeout_and_the_context_stays_usable():
    # a wait that can never complete gives up, the status reads TIMEOUT, and work runs on
    from paper_2510_20929_gb300 import api
    p = problem(N=32, M=2, H=72, W=76, J=6, step=6.0)
    (O, P, pos, _), (dO, dP, dpos, _) = _dev(p)
    d = api.dims_of(dO, dP, dpos)
    ws = api.workspace(d, 4, dO.device)
    ws.status()                                   # clear
    assert api.lib().ptycho_selftest_wait_timeout(api._P(ws.ptr), ws.nbytes, api._stream()) == 0
    assert ws.status() == 5                       # PTYCHO_ERR_TIMEOUT
    assert ws.status() == 0                       # read clears it
    I = api.forward(dO, dP, dpos, precision="bf16x3", batch=4).cpu().numpy()
    assert err(I, orc.forward(O, P, pos)) < TOL_BF16
