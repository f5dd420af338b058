"""Edge cases of the GPU path: positions outside the object and bad order
entries (skipped and reported), non-finite counts (reported), empty inputs,
one-position and whole-set minibatches, positions on the bounds limits,
integer positions, and the maximum mode and slice counts."""
import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from tests.parity_util import TOL_EPOCH, TOL_FWD, TOL_GRAD, c64, err, f32pos, problem, to_dev

pytestmark = pytest.mark.gpu


def _inputs(p):
    import torch
    O, P, pos, I_m = c64(p["O"]), c64(p["P"]), f32pos(p["pos"]), np.float32(p["I_m"]).astype(np.float64)
    return (O, P, pos, I_m), (to_dev(O, torch.complex64), to_dev(P, torch.complex64), to_dev(pos, torch.float32),
                              to_dev(I_m, torch.float32))


def _status(d, batch, device):
    from paper_2510_20929_gb300 import api
    return api.workspace(d, batch, device).status()


def test_position_outside_the_object_is_skipped_and_reported():
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=32, M=2, H=72, W=76, J=12, step=6.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _inputs(p)
    bad = 5
    pos_bad = pos.copy()
    pos_bad[bad] = [3.0, 40.0]                       # tile would start at y = -13
    dpos_bad = to_dev(pos_bad, torch.float32)
    keep = [j for j in range(12) if j != bad]
    # forward: the bad position's block is left untouched, the others are right
    d = api.dims_of(dO, dP, dpos_bad)
    I = torch.full((12, 32, 32), -7.0, dtype=torch.float32, device=dO.device)
    ws = api.workspace(d, 1, dO.device)
    assert api.lib().ptycho_forward(api.ctypes.byref(d), api._ptr(dO), api._ptr(dP), api._ptr(dpos_bad),
                                    api._ptr(I), api._P(ws.ptr), ws.nbytes, api._stream()) == 0
    assert ws.status() == 2
    I = I.cpu().numpy()
    assert np.all(I[bad] == -7.0)
    assert err(I[keep], orc.forward(O, P, pos[keep])) < TOL_FWD
    # gradients: the sum over the valid positions only
    loss, gO, gP, gr = api.adjoint(dO, dP, dpos_bad, dI, "gaussian", eps=1e-6, batch=5, check=False)
    assert _status(d, 5, dO.device) == 2
    L, gO_ref, gP_ref, gr_ref = orc.loss_and_gradients(O, P, pos[keep], I_m[keep], orc.GAUSSIAN, 1e-6)
    assert abs(loss.item() - L) / L < TOL_GRAD
    assert err(gO.cpu().numpy(), gO_ref) < TOL_GRAD and err(gP.cpu().numpy(), gP_ref, axis=0) < TOL_GRAD
    assert err(gr.cpu().numpy()[keep], gr_ref, axis=1) < TOL_GRAD and np.all(gr.cpu().numpy()[bad] == 0)
    # epoch: the bad position's slot does nothing; its minibatch is one shorter
    order = np.random.default_rng(3).permutation(12).astype(np.int32)
    with pytest.raises(api.PtychoError) as ei:
        api.lsqml_epoch(dO, dP, dpos_bad, dI, to_dev(order, torch.int32), batch=5, delta_o=0.1, delta_p=0.1,
                        lam=1e-6, eps=1e-6)
    assert ei.value.status == 2
    # the oracle rejects out-of-bounds positions: run its minibatches without the bad one
    ref_O, ref_P = O.copy(), P.copy()
    opts = orc.LsqmlOptions(batch=5, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    for b0 in range(0, 12, 5):
        idx = [j for j in order[b0:b0 + 5] if j != bad]
        ref_O, ref_P, _, _ = orc.lsqml_batch(ref_O, ref_P, pos, I_m, idx, opts)
    assert err(dO.cpu().numpy(), ref_O) < TOL_EPOCH and err(dP.cpu().numpy(), ref_P, axis=0) < TOL_EPOCH


def test_bad_order_entries_are_skipped_and_reported():
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=16, M=1, H=40, W=44, J=9, step=4.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _inputs(p)
    order = np.array([3, 99, 0, 7, -1, 2, 8, 1, 5], np.int32)   # two entries outside [0, J)
    with pytest.raises(api.PtychoError) as ei:
        api.lsqml_epoch(dO, dP, dpos, dI, to_dev(order, torch.int32), batch=4, delta_o=0.1, delta_p=0.1, eps=1e-6)
    assert ei.value.status == 2
    opts = orc.LsqmlOptions(batch=4, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    ref_O, ref_P = O.copy(), P.copy()
    for b0 in range(0, 9, 4):
        idx = [j for j in order[b0:b0 + 4] if 0 <= j < 9]
        ref_O, ref_P, _, _ = orc.lsqml_batch(ref_O, ref_P, pos, I_m, idx, opts)
    assert err(dO.cpu().numpy(), ref_O) < TOL_EPOCH and err(dP.cpu().numpy(), ref_P, axis=0) < TOL_EPOCH


@pytest.mark.parametrize("value", [float("nan"), float("inf"), -1.0])
def test_non_finite_or_negative_counts_are_reported(value):
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=16, M=1, H=40, W=44, J=6, step=4.0)
    _, (dO, dP, dpos, dI) = _inputs(p)
    dI[2, 3, 4] = value
    with pytest.raises(api.PtychoError) as ei:
        api.adjoint(dO, dP, dpos, dI, "poisson", eps=1e-6)
    assert ei.value.status == 3
    with pytest.raises(api.PtychoError) as ei:
        api.lsqml_epoch(dO, dP, dpos, dI, None, batch=3, eps=1e-6)
    assert ei.value.status == 3


def test_empty_inputs_leave_everything_untouched():
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=16, M=2, H=40, W=44, J=4, step=4.0)
    _, (dO, dP, dpos, dI) = _inputs(p)
    pos0 = dpos[:0].contiguous()
    I = api.forward(dO, dP, pos0)
    assert I.shape == (0, 16, 16)
    loss, gO, gP, gr = api.adjoint(dO, dP, pos0, dI[:0].contiguous(), "gaussian")
    assert loss.item() == 0.0 and gO.abs().max().item() == 0.0 and gP.abs().max().item() == 0.0
    O0, P0 = dO.clone(), dP.clone()
    loss, _ = api.lsqml_epoch(dO, dP, pos0, dI[:0].contiguous(), None, batch=4)
    assert loss.item() == 0.0 and torch.equal(dO, O0) and torch.equal(dP, P0)


@pytest.mark.parametrize("batch", [1, 100])
def test_one_position_and_whole_set_minibatches(batch):
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=32, M=2, H=72, W=76, J=9, step=6.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _inputs(p)
    order = np.random.default_rng(5).permutation(9).astype(np.int32)
    kw = dict(batch=batch, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    O1, P1, L1, a1 = orc.lsqml_epoch(O, P, pos, I_m, order, orc.LsqmlOptions(**kw))
    loss, alpha = api.lsqml_epoch(dO, dP, dpos, dI, to_dev(order, torch.int32), want_alpha=True, **kw)
    e = (err(dO.cpu().numpy(), O1), err(dP.cpu().numpy(), P1, axis=0), err(alpha.cpu().numpy(), a1, axis=1))
    print(f"batch {batch}:", e)
    assert max(e) < TOL_EPOCH


def test_positions_on_the_bounds_limits_and_integer_positions():
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=16, M=2, H=40, W=44, J=5, step=4.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _inputs(p)
    # r - N/2 = 0 (first tile row/column), the largest float32 below H - N, and integers
    lim = np.array([[8.0, 8.0], [np.float32(40 - 16 + 8) - np.float32(2 ** -18), np.float32(44 - 16 + 8) -
                                 np.float32(2 ** -18)], [20.0, 21.0], [8.0, 35.99], [31.5, 8.0]])
    lim = f32pos(lim)
    assert all(orc.in_bounds(r, 16, 40, 44) for r in lim)
    dlim = to_dev(lim, torch.float32)
    I = api.forward(dO, dP, dlim).cpu().numpy()
    assert err(I, orc.forward(O, P, lim)) < TOL_FWD
    L, gO_ref, gP_ref, gr_ref = orc.loss_and_gradients(O, P, lim, I_m, orc.GAUSSIAN, 1e-6)
    loss, gO, gP, gr = api.adjoint(dO, dP, dlim, dI, "gaussian", eps=1e-6)
    assert err(gO.cpu().numpy(), gO_ref) < TOL_GRAD and err(gr.cpu().numpy(), gr_ref, axis=1) < TOL_GRAD
    # one step past the limit is rejected
    over = lim.copy()
    over[1, 0] = 40 - 16 + 8
    with pytest.raises(api.PtychoError) as ei:
        api.forward(dO, dP, to_dev(over, torch.float32))
    assert ei.value.status == 2


def test_maximum_mode_and_slice_counts():
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=16, M=16, H=40, W=44, J=6, step=4.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _inputs(p)
    assert err(api.forward(dO, dP, dpos).cpu().numpy(), orc.forward(O, P, pos)) < TOL_FWD
    L, gO_ref, gP_ref, _ = orc.loss_and_gradients(O, P, pos, I_m, orc.GAUSSIAN, 1e-6)
    loss, gO, gP, _ = api.adjoint(dO, dP, dpos, dI, "gaussian", eps=1e-6)
    assert err(gO.cpu().numpy(), gO_ref) < TOL_GRAD and err(gP.cpu().numpy(), gP_ref, axis=0) < TOL_GRAD
    # 16 slices
    Os = np.stack([O ** (1.0 / 16)] * 16)
    Hf = orc.asm_propagator(16, 10e-9, 0.1e-9, 5e-6)
    ms = api.make_multislice(16, 5e-6, 0.1e-9, 10e-9)
    I = api.forward_ms(to_dev(c64(Os), torch.complex64), dP[:2].contiguous(), dpos, ms).cpu().numpy()
    assert err(I, orc.forward_ms(c64(Os), P[:2], pos, Hf)) < 10 * TOL_FWD
