"""Cluster windows (256 x 256 on four CTAs, 192 x 192 on three) against the FP64
oracle: forward intensities, gradients and LSQML epochs, including a ragged
last batch."""
import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from tests.parity_util import TOL_EPOCH, TOL_FWD, TOL_GRAD, c64, err, f32pos, problem, to_dev

pytestmark = pytest.mark.gpu


def _dev(p):
    import torch
    O, P, pos, I_m = c64(p["O"]), c64(p["P"]), f32pos(p["pos"]), np.float32(p["I_m"]).astype(np.float64)
    return (O, P, pos, I_m), (to_dev(O, torch.complex64), to_dev(P, torch.complex64),
                              to_dev(pos, torch.float32), to_dev(I_m, torch.float32))


@pytest.mark.parametrize("N,M", [(256, 1), (256, 3), (192, 1), (192, 3)])
def test_forward_cluster(N, M):
    from paper_2510_20929_gb300 import api
    p = problem(N=N, M=M, H=N + 74, W=N + 84, J=6, step=20.0)
    (O, P, pos, _), (dO, dP, dpos, _) = _dev(p)
    I = api.forward(dO, dP, dpos).cpu().numpy()
    ref = orc.forward(O, P, pos)
    e = err(I, ref)
    print(f"forward N={N} M={M}: {e:.3e}")
    assert e < 1e-5


@pytest.mark.parametrize("N", [256, 192])
@pytest.mark.parametrize("noise", ["gaussian", "poisson"])
def test_gradients_cluster(noise, N):
    from paper_2510_20929_gb300 import api
    p = problem(N=N, M=2, H=N + 64, W=N + 74, J=5, step=20.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    nz = orc.GAUSSIAN if noise == "gaussian" else orc.POISSON
    L, gO, gP, gr = orc.loss_and_gradients(O, P, pos, I_m, nz, 1e-6)
    loss, dgO, dgP, dgr = api.adjoint(dO, dP, dpos, dI, noise, eps=1e-6, batch=3)
    e = (abs(loss.item() - L) / abs(L), err(dgO.cpu().numpy(), gO), err(dgP.cpu().numpy(), gP, axis=0),
         err(dgr.cpu().numpy(), gr, axis=1))
    print(f"grad N={N} {noise}: {e}")
    assert e[0] < TOL_FWD and max(e[1:]) < TOL_GRAD


@pytest.mark.parametrize("N", [256, 192])
def test_lsqml_epoch_cluster(N):
    import torch
    from paper_2510_20929_gb300 import api
    p = problem(N=N, M=2, H=N + 64, W=N + 74, J=7, step=18.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    order = np.random.default_rng(1).permutation(7).astype(np.int32)
    opts = orc.LsqmlOptions(batch=3, delta_o=0.1, delta_p=0.1, eps=1e-6)
    O_ref, P_ref, L_ref, a_ref = orc.lsqml_epoch(O, P, pos, I_m, order, opts)
    loss, alpha = api.lsqml_epoch(dO, dP, dpos, dI, to_dev(order, torch.int32), batch=3, delta_o=0.1,
                                  delta_p=0.1, eps=1e-6, want_alpha=True)
    e = (err(dO.cpu().numpy(), O_ref), err(dP.cpu().numpy(), P_ref, axis=0), err(alpha.cpu().numpy(), a_ref, axis=1),
         abs(loss.item() - L_ref) / abs(L_ref))
    print(f"epoch N={N}: {e}")
    assert max(e) < TOL_EPOCH
