"""The autograd front end: gradients of the FarField and DataTerm Functions
against the FP64 oracle's adjoint, a finite-difference check on the GPU, and the
Adam reconstructor on object, probe and positions with perturbed positions."""
import math

import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2510_20929_gb300 import synth
from tests.parity_util import TOL_FWD, TOL_GRAD, c64, err, f32pos, problem, to_dev

pytestmark = pytest.mark.gpu


def _dev(p):
    import torch
    O, P, pos, I_m = c64(p["O"]), c64(p["P"]), f32pos(p["pos"]), np.float32(p["I_m"]).astype(np.float64)
    return (O, P, pos, I_m), (to_dev(O, torch.complex64), to_dev(P, torch.complex64), to_dev(pos, torch.float32),
                              to_dev(I_m, torch.float32))


def test_far_field_gradients_match_oracle_vjp():
    import torch
    from paper_2510_20929_gb300.autograd import far_field
    p = problem(N=32, M=3, H=72, W=76, J=16, step=6.0)
    (O, P, pos, _), (dO, dP, dpos, _) = _dev(p)
    wts = np.float32(np.random.default_rng(3).standard_normal((16, 32, 32))).astype(np.float64)
    for t in (dO, dP, dpos):
        t.requires_grad_(True)
    I = far_field(dO, dP, dpos)
    (I * to_dev(wts, torch.float32)).sum().backward()
    gO, gP, gr = orc.vjp(O, P, pos, wts)
    e = (err(dO.grad.cpu().numpy(), gO), err(dP.grad.cpu().numpy(), gP, axis=0), err(dpos.grad.cpu().numpy(), gr, axis=1))
    print("far_field grads:", e)
    assert max(e) < TOL_GRAD


def test_data_term_gradients_match_oracle():
    from paper_2510_20929_gb300.autograd import data_term
    p = problem(N=64, M=2, H=150, W=160, J=20, step=12.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    for t in (dO, dP, dpos):
        t.requires_grad_(True)
    loss = data_term(dO, dP, dpos, dI, "gaussian", 1e-6)
    (2.5 * loss).backward()
    L, gO, gP, gr = orc.loss_and_gradients(O, P, pos, I_m, orc.GAUSSIAN, 1e-6)
    e = (abs(loss.item() - L) / L, err(dO.grad.cpu().numpy(), 2.5 * gO), err(dP.grad.cpu().numpy(), 2.5 * gP, axis=0),
         err(dpos.grad.cpu().numpy(), 2.5 * gr, axis=1))
    print("data_term:", e)
    assert e[0] < TOL_FWD and max(e[1:]) < TOL_GRAD


@pytest.mark.parametrize("noise", ["gaussian", "poisson"])
@pytest.mark.parametrize("N,M,H,W,J,step", [(64, 2, 150, 160, 20, 12.0), (256, 1, 300, 310, 6, 12.0)])
def test_loss_only_evaluation_matches_oracle(noise, N, M, H, W, J, step):
    # without gradient buffers the adjoint evaluates the loss alone; the data
    # term takes that path when nothing needs a gradient (no_grad)
    import torch
    from paper_2510_20929_gb300 import api
    from paper_2510_20929_gb300.autograd import data_term
    p = problem(N=N, M=M, H=H, W=W, J=J, step=step)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    nz = orc.GAUSSIAN if noise == "gaussian" else orc.POISSON
    L = sum(orc.pattern_loss(I, Im, nz, 1e-6) for I, Im in zip(orc.forward(O, P, pos), I_m))
    loss, gO, gP, gr = api.adjoint(dO, dP, dpos, dI, noise, eps=1e-6, batch=7, gradients=False)
    assert gO is None and gP is None and gr is None
    full, _, _, _ = api.adjoint(dO, dP, dpos, dI, noise, eps=1e-6, batch=7)
    with torch.no_grad():
        dt = data_term(dO.requires_grad_(True), dP, dpos, dI, noise, 1e-6)
    e = (abs(loss.item() - L) / abs(L), abs(dt.item() - L) / abs(L))
    print(f"loss only {noise} N={N}: {e[0]:.2e} {e[1]:.2e}")
    assert max(e) < 1e-5 and abs(loss.item() - full.item()) <= 1e-6 * abs(full.item())


@pytest.mark.parametrize("which", ["far_field", "data_term"])
def test_split_bf16_autograd_matches_oracle(which):
    # the same Functions with the far field as split-BF16 DFT-GEMMs (tolerance 1e-3)
    import torch
    from paper_2510_20929_gb300.autograd import data_term, far_field
    p = problem(N=64, M=2, H=150, W=160, J=20, step=12.0)
    (O, P, pos, I_m), (dO, dP, dpos, dI) = _dev(p)
    for t in (dO, dP, dpos):
        t.requires_grad_(True)
    if which == "far_field":
        wts = np.float32(np.random.default_rng(3).standard_normal((20, 64, 64))).astype(np.float64)
        (far_field(dO, dP, dpos, precision="bf16x3") * to_dev(wts, torch.float32)).sum().backward()
        gO, gP, gr = orc.vjp(O, P, pos, wts)
        e = (0.0,)
    else:
        loss = data_term(dO, dP, dpos, dI, "gaussian", 1e-6, precision="bf16x3")
        loss.backward()
        L, gO, gP, gr = orc.loss_and_gradients(O, P, pos, I_m, orc.GAUSSIAN, 1e-6)
        e = (abs(loss.item() - L) / L,)
    e += (err(dO.grad.cpu().numpy(), gO), err(dP.grad.cpu().numpy(), gP, axis=0), err(dpos.grad.cpu().numpy(), gr, axis=1))
    print(f"{which} split BF16:", e)
    assert max(e) < 1e-3


def test_data_term_matches_finite_differences_on_gpu():
    import torch
    from paper_2510_20929_gb300.autograd import data_term
    p = problem(N=32, M=2, H=72, W=76, J=16, step=6.0, perturb=0.3)
    _, (dO, dP, dpos, dI) = _dev(p)
    g = torch.Generator(device=dO.device).manual_seed(0)
    for t in (dO, dP, dpos):
        t.requires_grad_(True)
    loss = data_term(dO, dP, dpos, dI, "poisson", 1.0)
    loss.backward()
    with torch.no_grad():
        for x, rel_h in ((dO, 1e-3), (dP, 1e-3), (dpos, 1e-3)):
            d = torch.randn(x.shape, generator=g, device=x.device, dtype=torch.float32)
            if x.is_complex():
                d = torch.complex(d, torch.randn(x.shape, generator=g, device=x.device, dtype=torch.float32))
            h = rel_h * (x.abs().max() / d.abs().max()).item() if x is not dpos else 1e-2
            x0 = x.detach().clone()
            Lp = data_term(x0 + h * d if x is dO else dO.detach(), x0 + h * d if x is dP else dP.detach(),
                           x0 + h * d if x is dpos else dpos.detach(), dI, "poisson", 1.0).item()
            Lm = data_term(x0 - h * d if x is dO else dO.detach(), x0 - h * d if x is dP else dP.detach(),
                           x0 - h * d if x is dpos else dpos.detach(), dI, "poisson", 1.0).item()
            fd = (Lp - Lm) / (2 * h)
            an = torch.real(torch.vdot(x.grad.flatten(), d.flatten())).item() if x.is_complex() else \
                (x.grad * d).sum().item()
            print("fd", fd, "autograd", an)
            assert abs(fd - an) < 2e-2 * abs(an)


def test_adam_reconstructor_corrects_perturbed_positions():
    import torch
    from paper_2510_20929_gb300 import api
    from paper_2510_20929_gb300.autograd import data_term, reconstruct_adam
    w = synth.workload_small(N=64, M=2, H=200, W=200, J=36, seed=31, step=14.0)
    # a smooth object (4 px correlation) so that 1.5 px position errors sit inside the basin
    obj = synth.make_object(200, 200, 31, phase_sigma=4.0, amp_sigma=4.0, phase_max=1.0, amp_lo=0.5)
    O_true = to_dev(c64(obj), torch.complex64)
    P = to_dev(c64(w["probe"] * 30.0), torch.complex64)
    pos_true = to_dev(f32pos(w["pos"]), torch.float32)
    I_m = api.forward(O_true, P, pos_true)
    err = torch.randn(pos_true.shape, generator=torch.Generator().manual_seed(2)).to(pos_true.device) * 1.5
    pos = (pos_true + err).contiguous()
    O = O_true.clone()
    rmse0 = (pos - pos_true).pow(2).mean().sqrt().item()
    hist = reconstruct_adam(O, P.clone(), pos, I_m, epochs=100, lr_pos=0.1, update=("positions",))
    hist += reconstruct_adam(O, P.clone(), pos, I_m, epochs=60, lr_pos=0.02, update=("positions",))
    rmse = (pos - pos_true).pow(2).mean().sqrt().item()
    print("position rmse", rmse0, "->", rmse, "loss", hist[0], "->", hist[-1])
    assert hist[-1] < 0.2 * hist[0] and rmse < 0.5 * rmse0
