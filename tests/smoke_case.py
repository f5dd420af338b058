"""One small forward + gradient + LSQML epoch on cuda:0, checked against the FP64 oracle
(the FP32 FFT path), and the forward model with the split-BF16 DFT-GEMM on the tensor cores."""
import numpy as np


def run_smoke():
    import torch
    from oracle import ptycho_oracle as orc
    from paper_2510_20929_gb300 import api
    from tests.parity_util import c64, f32pos, problem, rel, to_dev

    if not torch.cuda.is_available():
        raise RuntimeError("smoke() needs a CUDA device")
    p = problem(N=32, M=2, H=72, W=76, J=16, step=6.0)
    O, P, pos, I_m = c64(p["O"]), c64(p["P"]), f32pos(p["pos"]), np.float32(p["I_m"]).astype(np.float64)
    dO, dP = to_dev(O, torch.complex64), to_dev(P, torch.complex64)
    dpos, dI = to_dev(pos, torch.float32), to_dev(I_m, torch.float32)

    I_ref = orc.forward(O, P, pos)
    I = api.forward(dO, dP, dpos).cpu().numpy()
    e_fwd = rel(I, I_ref)
    e_tc = rel(api.forward(dO, dP, dpos, precision="bf16x3", batch=8).cpu().numpy(), I_ref)

    loss, gO, gP, gr = api.adjoint(dO, dP, dpos, dI, "gaussian", eps=1e-6)
    L_ref, gO_ref, gP_ref, gr_ref = orc.loss_and_gradients(O, P, pos, I_m, orc.GAUSSIAN, 1e-6)
    e_grad = max(rel(gO.cpu().numpy(), gO_ref), rel(gP.cpu().numpy(), gP_ref), rel(gr.cpu().numpy(), gr_ref))
    e_loss = abs(loss.item() - L_ref) / L_ref

    order = np.random.default_rng(3).permutation(16).astype(np.int32)
    opts = orc.LsqmlOptions(noise=orc.GAUSSIAN, batch=6, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
    O_ref, P_ref, L_ep, _ = orc.lsqml_epoch(O, P, pos, I_m, order, opts)
    l2, _ = api.lsqml_epoch(dO, dP, dpos, dI, to_dev(order, torch.int32), batch=6, delta_o=0.1,
                            delta_p=0.1, lam=1e-6, eps=1e-6)
    e_ep = max(rel(dO.cpu().numpy(), O_ref), rel(dP.cpu().numpy(), P_ref))
    print(f"smoke: forward {e_fwd:.2e}  grad {e_grad:.2e}  loss {e_loss:.2e}  epoch {e_ep:.2e}  "
          f"forward split-BF16 {e_tc:.2e}")
    assert e_fwd < 1e-5 and e_grad < 1e-4 and e_loss < 1e-5 and e_ep < 1e-4 and e_tc < 1e-3
