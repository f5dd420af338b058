"""Differentiable forms of the ptychographic forward model (autograd front end).

* :class:`FarField` maps (object, probe modes, positions) to the predicted
  intensities I_j = sum_k |F(P_k S_j(O))|^2 (Pty-Chi Sec. 2.1, Eq. 4); its
  backward calls the library's adjoint in vector-Jacobian mode, which
  recomputes the exit waves instead of storing them, and returns gradients for
  all three inputs in PyTorch's complex convention (2 dL/dz*).
* :class:`DataTerm` fuses the forward model with the amplitude (Eq. 1,
  unnormalised) or Poisson data term and returns the scalar loss; its backward
  is the fused adjoint (Eq. 2 extended to probe and positions) and never
  materialises I.
* :func:`reconstruct_adam` is the automatic-differentiation reconstructor of
  Sec. 2.2 with torch.optim.Adam on object, probe and positions.
* :class:`DataTermOPR` is the data term with orthogonal probe relaxation
  (Sec. 2.1: the primary mode of position j is sum_m w_jm U_m), differentiable
  in the object, the eigenmodes U, the real weights w, the shared modes and
  the positions; :func:`reconstruct_adam_opr` runs Adam on all of them.
* :class:`FarFieldMS` and :class:`DataTermMS` are the multislice forms
  (object slices [S, H, W], angular-spectrum propagation between slices);
  :func:`reconstruct_adam_ms` runs Adam on the slices, probe and positions.

Both Functions only marshal tensors to the C ABI; every arithmetic step runs
in the CUDA library.
"""
from __future__ import annotations

import torch

from . import api


class FarField(torch.autograd.Function):
    @staticmethod
    def forward(ctx, obj, probe, pos, precision="fp32"):
        obj, probe, pos = obj.contiguous(), probe.contiguous(), pos.contiguous()
        ctx.save_for_backward(obj, probe, pos)
        ctx.precision = precision
        return api.forward(obj, probe, pos, precision=precision)

    @staticmethod
    def backward(ctx, gI):
        obj, probe, pos = ctx.saved_tensors
        _, gO, gP, gr = api.adjoint(obj, probe, pos, gI.contiguous().to(torch.float32), "vjp",
                                    batch=256, positions_grad=ctx.needs_input_grad[2], precision=ctx.precision)
        return (gO if ctx.needs_input_grad[0] else None, gP if ctx.needs_input_grad[1] else None,
                gr if ctx.needs_input_grad[2] else None, None)


class DataTerm(torch.autograd.Function):
    @staticmethod
    def forward(ctx, obj, probe, pos, meas, noise="gaussian", eps=1e-9, precision="fp32"):
        obj, probe, pos, meas = obj.contiguous(), probe.contiguous(), pos.contiguous(), meas.contiguous()
        if not any(ctx.needs_input_grad[:3]):
            # a loss evaluation only: forward model and data term, no back-propagation
            loss, _, _, _ = api.adjoint(obj, probe, pos, meas, noise, eps=eps, batch=256, precision=precision,
                                        gradients=False)
            return loss
        loss, gO, gP, gr = api.adjoint(obj, probe, pos, meas, noise, eps=eps, batch=256,
                                       positions_grad=ctx.needs_input_grad[2], precision=precision)
        ctx.save_for_backward(gO, gP, gr)
        return loss

    @staticmethod
    def backward(ctx, gL):
        gO, gP, gr = ctx.saved_tensors
        s = gL.to(torch.float32)
        return (gO * s if ctx.needs_input_grad[0] else None, gP * s if ctx.needs_input_grad[1] else None,
                gr * s if ctx.needs_input_grad[2] else None, None, None, None, None)


class DataTermOPR(torch.autograd.Function):
    @staticmethod
    def forward(ctx, obj, U, w, P_rest, pos, meas, noise="gaussian", eps=1e-9):
        c = [t.contiguous() if t is not None else None for t in (obj, U, w, P_rest, pos, meas)]
        loss, gO, gU, gw, gP, gr = api.adjoint_opr(*c, noise, eps=eps, batch=256)
        ctx.has_rest = gP is not None
        ctx.save_for_backward(gO, gU, gw, gr, *([gP] if gP is not None else []))
        return loss

    @staticmethod
    def backward(ctx, gL):
        gO, gU, gw, gr, *rest = ctx.saved_tensors
        gP = rest[0] if ctx.has_rest else None
        s = gL.to(torch.float32)
        need = ctx.needs_input_grad
        return (gO * s if need[0] else None, gU * s if need[1] else None, gw * s if need[2] else None,
                gP * s if (need[3] and gP is not None) else None, gr * s if need[4] else None, None, None, None)


class FarFieldMS(torch.autograd.Function):
    @staticmethod
    def forward(ctx, obj, probe, pos, ms):
        obj, probe, pos = obj.contiguous(), probe.contiguous(), pos.contiguous()
        ctx.save_for_backward(obj, probe, pos)
        ctx.ms = ms
        return api.forward_ms(obj, probe, pos, ms)

    @staticmethod
    def backward(ctx, gI):
        obj, probe, pos = ctx.saved_tensors
        _, gO, gP, gr = api.adjoint_ms(obj, probe, pos, gI.contiguous().to(torch.float32), ctx.ms, "vjp",
                                       positions_grad=ctx.needs_input_grad[2])
        need = ctx.needs_input_grad
        return gO if need[0] else None, gP if need[1] else None, gr if need[2] else None, None


class DataTermMS(torch.autograd.Function):
    @staticmethod
    def forward(ctx, obj, probe, pos, meas, ms, noise="gaussian", eps=1e-9, batch=256):
        loss, gO, gP, gr = api.adjoint_ms(obj.contiguous(), probe.contiguous(), pos.contiguous(), meas.contiguous(),
                                          ms, noise, eps=eps, batch=batch, positions_grad=True)
        ctx.save_for_backward(gO, gP, gr)
        return loss

    @staticmethod
    def backward(ctx, gL):
        gO, gP, gr = ctx.saved_tensors
        s = gL.to(torch.float32)
        need = ctx.needs_input_grad
        return (gO * s if need[0] else None, gP * s if need[1] else None, gr * s if need[2] else None,
                None, None, None, None, None)


def far_field_ms(obj, probe, pos, ms):
    """Multislice intensities, differentiable in the object slices, probe modes and positions."""
    return FarFieldMS.apply(obj, probe, pos, ms)


def data_term_ms(obj, probe, pos, meas, ms, noise="gaussian", eps=1e-9, batch=256):
    """Scalar data term of the multislice model (differentiable in slices, probe, positions);
    positions are processed in minibatches of ``batch`` inside the library call."""
    return DataTermMS.apply(obj, probe, pos, meas, ms, noise, eps, batch)


def data_term_opr(obj, U, w, P_rest, pos, meas, noise="gaussian", eps=1e-9):
    """Scalar data term with the relaxed primary mode (differentiable in obj, U, w, P_rest, pos)."""
    return DataTermOPR.apply(obj, U, w, P_rest, pos, meas, noise, eps)


def far_field(obj, probe, pos, precision="fp32"):
    """Predicted intensities, differentiable in object, probe modes and positions
    (``precision`` "bf16x3": the far field as split-BF16 DFT-GEMMs, windows 32-128)."""
    return FarField.apply(obj, probe, pos, precision)


def data_term(obj, probe, pos, meas, noise="gaussian", eps=1e-9, precision="fp32"):
    """Scalar data term (Gaussian amplitude or Poisson), differentiable in object, probe, positions."""
    return DataTerm.apply(obj, probe, pos, meas, noise, eps, precision)


def reconstruct_adam(obj, probe, pos, meas, epochs=10, lr_object=1e-2, lr_probe=1e-2, lr_pos=1e-1,
                     noise="gaussian", eps=1e-9, update=("object", "probe", "positions"), precision="fp32"):
    """Adam on object, probe modes and positions (whole data set per step); returns the loss history.

    Learning rates are in the units of each variable (object and probe
    amplitudes, pixels for positions). The tensors are updated in place.
    """
    params = []
    obj.requires_grad_("object" in update)
    probe.requires_grad_("probe" in update)
    pos.requires_grad_("positions" in update)
    if "object" in update:
        params.append({"params": [obj], "lr": lr_object})
    if "probe" in update:
        params.append({"params": [probe], "lr": lr_probe})
    if "positions" in update:
        params.append({"params": [pos], "lr": lr_pos})
    opt = torch.optim.Adam(params)
    hist = []
    for _ in range(epochs):
        opt.zero_grad(set_to_none=True)
        loss = data_term(obj, probe, pos, meas, noise, eps, precision)
        loss.backward()
        opt.step()
        hist.append(loss.item())
    obj.requires_grad_(False)
    probe.requires_grad_(False)
    pos.requires_grad_(False)
    return hist


def reconstruct_adam_opr(obj, U, w, P_rest, pos, meas, epochs=10, lr_object=1e-2, lr_probe=1e-2,
                         lr_weights=1e-2, lr_pos=1e-1, noise="gaussian", eps=1e-9,
                         update=("object", "eigenmodes", "weights", "probe", "positions")):
    """Adam with orthogonal probe relaxation; returns the loss history (tensors updated in place).

    "probe" in ``update`` refers to the shared modes P_rest (ignored when None).
    """
    groups = [("object", obj, lr_object), ("eigenmodes", U, lr_probe), ("weights", w, lr_weights),
              ("probe", P_rest, lr_probe), ("positions", pos, lr_pos)]
    params = []
    for name, t, lr in groups:
        if t is None:
            continue
        t.requires_grad_(name in update)
        if name in update:
            params.append({"params": [t], "lr": lr})
    opt = torch.optim.Adam(params)
    hist = []
    for _ in range(epochs):
        opt.zero_grad(set_to_none=True)
        loss = data_term_opr(obj, U, w, P_rest, pos, meas, noise, eps)
        loss.backward()
        opt.step()
        hist.append(loss.item())
    for _, t, _ in groups:
        if t is not None:
            t.requires_grad_(False)
    return hist


def reconstruct_adam_ms(obj, probe, pos, meas, ms, epochs=10, lr_object=1e-2, lr_probe=1e-2, lr_pos=1e-1,
                        noise="gaussian", eps=1e-9, update=("object", "probe", "positions")):
    """Adam on the object slices [S, H, W], probe modes and positions of the
    multislice model; returns the loss history (tensors updated in place)."""
    groups = [("object", obj, lr_object), ("probe", probe, lr_probe), ("positions", pos, lr_pos)]
    params = []
    for name, t, lr in groups:
        t.requires_grad_(name in update)
        if name in update:
            params.append({"params": [t], "lr": lr})
    opt = torch.optim.Adam(params)
    hist = []
    for _ in range(epochs):
        opt.zero_grad(set_to_none=True)
        loss = data_term_ms(obj, probe, pos, meas, ms, noise, eps)
        loss.backward()
        opt.step()
        hist.append(loss.item())
    for _, t, _ in groups:
        t.requires_grad_(False)
    return hist
