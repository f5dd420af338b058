"""Thin ctypes binding of libptycho (argument marshalling only).

Every function here validates tensor dtypes, shapes and devices, passes raw
device pointers and the current CUDA stream to the C ABI declared in
include/ptycho.h, and raises :class:`PtychoError` on a non-OK status. All
arithmetic runs in the library's sm_103a kernels; there is no CPU or PyTorch
fallback, and loading fails loudly if the library has not been built.

Tensor conventions: object complex64 [H, W]; probe complex64 [M, N, N];
positions float32 [J, 2] (y, x) probe centres; intensities float32 [J, N, N]
with the zero frequency at [0, 0]; batch order int32 [J].
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libptycho.so")

GAUSSIAN, POISSON, VJP = 0, 1, 2
FLAG_GRAPH = 1
FLAG_AUTOTUNE = 2
_NOISE = {"gaussian": GAUSSIAN, "poisson": POISSON, "vjp": VJP}

STATUS = {0: "PTYCHO_OK", 1: "PTYCHO_ERR_ARG", 2: "PTYCHO_ERR_BOUNDS", 3: "PTYCHO_ERR_NONFINITE",
          4: "PTYCHO_ERR_CUDA", 5: "PTYCHO_ERR_TIMEOUT", 6: "PTYCHO_ERR_UNSUPPORTED",
          7: "PTYCHO_ERR_WORKSPACE", 8: "PTYCHO_ERR_TOO_LARGE"}


class PtychoError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({status_string(status)})")


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("total_ms", ctypes.c_double)]


class Dims(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("N", ctypes.c_int32),
                ("M", ctypes.c_int32), ("J", ctypes.c_int32)]


class LsqmlOpts(ctypes.Structure):
    _fields_ = [("noise", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("update_object", ctypes.c_int32), ("update_probe", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("update_positions", ctypes.c_int32),
                ("object_per_epoch", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("delta_o", ctypes.c_double), ("delta_p", ctypes.c_double),
                ("lambda_reg", ctypes.c_double), ("eps", ctypes.c_double),
                ("pos_step", ctypes.c_double), ("pos_max_shift", ctypes.c_double)]


class Multislice(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int32), ("recompute", ctypes.c_int32), ("dz", ctypes.c_double),
                ("wavelength", ctypes.c_double), ("pixel_size", ctypes.c_double)]


class OprOpts(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("update_weights", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2),
                ("weight_step", ctypes.c_double)]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Load libptycho.so (once); raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        dims_p = ctypes.POINTER(Dims)
        opts_p = ctypes.POINTER(LsqmlOpts)
        opr_p = ctypes.POINTER(OprOpts)
        ms_p = ctypes.POINTER(Multislice)
        sigs = {
            "ptycho_workspace_bytes_ms": (ctypes.c_size_t, [dims_p, ms_p, ctypes.c_int32]),
            "ptycho_forward_ms": (ctypes.c_int, [dims_p, ms_p, _P, _P, _P, _P, ctypes.c_int32, _P, ctypes.c_size_t,
                                                 _P]),
            "ptycho_adjoint_ms": (ctypes.c_int, [dims_p, ms_p, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_double,
                                                 ctypes.c_int32, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
            "ptycho_workspace_bytes_lsqml_ms": (ctypes.c_size_t, [dims_p, ms_p, opts_p]),
            "ptycho_lsqml_epoch_ms": (ctypes.c_int, [dims_p, ms_p, _P, _P, _P, _P, _P, opts_p, _P, _P, _P,
                                                     ctypes.c_size_t, _P]),
            "ptycho_workspace_bytes_opr": (ctypes.c_size_t, [dims_p, ctypes.c_int32, ctypes.c_int32]),
            "ptycho_forward_opr": (ctypes.c_int, [dims_p, ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P,
                                                  ctypes.c_size_t, _P]),
            "ptycho_adjoint_opr": (ctypes.c_int, [dims_p, ctypes.c_int32, _P, _P, _P, _P, _P, _P, ctypes.c_int32,
                                                  ctypes.c_double, ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P,
                                                  ctypes.c_size_t, _P]),
            "ptycho_lsqml_epoch_opr": (ctypes.c_int, [dims_p, opr_p, _P, _P, _P, _P, _P, _P, _P, opts_p, _P, _P,
                                                      _P, ctypes.c_size_t, _P]),
            "ptycho_workspace_bytes_opr_batched": (ctypes.c_size_t, [ctypes.c_int32, dims_p, opr_p, opts_p]),
            "ptycho_lsqml_epoch_opr_batched": (ctypes.c_int, [ctypes.c_int32, dims_p, opr_p, _P, _P, _P, _P, _P,
                                                              _P, _P, opts_p, _P, _P, ctypes.c_size_t, _P]),
            "ptycho_workspace_bytes": (ctypes.c_size_t, [dims_p, ctypes.c_int32]),
            "ptycho_workspace_bytes_opts": (ctypes.c_size_t, [dims_p, opts_p]),
            "ptycho_sampler_order": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                    ctypes.c_uint64, _P]),
            "ptycho_host_workspace_bytes_opts": (ctypes.c_size_t, [dims_p, opts_p]),
            "ptycho_host_workspace_bytes": (ctypes.c_size_t, [dims_p, ctypes.c_int32]),
            "ptycho_workspace_init": (ctypes.c_int, [_P, ctypes.c_size_t, _P]),
            "ptycho_forward": (ctypes.c_int, [dims_p, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
            "ptycho_forward_ex": (ctypes.c_int, [dims_p, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, _P,
                                                 ctypes.c_size_t, _P]),
            "ptycho_adjoint_ex": (ctypes.c_int, [dims_p, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int32,
                                                 ctypes.c_double, ctypes.c_int32, _P, _P, _P, _P, _P,
                                                 ctypes.c_size_t, _P]),
            "ptycho_adjoint": (ctypes.c_int, [dims_p, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_double,
                                              ctypes.c_int32, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
            "ptycho_lsqml_epoch": (ctypes.c_int, [dims_p, _P, _P, _P, _P, _P, opts_p, _P, _P, _P,
                                                  ctypes.c_size_t, _P]),
            "ptycho_lsqml_epoch_host": (ctypes.c_int, [dims_p, _P, _P, _P, _P, _P, opts_p, _P, _P,
                                                       ctypes.c_size_t, _P]),
            "ptycho_lsqml_epoch_static": (ctypes.c_int, [dims_p, _P, _P, _P, _P, _P, opts_p, _P, _P, _P]),
            "ptycho_workspace_bytes_batched": (ctypes.c_size_t, [ctypes.c_int32, dims_p, opts_p]),
            "ptycho_tuning_read": (ctypes.c_int32, [dims_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                                    ctypes.POINTER(ctypes.c_float)]),
            "ptycho_tuning_set": (ctypes.c_int, [dims_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
            "ptycho_lsqml_epoch_batched": (ctypes.c_int, [ctypes.c_int32, dims_p, _P, _P, _P, _P, _P, opts_p, _P,
                                                          _P, ctypes.c_size_t, _P]),
            "ptycho_status_read": (ctypes.c_int, [_P, _P]),
            "ptycho_selftest_wait_timeout": (ctypes.c_int, [_P, ctypes.c_size_t, _P]),
            "ptycho_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "ptycho_version": (ctypes.c_char_p, []),
            "ptycho_profile_enable": (ctypes.c_int, [ctypes.c_int32]),
            "ptycho_profile_read": (ctypes.c_int32, [ctypes.POINTER(KernelTime), ctypes.c_int32]),
            "ptycho_profile_select": (ctypes.c_int32, [ctypes.c_char_p]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def status_string(status: int) -> str:
    return lib().ptycho_status_string(int(status)).decode()


def profile_enable(on: bool = True, only: str | None = None) -> None:
    """Bracket every library kernel launch (or only those of kernel ``only``)
    with CUDA events on its stream."""
    if not lib().ptycho_profile_select(only.encode() if only else None):
        raise ValueError(f"unknown kernel name {only!r}")
    _check(lib().ptycho_profile_enable(1 if on else 0), "ptycho_profile_enable")


def profile_read() -> dict:
    """{kernel name: (launches, total ms)} since the last read (synchronises)."""
    buf = (KernelTime * 32)()
    n = lib().ptycho_profile_read(buf, 32)
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(min(n, 32))}


def _check(st: int, where: str) -> None:
    if st != 0:
        raise PtychoError(st, where)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return _P(s.cuda_stream)


def _ptr(t):
    return _P(t.data_ptr()) if t is not None else _P(0)


def _need(t, name, dtype, shape=None, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def dims_of(obj, probe, pos) -> Dims:
    H, W = obj.shape
    M, N, N2 = probe.shape
    if N != N2:
        raise ValueError("probe modes must be square")
    return Dims(H, W, N, M, pos.shape[0])


class Workspace:
    """Caller-owned device scratch for the library (a uint8 torch tensor, 256-B aligned)."""

    def __init__(self, nbytes: int, device, stream=None):
        self.nbytes = int(nbytes)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.buf.data_ptr()) % 256
        self.ptr = self.buf.data_ptr() + off
        _check(lib().ptycho_workspace_init(_P(self.ptr), self.nbytes, _stream(stream)), "workspace_init")

    def status(self, stream=None) -> int:
        """Synchronise and return (and clear) the device-side status."""
        return lib().ptycho_status_read(_P(self.ptr), _stream(stream))


_ws_cache: dict = {}


def workspace(dims: Dims, batch: int, device, host: bool = False, opr_K: int = 0, opts=None) -> Workspace:
    """A cached workspace large enough for these dimensions and minibatch size
    (with opr_K > 0, for the relaxed-probe entry points with K eigenmodes; with
    ``opts``, for an LSQML epoch with those options)."""
    if opr_K > 0:
        need = lib().ptycho_workspace_bytes_opr(ctypes.byref(dims), int(opr_K), int(batch))
    elif opts is not None:
        fn = lib().ptycho_host_workspace_bytes_opts if host else lib().ptycho_workspace_bytes_opts
        need = fn(ctypes.byref(dims), ctypes.byref(opts))
    else:
        fn = lib().ptycho_host_workspace_bytes if host else lib().ptycho_workspace_bytes
        need = fn(ctypes.byref(dims), int(batch))
    if need == 0:
        raise PtychoError(6, "workspace_bytes")
    key = (str(device), host)
    ws = _ws_cache.get(key)
    if ws is None or ws.nbytes < need:
        ws = Workspace(need, device)
        _ws_cache[key] = ws
    return ws


def _finish(ws: Workspace, where: str, check: bool):
    if check:
        _check(ws.status(), where)


PRECISIONS = {"fp32": 0, "bf16x3": 1}


def _precision(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def forward(obj, probe, pos, *, precision="fp32", batch: int = 256, check: bool = True):
    """Predicted intensities I [J, N, N] = sum_k |F(P_k S_j(O))|^2.

    ``precision`` "bf16x3" evaluates F as split-BF16 DFT-GEMMs on the tensor
    cores (windows 32, 64, 128), in chunks of ``batch`` positions."""
    _need(obj, "object", torch.complex64)
    _need(probe, "probe", torch.complex64, device=obj.device)
    _need(pos, "positions", torch.float32, device=obj.device)
    d = dims_of(obj, probe, pos)
    I = torch.empty((d.J, d.N, d.N), dtype=torch.float32, device=obj.device)
    pr = _precision(precision)
    B = max(1, min(int(batch), max(d.J, 1)))
    ws = workspace(d, B if pr else 1, obj.device)
    _check(lib().ptycho_forward_ex(ctypes.byref(d), pr, B, _ptr(obj), _ptr(probe), _ptr(pos), _ptr(I),
                                   _P(ws.ptr), ws.nbytes, _stream()), "ptycho_forward_ex")
    _finish(ws, "ptycho_forward_ex", check)
    return I


def adjoint(obj, probe, pos, meas, noise="gaussian", eps: float = 0.0, batch: int = 256, *,
            positions_grad: bool = True, precision="fp32", check: bool = True, gradients: bool = True):
    """Loss and gradients (grad = 2 dL/dz*): returns (loss, g_object, g_probe, g_pos).

    ``noise`` is "gaussian", "poisson", or "vjp" (then ``meas`` holds dL/dI and
    the returned loss is None). ``precision`` "bf16x3" evaluates the far field as
    split-BF16 DFT-GEMMs on the tensor cores (windows 32, 64, 128). With
    ``gradients=False`` only the loss is evaluated (forward model and data
    term, no back-propagation) and the three gradients are None.
    """
    nz = _NOISE[noise] if isinstance(noise, str) else int(noise)
    _need(obj, "object", torch.complex64)
    _need(probe, "probe", torch.complex64, device=obj.device)
    _need(pos, "positions", torch.float32, device=obj.device)
    d = dims_of(obj, probe, pos)
    _need(meas, "meas", torch.float32, (d.J, d.N, d.N), device=obj.device)
    if not gradients and nz == VJP:
        raise ValueError("the vjp mode has no loss to evaluate without gradients")
    B = max(1, min(int(batch), max(d.J, 1)))
    gO = torch.zeros_like(obj) if gradients else None
    gP = torch.zeros_like(probe) if gradients else None
    gr = torch.zeros((d.J, 2), dtype=torch.float32, device=obj.device) if (positions_grad and gradients) else None
    loss = torch.zeros((), dtype=torch.float64, device=obj.device)
    ws = workspace(d, B, obj.device)
    _check(lib().ptycho_adjoint_ex(ctypes.byref(d), _precision(precision), _ptr(obj), _ptr(probe), _ptr(pos),
                                   _ptr(meas), nz, float(eps), B, _ptr(gO), _ptr(gP), _ptr(gr),
                                   _ptr(loss) if nz != VJP else _P(0), _P(ws.ptr), ws.nbytes, _stream()),
           "ptycho_adjoint_ex")
    _finish(ws, "ptycho_adjoint_ex", check)
    return (None if nz == VJP else loss), gO, gP, gr


SAMPLERS = {"random": 0, "uniform": 1, "compact": 2}


def sampler_order(pos, batch: int, kind="compact", seed: int = 0):
    """Minibatch order (int32 CPU tensor [J]) of the random, uniform or compact
    sampler for positions ``pos`` (float32 [J, 2], any device; copied to the host)."""
    p = pos.detach().to("cpu", torch.float32).contiguous() if isinstance(pos, torch.Tensor) else \
        torch.as_tensor(pos, dtype=torch.float32).contiguous()
    J = p.shape[0]
    out = torch.empty(J, dtype=torch.int32)
    k = SAMPLERS[kind] if isinstance(kind, str) else int(kind)
    _check(lib().ptycho_sampler_order(_P(p.data_ptr()), J, int(batch), k, int(seed) & ((1 << 64) - 1),
                                      _P(out.data_ptr())), "ptycho_sampler_order")
    return out


def make_opts(noise="gaussian", batch: int = 256, delta_o: float = 0.1, delta_p: float = 0.1,
              lam: float = 1e-6, eps: float = 1e-9, update_object: bool = True,
              update_probe: bool = True, graph: bool = False, autotune: bool = False,
              update_positions: bool = False, pos_step: float = 1.0, pos_max_shift: float = 1.0,
              object_per_epoch: bool = False, precision="fp32") -> LsqmlOpts:
    """LSQML epoch options (the fields of ptycho_lsqml_opts). ``precision``:
    "fp32" (shared-memory FFTs) or "bf16x3" (split-BF16 DFT-GEMMs on the tensor
    cores, windows 32, 64, 128)."""
    o = LsqmlOpts()
    o.flags = (FLAG_GRAPH if graph else 0) | (FLAG_AUTOTUNE if autotune else 0)
    o.noise = _NOISE[noise] if isinstance(noise, str) else int(noise)
    o.batch = int(batch)
    o.update_object = int(bool(update_object))
    o.update_probe = int(bool(update_probe))
    o.update_positions = int(bool(update_positions))
    o.object_per_epoch = int(bool(object_per_epoch))
    o.precision = _precision(precision)
    o.delta_o, o.delta_p, o.lambda_reg, o.eps = float(delta_o), float(delta_p), float(lam), float(eps)
    o.pos_step, o.pos_max_shift = float(pos_step), float(pos_max_shift)
    return o


def lsqml_epoch(obj, probe, pos, meas, order=None, opts: LsqmlOpts | None = None, *,
                want_alpha: bool = False, check: bool = True, **kw):
    """One LSQML epoch, updating ``obj`` and ``probe`` (and, with
    ``update_positions``, ``pos``) in place.

    Returns (loss, alpha): loss is a float64 device scalar; alpha a float64
    [J, 2] device tensor of (alpha_O, alpha_P) or None.
    """
    if opts is None:
        opts = make_opts(**kw)
    _need(obj, "object", torch.complex64)
    _need(probe, "probe", torch.complex64, device=obj.device)
    _need(pos, "positions", torch.float32, device=obj.device)
    d = dims_of(obj, probe, pos)
    _need(meas, "meas", torch.float32, (d.J, d.N, d.N), device=obj.device)
    if order is not None:
        _need(order, "order", torch.int32, (d.J,), device=obj.device)
    loss = torch.zeros((), dtype=torch.float64, device=obj.device)
    alpha = torch.zeros((pos.shape[0], 2), dtype=torch.float64, device=obj.device) if want_alpha else None
    ws = workspace(d, opts.batch, obj.device, opts=opts)
    _check(lib().ptycho_lsqml_epoch(ctypes.byref(d), _ptr(obj), _ptr(probe), _ptr(pos), _ptr(meas),
                                    _ptr(order), ctypes.byref(opts), _ptr(loss), _ptr(alpha),
                                    _P(ws.ptr), ws.nbytes, _stream()), "ptycho_lsqml_epoch")
    _finish(ws, "ptycho_lsqml_epoch", check)
    return loss, alpha


TUNED = ("pass1", "pass2", "probe_reduce")   # the kernels the autotuner chooses variants of
TUNE_MAX = 4


def tuning(dims: Dims, batch: int):
    """Autotuner choice for these dimensions on the current device, or None:
    {"pass1": variant, "pass2": variant, "probe_reduce": variant,
     "pass1_ms": [candidate ms...], "pass2_ms": [...], "probe_reduce_ms": [...]}."""
    v = (ctypes.c_int32 * len(TUNED))()
    m = (ctypes.c_float * (len(TUNED) * TUNE_MAX))()
    if not lib().ptycho_tuning_read(ctypes.byref(dims), int(batch), v, m):
        return None
    out = {k: v[i] for i, k in enumerate(TUNED)}
    out.update({k + "_ms": list(m[i * TUNE_MAX:(i + 1) * TUNE_MAX]) for i, k in enumerate(TUNED)})
    return out


def set_tuning(dims: Dims, batch: int, pass1: int = 0, pass2: int = 0, probe_reduce: int = 0):
    """Pins the kernel variants used for these dimensions and batch on the current device."""
    v = (ctypes.c_int32 * len(TUNED))(int(pass1), int(pass2), int(probe_reduce))
    _check(lib().ptycho_tuning_set(ctypes.byref(dims), int(batch), v), "ptycho_tuning_set")


def lsqml_epoch_batched(recons, opts, *, check: bool = True):
    """One epoch for each of several independent reconstructions, run concurrently.

    ``recons`` is a list of (obj, probe, pos, meas, order) tuples of CUDA
    tensors (order may be None); ``opts`` one LsqmlOpts or a list of them.
    Objects and probes are updated in place; returns the float64 [n] losses.
    """
    n = len(recons)
    if n == 0:
        raise ValueError("no reconstructions")
    opts_list = opts if isinstance(opts, (list, tuple)) else [opts] * n
    dev = recons[0][0].device
    dims = (Dims * n)()
    OA = (LsqmlOpts * n)(*opts_list)
    ptrs = {k: (ctypes.c_void_p * n)() for k in ("o", "p", "r", "m", "q")}
    for i, (obj, probe, pos, meas, order) in enumerate(recons):
        _need(obj, "object", torch.complex64, device=dev)
        _need(probe, "probe", torch.complex64, device=dev)
        _need(pos, "positions", torch.float32, device=dev)
        d = dims_of(obj, probe, pos)
        _need(meas, "meas", torch.float32, (d.J, d.N, d.N), device=dev)
        if order is not None:
            _need(order, "order", torch.int32, (d.J,), device=dev)
        dims[i] = d
        ptrs["o"][i], ptrs["p"][i], ptrs["r"][i], ptrs["m"][i] = (obj.data_ptr(), probe.data_ptr(),
                                                                   pos.data_ptr(), meas.data_ptr())
        ptrs["q"][i] = order.data_ptr() if order is not None else None
    need = lib().ptycho_workspace_bytes_batched(n, dims, OA)
    if need == 0:
        raise PtychoError(6, "workspace_bytes_batched")
    key = (str(dev), "batched")
    ws = _ws_cache.get(key)
    if ws is None or ws.nbytes < need:
        ws = Workspace(need, dev)
        _ws_cache[key] = ws
    losses = torch.zeros(n, dtype=torch.float64, device=dev)
    _check(lib().ptycho_lsqml_epoch_batched(n, dims, ptrs["o"], ptrs["p"], ptrs["r"], ptrs["m"], ptrs["q"], OA,
                                            _ptr(losses), _P(ws.ptr), ws.nbytes, _stream()),
           "ptycho_lsqml_epoch_batched")
    if check:
        off = 0
        for i in range(n):
            _check(lib().ptycho_status_read(_P(ws.ptr + off), _stream()), f"ptycho_lsqml_epoch_batched[{i}]")
            off += lib().ptycho_workspace_bytes_opts(ctypes.byref(dims[i]), ctypes.byref(OA[i]))
    return losses


def lsqml_epoch_host(obj, probe, pos, meas, order, opts: LsqmlOpts, device=None):
    """LSQML epoch on HOST (CPU, ideally pinned) tensors through the host-buffer entry point.

    ``obj`` and ``probe`` (complex64, CPU; ``pos`` too with update_positions)
    are updated in place; returns the loss.
    """
    for t, name, dt in ((obj, "object", torch.complex64), (probe, "probe", torch.complex64),
                        (pos, "positions", torch.float32), (meas, "meas", torch.float32)):
        if t.device.type != "cpu" or t.dtype != dt or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CPU {dt} tensor")
    if order is not None and (order.device.type != "cpu" or order.dtype != torch.int32):
        raise ValueError("order must be a CPU int32 tensor")
    device = device or torch.device("cuda", torch.cuda.current_device())
    d = dims_of(obj, probe, pos)
    ws = workspace(d, opts.batch, device, host=True, opts=opts)
    loss = ctypes.c_double(0.0)
    _check(lib().ptycho_lsqml_epoch_host(ctypes.byref(d), _ptr(obj), _ptr(probe), _ptr(pos), _ptr(meas),
                                         _ptr(order), ctypes.byref(opts), ctypes.byref(loss),
                                         _P(ws.ptr), ws.nbytes, _stream()), "ptycho_lsqml_epoch_host")
    _check(ws.status(), "ptycho_lsqml_epoch_host")
    return loss.value


# ---------------------------------------------------------------------------
# Orthogonal probe relaxation: primary mode P_j0 = sum_m w[j, m] U[m] over K
# eigenmodes U complex64 [K, N, N] with real weights w float32 [J, K]; the
# shared modes P_rest complex64 [M - 1, N, N] (None when there are none).
# ---------------------------------------------------------------------------
def _opr_dims(obj, U, w, P_rest, pos) -> Dims:
    _need(obj, "object", torch.complex64)
    _need(U, "eigenmodes", torch.complex64, device=obj.device)
    K, N, N2 = U.shape
    if N != N2:
        raise ValueError("eigenmodes must be square")
    _need(pos, "positions", torch.float32, device=obj.device)
    J = pos.shape[0]
    _need(w, "weights", torch.float32, (J, K), device=obj.device)
    Mr = 0
    if P_rest is not None:
        _need(P_rest, "shared modes", torch.complex64, device=obj.device)
        if tuple(P_rest.shape[1:]) != (N, N):
            raise ValueError("shared modes must match the eigenmodes' window")
        Mr = P_rest.shape[0]
    H, W = obj.shape
    return Dims(H, W, N, 1 + Mr, J)


def forward_opr(obj, U, w, P_rest, pos, *, check: bool = True):
    """Predicted intensities [J, N, N] with the relaxed primary mode."""
    d = _opr_dims(obj, U, w, P_rest, pos)
    I = torch.empty((d.J, d.N, d.N), dtype=torch.float32, device=obj.device)
    ws = workspace(d, 1, obj.device)
    _check(lib().ptycho_forward_opr(ctypes.byref(d), U.shape[0], _ptr(obj), _ptr(U), _ptr(w), _ptr(P_rest),
                                    _ptr(pos), _ptr(I), _P(ws.ptr), ws.nbytes, _stream()), "ptycho_forward_opr")
    _finish(ws, "ptycho_forward_opr", check)
    return I


def adjoint_opr(obj, U, w, P_rest, pos, meas, noise="gaussian", eps: float = 0.0, batch: int = 256, *,
                positions_grad: bool = True, weights_grad: bool = True, check: bool = True):
    """Loss and gradients through the relaxed model: (loss, g_object, g_U, g_w, g_P_rest, g_pos).

    Complex gradients are 2 dL/dz*; g_w = dL/dw (real). ``noise`` as in :func:`adjoint`.
    """
    nz = _NOISE[noise] if isinstance(noise, str) else int(noise)
    d = _opr_dims(obj, U, w, P_rest, pos)
    K = U.shape[0]
    _need(meas, "meas", torch.float32, (d.J, d.N, d.N), device=obj.device)
    B = max(1, min(int(batch), max(d.J, 1)))
    gO, gU = torch.zeros_like(obj), torch.zeros_like(U)
    gw = torch.zeros_like(w) if weights_grad else None
    gP = torch.zeros_like(P_rest) if P_rest is not None else None
    gr = torch.zeros((d.J, 2), dtype=torch.float32, device=obj.device) if positions_grad else None
    loss = torch.zeros((), dtype=torch.float64, device=obj.device)
    ws = workspace(d, B, obj.device, opr_K=K)
    _check(lib().ptycho_adjoint_opr(ctypes.byref(d), K, _ptr(obj), _ptr(U), _ptr(w), _ptr(P_rest), _ptr(pos),
                                    _ptr(meas), nz, float(eps), B, _ptr(gO), _ptr(gU), _ptr(gw), _ptr(gP), _ptr(gr),
                                    _ptr(loss) if nz != VJP else _P(0), _P(ws.ptr), ws.nbytes, _stream()),
           "ptycho_adjoint_opr")
    _finish(ws, "ptycho_adjoint_opr", check)
    return (None if nz == VJP else loss), gO, gU, gw, gP, gr


def make_opr_opts(K: int, update_weights: bool = True, weight_step: float = 1.0) -> OprOpts:
    r = OprOpts()
    r.K = int(K)
    r.update_weights = int(bool(update_weights))
    r.weight_step = float(weight_step)
    return r


def lsqml_epoch_opr(obj, U, w, P_rest, pos, meas, order=None, opts: LsqmlOpts | None = None,
                    opr: OprOpts | None = None, *, want_alpha: bool = False, check: bool = True, **kw):
    """One LSQML epoch with the relaxed primary mode; updates obj, U, w, P_rest in place.

    Returns (loss, alpha) as :func:`lsqml_epoch`.
    """
    if opts is None:
        opts = make_opts(**kw)
    d = _opr_dims(obj, U, w, P_rest, pos)
    if opr is None:
        opr = make_opr_opts(U.shape[0])
    if opr.K != U.shape[0]:
        raise ValueError("opr.K must equal the number of eigenmodes")
    _need(meas, "meas", torch.float32, (d.J, d.N, d.N), device=obj.device)
    if order is not None:
        _need(order, "order", torch.int32, device=obj.device)
    loss = torch.zeros((), dtype=torch.float64, device=obj.device)
    alpha = torch.zeros((d.J, 2), dtype=torch.float64, device=obj.device) if want_alpha else None
    ws = workspace(d, opts.batch, obj.device, opr_K=opr.K)
    _check(lib().ptycho_lsqml_epoch_opr(ctypes.byref(d), ctypes.byref(opr), _ptr(obj), _ptr(U), _ptr(w),
                                        _ptr(P_rest), _ptr(pos), _ptr(meas), _ptr(order), ctypes.byref(opts),
                                        _ptr(loss), _ptr(alpha), _P(ws.ptr), ws.nbytes, _stream()),
           "ptycho_lsqml_epoch_opr")
    _finish(ws, "ptycho_lsqml_epoch_opr", check)
    return loss, alpha


def lsqml_epoch_opr_batched(recons, opts, oprs, *, check: bool = True):
    """One relaxed-probe LSQML epoch for each of several reconstructions, run concurrently.

    ``recons`` is a list of (obj, U, w, P_rest, pos, meas, order) tuples (P_rest
    and order may be None); ``opts`` and ``oprs`` one options struct or a list.
    Updates obj, U, w, P_rest in place; returns the float64 [n] losses.
    """
    n = len(recons)
    if n == 0:
        raise ValueError("no reconstructions")
    opts_list = opts if isinstance(opts, (list, tuple)) else [opts] * n
    opr_list = oprs if isinstance(oprs, (list, tuple)) else [oprs] * n
    dev = recons[0][0].device
    dims = (Dims * n)()
    OA = (LsqmlOpts * n)(*opts_list)
    RA = (OprOpts * n)(*opr_list)
    ptrs = {k: (ctypes.c_void_p * n)() for k in ("o", "u", "w", "p", "r", "m", "q")}
    any_rest = False
    for i, (obj, U, w, P_rest, pos, meas, order) in enumerate(recons):
        d = _opr_dims(obj, U, w, P_rest, pos)
        if RA[i].K != U.shape[0]:
            raise ValueError("opr.K must equal the number of eigenmodes")
        _need(meas, "meas", torch.float32, (d.J, d.N, d.N), device=dev)
        if order is not None:
            _need(order, "order", torch.int32, (d.J,), device=dev)
        dims[i] = d
        ptrs["o"][i], ptrs["u"][i], ptrs["w"][i] = obj.data_ptr(), U.data_ptr(), w.data_ptr()
        ptrs["p"][i] = P_rest.data_ptr() if P_rest is not None else None
        any_rest = any_rest or P_rest is not None
        ptrs["r"][i], ptrs["m"][i] = pos.data_ptr(), meas.data_ptr()
        ptrs["q"][i] = order.data_ptr() if order is not None else None
    need = lib().ptycho_workspace_bytes_opr_batched(n, dims, RA, OA)
    if need == 0:
        raise PtychoError(6, "workspace_bytes_opr_batched")
    key = (str(dev), "batched")
    ws = _ws_cache.get(key)
    if ws is None or ws.nbytes < need:
        ws = Workspace(need, dev)
        _ws_cache[key] = ws
    losses = torch.zeros(n, dtype=torch.float64, device=dev)
    _check(lib().ptycho_lsqml_epoch_opr_batched(n, dims, RA, ptrs["o"], ptrs["u"], ptrs["w"],
                                                ptrs["p"] if any_rest else None, ptrs["r"], ptrs["m"], ptrs["q"], OA,
                                                _ptr(losses), _P(ws.ptr), ws.nbytes, _stream()),
           "ptycho_lsqml_epoch_opr_batched")
    if check:
        off = 0
        for i in range(n):
            _check(lib().ptycho_status_read(_P(ws.ptr + off), _stream()), f"ptycho_lsqml_epoch_opr_batched[{i}]")
            off += lib().ptycho_workspace_bytes_opr(ctypes.byref(dims[i]), RA[i].K, OA[i].batch)
    return losses


# ---------------------------------------------------------------------------
# Multislice: object slices complex64 [S, H, W], angular-spectrum propagation
# between slices (spacing dz, wavelength and pixel size in one unit).
# ---------------------------------------------------------------------------
def make_multislice(S: int, dz: float, wavelength: float, pixel_size: float, *,
                    recompute: bool = False) -> Multislice:
    """recompute: the backward passes recompute each mode's incident waves
    instead of keeping every mode's from the forward pass (less workspace and
    DRAM traffic, 2 (S-1) more 2-D transforms per mode)."""
    m = Multislice()
    m.S, m.dz, m.wavelength, m.pixel_size = int(S), float(dz), float(wavelength), float(pixel_size)
    m.recompute = int(bool(recompute))
    return m


def _ms_dims(obj, probe, pos, ms):
    _need(obj, "object slices", torch.complex64)
    _need(probe, "probe", torch.complex64, device=obj.device)
    _need(pos, "positions", torch.float32, device=obj.device)
    if obj.dim() != 3 or obj.shape[0] != ms.S:
        raise ValueError("object must be [S, H, W] with S = ms.S")
    M, N, N2 = probe.shape
    if N != N2:
        raise ValueError("probe modes must be square")
    return Dims(obj.shape[1], obj.shape[2], N, M, pos.shape[0])


def _ms_workspace(d, ms, batch, device):
    need = lib().ptycho_workspace_bytes_ms(ctypes.byref(d), ctypes.byref(ms), int(batch))
    if need == 0:
        raise PtychoError(6, "workspace_bytes_ms")
    key = (str(device), "ms")
    ws = _ws_cache.get(key)
    if ws is None or ws.nbytes < need:
        ws = Workspace(need, device)
        _ws_cache[key] = ws
    return ws


def forward_ms(obj, probe, pos, ms: Multislice, batch: int = 256, *, check: bool = True):
    """Predicted intensities [J, N, N] of the multislice model."""
    d = _ms_dims(obj, probe, pos, ms)
    B = max(1, min(int(batch), max(d.J, 1)))
    I = torch.empty((d.J, d.N, d.N), dtype=torch.float32, device=obj.device)
    ws = _ms_workspace(d, ms, B, obj.device)
    _check(lib().ptycho_forward_ms(ctypes.byref(d), ctypes.byref(ms), _ptr(obj), _ptr(probe), _ptr(pos), _ptr(I), B,
                                   _P(ws.ptr), ws.nbytes, _stream()), "ptycho_forward_ms")
    _finish(ws, "ptycho_forward_ms", check)
    return I


def adjoint_ms(obj, probe, pos, meas, ms: Multislice, noise="gaussian", eps: float = 0.0, batch: int = 256, *,
               positions_grad: bool = True, check: bool = True):
    """Loss and gradients through the multislice model: (loss, g_object [S, H, W], g_probe, g_pos)."""
    nz = _NOISE[noise] if isinstance(noise, str) else int(noise)
    d = _ms_dims(obj, probe, pos, ms)
    _need(meas, "meas", torch.float32, (d.J, d.N, d.N), device=obj.device)
    B = max(1, min(int(batch), max(d.J, 1)))
    gO, gP = torch.zeros_like(obj), torch.zeros_like(probe)
    gr = torch.zeros((d.J, 2), dtype=torch.float32, device=obj.device) if positions_grad else None
    loss = torch.zeros((), dtype=torch.float64, device=obj.device)
    ws = _ms_workspace(d, ms, B, obj.device)
    _check(lib().ptycho_adjoint_ms(ctypes.byref(d), ctypes.byref(ms), _ptr(obj), _ptr(probe), _ptr(pos), _ptr(meas),
                                   nz, float(eps), B, _ptr(gO), _ptr(gP), _ptr(gr),
                                   _ptr(loss) if nz != VJP else _P(0), _P(ws.ptr), ws.nbytes, _stream()),
           "ptycho_adjoint_ms")
    _finish(ws, "ptycho_adjoint_ms", check)
    return (None if nz == VJP else loss), gO, gP, gr


def lsqml_epoch_ms(obj, probe, pos, meas, order, ms: Multislice, opts: LsqmlOpts | None = None, *,
                   want_alpha: bool = False, check: bool = True, **kw):
    """One LSQML epoch with a multislice object (slices [S, H, W]), updating
    ``obj`` and ``probe`` in place. Returns (loss, alpha): alpha is a float64
    [J, 2] device tensor (alpha_O shared by the slices, alpha_P) or None."""
    if opts is None:
        opts = make_opts(**kw)
    d = _ms_dims(obj, probe, pos, ms)
    _need(meas, "meas", torch.float32, (d.J, d.N, d.N), device=obj.device)
    if order is not None:
        _need(order, "order", torch.int32, (d.J,), device=obj.device)
    need = lib().ptycho_workspace_bytes_lsqml_ms(ctypes.byref(d), ctypes.byref(ms), ctypes.byref(opts))
    if need == 0:
        raise PtychoError(6, "workspace_bytes_lsqml_ms")
    key = (str(obj.device), "lsqml_ms")
    ws = _ws_cache.get(key)
    if ws is None or ws.nbytes < need:
        ws = Workspace(need, obj.device)
        _ws_cache[key] = ws
    loss = torch.zeros((), dtype=torch.float64, device=obj.device)
    alpha = torch.zeros((d.J, 2), dtype=torch.float64, device=obj.device) if want_alpha else None
    _check(lib().ptycho_lsqml_epoch_ms(ctypes.byref(d), ctypes.byref(ms), _ptr(obj), _ptr(probe), _ptr(pos),
                                       _ptr(meas), _ptr(order), ctypes.byref(opts), _ptr(loss), _ptr(alpha),
                                       _P(ws.ptr), ws.nbytes, _stream()), "ptycho_lsqml_epoch_ms")
    _finish(ws, "ptycho_lsqml_epoch_ms", check)
    return loss, alpha
