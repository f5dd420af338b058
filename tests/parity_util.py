"""Helpers shared by the GPU parity tests and the smoke run: seeded problems
(inputs from paper_2510_20929_gb300.synth, measured data from the FP64 oracle)
and error metrics."""
import json
import math
import os

import numpy as np

from oracle import ptycho_oracle as orc
from paper_2510_20929_gb300 import synth


def rel(a, b):
    """Norm-wise relative error ||a - b|| / ||b||."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


def elem(a, b, axis=None):
    """Element-wise relative error max|a - b| / max|b|.

    With ``axis`` every slice along that axis is measured against its own
    maximum and the worst slice is returned: axis 0 of a probe [M, N, N] gives
    the worst mode, axis 1 of step sizes [J, 2] the worst of alpha_O and
    alpha_P (each over all positions), so that one wrong mode plane or one
    wrong position shows even when the norm of the whole array hides it.
    """
    a = np.asarray(a)
    b = np.asarray(b)
    if axis is None:
        mb = float(np.max(np.abs(b))) if b.size else 0.0
        return float(np.max(np.abs(a - b)) / (mb if mb > 0 else 1.0)) if b.size else 0.0
    return max((elem(np.take(a, i, axis=axis), np.take(b, i, axis=axis)) for i in range(b.shape[axis])),
               default=0.0)


# FP32 tolerances against the FP64 oracle (as err() measures them). A
# radix-16x8 FP32 FFT of length 128 has an rms relative error near
# u log2(N^2) ~ 1e-6 (u = 6e-8): forward intensities are held to 1e-5. The
# gradient factor (1 - rho) loses up to a decade to cancellation where the
# prediction already fits the data, and an epoch compounds a few minibatches
# of that through the preconditioned update: gradients and epoch outputs are
# held to 3e-5 (measured at most 1.5e-5 norm-wise, 3e-5 element-wise). These
# bars assume a well-conditioned problem; see full_epoch_bar() for the case
# where the data term itself amplifies rounding.
TOL_FWD = 1e-5
TOL_GRAD = 3e-5
TOL_EPOCH = 3e-5

# The largest element-wise error admitted per unit of norm-wise tolerance. For n
# independent rounding errors of rms s the largest is near s sqrt(2 ln n)
# (4.3 for n = 1e4, 5.3 for n = 1e6), and max|b| is at least the rms of b, so
# an element-wise bar of 5x the norm-wise one passes rounding noise while a
# localised mistake (one wrong column, mode plane or position) exceeds it.
ELEM_FACTOR = 5.0

_LOG = []


def err(a, b, axis=None, label=None):
    """max(norm-wise error, element-wise error / ELEM_FACTOR): below a tolerance
    t means ||a - b|| < t ||b|| and max|a - b| < 5 t max|b| (per slice of
    ``axis``). Both parts are recorded for the parity log."""
    n, e = rel(a, b), elem(a, b, axis)
    _LOG.append({"label": label, "norm": n, "elem": e})
    return max(n, e / ELEM_FACTOR)


def write_log(path, test_id):
    """Appends the errors recorded since the last call, tagged with the test id."""
    global _LOG
    if path and _LOG:
        with open(path, "a") as f:
            for r in _LOG:
                f.write(json.dumps({"test": test_id, **r}) + "\n")
    _LOG = []


def problem(N=16, M=2, H=40, W=44, J=12, seed=7, step=4.0, counts=2e4, perturb=0.15, noisy=True):
    """Truth, a perturbed estimate, and Poisson-noised intensities (oracle forward)."""
    w = synth.workload_small(N=N, M=M, H=H, W=W, J=J, seed=seed, step=step)
    O_true, P, pos = w["object"], w["probe"], w["pos"]
    I0 = orc.forward(O_true, P, pos)
    scale = counts / I0.sum(axis=(1, 2)).mean()
    P = P * math.sqrt(scale)
    I_true = I0 * scale
    I_m = synth.poisson_counts(I_true, seed + 11) if noisy else I_true
    g = np.random.default_rng(seed + 5)
    O = O_true * (1 + perturb * (g.standard_normal(O_true.shape) + 1j * g.standard_normal(O_true.shape)))
    return dict(O_true=O_true, O=O, P=P, pos=pos, I_m=I_m, I_true=I_true)


def to_dev(x, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype).cuda().contiguous()


def f32pos(pos):
    """Positions as the float32 values both sides see."""
    return np.asarray(pos, np.float32).astype(np.float64)


def c64(x):
    """Round a complex array to complex64 and back (the inputs both sides see)."""
    return np.asarray(x, np.complex64).astype(np.complex128)


def opr_problem(N=16, K=3, M=2, H=40, W=44, J=12, seed=7, step=4.0, counts=2e4, perturb=0.15, w_perturb=0.05,
                noisy=True):
    """Relaxed-probe problem: K eigenmodes and M - 1 shared modes (Hermite-Gaussian
    modes of one probe), true weights drawn from N(1, 0.1), Poisson-noised
    intensities from the oracle's relaxed forward model, and a start with a
    perturbed object and perturbed weights."""
    w = synth.workload_small(N=N, M=K + M - 1, H=H, W=W, J=J, seed=seed, step=step)
    O_true, modes, pos = w["object"], w["probe"], w["pos"]
    if K + M - 1 == 1:
        modes = modes[None] if modes.ndim == 2 else modes
    g = np.random.default_rng(seed + 21)
    w_true = 1.0 + 0.1 * g.standard_normal((J, K))
    U, P_rest = modes[:K], (modes[K:] if M > 1 else None)
    I0 = orc.forward_opr(O_true, U, w_true, P_rest, pos)
    s = math.sqrt(counts / I0.sum(axis=(1, 2)).mean())
    U = U * s
    P_rest = P_rest * s if P_rest is not None else None
    I_true = I0 * s * s
    I_m = synth.poisson_counts(I_true, seed + 11) if noisy else I_true
    O = O_true * (1 + perturb * (g.standard_normal(O_true.shape) + 1j * g.standard_normal(O_true.shape)))
    w0 = w_true + w_perturb * g.standard_normal(w_true.shape)
    return dict(O_true=O_true, O=O, U=U, w=w0, w_true=w_true, P_rest=P_rest, pos=pos, I_m=I_m)
