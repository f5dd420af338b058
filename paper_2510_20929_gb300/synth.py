"""Seeded synthetic inputs shaped like the paper's ptychography workloads.

This module generates inputs only: objects, probe modes, scan positions, batch
orders and Poisson counts. It holds none of the reconstruction arithmetic
(no patch extraction, no propagation, no data term), so that the CPU oracle
and the CUDA library can both be fed from it without sharing method code.
Measured intensities are made by the caller: it propagates the true object
with its own forward model and passes the noiseless intensities to
:func:`poisson_counts`.

Recipes (all float64 numpy, seeded with ``numpy.random.default_rng``):

* object: amplitude U[0.8, 1]; phase = white noise smoothed by a Gaussian of
  ``phase_sigma`` px (periodic boundary), rescaled to +-``phase_max`` rad.
* single-mode probe: Gaussian amplitude exp(-rho^2 / (2 sigma^2)) times the
  quadratic phase exp(i q rho^2), rho measured from the window centre N/2.
* multi-mode probe: Hermite-Gaussian modes H_m(sqrt2 y/w) H_n(sqrt2 x/w)
  exp(-rho^2/w^2) with the same quadratic phase, orthonormalised by
  Gram-Schmidt and scaled to the requested power fractions.
* positions: a jittered raster, or a Fermat spiral r_n = c sqrt(n),
  theta_n = n * 137.508 deg, both given as probe centres (y, x) in object px.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN_ANGLE_DEG = 137.508


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def make_object(H: int, W: int, seed: int, amp_lo: float = 0.8, amp_hi: float = 1.0,
                phase_sigma: float = 3.0, phase_max: float = 0.5,
                amp_sigma: float | None = None) -> np.ndarray:
    """Complex [H, W] object: U[amp_lo, amp_hi] amplitude, smoothed random phase.

    With ``amp_sigma`` the amplitude is smoothed white noise mapped onto
    [amp_lo, amp_hi] instead of independent uniform draws.
    """
    from scipy.ndimage import gaussian_filter

    g = rng(seed)
    amp = g.uniform(amp_lo, amp_hi, size=(H, W))
    if amp_sigma is not None:
        a = gaussian_filter(g.standard_normal((H, W)), sigma=amp_sigma, mode="wrap")
        amp = amp_lo + (amp_hi - amp_lo) * (a - a.min()) / (a.max() - a.min())
    noise = g.standard_normal((H, W))
    ph = gaussian_filter(noise, sigma=phase_sigma, mode="wrap")
    ph = ph * (phase_max / np.max(np.abs(ph)))
    return amp * np.exp(1j * ph)


def _window_coords(N: int):
    a = np.arange(N, dtype=np.float64) - N / 2.0
    return np.meshgrid(a, a, indexing="ij")


def gaussian_probe(N: int, sigma: float = 10.0, quad_phase: float = 0.01) -> np.ndarray:
    """Single-mode probe [1, N, N]: Gaussian amplitude with a quadratic phase."""
    y, x = _window_coords(N)
    rho2 = y * y + x * x
    return (np.exp(-rho2 / (2.0 * sigma * sigma)) * np.exp(1j * quad_phase * rho2))[None]


def _hermite(n: int, t: np.ndarray) -> np.ndarray:
    """Physicists' Hermite polynomial H_n by the three-term recurrence."""
    h0 = np.ones_like(t)
    if n == 0:
        return h0
    h1 = 2.0 * t
    for k in range(1, n):
        h0, h1 = h1, 2.0 * t * h1 - 2.0 * k * h0
    return h1


HG_ORDERS = [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (0, 2), (2, 1), (1, 2),
             (3, 0), (0, 3), (2, 2), (3, 1), (1, 3), (4, 0), (0, 4), (3, 2)]


def orthonormalise(modes: np.ndarray) -> np.ndarray:
    """Modified Gram-Schmidt over the flattened modes (float64/complex128)."""
    M = modes.shape[0]
    out = np.array(modes, dtype=np.complex128, copy=True).reshape(M, -1)
    for k in range(M):
        for i in range(k):
            out[k] -= np.vdot(out[i], out[k]) * out[i]
        out[k] /= np.linalg.norm(out[k])
    return out.reshape(modes.shape)


def hg_probe(N: int, powers, waist: float = 25.0, quad_phase: float = 0.01,
             total_power: float | None = None) -> np.ndarray:
    """Incoherent probe [M, N, N] of Hermite-Gaussian modes with power fractions ``powers``."""
    powers = np.asarray(powers, np.float64)
    powers = powers / powers.sum()
    y, x = _window_coords(N)
    rho2 = y * y + x * x
    s = math.sqrt(2.0) / waist
    modes = []
    for k in range(len(powers)):
        m, n = HG_ORDERS[k]
        modes.append(_hermite(m, s * y) * _hermite(n, s * x) * np.exp(-rho2 / waist ** 2)
                     * np.exp(1j * quad_phase * rho2))
    modes = orthonormalise(np.stack(modes))
    if total_power is None:
        total_power = math.pi * waist * waist / 2.0
    return modes * np.sqrt(powers * total_power)[:, None, None]


def raster_positions(ny: int, nx: int, step: float, center, jitter: float, seed: int) -> np.ndarray:
    """Jittered raster of probe centres [ny*nx, 2] (y, x), centred on ``center``."""
    g = rng(seed)
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    y = center[0] + (iy.ravel() - (ny - 1) / 2.0) * step
    x = center[1] + (ix.ravel() - (nx - 1) / 2.0) * step
    pos = np.stack([y, x], axis=1)
    pos += g.uniform(-jitter, jitter, size=pos.shape)
    return pos


def fermat_spiral(J: int, c: float, center) -> np.ndarray:
    """Fermat spiral of probe centres [J, 2] (y, x): r_n = c sqrt(n), theta_n = n * golden angle."""
    n = np.arange(J, dtype=np.float64)
    r = c * np.sqrt(n)
    th = np.deg2rad(GOLDEN_ANGLE_DEG) * n
    return np.stack([center[0] + r * np.sin(th), center[1] + r * np.cos(th)], axis=1)


def random_order(J: int, seed: int) -> np.ndarray:
    """Random minibatch order (a permutation of 0..J-1), int32."""
    return rng(seed).permutation(J).astype(np.int32)


def poisson_counts(I_true: np.ndarray, seed: int) -> np.ndarray:
    """Poisson-sampled counts with mean ``I_true`` (float64 array of non-negative means)."""
    return rng(seed).poisson(np.maximum(I_true, 0.0)).astype(np.float64)


def count_scale(total_intensity: float, total_counts: float) -> float:
    """Factor that maps a total predicted intensity onto ``total_counts`` detector counts."""
    return float(total_counts) / float(total_intensity)


# ---------------------------------------------------------------------------
# Workloads (probe, true object, positions) for the paper-shaped configurations.
# ---------------------------------------------------------------------------
def workload_raster64(seed: int = 1001):
    """Plain LSQML case: probe 64^2 (sigma 10 px, 0.01 rad/px^2), object 256^2,
    100 positions on a 10 x 10 raster with 16 px steps and +-0.5 px jitter."""
    H = W = 256
    N = 64
    obj = make_object(H, W, seed)
    probe = gaussian_probe(N, sigma=10.0, quad_phase=0.01)
    pos = raster_positions(10, 10, 16.0, (H / 2.0, W / 2.0), 0.5, seed + 7)
    return dict(name="raster64", H=H, W=W, N=N, M=1, J=100, batch=100,
                object=obj, probe=probe, pos=pos, total_counts=1e6, counts_per="all")


def workload_spiral128(seed: int = 1002, J: int = 4096):
    """Batched LSQML case: 5 Hermite-Gaussian modes (60/20/10/6/4 %), probe 128^2,
    object 1024^2, 4096 Fermat-spiral positions (c = 6.9 px), batch 256."""
    H = W = 1024
    N = 128
    obj = make_object(H, W, seed)
    probe = hg_probe(N, [0.60, 0.20, 0.10, 0.06, 0.04], waist=25.0, quad_phase=0.01)
    pos = fermat_spiral(J, 6.9, (H / 2.0, W / 2.0))
    return dict(name="spiral128", H=H, W=W, N=N, M=5, J=J, batch=256,
                object=obj, probe=probe, pos=pos, total_counts=1e6, counts_per="pattern")


def workload_spiral256(seed: int = 1003, J: int = 10000, pos_error: float = 1.5):
    """Differentiable case: 8 Hermite-Gaussian modes (orders up to 3; power
    halving per mode), probe 256^2, object 2048^2, 10,000 Fermat-spiral
    positions (c = 8.85 px), initial positions = truth + N(0, pos_error px)."""
    H = W = 2048
    N = 256
    obj = make_object(H, W, seed)
    powers = [0.5 ** k for k in range(8)]
    probe = hg_probe(N, powers, waist=40.0, quad_phase=0.005)
    pos = fermat_spiral(J, 8.85, (H / 2.0, W / 2.0))
    pos0 = pos + rng(seed + 1).normal(0.0, pos_error, size=pos.shape)
    return dict(name="spiral256", H=H, W=W, N=N, M=8, J=J, batch=256, object=obj, probe=probe, pos=pos,
                pos_init=pos0, total_counts=1e6, counts_per="pattern")


def workload_multislice256(seed: int = 1004, J: int = 8000, S: int = 4):
    """Multislice case: S slices of 2048^2 (each with the object recipe, the
    phase range divided among the slices), slice spacing 2 um, wavelength
    0.1 nm, pixel 10 nm; probe 256^2 with 4 Hermite-Gaussian modes (power
    halving per mode, waist 40 px); 8000 Fermat-spiral positions (c = 9.9 px);
    minibatch 512."""
    H = W = 2048
    N = 256
    slices = np.stack([make_object(H, W, seed * 10 + s, amp_lo=0.8 ** (1.0 / S), phase_max=0.5 / S)
                       for s in range(S)])
    probe = hg_probe(N, [0.5 ** k for k in range(4)], waist=40.0, quad_phase=0.005)
    pos = fermat_spiral(J, 9.9, (H / 2.0, W / 2.0))
    return dict(name="multislice256", H=H, W=W, N=N, M=4, S=S, J=J, batch=512, slices=slices, probe=probe,
                pos=pos, dz=2e-6, wavelength=0.1e-9, pixel_size=10e-9, total_counts=1e6, counts_per="pattern")


def workload_small(N: int = 16, M: int = 2, H: int = 40, W: int = 44, J: int = 12,
                   seed: int = 7, step: float = 4.0):
    """Small seeded problem for parity tests: raster positions with sub-pixel jitter."""
    obj = make_object(H, W, seed, phase_sigma=1.5)
    if M == 1:
        probe = gaussian_probe(N, sigma=N / 6.0, quad_phase=0.02)
    else:
        probe = hg_probe(N, np.linspace(1.0, 0.3, M), waist=N / 5.0, quad_phase=0.02)
    ny = int(math.ceil(math.sqrt(J)))
    nx = int(math.ceil(J / ny))
    pos = raster_positions(ny, nx, step, (H / 2.0, W / 2.0), 0.45, seed + 3)[:J]
    return dict(name=f"small{N}", H=H, W=W, N=N, M=M, J=J, batch=J,
                object=obj, probe=probe, pos=pos)


def workload_uneven(n: int = 16, seed: int = 1005, N_choices=(64, 128, 192, 256), J_range=(500, 20000),
                    counts_range=(1e5, 1e7), opr_K: int = 0):
    """Independent reconstructions of uneven size for batched serving: per
    reconstruction a window N drawn from ``N_choices``, J ~ U[J_range], a
    Gaussian probe (1/e^2 diameter D = 0.4 N), a Fermat spiral with spacing
    0.6 D (about 40% overlap), an object of side 2 (c sqrt(J) + N/2 + 2)
    rounded up to a multiple of 32, and total counts log-uniform in
    ``counts_range`` per pattern set. With ``opr_K`` > 0 each reconstruction
    also gets ``opr_K`` eigenmodes of its primary probe mode and per-position
    weights drawn from N(1, 0.1) (orthogonal probe relaxation)."""
    g = rng(seed)
    out = []
    for i in range(n):
        N = int(g.choice(N_choices))
        J = int(g.integers(J_range[0], J_range[1] + 1))
        D = 0.4 * N
        c = 0.6 * D / math.sqrt(math.pi)   # mean nearest-neighbour spacing of r = c sqrt(n) is c sqrt(pi)
        side = int(math.ceil(2 * (c * math.sqrt(J) + N / 2 + 2) / 32.0) * 32)
        obj = make_object(side, side, seed * 100 + i)
        probe = gaussian_probe(N, sigma=D / 4.0, quad_phase=0.2 / N)
        pos = fermat_spiral(J, c, (side / 2.0, side / 2.0))
        counts = float(np.exp(g.uniform(math.log(counts_range[0]), math.log(counts_range[1]))))
        out.append(dict(name=f"uneven{i}", H=side, W=side, N=N, M=1, J=J, batch=min(256, J), object=obj,
                        probe=probe, pos=pos, total_counts=counts, counts_per="all"))
        if opr_K:
            # relaxed primary mode: K Hermite-Gaussian eigenmodes (waist D/2,
            # power falling off from the fundamental) with weights N(1, 0.1)
            powers = [1.0] + [0.3 * 0.6 ** k for k in range(opr_K - 1)]
            out[-1]["opr_U"] = hg_probe(N, powers, waist=D / 2.0, quad_phase=0.2 / N)
            out[-1]["opr_w"] = 1.0 + 0.1 * rng(seed * 1000 + 17 + i).standard_normal((J, opr_K))
    return out
