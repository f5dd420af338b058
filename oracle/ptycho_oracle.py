"""FP64 CPU oracle for the LSQML ptychography hot path (Pty-Chi, arXiv 2510.20929).

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import or call this
module: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it. It shares no code with the CUDA library; both sides only
share the seeded input generators, which hold none of the method's arithmetic.

Everything here is plain numpy in float64 / complex128, written to be read
against the paper, not to be fast:

* Forward model (Sec. 2.1; Eq. 4's F(o, p, Lambda); the exit wave psi = p * o
  named under Eq. 2): per scan position j the object patch o_j = S_j(O) is cut
  out at a sub-pixel position, multiplied by each incoherent probe mode P_k,
  propagated to the far field with a unitary 2-D DFT and the modes are summed
  incoherently, I_j = sum_k |F(P_k o_j)|^2.
* Gaussian data term (Eq. 1, amplitude MSE, unnormalised) and its gradient
  (Eq. 2, the conjugate probe times the exit-wave change), plus the Poisson
  negative log-likelihood.
* The LSQML reconstructor named in Sec. 2.2 (self-adaptive step sizes) with
  the illumination preconditioner of Sec. 1 / Sec. 4, one minibatch at a time
  (per-batch update, Sec. 2.2 third bullet for the non-compact sampler).

The paper does not print LSQML's update equations. The readings used here
(bilinear sub-pixel shift, unitary FFT without fftshift, probe-centre
positions, relative preconditioner regularisers, Tikhonov-regularised 2x2
step solve, alpha-weighted object scatter, mean-alpha probe step, the
Poisson exit-wave step) are the repository's documented readings of the
method; parity of the full iteration against Pty-Chi itself is unpinned
(no code or printed numbers exist to pin it to). Every other function is
pinned by the CPU tests (brute-force DFT, Parseval, adjoint dot products,
finite differences, closed-form special cases, brute-force step search,
convergence on noiseless data).

Conventions
-----------
* Object O: complex [H, W]; probe P: complex [M, N, N]; positions pos:
  float [J, 2] in (y, x) order, the probe centre in object pixels.
* Tile origin t = floor(r - N/2), fraction f = r - N/2 - t in [0, 1); the
  bilinear tile spans (N+1) x (N+1) object pixels starting at t, which must
  lie inside the object.
* F is the unitary ("ortho") 2-D DFT with DC at index [0, 0]; measured
  intensities are stored in that order.
* Gradients follow the complex convention grad = 2 dL/dz* (PyTorch's), so a
  real perturbation changes the loss by Re<grad, dz>.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GAUSSIAN = 0
POISSON = 1


# ---------------------------------------------------------------------------
# Unitary 2-D DFT (the far-field propagator of the forward model, Sec. 2.1).
# ---------------------------------------------------------------------------
def dft2(x: np.ndarray) -> np.ndarray:
    """Unitary 2-D DFT over the last two axes, DC at [0, 0] (no fftshift)."""
    return np.fft.fft2(np.asarray(x, dtype=np.complex128), norm="ortho")


def idft2(X: np.ndarray) -> np.ndarray:
    """Inverse of :func:`dft2` (its adjoint, since the transform is unitary)."""
    return np.fft.ifft2(np.asarray(X, dtype=np.complex128), norm="ortho")


# ---------------------------------------------------------------------------
# Sub-pixel patch extraction S_j and its adjoint S_j^T (object class routine,
# Sec. 2.1: "object patch extraction/update").
# ---------------------------------------------------------------------------
def tile_origin(r, N: int):
    """Integer tile origin t = floor(r - N/2) and fraction f = r - N/2 - t."""
    r = np.asarray(r, dtype=np.float64)
    s = r - N / 2.0
    t = np.floor(s)
    return t.astype(np.int64), s - t


def in_bounds(r, N: int, H: int, W: int) -> bool:
    """True when the (N+1)^2 bilinear tile of position r lies inside [H, W]."""
    t, _ = tile_origin(r, N)
    return bool(t[0] >= 0 and t[1] >= 0 and t[0] + N + 1 <= H and t[1] + N + 1 <= W)


def _corners(O: np.ndarray, t, N: int):
    ty, tx = int(t[0]), int(t[1])
    O00 = O[ty:ty + N, tx:tx + N]
    O01 = O[ty:ty + N, tx + 1:tx + N + 1]
    O10 = O[ty + 1:ty + N + 1, tx:tx + N]
    O11 = O[ty + 1:ty + N + 1, tx + 1:tx + N + 1]
    return O00, O01, O10, O11


def extract(O: np.ndarray, r, N: int) -> np.ndarray:
    """o_j = S_j(O): bilinear interpolation of O on the N x N grid t + f + (a, b)."""
    t, f = tile_origin(r, N)
    if not in_bounds(r, N, O.shape[0], O.shape[1]):
        raise ValueError("position outside the object")
    fy, fx = f
    O00, O01, O10, O11 = _corners(O, t, N)
    return ((1 - fy) * (1 - fx) * O00 + (1 - fy) * fx * O01
            + fy * (1 - fx) * O10 + fy * fx * O11)


def extract_dr(O: np.ndarray, r, N: int):
    """Derivatives (d o_j / d y, d o_j / d x) of the bilinear patch w.r.t. the position."""
    t, f = tile_origin(r, N)
    fy, fx = f
    O00, O01, O10, O11 = _corners(O, t, N)
    d_dy = (1 - fx) * (O10 - O00) + fx * (O11 - O01)
    d_dx = (1 - fy) * (O01 - O00) + fy * (O11 - O10)
    return d_dy, d_dx


def scatter(patch: np.ndarray, r, H: int, W: int) -> np.ndarray:
    """S_j^T: adds the N x N patch back into an H x W canvas with the bilinear weights."""
    N = patch.shape[-1]
    t, f = tile_origin(r, N)
    if not in_bounds(r, N, H, W):
        raise ValueError("position outside the object")
    fy, fx = f
    ty, tx = int(t[0]), int(t[1])
    out = np.zeros((H, W), dtype=np.result_type(patch.dtype, np.float64))
    out[ty:ty + N, tx:tx + N] += (1 - fy) * (1 - fx) * patch
    out[ty:ty + N, tx + 1:tx + N + 1] += (1 - fy) * fx * patch
    out[ty + 1:ty + N + 1, tx:tx + N] += fy * (1 - fx) * patch
    out[ty + 1:ty + N + 1, tx + 1:tx + N + 1] += fy * fx * patch
    return out


# ---------------------------------------------------------------------------
# Forward model: I_j = sum_k |F(P_k * S_j(O))|^2 (Sec. 2.1, Eq. 4).
# ---------------------------------------------------------------------------
def exit_waves(O, P, r):
    """psi_jk = P_k * o_j for one position (array [M, N, N])."""
    N = P.shape[-1]
    return P * extract(O, r, N)[None]


def forward(O: np.ndarray, P: np.ndarray, pos: np.ndarray) -> np.ndarray:
    """Predicted far-field intensities [J, N, N], DC at [0, 0]."""
    J, N = pos.shape[0], P.shape[-1]
    out = np.empty((J, N, N), dtype=np.float64)
    for j in range(J):
        Psi = dft2(exit_waves(O, P, pos[j]))
        out[j] = np.sum(np.abs(Psi) ** 2, axis=0)
    return out


# ---------------------------------------------------------------------------
# Data terms. Gaussian = Eq. 1 without its 1/(BHW) prefactor, with eps inside
# the square root so that its derivative is exact; Poisson = negative
# log-likelihood up to a data-only constant.
# ---------------------------------------------------------------------------
def pattern_loss(I, I_m, noise: int, eps: float) -> float:
    I = np.asarray(I, np.float64)
    I_m = np.asarray(I_m, np.float64)
    if noise == GAUSSIAN:
        return float(np.sum((np.sqrt(I + eps) - np.sqrt(I_m)) ** 2))
    if noise == POISSON:
        return float(np.sum(I - I_m * np.log(I + eps)))
    raise ValueError("noise model")


def dloss_dI(I, I_m, noise: int, eps: float) -> np.ndarray:
    """dL/dI per detector pixel for the two data terms above."""
    if noise == GAUSSIAN:
        return 1.0 - np.sqrt(I_m) / np.sqrt(I + eps)
    if noise == POISSON:
        return 1.0 - I_m / (I + eps)
    raise ValueError("noise model")


def modulus_ratio(I, I_m, noise: int, eps: float) -> np.ndarray:
    """rho such that the projected far field is Psi' = rho * Psi for every mode.

    Gaussian: the magnitude is replaced by the measured amplitude (the psi' of
    Eq. 2). Poisson: half a gradient step on the likelihood, rho = 1 + (I_m/I - 1)/2.
    """
    if noise == GAUSSIAN:
        return np.sqrt(I_m) / np.sqrt(I + eps)
    if noise == POISSON:
        return 1.0 + 0.5 * (I_m / (I + eps) - 1.0)
    raise ValueError("noise model")


# ---------------------------------------------------------------------------
# Gradients (Eq. 2 generalised to probe and positions; AD reconstructor, Sec. 2.2).
# ---------------------------------------------------------------------------
def vjp(O, P, pos, G):
    """Gradients of L through the forward model given G = dL/dI [J, N, N].

    grad_Psi_k = 2 G Psi_k; grad_psi_k = F^H grad_Psi_k;
    grad_o_j = sum_k conj(P_k) grad_psi_k; grad_O = sum_j S_j^T grad_o_j;
    grad_P_k = sum_j conj(o_j) grad_psi_jk; dL/dr_j = Re sum conj(grad_o_j) d o_j/d r.
    """
    H, W = O.shape
    M, N = P.shape[0], P.shape[-1]
    J = pos.shape[0]
    gO = np.zeros((H, W), np.complex128)
    gP = np.zeros((M, N, N), np.complex128)
    gr = np.zeros((J, 2), np.float64)
    for j in range(J):
        o = extract(O, pos[j], N)
        Psi = dft2(P * o[None])
        gpsi = idft2(2.0 * G[j][None] * Psi)
        go = np.sum(np.conj(P) * gpsi, axis=0)
        gO += scatter(go, pos[j], H, W)
        gP += np.conj(o)[None] * gpsi
        d_dy, d_dx = extract_dr(O, pos[j], N)
        gr[j, 0] = np.real(np.sum(np.conj(go) * d_dy))
        gr[j, 1] = np.real(np.sum(np.conj(go) * d_dx))
    return gO, gP, gr


def loss_and_gradients(O, P, pos, I_m, noise: int = GAUSSIAN, eps: float = 0.0):
    """Total loss sum_j L_j and its gradients w.r.t. object, probe modes and positions."""
    I = forward(O, P, pos)
    loss = sum(pattern_loss(I[j], I_m[j], noise, eps) for j in range(pos.shape[0]))
    G = dloss_dI(I, I_m, noise, eps)
    gO, gP, gr = vjp(O, P, pos, G)
    return loss, gO, gP, gr


# ---------------------------------------------------------------------------
# LSQML (Sec. 2.2; object preconditioner Sec. 1 and Sec. 4).
# ---------------------------------------------------------------------------
@dataclass
class LsqmlOptions:
    noise: int = GAUSSIAN
    batch: int = 256
    delta_o: float = 1e-3      # relative: delta_O = delta_o * max(illumination)
    delta_p: float = 1e-3      # relative: delta_P = delta_p * max(sum_j |o_j|^2)
    lam: float = 1e-6          # 2x2 Tikhonov term, relative to trace(A)/2
    eps: float = 0.0           # added to I_pred in the data term
    update_object: bool = True
    update_probe: bool = True
    update_positions: bool = False   # least-squares position correction per minibatch
    pos_step: float = 1.0            # relaxation of the position step
    pos_max_shift: float = 1.0       # per-minibatch clamp of each position component (px)
    object_per_epoch: bool = False   # accumulate the object update over the epoch, apply once


def step_solve(A11, A12, A22, b1, b2, lam):
    """Per-position step sizes (alpha_O, alpha_P) from the 2x2 normal equations.

    A is regularised by lam * trace(A)/2 on the diagonal. If the determinant is
    not positive, each step falls back to its own 1x1 solve (zero when the
    curvature is zero).
    """
    tr = 0.5 * (A11 + A22)
    a11 = A11 + lam * tr
    a22 = A22 + lam * tr
    det = a11 * a22 - A12 * A12
    if det > 0.0:
        return (a22 * b1 - A12 * b2) / det, (a11 * b2 - A12 * b1) / det
    return (b1 / a11 if a11 > 0 else 0.0), (b2 / a22 if a22 > 0 else 0.0)


POS_MARGIN = 1.0 / 64.0   # corrected positions stay this far inside the bounds rule's upper limit


def position_step(O, P, r, g, lam):
    """Least-squares shift of one scan position (position correction, Sec. 1 / Sec. 2.1).

    A shift dr moves the exit waves by P_k (d o / d r) dr; the step is
    argmin_dr sum_k ||chi_k - P_k (d_y dr_y + d_x dr_x)||^2 with the patch
    derivatives d = d o_j / d r of the bilinear extraction. Its normal
    equations sum the modes into Sp = sum_k |P_k|^2 and g = sum_k conj(P_k) chi_k:
      A = sum_p Sp [|d_y|^2, Re(conj(d_y) d_x); ., |d_x|^2],
      b = sum_p [Re(conj(d_y) g), Re(conj(d_x) g)],
    solved like the step sizes (damping lam tr(A)/2, 1x1 fallbacks).
    """
    N = P.shape[-1]
    d_y, d_x = extract_dr(O, r, N)
    Sp = np.sum(np.abs(P) ** 2, axis=0)
    A11 = float(np.sum(Sp * np.abs(d_y) ** 2))
    A12 = float(np.sum(Sp * np.real(np.conj(d_y) * d_x)))
    A22 = float(np.sum(Sp * np.abs(d_x) ** 2))
    b1 = float(np.real(np.sum(np.conj(d_y) * g)))
    b2 = float(np.real(np.sum(np.conj(d_x) * g)))
    return np.array(step_solve(A11, A12, A22, b1, b2, lam))


def corrected_position(r, dr, opts: LsqmlOptions, N: int, H: int, W: int):
    """r + pos_step * clip(dr, +-pos_max_shift), kept inside the bounds rule."""
    m = opts.pos_max_shift
    new = np.asarray(r, np.float64) + opts.pos_step * np.clip(dr, -m, m)
    return np.array([np.clip(new[0], N / 2.0, H - N / 2.0 - POS_MARGIN),
                     np.clip(new[1], N / 2.0, W - N / 2.0 - POS_MARGIN)])


def lsqml_batch(O, P, pos, I_m, idx, opts: LsqmlOptions, record: dict | None = None):
    """One LSQML minibatch over the positions ``idx``; returns (O, P, loss, alpha).

    Steps, per position j of the batch and modes k:
      o_j = S_j(O); psi_jk = P_k o_j; Psi_jk = F psi_jk; I_j = sum_k |Psi_jk|^2;
      chi_jk = F^{-1}[(rho_j - 1) Psi_jk] (= F^{-1} Psi'_jk - psi_jk);
      g_j = sum_k conj(P_k) chi_jk;  h_jk = conj(o_j) chi_jk.
    Batch accumulators and preconditioned directions:
      dO_acc = sum_j S_j^T g_j;  illum = sum_j S_j^T sum_k |P_k|^2;
      dP_acc_k = sum_j h_jk;  Dp = sum_j |o_j|^2;
      dO_hat = dO_acc / (illum + delta_O);  dP_k = dP_acc_k / (Dp + delta_P).
    Step sizes: u_jk = S_j(dO_hat) P_k, v_jk = o_j dP_k; A and b are the normal
    equations of min ||chi_j - a_O u_j - a_P v_j||^2 summed over modes and pixels.
    Update: O += sum_j S_j^T(alpha_O,j g_j) / (illum + delta_O);
            P_k += mean_j(alpha_P,j) dP_k.
    """
    H, W = O.shape
    M, N = P.shape[0], P.shape[-1]
    idx = [int(i) for i in idx]
    B = len(idx)
    Sp = np.sum(np.abs(P) ** 2, axis=0)

    loss = 0.0
    o_all, chi_all, g_all = [], [], []
    dO_acc = np.zeros((H, W), np.complex128)
    illum = np.zeros((H, W), np.float64)
    dP_acc = np.zeros((M, N, N), np.complex128)
    Dp = np.zeros((N, N), np.float64)
    for j in idx:
        o = extract(O, pos[j], N)
        psi = P * o[None]
        Psi = dft2(psi)
        I = np.sum(np.abs(Psi) ** 2, axis=0)
        loss += pattern_loss(I, I_m[j], opts.noise, opts.eps)
        rho = modulus_ratio(I, I_m[j], opts.noise, opts.eps)
        chi = idft2((rho - 1.0)[None] * Psi)
        g = np.sum(np.conj(P) * chi, axis=0)
        dO_acc += scatter(g, pos[j], H, W)
        illum += scatter(Sp, pos[j], H, W)
        dP_acc += np.conj(o)[None] * chi
        Dp += np.abs(o) ** 2
        o_all.append(o)
        chi_all.append(chi)
        g_all.append(g)

    delta_O = opts.delta_o * float(np.max(illum))
    delta_P = opts.delta_p * float(np.max(Dp))
    dO_hat = dO_acc / (illum + delta_O)
    if not opts.update_object:
        dO_hat = np.zeros_like(dO_hat)
    if opts.update_probe:
        dP = dP_acc / (Dp + delta_P)[None]
    else:
        dP = np.zeros_like(dP_acc)

    alpha = np.zeros((B, 2), np.float64)
    for i, j in enumerate(idx):
        o, chi = o_all[i], chi_all[i]
        u = extract(dO_hat, pos[j], N)[None] * P
        v = o[None] * dP
        A11 = float(np.sum(np.abs(u) ** 2))
        A12 = float(np.real(np.sum(np.conj(u) * v)))
        A22 = float(np.sum(np.abs(v) ** 2))
        b1 = float(np.real(np.sum(np.conj(u) * chi)))
        b2 = float(np.real(np.sum(np.conj(v) * chi)))
        alpha[i] = step_solve(A11, A12, A22, b1, b2, opts.lam)

    O_new = O.copy()
    dO = np.zeros((H, W), np.complex128)
    if opts.update_object:
        upd = np.zeros((H, W), np.complex128)
        for i, j in enumerate(idx):
            upd += scatter(alpha[i, 0] * g_all[i], pos[j], H, W)
        dO = upd / (illum + delta_O)
        if not opts.object_per_epoch:
            O_new = O + dO
    P_new = P.copy()
    if opts.update_probe:
        P_new = P + float(np.mean(alpha[:, 1])) * dP
    pos_new = np.array(pos, np.float64, copy=True)
    if opts.update_positions:   # shifts from this minibatch's chi, at the object it started from
        for i, j in enumerate(idx):
            dr = position_step(O, P, pos[j], g_all[i], opts.lam)
            pos_new[j] = corrected_position(pos[j], dr, opts, N, H, W)

    if record is not None:
        record.update(dict(dO_acc=dO_acc, illum=illum, dP_acc=dP_acc, Dp=Dp,
                           delta_O=delta_O, delta_P=delta_P, dO_hat=dO_hat, dP=dP,
                           chi=np.stack(chi_all), g=np.stack(g_all), alpha=alpha, dO=dO, pos=pos_new))
    return O_new, P_new, loss, alpha


def lsqml_epoch(O, P, pos, I_m, order, opts: LsqmlOptions):
    """One epoch: minibatches of ``opts.batch`` positions taken from ``order`` in turn.

    Returns (O, P, loss, alpha); :func:`lsqml_epoch_state` also returns the
    corrected positions.
    """
    O, P, _, loss, alpha = lsqml_epoch_state(O, P, pos, I_m, order, opts)
    return O, P, loss, alpha


def lsqml_epoch_state(O, P, pos, I_m, order, opts: LsqmlOptions):
    """One epoch; returns (O, P, pos, loss, alpha).

    With ``opts.object_per_epoch`` (the mode LSQML takes with the compact
    sampler, Sec. 2.2) every minibatch sees the object the epoch started from;
    the minibatches' object updates are summed and applied once at the end.
    The probe and (with ``update_positions``) the positions change per minibatch.
    """
    O = np.asarray(O, np.complex128).copy()
    P = np.asarray(P, np.complex128).copy()
    pos = np.asarray(pos, np.float64).copy()
    order = np.asarray(order)
    J = order.shape[0]
    loss = 0.0
    alpha = np.zeros((pos.shape[0], 2), np.float64)
    dO_epoch = np.zeros_like(O)
    for b0 in range(0, J, opts.batch):
        idx = order[b0:b0 + opts.batch]
        rec = {}
        O, P, l, a = lsqml_batch(O, P, pos, I_m, idx, opts, rec)
        pos = rec["pos"]
        dO_epoch += rec["dO"]
        loss += l
        alpha[idx] = a
    if opts.object_per_epoch:
        O = O + dO_epoch
    return O, P, pos, loss, alpha


def align_global_phase(O, O_ref, mask=None):
    """Multiply O by the unit phase e^{i phi} minimising ||O e^{i phi} - O_ref|| on mask."""
    if mask is None:
        mask = np.ones(O.shape, bool)
    c = np.sum(np.conj(O[mask]) * O_ref[mask])
    return O * (c / abs(c)) if abs(c) > 0 else O


# ---------------------------------------------------------------------------
# Orthogonal probe relaxation (Sec. 2.1: scan-point-specific probes; Sec. 3.2).
# The primary probe mode of position j is sum_m w_jm U_m over K eigenmodes U
# with real weights w [J, K]; the other incoherent modes are shared.
# ---------------------------------------------------------------------------
def opr_primary(U, w_j):
    """Primary probe mode of one position: sum_m w_jm U_m."""
    return np.tensordot(np.asarray(w_j, np.float64), U, axes=(0, 0))


def opr_modes(U, w_j, P_rest):
    """All incoherent modes of one position: [sum_m w_jm U_m, P_rest...]."""
    P0 = opr_primary(U, w_j)[None]
    return np.concatenate([P0, P_rest], axis=0) if P_rest is not None and len(P_rest) else P0


def forward_opr(O, U, w, P_rest, pos):
    """Predicted intensities with position-dependent primary modes [J, N, N]."""
    J, N = pos.shape[0], U.shape[-1]
    out = np.empty((J, N, N), np.float64)
    for j in range(J):
        Psi = dft2(opr_modes(U, w[j], P_rest) * extract(O, pos[j], N)[None])
        out[j] = np.sum(np.abs(Psi) ** 2, axis=0)
    return out


def vjp_opr(O, U, w, P_rest, pos, G):
    """Gradients through the OPR forward model given G = dL/dI.

    With g_P0 = conj(o_j) grad_psi_j0: grad U_m = sum_j w_jm g_P0 and
    dL/dw_jm = Re<U_m, g_P0> (w real); the rest as in :func:`vjp`.
    """
    H, W = O.shape
    K, N = U.shape[0], U.shape[-1]
    J = pos.shape[0]
    gO = np.zeros((H, W), np.complex128)
    gU = np.zeros_like(U, dtype=np.complex128)
    gw = np.zeros((J, K), np.float64)
    gP = np.zeros_like(P_rest, dtype=np.complex128) if P_rest is not None else None
    gr = np.zeros((J, 2), np.float64)
    for j in range(J):
        o = extract(O, pos[j], N)
        Pj = opr_modes(U, w[j], P_rest)
        gpsi = idft2(2.0 * G[j][None] * dft2(Pj * o[None]))
        go = np.sum(np.conj(Pj) * gpsi, axis=0)
        gO += scatter(go, pos[j], H, W)
        gP0 = np.conj(o) * gpsi[0]
        gU += np.asarray(w[j], np.float64)[:, None, None] * gP0[None]
        gw[j] = np.real(np.sum(np.conj(U) * gP0[None], axis=(1, 2)))
        if gP is not None:
            gP += np.conj(o)[None] * gpsi[1:]
        d_dy, d_dx = extract_dr(O, pos[j], N)
        gr[j, 0] = np.real(np.sum(np.conj(go) * d_dy))
        gr[j, 1] = np.real(np.sum(np.conj(go) * d_dx))
    return gO, gU, gw, gP, gr


def loss_and_gradients_opr(O, U, w, P_rest, pos, I_m, noise=GAUSSIAN, eps=0.0):
    I = forward_opr(O, U, w, P_rest, pos)
    loss = sum(pattern_loss(I[j], I_m[j], noise, eps) for j in range(pos.shape[0]))
    return (loss,) + vjp_opr(O, U, w, P_rest, pos, dloss_dI(I, I_m, noise, eps))


@dataclass
class OprOptions:
    """Options of the LSQML minibatch with orthogonal probe relaxation."""
    update_weights: bool = True
    weight_step: float = 1.0      # relaxation of the per-position weight update


def weight_solve(A, b, lam):
    """Damped normal equations (A + lam (tr A / K) I) dw = b in FP64 (Cholesky).

    A singular (or non-positive) damped system gives dw = 0.
    """
    A = np.asarray(A, np.float64)
    K = A.shape[0]
    Ad = A + lam * (np.trace(A) / K) * np.eye(K)
    try:
        L = np.linalg.cholesky(Ad)
    except np.linalg.LinAlgError:
        return np.zeros(K)
    y = np.linalg.solve(L, np.asarray(b, np.float64))
    return np.linalg.solve(L.T, y)


def lsqml_batch_opr(O, U, w, P_rest, pos, I_m, idx, opts: LsqmlOptions, opr: OprOptions,
                    record: dict | None = None):
    """One LSQML minibatch with a relaxed primary probe mode (Sec. 2.1, OPR).

    Returns (O, U, w, P_rest, loss, alpha). Position j's modes are
    [P_j0, P_rest...] with P_j0 = sum_m w_jm U_m (U [K, N, N], w [J, K] real).
    The exit waves, chi, g_j = sum_k conj(P_jk) chi_jk, h_jk = conj(o_j) chi_jk,
    the object direction and the shared modes' directions are those of
    :func:`lsqml_batch` with the per-position primary mode, the illumination
    included. The eigenmodes take the weighted probe direction
      dU_m = (sum_j w_jm h_j0) / (D_m + delta_P),  D_m = sum_j w_jm^2 |o_j|^2,
    with delta_P = delta_p max(max Dp, max_m D_m); the primary-mode direction
    of position j is then dP_j0 = sum_m w_jm dU_m in the step-size system, and
    U_m += mean(alpha_P) dU_m with the shared modes. The weights of each
    position move by the least-squares fit of the primary mode's exit-wave
    change onto the eigenmodes' exit waves: min over real dw of
    ||chi_j0 - sum_m dw_m U_m o_j||^2 (normal equations A_mn = Re<U_m o_j, U_n o_j>,
    b_m = Re<U_m o_j, chi_j0>, damped by lam tr(A)/K), w_j += weight_step dw,
    taken with this batch's U and chi.
    """
    H, W = O.shape
    K, N = U.shape[0], U.shape[-1]
    Mr = 0 if P_rest is None else P_rest.shape[0]
    idx = [int(i) for i in idx]
    B = len(idx)
    Sp_rest = np.sum(np.abs(P_rest) ** 2, axis=0) if Mr else np.zeros((N, N))

    loss = 0.0
    o_all, chi_all, g_all = [], [], []
    dO_acc = np.zeros((H, W), np.complex128)
    illum = np.zeros((H, W), np.float64)
    dP_acc = np.zeros((Mr, N, N), np.complex128)
    dU_acc = np.zeros((K, N, N), np.complex128)
    Dp = np.zeros((N, N), np.float64)
    D = np.zeros((K, N, N), np.float64)
    for j in idx:
        o = extract(O, pos[j], N)
        Pj = opr_modes(U, w[j], P_rest)
        Psi = dft2(Pj * o[None])
        I = np.sum(np.abs(Psi) ** 2, axis=0)
        loss += pattern_loss(I, I_m[j], opts.noise, opts.eps)
        rho = modulus_ratio(I, I_m[j], opts.noise, opts.eps)
        chi = idft2((rho - 1.0)[None] * Psi)
        g = np.sum(np.conj(Pj) * chi, axis=0)
        dO_acc += scatter(g, pos[j], H, W)
        illum += scatter(Sp_rest + np.abs(Pj[0]) ** 2, pos[j], H, W)
        h = np.conj(o)[None] * chi
        dP_acc += h[1:]
        dU_acc += np.asarray(w[j], np.float64)[:, None, None] * h[0][None]
        Dp += np.abs(o) ** 2
        D += (np.asarray(w[j], np.float64) ** 2)[:, None, None] * (np.abs(o) ** 2)[None]
        o_all.append(o)
        chi_all.append(chi)
        g_all.append(g)

    delta_O = opts.delta_o * float(np.max(illum))
    delta_P = opts.delta_p * max(float(np.max(Dp)), float(np.max(D)))
    dO_hat = dO_acc / (illum + delta_O) if opts.update_object else np.zeros((H, W), np.complex128)
    if opts.update_probe:
        dP = dP_acc / (Dp + delta_P)[None]
        dU = dU_acc / (D + delta_P)
    else:
        dP, dU = np.zeros_like(dP_acc), np.zeros_like(dU_acc)

    alpha = np.zeros((B, 2), np.float64)
    dw = np.zeros((B, K), np.float64)
    for i, j in enumerate(idx):
        o, chi = o_all[i], chi_all[i]
        Pj = opr_modes(U, w[j], P_rest)
        dPj = np.concatenate([opr_primary(dU, w[j])[None], dP], axis=0)
        u = extract(dO_hat, pos[j], N)[None] * Pj
        v = o[None] * dPj
        A11 = float(np.sum(np.abs(u) ** 2))
        A12 = float(np.real(np.sum(np.conj(u) * v)))
        A22 = float(np.sum(np.abs(v) ** 2))
        b1 = float(np.real(np.sum(np.conj(u) * chi)))
        b2 = float(np.real(np.sum(np.conj(v) * chi)))
        alpha[i] = step_solve(A11, A12, A22, b1, b2, opts.lam)
        if opr.update_weights:
            E = U * o[None]                                   # eigenmode exit waves
            A = np.real(np.einsum("mxy,nxy->mn", np.conj(E), E))
            b = np.real(np.einsum("mxy,xy->m", np.conj(E), chi[0]))
            dw[i] = weight_solve(A, b, opts.lam)

    O_new = O.copy()
    if opts.update_object:
        upd = np.zeros((H, W), np.complex128)
        for i, j in enumerate(idx):
            upd += scatter(alpha[i, 0] * g_all[i], pos[j], H, W)
        O_new = O + upd / (illum + delta_O)
    U_new, P_new = U.copy(), (P_rest.copy() if Mr else P_rest)
    if opts.update_probe:
        a_p = float(np.mean(alpha[:, 1]))
        U_new = U + a_p * dU
        if Mr:
            P_new = P_rest + a_p * dP
    w_new = np.array(w, np.float64, copy=True)
    if opr.update_weights:
        for i, j in enumerate(idx):
            w_new[j] += opr.weight_step * dw[i]

    if record is not None:
        record.update(dict(dO_acc=dO_acc, illum=illum, dP_acc=dP_acc, dU_acc=dU_acc, Dp=Dp, D=D,
                           delta_O=delta_O, delta_P=delta_P, dU=dU, dP=dP, dw=dw,
                           chi=np.stack(chi_all), alpha=alpha))
    return O_new, U_new, w_new, P_new, loss, alpha


def lsqml_epoch_opr(O, U, w, P_rest, pos, I_m, order, opts: LsqmlOptions, opr: OprOptions):
    """One OPR epoch: minibatches of ``opts.batch`` positions taken from ``order`` in turn."""
    O = np.asarray(O, np.complex128).copy()
    U = np.asarray(U, np.complex128).copy()
    w = np.asarray(w, np.float64).copy()
    P_rest = None if P_rest is None else np.asarray(P_rest, np.complex128).copy()
    order = np.asarray(order)
    loss = 0.0
    alpha = np.zeros((pos.shape[0], 2), np.float64)
    for b0 in range(0, order.shape[0], opts.batch):
        idx = order[b0:b0 + opts.batch]
        O, U, w, P_rest, l, a = lsqml_batch_opr(O, U, w, P_rest, pos, I_m, idx, opts, opr)
        loss += l
        alpha[idx] = a
    return O, U, w, P_rest, loss, alpha


# ---------------------------------------------------------------------------
# Minibatch samplers (Sec. 2.1: random, uniform and compact batches).
# Index work, compared bit-exactly with the library; positions as float32.
# ---------------------------------------------------------------------------
SAMPLER_RANDOM, SAMPLER_UNIFORM, SAMPLER_COMPACT = 0, 1, 2
_MASK64 = (1 << 64) - 1


def splitmix64(state: int):
    """One SplitMix64 step (Steele, Lea and Flood 2014): returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & _MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return state, z ^ (z >> 31)


def _kd_split(pos32, idx, groups, cap, out):
    """Recursive spatial split of the index list ``idx`` into ``groups`` clusters."""
    n = len(idx)
    if groups <= 1 or n <= 1:
        out.append(list(idx))
        return
    ys, xs = pos32[idx, 0], pos32[idx, 1]
    axis = 0 if (ys.max() - ys.min()) >= (xs.max() - xs.min()) else 1
    idx = [idx[i] for i in np.argsort(pos32[idx, axis], kind="stable")]
    g1 = groups // 2
    g2 = groups - g1
    n1 = min(n, g1 * cap) if cap > 0 else (n * g1 + groups // 2) // groups
    _kd_split(pos32, idx[:n1], g1, cap, out)
    _kd_split(pos32, idx[n1:], g2, cap, out)


def sampler_order(pos, batch: int, kind: int, seed: int = 0) -> np.ndarray:
    """Batch order of the random, uniform or compact sampler (see the C header)."""
    pos32 = np.asarray(pos, np.float32)
    J = pos32.shape[0]
    if kind == SAMPLER_RANDOM:
        idx = list(range(J))
        state = seed & _MASK64
        for i in range(J - 1, 0, -1):
            state, z = splitmix64(state)
            k = z % (i + 1)
            idx[i], idx[k] = idx[k], idx[i]
        return np.array(idx, np.int32)
    groups = []
    if kind == SAMPLER_COMPACT:
        _kd_split(pos32, list(range(J)), -(-J // batch), batch, groups)
        return np.array([i for g in groups for i in g], np.int32)
    _kd_split(pos32, list(range(J)), min(batch, max(J, 1)), 0, groups)
    longest = max(len(g) for g in groups)
    return np.array([g[t] for t in range(longest) for g in groups if t < len(g)], np.int32)


# ---------------------------------------------------------------------------
# Multislice (Sec. 1 and Sec. 2.1: multislice modelling). The object has S
# slices [S, H, W]; the wave is multiplied by each slice's patch and carried to
# the next slice by the angular-spectrum propagator.
# ---------------------------------------------------------------------------
def asm_propagator(N: int, pixel_size: float, wavelength: float, dz: float) -> np.ndarray:
    """Angular-spectrum transfer function on the N x N FFT grid (no fftshift).

    H(f) = exp(i 2 pi dz (sqrt(1/lambda^2 - |f|^2) - 1/lambda)) with the
    spatial frequencies f = k / (N pixel_size); the constant phase 2 pi dz /
    lambda is dropped (a global phase) and evanescent frequencies are set to 0.
    The bracket is evaluated as -|f|^2 / (sqrt(1/lambda^2 - |f|^2) + 1/lambda).
    """
    f = np.fft.fftfreq(N, d=pixel_size)
    fy, fx = np.meshgrid(f, f, indexing="ij")
    f2 = fy * fy + fx * fx
    inv_l2 = 1.0 / (wavelength * wavelength)
    prop = f2 < inv_l2
    kz = np.sqrt(np.where(prop, inv_l2 - f2, 0.0))
    phase = 2.0 * np.pi * dz * (-f2 / (kz + 1.0 / wavelength))
    return np.where(prop, np.exp(1j * phase), 0.0)


def propagate(psi: np.ndarray, Hf: np.ndarray) -> np.ndarray:
    """F^-1 [H F psi] over the last two axes."""
    return idft2(Hf * dft2(psi))


def exit_waves_ms(Os, P, r, Hf):
    """Per-mode exit waves after the last slice, and each slice's incident wave.

    Os: [S, H, W]; returns (psi_out [M, N, N], incident [S, M, N, N], patches [S, N, N]).
    """
    N = P.shape[-1]
    S = Os.shape[0]
    o = np.stack([extract(Os[s], r, N) for s in range(S)])
    inc = np.empty((S,) + P.shape, np.complex128)
    psi = np.asarray(P, np.complex128)
    for s in range(S):
        if s > 0:
            psi = propagate(psi, Hf)
        inc[s] = psi
        psi = psi * o[s][None]
    return psi, inc, o


def forward_ms(Os, P, pos, Hf):
    """Predicted intensities [J, N, N] of the multislice model."""
    out = np.empty((pos.shape[0], P.shape[-1], P.shape[-1]), np.float64)
    for j in range(pos.shape[0]):
        psi, _, _ = exit_waves_ms(Os, P, pos[j], Hf)
        out[j] = np.sum(np.abs(dft2(psi)) ** 2, axis=0)
    return out


def vjp_ms(Os, P, pos, Hf, G):
    """Gradients (2 dL/dz*) of the multislice model given G = dL/dI.

    Backward through the slices: at slice s the wave leaving it is
    incident_s * o_s, so g(o_s) += conj(incident_s) g_out and the gradient
    reaching the slice entrance is conj(o_s) g_out; the propagator's adjoint
    is F^-1 [conj(H) F .]. The probe gradient is the entrance gradient of
    slice 0; the position gradient sums each slice's patch derivative.
    """
    S, H, W = Os.shape
    N = P.shape[-1]
    gO = np.zeros((S, H, W), np.complex128)
    gP = np.zeros_like(P, dtype=np.complex128)
    gr = np.zeros((pos.shape[0], 2), np.float64)
    Hc = np.conj(Hf)
    for j in range(pos.shape[0]):
        psi, inc, o = exit_waves_ms(Os, P, pos[j], Hf)
        g = idft2(2.0 * G[j][None] * dft2(psi))       # gradient w.r.t. the exit waves
        go = np.zeros((S, N, N), np.complex128)
        for s in range(S - 1, -1, -1):
            go[s] = np.sum(np.conj(inc[s]) * g, axis=0)
            g = np.conj(o[s])[None] * g
            if s > 0:
                g = propagate(g, Hc)
        gP += g
        for s in range(S):
            gO[s] += scatter(go[s], pos[j], H, W)
            d_dy, d_dx = extract_dr(Os[s], pos[j], N)
            gr[j, 0] += np.real(np.sum(np.conj(go[s]) * d_dy))
            gr[j, 1] += np.real(np.sum(np.conj(go[s]) * d_dx))
    return gO, gP, gr


def loss_and_gradients_ms(Os, P, pos, Hf, I_m, noise=GAUSSIAN, eps=0.0):
    I = forward_ms(Os, P, pos, Hf)
    loss = sum(pattern_loss(I[j], I_m[j], noise, eps) for j in range(pos.shape[0]))
    return (loss,) + vjp_ms(Os, P, pos, Hf, dloss_dI(I, I_m, noise, eps))


# ---------------------------------------------------------------------------
# LSQML with a multislice object (Sec. 1 and Sec. 2.1: multislice modelling is
# a forward-model option of every reconstructor; LSQML, Sec. 2.2).
# ---------------------------------------------------------------------------
def lsqml_batch_ms(Os, P, pos, I_m, idx, Hf, opts: LsqmlOptions, record: dict | None = None):
    """One LSQML minibatch with an object of S slices; returns (Os, P, loss, alpha [B, 2]).

    Per position j and mode k, the exit-plane change is that of the
    single-slice method, chi_jk = F^-1[(rho_j - 1) Psi_jk], with Psi the far
    field of the last slice's exit wave. It is carried back through the slices
    (s = S-1 .. 0): slice s, whose exit wave is inc_jsk o_js, receives
        g_js = sum_k conj(inc_jsk) chi_jsk   (its direction numerator),
        w_js = sum_k |inc_jsk|^2             (its illumination),
    with chi_j(S-1)k = chi_jk and chi_j(s-1)k = H^H[conj(o_js) chi_jsk]; the
    probe (the wave entering slice 0) receives h_jk = conj(o_j0) chi_j0k.
    Directions: dO_s = sum_j S_j^T g_js / (illum_s + delta_o max illum_s) with
    illum_s = sum_j S_j^T w_js, one preconditioner per slice;
    dP_k = sum_j h_jk / (Dp + delta_p max Dp), Dp = sum_j |o_j0|^2.
    Step sizes, per position, the least-squares fit of the exit-plane change by
    the first-order changes of the exit waves: u_jk when every slice moves
    along its direction (the tangent of the forward model, carried through the
    slices: u = dO_0 P at slice 0, then u <- H(u) o_s + inc_s dO_s(r_j)), v_jk
    when the probe moves along dP (v = o_0 dP, then v <- H(v) o_s); the 2x2
    system and its solve are those of :func:`lsqml_batch`.
    Update: O_s += sum_j S_j^T(alpha_O,j g_js) / (illum_s + delta_O,s);
    P_k += mean_j(alpha_P,j) dP_k. With S = 1 this is :func:`lsqml_batch`.
    """
    S, H, W = Os.shape
    M, N = P.shape[0], P.shape[-1]
    idx = [int(i) for i in idx]
    B = len(idx)
    Hc = np.conj(Hf)
    loss = 0.0
    rec = []
    dO_acc = np.zeros((S, H, W), np.complex128)
    illum = np.zeros((S, H, W), np.float64)
    dP_acc = np.zeros((M, N, N), np.complex128)
    Dp = np.zeros((N, N), np.float64)
    for j in idx:
        psi, inc, o = exit_waves_ms(Os, P, pos[j], Hf)
        Psi = dft2(psi)
        I = np.sum(np.abs(Psi) ** 2, axis=0)
        loss += pattern_loss(I, I_m[j], opts.noise, opts.eps)
        rho = modulus_ratio(I, I_m[j], opts.noise, opts.eps)
        chi = idft2((rho - 1.0)[None] * Psi)             # exit-plane change of the last slice
        g = np.zeros((S, N, N), np.complex128)
        w = np.zeros((S, N, N), np.float64)
        chis = np.zeros((S,) + P.shape, np.complex128)
        for s in range(S - 1, -1, -1):
            chis[s] = chi
            g[s] = np.sum(np.conj(inc[s]) * chi, axis=0)
            w[s] = np.sum(np.abs(inc[s]) ** 2, axis=0)
            chi = np.conj(o[s])[None] * chi
            if s > 0:
                chi = propagate(chi, Hc)
        h = chi                                          # conj(o_j0) chi_j0 per mode
        for s in range(S):
            dO_acc[s] += scatter(g[s], pos[j], H, W)
            illum[s] += scatter(w[s], pos[j], H, W)
        dP_acc += h
        Dp += np.abs(o[0]) ** 2
        rec.append((o, inc, g, w, chis))

    delta_O = opts.delta_o * np.max(illum.reshape(S, -1), axis=1)
    delta_P = opts.delta_p * float(np.max(Dp))
    dO_hat = dO_acc / (illum + delta_O[:, None, None])
    if not opts.update_object:
        dO_hat = np.zeros_like(dO_hat)
    dP = dP_acc / (Dp + delta_P)[None] if opts.update_probe else np.zeros_like(dP_acc)

    alpha = np.zeros((B, 2), np.float64)
    tangents = []
    for i, j in enumerate(idx):
        o, inc, g, w, chis = rec[i]
        u = extract(dO_hat[0], pos[j], N)[None] * P
        v = o[0][None] * dP
        for s in range(1, S):
            u = propagate(u, Hf) * o[s][None] + inc[s] * extract(dO_hat[s], pos[j], N)[None]
            v = propagate(v, Hf) * o[s][None]
        chi = chis[S - 1]
        A11 = float(np.sum(np.abs(u) ** 2))
        A12 = float(np.real(np.sum(np.conj(u) * v)))
        A22 = float(np.sum(np.abs(v) ** 2))
        b1 = float(np.real(np.sum(np.conj(u) * chi)))
        b2 = float(np.real(np.sum(np.conj(v) * chi)))
        alpha[i] = step_solve(A11, A12, A22, b1, b2, opts.lam)
        tangents.append((u, v))

    Os_new = Os.copy()
    if opts.update_object:
        for s in range(S):
            upd = np.zeros((H, W), np.complex128)
            for i, j in enumerate(idx):
                upd += scatter(alpha[i, 0] * rec[i][2][s], pos[j], H, W)
            Os_new[s] = Os[s] + upd / (illum[s] + delta_O[s])
    P_new = P + float(np.mean(alpha[:, 1])) * dP if opts.update_probe else P.copy()
    if record is not None:
        record.update(dict(dO_acc=dO_acc, illum=illum, dP_acc=dP_acc, Dp=Dp, delta_O=delta_O, delta_P=delta_P,
                           dO_hat=dO_hat, dP=dP, alpha=alpha, g=np.stack([r[2] for r in rec]),
                           w=np.stack([r[3] for r in rec]), chi=np.stack([r[4] for r in rec]),
                           u=np.stack([t[0] for t in tangents]), v=np.stack([t[1] for t in tangents])))
    return Os_new, P_new, loss, alpha


def lsqml_epoch_ms(Os, P, pos, I_m, order, Hf, opts: LsqmlOptions):
    """One epoch of multislice LSQML minibatches (``opts.batch`` positions of
    ``order`` in turn); returns (Os, P, loss, alpha [J, 2])."""
    Os = np.asarray(Os, np.complex128).copy()
    P = np.asarray(P, np.complex128).copy()
    order = np.asarray(order)
    loss = 0.0
    alpha = np.zeros((pos.shape[0], 2), np.float64)
    for b0 in range(0, order.shape[0], opts.batch):
        idx = order[b0:b0 + opts.batch]
        Os, P, l, a = lsqml_batch_ms(Os, P, pos, I_m, idx, Hf, opts)
        loss += l
        alpha[idx] = a
    return Os, P, loss, alpha
