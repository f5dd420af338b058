/* ptycho.h -- C ABI of the GB300 LSQML ptychography hot path.
 *
 * The library implements the data-parallel per-scan-position path of the
 * LSQML reconstructor described in Pty-Chi (Du et al., arXiv 2510.20929):
 * the far-field forward model F(o, p, Lambda) of Sec. 2.1 / Eq. 4 (sub-pixel
 * object patch, incoherent probe modes, unitary 2-D FFT, intensity), the
 * amplitude data term of Eq. 1 (and the Poisson likelihood), its gradient
 * (Eq. 2, extended to the probe modes and the scan positions), and one LSQML
 * epoch: modulus-projected exit-wave update, illumination-preconditioned
 * object and probe directions (Sec. 1, Sec. 4), per-position least-squares
 * step sizes (Sec. 2.2), and the minibatch update.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All array arguments are DEVICE pointers owned by the caller, row-major
 *   and contiguous. "complex64" means interleaved (re, im) float pairs.
 * - Object O: complex64 [H, W]. Probe P: complex64 [M, N, N] (M incoherent
 *   modes). Positions: float32 [J, 2], (y, x) probe centre in object pixels.
 *   Intensities: float32 [J, N, N] with the zero frequency at [0, 0]
 *   (no fftshift).
 * - Patch extraction is bilinear: t = floor(r - N/2), f = r - N/2 - t; the
 *   (N+1) x (N+1) tile starting at t must lie inside the object, i.e.
 *   0 <= r - N/2 < H - N (same for x). The far-field propagator is the
 *   unitary ("ortho") 2-D DFT.
 * - Gradients follow the complex convention grad = 2 dL/dz* (PyTorch's), so
 *   dL = Re<grad, dz> for a perturbation dz.
 * - Supported window sizes N: 16, 32, 64, 128, 192, 256 (192 and 256 run on
 *   clusters of six and eight CTAs, 32 rows each, sharing the tile through
 *   distributed shared memory).
 *   Modes: 1 <= M <= 16.
 * - The library never allocates device memory. Scratch lives in a caller
 *   workspace of ptycho_workspace_bytes() bytes (256-byte aligned).
 * - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *   default stream). Argument errors are returned synchronously before any
 *   launch. Data errors found on the device (a position whose tile leaves the
 *   object, an `order` entry outside [0, J), a negative or non-finite measured
 *   intensity) are recorded in the workspace and returned by
 *   ptycho_status_read(); such positions are skipped, never read out of bounds.
 */
#ifndef PTYCHO_H
#define PTYCHO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t H, W; /* object size */
  int32_t N;    /* probe window (N x N) */
  int32_t M;    /* incoherent probe modes */
  int32_t J;    /* scan positions */
} ptycho_dims;

typedef enum {
  PTYCHO_OK = 0,
  PTYCHO_ERR_ARG = 1,         /* null pointer, bad size, bad option */
  PTYCHO_ERR_BOUNDS = 2,      /* (device) a position's tile leaves the object, or a bad order entry */
  PTYCHO_ERR_NONFINITE = 3,   /* (device) negative or non-finite measured intensity */
  PTYCHO_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  PTYCHO_ERR_TIMEOUT = 5,     /* (device) a bounded wait of the tensor-core pipeline gave up */
  PTYCHO_ERR_UNSUPPORTED = 6, /* window size or mode count not built */
  PTYCHO_ERR_WORKSPACE = 7,   /* workspace missing, misaligned or too small */
  PTYCHO_ERR_TOO_LARGE = 8    /* problem needs more scratch than ptycho_lsqml_epoch_static holds */
} ptycho_status;

typedef enum {
  PTYCHO_NOISE_GAUSSIAN = 0, /* L = sum (sqrt(I + eps) - sqrt(I_m))^2 (Eq. 1, unnormalised) */
  PTYCHO_NOISE_POISSON = 1,  /* L = sum (I - I_m log(I + eps)) */
  PTYCHO_NOISE_VJP = 2       /* ptycho_adjoint only: the `meas` array holds dL/dI */
} ptycho_noise;

typedef struct {
  int32_t noise;            /* PTYCHO_NOISE_GAUSSIAN or PTYCHO_NOISE_POISSON */
  int32_t batch;            /* minibatch size B >= 1 */
  int32_t update_object;    /* 0/1 */
  int32_t update_probe;     /* 0/1 */
  int32_t flags;            /* PTYCHO_FLAG_* bits */
  int32_t update_positions; /* 0/1: least-squares position correction per minibatch; the
                               positions array is then updated in place */
  int32_t object_per_epoch; /* 0/1: accumulate the object update over the epoch and apply it
                               once at its end (the update cadence LSQML takes with the
                               compact sampler, Sec. 2.2); needs the larger workspace of
                               ptycho_workspace_bytes_opts */
  int32_t precision;        /* PTYCHO_PRECISION_FP32 or PTYCHO_PRECISION_BF16X3 */
  double delta_o;           /* object preconditioner damping, relative to max(illumination) */
  double delta_p;           /* probe preconditioner damping, relative to max(sum_j |o_j|^2) */
  double lambda_reg;        /* 2x2 step-size Tikhonov term, relative to trace/2 */
  double eps;               /* added to the predicted intensity in the data term */
  double pos_step;          /* relaxation of the position step (1 = the least-squares step) */
  double pos_max_shift;     /* clamp of each component of a minibatch's position step, px */
} ptycho_lsqml_opts;

/* opts->precision: how the far-field transforms F and F^-1 are evaluated.
 * FP32: shared-memory radix FFTs in FP32 (every window size).
 * BF16X3: the 2-D DFT as dense complex GEMMs on the tensor cores (tcgen05,
 * FP32 accumulation in tensor memory) with every operand split into BF16
 * hi + lo parts and three products per real product (hi*hi + lo*hi + hi*lo);
 * windows N = 32, 64 and 128 (others: PTYCHO_ERR_UNSUPPORTED), the shared
 * probe only (the relaxed-probe and multislice entry points take FP32); the
 * measured-intensity array must be 16-byte aligned (else PTYCHO_ERR_ARG). Each
 * operand is represented to within 2^-16 of its magnitude (about 2^-17
 * typically), and the dropped lo*lo term is of the same order; the transform's
 * norm-wise error is near 1e-5. */
#define PTYCHO_PRECISION_FP32 0
#define PTYCHO_PRECISION_BF16X3 1

/* opts->flags: capture the epoch's launch sequence into a CUDA graph on the
 * first call with a given set of arguments (pointers, sizes, options) and
 * replay it on later identical calls, which then cost one graph launch. The
 * first such call must not itself be inside a stream capture. */
#define PTYCHO_FLAG_GRAPH 1
/* opts->flags: on the first epoch for a given device and (N, M, H, W, batch),
 * time the candidate variants of three kernels of the epoch on the first
 * minibatch (synchronising the stream; skipped while capturing) and use the
 * fastest of each from then on. Without it, or before tuning, the
 * per-position and step-size passes use variant 0 and the probe reduction
 * variant 3 (the fastest candidate on every workload measured). The
 * candidates (the "variants" below):
 *   [0] the per-position pass: windows <= 64: CTA sizes default / alternative;
 *       window 128: 1024 threads (0), 512 threads (1), a pair of CTAs of 512
 *       threads with 64 rows each exchanging the column transforms through
 *       distributed shared memory, two pairs per SM (2); windows 192/256: one;
 *   [1] the step-size pass: one kernel per position (0), or the partial sums
 *       spread over 8 chunks of every position, then a
 *       per-position solve and update (1), or (windows <= 128) a cluster of 4
 *       CTAs per position adding their partial sums over distributed shared
 *       memory, at 4 (2) or 3 (3) CTAs per SM;
 *   [2] the probe reduction: 16 (0), 8 (1) or 32 (2) positions in flight per
 *       thread, or the minibatch split into 4 ranges summed by 4 threads of
 *       a block with 8 positions in flight each (3). */
#define PTYCHO_FLAG_AUTOTUNE 2
#define PTYCHO_TUNE_KERNELS 3
#define PTYCHO_TUNE_MAX 4

/* Autotuner choice for these dimensions and batch on the current device:
 * returns 1 and fills variants[PTYCHO_TUNE_KERNELS] and the measured
 * milliseconds ms[PTYCHO_TUNE_KERNELS * PTYCHO_TUNE_MAX] (row i: kernel i's
 * candidates, 0 where not timed; either pointer may be NULL), or 0 if these
 * dimensions were not tuned (or were pinned by ptycho_tuning_set, which
 * records no times). */
int32_t ptycho_tuning_read(const ptycho_dims* dims, int32_t batch, int32_t* variants, float* ms);

/* Pins the variants used for these dimensions and batch on the current
 * device (as if the autotuner had chosen them; a later PTYCHO_FLAG_AUTOTUNE
 * call does not retune them). PTYCHO_ERR_ARG for a variant outside its
 * kernel's candidates, PTYCHO_ERR_UNSUPPORTED for unsupported dimensions. */
ptycho_status ptycho_tuning_set(const ptycho_dims* dims, int32_t batch, const int32_t* variants);

/* Bytes of workspace needed by every entry point below for these dimensions
 * and minibatch size (ptycho_adjoint processes positions in chunks of
 * `batch`) with object_per_epoch = 0. Returns 0 for unsupported dimensions.
 * ptycho_workspace_bytes_opts gives the size for a set of epoch options
 * (object_per_epoch adds an H x W complex64 epoch accumulator). */
size_t ptycho_workspace_bytes(const ptycho_dims* dims, int32_t batch);
size_t ptycho_workspace_bytes_opts(const ptycho_dims* dims, const ptycho_lsqml_opts* opts);

/* Clears the workspace header (its device status word). Call once on a fresh
 * workspace before the first entry point that uses it. */
ptycho_status ptycho_workspace_init(void* ws, size_t ws_bytes, void* stream);

/* Forward model (Sec. 2.1, Eq. 4): I_pred[j] = sum_k |F(P_k * S_j(O))|^2 for
 * all J positions. I_pred: float32 [J, N, N], overwritten. Positions that
 * fail the bounds rule leave their I_pred block untouched. */
ptycho_status ptycho_forward(const ptycho_dims* dims, const float* object, const float* probe,
                             const float* pos, float* I_pred, void* ws, size_t ws_bytes,
                             void* stream);

/* Data term and its gradients (Eq. 1 and Eq. 2, extended to probe modes and
 * positions), exit waves recomputed, never stored. `meas` is the measured
 * intensity for GAUSSIAN/POISSON, or dL/dI for VJP. All outputs are
 * ACCUMULATED (+=), so sums over position subsets add up to the full-set
 * result; zero them first for a plain evaluation:
 *   g_object complex64 [H, W], g_probe complex64 [M, N, N],
 *   g_pos float32 [J, 2] (may be NULL), loss float64 scalar (may be NULL;
 *   untouched for VJP). Positions are processed in chunks of `batch`.
 * With g_object, g_probe and g_pos all NULL (GAUSSIAN or POISSON, `loss`
 * given) only the forward model and the data term run: the loss alone, at
 * about half the cost (no back-propagation). */
ptycho_status ptycho_adjoint(const ptycho_dims* dims, const float* object, const float* probe,
                             const float* pos, const float* meas, int32_t noise, double eps,
                             int32_t batch, float* g_object, float* g_probe, float* g_pos,
                             double* loss, void* ws, size_t ws_bytes, void* stream);

/* ptycho_forward (Sec. 2.1, Eq. 4) and ptycho_adjoint (Eq. 1-2) with the
 * far-field precision chosen (PTYCHO_PRECISION_*); every other argument has
 * the meaning, layout and ownership given above, and the same synchronous
 * argument checks and device status apply. precision other than FP32 and
 * BF16X3 is PTYCHO_ERR_ARG; BF16X3 on a window other than 32, 64 or 128 is
 * PTYCHO_ERR_UNSUPPORTED, and with `meas` not 16-byte aligned PTYCHO_ERR_ARG.
 * The forward form processes positions in chunks of `batch` (>= 1) and with
 * BF16X3 needs ptycho_workspace_bytes(dims, batch) of workspace (with FP32
 * the header suffices, as for ptycho_forward). A bounded wait of the
 * tensor-core kernel that gives up is reported as PTYCHO_ERR_TIMEOUT by
 * ptycho_status_read. */
ptycho_status ptycho_forward_ex(const ptycho_dims* dims, int32_t precision, int32_t batch,
                                const float* object, const float* probe, const float* pos,
                                float* I_pred, void* ws, size_t ws_bytes, void* stream);
ptycho_status ptycho_adjoint_ex(const ptycho_dims* dims, int32_t precision, const float* object,
                                const float* probe, const float* pos, const float* meas,
                                int32_t noise, double eps, int32_t batch, float* g_object,
                                float* g_probe, float* g_pos, double* loss, void* ws,
                                size_t ws_bytes, void* stream);

/* One LSQML epoch (Sec. 2.2): minibatches of opts->batch positions taken from
 * `order` (int32 [J], a permutation or any list of indices in [0, J); NULL =
 * 0..J-1). Per minibatch: exit-wave changes chi_jk, preconditioned object and
 * probe directions, per-position FP64 2x2 step sizes, then
 *   O += sum_j S_j^T(alpha_O,j g_j) / (illum + delta_O),
 *   P_k += mean_j(alpha_P,j) dP_k.
 * object and probe are updated in place. loss (float64 scalar, may be NULL)
 * receives the epoch's data term summed over positions, each evaluated at the
 * state its minibatch started from. alpha (float64 [J, 2], may be NULL)
 * receives (alpha_O, alpha_P) per position.
 * With opts->update_positions each position of a minibatch also moves by
 * pos_step times its least-squares shift (position correction, Sec. 1 /
 * Sec. 2.1): argmin_dr sum_k ||chi_jk - P_k (d o_j / d r) dr||^2 over the
 * bilinear patch derivatives at the object the minibatch started from,
 * solved in FP64 like the step sizes, each component clamped to
 * +-pos_max_shift and the result kept inside the bounds rule (at most
 * H - N/2 - 1/64). With opts->object_per_epoch every minibatch sees the
 * epoch's starting object and the object updates are applied together at
 * the end of the epoch. */
ptycho_status ptycho_lsqml_epoch(const ptycho_dims* dims, float* object, float* probe,
                                 float* pos, const float* meas, const int32_t* order,
                                 const ptycho_lsqml_opts* opts, double* loss, double* alpha,
                                 void* ws, size_t ws_bytes, void* stream);

/* Batched serving: one LSQML epoch for each of n independent reconstructions
 * of possibly different sizes (arrays of n dimensions, options and device
 * pointers; `orders` may be NULL, or hold NULL entries). losses: float64 [n]
 * device array or NULL. Workspace: ptycho_workspace_bytes_batched() bytes,
 * split into one section per reconstruction in argument order. Each
 * reconstruction computes exactly what ptycho_lsqml_epoch computes for it;
 * their minibatches run concurrently on internal worker streams forked from
 * and joined back into `stream`. If every opts[i].flags has PTYCHO_FLAG_GRAPH,
 * the launch sequence is captured once and replayed as one graph launch.
 * Section i starts at the sum of ptycho_workspace_bytes(dims[k], opts[k].batch)
 * over k < i; its status word is cleared at the start of the call and read
 * with ptycho_status_read(section). */
size_t ptycho_workspace_bytes_batched(int32_t n, const ptycho_dims* dims, const ptycho_lsqml_opts* opts);
ptycho_status ptycho_lsqml_epoch_batched(int32_t n, const ptycho_dims* dims, float* const* objects,
                                         float* const* probes, float* const* pos,
                                         const float* const* meas, const int32_t* const* orders,
                                         const ptycho_lsqml_opts* opts, double* losses, void* ws,
                                         size_t ws_bytes, void* stream);

/* Same epoch with HOST buffers: copies pos, meas and order (and the object and
 * probe) into device staging areas carved from `ws` (ws_bytes must be at least
 * ptycho_host_workspace_bytes(), or ptycho_host_workspace_bytes_opts() for
 * these options), runs the epoch on `stream`, copies object, probe, loss (and
 * the positions when they are corrected) back, and synchronises the stream
 * before returning. Host buffers should be pinned for full copy bandwidth.
 * With PTYCHO_PRECISION_FP32, a `meas` array in pinned host memory that is
 * mapped into the device address space (cudaHostAlloc, or page-locked tensors
 * on a unified-addressing system) is not staged before the epoch: a gather
 * kernel on one of the library's worker streams (the one
 * ptycho_lsqml_epoch_batched also uses) reads it over the host link into `ws`
 * minibatch by minibatch, in the epoch's order, and each minibatch waits only
 * for its own positions, so the transfer overlaps the compute. */
size_t ptycho_host_workspace_bytes(const ptycho_dims* dims, int32_t batch);
size_t ptycho_host_workspace_bytes_opts(const ptycho_dims* dims, const ptycho_lsqml_opts* opts);
ptycho_status ptycho_lsqml_epoch_host(const ptycho_dims* dims, float* object, float* probe,
                                      float* pos, const float* meas, const int32_t* order,
                                      const ptycho_lsqml_opts* opts, double* loss, void* ws,
                                      size_t ws_bytes, void* stream);

/* Allocation-free epoch, for callers that cannot allocate device memory:
 * applications that reserve the whole device memory budget up front through
 * their own allocator, or real-time pipelines that must not call cudaMalloc
 * because it can synchronise the device. It computes exactly what
 * ptycho_lsqml_epoch computes (same arguments, minus the workspace), with its
 * scratch taken from a fixed device array of PTYCHO_STATIC_WS_BYTES bytes that
 * every GPU loading the library keeps until the process exits. The paper has
 * no counterpart: this is an interface for embedding the library.
 * - Returns PTYCHO_ERR_TOO_LARGE, before touching the device, when
 *   ptycho_workspace_bytes_opts(dims, opts) exceeds PTYCHO_STATIC_WS_BYTES.
 * - Argument errors return the statuses ptycho_lsqml_epoch returns for the
 *   same arguments. PTYCHO_FLAG_GRAPH in opts->flags is ignored: the epoch
 *   runs as eager launches (an executable graph would make the driver
 *   allocate).
 * - The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current, and so does the first
 *   call after that device's CUDA context was destroyed and created again;
 *   make that call before any stream capture.
 * - All calls share the one array per device: calls whose work overlaps on the
 *   GPU (other streams, other host threads) race and must be serialised by
 *   the caller.
 * - Synchronises `stream` at the end and returns the device-side status as
 *   ptycho_status_read() would. No device memory is allocated. */
#define PTYCHO_STATIC_WS_BYTES (64u * 1024u * 1024u)
ptycho_status ptycho_lsqml_epoch_static(const ptycho_dims* dims, float* object, float* probe,
                                        float* pos, const float* meas, const int32_t* order,
                                        const ptycho_lsqml_opts* opts, double* loss, double* alpha,
                                        void* stream);

/* ---------------------------------------------------------------------------
 * Orthogonal probe relaxation (Sec. 2.1: scan-point-specific probes). The
 * primary probe mode of position j is P_j0 = sum_m w[j][m] U[m] over K
 * eigenmodes U (complex64 [K, N, N], 1 <= K <= 8) with real weights w
 * (float32 [J, K]); the other dims->M - 1 modes are shared by all positions
 * (P_rest, complex64 [M - 1, N, N]; may be NULL when M == 1). dims->M counts
 * every mode, the primary one included. The per-position kernels synthesise
 * P_j0 on chip.
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t K;              /* eigenmodes, 1..8 */
  int32_t update_weights; /* 0/1: per-position least-squares weight update */
  int32_t reserved[2];    /* must be zero */
  double weight_step;     /* relaxation of the weight update (1 = the full least-squares step) */
} ptycho_opr_opts;

/* Workspace bytes of the three OPR entry points below (0 if unsupported). */
size_t ptycho_workspace_bytes_opr(const ptycho_dims* dims, int32_t K, int32_t batch);

/* Forward model with the relaxed primary mode: I_pred[j] = |F(P_j0 S_j(O))|^2
 * + sum_k |F(P_rest_k S_j(O))|^2. As ptycho_forward otherwise. */
ptycho_status ptycho_forward_opr(const ptycho_dims* dims, int32_t K, const float* object, const float* U,
                                 const float* w, const float* P_rest, const float* pos, float* I_pred,
                                 void* ws, size_t ws_bytes, void* stream);

/* Gradients of the data term through the relaxed model, ACCUMULATED (+=) as
 * in ptycho_adjoint: g_object [H, W], g_U complex64 [K, N, N]
 * (sum_j w_jm conj(o_j) times the exit-wave gradient of mode 0), g_w float32
 * [J, K] (Re<U_m, that product>, may be NULL), g_P_rest [M - 1, N, N] (NULL
 * when M == 1), g_pos [J, 2] (may be NULL), loss (may be NULL). */
ptycho_status ptycho_adjoint_opr(const ptycho_dims* dims, int32_t K, const float* object, const float* U,
                                 const float* w, const float* P_rest, const float* pos, const float* meas,
                                 int32_t noise, double eps, int32_t batch, float* g_object, float* g_U,
                                 float* g_w, float* g_P_rest, float* g_pos, double* loss, void* ws,
                                 size_t ws_bytes, void* stream);

/* One LSQML epoch with the relaxed primary mode. Per minibatch, as
 * ptycho_lsqml_epoch with these differences: the illumination and the step
 * sizes use each position's own primary mode; the eigenmodes move with the
 * probe step, U_m += mean_j(alpha_P,j) dU_m, along
 *   dU_m = sum_j w_jm conj(o_j) chi_j0 / (D_m + delta_P),
 *   D_m = sum_j w_jm^2 |o_j|^2, delta_P = delta_p max(sum_j |o_j|^2, D),
 * whose per-position image sum_m w_jm dU_m is the primary mode's direction in
 * the step-size system; and, with opr->update_weights, each position's
 * weights move by weight_step times the least-squares fit (FP64, damped by
 * lambda_reg tr(A)/K) of chi_j0 with the exit waves U_m o_j, taken with this
 * minibatch's U and chi. U, w, P_rest and the object are updated in place.
 * PTYCHO_FLAG_GRAPH is honoured; PTYCHO_FLAG_AUTOTUNE is ignored (default CTA
 * sizes); update_positions and object_per_epoch are not supported with OPR
 * (PTYCHO_ERR_UNSUPPORTED). */
ptycho_status ptycho_lsqml_epoch_opr(const ptycho_dims* dims, const ptycho_opr_opts* opr, float* object,
                                     float* U, float* w, float* P_rest, const float* pos, const float* meas,
                                     const int32_t* order, const ptycho_lsqml_opts* opts, double* loss,
                                     double* alpha, void* ws, size_t ws_bytes, void* stream);

/* Batched serving with the relaxed primary mode: ptycho_lsqml_epoch_opr for
 * each of n reconstructions, run concurrently as ptycho_lsqml_epoch_batched
 * runs its reconstructions (arrays of n entries; P_rest may be NULL when
 * every dims[i].M == 1, `orders` may be NULL or hold NULL entries). Section i
 * of the workspace has ptycho_workspace_bytes_opr(dims[i], opr[i].K,
 * opts[i].batch) bytes. */
size_t ptycho_workspace_bytes_opr_batched(int32_t n, const ptycho_dims* dims, const ptycho_opr_opts* opr,
                                          const ptycho_lsqml_opts* opts);
ptycho_status ptycho_lsqml_epoch_opr_batched(int32_t n, const ptycho_dims* dims, const ptycho_opr_opts* opr,
                                             float* const* objects, float* const* U, float* const* w,
                                             float* const* P_rest, const float* const* pos,
                                             const float* const* meas, const int32_t* const* orders,
                                             const ptycho_lsqml_opts* opts, double* losses, void* ws,
                                             size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Multislice (Sec. 1 and Sec. 2.1: multislice modelling). The object has S
 * slices, complex64 [S, H, W]. For position j and mode k the wave entering
 * slice 0 is P_k; the wave leaving slice s is its incident wave times
 * S_j(O^(s)); between slices the wave is propagated by the angular spectrum,
 * F^-1[H F psi] with H(f) = exp(i 2 pi dz (sqrt(1/lambda^2 - |f|^2) - 1/lambda))
 * on the FFT grid f = k / (N pixel_size) (the constant phase 2 pi dz / lambda
 * dropped, evanescent frequencies zero; computed in FP64 on the device); the
 * far field of the last slice gives I_j = sum_k |F psi_jk|^2. Every window
 * size, 1 <= S <= 16. The backward pass needs the incident waves of slices
 * 1..S-1. With recompute = 0 the forward pass keeps every mode's in the
 * workspace (B M (S-1) N^2 complex64). With recompute = 1 it keeps none: the
 * backward pass runs each mode through the slices again just before carrying
 * its exit-plane change back (2 (S-1) more 2-D transforms per mode; the LSQML
 * tangent pass does the same), and the workspace holds one mode's waves per
 * position (B (S-1) N^2 complex64), which stay mostly in L2 between their
 * write and their read. Both give the same waves, bit for bit.
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t S;          /* object slices */
  int32_t recompute;  /* 0: incident waves kept by the forward pass, 1: recomputed
                         in the backward pass; any other value: PTYCHO_ERR_ARG */
  double dz;          /* slice spacing */
  double wavelength;  /* same unit as dz */
  double pixel_size;  /* object pixel, same unit */
} ptycho_multislice;

/* Workspace bytes of the two multislice entry points (0 if unsupported). */
size_t ptycho_workspace_bytes_ms(const ptycho_dims* dims, const ptycho_multislice* ms, int32_t batch);

/* Multislice forward model, positions in chunks of `batch`. I_pred float32
 * [J, N, N], overwritten. */
ptycho_status ptycho_forward_ms(const ptycho_dims* dims, const ptycho_multislice* ms, const float* object,
                                const float* probe, const float* pos, float* I_pred, int32_t batch, void* ws,
                                size_t ws_bytes, void* stream);

/* Data term and gradients (2 dL/dz*) through the multislice model, all
 * ACCUMULATED (+=): g_object complex64 [S, H, W], g_probe [M, N, N], g_pos
 * float32 [J, 2] (may be NULL), loss (may be NULL; untouched for VJP). As
 * ptycho_adjoint otherwise. */
ptycho_status ptycho_adjoint_ms(const ptycho_dims* dims, const ptycho_multislice* ms, const float* object,
                                const float* probe, const float* pos, const float* meas, int32_t noise,
                                double eps, int32_t batch, float* g_object, float* g_probe, float* g_pos,
                                double* loss, void* ws, size_t ws_bytes, void* stream);

/* One LSQML epoch with a multislice object (Sec. 1 and Sec. 2.1: multislice
 * modelling as a forward-model option of every reconstructor; LSQML, Sec.
 * 2.2), updating `object` ([S, H, W]) and `probe` in place. Per position the
 * exit-plane change chi = F^-1[(rho - 1) Psi] of the last slice is carried
 * back through the slices (adjoint propagation, times conj of each slice's
 * patch); every slice s gets the direction numerator sum_k conj(inc_sk) chi_sk
 * and the illumination sum_k |inc_sk|^2 of its incident waves and its own
 * object-frame preconditioner (damping delta_o times its maximum); the probe
 * direction is conj(o_0) chi_0 / (sum |o_0|^2 + delta_p max). The step sizes
 * are the 2x2 least-squares fit of the exit-plane change by the tangents of
 * the forward model (the first-order change of the exit waves when every
 * slice moves along its direction, and when the probe moves along its own),
 * solved like ptycho_lsqml_epoch's; every slice moves by the position's
 * alpha_O, the probe by the mean alpha_P. With S = 1 this is
 * ptycho_lsqml_epoch. alpha: float64 [J, 2] (alpha_O, alpha_P) or NULL.
 * opts as for ptycho_lsqml_epoch, except that precision BF16X3,
 * update_positions and object_per_epoch return PTYCHO_ERR_UNSUPPORTED
 * (PTYCHO_FLAG_AUTOTUNE has no variants to choose here). Workspace:
 * ptycho_workspace_bytes_lsqml_ms(dims, ms, opts); the incident waves are kept
 * (or, with ms->recompute, one mode's parked) there as for the adjoint, plus S
 * accumulator planes [S, H, W] of 16 bytes,
 * the slices' illumination and directions per slot and one tangent plane per
 * slot. */
size_t ptycho_workspace_bytes_lsqml_ms(const ptycho_dims* dims, const ptycho_multislice* ms,
                                        const ptycho_lsqml_opts* opts);
ptycho_status ptycho_lsqml_epoch_ms(const ptycho_dims* dims, const ptycho_multislice* ms, float* object,
                                    float* probe, const float* pos, const float* meas, const int32_t* order,
                                    const ptycho_lsqml_opts* opts, double* loss, double* alpha, void* ws,
                                    size_t ws_bytes, void* stream);

/* Minibatch samplers (Sec. 2.1: random, uniform and compact batches).
 * Writes `order` (int32 [J], a permutation of 0..J-1) for the epoch entry
 * points, whose consecutive chunks of `batch` entries are the minibatches.
 * HOST pointers; pos float32 [J, 2] (y, x). Pure host code, no GPU work.
 *   RANDOM:  Fisher-Yates driven by SplitMix64 from `seed`.
 *   COMPACT: spatially connected clusters: recursive splits at an index along
 *            the longer side of the bounding box (stable sort by that
 *            coordinate), every cluster but the last exactly `batch` long, so
 *            each minibatch is one cluster (pair it with object_per_epoch).
 *   UNIFORM: `batch` balanced compact clusters read round-robin, so each
 *            minibatch takes one position from every part of the scan field.
 * Returns PTYCHO_ERR_ARG for a bad kind, batch < 1, null pointers with J > 0,
 * or a non-finite position. `seed` is used by RANDOM only. */
typedef enum {
  PTYCHO_SAMPLER_RANDOM = 0,
  PTYCHO_SAMPLER_UNIFORM = 1,
  PTYCHO_SAMPLER_COMPACT = 2
} ptycho_sampler;
ptycho_status ptycho_sampler_order(const float* pos, int32_t J, int32_t batch, int32_t kind, uint64_t seed,
                                   int32_t* order);

/* Synchronises `stream`, returns (and clears) the device-side status recorded
 * in `ws` since the last read: PTYCHO_OK, PTYCHO_ERR_TIMEOUT, PTYCHO_ERR_BOUNDS
 * or PTYCHO_ERR_NONFINITE (reported in that order of precedence), or
 * PTYCHO_ERR_CUDA. */
ptycho_status ptycho_status_read(void* ws, void* stream);

/* Diagnostic of the bounded waits: launches on `stream` one kernel whose
 * mbarrier wait cannot complete; the wait gives up after about 2^26 SM clock
 * cycles (tens of milliseconds) and records the timeout in the workspace
 * status, which the next ptycho_status_read() returns as PTYCHO_ERR_TIMEOUT.
 * The GPU context stays usable. ws as for the other entry points (header
 * size at least). */
ptycho_status ptycho_selftest_wait_timeout(void* ws, size_t ws_bytes, void* stream);

/* Static description of a status code. */
const char* ptycho_status_string(ptycho_status status);

/* Per-kernel timing. When enabled, each kernel launch of the entry points
 * above is bracketed by a CUDA event pair recorded on the caller's stream
 * (this adds two event records per launch and is meant for measurement runs,
 * not production). ptycho_profile_read() synchronises the recorded events,
 * writes up to `cap` records (kernels with at least one launch since the last
 * read) and returns how many kernels had launches; it then resets the
 * counters. */
typedef struct {
  char name[32];
  int32_t launches;
  int32_t pad;
  double total_ms;
} ptycho_kernel_time;
ptycho_status ptycho_profile_enable(int32_t on);
/* Restricts the recording to the kernel of this name (as reported by
 * ptycho_profile_read), or records every kernel again for NULL. Returns 1, or
 * 0 (and changes nothing) for an unknown name. Recording one kernel costs two
 * event records per launch of that kernel only. */
int32_t ptycho_profile_select(const char* name);
int32_t ptycho_profile_read(ptycho_kernel_time* out, int32_t cap);

/* Library version string. */
const char* ptycho_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PTYCHO_H */
