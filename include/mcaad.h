/*
 * mcaad.h -- C ABI of libmcaad.so: the Monte Carlo value and adjoint gradient
 * of the calibration objective
 *
 *     G(theta) = 1/2 sum_{i=1..m} (E y_i(theta) - C_i)^2            (eq. 241118A)
 *
 * of Goloubentsev & Lakshtanov, "Remarks on Automatic Adjoint Differentiation
 * for gradient descent and models calibration" (arXiv 1901.04200), computed
 * with the paper's two-step algorithm: step 1, E y_i by a forward sweep over
 * paths (eq. 1211A); step 2, per path, the reverse algorithm R seeded with
 * lambda_i = E y_i - C_i (eq. 0711A), re-running F from checkpoints because the
 * forward results are not all stored; step 3, the sum over paths.  Total cost
 * (2 K_F + K_R)/c * paths * Cost(F) (eq. 0711C).
 *
 * Conventions for every entry point:
 *  - All pointers are DEVICE pointers unless the name ends in `_host`.
 *    The caller owns every buffer it passes; the library never frees them.
 *  - Work is enqueued on the caller's `stream` (a cudaStream_t passed as
 *    void*; NULL = legacy default stream) and is asynchronous: outputs are
 *    valid once the stream reaches that point.
 *  - Every call returns an mc_status.  Argument errors are detected on the
 *    host before any work is enqueued (MC_ERR_INVALID_ARG, nothing written).
 *    A launch error returns MC_ERR_CUDA.  Errors from earlier asynchronous
 *    work surface in a later call or in mc_sync.  mc_last_error() gives a
 *    message owned by the context (valid until the next call on it).
 *  - A context is used from one host thread at a time; calls enqueued on
 *    different streams that share a context race on its workspace.
 *  - Floating-point inputs and outputs at the boundary are FP64.  Path
 *    arithmetic runs in the model's precision (MC_FP32 or MC_FP64); sums over
 *    paths, E y, lambda, G and grad G are FP64.
 *
 * Random numbers: normal j of global path p is Box-Muller on the
 * Philox-4x32-10 block (Salmon et al., SC'11) with counter
 * (j>>2 as 64-bit in words 0-1, p as 64-bit in words 2-3) and key
 * (seed & 0xffffffff, seed >> 32); u(w) = ((w >> 9) + 0.5) * 2^-23;
 * block words (o0,o1) give normals 0,1 and (o2,o3) give 2,3 with
 * rad = sqrt(-2 ln u(o_2q)), z_2q = rad cos(2 pi u(o_2q+1)),
 * z_2q+1 = rad sin(2 pi u(o_2q+1)).  Global path indices make results
 * independent of how a path range is split across calls or devices.
 */
#ifndef MCAAD_H
#define MCAAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MC_OK = 0,
    MC_ERR_INVALID_ARG = 1,
    MC_ERR_CUDA = 2,
    MC_ERR_OOM = 3,
    MC_ERR_UNSUPPORTED = 4,
    MC_ERR_STATE = 5
} mc_status;

typedef enum {
    MC_MODEL_GBM_PWC = 0,     /* GBM, piecewise-constant vol, log-Euler       */
    MC_MODEL_HESTON_FT = 1,   /* Heston, full-truncation Euler                */
    MC_MODEL_LV_BILINEAR = 2, /* local vol, bilinear node surface, log-Euler  */
    MC_MODEL_HESTON_SLV = 3   /* Heston stochastic local vol (leverage surface) */
} mc_model_kind;

typedef enum { MC_FP64 = 0, MC_FP32 = 1 } mc_precision;

/* How the reverse sweep gets the forward sweep's results (two-step algorithm,
 * step 2, stored results against recomputation):
 *   MC_STORAGE_CHECKPOINT  the state every ckpt_every steps; the reverse sweep
 *                          re-runs F between checkpoints, normals included
 *                          (cost K_F + K_R per path).
 *   MC_STORAGE_FULL        every step's tape (K_R only; HBM per path-step: the
 *                          model's tape fields x 4 or 8 bytes, written once and
 *                          read once).
 *   MC_STORAGE_NORMALS     the checkpoints and every normal drawn (1 per step
 *                          for GBM and LV, 2 for Heston and SLV, x 4 or 8 bytes
 *                          per path-step); the reverse sweep re-runs the model
 *                          step between checkpoints on the stored normals.
 *   MC_STORAGE_STATES      (local vol only) the state before every step (one
 *                          word per path-step, no normals, no checkpoints); the
 *                          reverse sweep runs only the adjoint, taking each
 *                          step's sqrt(dt) z from the states at its two ends
 *                          (the step's increment minus its drift, over sigma):
 *                          valid where the surface is nonzero along the paths
 *                          (a zero sigma gives a non-finite gradient).
 * All run the same forward step arithmetic, so E y is the same and the
 * gradients agree to rounding (the compiler may fuse a multiply and an add
 * differently in different kernels; the stored-states adjoint divides by
 * sigma).  The mode is fixed per context; mc_workspace_size accounts for the
 * storage it needs. */
typedef enum {
    MC_STORAGE_CHECKPOINT = 0,
    MC_STORAGE_FULL = 1,
    MC_STORAGE_NORMALS = 2,
    MC_STORAGE_AUTO = 3, /* local vol: STATES, the other models: NORMALS, when that storage for
                            max_paths takes at most a quarter of the device's total memory,
                            else CHECKPOINT */
    MC_STORAGE_STATES = 4
} mc_storage;

/*
 * The stochastic model F (paper: F maps M parameters and N random numbers to
 * the m payoffs of one path; Heston SLV test paragraph: Euler discretisation).
 * State x = ln(S/S0) starts at 0.  Step n (time n*dt) of each model:
 *   GBM_PWC:     theta[b] = vol of bucket b; step n is in the first bucket b
 *                with n < bucket_end_host[b];
 *                x += (r - theta_b^2/2) dt + theta_b sqrt(dt) z_n.       M = n_buckets
 *   HESTON_FT:   theta = (kappa, theta_h, xi, rho, v0); v+ = max(v,0);
 *                x += (r - v+/2) dt + sqrt(v+ dt) z1;
 *                v += kappa (theta_h - v+) dt + xi sqrt(v+ dt) (rho z1 + sqrt(1-rho^2) z2),
 *                z1, z2 = normals 2n, 2n+1; v starts at v0.             M = 5
 *                The gradient needs |rho| < 1: d sqrt(1-rho^2)/d rho is unbounded
 *                at |rho| = 1, where the rho component is not finite (theta
 *                lives on the device and is not checked on the host).
 *   LV_BILINEAR: theta[j*nx + c] = sigma at t_j = j t_max/(nt-1),
 *                x_c = x_lo + c (x_hi-x_lo)/(nx-1); sigma(t_n, x_n) bilinear
 *                with flat extrapolation;
 *                x += (r - sigma^2/2) dt + sigma sqrt(dt) z_n.           M = nt*nx
 *   HESTON_SLV:  theta = (kappa, theta_h, xi, rho, v0, L[j*nx + c]): the
 *                paper's test model (Heston SLV test paragraph); leverage L
 *                on the LV node grid, bilinear; v as HESTON_FT and
 *                x += (r - L^2 v+/2) dt + L sqrt(v+ dt) z1.         M = 5 + nt*nx
 * ckpt_every: checkpoint interval k of the reverse sweep (0 = library
 * default); it must divide every maturity step.
 * paths_per_thread: independent paths per GPU thread, 1 to 4 where that
 * (model, precision, ckpt_every) combination is built (MC_ERR_UNSUPPORTED
 * otherwise; 0 = library default); results agree to rounding of the FP32
 * warp sums.
 * normals: optional device FP64 table [rows][n_steps * normals_per_step]
 * (row = global path - normals_path0) used instead of Philox; GBM only.
 */
typedef struct {
    int32_t kind;        /* mc_model_kind */
    int32_t precision;   /* mc_precision  */
    double S0, r, dt;
    int32_t n_steps;
    int32_t ckpt_every;
    int32_t n_buckets;
    const int32_t *bucket_end_host;
    int32_t nt, nx;
    double t_max, x_lo, x_hi;
    const double *normals;
    uint64_t normals_path0;
    uint64_t normals_rows;
    int32_t paths_per_thread;
    int32_t storage;     /* mc_storage */
} mc_model;

/* European calls y_i = exp(-r T_i) max(S0 e^{x_{n_i}} - K_i, 0), T_i = n_i dt
 * (Heston SLV test paragraph: European options as the y_i).  Host arrays,
 * copied at context creation; 1 <= mat_step_host[i] <= n_steps. */
typedef struct {
    int32_t m;
    const double *K_host;
    const int32_t *mat_step_host;
} mc_instruments;

typedef struct mc_ctx mc_ctx;

/* Bytes of device workspace a context needs for up to max_paths paths per
 * call (checkpoints, per-block partial sums, seeds, model tables).
 * Errors: MC_ERR_INVALID_ARG for an invalid model/instruments (same checks
 * as mc_context_create). */
mc_status mc_workspace_size(const mc_model *model, const mc_instruments *inst,
                            uint64_t max_paths, int device, size_t *bytes_out);

/* Create a context on `device` for one model and instrument set (a plan:
 * tables and launch shapes are fixed here, nothing is allocated per call).
 * workspace: caller-owned device buffer of >= mc_workspace_size bytes,
 * 256-byte aligned; NULL makes the context cudaMalloc (and later free) its own.
 * The model's `normals` table pointer, if any, must stay valid for the
 * context's life.  Synchronous.  Errors: MC_ERR_INVALID_ARG (bad model,
 * maturities not multiples of ckpt_every, workspace too small or misaligned),
 * MC_ERR_OOM, MC_ERR_CUDA.  Tuning: the environment variables
 * MCAAD_MAX_BLOCKS_FWD / MCAAD_MAX_BLOCKS_REV (positive integers), read here,
 * cap the resident blocks per SM of the forward / reverse path kernels. */
mc_status mc_context_create(int device, const mc_model *model, const mc_instruments *inst,
                            uint64_t max_paths, void *workspace, size_t workspace_bytes,
                            mc_ctx **out);
void mc_context_destroy(mc_ctx *ctx);
const char *mc_last_error(const mc_ctx *ctx);
/* Parameter count M and instrument count m of a context. */
int32_t mc_n_params(const mc_ctx *ctx);
int32_t mc_n_instruments(const mc_ctx *ctx);
/* The storage mode a context runs (MC_STORAGE_AUTO resolved); -1 for a null context. */
int32_t mc_storage_mode(const mc_ctx *ctx);
/* Synchronise `stream` and report any asynchronous CUDA error. */
mc_status mc_sync(mc_ctx *ctx, void *stream);

/* Step 1 of the two-step algorithm (eq. 1211A): Ey_out[i] = mean over global
 * paths [path0, path0+n_paths) of y_i.  theta: FP64 [M]; Ey_out: FP64 [m].
 * keep_checkpoints != 0 stores the state every ckpt_every steps so that a
 * following mc_vjp can run the reverse sweep; theta must then stay unchanged
 * until that mc_vjp.  1 <= n_paths <= max_paths.  For a GBM normals table,
 * the paths must lie inside its rows. */
mc_status mc_forward(mc_ctx *ctx, const double *theta, uint64_t seed, uint64_t path0,
                     uint64_t n_paths, double *Ey_out, int keep_checkpoints, void *stream);

/* Steps 2-3 after mc_forward(keep_checkpoints=1): theta_bar_out[j] =
 * sum_i ybar[i] d(E y_i)/d theta_j for the last forward's paths and theta
 * (eq. 0711A per path, re-running F between checkpoints, then the mean over
 * paths).  ybar: FP64 [m]; theta_bar_out: FP64 [M].  MC_ERR_STATE if no
 * forward kept checkpoints. */
mc_status mc_vjp(mc_ctx *ctx, const double *ybar, double *theta_bar_out, void *stream);

/* The whole two-step algorithm: E y, lambda = E y - C, G = 1/2 |lambda|^2
 * (eq. 241118A) and grad G = E(sum_i lambda_i dy_i/dtheta) (gradient
 * identity), with no host round trip.  theta, grad_out: FP64 [M]; C: FP64 [m];
 * G_out: FP64 [1]; Ey_out: FP64 [m] or NULL.  Leaves checkpoints for mc_vjp. */
mc_status mc_value_and_grad(mc_ctx *ctx, const double *theta, const double *C, uint64_t seed,
                            uint64_t path0, uint64_t n_paths, double *G_out, double *grad_out,
                            double *Ey_out, void *stream);

/* Forward-mode Jacobian for many Heston parameter vectors (the gradient
 * identity's pathwise derivatives dy_i/dtheta_j, carried forward as five
 * tangents per path instead of one reverse sweep per instrument; the labels
 * of the pricing surrogate).  For t < n_theta: Ey_out[t][i] = mean of y_i and
 * J_out[t][i][j] = mean of dy_i/dtheta_j over global paths
 * [t n_paths, (t+1) n_paths) of `seed`, at thetas[t][0..5) (Heston contexts
 * only; MC_ERR_UNSUPPORTED otherwise).  strikes: optional FP64 [n_theta][m]
 * replacing the context's strikes per t (maturities stay the context's).
 * Ey_out (nullable) FP64 [n_theta][m]; J_out FP64 [n_theta][m][5]; scratch:
 * device buffer of mc_price_jacobian_scratch_size bytes.  Kink conventions
 * as the reverse sweep.  1 <= n_theta <= 65535. */
mc_status mc_price_jacobian_scratch_size(mc_ctx *ctx, int32_t n_theta, uint64_t n_paths, size_t *bytes_out);
mc_status mc_price_jacobian(mc_ctx *ctx, const double *thetas, const double *strikes, int32_t n_theta,
                            uint64_t seed, uint64_t n_paths, double *Ey_out, double *J_out, void *scratch,
                            size_t scratch_bytes, void *stream);

/* G and grad G by forward-mode tangents instead of the reverse sweep (Heston
 * contexts, M = 5): one sweep over global paths [path0, path0 + n_paths) of
 * `seed` carries d(x, v)/d theta_j along each path and gives E y_i and
 * J_ij = d E y_i / d theta_j; then lambda = E y - C, G = 1/2 |lambda|^2
 * (eq. 241118A) and grad G = J^T lambda (the gradient identity, with the
 * expectation taken per instrument before the contraction with lambda).  The
 * same estimator as mc_value_and_grad (same paths, normals and kink
 * conventions); its cost grows with M where the adjoint's does not, and it
 * stores nothing for a reverse sweep (so mc_vjp does not follow it).
 * theta, grad_out: FP64 [M]; C: FP64 [m]; G_out: FP64 [1]; Ey_out: FP64 [m]
 * or NULL; scratch: device buffer of mc_value_and_grad_tangent_scratch_size
 * bytes, 256-byte aligned. */
mc_status mc_value_and_grad_tangent_scratch_size(mc_ctx *ctx, uint64_t n_paths, size_t *bytes_out);
mc_status mc_value_and_grad_tangent(mc_ctx *ctx, const double *theta, const double *C, uint64_t seed,
                                    uint64_t path0, uint64_t n_paths, double *G_out, double *grad_out,
                                    double *Ey_out, void *scratch, size_t scratch_bytes, void *stream);

/* The tensor-core GEMM used by the pricing surrogate, as a plain operation:
 * D[s][M][N] (row stride ldd, slice stride M*ldd) = A[:, s*k_slice .. +k_slice)
 * B[:, same]^T for s < K / k_slice, with A [M][lda] and B [N][ldb] BF16 (K
 * contiguous), FP32 accumulation on tcgen05 tensor cores.  M % 128 == 0,
 * N % 16 == 0 and N <= 256, K and k_slice multiples of 64, lda/ldb multiples
 * of 8, A and B 16-byte aligned.  err: optional device int set to 1 if a
 * wait on the tensor cores exceeded its limit (the result is then invalid). */
mc_status mc_tc_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, int32_t M, int32_t N, int32_t K,
                          int32_t k_slice, float *D, int64_t ldd, int32_t *err, void *stream);

/* ---- Pricing surrogate (learned part; no counterpart in the paper, which
 * prices every calibration step by Monte Carlo).  MLP 7 -> 256 -> 256 -> 256
 * -> 256 -> 1, SiLU, input (Heston theta[5], K, T) normalised by the caller,
 * BF16 operands and FP32 accumulation on tcgen05 tensor cores, FP32 master
 * parameters in a flat caller-owned buffer of mlp_n_params() floats laid out
 * W1 [256][7], b1, W2 [256][256], b2, W3, b3, W4, b4, w5 [256], b5.
 * A context owns the activation workspace for `batch` rows (a multiple of 128)
 * and the BF16 copies of the weights; mlp_set_weights (or mlp_adam_step)
 * refreshes those copies from the FP32 parameters.  Stream-ordered; the
 * status conventions are those of the mc_ entry points. */
typedef struct mlp_ctx mlp_ctx;
int64_t mlp_n_params(void);
mc_status mlp_workspace_size(int32_t batch, size_t *bytes_out);
/* workspace: caller-owned device buffer (256-byte aligned, >= mlp_workspace_size)
 * or NULL to let the context allocate its own.  Synchronous (zeroes it). */
mc_status mlp_create(int device, int32_t batch, void *workspace, size_t workspace_bytes, mlp_ctx **out);
void mlp_destroy(mlp_ctx *ctx);
mc_status mlp_set_weights(mlp_ctx *ctx, const float *params, void *stream);
/* out[r] = net(X[r]) for r < n_rows <= batch; X FP32 [n_rows][7]; dout_dx
 * (nullable) FP32 [n_rows][7] = d net/d x (the input gradient). */
mc_status mlp_forward(mlp_ctx *ctx, const float *params, const float *X, int32_t n_rows, float *out,
                      float *dout_dx, void *stream);
/* Differential loss over one full batch, L = mean (net - y)^2 + alpha mean
 * sum_{j<5} (d net/d x_j - dy_j)^2, and its gradient with respect to every
 * parameter (double backward through the input gradient).  X [batch][7],
 * y [batch], dy [batch][5]; loss_out (nullable) FP32 [1]; grads FP32 [n_params]. */
mc_status mlp_loss_grad(mlp_ctx *ctx, const float *params, const float *X, const float *y, const float *dy,
                        float alpha, float *loss_out, float *grads, void *stream);
/* Adam (Kingma & Ba) step t >= 1 on the FP32 parameters and moments, then the
 * BF16 weight copies are refreshed. */
mc_status mlp_adam_step(mlp_ctx *ctx, float *params, const float *grads, float *m, float *v, int32_t t, float lr,
                        float beta1, float beta2, float eps, void *stream);
/* One training step: mlp_loss_grad on the batch (X [batch][7], y [batch], dy [batch][5]), then
 * mlp_adam_step t with learning rate lr (no counterpart in the paper: the learned surrogate).
 * The batch is first copied into buffers of the context, so the caller's batch may live
 * anywhere and change every step.  The first call with a given set of params, grads, loss_out,
 * m and v buffers and (alpha, beta1, beta2, eps) runs eagerly and then records the step as a
 * CUDA graph on a stream of the context; later calls with the same set replay that graph on
 * `stream`, with only t and lr changed, which removes the per-kernel launch cost of the ~40
 * kernels of a step.  Results equal those of mlp_loss_grad followed by mlp_adam_step.  Calls on
 * one context must not overlap on the GPU (they share its buffers). */
mc_status mlp_train_step(mlp_ctx *ctx, float *params, const float *X, const float *y, const float *dy, float alpha,
                         float *grads, float *loss_out, float *m, float *v, int32_t t, float lr, float beta1,
                         float beta2, float eps, void *stream);
/* Host copy of the tensor-core wait-expiry flag (0 = every wait completed). Synchronous. */
mc_status mlp_error_flag(mlp_ctx *ctx, int32_t *flag_host);

/* Test hooks for the generator of F's N random inputs (definition of F; the
 * paper names no generator: Philox-4x32-10 and Box-Muller as described at the
 * top of this file).  mc_philox_fill: out uint32
 * [n_paths][n_calls][4], block (call c, path path0+i).  mc_normals_fill:
 * out [n_paths][n_per_path] of normals 0.. of each path, FP64 when
 * precision == MC_FP64 (double*), else FP32 (float*), computed exactly as the
 * path kernels compute them. */
mc_status mc_philox_fill(uint64_t seed, uint64_t path0, uint32_t n_paths, uint32_t n_calls,
                         uint32_t *out, void *stream);
mc_status mc_normals_fill(uint64_t seed, uint64_t path0, uint32_t n_paths, uint32_t n_per_path,
                          int32_t precision, void *out, void *stream);

/* Per-kernel timing with CUDA events recorded on the launching stream around
 * every kernel the context launches (no counterpart in the paper; it measures
 * the terms of eq. 0711C).  Kernel ids: MC_K_FORWARD (forward sweep),
 * MC_K_FINALIZE_Y (E y / lambda / G), MC_K_SEED (mc_vjp seeds),
 * MC_K_REVERSE (reverse sweep), MC_K_FINALIZE_G (grad G), MC_K_TANGENT and
 * MC_K_FINALIZE_T (mc_value_and_grad_tangent).
 * mc_profile_begin creates events for up to max_launches launches (host
 * call).  mc_profile_end waits for the recorded events, writes the summed
 * milliseconds and kernel launches per kernel id into ms_out[MC_N_KERNELS]
 * and launches_out[MC_N_KERNELS] (either may be NULL; a finalize that first
 * folds many partial rows in a second kernel counts two launches under one
 * event pair, max_launches counts event pairs), and stops recording. */
enum { MC_K_FORWARD = 0, MC_K_FINALIZE_Y = 1, MC_K_SEED = 2, MC_K_REVERSE = 3, MC_K_FINALIZE_G = 4,
       MC_K_TANGENT = 5, MC_K_FINALIZE_T = 6, MC_N_KERNELS = 7 };
mc_status mc_profile_begin(mc_ctx *ctx, int32_t max_launches);
mc_status mc_profile_end(mc_ctx *ctx, double *ms_out, int32_t *launches_out);

/* E y with no device allocation at all: the same forward sweep and E y
 * finalize as mc_forward, for callers that cannot call cudaMalloc -- for
 * example code running in a process whose device memory is owned by another
 * allocator's pool, or a latency-critical loop that must not pay
 * cudaMalloc's implicit device synchronisation.  The paper has no
 * counterpart; it is a deployment convenience.
 * The caller passes the model, instruments (as for mc_context_create), theta
 * (FP64 [M], device) and Ey_out (FP64 [m], device); no context is needed.
 * Scratch (model tables and per-block partial sums) lives in one fixed
 * device array of MC_STATIC_SCRATCH_BYTES that every GPU loading the library
 * holds until the process exits.  The first call on a device looks up that
 * array's device address, so make the first call on each device before any
 * stream capture.  Each call copies the model tables into the array with one
 * cudaMemcpyAsync from pageable host memory, which waits for the work already
 * on the stream, unless they are byte-identical to the tables the previous
 * call on this device uploaded (then nothing is copied).  A path range that
 * wraps around 2^64 returns MC_ERR_INVALID_ARG.  The forward sweep's shared
 * memory is checked first: tables beyond it return MC_ERR_UNSUPPORTED.  A
 * problem whose tables and one row of partial sums exceed the array would
 * return MC_ERR_INVALID_ARG, but the shared-memory limit (which holds the same
 * tables) refuses every such problem first; that check is a backstop.  Every
 * call shares the array and leaves the last call's contents in it (nothing is
 * read before this call writes it); calls that overlap on the GPU, on any
 * stream, race on it.  No checkpoints are kept (use a context for mc_vjp). */
#define MC_STATIC_SCRATCH_BYTES ((size_t)4 << 20)
mc_status mc_forward_static(const mc_model *model, const mc_instruments *inst, const double *theta,
                            uint64_t seed, uint64_t path0, uint64_t n_paths, double *Ey_out,
                            void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MCAAD_H */
