// mc_api.cu -- host side of the C ABI declared in include/mcaad.h: argument
// checks, the context (a plan holding the model tables, launch shapes and
// workspace), and the stream-ordered launch sequences of the two-step
// algorithm (arXiv 1901.04200): forward sweep -> finalize (E y, lambda, G)
// -> reverse sweep -> finalize (grad G).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "mcaad.h"
#include "mc_internal.h"
#include "mc_paths.cuh"

using namespace mcaad;

// The path kernels a context launches (chosen by its storage mode) and their
// shapes: the forward sweep without checkpoints (mc_forward alone), the
// forward sweep that leaves what the reverse sweep reads, the reverse sweep.
struct Launch {
    const void *fwd = nullptr, *fwd_keep = nullptr, *rev = nullptr;
    int grid_fwd = 1, grid_fwd_keep = 1, grid_rev = 1;  // (resident blocks per SM) x SMs
    size_t smem_fwd = 0, smem_rev = 0;
    int grid_max() const {
        const int g = grid_fwd > grid_fwd_keep ? grid_fwd : grid_fwd_keep;
        return g > grid_rev ? g : grid_rev;
    }
};

struct mc_ctx {
    int device = 0;
    int kind = 0, precision = 0, K = 1, ppt = 1;
    int m = 0, M = 0, n_groups = 0, n_seg = 0, state_dim = 1;
    uint64_t max_paths = 0, ckpt_stride = 0;
    int n_sm = 1;
    int grid_max = 1;
    int storage = 0;  // mc_storage
    KernelPair kern;
    Launch ln;        // the kernels of the storage mode and their launch shapes
    DevProblem pb{};
    // workspace
    bool owns_ws = false;
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0;
    void *ckpt = nullptr;
    void *tape = nullptr, *xmat = nullptr;
    double *part_y = nullptr, *part_g = nullptr, *seed_w = nullptr, *lam2 = nullptr;
    double *part1_y = nullptr, *part1_g = nullptr;  // first-level sums of the finalize
    unsigned int *ticket = nullptr;
    unsigned long long *queue = nullptr;  // the path sweeps' chunk queue (two words, zero between launches)
    // state for mc_vjp
    bool have_ckpt = false;
    DevCall last{};
    std::string err;
    // per-kernel event timing
    bool prof_on = false;
    int prof_max = 0, prof_n = 0;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_id, prof_k;  // per bracket: kernel part, kernels launched
};

namespace {

mc_status fail(mc_ctx *ctx, mc_status st, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
mc_status fail(mc_ctx *ctx, mc_status st, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

mc_status cuda_fail(mc_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? MC_ERR_OOM : MC_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

const int kGbmK[] = {16, 8, 4, 2, 1};
const int kHestonK[] = {8, 4, 2, 1};
const int kLvK[] = {25, 5, 1};

int model_params(const mc_model *md) {
    switch (md->kind) {
    case MC_MODEL_GBM_PWC: return md->n_buckets;
    case MC_MODEL_HESTON_FT: return 5;
    case MC_MODEL_LV_BILINEAR: return md->nt * md->nx;
    case MC_MODEL_HESTON_SLV: return 5 + md->nt * md->nx;
    }
    return -1;
}

bool kernels_raw(int kind, int precision, int K, int ppt, KernelPair *kp) {
    switch (kind) {
    case kGbm: return gbm_kernels(precision, K, ppt, kp);
    case kHeston: return heston_kernels(precision, K, ppt, kp);
    case kLv: return lv_kernels(precision, K, ppt, kp);
    case kSlv: return slv_kernels(precision, K, ppt, kp);
    }
    return false;
}

// Paths per thread when the model leaves it at 0: two independent Heston
// recursions per thread measured fastest in FP32 (K = 8: 2.69 ms against
// 2.93 ms per value-and-gradient on 2^20 x 512 paths).
int default_ppt(int kind, int precision) { return (kind == kHeston && precision == MC_FP32) ? 2 : 1; }

// Path stride of the workspace arrays: whole pairs of warp chunks (64 * ppt paths), so the
// segment tiles of every chunk of a call fit.
uint64_t path_stride(uint64_t max_paths, int ppt) {
    const uint64_t q = 2 * (uint64_t)kWarp * (uint64_t)ppt;
    return (max_paths + q - 1) / q * q;
}

// Everything a context derives from (model, instruments), computed on the host.
struct Plan {
    int kind, precision, K, ppt, n_last, n_seg, m, M, n_groups, state_dim, storage, tape_fields, dz;
    std::vector<int> order;  // sorted position -> caller index
    std::vector<double> strike, disc;
    std::vector<int> perm, grp_seg, grp_begin, bucket, lv_jt;
    std::vector<double> lv_a;
    double hx = 1.0;
};

mc_status make_plan(const mc_model *md, const mc_instruments *in, Plan &p, std::string &why) {
    char buf[256];
    auto bad = [&](const char *msg) {
        why = msg;
        return MC_ERR_INVALID_ARG;
    };
    if (!md || !in) return bad("null model or instruments");
    if (md->kind < 0 || md->kind > 3) return bad("unknown model kind");
    if (md->precision != MC_FP32 && md->precision != MC_FP64) return bad("unknown precision");
    if (!(md->S0 > 0.0) || !(md->dt > 0.0) || !std::isfinite(md->r)) return bad("need S0 > 0, dt > 0, finite r");
    if (md->n_steps < 1) return bad("n_steps must be >= 1");
    if (in->m < 1 || in->m > kMaxInstruments) return bad("instrument count out of range [1, 1024]");
    if (!in->K_host || !in->mat_step_host) return bad("null instrument arrays");
    p.kind = md->kind;
    p.precision = md->precision;
    p.m = in->m;
    p.M = model_params(md);
    if (p.M < 1 || p.M > kMaxParams) return bad("parameter count out of range [1, 256]");
    const bool lv_grid = md->kind == MC_MODEL_LV_BILINEAR || md->kind == MC_MODEL_HESTON_SLV;
    p.state_dim = (md->kind == MC_MODEL_HESTON_FT || md->kind == MC_MODEL_HESTON_SLV) ? 2 : 1;
    int n_last = 0, g = 0;
    for (int i = 0; i < in->m; ++i) {
        const int s = in->mat_step_host[i];
        if (s < 1 || s > md->n_steps) return bad("maturity step outside [1, n_steps]");
        if (!std::isfinite(in->K_host[i])) return bad("non-finite strike");
        n_last = s > n_last ? s : n_last;
        g = std::gcd(g, s);
    }
    p.n_last = n_last;
    if (md->kind == MC_MODEL_GBM_PWC) {
        if (md->n_buckets < 1 || !md->bucket_end_host) return bad("GBM needs bucket ends");
        for (int b = 0; b < md->n_buckets; ++b) {
            const int prev = b ? md->bucket_end_host[b - 1] : 0;
            if (md->bucket_end_host[b] <= prev) return bad("bucket ends must increase");
        }
        if (md->bucket_end_host[md->n_buckets - 1] < n_last) return bad("buckets end before the last maturity");
    } else if (md->normals) {
        return bad("a normals table is supported for GBM only");
    }
    if (lv_grid) {
        if (md->nt < 2 || md->nx < 2 || !(md->t_max > 0.0) || !(md->x_hi > md->x_lo))
            return bad("LV needs nt, nx >= 2, t_max > 0, x_hi > x_lo");
        if (md->nx > 32) return bad("LV needs nx <= 32");
    }
    if (md->paths_per_thread < 0 || md->paths_per_thread > 4) return bad("paths_per_thread must be in [0, 4]");
    if (md->storage < MC_STORAGE_CHECKPOINT || md->storage > MC_STORAGE_STATES) return bad("unknown storage mode");
    if (md->storage == MC_STORAGE_STATES && md->kind != MC_MODEL_LV_BILINEAR) {
        why = "stored states are implemented for local vol only";
        return MC_ERR_UNSUPPORTED;
    }
    p.storage = md->storage;
    p.dz = p.state_dim;  // normals per step: 1 (GBM, LV) or 2 (Heston, SLV)
    p.tape_fields = md->kind == MC_MODEL_GBM_PWC ? 1 : md->kind == MC_MODEL_HESTON_FT ? 4 : md->kind == MC_MODEL_LV_BILINEAR ? 2 : 5;
    p.ppt = md->paths_per_thread ? md->paths_per_thread : default_ppt(md->kind, md->precision);
    // segment length: must divide every maturity step
    const bool hs_k = md->kind == MC_MODEL_HESTON_FT || md->kind == MC_MODEL_HESTON_SLV;
    const int *ks = md->kind == MC_MODEL_GBM_PWC ? kGbmK : hs_k ? kHestonK : kLvK;
    const int nk = md->kind == MC_MODEL_GBM_PWC ? 5 : hs_k ? 4 : 3;
    KernelPair probe;
    p.K = 0;
    if (md->ckpt_every > 0) {
        if (g % md->ckpt_every != 0) {
            snprintf(buf, sizeof buf, "ckpt_every=%d does not divide every maturity step (gcd %d)",
                     md->ckpt_every, g);
            why = buf;
            return MC_ERR_INVALID_ARG;
        }
        if (kernels_raw(md->kind, md->precision, md->ckpt_every, p.ppt, &probe)) p.K = md->ckpt_every;
        if (!p.K) {
            snprintf(buf, sizeof buf, "ckpt_every=%d with %d paths per thread is not instantiated",
                     md->ckpt_every, p.ppt);
            why = buf;
            return MC_ERR_UNSUPPORTED;
        }
    } else {
        for (int q = 0; q < nk && !p.K; ++q)
            if (g % ks[q] == 0 && kernels_raw(md->kind, md->precision, ks[q], p.ppt, &probe)) p.K = ks[q];
        if (!p.K) {
            why = "no instantiated segment length divides every maturity step";
            return MC_ERR_UNSUPPORTED;
        }
    }
    p.n_seg = n_last / p.K;
    // instruments sorted by maturity (stable), grouped per maturity step
    p.order.resize(p.m);
    std::iota(p.order.begin(), p.order.end(), 0);
    std::stable_sort(p.order.begin(), p.order.end(),
                     [&](int a, int b) { return in->mat_step_host[a] < in->mat_step_host[b]; });
    p.strike.resize(p.m);
    p.disc.resize(p.m);
    p.perm.resize(p.m);
    p.grp_begin.clear();
    p.grp_seg.clear();
    int prev = -1;
    for (int q = 0; q < p.m; ++q) {
        const int i = p.order[q];
        const int s = in->mat_step_host[i];
        p.strike[q] = in->K_host[i];
        p.disc[q] = std::exp(-md->r * (double)s * md->dt);
        p.perm[q] = i;
        if (s != prev) {
            p.grp_begin.push_back(q);
            p.grp_seg.push_back(s / p.K - 1);
            prev = s;
        }
    }
    p.n_groups = (int)p.grp_seg.size();
    p.grp_begin.push_back(p.m);
    if (md->kind == MC_MODEL_GBM_PWC) {
        p.bucket.resize(n_last);
        int b = 0;
        for (int n = 0; n < n_last; ++n) {
            while (n >= md->bucket_end_host[b]) ++b;
            p.bucket[n] = b;
        }
    }
    if (lv_grid) {
        // time cell and weight of step n, in FP64 as u_t = (n dt) / (t_max / (nt - 1))
        const double ht = md->t_max / (double)(md->nt - 1);
        p.lv_jt.resize(n_last);
        p.lv_a.resize(n_last);
        for (int n = 0; n < n_last; ++n) {
            const double ut = ((double)n * md->dt) / ht;
            int jt = (int)std::floor(ut);
            jt = jt < 0 ? 0 : (jt > md->nt - 2 ? md->nt - 2 : jt);
            double a = ut - (double)jt;
            a = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
            p.lv_jt[n] = jt;
            p.lv_a[n] = a;
        }
        p.hx = (md->x_hi - md->x_lo) / (double)(md->nx - 1);
    }
    return MC_OK;
}

// Workspace carve-out (256-byte aligned pieces).
struct WsLayout {
    size_t strike, disc, perm, grp_seg, grp_begin, bucket, lv_jt, lv_a, seed_w, lam2, ticket, queue, part_y, part_g,
        part1_y, part1_g,
        ckpt, tape, xmat, total;
    WsLayout(const Plan &p, int grid_max, uint64_t ckpt_stride) {
        size_t o = 0;
        auto take = [&](size_t bytes) {
            size_t at = o;
            o = align_up(o + bytes, 256);
            return at;
        };
        strike = take(p.m * 8);
        disc = take(p.m * 8);
        perm = take(p.m * 4);
        grp_seg = take(p.n_groups * 4);
        grp_begin = take((p.n_groups + 1) * 4);
        bucket = take(p.bucket.size() * 4);
        lv_jt = take(p.lv_jt.size() * 4);
        lv_a = take(p.lv_a.size() * 8);
        seed_w = take(p.m * 8);
        lam2 = take(p.m * 8);
        ticket = take(4);
        queue = take(16);
        // partial sums: one row per block (static chunk assignment) or per warp chunk (queue)
        const size_t part_rows = std::max((size_t)grid_max, ckpt_stride / (32 * (size_t)p.ppt));
        part_y = take(part_rows * p.m * 8);
        part_g = take(part_rows * p.M * 8);
        const size_t rows1 = (part_rows + kRowsPerBlock - 1) / kRowsPerBlock;
        part1_y = take(rows1 * p.m * 8);
        part1_g = take(rows1 * p.M * 8);
        const size_t real = p.precision == MC_FP64 ? 8 : 4;
        // checkpoint tiles (SegTile): per warp chunk of 32*ppt paths and segment, the state
        // words and, with stored normals, the segment's K * dz normals of each path, in rows of
        // 32 paths padded to whole 16-byte groups; ckpt_stride covers whole chunks
        // (stored states: the state before each step of the segment, no checkpoint rows, and one
        // extra tile for the state after the last step)
        const bool full = p.storage == MC_STORAGE_FULL, states = p.storage == MC_STORAGE_STATES;
        const size_t rows = states ? (size_t)p.ppt * p.K * p.state_dim
                                   : (size_t)p.ppt * (p.state_dim + (p.storage == MC_STORAGE_NORMALS ? (size_t)p.K * p.dz : 0));
        const size_t group = 16 / real;
        const size_t rows_padded = (rows + group - 1) / group * group;
        const size_t chunks = ckpt_stride / (32 * (size_t)p.ppt);
        const size_t tiles = (size_t)p.n_seg + (states ? 1 : 0);
        ckpt = take(full ? 0 : tiles * chunks * rows_padded * 32 * real);
        tape = take(full ? (size_t)p.n_last * p.tape_fields * ckpt_stride * real : 0);
        xmat = take(full ? (size_t)p.n_groups * ckpt_stride * real : 0);
        total = o;
    }
};

// MC_STORAGE_AUTO: the stored normals when they take at most a quarter of the
// device's total memory (a fixed property, so mc_workspace_size and
// mc_context_create resolve alike), else checkpoints alone.
mc_status resolve_storage(Plan &p, uint64_t max_paths, int device, std::string &why) {
    if (p.storage != MC_STORAGE_AUTO) return MC_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    size_t free_b = 0, total_b = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        why = cudaGetErrorString(e);
        return MC_ERR_CUDA;
    }
    const uint64_t stride = path_stride(max_paths, p.ppt);
    // local vol stores its states (one word per path-step), the other models their normals
    const bool states = p.kind == MC_MODEL_LV_BILINEAR;
    const double bytes = (double)p.n_last * (states ? p.state_dim : p.dz) * (double)stride * (p.precision == MC_FP64 ? 8 : 4);
    p.storage = bytes <= 0.25 * (double)total_b ? (states ? MC_STORAGE_STATES : MC_STORAGE_NORMALS) : MC_STORAGE_CHECKPOINT;
    return MC_OK;
}

bool kernels_for(const Plan &p, KernelPair *kp) { return kernels_raw(p.kind, p.precision, p.K, p.ppt, kp); }

// Launch shape: blocks of kBlock threads, at most (resident blocks per SM) x
// (SMs) of them; each warp loops over 32-path chunks.  The environment
// variables MCAAD_MAX_BLOCKS_FWD / MCAAD_MAX_BLOCKS_REV (positive integers) cap
// the resident blocks per SM of the forward / reverse path kernels, for tuning.
int env_int(const char *name) {
    const char *v = getenv(name);
    return v ? atoi(v) : 0;
}

// Raise a kernel's dynamic shared-memory limit to at least `bytes`, never lower it: every
// context and call that shares the kernel keeps the limit it was planned with.
static std::mutex g_smem_mu;
cudaError_t ensure_smem(const void *fn, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_smem_mu);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void block_caps(int *fwd, int *rev) {
    *fwd = env_int("MCAAD_MAX_BLOCKS_FWD") > 0 ? env_int("MCAAD_MAX_BLOCKS_FWD") : 0;
    *rev = env_int("MCAAD_MAX_BLOCKS_REV") > 0 ? env_int("MCAAD_MAX_BLOCKS_REV") : 0;
}

// The forward sweep's shape alone (mc_forward_static): its shared memory and
// resident blocks, (blocks per SM) x SMs.
mc_status forward_shape(const Plan &p, int device, const void *fwd, int nx, int *grid, size_t *smem,
                        std::string &why) {
    int n_sm = 1;
    cudaError_t e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        why = cudaGetErrorString(e);
        return MC_ERR_CUDA;
    }
    const int real = p.precision == MC_FP64 ? 8 : 4;
    *smem = SmemPlan(p.kind, real, p.m, p.n_groups, p.M, p.n_seg * p.K, nx, false).total;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (*smem > (size_t)optin) {
        why = "problem tables exceed shared memory";
        return MC_ERR_UNSUPPORTED;
    }
    e = ensure_smem(fwd, *smem);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fwd, kBlock, *smem);
    if (e != cudaSuccess || occ < 1) {
        why = e != cudaSuccess ? cudaGetErrorString(e) : "path kernel does not fit on an SM";
        return e != cudaSuccess ? MC_ERR_CUDA : MC_ERR_UNSUPPORTED;
    }
    int cap_fwd, cap_rev;
    block_caps(&cap_fwd, &cap_rev);
    if (cap_fwd > 0 && occ > cap_fwd) occ = cap_fwd;
    *grid = occ * n_sm;
    return MC_OK;
}

mc_status launch_shape(const Plan &p, int device, const KernelPair &kp, int nx, int *n_sm, Launch &ln,
                       std::string &why) {
    cudaError_t e = cudaDeviceGetAttribute(n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        why = cudaGetErrorString(e);
        return MC_ERR_CUDA;
    }
    const int real = p.precision == MC_FP64 ? 8 : 4;
    const int n_steps = p.n_seg * p.K;
    const size_t zst = p.storage == MC_STORAGE_NORMALS      ? kp.stage_bytes_z
                       : p.storage == MC_STORAGE_CHECKPOINT ? kp.stage_bytes_ckpt
                       : p.storage == MC_STORAGE_STATES     ? kp.stage_bytes_x
                                                            : 0;
    ln.smem_fwd = SmemPlan(p.kind, real, p.m, p.n_groups, p.M, n_steps, nx, false).total;
    ln.smem_rev = SmemPlan(p.kind, real, p.m, p.n_groups, p.M, n_steps, nx, true, zst,
                           p.storage == MC_STORAGE_STATES ||
                               (p.storage == MC_STORAGE_CHECKPOINT && kp.rev_node_table)).total;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (ln.smem_fwd > (size_t)optin || ln.smem_rev > (size_t)optin) {
        why = "problem tables exceed shared memory";
        return MC_ERR_UNSUPPORTED;
    }
    ln.fwd = kp.fwd;
    ln.fwd_keep = p.storage == MC_STORAGE_FULL      ? kp.fwd_store
                  : p.storage == MC_STORAGE_NORMALS ? kp.fwd_z
                  : p.storage == MC_STORAGE_STATES  ? kp.fwd_x
                                                    : kp.fwd;
    ln.rev = p.storage == MC_STORAGE_FULL      ? kp.rev_tape
             : p.storage == MC_STORAGE_NORMALS ? kp.rev_z
             : p.storage == MC_STORAGE_STATES  ? kp.rev_x
                                               : kp.rev;
    if (!ln.fwd_keep || !ln.rev) {
        why = "storage mode not instantiated for this model";
        return MC_ERR_UNSUPPORTED;
    }
    const void *fns[3] = {ln.fwd, ln.fwd_keep, ln.rev};
    const size_t sm[3] = {ln.smem_fwd, ln.smem_fwd, ln.smem_rev};
    int *grids[3] = {&ln.grid_fwd, &ln.grid_fwd_keep, &ln.grid_rev};
    int cap_fwd, cap_rev;
    block_caps(&cap_fwd, &cap_rev);
    const int caps[3] = {cap_fwd, cap_fwd, cap_rev};
    for (int q = 0; q < 3; ++q) {
        e = ensure_smem(fns[q], sm[q]);
        if (e != cudaSuccess) {
            why = cudaGetErrorString(e);
            return MC_ERR_CUDA;
        }
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fns[q], kBlock, sm[q]);
        if (e != cudaSuccess || occ < 1) {
            why = e != cudaSuccess ? cudaGetErrorString(e) : "path kernel does not fit on an SM";
            return e != cudaSuccess ? MC_ERR_CUDA : MC_ERR_UNSUPPORTED;
        }
        if (caps[q] > 0 && occ > caps[q]) occ = caps[q];
        *grids[q] = occ * *n_sm;
    }
    return MC_OK;
}

// Blocks for a launch over n_paths: up to grid_max = (resident blocks per SM)
// x (SMs), each warp looping over 32*ppt-path chunks.  Every chunk costs the
// same, so the time goes with the number of rounds, ceil(chunks / warps); with
// n_sm given, fewer resident blocks per SM b (down to occ/2) are used only when
// that makes the rounds at least 2 % fuller than at full occupancy (fewer
// warps hide less latency).
int grid_for_paths(int grid_max, uint64_t n_paths, int ppt, int n_sm = 0) {
    const uint64_t chunks = (n_paths + (uint64_t)kWarp * ppt - 1) / ((uint64_t)kWarp * ppt);
    const uint64_t want = (chunks + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (want <= (uint64_t)grid_max || n_sm <= 0 || grid_max % n_sm) return (int)(want < (uint64_t)grid_max ? want : grid_max);
    const int occ = grid_max / n_sm;
    auto eff = [&](int b) {
        const uint64_t warps = (uint64_t)b * n_sm * kWarpsPerBlock;
        const uint64_t rounds = (chunks + warps - 1) / warps;
        return (double)chunks / (double)(rounds * warps);
    };
    int best_b = occ;
    double best_eff = eff(occ);
    for (int b = occ - 1; b >= (occ + 1) / 2; --b) {
        const double e = eff(b);
        if (e > best_eff + 0.02) {
            best_eff = e;
            best_b = b;
        }
    }
    return best_b * n_sm;
}

// Warp chunks of n_paths (32 * ppt paths each).
uint64_t chunk_count(uint64_t n_paths, int ppt) { return (n_paths + (uint64_t)kWarp * ppt - 1) / ((uint64_t)kWarp * ppt); }

// Blocks of a queue-fed sweep: every resident block (no round to balance), at most one warp per
// chunk.
int queue_grid(int grid_max, uint64_t n_paths, int ppt) {
    const uint64_t want = (chunk_count(n_paths, ppt) + kWarpsPerBlock - 1) / kWarpsPerBlock;
    return (int)(want < (uint64_t)grid_max ? want : grid_max);
}

cudaError_t launch(const void *fn, int grid, size_t smem, const DevProblem &pb, const DevCall &cl,
                   cudaStream_t st) {
    void *args[2] = {(void *)&pb, (void *)&cl};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kBlock), args, smem, st);
}

// Launch f() (`kernels` kernel launches) on st; when profiling, bracket it with events tagged `id`.
template <class F>
cudaError_t timed(mc_ctx *ctx, int id, cudaStream_t st, F &&f, int kernels = 1) {
    const bool rec = ctx->prof_on && ctx->prof_n < ctx->prof_max;
    if (rec) cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], st);
    cudaError_t e = f();
    if (rec) {
        cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n + 1], st);
        ctx->prof_id[ctx->prof_n] = id;
        ctx->prof_k[ctx->prof_n++] = kernels;
    }
    return e;
}

void prof_free(mc_ctx *ctx) {
    for (cudaEvent_t ev : ctx->prof_ev) cudaEventDestroy(ev);
    ctx->prof_ev.clear();
    ctx->prof_id.clear();
    ctx->prof_k.clear();
    ctx->prof_on = false;
    ctx->prof_max = ctx->prof_n = 0;
}

template <typename T>
bool aligned8(const T *p) {
    return ((uintptr_t)p & 7u) == 0;
}

}  // namespace

extern "C" {

mc_status mc_workspace_size(const mc_model *model, const mc_instruments *inst, uint64_t max_paths,
                            int device, size_t *bytes_out) {
    if (!bytes_out || max_paths == 0) return MC_ERR_INVALID_ARG;
    Plan p;
    std::string why;
    mc_status st = make_plan(model, inst, p, why);
    if (st != MC_OK) return st;
    st = resolve_storage(p, max_paths, device, why);
    if (st != MC_OK) return st;
    KernelPair kp;
    if (!kernels_for(p, &kp)) return MC_ERR_UNSUPPORTED;
    int n_sm;
    Launch ln;
    st = launch_shape(p, device, kp, model->nx, &n_sm, ln, why);
    if (st != MC_OK) return st;
    const uint64_t stride = path_stride(max_paths, p.ppt);
    *bytes_out = WsLayout(p, ln.grid_max(), stride).total;
    return MC_OK;
}

mc_status mc_context_create(int device, const mc_model *model, const mc_instruments *inst,
                            uint64_t max_paths, void *workspace, size_t workspace_bytes,
                            mc_ctx **out) {
    if (!out) return MC_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_paths == 0) return MC_ERR_INVALID_ARG;
    Plan p;
    std::string why;
    mc_status st = make_plan(model, inst, p, why);
    if (st == MC_OK) st = resolve_storage(p, max_paths, device, why);
    if (st != MC_OK) {
        fprintf(stderr, "mc_context_create: %s\n", why.c_str());
        return st;
    }
    KernelPair kp;
    if (!kernels_for(p, &kp)) return MC_ERR_UNSUPPORTED;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        fprintf(stderr, "mc_context_create: cudaSetDevice: %s\n", cudaGetErrorString(e));
        return MC_ERR_CUDA;
    }
    mc_ctx *ctx = new (std::nothrow) mc_ctx();
    if (!ctx) return MC_ERR_OOM;
    ctx->device = device;
    ctx->kind = p.kind;
    ctx->precision = p.precision;
    ctx->K = p.K;
    ctx->ppt = p.ppt;
    ctx->m = p.m;
    ctx->M = p.M;
    ctx->n_groups = p.n_groups;
    ctx->n_seg = p.n_seg;
    ctx->state_dim = p.state_dim;
    ctx->kern = kp;
    ctx->storage = p.storage;
    st = launch_shape(p, device, kp, model->nx, &ctx->n_sm, ctx->ln, why);
    if (st != MC_OK) {
        fprintf(stderr, "mc_context_create: %s\n", why.c_str());
        delete ctx;
        return st;
    }
    ctx->grid_max = ctx->ln.grid_max();
    ctx->max_paths = max_paths;
    ctx->ckpt_stride = path_stride(max_paths, p.ppt);
    WsLayout L(p, ctx->grid_max, ctx->ckpt_stride);
    if (workspace) {
        if (workspace_bytes < L.total || ((uintptr_t)workspace & 255u)) {
            fprintf(stderr, "mc_context_create: workspace needs %zu bytes, 256-byte aligned\n", L.total);
            delete ctx;
            return MC_ERR_INVALID_ARG;
        }
        ctx->ws = (unsigned char *)workspace;
        ctx->owns_ws = false;
    } else {
        e = cudaMalloc((void **)&ctx->ws, L.total);
        if (e != cudaSuccess) {
            fprintf(stderr, "mc_context_create: cudaMalloc(%zu): %s\n", L.total, cudaGetErrorString(e));
            delete ctx;
            return e == cudaErrorMemoryAllocation ? MC_ERR_OOM : MC_ERR_CUDA;
        }
        ctx->owns_ws = true;
    }
    ctx->ws_bytes = L.total;
    unsigned char *w = ctx->ws;
    auto up = [&](size_t off, const void *src, size_t bytes) {
        return bytes ? cudaMemcpy(w + off, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    e = up(L.strike, p.strike.data(), p.m * 8);
    if (e == cudaSuccess) e = up(L.disc, p.disc.data(), p.m * 8);
    if (e == cudaSuccess) e = up(L.perm, p.perm.data(), p.m * 4);
    if (e == cudaSuccess) e = up(L.grp_seg, p.grp_seg.data(), p.n_groups * 4);
    if (e == cudaSuccess) e = up(L.grp_begin, p.grp_begin.data(), (p.n_groups + 1) * 4);
    if (e == cudaSuccess) e = up(L.bucket, p.bucket.data(), p.bucket.size() * 4);
    if (e == cudaSuccess) e = up(L.lv_jt, p.lv_jt.data(), p.lv_jt.size() * 4);
    if (e == cudaSuccess) e = up(L.lv_a, p.lv_a.data(), p.lv_a.size() * 8);
    if (e == cudaSuccess) e = cudaMemset(w + L.ticket, 0, 4);
    if (e == cudaSuccess) e = cudaMemset(w + L.queue, 0, 16);
    if (e != cudaSuccess) {
        fprintf(stderr, "mc_context_create: table upload: %s\n", cudaGetErrorString(e));
        mc_context_destroy(ctx);
        return MC_ERR_CUDA;
    }
    ctx->ckpt = w + L.ckpt;
    ctx->tape = w + L.tape;
    ctx->xmat = w + L.xmat;
    ctx->part_y = (double *)(w + L.part_y);
    ctx->part_g = (double *)(w + L.part_g);
    ctx->part1_y = (double *)(w + L.part1_y);
    ctx->part1_g = (double *)(w + L.part1_g);
    ctx->seed_w = (double *)(w + L.seed_w);
    ctx->lam2 = (double *)(w + L.lam2);
    ctx->ticket = (unsigned int *)(w + L.ticket);
    ctx->queue = (unsigned long long *)(w + L.queue);
    DevProblem &pb = ctx->pb;
    pb.kind = p.kind;
    pb.K = p.K;
    pb.n_seg = p.n_seg;
    pb.m = p.m;
    pb.M = p.M;
    pb.n_groups = p.n_groups;
    pb.S0 = model->S0;
    pb.r = model->r;
    pb.dt = model->dt;
    pb.strike = (const double *)(w + L.strike);
    pb.disc = (const double *)(w + L.disc);
    pb.perm = (const int *)(w + L.perm);
    pb.grp_seg = (const int *)(w + L.grp_seg);
    pb.grp_begin = (const int *)(w + L.grp_begin);
    pb.bucket_of_step = (const int *)(w + L.bucket);
    pb.lv_jt = (const int *)(w + L.lv_jt);
    pb.lv_a = (const double *)(w + L.lv_a);
    pb.nt = model->nt;
    pb.nx = model->nx;
    pb.x_lo = model->x_lo;
    pb.hx = p.hx;
    pb.normals = model->normals;
    pb.normals_path0 = model->normals_path0;
    pb.normals_rows = model->normals_rows;
    pb.normals_stride = model->n_steps * (p.state_dim == 2 ? 2 : 1);
    *out = ctx;
    return MC_OK;
}

void mc_context_destroy(mc_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    prof_free(ctx);
    if (ctx->owns_ws && ctx->ws) cudaFree(ctx->ws);
    delete ctx;
}

const char *mc_last_error(const mc_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }
int32_t mc_n_params(const mc_ctx *ctx) { return ctx ? ctx->M : -1; }
int32_t mc_n_instruments(const mc_ctx *ctx) { return ctx ? ctx->m : -1; }
int32_t mc_storage_mode(const mc_ctx *ctx) { return ctx ? ctx->storage : -1; }

mc_status mc_sync(mc_ctx *ctx, void *stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    return MC_OK;
}

static mc_status check_call(mc_ctx *ctx, const double *theta, uint64_t path0, uint64_t n_paths) {
    if (!theta || !aligned8(theta)) return fail(ctx, MC_ERR_INVALID_ARG, "theta must be a non-null FP64 device pointer");
    if (n_paths == 0 || n_paths > ctx->max_paths)
        return fail(ctx, MC_ERR_INVALID_ARG, "n_paths=%llu outside [1, max_paths=%llu]",
                    (unsigned long long)n_paths, (unsigned long long)ctx->max_paths);
    if (path0 + n_paths < path0) return fail(ctx, MC_ERR_INVALID_ARG, "path range overflows");
    if (ctx->pb.normals) {
        if (path0 < ctx->pb.normals_path0 || path0 + n_paths > ctx->pb.normals_path0 + ctx->pb.normals_rows)
            return fail(ctx, MC_ERR_INVALID_ARG, "paths outside the normals table");
    }
    return MC_OK;
}

static mc_status do_forward(mc_ctx *ctx, const double *theta, uint64_t seed, uint64_t path0,
                            uint64_t n_paths, int keep, cudaStream_t st, DevCall &cl, int &grid) {
    cl = DevCall{};
    cl.theta = theta;
    cl.seed = seed;
    cl.rk = philox_round_keys(seed);
    cl.path0 = path0;
    cl.n_paths = n_paths;
    cl.ckpt = ctx->ckpt;
    cl.ckpt_stride = ctx->ckpt_stride;
    cl.keep_ckpt = keep;
    cl.part_y = ctx->part_y;
    cl.part_g = ctx->part_g;
    cl.seed_w = ctx->seed_w;
    cl.tape = ctx->tape;
    cl.xmat = ctx->xmat;
    const Launch &ln = ctx->ln;
    // the sweeps take their chunks from the queue (all resident blocks busy to the end, one
    // partial row per chunk), except the full-tape kernels (static assignment, per-block rows)
    const bool dyn = !(keep && ctx->storage == MC_STORAGE_FULL);
    cl.queue = dyn ? ctx->queue : nullptr;
    const int gmax = keep ? ln.grid_fwd_keep : ln.grid_fwd;
    grid = dyn ? queue_grid(gmax, n_paths, ctx->ppt) : grid_for_paths(gmax, n_paths, ctx->ppt, ctx->n_sm);
    const void *fn = keep ? ln.fwd_keep : ln.fwd;
    cudaError_t e = timed(ctx, MC_K_FORWARD, st, [&] { return launch(fn, grid, ln.smem_fwd, ctx->pb, cl, st); });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "forward sweep launch");
    if (dyn) grid = (int)chunk_count(n_paths, ctx->ppt);  // the rows the finalize sums
    return MC_OK;
}

static mc_status do_reverse(mc_ctx *ctx, cudaStream_t st, double *grad_out) {
    const Launch &ln = ctx->ln;
    const bool dyn = ctx->last.queue != nullptr;
    const int grid = dyn ? queue_grid(ln.grid_rev, ctx->last.n_paths, ctx->ppt)
                         : grid_for_paths(ln.grid_rev, ctx->last.n_paths, ctx->ppt, ctx->n_sm);
    const int rows = dyn ? (int)chunk_count(ctx->last.n_paths, ctx->ppt) : grid;
    cudaError_t e = timed(ctx, MC_K_REVERSE, st, [&] { return launch(ln.rev, grid, ln.smem_rev, ctx->pb, ctx->last, st); });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reverse sweep launch");
    e = timed(ctx, MC_K_FINALIZE_G, st, [&] {
        return launch_finalize_grad(ctx->part_g, rows, ctx->M, 1.0 / (double)ctx->last.n_paths, grad_out, st,
                                    ctx->part1_g);
    }, finalize_kernels(rows, ctx->part1_g));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gradient finalize launch");
    return MC_OK;
}

mc_status mc_forward(mc_ctx *ctx, const double *theta, uint64_t seed, uint64_t path0,
                     uint64_t n_paths, double *Ey_out, int keep_checkpoints, void *stream) {
    if (!ctx) return MC_ERR_INVALID_ARG;
    mc_status s = check_call(ctx, theta, path0, n_paths);
    if (s != MC_OK) return s;
    if (!Ey_out || !aligned8(Ey_out)) return fail(ctx, MC_ERR_INVALID_ARG, "Ey_out must be a non-null FP64 device pointer");
    cudaStream_t st = (cudaStream_t)stream;
    DevCall cl;
    int grid;
    ctx->have_ckpt = false;
    s = do_forward(ctx, theta, seed, path0, n_paths, keep_checkpoints ? 1 : 0, st, cl, grid);
    if (s != MC_OK) return s;
    cudaError_t e = timed(ctx, MC_K_FINALIZE_Y, st, [&] {
        return launch_finalize_forward(ctx->part_y, grid, ctx->m, 1.0 / (double)n_paths, ctx->pb.disc,
                                       ctx->pb.perm, nullptr, Ey_out, nullptr, nullptr, nullptr, nullptr, st,
                                       ctx->part1_y);
    }, finalize_kernels(grid, ctx->part1_y));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "forward finalize launch");
    if (keep_checkpoints) {
        ctx->last = cl;
        ctx->have_ckpt = true;
    }
    return MC_OK;
}

mc_status mc_vjp(mc_ctx *ctx, const double *ybar, double *theta_bar_out, void *stream) {
    if (!ctx) return MC_ERR_INVALID_ARG;
    if (!ctx->have_ckpt) return fail(ctx, MC_ERR_STATE, "mc_vjp needs a preceding mc_forward with keep_checkpoints");
    if (!ybar || !theta_bar_out || !aligned8(ybar) || !aligned8(theta_bar_out))
        return fail(ctx, MC_ERR_INVALID_ARG, "ybar and theta_bar_out must be non-null FP64 device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = timed(ctx, MC_K_SEED, st, [&] {
        return launch_seed_from_ybar(ybar, ctx->pb.perm, ctx->pb.disc, ctx->m, ctx->seed_w, st);
    });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "seed launch");
    return do_reverse(ctx, st, theta_bar_out);
}

mc_status mc_value_and_grad(mc_ctx *ctx, const double *theta, const double *C, uint64_t seed,
                            uint64_t path0, uint64_t n_paths, double *G_out, double *grad_out,
                            double *Ey_out, void *stream) {
    if (!ctx) return MC_ERR_INVALID_ARG;
    mc_status s = check_call(ctx, theta, path0, n_paths);
    if (s != MC_OK) return s;
    if (!C || !G_out || !grad_out || !aligned8(C) || !aligned8(G_out) || !aligned8(grad_out) ||
        (Ey_out && !aligned8(Ey_out)))
        return fail(ctx, MC_ERR_INVALID_ARG, "C, G_out, grad_out must be non-null FP64 device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    DevCall cl;
    int grid;
    ctx->have_ckpt = false;
    s = do_forward(ctx, theta, seed, path0, n_paths, 1, st, cl, grid);
    if (s != MC_OK) return s;
    cudaError_t e = timed(ctx, MC_K_FINALIZE_Y, st, [&] {
        return launch_finalize_forward(ctx->part_y, grid, ctx->m, 1.0 / (double)n_paths, ctx->pb.disc,
                                       ctx->pb.perm, C, Ey_out, ctx->seed_w, ctx->lam2, ctx->ticket, G_out, st,
                                       ctx->part1_y);
    }, finalize_kernels(grid, ctx->part1_y));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "forward finalize launch");
    ctx->last = cl;
    ctx->have_ckpt = true;
    return do_reverse(ctx, st, grad_out);
}

mc_status mc_profile_begin(mc_ctx *ctx, int32_t max_launches) {
    if (!ctx || max_launches < 1) return MC_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    prof_free(ctx);
    ctx->prof_ev.resize(2 * (size_t)max_launches, nullptr);
    ctx->prof_id.resize(max_launches, -1);
    ctx->prof_k.resize(max_launches, 0);
    for (auto &ev : ctx->prof_ev) {
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) {
            prof_free(ctx);
            return cuda_fail(ctx, e, "profile event create");
        }
    }
    ctx->prof_max = max_launches;
    ctx->prof_n = 0;
    ctx->prof_on = true;
    return MC_OK;
}

mc_status mc_profile_end(mc_ctx *ctx, double *ms_out, int32_t *launches_out) {
    if (!ctx || !ctx->prof_on) return ctx ? fail(ctx, MC_ERR_STATE, "profiling was not started") : MC_ERR_INVALID_ARG;
    double ms[MC_N_KERNELS] = {0};
    int32_t cnt[MC_N_KERNELS] = {0};
    mc_status st = MC_OK;
    for (int q = 0; q < ctx->prof_n; ++q) {
        cudaError_t e = cudaEventSynchronize(ctx->prof_ev[2 * q + 1]);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ctx->prof_ev[2 * q], ctx->prof_ev[2 * q + 1]);
        if (e != cudaSuccess) {
            st = cuda_fail(ctx, e, "profile event read");
            break;
        }
        ms[ctx->prof_id[q]] += t;
        cnt[ctx->prof_id[q]] += ctx->prof_k[q];
    }
    prof_free(ctx);
    for (int k = 0; k < MC_N_KERNELS; ++k) {
        if (ms_out) ms_out[k] = ms[k];
        if (launches_out) launches_out[k] = cnt[k];
    }
    return st;
}

// Blocks per parameter vector: one when there are enough vectors to fill the
// GPU, otherwise enough to give it about four blocks per SM.
// Blocks per parameter vector: enough for every SM to hold as many blocks as
// fit (few vectors: one vector fills the GPU), at most one per four warp chunks.
static int jacobian_bpt(const mc_ctx *ctx, int n_theta, uint64_t n_paths) {
    const uint64_t chunk = (uint64_t)kWarp * jacobian_ppt(ctx->precision);
    const uint64_t chunks = (n_paths + chunk - 1) / chunk;
    int occ = 0;
    const size_t smem = jacobian_smem_bytes(ctx->m, ctx->n_groups, ctx->precision);
    if (cudaFuncSetAttribute(jacobian_kernel(ctx->precision), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobian_kernel(ctx->precision), kBlock, smem) !=
            cudaSuccess ||
        occ < 1)
        occ = 4;
    const uint64_t target = (uint64_t)ctx->n_sm * occ;
    uint64_t bpt = (target + n_theta - 1) / (uint64_t)n_theta;
    const uint64_t cap = (chunks + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (bpt > cap) bpt = cap;
    if (bpt > 4096) bpt = 4096;
    return (int)(bpt ? bpt : 1);
}

mc_status mc_price_jacobian_scratch_size(mc_ctx *ctx, int32_t n_theta, uint64_t n_paths, size_t *bytes_out) {
    if (!ctx || !bytes_out || n_theta < 1 || n_theta > 65535 || n_paths == 0) return MC_ERR_INVALID_ARG;
    const int bpt = jacobian_bpt(ctx, n_theta, n_paths);
    *bytes_out = (size_t)n_theta * bpt * 6 * ctx->m * sizeof(double);
    return MC_OK;
}

mc_status mc_price_jacobian(mc_ctx *ctx, const double *thetas, const double *strikes, int32_t n_theta,
                            uint64_t seed, uint64_t n_paths, double *Ey_out, double *J_out, void *scratch,
                            size_t scratch_bytes, void *stream) {
    if (!ctx) return MC_ERR_INVALID_ARG;
    if (ctx->kind != kHeston) return fail(ctx, MC_ERR_UNSUPPORTED, "the forward-mode Jacobian is built for the Heston model");
    if (!thetas || !J_out || !scratch || !aligned8(thetas) || !aligned8(J_out) || !aligned8(scratch) ||
        (Ey_out && !aligned8(Ey_out)) || (strikes && !aligned8(strikes)))
        return fail(ctx, MC_ERR_INVALID_ARG, "thetas, J_out and scratch must be non-null FP64-aligned device pointers");
    if (n_theta < 1 || n_theta > 65535 || n_paths == 0 || (uint64_t)n_theta * n_paths < n_paths)
        return fail(ctx, MC_ERR_INVALID_ARG, "need 1 <= n_theta <= 65535 and n_paths >= 1");
    size_t need = 0;
    mc_price_jacobian_scratch_size(ctx, n_theta, n_paths, &need);
    if (scratch_bytes < need) return fail(ctx, MC_ERR_INVALID_ARG, "scratch needs %zu bytes", need);
    const int bpt = jacobian_bpt(ctx, n_theta, n_paths);
    const size_t smem = jacobian_smem_bytes(ctx->m, ctx->n_groups, ctx->precision);
    cudaError_t e = cudaFuncSetAttribute(jacobian_kernel(ctx->precision), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "jacobian shared memory");
    cudaStream_t st = (cudaStream_t)stream;
    e = launch_jacobian(ctx->pb, ctx->precision, thetas, strikes, n_theta, seed, 0, n_paths, bpt, smem,
                        (double *)scratch, ctx->pb.disc, ctx->pb.perm, Ey_out, J_out, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "jacobian launch");
    return MC_OK;
}

// Scratch of mc_value_and_grad_tangent: the jacobian's per-block sums, then
// E y [m] and J [m][5] (256-byte aligned pieces).
static size_t tangent_scratch(mc_ctx *ctx, uint64_t n_paths, size_t *off_ey, size_t *off_j) {
    size_t part = 0;
    mc_price_jacobian_scratch_size(ctx, 1, n_paths, &part);
    *off_ey = align_up(part, 256);
    *off_j = align_up(*off_ey + (size_t)ctx->m * 8, 256);
    return align_up(*off_j + (size_t)ctx->m * 5 * 8, 256);
}

mc_status mc_value_and_grad_tangent_scratch_size(mc_ctx *ctx, uint64_t n_paths, size_t *bytes_out) {
    if (!ctx || !bytes_out || n_paths == 0) return MC_ERR_INVALID_ARG;
    size_t a, b;
    *bytes_out = tangent_scratch(ctx, n_paths, &a, &b);
    return MC_OK;
}

mc_status mc_value_and_grad_tangent(mc_ctx *ctx, const double *theta, const double *C, uint64_t seed,
                                    uint64_t path0, uint64_t n_paths, double *G_out, double *grad_out,
                                    double *Ey_out, void *scratch, size_t scratch_bytes, void *stream) {
    if (!ctx) return MC_ERR_INVALID_ARG;
    if (ctx->kind != kHeston) return fail(ctx, MC_ERR_UNSUPPORTED, "forward-mode tangents are built for the Heston model");
    mc_status s = check_call(ctx, theta, path0, n_paths);
    if (s != MC_OK) return s;
    if (!C || !G_out || !grad_out || !scratch || !aligned8(C) || !aligned8(G_out) || !aligned8(grad_out) ||
        (Ey_out && !aligned8(Ey_out)) || ((uintptr_t)scratch & 255u))
        return fail(ctx, MC_ERR_INVALID_ARG, "C, G_out, grad_out must be FP64 device pointers, scratch 256-byte aligned");
    size_t off_ey, off_j;
    const size_t need = tangent_scratch(ctx, n_paths, &off_ey, &off_j);
    if (scratch_bytes < need) return fail(ctx, MC_ERR_INVALID_ARG, "scratch needs %zu bytes", need);
    unsigned char *sc = (unsigned char *)scratch;
    double *Ey = Ey_out ? Ey_out : (double *)(sc + off_ey);
    double *J = (double *)(sc + off_j);
    const int bpt = jacobian_bpt(ctx, 1, n_paths);
    const size_t smem = jacobian_smem_bytes(ctx->m, ctx->n_groups, ctx->precision);
    cudaStream_t st = (cudaStream_t)stream;
    ctx->have_ckpt = false;
    cudaError_t e = timed(ctx, MC_K_TANGENT, st, [&] {
        return launch_jacobian(ctx->pb, ctx->precision, theta, nullptr, 1, seed, path0, n_paths, bpt, smem,
                               (double *)sc, ctx->pb.disc, ctx->pb.perm, Ey, J, st);
    });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tangent sweep launch");
    e = timed(ctx, MC_K_FINALIZE_T, st, [&] { return launch_tangent_finalize(Ey, J, C, ctx->m, G_out, grad_out, st); });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tangent finalize launch");
    return MC_OK;
}

mc_status mc_philox_fill(uint64_t seed, uint64_t path0, uint32_t n_paths, uint32_t n_calls,
                         uint32_t *out, void *stream) {
    if (!out || n_paths == 0 || n_calls == 0 || ((uintptr_t)out & 15u)) return MC_ERR_INVALID_ARG;
    return launch_philox_fill(seed, path0, n_paths, n_calls, out, (cudaStream_t)stream) == cudaSuccess
               ? MC_OK
               : MC_ERR_CUDA;
}

mc_status mc_normals_fill(uint64_t seed, uint64_t path0, uint32_t n_paths, uint32_t n_per_path,
                          int32_t precision, void *out, void *stream) {
    if (!out || n_paths == 0 || n_per_path == 0) return MC_ERR_INVALID_ARG;
    if (precision != MC_FP32 && precision != MC_FP64) return MC_ERR_INVALID_ARG;
    if (((uintptr_t)out & (precision == MC_FP64 ? 7u : 3u))) return MC_ERR_INVALID_ARG;
    return launch_normals_fill(seed, path0, n_paths, n_per_path, precision, out,
                               (cudaStream_t)stream) == cudaSuccess
               ? MC_OK
               : MC_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// mc_forward_static: E y with no device allocation by anyone.  Its scratch
// (model tables and per-block partial sums) lives in one file-scope device
// array that every GPU loading this library holds until the process exits.
// Host code may not use the array's name as an address; the device address
// is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kStaticScratchBytes = (size_t)4 << 20;  // MC_STATIC_SCRATCH_BYTES
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned char *g_static_ptr[kMaxDevices] = {nullptr};
// The table image each device's scratch last received (host copy), so an unchanged problem
// skips the upload.
std::vector<unsigned char> g_static_image[kMaxDevices];

}  // namespace

extern "C" mc_status mc_forward_static(const mc_model *model, const mc_instruments *inst,
                                       const double *theta, uint64_t seed, uint64_t path0,
                                       uint64_t n_paths, double *Ey_out, void *stream) {
    if (!theta || !Ey_out || ((uintptr_t)theta & 7u) || ((uintptr_t)Ey_out & 7u) || n_paths == 0) {
        fprintf(stderr, "mc_forward_static: theta and Ey_out must be FP64 device pointers, n_paths >= 1\n");
        return MC_ERR_INVALID_ARG;
    }
    Plan p;
    std::string why;
    mc_status st = make_plan(model, inst, p, why);
    if (st != MC_OK) {
        fprintf(stderr, "mc_forward_static: %s\n", why.c_str());
        return st;
    }
    if (path0 + n_paths < path0) {
        fprintf(stderr, "mc_forward_static: path range wraps around 2^64\n");
        return MC_ERR_INVALID_ARG;
    }
    if (model->normals) {
        if (path0 < model->normals_path0 || path0 + n_paths > model->normals_path0 + model->normals_rows) {
            fprintf(stderr, "mc_forward_static: paths outside the normals table\n");
            return MC_ERR_INVALID_ARG;
        }
    }
    KernelPair kp;
    if (!kernels_for(p, &kp)) return MC_ERR_UNSUPPORTED;
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess || device < 0 || device >= kMaxDevices) {
        fprintf(stderr, "mc_forward_static: no usable current device\n");
        return MC_ERR_CUDA;
    }
    unsigned char *scratch = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_ptr[device]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess || !ptr) {
                fprintf(stderr, "mc_forward_static: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
                return MC_ERR_CUDA;
            }
            g_static_ptr[device] = (unsigned char *)ptr;
        }
        scratch = g_static_ptr[device];
    }
    int grid_fwd = 1;
    size_t smem_fwd = 0;
    st = forward_shape(p, device, kp.fwd, model->nx, &grid_fwd, &smem_fwd, why);
    if (st != MC_OK) {
        fprintf(stderr, "mc_forward_static: %s\n", why.c_str());
        return st;
    }
    // scratch layout: the context's table layout with no checkpoints, then as
    // many per-block partial rows as fit
    WsLayout L(p, 0, 0);
    const size_t part_bytes = (size_t)p.m * 8;
    if (L.total + part_bytes > kStaticScratchBytes) {
        fprintf(stderr, "mc_forward_static: problem needs %zu bytes of scratch, limit %zu\n",
                L.total + part_bytes, kStaticScratchBytes);
        return MC_ERR_INVALID_ARG;
    }
    const int fit = (int)((kStaticScratchBytes - L.total) / part_bytes);
    int grid = grid_for_paths(grid_fwd < fit ? grid_fwd : fit, n_paths, p.ppt);
    cudaStream_t s = (cudaStream_t)stream;
    // The tables as one image of the scratch's first L.total bytes, uploaded with one copy and
    // only when it differs from the image this device last received.
    std::vector<unsigned char> img(L.total, 0);
    auto put = [&](size_t off, const void *src, size_t bytes) {
        if (bytes) memcpy(img.data() + off, src, bytes);
    };
    put(L.strike, p.strike.data(), p.m * 8);
    put(L.disc, p.disc.data(), p.m * 8);
    put(L.perm, p.perm.data(), p.m * 4);
    put(L.grp_seg, p.grp_seg.data(), p.n_groups * 4);
    put(L.grp_begin, p.grp_begin.data(), (p.n_groups + 1) * 4);
    put(L.bucket, p.bucket.data(), p.bucket.size() * 4);
    put(L.lv_jt, p.lv_jt.data(), p.lv_jt.size() * 4);
    put(L.lv_a, p.lv_a.data(), p.lv_a.size() * 8);
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        std::vector<unsigned char> &last = g_static_image[device];
        if (last != img) {
            last.swap(img);
            e = cudaMemcpyAsync(scratch, last.data(), last.size(), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                last.clear();
                fprintf(stderr, "mc_forward_static: table upload: %s\n", cudaGetErrorString(e));
                return MC_ERR_CUDA;
            }
        }
    }
    DevProblem pb{};
    pb.kind = p.kind;
    pb.K = p.K;
    pb.n_seg = p.n_seg;
    pb.m = p.m;
    pb.M = p.M;
    pb.n_groups = p.n_groups;
    pb.S0 = model->S0;
    pb.r = model->r;
    pb.dt = model->dt;
    pb.strike = (const double *)(scratch + L.strike);
    pb.disc = (const double *)(scratch + L.disc);
    pb.perm = (const int *)(scratch + L.perm);
    pb.grp_seg = (const int *)(scratch + L.grp_seg);
    pb.grp_begin = (const int *)(scratch + L.grp_begin);
    pb.bucket_of_step = (const int *)(scratch + L.bucket);
    pb.lv_jt = (const int *)(scratch + L.lv_jt);
    pb.lv_a = (const double *)(scratch + L.lv_a);
    pb.nt = model->nt;
    pb.nx = model->nx;
    pb.x_lo = model->x_lo;
    pb.hx = p.hx;
    pb.normals = model->normals;
    pb.normals_path0 = model->normals_path0;
    pb.normals_rows = model->normals_rows;
    pb.normals_stride = model->n_steps * (p.state_dim == 2 ? 2 : 1);
    DevCall cl{};
    cl.theta = theta;
    cl.seed = seed;
    cl.rk = philox_round_keys(seed);
    cl.path0 = path0;
    cl.n_paths = n_paths;
    cl.keep_ckpt = 0;
    cl.part_y = (double *)(scratch + L.total);
    e = launch(kp.fwd, grid, smem_fwd, pb, cl, s);
    if (e == cudaSuccess)
        e = launch_finalize_forward(cl.part_y, grid, p.m, 1.0 / (double)n_paths, pb.disc, pb.perm, nullptr,
                                    Ey_out, nullptr, nullptr, nullptr, nullptr, s);
    if (e != cudaSuccess) {
        fprintf(stderr, "mc_forward_static: launch: %s\n", cudaGetErrorString(e));
        return MC_ERR_CUDA;
    }
    return MC_OK;
}
