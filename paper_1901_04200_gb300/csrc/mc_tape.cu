// mc_tape.cu -- expected-backward AD of a whole Monte-Carlo program on the
// GPU (arXiv 1901.04200, Appendix, after Fries).  The program, the rule and
// the stage structure are described in include/mctape.h.
//
// Host plan.  Each node is deterministic (DET) or per-path (PATH).  PARAM and
// CONST are DET, NORMAL is PATH, an expectation of a PATH node is DET (an
// expectation of a DET node is the node itself), any other op is PATH if an
// argument is.  A node's stage is the latest stage at which its arguments
// are available; an expectation belongs to the stage of its argument and is
// available from the next one.  Per stage the order det-nodes -> path-nodes
// -> expectations is topological, so the forward sweep runs per stage
//   det_forward (one thread) -> path_forward (one thread per path, values to
//   the tape, per-warp sums of the expectations' arguments) -> expect_finalize
// and the backward sweep runs the stages in reverse, per stage
//   path_backward (adds E(D) of each expectation to its argument's per-path
//   adjoint, then the per-path nodes in reverse; per-warp sums of the
//   adjoint contributions to deterministic arguments) -> darg_finalize (their
//   means) -> det_backward (one thread, the deterministic nodes in reverse;
//   a parameter's adjoint mean is its gradient).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "mc_common.cuh"
#include "mc_common_src.h"  // kMcCommonSrc: this header's text, for the run-time compiler
#include "mctape.h"

using namespace mcaad;

namespace {

constexpr int kMaxNodes = 1 << 24;
constexpr int kMaxStageSums = 2048;  // expectations, or distinct DET arguments, per stage
constexpr int kRing = 32;            // per-thread shared-memory window of recent per-path nodes
constexpr int kGroup = 8;            // nodes whose HBM loads are issued together (<= kRing)
constexpr int kTile = 128;           // node descriptors a block stages in shared memory at a time

// Node flags.  kStore: the value goes to the HBM tape (a far or later-stage
// user, an expectation, or a backward partial needs it from there).  kFar:
// some user's adjoint contribution goes to the HBM adjoint array (a far or
// later-stage user, or an expectation), so the backward sweep reads it.
constexpr int kStore = 1, kFar = 2;

// Device form of a node.  References to values: r >= 0 is row r of the
// per-path tape, r < 0 is deterministic slot -r-1.  sm: the node's slot in
// the per-thread ring (its position in the stage's per-path list mod kRing);
// sa, sb: the ring slot of a per-path argument fewer than kRing positions
// earlier in the same stage (read from the ring, not HBM), -1 else.  la, lb:
// index of a DET argument among the stage's accumulated DET arguments
// (backward), -1 else.
struct DevNode {
    int op, flags;
    int ra, rb, rm;
    int sa, sb, sm;
    int la, lb;
    double c;
};

struct StagePlan {
    std::vector<int> det, path, expect;  // node indices, program order
    std::vector<int> dargs;              // DET nodes used by the stage's PATH nodes (first use order)
};

struct TapePlan {
    int n_nodes = 0, objective = 0, n_params = 0, n_stages = 0, n_rows = 0, n_det = 0;
    int max_exp = 0, max_darg = 0;
    std::vector<int> cls;    // 0 DET, 1 PATH
    std::vector<int> stage;  // stage where the node is computed
    std::vector<int> ref;    // row (PATH) or -slot-1 (DET)
    std::vector<StagePlan> st;
};

__host__ __device__ inline int n_args(int op) {
    switch (op) {
    case MC_OP_PARAM:
    case MC_OP_CONST:
    case MC_OP_NORMAL:
        return 0;
    case MC_OP_ADD:
    case MC_OP_SUB:
    case MC_OP_MUL:
    case MC_OP_DIV:
        return 2;
    default:
        return 1;
    }
}

mc_status make_tape_plan(const mc_tape_node *nodes, int n, int objective, int n_params, TapePlan &p,
                         std::string &why) {
    char buf[256];
    auto bad = [&](mc_status s, const char *fmt, ...) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        why = buf;
        return s;
    };
    if (!nodes || n < 1) return bad(MC_ERR_INVALID_ARG, "empty program");
    if (n > kMaxNodes) return bad(MC_ERR_UNSUPPORTED, "more than %d nodes", kMaxNodes);
    if (objective < 0 || objective >= n) return bad(MC_ERR_INVALID_ARG, "objective %d outside the program", objective);
    if (n_params < 0) return bad(MC_ERR_INVALID_ARG, "negative parameter count");
    p = TapePlan();
    p.n_nodes = n;
    p.objective = objective;
    p.n_params = n_params;
    p.cls.assign(n, 0);
    p.stage.assign(n, 0);
    p.ref.assign(n, 0);
    std::vector<int> avail(n, 0);
    for (int i = 0; i < n; ++i) {
        const mc_tape_node &d = nodes[i];
        if (d.op < 0 || d.op >= MC_N_OPS) return bad(MC_ERR_INVALID_ARG, "node %d: unknown op %d", i, d.op);
        const int na = n_args(d.op);
        const int args[2] = {d.a, d.b};
        for (int q = 0; q < 2; ++q) {
            if (q < na) {
                if (args[q] < 0 || args[q] >= i)
                    return bad(MC_ERR_INVALID_ARG, "node %d: argument %d does not precede it", i, args[q]);
            } else if (args[q] != -1) {
                return bad(MC_ERR_INVALID_ARG, "node %d: op %d takes %d arguments", i, d.op, na);
            }
        }
        if (d.op == MC_OP_PARAM && !(d.c >= 0 && d.c < n_params && d.c == floor(d.c)))
            return bad(MC_ERR_INVALID_ARG, "node %d: parameter index %g outside [0, %d)", i, d.c, n_params);
        if (d.op == MC_OP_NORMAL && !(d.c >= 0 && d.c < 4294967296.0 * 4.0 && d.c == floor(d.c)))
            return bad(MC_ERR_INVALID_ARG, "node %d: bad normal index %g", i, d.c);
        if (!std::isfinite(d.c)) return bad(MC_ERR_INVALID_ARG, "node %d: non-finite constant", i);
        if (d.op == MC_OP_PARAM || d.op == MC_OP_CONST) {
            p.cls[i] = 0;
            p.stage[i] = avail[i] = 0;
        } else if (d.op == MC_OP_NORMAL) {
            p.cls[i] = 1;
            p.stage[i] = avail[i] = 0;
        } else if (d.op == MC_OP_EXPECT) {
            p.cls[i] = 0;
            if (p.cls[d.a] == 0) {  // E of a deterministic value: the value itself
                p.stage[i] = avail[i] = avail[d.a];
            } else {
                p.stage[i] = p.stage[d.a];
                avail[i] = p.stage[d.a] + 1;
            }
        } else {
            int cls = 0, s = 0;
            for (int q = 0; q < na; ++q) {
                cls |= p.cls[args[q]];
                s = std::max(s, avail[args[q]]);
            }
            p.cls[i] = cls;
            p.stage[i] = avail[i] = s;
        }
    }
    if (p.cls[objective] != 0) return bad(MC_ERR_INVALID_ARG, "the objective (node %d) is not deterministic", objective);
    int ns = 1;
    for (int i = 0; i < n; ++i) ns = std::max(ns, p.stage[i] + 1);
    p.n_stages = ns;
    p.st.assign(ns, StagePlan());
    for (int i = 0; i < n; ++i) {
        StagePlan &sp = p.st[p.stage[i]];
        if (p.cls[i] == 1) {
            p.ref[i] = p.n_rows++;
            sp.path.push_back(i);
        } else {
            p.ref[i] = -(p.n_det++) - 1;
            const bool exp_of_path = nodes[i].op == MC_OP_EXPECT && p.cls[nodes[i].a] == 1;
            (exp_of_path ? sp.expect : sp.det).push_back(i);
        }
    }
    for (int s = 0; s < ns; ++s) {
        StagePlan &sp = p.st[s];
        for (int i : sp.path) {
            const int args[2] = {nodes[i].a, nodes[i].b};
            for (int q = 0; q < n_args(nodes[i].op); ++q)
                if (p.cls[args[q]] == 0 && std::find(sp.dargs.begin(), sp.dargs.end(), args[q]) == sp.dargs.end())
                    sp.dargs.push_back(args[q]);
        }
        if ((int)sp.expect.size() > kMaxStageSums)
            return bad(MC_ERR_UNSUPPORTED, "stage %d has %zu expectations (limit %d)", s, sp.expect.size(), kMaxStageSums);
        if ((int)sp.dargs.size() > kMaxStageSums)
            return bad(MC_ERR_UNSUPPORTED, "stage %d uses %zu deterministic values per path (limit %d)", s,
                       sp.dargs.size(), kMaxStageSums);
        p.max_exp = std::max(p.max_exp, (int)sp.expect.size());
        p.max_darg = std::max(p.max_darg, (int)sp.dargs.size());
    }
    return MC_OK;
}

// Device node lists: per stage [det | path | expect] blocks, flattened.
struct DevLists {
    std::vector<DevNode> all;
    std::vector<int> det_off, path_off, exp_off, darg_off;  // per stage, + 1 end entry each
    std::vector<int> darg_slot;                              // flattened: DET slot of each accumulated argument
    std::vector<char> stored;                                // per node: its per-path values are on the tape
    std::vector<int> far_rows;                               // tape rows whose adjoints accumulate in HBM
};

// Whether the backward partials of op need the value of argument q (0: a, 1: b) or the node's own.
bool needs_arg_value(int op, int q) {
    if (op == MC_OP_MUL || op == MC_OP_DIV) return true;
    return q == 0 && (op == MC_OP_LOG || op == MC_OP_SQRT || op == MC_OP_RELU || op == MC_OP_ABS);
}
bool needs_own_value(int op) { return op == MC_OP_EXP || op == MC_OP_SQRT; }

DevLists make_lists(const mc_tape_node *nodes, const TapePlan &p, size_t *bytes_per_path = nullptr,
                    size_t rb = 8) {
    DevLists L;
    const int n = p.n_nodes;
    // position of each per-path node in its stage's list; flags from its users
    std::vector<int> pos(n, -1), flags(n, 0);
    for (int s = 0; s < p.n_stages; ++s)
        for (size_t k = 0; k < p.st[s].path.size(); ++k) pos[p.st[s].path[k]] = (int)k;
    auto near = [&](int user, int arg) {
        return p.cls[arg] == 1 && p.cls[user] == 1 && p.stage[user] == p.stage[arg] && pos[user] - pos[arg] < kRing;
    };
    for (int i = 0; i < n; ++i) {
        const int args[2] = {nodes[i].a, nodes[i].b};
        for (int q = 0; q < n_args(nodes[i].op); ++q) {
            const int a = args[q];
            if (p.cls[a] != 1) continue;
            if (!near(i, a)) flags[a] |= kStore | kFar;  // far user, later stage, or an expectation
            if (needs_arg_value(nodes[i].op, q)) flags[a] |= kStore;
        }
        if (p.cls[i] == 1 && needs_own_value(nodes[i].op)) flags[i] |= kStore;
    }
    auto dev = [&](int i, const StagePlan *sp) {
        DevNode d;
        d.op = nodes[i].op;
        d.flags = flags[i];
        d.c = nodes[i].c;
        d.rm = p.ref[i];
        d.ra = nodes[i].a >= 0 ? p.ref[nodes[i].a] : 0;
        d.rb = nodes[i].b >= 0 ? p.ref[nodes[i].b] : 0;
        d.sm = pos[i] >= 0 ? pos[i] % kRing : -1;
        d.sa = nodes[i].a >= 0 && near(i, nodes[i].a) ? pos[nodes[i].a] % kRing : -1;
        d.sb = nodes[i].b >= 0 && near(i, nodes[i].b) ? pos[nodes[i].b] % kRing : -1;
        d.la = d.lb = -1;
        if (sp) {
            auto local = [&](int arg) {
                if (arg < 0 || p.cls[arg] == 1) return -1;
                return (int)(std::find(sp->dargs.begin(), sp->dargs.end(), arg) - sp->dargs.begin());
            };
            d.la = local(nodes[i].a);
            d.lb = local(nodes[i].b);
        }
        return d;
    };
    L.stored.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        L.stored[i] = p.cls[i] == 1 && (flags[i] & kStore);
        if (p.cls[i] == 1 && (flags[i] & kFar)) L.far_rows.push_back(p.ref[i]);
    }
    if (bytes_per_path) {
        // HBM bytes per path of one value and gradient under the kernels' rules (FP64)
        size_t b = 0;
        for (int i = 0; i < n; ++i) {
            const int op = nodes[i].op;
            if (op == MC_OP_EXPECT) {
                if (p.cls[nodes[i].a] == 1) b += 3 * rb;  // argument read for the sum; E(D) added to its adjoint
                continue;
            }
            if (p.cls[i] != 1) continue;
            if (flags[i] & kStore) b += rb;          // forward: value to the tape
            if (flags[i] & kFar) b += rb;            // backward: adjoint from HBM
            if (needs_own_value(op)) b += rb;        // backward: own value
            const int args[2] = {nodes[i].a, nodes[i].b};
            for (int q = 0; q < n_args(op); ++q) {
                const int a = args[q];
                if (p.cls[a] != 1) continue;
                if (!near(i, a)) b += 3 * rb;        // forward load; backward adjoint update
                if (needs_arg_value(op, q)) b += rb; // backward: argument value
            }
        }
        *bytes_per_path = b;
    }
    for (int s = 0; s < p.n_stages; ++s) {
        const StagePlan &sp = p.st[s];
        L.det_off.push_back((int)L.all.size());
        for (int i : sp.det) L.all.push_back(dev(i, nullptr));
        L.path_off.push_back((int)L.all.size());
        for (int i : sp.path) L.all.push_back(dev(i, &sp));
        L.exp_off.push_back((int)L.all.size());
        for (int i : sp.expect) L.all.push_back(dev(i, nullptr));
        L.darg_off.push_back((int)L.darg_slot.size());
        for (int i : sp.dargs) L.darg_slot.push_back(-p.ref[i] - 1);
    }
    L.det_off.push_back((int)L.all.size());
    L.path_off.push_back((int)L.all.size());
    L.exp_off.push_back((int)L.all.size());
    L.darg_off.push_back((int)L.darg_slot.size());
    return L;
}

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct TapeWs {
    size_t nodes, dslot, frows, det, ddet, part, tape, adj, total;
    TapeWs(const TapePlan &p, size_t n_all, size_t n_dslot, size_t n_far, int grid, uint64_t stride, size_t rb) {
        size_t o = 0;
        auto take = [&](size_t bytes) {
            size_t at = o;
            o = round_up(o + bytes, 256);
            return at;
        };
        nodes = take(n_all * sizeof(DevNode));
        dslot = take(n_dslot * 4 + 4);
        frows = take(n_far * 4 + 4);
        det = take((size_t)p.n_det * 8);
        ddet = take((size_t)p.n_det * 8);
        part = take((size_t)grid * std::max(1, std::max(p.max_exp, p.max_darg)) * 8);
        tape = take((size_t)p.n_rows * stride * rb);
        adj = take((size_t)p.n_rows * stride * rb);
        total = o;
    }
};

// ------------------------------------------------------------- kernels ----

template <typename Real>
__device__ __forceinline__ Real ld(const Real *tape, const double *det, int r, uint64_t stride, uint64_t p) {
    return r >= 0 ? tape[(size_t)r * stride + p] : (Real)det[-r - 1];
}

__device__ __forceinline__ float exp_t(float x) { return expf(x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }
__device__ __forceinline__ float log_t(float x) { return logf(x); }
__device__ __forceinline__ double log_t(double x) { return log(x); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }

template <typename T>
__device__ __forceinline__ T apply_op(int op, T a, T b, T c) {
    switch (op) {
    case MC_OP_ADD: return a + b;
    case MC_OP_SUB: return a - b;
    case MC_OP_MUL: return a * b;
    case MC_OP_DIV: return a / b;
    case MC_OP_ADDC: return a + c;
    case MC_OP_MULC: return a * c;
    case MC_OP_NEG: return -a;
    case MC_OP_EXP: return exp_t(a);
    case MC_OP_LOG: return log_t(a);
    case MC_OP_SQRT: return sqrt_t(a);
    case MC_OP_RELU: return a > T(0) ? a : T(0);
    case MC_OP_ABS: return a < T(0) ? -a : a;
    default: return a;  // EXPECT of a deterministic value
    }
}

// Partial derivatives of node value m = op(a, b) with respect to a and b.
template <typename T>
__device__ __forceinline__ void partials(int op, T a, T b, T m, T c, T &pa, T &pb) {
    pa = T(0);
    pb = T(0);
    switch (op) {
    case MC_OP_ADD: pa = T(1); pb = T(1); break;
    case MC_OP_SUB: pa = T(1); pb = T(-1); break;
    case MC_OP_MUL: pa = b; pb = a; break;
    case MC_OP_DIV: pa = T(1) / b; pb = -a / (b * b); break;
    case MC_OP_ADDC: pa = T(1); break;
    case MC_OP_MULC: pa = c; break;
    case MC_OP_NEG: pa = T(-1); break;
    case MC_OP_EXP: pa = m; break;
    case MC_OP_LOG: pa = T(1) / a; break;
    case MC_OP_SQRT: pa = a > T(0) ? T(0.5) / m : T(0); break;
    case MC_OP_RELU: pa = a > T(0) ? T(1) : T(0); break;
    case MC_OP_ABS: pa = a > T(0) ? T(1) : (a < T(0) ? T(-1) : T(0)); break;
    case MC_OP_EXPECT: pa = T(1); break;  // of a deterministic value: identity
    default: break;
    }
}

// The block's copy of descriptors nd[k0 .. k0 + cnt) into shared memory (16-byte words).
__device__ __forceinline__ void stage_tile(DevNode *tile, const DevNode *__restrict__ nd, int k0, int cnt) {
    static_assert(sizeof(DevNode) % 16 == 0, "descriptor size");
    constexpr int kWords = (int)(sizeof(DevNode) / 16);
    const int4 *src = (const int4 *)(nd + k0);
    int4 *dst = (int4 *)tile;
    for (int q = threadIdx.x; q < cnt * kWords; q += blockDim.x) dst[q] = src[q];
}

// Deterministic nodes of a stage, in program order, by one thread.  The block
// stages the node descriptors in shared memory, kDetTile at a time, and the
// deterministic values too when they fit (in_smem), so the walk's dependent
// loads do not go to L2.
constexpr int kDetTile = 256;
constexpr size_t kDetTileBytes = (size_t)kDetTile * sizeof(DevNode);
constexpr int kDetSmemBytes = 36 * 1024;  // values; with the tile within the default 48 KB

__global__ void tape_det_forward(const DevNode *__restrict__ nd, int n, const double *__restrict__ theta,
                                 double *__restrict__ det, int n_det, int in_smem) {
    extern __shared__ __align__(16) unsigned char dsm[];
    DevNode *tile = (DevNode *)dsm;
    double *sdet = (double *)(dsm + kDetTileBytes);
    double *V = in_smem ? sdet : det;
    if (in_smem)
        for (int q = threadIdx.x; q < n_det; q += blockDim.x) sdet[q] = det[q];
    for (int t0 = 0; t0 < n; t0 += kDetTile) {
        const int tn = min(kDetTile, n - t0);
        __syncthreads();  // values staged; the previous tile consumed
        stage_tile(tile, nd, t0, tn);
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 0; k < tn; ++k) {
                const DevNode &d = tile[k];
                double v;
                if (d.op == MC_OP_PARAM) {
                    v = theta[(int)d.c];
                } else if (d.op == MC_OP_CONST) {
                    v = d.c;
                } else {
                    const double a = V[-d.ra - 1];
                    const double b = n_args(d.op) == 2 ? V[-d.rb - 1] : 0.0;
                    v = apply_op<double>(d.op, a, b, d.c);
                }
                V[-d.rm - 1] = v;
            }
        }
    }
    if (in_smem) {
        __syncthreads();
        for (int q = threadIdx.x; q < n_det; q += blockDim.x) det[q] = sdet[q];
    }
}

// Per-path nodes of a stage, one thread per path.  Each thread keeps its last
// kRing per-path values in shared memory (ring[slot][thread]); arguments
// further back, of earlier stages, or deterministic ones are loaded for a
// group of kGroup nodes at once before the group is computed.  Values flagged
// kStore also go to the HBM tape.  Then per-warp FP64 sums of the
// expectations' arguments (warp shuffle, lane k%32 adds), per block in warp
// order -> part[block][k].
template <typename Real>
__global__ void __launch_bounds__(kBlock) tape_path_forward(const DevNode *__restrict__ nd, int n,
                                                            const DevNode *__restrict__ ex, int n_exp,
                                                            const double *__restrict__ det, Real *__restrict__ tape,
                                                            uint64_t stride, RoundKeys rk, uint64_t path0,
                                                            uint64_t n_paths, double *__restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem[];
    DevNode *tile = (DevNode *)smem;                                     // [kTile] descriptors
    unsigned char *after = smem + (size_t)kTile * sizeof(DevNode);
    Real *ring = (Real *)after + threadIdx.x;                                 // [kRing][kBlock]
    double *wacc = (double *)(after + (size_t)kRing * kBlock * sizeof(Real));  // [kWarpsPerBlock][n_exp]
    for (int q = threadIdx.x; q < kWarpsPerBlock * n_exp; q += blockDim.x) wacc[q] = 0.0;
    __syncthreads();
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    const uint64_t chunks = (n_paths + kWarp - 1) / kWarp;
    // the block's warps take chunks base + warp in lockstep (block-uniform loop: they share the tiles)
    for (uint64_t base = (uint64_t)blockIdx.x * kWarpsPerBlock; base < chunks;
         base += (uint64_t)gridDim.x * kWarpsPerBlock) {
        const uint64_t ch = base + warp;
        const bool live = ch < chunks;  // a warp past the last chunk only takes part in the tiles
        const uint64_t p = ch * kWarp + lane;
        const bool active = live && p < n_paths;
        PathNormals<Real> rng;
        rng.init(path0 + (active ? p : 0));
        uint64_t last_call = ~0ull;
        for (int t0 = 0; t0 < n; t0 += kTile) {
        const int tn = min(kTile, n - t0);
        __syncthreads();  // the previous tile is consumed
        stage_tile(tile, nd, t0, tn);
        __syncthreads();
        for (int k0 = 0; k0 < tn; k0 += kGroup) {
            Real fa[kGroup], fb[kGroup];
#pragma unroll
            for (int g = 0; g < kGroup; ++g) {
                fa[g] = fb[g] = Real(0);
                if (live && k0 + g < tn) {
                    const DevNode &d = tile[k0 + g];
                    const int na = d.op == MC_OP_NORMAL ? 0 : n_args(d.op);
                    if (na >= 1 && d.sa < 0) fa[g] = ld(tape, det, d.ra, stride, p);
                    if (na == 2 && d.sb < 0) fb[g] = ld(tape, det, d.rb, stride, p);
                }
            }
#pragma unroll
            for (int g = 0; g < kGroup; ++g) {
                if (k0 + g >= tn) break;
                const DevNode &d = tile[k0 + g];
                Real v;
                if (d.op == MC_OP_NORMAL) {
                    const uint64_t j = (uint64_t)d.c;
                    if ((j >> 2) != last_call) {
                        last_call = j >> 2;
                        rng.fill((uint32_t)last_call, rk);
                    }
                    v = rng.pick((uint32_t)(j & 3u));
                } else {
                    const Real a = d.sa >= 0 ? ring[d.sa * kBlock] : fa[g];
                    const Real b = d.sb >= 0 ? ring[d.sb * kBlock] : fb[g];
                    v = apply_op<Real>(d.op, a, b, (Real)d.c);
                }
                ring[d.sm * kBlock] = v;
                if (live && (d.flags & kStore)) tape[(size_t)d.rm * stride + p] = v;
            }
        }
        }
        double *wrow = wacc + warp * n_exp;
        for (int k0 = 0; k0 < n_exp; k0 += kWarp) {
            const int cnt = min(kWarp, n_exp - k0);
            Real mine = Real(0);
            for (int j = 0; j < cnt; ++j) {
                const Real v = active ? tape[(size_t)ex[k0 + j].ra * stride + p] : Real(0);
                const Real s = warp_sum(v);
                mine = lane == j ? s : mine;
            }
            if (lane < cnt) wrow[k0 + lane] += (double)mine;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_exp; k += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kWarpsPerBlock; ++w) s += wacc[w * n_exp + k];
        part[(size_t)blockIdx.x * n_exp + k] = s;
    }
}

// Expectation k = (sum over blocks) / n: one warp per expectation, lane l
// sums blocks l, l + 32, ... in order, then a fixed shuffle tree.
__global__ void tape_expect_finalize(const double *__restrict__ part, int nb, const DevNode *__restrict__ ex,
                                     int n_exp, double inv_n, double *__restrict__ det) {
    const int lane = threadIdx.x % kWarp;
    const int warps = gridDim.x * blockDim.x / kWarp;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) / kWarp; k < n_exp; k += warps) {
        double s = 0.0;
        for (int b = lane; b < nb; b += kWarp) s += part[(size_t)b * n_exp + k];
        s = warp_sum(s);
        if (lane == 0) det[-ex[k].rm - 1] = s * inv_n;
    }
}

// Backward sweep of a stage's per-path nodes: first E(D) of each expectation
// into its argument's adjoint (HBM), then the nodes in reverse.  A node's
// adjoint is the sum of its near users' contributions, kept in a per-thread
// shared-memory ring like the forward values, and (flag kFar) of the far
// users' contributions in the HBM adjoint array.  The values the partials
// need are loaded from the tape for a group of kGroup nodes at once;
// contributions to deterministic arguments are warp-summed into per-warp
// accumulators.
template <typename Real>
__global__ void __launch_bounds__(kBlock) tape_path_backward(const DevNode *__restrict__ nd, int n,
                                                             const DevNode *__restrict__ ex, int n_exp, int n_darg,
                                                             const double *__restrict__ det,
                                                             const double *__restrict__ ddet,
                                                             const Real *__restrict__ tape, Real *__restrict__ adj,
                                                             uint64_t stride, uint64_t n_paths,
                                                             double *__restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem[];
    DevNode *tile = (DevNode *)smem;                                     // [kTile] descriptors
    unsigned char *after = smem + (size_t)kTile * sizeof(DevNode);
    Real *ring = (Real *)after + threadIdx.x;                                 // [kRing][kBlock] adjoints
    double *wacc = (double *)(after + (size_t)kRing * kBlock * sizeof(Real));  // [kWarpsPerBlock][n_darg]
    for (int q = threadIdx.x; q < kWarpsPerBlock * n_darg; q += blockDim.x) wacc[q] = 0.0;
    __syncthreads();
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    double *wrow = wacc + warp * n_darg;
    const uint64_t chunks = (n_paths + kWarp - 1) / kWarp;
    for (uint64_t base = (uint64_t)blockIdx.x * kWarpsPerBlock; base < chunks;
         base += (uint64_t)gridDim.x * kWarpsPerBlock) {
        const uint64_t ch = base + warp;
        const bool live = ch < chunks;
        const uint64_t p = ch * kWarp + lane;
        const bool active = live && p < n_paths;
#pragma unroll
        for (int q = 0; q < kRing; ++q) ring[q * kBlock] = Real(0);
        if (active)
            for (int k = 0; k < n_exp; ++k) adj[(size_t)ex[k].ra * stride + p] += (Real)ddet[-ex[k].rm - 1];
        for (int t1 = n; t1 > 0; t1 -= kTile) {
        const int t0 = max(0, t1 - kTile), tn = t1 - t0;
        __syncthreads();  // the previous tile is consumed
        stage_tile(tile, nd, t0, tn);
        __syncthreads();
        for (int k0 = tn - 1; k0 >= 0; k0 -= kGroup) {
            Real va[kGroup], vb[kGroup], vm[kGroup], dg[kGroup];
#pragma unroll
            for (int g = 0; g < kGroup; ++g) {
                va[g] = vb[g] = vm[g] = dg[g] = Real(0);
                if (live && k0 - g >= 0) {
                    const DevNode &d = tile[k0 - g];
                    if (d.op != MC_OP_NORMAL) {
                        const bool need_ab = d.op == MC_OP_MUL || d.op == MC_OP_DIV;
                        const bool need_a = need_ab || d.op == MC_OP_LOG || d.op == MC_OP_SQRT ||
                                            d.op == MC_OP_RELU || d.op == MC_OP_ABS;
                        if (need_a) va[g] = ld(tape, det, d.ra, stride, p);
                        if (need_ab) vb[g] = ld(tape, det, d.rb, stride, p);
                        if (d.op == MC_OP_EXP || d.op == MC_OP_SQRT) vm[g] = tape[(size_t)d.rm * stride + p];
                    }
                    if ((d.flags & kFar) && active) dg[g] = adj[(size_t)d.rm * stride + p];
                }
            }
#pragma unroll
            for (int g = 0; g < kGroup; ++g) {
                if (k0 - g < 0) break;
                const DevNode &d = tile[k0 - g];
                const Real D = active ? ring[d.sm * kBlock] + dg[g] : Real(0);
                ring[d.sm * kBlock] = Real(0);
                if (d.op == MC_OP_NORMAL) continue;
                const bool two = n_args(d.op) == 2;
                Real pa, pb;
                partials<Real>(d.op, va[g], vb[g], vm[g], (Real)d.c, pa, pb);
                const Real ga = active ? D * pa : Real(0), gb = active ? D * pb : Real(0);
                if (d.sa >= 0) {
                    ring[d.sa * kBlock] += ga;
                } else if (d.ra >= 0) {
                    if (active) adj[(size_t)d.ra * stride + p] += ga;
                } else {
                    const Real sum = warp_sum(ga);
                    if (lane == 0) wrow[d.la] += (double)sum;
                }
                if (two) {
                    if (d.sb >= 0) {
                        ring[d.sb * kBlock] += gb;
                    } else if (d.rb >= 0) {
                        if (active) adj[(size_t)d.rb * stride + p] += gb;
                    } else {
                        const Real sum = warp_sum(gb);
                        if (lane == 0) wrow[d.lb] += (double)sum;
                    }
                }
            }
        }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_darg; k += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kWarpsPerBlock; ++w) s += wacc[w * n_darg + k];
        part[(size_t)blockIdx.x * n_darg + k] = s;
    }
}

// Adjoint means of the stage's deterministic arguments: += (sum over blocks) / n,
// one warp per argument as in tape_expect_finalize.
__global__ void tape_darg_finalize(const double *__restrict__ part, int nb, const int *__restrict__ slot,
                                   int n_darg, double inv_n, double *__restrict__ ddet) {
    const int lane = threadIdx.x % kWarp;
    const int warps = gridDim.x * blockDim.x / kWarp;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) / kWarp; k < n_darg; k += warps) {
        double s = 0.0;
        for (int b = lane; b < nb; b += kWarp) s += part[(size_t)b * n_darg + k];
        s = warp_sum(s);
        if (lane == 0) ddet[slot[k]] += s * inv_n;
    }
}

// Deterministic nodes of a stage in reverse, by one thread (values and
// adjoints staged in shared memory when they fit); a parameter's adjoint mean
// is added to its gradient component.
__global__ void tape_det_backward(const DevNode *__restrict__ nd, int n, const double *__restrict__ det,
                                  double *__restrict__ ddet, double *__restrict__ grad, int n_det, int in_smem) {
    extern __shared__ __align__(16) unsigned char dsm[];
    DevNode *tile = (DevNode *)dsm;
    double *sdet = (double *)(dsm + kDetTileBytes);
    const double *V = in_smem ? sdet : det;
    double *A = in_smem ? sdet + n_det : ddet;
    if (in_smem)
        for (int q = threadIdx.x; q < n_det; q += blockDim.x) {
            sdet[q] = det[q];
            sdet[n_det + q] = ddet[q];
        }
    for (int t1 = n; t1 > 0; t1 -= kDetTile) {
        const int t0 = max(0, t1 - kDetTile), tn = t1 - t0;
        __syncthreads();  // values staged; the previous tile consumed
        stage_tile(tile, nd, t0, tn);
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = tn - 1; k >= 0; --k) {
                const DevNode &d = tile[k];
                const double D = A[-d.rm - 1];
                if (d.op == MC_OP_PARAM) {
                    grad[(int)d.c] += D;
                    continue;
                }
                if (d.op == MC_OP_CONST) continue;
                const bool two = n_args(d.op) == 2;
                const double a = V[-d.ra - 1];
                const double b = two ? V[-d.rb - 1] : 0.0;
                double pa, pb;
                partials<double>(d.op, a, b, V[-d.rm - 1], d.c, pa, pb);
                A[-d.ra - 1] += D * pa;
                if (two) A[-d.rb - 1] += D * pb;
            }
        }
    }
    if (in_smem) {
        __syncthreads();
        for (int q = threadIdx.x; q < n_det; q += blockDim.x) ddet[q] = sdet[n_det + q];
    }
}

// Launchers (shared by the interpreter and the compiled program).
void launch_det_forward(const DevNode *nd, int n, const double *theta, double *det, int n_det, cudaStream_t st) {
    const bool sm = (size_t)n_det * 8 <= (size_t)kDetSmemBytes;
    tape_det_forward<<<1, kBlock, kDetTileBytes + (sm ? (size_t)n_det * 8 : 0), st>>>(nd, n, theta, det, n_det,
                                                                                       sm ? 1 : 0);
}
void launch_det_backward(const DevNode *nd, int n, const double *det, double *ddet, double *grad, int n_det,
                         cudaStream_t st) {
    const bool sm = (size_t)n_det * 16 <= (size_t)kDetSmemBytes;
    tape_det_backward<<<1, kBlock, kDetTileBytes + (sm ? (size_t)n_det * 16 : 0), st>>>(nd, n, det, ddet, grad,
                                                                                        n_det, sm ? 1 : 0);
}
void launch_expect_finalize(const double *part, int nb, const DevNode *ex, int n_exp, double inv_n, double *det,
                            cudaStream_t st) {
    tape_expect_finalize<<<(n_exp * kWarp + kBlock - 1) / kBlock, kBlock, 0, st>>>(part, nb, ex, n_exp, inv_n, det);
}
void launch_darg_finalize(const double *part, int nb, const int *slot, int n_darg, double inv_n, double *ddet,
                          cudaStream_t st) {
    tape_darg_finalize<<<(n_darg * kWarp + kBlock - 1) / kBlock, kBlock, 0, st>>>(part, nb, slot, n_darg, inv_n, ddet);
}

__global__ void tape_begin_backward(double *__restrict__ ddet, int n_det, int obj_slot, double *__restrict__ grad,
                                    int n_params) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_det; k += gridDim.x * blockDim.x)
        ddet[k] = k == obj_slot ? 1.0 : 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_params; k += gridDim.x * blockDim.x) grad[k] = 0.0;
}

__global__ void tape_copy_value(const double *__restrict__ det, int slot, double *__restrict__ out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *out = det[slot];
}

// Zero, for the evaluated paths, the adjoint rows that accumulate contributions
// in HBM (nodes with a far or later-stage user or an expectation); no other
// row of the adjoint array is read.  Block row y walks rows y, y + gridDim.y, ...
template <typename Real>
__global__ void tape_zero_rows(Real *__restrict__ adj, const int *__restrict__ rows, int n_rows, uint64_t stride,
                               uint64_t n_paths) {
    for (int r = blockIdx.y; r < n_rows; r += gridDim.y) {
        Real *row = adj + (size_t)rows[r] * stride;
        for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_paths;
             q += (uint64_t)gridDim.x * blockDim.x)
            row[q] = Real(0);
    }
}

template <typename Real>
void launch_zero_rows(Real *adj, const int *rows, int n_rows, uint64_t stride, uint64_t n_paths, cudaStream_t st) {
    if (n_rows <= 0) return;
    const int gx = (int)std::min<uint64_t>((n_paths + 1023) / 1024, 1024);
    const int gy = std::min(n_rows, 1024);
    tape_zero_rows<Real><<<dim3(gx, gy), 256, 0, st>>>(adj, rows, n_rows, stride, n_paths);
}

__global__ void tape_widen(const float *__restrict__ in, uint64_t n, double *__restrict__ out) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x)
        out[k] = in[k];
}

}  // namespace

// ------------------------------------------------------- tape compiler ----
// A stage's per-path nodes are cut into segments of consecutive nodes; each
// segment becomes two straight-line kernels (forward: values in registers;
// backward: adjoints in registers) compiled at run time.  A value crosses a
// segment or stage boundary, or feeds an expectation or a backward partial,
// through the HBM tape; an adjoint contribution to a node outside the segment
// goes to the HBM adjoint array.
struct JitSeg {
    int stage = 0;
    std::vector<int> nodes;  // per-path nodes, program order
    std::vector<int> dargs;  // deterministic nodes they use, first-use order
    int darg_off = 0;        // offset of this segment's DET slots in the device list
    std::string src, log;
    std::vector<char> cubin;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t fwd = nullptr, bwd = nullptr;
    int grid_f = 1, grid_b = 1;
    size_t smem_b = 0;
};

struct JitPlan {
    bool recompute = false;             // backward kernels re-run their segment's forward
    int piece = 0;                      // with recompute: pieces of this many nodes (0: the whole segment)
    std::vector<JitSeg> segs;           // stage order, then program order
    std::vector<int> seg_begin;         // per stage: first segment; + end entry
    std::vector<char> store, far;       // per node, compiled mode
    std::vector<int> dslot;             // DET slot of every segment's accumulated arguments
    int *dslot_dev = nullptr;
    std::vector<int> far_rows;          // tape rows whose adjoints accumulate in HBM (far nodes)
    int *frows_dev = nullptr;
    size_t bytes_per_path = 0;
};

struct mc_tape {
    int device = 0, precision = MC_FP64;
    std::vector<mc_tape_node> src_nodes;  // the program as given (for the tape compiler)
    JitPlan *jit = nullptr;               // compiled program, or null (interpreter)
    TapePlan plan;
    DevLists lists;
    int grid_f = 1, grid_b = 1, n_sm = 1;  // blocks of the path forward / backward kernels
    uint64_t max_paths = 0, stride = 0;
    size_t smem_fwd = 0, smem_bwd = 0;
    bool owns_ws = false;
    unsigned char *ws = nullptr;
    DevNode *nodes = nullptr;
    int *dslot = nullptr;
    int *frows = nullptr;  // the interpreter's HBM-accumulated adjoint rows (lists.far_rows)
    double *det = nullptr, *ddet = nullptr, *part = nullptr;
    void *tape = nullptr, *adj = nullptr;  // [n_rows][stride] of FP64 or FP32
    uint64_t last_n = 0;
    std::string err;
};

namespace {

mc_status tfail(mc_tape *t, mc_status st, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
mc_status tfail(mc_tape *t, mc_status st, const char *fmt, ...) {
    if (t) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        t->err = buf;
    }
    return st;
}

uint64_t tape_stride(uint64_t max_paths) { return (max_paths + kWarp - 1) / kWarp * kWarp; }

// Blocks: (resident blocks per SM) x SMs of the heavier path kernel, capped at
// one block per 4 chunks of 32 paths.
template <typename Real>
mc_status tape_launch_shape(int device, const TapePlan &p, uint64_t max_paths, int *grid_f, int *grid_b, int *n_sm,
                            size_t *smem_fwd, size_t *smem_bwd, std::string &why) {
    cudaError_t e = cudaDeviceGetAttribute(n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        why = cudaGetErrorString(e);
        return MC_ERR_CUDA;
    }
    const size_t fixed = (size_t)kTile * sizeof(DevNode) + (size_t)kRing * kBlock * sizeof(Real);
    *smem_fwd = fixed + (size_t)kWarpsPerBlock * p.max_exp * 8;
    *smem_bwd = fixed + (size_t)kWarpsPerBlock * p.max_darg * 8;
    int occ_f = 0, occ_b = 0;
    e = cudaFuncSetAttribute(tape_path_forward<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem_fwd);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tape_path_backward<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)*smem_bwd);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, tape_path_forward<Real>, kBlock, *smem_fwd);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, tape_path_backward<Real>, kBlock, *smem_bwd);
    if (e != cudaSuccess) {
        why = cudaGetErrorString(e);
        return MC_ERR_CUDA;
    }
    const uint64_t want = std::max<uint64_t>(((max_paths + kWarp - 1) / kWarp + kWarpsPerBlock - 1) / kWarpsPerBlock, 1);
    *grid_f = (int)std::min<uint64_t>((uint64_t)std::max(occ_f, 1) * *n_sm, want);
    *grid_b = (int)std::min<uint64_t>((uint64_t)std::max(occ_b, 1) * *n_sm, want);
    return MC_OK;
}

}  // namespace

namespace {

// One value and gradient: the forward stages, then the backward stages in reverse.
template <typename Real>
mc_status run_tape(mc_tape *t, const double *theta, uint64_t seed, uint64_t path0, uint64_t n_paths,
                   double *value_out, double *grad_out, cudaStream_t st) {
    const TapePlan &p = t->plan;
    const DevLists &L = t->lists;
    const RoundKeys rk = philox_round_keys(seed);
    const double inv_n = 1.0 / (double)n_paths;
    const uint64_t want = ((n_paths + kWarp - 1) / kWarp + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int grid_f = (int)std::min<uint64_t>((uint64_t)t->grid_f, want);
    const int grid_b = (int)std::min<uint64_t>((uint64_t)t->grid_b, want);
    Real *tape = (Real *)t->tape, *adj = (Real *)t->adj;
    const size_t ring = (size_t)kTile * sizeof(DevNode) + (size_t)kRing * kBlock * sizeof(Real);
    auto ck = [&](const char *what) -> mc_status {
        const cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? MC_OK : tfail(t, MC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    };
    // ---- forward sweep
    for (int s = 0; s < p.n_stages; ++s) {
        const int nd = L.path_off[s] - L.det_off[s], np = L.exp_off[s] - L.path_off[s];
        const int ne = L.det_off[s + 1] - L.exp_off[s];
        if (nd > 0) launch_det_forward(t->nodes + L.det_off[s], nd, theta, t->det, p.n_det, st);
        if (np > 0 || ne > 0)
            tape_path_forward<Real><<<grid_f, kBlock, ring + (size_t)kWarpsPerBlock * ne * 8, st>>>(
                t->nodes + L.path_off[s], np, t->nodes + L.exp_off[s], ne, t->det, tape, t->stride, rk, path0,
                n_paths, t->part);
        if (ne > 0)
            launch_expect_finalize(t->part, grid_f, t->nodes + L.exp_off[s], ne, inv_n, t->det, st);
        mc_status r = ck("forward sweep");
        if (r != MC_OK) return r;
    }
    tape_copy_value<<<1, 1, 0, st>>>(t->det, -p.ref[p.objective] - 1, value_out);
    // ---- backward sweep
    launch_zero_rows<Real>(adj, t->frows, (int)L.far_rows.size(), t->stride, n_paths, st);
    tape_begin_backward<<<(std::max(p.n_det, p.n_params) + 255) / 256 + 1, 256, 0, st>>>(
        t->ddet, p.n_det, -p.ref[p.objective] - 1, grad_out, p.n_params);
    for (int s = p.n_stages - 1; s >= 0; --s) {
        const int nd = L.path_off[s] - L.det_off[s], np = L.exp_off[s] - L.path_off[s];
        const int ne = L.det_off[s + 1] - L.exp_off[s];
        const int na = L.darg_off[s + 1] - L.darg_off[s];
        if (np > 0 || ne > 0)
            tape_path_backward<Real><<<grid_b, kBlock, ring + (size_t)kWarpsPerBlock * na * 8, st>>>(
                t->nodes + L.path_off[s], np, t->nodes + L.exp_off[s], ne, na, t->det, t->ddet, tape, adj, t->stride,
                n_paths, t->part);
        if (na > 0)
            launch_darg_finalize(t->part, grid_b, t->dslot + L.darg_off[s], na, inv_n, t->ddet, st);
        if (nd > 0) launch_det_backward(t->nodes + L.det_off[s], nd, t->det, t->ddet, grad_out, p.n_det, st);
        mc_status r = ck("backward sweep");
        if (r != MC_OK) return r;
    }
    return MC_OK;
}

}  // namespace

namespace {

// ------------------------------------------------ tape compiler: plan ----

// piece > 0 (with recompute): the backward kernel re-runs and differentiates its segment in
// pieces of `piece` consecutive nodes, last piece first; a value one piece computes and a later
// piece of the same segment uses is kept by the forward kernel on the tape, so each piece starts
// from loads and only one piece's values are live at a time.
JitPlan *make_jit_plan(const std::vector<mc_tape_node> &nodes, const TapePlan &p, int seg_nodes, size_t rb,
                       bool recompute, int piece = 0) {
    JitPlan *J = new JitPlan;
    J->recompute = recompute;
    J->piece = recompute ? std::max(piece, 0) : 0;
    const int n = p.n_nodes;
    std::vector<int> seg_of(n, -1), piece_of(n, -1);
    for (int s = 0; s < p.n_stages; ++s) {
        J->seg_begin.push_back((int)J->segs.size());
        const std::vector<int> &path = p.st[s].path;
        for (size_t k0 = 0; k0 < path.size(); k0 += (size_t)seg_nodes) {
            JitSeg sg;
            sg.stage = s;
            for (size_t k = k0; k < std::min(path.size(), k0 + (size_t)seg_nodes); ++k) {
                sg.nodes.push_back(path[k]);
                seg_of[path[k]] = (int)J->segs.size();
                piece_of[path[k]] = J->piece > 0 ? (int)((k - k0) / (size_t)J->piece) : 0;
            }
            J->segs.push_back(std::move(sg));
        }
    }
    J->seg_begin.push_back((int)J->segs.size());
    J->store.assign(n, 0);
    J->far.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        const int args[2] = {nodes[i].a, nodes[i].b};
        for (int q = 0; q < n_args(nodes[i].op); ++q) {
            const int a = args[q];
            if (p.cls[a] != 1) continue;
            if (!(p.cls[i] == 1 && seg_of[i] == seg_of[a])) J->store[a] = J->far[a] = 1;  // outside user
            else if (piece_of[i] != piece_of[a]) J->store[a] = 1;  // a later piece's input
            if (!recompute && needs_arg_value(nodes[i].op, q)) J->store[a] = 1;
        }
        if (!recompute && p.cls[i] == 1 && needs_own_value(nodes[i].op)) J->store[i] = 1;
    }
    for (int i = 0; i < n; ++i)
        if (J->far[i]) J->far_rows.push_back(p.ref[i]);
    size_t b = 0;
    for (int i = 0; i < n; ++i)
        if (nodes[i].op == MC_OP_EXPECT && p.cls[nodes[i].a] == 1) b += 3 * rb;
    for (size_t k = 0; k < J->segs.size(); ++k) {
        JitSeg &sg = J->segs[k];
        sg.darg_off = (int)J->dslot.size();
        std::vector<int> fwd_loads, bwd_loads, far_rows;
        auto add = [](std::vector<int> &v, int x) {
            if (std::find(v.begin(), v.end(), x) == v.end()) v.push_back(x);
        };
        for (int i : sg.nodes) {
            const int args[2] = {nodes[i].a, nodes[i].b};
            if (J->store[i]) b += rb;
            if (J->far[i]) b += rb;
            if (needs_own_value(nodes[i].op)) add(bwd_loads, i);
            for (int q = 0; q < n_args(nodes[i].op); ++q) {
                const int a = args[q];
                if (p.cls[a] == 0) {
                    add(sg.dargs, a);
                    continue;
                }
                if (seg_of[a] != (int)k) {
                    add(fwd_loads, a);
                    add(far_rows, a);
                }
                if (needs_arg_value(nodes[i].op, q)) add(bwd_loads, a);
            }
        }
        // with recompute the backward kernel loads what the forward kernel loads (in pieces: also each
        // piece's inputs from earlier pieces), and nothing more
        size_t piece_loads = 0;
        if (J->piece > 0) {
            std::vector<std::pair<int, int>> seen;  // (piece, value)
            for (int i : sg.nodes) {
                const int args[2] = {nodes[i].a, nodes[i].b};
                for (int q = 0; q < n_args(nodes[i].op); ++q) {
                    const int a = args[q];
                    if (p.cls[a] == 1 && seg_of[a] == (int)k && piece_of[a] != piece_of[i]) {
                        const std::pair<int, int> key(piece_of[i], a);
                        if (std::find(seen.begin(), seen.end(), key) == seen.end()) seen.push_back(key);
                    }
                }
            }
            piece_loads = seen.size();
        }
        b += rb * (fwd_loads.size() + (recompute ? fwd_loads.size() + piece_loads : bwd_loads.size())) +
             2 * rb * far_rows.size();
        for (int d : sg.dargs) J->dslot.push_back(-p.ref[d] - 1);
    }
    J->bytes_per_path = b;
    return J;
}

// ---------------------------------------------- tape compiler: codegen ----

std::string lit(double c) {
    char buf[64];
    snprintf(buf, sizeof buf, "%.17g", c);
    std::string t(buf);
    if (t.find_first_of(".eE") == std::string::npos) t += ".0";
    return "R(" + t + ")";
}

std::string gen_segment(const std::vector<mc_tape_node> &nodes, const TapePlan &p, const JitPlan &J, int k,
                        int precision) {
    const JitSeg &sg = J.segs[k];
    const bool f64 = precision == MC_FP64;
    std::vector<int> local(p.n_nodes, -1);
    for (size_t q = 0; q < sg.nodes.size(); ++q) local[sg.nodes[q]] = (int)q;
    std::vector<int> dl(p.n_nodes, -1);
    for (size_t q = 0; q < sg.dargs.size(); ++q) dl[sg.dargs[q]] = (int)q;
    auto det_ref = [&](int a) { return "R(det[" + std::to_string(-p.ref[a] - 1) + "])"; };
    std::ostringstream o;
    o << "#include \"mc_common.cuh\"\ntypedef " << (f64 ? "double" : "float") << " R;\ntypedef unsigned long long u64;\n";

    // The segment's forward body: values in registers; values from outside the segment loaded
    // at first use through `ptr` (w<row>); with `stores`, values flagged kept go to the tape.
    // Nodes [q0, q1) of the segment (all of them by default): values computed before q0 count as
    // loaded from the tape like values from outside the segment.
    auto emit_forward = [&](bool stores, const char *ptr, size_t q0 = 0, size_t q1 = (size_t)-1) {
        if (q1 > sg.nodes.size()) q1 = sg.nodes.size();
        std::vector<char> loaded(p.n_nodes, 0);
        long long call = -1;
        auto val = [&](int a) -> std::string {
            if (p.cls[a] == 0) return det_ref(a);
            if (local[a] >= (int)q0) return "v" + std::to_string(local[a]);
            if (!loaded[a]) {
                o << "  const R w" << p.ref[a] << " = " << ptr << "[(u64)" << p.ref[a] << " * stride];\n";
                loaded[a] = 1;
            }
            return "w" + std::to_string(p.ref[a]);
        };
        for (size_t q = q0; q < q1; ++q) {
            const int i = sg.nodes[q];
            const mc_tape_node &d = nodes[i];
            const std::string A = n_args(d.op) >= 1 ? val(d.a) : std::string();
            const std::string B = n_args(d.op) == 2 ? val(d.b) : std::string();
            std::string e;
            switch (d.op) {
            case MC_OP_NORMAL: {
                const unsigned long long j = (unsigned long long)d.c;
                if ((long long)(j >> 2) != call) {
                    call = (long long)(j >> 2);
                    o << "  rng.fill(" << call << "u, rk);\n";
                }
                e = "rng.z" + std::to_string(j & 3u);
                break;
            }
            case MC_OP_ADD: e = A + " + " + B; break;
            case MC_OP_SUB: e = A + " - " + B; break;
            case MC_OP_MUL: e = A + " * " + B; break;
            case MC_OP_DIV: e = A + " / " + B; break;
            case MC_OP_ADDC: e = A + " + " + lit(d.c); break;
            case MC_OP_MULC: e = A + " * " + lit(d.c); break;
            case MC_OP_NEG: e = "-" + A; break;
            case MC_OP_EXP: e = std::string(f64 ? "exp(" : "expf(") + A + ")"; break;
            case MC_OP_LOG: e = std::string(f64 ? "log(" : "logf(") + A + ")"; break;
            case MC_OP_SQRT: e = std::string(f64 ? "sqrt(" : "sqrtf(") + A + ")"; break;
            case MC_OP_RELU: e = "(" + A + " > R(0) ? " + A + " : R(0))"; break;
            case MC_OP_ABS: e = "(" + A + " < R(0) ? -" + A + " : " + A + ")"; break;
            default: e = A; break;
            }
            o << "  const R v" << q << " = " << e << ";\n";
            if (stores && J.store[i]) o << "  " << ptr << "[(u64)" << p.ref[i] << " * stride] = v" << q << ";\n";
        }
    };

    // forward kernel
    o << "extern \"C\" __global__ void __launch_bounds__(128) fwd(const double *__restrict__ det, R *__restrict__ tape,"
         " u64 stride, mcaad::RoundKeys rk, u64 path0, u64 n_paths) {\n"
         " const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;\n"
         " const u64 chunks = (n_paths + 31) / 32;\n"
         " for (u64 ch = (u64)blockIdx.x * 4 + warp; ch < chunks; ch += (u64)gridDim.x * 4) {\n"
         "  const u64 p = ch * 32 + lane;\n"
         "  const bool active = p < n_paths;\n"
         "  R *tp = tape + p;\n"
         "  mcaad::PathNormals<R> rng;\n"
         "  rng.init(path0 + (active ? p : 0));\n";
    emit_forward(true, "tp");
    o << " }\n}\n";

    // backward: adjoints of the segment's nodes in registers; values its partials need loaded
    // from the tape; contributions to nodes outside summed per row and added once; those to
    // deterministic arguments summed per thread, warp-summed once per chunk
    std::vector<int> far_rows;
    for (int i : sg.nodes) {
        const int args[2] = {nodes[i].a, nodes[i].b};
        for (int q = 0; q < n_args(nodes[i].op); ++q) {
            const int a = args[q];
            if (p.cls[a] == 1 && local[a] < 0 && std::find(far_rows.begin(), far_rows.end(), a) == far_rows.end())
                far_rows.push_back(a);
        }
    }
    // at least four resident blocks: the straight-line backward code of a long segment would take
    // up to 255 registers (two blocks per SM); capped at 128 the spills cost less than the lost
    // occupancy (Heston program, 768-node segments: 1.88 ms per evaluation against 2.00)
    o << "extern \"C\" __global__ void __launch_bounds__(128, 4) bwd(const double *__restrict__ det,"
         " const R *__restrict__ tape, R *__restrict__ adj, u64 stride, u64 n_paths, double *__restrict__ part,"
         " int n_darg, mcaad::RoundKeys rk, u64 path0) {\n"
         " extern __shared__ double wacc[];\n"
         " for (int q = threadIdx.x; q < 4 * n_darg; q += blockDim.x) wacc[q] = 0.0;\n"
         " __syncthreads();\n"
         " const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;\n"
         " double *wrow = wacc + warp * n_darg;\n"
         " const u64 chunks = (n_paths + 31) / 32;\n"
         " for (u64 ch = (u64)blockIdx.x * 4 + warp; ch < chunks; ch += (u64)gridDim.x * 4) {\n"
         "  const u64 p = ch * 32 + lane;\n"
         "  const bool active = p < n_paths;\n"
         "  const R *tv = tape + p;\n"
         "  R *ta = adj + p;\n";
    // With recompute the segment's values are re-run in registers (the partials need no tape loads):
    // all at once, or piece by piece from the last piece, each piece's inputs loaded from the tape.
    const size_t nq = sg.nodes.size();
    const size_t piece = J.recompute && J.piece > 0 ? (size_t)J.piece : nq;
    if (J.recompute) o << "  mcaad::PathNormals<R> rng;\n  rng.init(path0 + (active ? p : 0));\n";
    if (J.recompute && piece >= nq) emit_forward(false, "tv");
    for (size_t q = 0; q < nq; ++q) o << "  R a" << q << " = R(0);\n";
    for (int a : far_rows) o << "  R f" << p.ref[a] << " = R(0);\n";
    for (size_t l = 0; l < sg.dargs.size(); ++l) o << "  R g" << l << " = R(0);\n";
    for (size_t q1 = nq; q1 > 0;) {
        const size_t q0 = (q1 - 1) / piece * piece;  // pieces start at multiples of `piece`, as planned
        const bool pieced = J.recompute && piece < nq;
        if (pieced) {
            o << "  {\n";
            emit_forward(false, "tv", q0, q1);
        }
        std::vector<char> vloaded(p.n_nodes, 0);
        auto value = [&](int a) -> std::string {
            if (p.cls[a] == 0) return det_ref(a);
            if (J.recompute) return local[a] >= (int)(pieced ? q0 : 0) ? "v" + std::to_string(local[a])
                                                                      : "w" + std::to_string(p.ref[a]);
            if (!vloaded[a]) {
                o << "  const R u" << p.ref[a] << " = tv[(u64)" << p.ref[a] << " * stride];\n";
                vloaded[a] = 1;
            }
            return "u" + std::to_string(p.ref[a]);
        };
        auto contrib = [&](int a, const std::string &g) {
            if (p.cls[a] == 0)
                o << "  g" << dl[a] << " += " << g << ";\n";
            else if (local[a] >= 0)
                o << "  a" << local[a] << " += " << g << ";\n";
            else
                o << "  f" << p.ref[a] << " += " << g << ";\n";
        };
        for (int q = (int)q1 - 1; q >= (int)q0; --q) {
            const int i = sg.nodes[q];
            const mc_tape_node &d = nodes[i];
            const std::string D = "D" + std::to_string(q);
            if (J.far[i])
                o << "  const R " << D << " = active ? a" << q << " + ta[(u64)" << p.ref[i] << " * stride] : R(0);\n";
            else
                o << "  const R " << D << " = active ? a" << q << " : R(0);\n";
            switch (d.op) {
            case MC_OP_NORMAL: break;
            case MC_OP_ADD: contrib(d.a, D); contrib(d.b, D); break;
            case MC_OP_SUB: contrib(d.a, D); contrib(d.b, "-" + D); break;
            case MC_OP_MUL: {
                const std::string va = value(d.a), vb = value(d.b);
                contrib(d.a, D + " * " + vb);
                contrib(d.b, D + " * " + va);
                break;
            }
            case MC_OP_DIV: {
                const std::string va = value(d.a), vb = value(d.b);
                contrib(d.a, D + " * (R(1) / " + vb + ")");
                contrib(d.b, D + " * (-" + va + " / (" + vb + " * " + vb + "))");
                break;
            }
            case MC_OP_ADDC: contrib(d.a, D); break;
            case MC_OP_MULC: contrib(d.a, D + " * " + lit(d.c)); break;
            case MC_OP_NEG: contrib(d.a, "-" + D); break;
            case MC_OP_EXP: contrib(d.a, D + " * " + value(i)); break;
            case MC_OP_LOG: contrib(d.a, D + " * (R(1) / " + value(d.a) + ")"); break;
            case MC_OP_SQRT: {
                const std::string va = value(d.a), m = value(i);
                contrib(d.a, D + " * (" + va + " > R(0) ? R(0.5) / " + m + " : R(0))");
                break;
            }
            case MC_OP_RELU: {
                const std::string va = value(d.a);
                contrib(d.a, D + " * (" + va + " > R(0) ? R(1) : R(0))");
                break;
            }
            case MC_OP_ABS: {
                const std::string va = value(d.a);
                contrib(d.a, D + " * (" + va + " > R(0) ? R(1) : (" + va + " < R(0) ? R(-1) : R(0)))");
                break;
            }
            default: break;
            }
        }
        if (pieced) o << "  }\n";
        q1 = q0;
    }
    for (int a : far_rows) o << "  if (active) ta[(u64)" << p.ref[a] << " * stride] += f" << p.ref[a] << ";\n";
    for (size_t l = 0; l < sg.dargs.size(); ++l)
        o << "  { const R s = mcaad::warp_sum(g" << l << "); if (lane == 0) wrow[" << l << "] += (double)s; }\n";
    o << " }\n"
         " __syncthreads();\n"
         " for (int k = threadIdx.x; k < n_darg; k += blockDim.x) {\n"
         "  double s = 0.0;\n"
         "  for (int w = 0; w < 4; ++w) s += wacc[w * n_darg + k];\n"
         "  part[(u64)blockIdx.x * n_darg + k] = s;\n"
         " }\n}\n";
    return o.str();
}

bool rtc_compile(JitSeg &sg) {
    nvrtcProgram prog;
    const char *hdr[] = {kMcCommonSrc};
    const char *hdr_name[] = {"mc_common.cuh"};
    if (nvrtcCreateProgram(&prog, sg.src.c_str(), "tape_segment.cu", 1, hdr, hdr_name) != NVRTC_SUCCESS) {
        sg.log = "nvrtcCreateProgram failed";
        return false;
    }
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=false"};
    const nvrtcResult r = nvrtcCompileProgram(prog, 3, opts);
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    sg.log.assign(ls, '\0');
    if (ls) nvrtcGetProgramLog(prog, &sg.log[0]);
    bool ok = r == NVRTC_SUCCESS;
    if (ok) {
        size_t cs = 0;
        ok = nvrtcGetCUBINSize(prog, &cs) == NVRTC_SUCCESS && cs > 0;
        if (ok) {
            sg.cubin.resize(cs);
            ok = nvrtcGetCUBIN(prog, sg.cubin.data()) == NVRTC_SUCCESS;
        }
    }
    nvrtcDestroyProgram(&prog);
    return ok;
}

void jit_free(JitPlan *J) {
    if (!J) return;
    for (JitSeg &sg : J->segs)
        if (sg.lib) cudaLibraryUnload(sg.lib);
    if (J->dslot_dev) cudaFree(J->dslot_dev);
    if (J->frows_dev) cudaFree(J->frows_dev);
    delete J;
}

// One value and gradient with the compiled segments (the deterministic nodes,
// the expectations' sums and adds, and the finalize steps as in the interpreter).
template <typename Real>
mc_status run_tape_jit(mc_tape *t, const double *theta, uint64_t seed, uint64_t path0, uint64_t n_paths,
                       double *value_out, double *grad_out, cudaStream_t st) {
    const TapePlan &p = t->plan;
    const DevLists &L = t->lists;
    const JitPlan &J = *t->jit;
    RoundKeys rk = philox_round_keys(seed);
    const double inv_n = 1.0 / (double)n_paths;
    const uint64_t want = ((n_paths + kWarp - 1) / kWarp + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int grid_f = (int)std::min<uint64_t>((uint64_t)t->grid_f, want);
    const int grid_b = (int)std::min<uint64_t>((uint64_t)t->grid_b, want);
    Real *tape = (Real *)t->tape, *adj = (Real *)t->adj;
    uint64_t stride = t->stride;
    const size_t ring = (size_t)kTile * sizeof(DevNode) + (size_t)kRing * kBlock * sizeof(Real);
    auto ck = [&](const char *what) -> mc_status {
        const cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? MC_OK : tfail(t, MC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    };
    for (int s = 0; s < p.n_stages; ++s) {
        const int nd = L.path_off[s] - L.det_off[s];
        const int ne = L.det_off[s + 1] - L.exp_off[s];
        if (nd > 0) launch_det_forward(t->nodes + L.det_off[s], nd, theta, t->det, p.n_det, st);
        for (int k = J.seg_begin[s]; k < J.seg_begin[s + 1]; ++k) {
            const JitSeg &sg = J.segs[k];
            const double *det = t->det;
            void *args[] = {(void *)&det, (void *)&tape, (void *)&stride, (void *)&rk, (void *)&path0, (void *)&n_paths};
            const int g = (int)std::min<uint64_t>((uint64_t)sg.grid_f, want);
            const cudaError_t e = cudaLaunchKernel((const void *)sg.fwd, dim3(g), dim3(kBlock), args, 0, st);
            if (e != cudaSuccess) return tfail(t, MC_ERR_CUDA, "compiled forward: %s", cudaGetErrorString(e));
        }
        if (ne > 0) {  // the expectations' sums, read back from the tape
            tape_path_forward<Real><<<grid_f, kBlock, ring + (size_t)kWarpsPerBlock * ne * 8, st>>>(
                t->nodes + L.path_off[s], 0, t->nodes + L.exp_off[s], ne, t->det, tape, stride, rk, path0, n_paths,
                t->part);
            launch_expect_finalize(t->part, grid_f, t->nodes + L.exp_off[s], ne, inv_n, t->det, st);
        }
        mc_status r = ck("forward sweep");
        if (r != MC_OK) return r;
    }
    tape_copy_value<<<1, 1, 0, st>>>(t->det, -p.ref[p.objective] - 1, value_out);
    launch_zero_rows<Real>(adj, J.frows_dev, (int)J.far_rows.size(), stride, n_paths, st);
    tape_begin_backward<<<(std::max(p.n_det, p.n_params) + 255) / 256 + 1, 256, 0, st>>>(
        t->ddet, p.n_det, -p.ref[p.objective] - 1, grad_out, p.n_params);
    for (int s = p.n_stages - 1; s >= 0; --s) {
        const int nd = L.path_off[s] - L.det_off[s];
        const int ne = L.det_off[s + 1] - L.exp_off[s];
        if (ne > 0)  // E(D) of each expectation into its argument's adjoint
            tape_path_backward<Real><<<grid_b, kBlock, ring, st>>>(t->nodes + L.path_off[s], 0, t->nodes + L.exp_off[s],
                                                                   ne, 0, t->det, t->ddet, tape, adj, stride, n_paths,
                                                                   t->part);
        for (int k = J.seg_begin[s + 1] - 1; k >= J.seg_begin[s]; --k) {
            const JitSeg &sg = J.segs[k];
            const double *det = t->det;
            double *part = t->part;
            int na = (int)sg.dargs.size();
            void *args[] = {(void *)&det, (void *)&tape,  (void *)&adj, (void *)&stride, (void *)&n_paths,
                            (void *)&part, (void *)&na,   (void *)&rk,  (void *)&path0};
            const int g = (int)std::min<uint64_t>((uint64_t)sg.grid_b, want);
            const cudaError_t e = cudaLaunchKernel((const void *)sg.bwd, dim3(g), dim3(kBlock), args, sg.smem_b, st);
            if (e != cudaSuccess) return tfail(t, MC_ERR_CUDA, "compiled backward: %s", cudaGetErrorString(e));
            if (na > 0)
                launch_darg_finalize(t->part, g, J.dslot_dev + sg.darg_off, na, inv_n, t->ddet, st);
        }
        if (nd > 0) launch_det_backward(t->nodes + L.det_off[s], nd, t->det, t->ddet, grad_out, p.n_det, st);
        mc_status r = ck("backward sweep");
        if (r != MC_OK) return r;
    }
    return MC_OK;
}

}  // namespace

extern "C" {

mc_status mc_tape_plan(const mc_tape_node *nodes, int32_t n_nodes, int32_t objective, int32_t n_params,
                       int32_t precision, uint64_t max_paths, int32_t *n_stages, int32_t *n_path_nodes,
                       size_t *workspace, size_t *hbm_bytes) {
    if (precision != MC_FP32 && precision != MC_FP64) return MC_ERR_INVALID_ARG;
    const size_t rb = precision == MC_FP64 ? 8 : 4;
    TapePlan p;
    std::string why;
    mc_status st = make_tape_plan(nodes, n_nodes, objective, n_params, p, why);
    if (st != MC_OK) {
        fprintf(stderr, "mc_tape_plan: %s\n", why.c_str());
        return st;
    }
    if (n_stages) *n_stages = p.n_stages;
    if (n_path_nodes) *n_path_nodes = p.n_rows;
    if (hbm_bytes) make_lists(nodes, p, hbm_bytes, rb);
    if (workspace) {
        if (max_paths == 0) return MC_ERR_INVALID_ARG;
        // the grid is bounded by one block per 128 paths and by 32 resident blocks on each of 1024 SMs
        const uint64_t blocks = std::min<uint64_t>((max_paths + kBlock - 1) / kBlock, 32u * 1024u);
        const DevLists L = make_lists(nodes, p);
        *workspace = TapeWs(p, L.all.size(), L.darg_slot.size(), L.far_rows.size(), (int)blocks,
                            tape_stride(max_paths), rb).total;
    }
    return MC_OK;
}

mc_status mc_tape_create(int device, const mc_tape_node *nodes, int32_t n_nodes, int32_t objective,
                         int32_t n_params, int32_t precision, uint64_t max_paths, void *workspace,
                         size_t workspace_bytes, mc_tape **out) {
    if (!out || max_paths == 0 || (precision != MC_FP32 && precision != MC_FP64)) return MC_ERR_INVALID_ARG;
    const size_t rb = precision == MC_FP64 ? 8 : 4;
    *out = nullptr;
    mc_tape *t = new (std::nothrow) mc_tape();
    if (!t) return MC_ERR_OOM;
    std::string why;
    mc_status st = make_tape_plan(nodes, n_nodes, objective, n_params, t->plan, why);
    if (st != MC_OK) {
        fprintf(stderr, "mc_tape_create: %s\n", why.c_str());
        delete t;
        return st;
    }
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete t;
        return MC_ERR_CUDA;
    }
    t->device = device;
    t->precision = precision;
    t->src_nodes.assign(nodes, nodes + n_nodes);
    t->max_paths = max_paths;
    t->stride = tape_stride(max_paths);
    t->lists = make_lists(nodes, t->plan);
    st = precision == MC_FP64
             ? tape_launch_shape<double>(device, t->plan, max_paths, &t->grid_f, &t->grid_b, &t->n_sm, &t->smem_fwd,
                                         &t->smem_bwd, why)
             : tape_launch_shape<float>(device, t->plan, max_paths, &t->grid_f, &t->grid_b, &t->n_sm, &t->smem_fwd,
                                        &t->smem_bwd, why);
    if (st != MC_OK) {
        fprintf(stderr, "mc_tape_create: %s\n", why.c_str());
        delete t;
        return st;
    }
    const uint64_t blocks_cap = std::min<uint64_t>((max_paths + kBlock - 1) / kBlock, 32u * 1024u);
    if ((uint64_t)t->grid_f > blocks_cap) t->grid_f = (int)std::max<uint64_t>(blocks_cap, 1);
    if ((uint64_t)t->grid_b > blocks_cap) t->grid_b = (int)std::max<uint64_t>(blocks_cap, 1);
    TapeWs W(t->plan, t->lists.all.size(), t->lists.darg_slot.size(), t->lists.far_rows.size(),
             (int)std::max<uint64_t>(blocks_cap, 1), t->stride, rb);
    if (workspace) {
        if (workspace_bytes < W.total || ((uintptr_t)workspace & 255u)) {
            fprintf(stderr, "mc_tape_create: workspace needs %zu bytes, 256-byte aligned\n", W.total);
            delete t;
            return MC_ERR_INVALID_ARG;
        }
        t->ws = (unsigned char *)workspace;
    } else {
        e = cudaMalloc((void **)&t->ws, W.total);
        if (e != cudaSuccess) {
            fprintf(stderr, "mc_tape_create: cudaMalloc(%zu): %s\n", W.total, cudaGetErrorString(e));
            delete t;
            return e == cudaErrorMemoryAllocation ? MC_ERR_OOM : MC_ERR_CUDA;
        }
        t->owns_ws = true;
    }
    t->nodes = (DevNode *)(t->ws + W.nodes);
    t->dslot = (int *)(t->ws + W.dslot);
    t->frows = (int *)(t->ws + W.frows);
    t->det = (double *)(t->ws + W.det);
    t->ddet = (double *)(t->ws + W.ddet);
    t->part = (double *)(t->ws + W.part);
    t->tape = t->ws + W.tape;
    t->adj = t->ws + W.adj;
    e = cudaMemcpy(t->nodes, t->lists.all.data(), t->lists.all.size() * sizeof(DevNode), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !t->lists.darg_slot.empty())
        e = cudaMemcpy(t->dslot, t->lists.darg_slot.data(), t->lists.darg_slot.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !t->lists.far_rows.empty())
        e = cudaMemcpy(t->frows, t->lists.far_rows.data(), t->lists.far_rows.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        fprintf(stderr, "mc_tape_create: upload: %s\n", cudaGetErrorString(e));
        mc_tape_destroy(t);
        return MC_ERR_CUDA;
    }
    *out = t;
    return MC_OK;
}

void mc_tape_destroy(mc_tape *t) {
    if (!t) return;
    cudaSetDevice(t->device);
    jit_free(t->jit);
    if (t->owns_ws && t->ws) cudaFree(t->ws);
    delete t;
}

const char *mc_tape_last_error(const mc_tape *t) { return t ? t->err.c_str() : "null tape"; }

mc_status mc_tape_value_and_grad(mc_tape *t, const double *theta, uint64_t seed, uint64_t path0,
                                 uint64_t n_paths, double *value_out, double *grad_out, void *stream) {
    if (!t) return MC_ERR_INVALID_ARG;
    const TapePlan &p = t->plan;
    if (n_paths == 0 || n_paths > t->max_paths)
        return tfail(t, MC_ERR_INVALID_ARG, "n_paths=%llu outside [1, max_paths=%llu]", (unsigned long long)n_paths,
                     (unsigned long long)t->max_paths);
    if ((p.n_params > 0 && (!theta || ((uintptr_t)theta & 7u))) || !value_out || !grad_out ||
        ((uintptr_t)value_out & 7u) || ((uintptr_t)grad_out & 7u))
        return tfail(t, MC_ERR_INVALID_ARG, "theta, value_out and grad_out must be FP64 device pointers");
    if (path0 + n_paths < path0) return tfail(t, MC_ERR_INVALID_ARG, "path range overflows");
    cudaStream_t st = (cudaStream_t)stream;
    mc_status r;
    if (t->jit)
        r = t->precision == MC_FP64 ? run_tape_jit<double>(t, theta, seed, path0, n_paths, value_out, grad_out, st)
                                    : run_tape_jit<float>(t, theta, seed, path0, n_paths, value_out, grad_out, st);
    else
        r = t->precision == MC_FP64 ? run_tape<double>(t, theta, seed, path0, n_paths, value_out, grad_out, st)
                                    : run_tape<float>(t, theta, seed, path0, n_paths, value_out, grad_out, st);
    if (r == MC_OK) t->last_n = n_paths;
    return r;
}

mc_status mc_tape_path_values(mc_tape *t, int32_t node, double *out, void *stream) {
    if (!t) return MC_ERR_INVALID_ARG;
    if (node < 0 || node >= t->plan.n_nodes || t->plan.cls[node] != 1 || !out || ((uintptr_t)out & 7u))
        return tfail(t, MC_ERR_INVALID_ARG, "node %d is not a per-path node, or out is not FP64-aligned", node);
    if (!(t->jit ? t->jit->store[node] : t->lists.stored[node]))
        return tfail(t, MC_ERR_UNSUPPORTED, "node %d is not kept on the tape (nothing reads it from there)", node);
    if (t->last_n == 0) return tfail(t, MC_ERR_STATE, "no evaluation yet");
    const size_t rb = t->precision == MC_FP64 ? 8 : 4;
    const unsigned char *row = (const unsigned char *)t->tape + (size_t)t->plan.ref[node] * t->stride * rb;
    cudaStream_t st = (cudaStream_t)stream;
    if (t->precision == MC_FP64) {
        const cudaError_t e = cudaMemcpyAsync(out, row, t->last_n * 8, cudaMemcpyDeviceToDevice, st);
        return e == cudaSuccess ? MC_OK : tfail(t, MC_ERR_CUDA, "copy: %s", cudaGetErrorString(e));
    }
    const int blocks = (int)std::min<uint64_t>((t->last_n + 255) / 256, 4096);
    tape_widen<<<blocks, 256, 0, st>>>((const float *)row, t->last_n, out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MC_OK : tfail(t, MC_ERR_CUDA, "widen: %s", cudaGetErrorString(e));
}

mc_status mc_tape_compile(mc_tape *t, int32_t seg_nodes, int32_t recompute, int32_t threads, double *seconds_out,
                          size_t *hbm_bytes_out) {
    if (!t) return MC_ERR_INVALID_ARG;
    if (seg_nodes <= 0) seg_nodes = 384;
    if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    const auto t0 = std::chrono::steady_clock::now();
    const size_t rb = t->precision == MC_FP64 ? 8 : 4;
    JitPlan *J = make_jit_plan(t->src_nodes, t->plan, seg_nodes, rb, recompute != 0, recompute > 1 ? recompute : 0);
    const int nseg = (int)J->segs.size();
    for (int k = 0; k < nseg; ++k) J->segs[k].src = gen_segment(t->src_nodes, t->plan, *J, k, t->precision);
    std::atomic<int> next(0), failed(-1);
    auto work = [&]() {
        for (int k = next++; k < nseg; k = next++)
            if (!rtc_compile(J->segs[k])) failed = k;
    };
    std::vector<std::thread> pool;
    for (int q = 0; q < std::min(threads, std::max(nseg, 1)); ++q) pool.emplace_back(work);
    for (std::thread &th : pool) th.join();
    if (failed >= 0) {
        const std::string head = J->segs[failed].log.substr(0, 400);
        jit_free(J);
        return tfail(t, MC_ERR_UNSUPPORTED, "run-time compilation of segment %d failed: %s", (int)failed, head.c_str());
    }
    cudaSetDevice(t->device);
    for (JitSeg &sg : J->segs) {
        cudaError_t e = cudaLibraryLoadData(&sg.lib, sg.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
        if (e == cudaSuccess) e = cudaLibraryGetKernel(&sg.fwd, sg.lib, "fwd");
        if (e == cudaSuccess) e = cudaLibraryGetKernel(&sg.bwd, sg.lib, "bwd");
        sg.smem_b = (size_t)kWarpsPerBlock * sg.dargs.size() * 8;
        if (e == cudaSuccess && sg.smem_b > 48 * 1024)
            e = cudaFuncSetAttribute((const void *)sg.bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sg.smem_b);
        int occ_f = 0, occ_b = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, (const void *)sg.fwd, kBlock, 0);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, (const void *)sg.bwd, kBlock, sg.smem_b);
        if (e != cudaSuccess) {
            jit_free(J);
            return tfail(t, MC_ERR_CUDA, "loading a compiled segment: %s", cudaGetErrorString(e));
        }
        const uint64_t cap = std::min<uint64_t>((t->max_paths + kBlock - 1) / kBlock, 32u * 1024u);
        sg.grid_f = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)std::max(occ_f, 1) * t->n_sm, cap));
        sg.grid_b = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)std::max(occ_b, 1) * t->n_sm, cap));
        sg.cubin.clear();
        sg.cubin.shrink_to_fit();
        sg.src.clear();
    }
    if (!J->dslot.empty()) {
        cudaError_t e = cudaMalloc((void **)&J->dslot_dev, J->dslot.size() * 4);
        if (e == cudaSuccess) e = cudaMemcpy(J->dslot_dev, J->dslot.data(), J->dslot.size() * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            jit_free(J);
            return tfail(t, MC_ERR_CUDA, "segment tables: %s", cudaGetErrorString(e));
        }
    }
    if (!J->far_rows.empty()) {
        cudaError_t e = cudaMalloc((void **)&J->frows_dev, J->far_rows.size() * 4);
        if (e == cudaSuccess)
            e = cudaMemcpy(J->frows_dev, J->far_rows.data(), J->far_rows.size() * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            jit_free(J);
            return tfail(t, MC_ERR_CUDA, "segment tables: %s", cudaGetErrorString(e));
        }
    }
    jit_free(t->jit);
    t->jit = J;
    t->last_n = 0;
    if (seconds_out)
        *seconds_out = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (hbm_bytes_out) *hbm_bytes_out = J->bytes_per_path;
    return MC_OK;
}

}  // extern "C"
