// mc_paths.cuh -- the forward sweep F_v and the reverse sweep R_v of the
// two-step algorithm (arXiv 1901.04200), one thread per Monte Carlo path.
//
// Paths are processed in chunks of 32*PPT consecutive global paths per warp:
// lane l carries paths chunk*32*PPT + q*32 + l for q < PPT (PPT independent
// recursions per thread give the scheduler instruction-level parallelism);
// a block of kBlock threads walks its warps over chunks blockIdx*W + warp,
// + gridDim*W, ...  The time axis is cut into segments of K steps (K a
// template constant, so a segment's steps are unrolled and the reverse
// sweep's tape lives in registers).  Every maturity lies on a segment end.
//
// Forward kernel (step 1, eq. 1211A): per segment, optionally store the state
// (checkpoint) and, in the stored-normals variant, the segment's normals into
// the warp chunk's tile (SegTile below: rows of 32 consecutive paths), run K
// Euler steps with Philox normals (segments visited in groups that fill whole
// Philox blocks), and at a maturity sum the undiscounted call payoffs of the
// warp's 32 paths (FP32 warp sum) into per-warp FP64 accumulators.  Block
// end: the warps' sums in warp order -> part_y[block][i].
//
// Reverse kernel (step 2, eq. 0711A): per path, segments from last to first:
// reload the checkpoint (staged in shared memory one segment ahead), re-run
// the segment's K steps (regenerating the normals, or reading the stored
// ones) while recording what the adjoint needs, add the payoff seeds
// lambda_i e^{-rT_i} 1{S>K_i} S of a maturity at the segment end to x-bar,
// then run the adjoint of the K steps backwards.  Parameter adjoints are
// summed per thread over its paths in the path precision, then warp-summed
// and added in FP64 to per-warp accumulators (one lane per value); block end
// -> part_g[block][j].  No atomics: the result is deterministic for a given
// launch shape.
#pragma once
#include "mc_common.cuh"

#include <type_traits>

namespace mcaad {

template <typename T>
__device__ __forceinline__ T rsqrt_r(T x);
template <>
__device__ __forceinline__ float rsqrt_r<float>(float x) { return rsqrt_approx(x); }  // x >= 1e-30 where used
template <>
__device__ __forceinline__ double rsqrt_r<double>(double x) { return rsqrt(x); }

// 1/x: the hardware approximation in FP32 (relative error about one ulp), exact division in FP64
template <typename T>
__device__ __forceinline__ T recip_r(T x);
template <>
__device__ __forceinline__ float recip_r<float>(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <>
__device__ __forceinline__ double recip_r<double>(double x) { return 1.0 / x; }

template <typename T>
__device__ __forceinline__ T exp_r(T x);
template <>
__device__ __forceinline__ float exp_r<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double exp_r<double>(double x) { return exp(x); }

template <typename T>
__device__ __forceinline__ T tiny_r();
template <>
__device__ __forceinline__ float tiny_r<float>() { return 1e-30f; }
template <>
__device__ __forceinline__ double tiny_r<double>() { return 1e-300; }

// ------------------------------------------------------- shared layout ----

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Dynamic shared memory of a path kernel, identical on host and device.
struct SmemPlan {
    size_t strike, grp_seg, grp_begin, seed_w, wacc_y, wacc_g, model, zstage, total;
    // zstage_bytes: the reverse sweep's staging buffers for stored normals (0 otherwise)
    // node_table: the local-vol surface as node pairs per time cell instead of per-step rows (the
    // stored-states reverse sweep, which looks the surface up once per step)
    __host__ __device__ SmemPlan(int kind, int real_bytes, int m, int n_groups, int M, int n_steps,
                                 int nx, bool reverse, size_t zstage_bytes = 0, bool node_table = false) {
        size_t o = 0;
        strike = o;    o = align_up(o + (size_t)m * real_bytes, 16);
        grp_seg = o;   o = align_up(o + (size_t)n_groups * 4, 16);
        grp_begin = o; o = align_up(o + (size_t)(n_groups + 1) * 4, 16);
        seed_w = o;    o = align_up(o + (reverse ? (size_t)m * real_bytes : 0), 16);
        wacc_y = o;    o = align_up(o + (reverse ? 0 : (size_t)kWarpsPerBlock * m * 8), 16);
        wacc_g = o;    o = align_up(o + (reverse ? (size_t)kWarpsPerBlock * M * 8 : 0), 16);
        model = o;
        if (kind == kGbm) {
            o += (size_t)M * real_bytes;
            o = align_up(o, 16);
            o += (size_t)n_steps * 4;
        } else if (kind == kLv || kind == kSlv) {
            if (node_table) o += (size_t)((kind == kSlv ? M - 5 : M) / nx - 1) * nx * 2 * real_bytes;  // node pairs
            else o += (size_t)n_steps * nx * real_bytes;  // time-interpolated node rows
            o = align_up(o, 16);
            o += (size_t)n_steps * real_bytes;       // time weight a_n
            o = align_up(o, 16);
            o += (size_t)n_steps * 4;                // time cell jt_n
            o = align_up(o, 16);
            if (reverse) o += (size_t)nx * 2 * real_bytes * kBlock;  // per-thread node adjoints
        }
        zstage = o = align_up(o, 16);
        o += zstage_bytes;
        total = align_up(o, 16);
    }
};

// Warp-sum n values v[0..n) and add sum j, in FP64, to wacc_row[idx0 + j];
// lane j performs the add for value j (one FP64 instruction per 32 values).
template <typename Real, int N>
__device__ __forceinline__ void warp_flush_n(double *wacc_row, int idx0, const Real (&v)[N], int lane) {
    Real mine = Real(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const Real s = warp_sum(v[j]);
        mine = (lane == (j & 31)) ? s : mine;
        if ((j & 31) == 31 || j == N - 1) {
            if (lane <= (j & 31)) wacc_row[idx0 + (j & ~31) + lane] += (double)mine;
            mine = Real(0);
        }
    }
}

// ================================================================ models ====
//
// Model interface used by the kernels:
//   State / Tape        per path; Tape is what the adjoint of one step needs
//   Acc                 per thread: linear sums over the thread's paths of a chunk
//   setup(...)          block-level preparation (shared tables, parameters)
//   step(st, z, n, ...) one Euler step; records the tape when given one
//   boundary(acc, n, ...)  before the adjoints of step n (warp-uniform): flush
//                       accumulators whose parameter slot changes
//   adjoint(tape, n, xb, vb, acc, ...)  adjoint of step n for one path
//   acc_end(acc, vb_sum, ...)  flush at the end of a chunk

// GBM, piecewise-constant volatility theta_b over buckets of steps, log-Euler:
// x += (r - theta_b^2/2) dt + theta_b sqrt(dt) z_n.
template <typename Real_>
struct GbmModel {
    using Real = Real_;
    static constexpr int kind = kGbm;
    static constexpr int DZ = 1, SD = 1;
    static constexpr bool kKeysInRegisters = false;
    static constexpr bool kPhiloxWide = true;   // Philox by wide multiplies
    struct State { Real x; };
    struct Tape { Real z; };
    struct Shared {
        const Real *vol;
        const int *bucket;
    };
    struct Par { Real rdt, dt, sdt; };
    struct Acc { Real g; int b; };

    __device__ static void setup(unsigned char *base, const SmemPlan &sp, const DevProblem &pb,
                                 const double *theta, int n_steps, Shared &sh, Par &par) {
        Real *vol = (Real *)(base + sp.model);
        int *bucket = (int *)(base + align_up(sp.model + (size_t)pb.M * sizeof(Real), 16));
        for (int j = threadIdx.x; j < pb.M; j += blockDim.x) vol[j] = (Real)theta[j];
        for (int n = threadIdx.x; n < n_steps; n += blockDim.x) bucket[n] = pb.bucket_of_step[n];
        sh.vol = vol;
        sh.bucket = bucket;
        par.dt = (Real)pb.dt;
        par.rdt = (Real)(pb.r * pb.dt);
        par.sdt = (Real)sqrt(pb.dt);
    }
    __device__ static State init(const Par &) { return State{Real(0)}; }
    __device__ __forceinline__ static void step(State &s, const Real *z, int n, const Par &p,
                                                const Shared &sh, Tape *t) {
        const Real vol = sh.vol[sh.bucket[n]];
        s.x = s.x + ((p.rdt - Real(0.5) * vol * vol * p.dt) + vol * p.sdt * z[0]);
        if (t) t->z = z[0];
    }
    __device__ static void acc_begin(Acc &a, int n_last, const Shared &sh) {
        a.g = Real(0);
        a.b = sh.bucket[n_last - 1];
    }
    __device__ __forceinline__ static void boundary(Acc &a, int n, const Shared &sh, double *wacc, int lane) {
        const int b = sh.bucket[n];
        if (b != a.b) {  // uniform across the warp: all lanes are at step n
            const Real v[1] = {a.g};
            warp_flush_n(wacc, a.b, v, lane);
            a.g = Real(0);
            a.b = b;
        }
    }
    // x_{n+1} = x_n + ... : x-bar passes through; theta_b-bar += xb (-vol dt + sqrt(dt) z).
    __device__ __forceinline__ static void adjoint(const Tape &t, int, Real &xb, Real &, Acc &a,
                                                   const Par &p, const Shared &sh) {
        const Real vol = sh.vol[a.b];
        a.g += xb * (p.sdt * t.z - vol * p.dt);
    }
    __device__ static void acc_end(Acc &a, Real, const Par &, const Shared &, double *wacc, int lane) {
        const Real v[1] = {a.g};
        warp_flush_n(wacc, a.b, v, lane);
    }
};

// Heston with full-truncation Euler, theta = (kappa, theta_h, xi, rho, v0):
// vdt = max(v,0) dt, sq = sqrt(vdt) (as vdt * rsqrt(max(vdt, tiny)), which is
// exactly 0 at vdt = 0), w = rho z1 + sqrt(1-rho^2) z2,
// x += (r dt - vdt/2) + sq z1,  v += (kappa theta_h dt - kappa vdt) + xi sq w.
template <typename Real_>
struct HestonModel {
    using Real = Real_;
    static constexpr int kind = kHeston;
    static constexpr int DZ = 2, SD = 2;
    static constexpr bool kKeysInRegisters = false;
    static constexpr bool kPhiloxWide = true;   // Philox by wide multiplies
    struct State { Real x, v; };
    struct Tape { Real vdt, rs, z1, w; };
    struct Shared {};
    struct Par { Real kappa, thh, xi, rho, rhob, v0, dt, rdt, kthdt; };
    // sums over paths: kappa-bar, vb, vb sq z1, vb sq w
    struct Acc { Real kb, cs, a, b; };

    __device__ static void setup(unsigned char *, const SmemPlan &, const DevProblem &pb,
                                 const double *theta, int, Shared &, Par &par) {
        const double kappa = theta[0], thh = theta[1], xi = theta[2], rho = theta[3];
        par.kappa = (Real)kappa;
        par.thh = (Real)thh;
        par.xi = (Real)xi;
        par.rho = (Real)rho;
        par.rhob = (Real)sqrt(1.0 - rho * rho);
        par.v0 = (Real)theta[4];
        par.dt = (Real)pb.dt;
        par.rdt = (Real)(pb.r * pb.dt);
        par.kthdt = (Real)(kappa * thh * pb.dt);
    }
    __device__ static State init(const Par &p) { return State{Real(0), p.v0}; }
    __device__ __forceinline__ static void step(State &s, const Real *z, int, const Par &p,
                                                const Shared &, Tape *t) {
        const Real vdt = fmax(s.v, Real(0)) * p.dt;
        const Real rs = rsqrt_r<Real>(fmax(vdt, tiny_r<Real>()));
        const Real sq = vdt * rs;
        const Real z1 = z[0];
        const Real w = fma(p.rho, z1, p.rhob * z[1]);
        s.x = s.x + fma(sq, z1, fma(Real(-0.5), vdt, p.rdt));
        s.v = s.v + fma(p.xi * sq, w, fma(-p.kappa, vdt, p.kthdt));
        if (t) {
            t->vdt = vdt;
            t->rs = rs;
            t->z1 = z1;
            t->w = w;
        }
    }
    __device__ static void acc_begin(Acc &a, int, const Shared &) { a.kb = a.cs = a.a = a.b = Real(0); }
    __device__ __forceinline__ static void boundary(Acc &, int, const Shared &, double *, int) {}
    // Adjoint of one step given xb, vb of the state after it:
    //   kappa-bar += vb (theta_h dt - vdt), theta_h-bar += vb kappa dt,
    //   xi-bar += vb sq w, rho-bar += vb xi sq dw/drho,
    //   vdt-bar = -xb/2 - kappa vb + (xb z1 + xi vb w) / (2 sq),
    //   vb_prev = vb + 1{v > 0} dt vdt-bar,  xb_prev = xb.
    __device__ __forceinline__ static void adjoint(const Tape &t, int, Real &xb, Real &vb, Acc &a,
                                                   const Par &p, const Shared &) {
        const Real sq = t.vdt * t.rs;
        const Real vsq = vb * sq;
        a.a = fma(vsq, t.z1, a.a);
        a.b = fma(vsq, t.w, a.b);
        a.cs += vb;
        a.kb = fma(vb, p.thh * p.dt - t.vdt, a.kb);
        const Real sqb = fma(xb, t.z1, p.xi * vb * t.w);
        const Real vdtb = fma(Real(0.5) * t.rs, sqb, fma(Real(-0.5), xb, -p.kappa * vb));
        vb = (t.vdt > Real(0)) ? fma(vdtb, p.dt, vb) : vb;
    }
    // theta-bar = (kb, kappa dt cs, b, xi (a - rho b) / (1 - rho^2), sum of vb at step 0);
    // d w / d rho = z1 - rho z2 / rhob = (z1 - rho w) / rhob^2.
    __device__ static void acc_end(Acc &a, Real vb_sum, const Par &p, const Shared &, double *wacc, int lane) {
        const Real v[5] = {a.kb, p.kappa * p.dt * a.cs, a.b, p.xi * (a.a - p.rho * a.b) / (p.rhob * p.rhob),
                           vb_sum};
        warp_flush_n(wacc, 0, v, lane);
    }
};

// Local volatility on a bilinear node surface theta[j*nx + c] over
// (t_j, x_c), flat extrapolation; log-Euler with sigma at (t_n, x_n):
// x += (r - sigma^2/2) dt + sigma sqrt(dt) z_n.  The time interpolation is the
// same for every path at step n, so each block first forms the rows
// row_n[c] = (1 - a_n) theta[jt_n][c] + a_n theta[jt_n + 1][c].
template <typename Real_>
struct LvModel {
    using Real = Real_;
    static constexpr int kind = kLv;
    static constexpr int DZ = 1, SD = 1;
    static constexpr bool kKeysInRegisters = true;
    static constexpr bool kPhiloxWide = false;  // Philox by low and high multiplies: measured faster here
    static constexpr int kMaxNx = 32;
    struct State { Real x; };
    struct Tape { Real u, z; };  // u = (x - x_lo)/hx, z
    struct Shared {
        const Real *row;  // [n_steps][nx]
        const Real *a;    // [n_steps]
        const int *jt;    // [n_steps]
        Real *racc;       // reverse: [nx][kBlock][2] per-thread node adjoints of rows jt, jt+1
        const Real *node; // node_table: [nt-1][nx][2] (theta[j][c], theta[j+1][c] - theta[j][c]) x sqrt(dt)
        int nx;
    };
    // u0 = -x_lo / hx, so that the scaled coordinate u = (x - x_lo) / hx is one FMA
    struct Par { Real rdt, dt, sdt, x_lo, inv_hx, u0, nxm1; int nxm2; };
    // jt: the time row being accumulated; at, oma: a_n and 1 - a_n of the step
    // whose adjoints run next
    struct Acc { int jt; Real at, oma; };

    // Local vol keeps its surface premultiplied by sqrt(dt): a row entry is h = sigma sqrt(dt),
    // the step's diffusion coefficient, so the step and its adjoint need no products with dt.
    // The reverse sweep is linear in its seeds, which load_tables scales by sqrt(dt) for local
    // vol, so the node adjoints come out as d/d theta = sqrt(dt) d/d h.  A leverage surface
    // (SlvModel) is kept as it is.
    __device__ static void setup(unsigned char *base, const SmemPlan &sp, const DevProblem &pb,
                                 const double *theta, int n_steps, Shared &sh, Par &par, bool node_table = false,
                                 bool leverage = false) {
        const int nx = pb.nx;
        const double sc = leverage ? 1.0 : sqrt(pb.dt);
        Real *row = (Real *)(base + sp.model);
        size_t o = align_up(sp.model + (node_table ? (size_t)(pb.nt - 1) * nx * 2 : (size_t)n_steps * nx) * sizeof(Real),
                            16);
        Real *a = (Real *)(base + o);
        o = align_up(o + (size_t)n_steps * sizeof(Real), 16);
        int *jt = (int *)(base + o);
        o = align_up(o + (size_t)n_steps * 4, 16);
        sh.racc = (Real *)(base + o);
        for (int n = threadIdx.x; n < n_steps; n += blockDim.x) {
            a[n] = (Real)pb.lv_a[n];
            jt[n] = pb.lv_jt[n];
        }
        if (node_table) {
            for (int q = threadIdx.x; q < (pb.nt - 1) * nx; q += blockDim.x) {
                row[2 * q] = (Real)(sc * theta[q]);
                row[2 * q + 1] = (Real)(sc * (theta[q + nx] - theta[q]));
            }
            sh.row = nullptr;
            sh.node = row;
        } else {
            for (int q = threadIdx.x; q < n_steps * nx; q += blockDim.x) {
                const int n = q / nx, c = q - n * nx;
                const int j = pb.lv_jt[n];
                const double w = pb.lv_a[n];
                row[q] = (Real)(sc * ((1.0 - w) * theta[j * nx + c] + w * theta[(j + 1) * nx + c]));
            }
            sh.node = nullptr;
        }
        sh.row = node_table ? nullptr : row;
        sh.a = a;
        sh.jt = jt;
        sh.nx = nx;
        par.dt = (Real)pb.dt;
        par.rdt = (Real)(pb.r * pb.dt);
        par.sdt = (Real)sqrt(pb.dt);
        par.x_lo = (Real)pb.x_lo;
        par.inv_hx = (Real)(1.0 / pb.hx);
        par.u0 = (Real)(-pb.x_lo / pb.hx);
        par.nxm1 = (Real)(nx - 1);
        par.nxm2 = nx - 2;
    }
    __device__ static State init(const Par &) { return State{Real(0)}; }

    // The scaled coordinate u = (x - x_lo) / hx.
    __device__ __forceinline__ static Real scaled(Real x, const Par &p) { return fma(x, p.inv_hx, p.u0); }
    // Cell c = clamp(floor(u), 0, nx-2) and weight b = clamp(u - c, 0, 1): with uc = clamp(u, 0,
    // nx-1), c = floor(min(uc, nx-2)) and b = uc - c lies in [0, 1] by construction; inside
    // (x not clamped, d sigma/dx not zero) is u == uc.  In FP32 the floor (of a value in
    // [0, 30]) comes from one addition of 1.5 2^23 rounded toward minus infinity: the sum's last
    // place is 1, so it holds 1.5 2^23 + floor, its low bits are the integer, and subtracting
    // 1.5 2^23 again is exact -- no conversion instructions.
    __device__ __forceinline__ static void cell(Real u, const Par &p, int &c, Real &b, bool &inside) {
        const Real uc = fmin(fmax(u, Real(0)), p.nxm1);
        Real f;
        if constexpr (sizeof(Real) == 4) {
            const float r = __fadd_rd(fminf(uc, (float)p.nxm2), 12582912.0f);
            f = r - 12582912.0f;
            c = __float_as_int(r) - 0x4B400000;
        } else {
            f = floor(fmin(uc, (Real)p.nxm2));
            c = (int)f;
        }
        b = uc - f;
        inside = u == uc;
    }
    __device__ __forceinline__ static void step(State &s, const Real *z, int n, const Par &p,
                                                const Shared &sh, Tape *t) {
        const Real u = scaled(s.x, p);
        int c;
        Real b;
        bool inside;
        cell(u, p, c, b, inside);
        const Real *rw = sh.row + n * sh.nx;
        const Real h0 = rw[c], h1 = rw[c + 1];
        const Real h = fma(b, h1 - h0, h0);  // sigma sqrt(dt)
        // x + r dt - sigma^2 dt / 2 + sigma sqrt(dt) z = x + (h (z - h / 2) + r dt): the small
        // increment is formed first and x rounded once per step
        s.x = s.x + fma(h, fma(Real(-0.5), h, z[0]), p.rdt);
        if (t) {
            t->u = u;
            t->z = z[0];
        }
    }
    // Node k's pair (row jt, row jt+1) of thread t: one 2-vector at (k * kBlock + t) * 2.
    __device__ __forceinline__ static Real *acc_slot(const Shared &sh, int k) {
        return sh.racc + (k * kBlock + (int)threadIdx.x) * 2;
    }
    __device__ __forceinline__ static void add_node(const Shared &sh, const Acc &a, int k, Real g) {
        Real *r = acc_slot(sh, k);
        if constexpr (sizeof(Real) == 4) {
            float2 v = *(float2 *)r;
            v.x = fma(a.oma, g, v.x);
            v.y = fma(a.at, g, v.y);
            *(float2 *)r = v;
        } else {
            double2 v = *(double2 *)r;
            v.x = fma(a.oma, g, v.x);
            v.y = fma(a.at, g, v.y);
            *(double2 *)r = v;
        }
    }
    __device__ static void acc_begin(Acc &a, int n_last, const Shared &sh) {
        a.jt = sh.jt[n_last - 1];
        a.at = a.oma = Real(0);
        for (int k = 0; k < sh.nx; ++k) {
            Real *r = acc_slot(sh, k);
            r[0] = r[1] = Real(0);
        }
    }
    // Rows jt and jt+1 are the contiguous node range [jt*nx, (jt+2)*nx); each node's pair is read
    // and cleared with one 2-vector access per lane (conflict-free: lanes hit consecutive pairs).
    __device__ __noinline__ static void flush_rows(Acc &a, const Shared &sh, double *wacc, int lane) {
        using Pair = typename std::conditional<sizeof(Real) == 4, float2, double2>::type;
        const int nx = sh.nx;
        Real mine0 = Real(0), mine1 = Real(0);
        for (int k = 0; k < nx; ++k) {
            Pair *r = (Pair *)acc_slot(sh, k);
            const Pair v = *r;
            Pair z;
            z.x = z.y = Real(0);
            *r = z;
            const Real s0 = warp_sum(v.x), s1 = warp_sum(v.y);
            mine0 = (lane == k) ? s0 : mine0;
            mine1 = (lane == k) ? s1 : mine1;
        }
        if (lane < nx) {
            wacc[a.jt * nx + lane] += (double)mine0;
            wacc[(a.jt + 1) * nx + lane] += (double)mine1;
        }
    }
    __device__ __forceinline__ static void boundary(Acc &a, int n, const Shared &sh, double *wacc, int lane) {
        const int jt = sh.jt[n];
        if (jt != a.jt) {  // uniform across the warp
            flush_rows(a, sh, wacc, lane);
            a.jt = jt;
        }
        a.at = sh.a[n];
        a.oma = Real(1) - a.at;
    }
    // h-bar = xb (z - h) (h = sigma sqrt(dt)); node adjoints h-bar times the bilinear weights
    // (xb carries the seeds' factor sqrt(dt)); xb += h-bar dh/dx (0 where x is clamped).
    __device__ __forceinline__ static void adjoint(const Tape &t, int n, Real &xb, Real &, Acc &a,
                                                   const Par &p, const Shared &sh) {
        int c;
        Real b;
        bool inside;
        cell(t.u, p, c, b, inside);
        const Real *rw = sh.row + n * sh.nx;
        const Real h0 = rw[c], h1 = rw[c + 1];
        const Real dh = h1 - h0;
        const Real h = fma(b, dh, h0);
        const Real hb = xb * (t.z - h);
        const Real g1 = hb * b, g0 = hb - g1;
        add_node(sh, a, c, g0);
        add_node(sh, a, c + 1, g1);
        if (inside) xb = fma(hb * p.inv_hx, dh, xb);
    }
    // Step n with the surface read from the per-time-cell node pairs (setup with node_table):
    // the row value at the step's time is theta_jt + a_n (theta_jt+1 - theta_jt), formed in Real
    // instead of read from a per-step row (the reverse sweep that re-runs segments into shared
    // memory, which holds the node table and not the rows).
    __device__ __forceinline__ static void step_nodes(State &s, Real z, int n, const Par &p, const Shared &sh) {
        const Real u = scaled(s.x, p);
        int c;
        Real b;
        bool inside;
        cell(u, p, c, b, inside);
        using P2 = typename std::conditional<sizeof(Real) == 4, float2, double2>::type;
        const Real at = sh.a[n];
        const P2 *nd = (const P2 *)sh.node + sh.jt[n] * sh.nx + c;
        const P2 n0 = nd[0], n1 = nd[1];
        const Real h0 = fma(at, n0.y, n0.x), h1 = fma(at, n1.y, n1.x);
        const Real h = fma(b, h1 - h0, h0);
        s.x = s.x + fma(h, fma(Real(-0.5), h, z), p.rdt);
    }
    // The adjoint of step n from the states at both of its ends (stored-states variant): the
    // step x1 = x0 + r dt + h z - h^2 / 2 (h = sigma sqrt(dt)) gives
    // d x1 / d h = z - h = (x1 - x0 - r dt - h^2 / 2) / h,
    // so the adjoint needs neither the normal nor a re-run of the step (sigma != 0).
    // The time cell's node pairs at x cells c and c+1: h = a0 + at d0 at node c, a1 + at d1 at c+1.
    struct NodePair { Real a0, d0, a1, d1; };
    __device__ __forceinline__ static NodePair node_pair(const Shared &sh, int jt, int c) {
        using P2 = typename std::conditional<sizeof(Real) == 4, float2, double2>::type;
        const P2 *nd = (const P2 *)sh.node + jt * sh.nx + c;
        const P2 n0 = nd[0], n1 = nd[1];
        return NodePair{n0.x, n0.y, n1.x, n1.y};
    }
    // Shared body of the two forms below, given the step's cell and its node pairs.
    __device__ __forceinline__ static void adjoint_states_with(const State &s0, const State &s1, int c, Real b,
                                                               bool inside, const NodePair &q, Real &xb, Acc &a,
                                                               const Par &p, const Shared &sh) {
        const Real v0 = fma(a.at, q.d0, q.a0), v1 = fma(a.at, q.d1, q.a1);
        const Real dh = v1 - v0;
        const Real h = fma(b, dh, v0);
        const Real dxdh = fma(Real(-0.5) * h, h, s1.x - s0.x - p.rdt) * recip_r<Real>(h);
        const Real hb = xb * dxdh;
        const Real g1 = hb * b, g0 = hb - g1;
        add_node(sh, a, c, g0);
        add_node(sh, a, c + 1, g1);
        if (inside) xb = fma(hb * p.inv_hx, dh, xb);
    }
    __device__ __forceinline__ static void adjoint_states(const State &s0, const State &s1, int n, Real &xb, Real &,
                                                          Acc &a, const Par &p, const Shared &sh) {
        const Real u = scaled(s0.x, p);
        int c;
        Real b;
        bool inside;
        cell(u, p, c, b, inside);
        adjoint_states_with(s0, s1, c, b, inside, node_pair(sh, a.jt, c), xb, a, p, sh);  // (a.jt, a.at: step n)
    }
    // The same with the last node pairs a path slot read kept in registers: a path stays in its cell
    // for most steps, so the reload (a shared-memory read by the lanes whose cell or time cell
    // changed) is predicated off for most lanes, and the warp's read costs one wavefront instead
    // of two per pair.
    struct NodeCache {
        int key;  // jt * 64 + c of the pairs held (nx <= kMaxNx = 32), -1 for none
        NodePair q;
    };
    __device__ __forceinline__ static void adjoint_states_cached(const State &s0, const State &s1, Real &xb, Acc &a,
                                                                 const Par &p, const Shared &sh, NodeCache &nc) {
        const Real u = scaled(s0.x, p);
        int c;
        Real b;
        bool inside;
        cell(u, p, c, b, inside);
        const int key = a.jt * 64 + c;
        if (key != nc.key) {
            nc.q = node_pair(sh, a.jt, c);
            nc.key = key;
        }
        adjoint_states_with(s0, s1, c, b, inside, nc.q, xb, a, p, sh);
    }
    __device__ static void acc_end(Acc &a, Real, const Par &, const Shared &sh, double *wacc, int lane) {
        flush_rows(a, sh, wacc, lane);
    }
};

// Heston stochastic local volatility (the paper's test model): the Heston
// variance process with full truncation, and x driven by sqrt(v+) times a
// leverage L(t_n, x_n) interpolated bilinearly on fixed nodes;
// theta = (kappa, theta_h, xi, rho, v0, L[j*nx + c]).  Per step:
//   x += (r dt - L^2 vdt / 2) + L sq z1,  v as HestonModel.
// The leverage surface reuses LvModel's tables, cell logic and per-thread row
// adjoints (node j*nx + c is parameter 5 + j*nx + c).
template <typename Real_>
struct SlvModel {
    using Real = Real_;
    using Lv = LvModel<Real_>;
    using Hs = HestonModel<Real_>;
    static constexpr int kind = kSlv;
    static constexpr int DZ = 2, SD = 2;
    static constexpr bool kKeysInRegisters = true;
    static constexpr bool kPhiloxWide = true;   // Philox by wide multiplies
    struct State { Real x, v; };
    struct Tape { Real u, vdt, rs, z1, w; };
    using Shared = typename Lv::Shared;
    struct Par {
        typename Hs::Par h;
        typename Lv::Par l;
    };
    struct Acc {
        typename Hs::Acc h;
        typename Lv::Acc l;
    };

    __device__ static void setup(unsigned char *base, const SmemPlan &sp, const DevProblem &pb,
                                 const double *theta, int n_steps, Shared &sh, Par &par) {
        typename Hs::Shared hs;
        Hs::setup(base, sp, pb, theta, n_steps, hs, par.h);
        Lv::setup(base, sp, pb, theta + 5, n_steps, sh, par.l, false, true);
    }
    __device__ static State init(const Par &p) { return State{Real(0), p.h.v0}; }
    __device__ __forceinline__ static void step(State &s, const Real *z, int n, const Par &p,
                                                const Shared &sh, Tape *t) {
        const Real u = Lv::scaled(s.x, p.l);
        int c;
        Real b;
        bool inside;
        Lv::cell(u, p.l, c, b, inside);
        const Real *rw = sh.row + n * sh.nx;
        const Real s0 = rw[c], s1 = rw[c + 1];
        const Real lev = fma(b, s1 - s0, s0);
        const Real vdt = fmax(s.v, Real(0)) * p.h.dt;
        const Real rs = rsqrt_r<Real>(fmax(vdt, tiny_r<Real>()));
        const Real sq = vdt * rs;
        const Real z1 = z[0];
        const Real w = fma(p.h.rho, z1, p.h.rhob * z[1]);
        s.x = s.x + fma(lev * sq, z1, fma(Real(-0.5) * lev * lev, vdt, p.h.rdt));
        s.v = s.v + fma(p.h.xi * sq, w, fma(-p.h.kappa, vdt, p.h.kthdt));
        if (t) {
            t->u = u;
            t->vdt = vdt;
            t->rs = rs;
            t->z1 = z1;
            t->w = w;
        }
    }
    __device__ static void acc_begin(Acc &a, int n_last, const Shared &sh) {
        Hs::acc_begin(a.h, n_last, typename Hs::Shared{});
        Lv::acc_begin(a.l, n_last, sh);
    }
    // Leverage rows flush into parameters 5 + node.
    __device__ __forceinline__ static void boundary(Acc &a, int n, const Shared &sh, double *wacc, int lane) {
        Lv::boundary(a.l, n, sh, wacc + 5, lane);
    }
    // Adjoint of one step given xb, vb of the state after it:
    //   L-bar = xb (sq z1 - L vdt) -> bilinear node weights (time weight a_n),
    //   Heston parameter sums as HestonModel with d x/d sq = L z1,
    //   vdt-bar = -xb L^2/2 - kappa vb + (xb L z1 + xi vb w) / (2 sq),
    //   vb_prev = vb + 1{v > 0} dt vdt-bar,  xb_prev = xb + L-bar dL/dx.
    __device__ __forceinline__ static void adjoint(const Tape &t, int n, Real &xb, Real &vb, Acc &a,
                                                   const Par &p, const Shared &sh) {
        int c;
        Real b;
        bool inside;
        Lv::cell(t.u, p.l, c, b, inside);
        const Real *rw = sh.row + n * sh.nx;
        const Real s0 = rw[c], s1 = rw[c + 1];
        const Real ds = s1 - s0;
        const Real lev = fma(b, ds, s0);
        const Real sq = t.vdt * t.rs;
        const Real lb = xb * fma(sq, t.z1, -lev * t.vdt);
        const Real g1 = lb * b, g0 = lb - g1;
        Lv::add_node(sh, a.l, c, g0);
        Lv::add_node(sh, a.l, c + 1, g1);
        const Real vsq = vb * sq;
        a.h.a = fma(vsq, t.z1, a.h.a);
        a.h.b = fma(vsq, t.w, a.h.b);
        a.h.cs += vb;
        a.h.kb = fma(vb, p.h.thh * p.h.dt - t.vdt, a.h.kb);
        const Real sqb = fma(xb * lev, t.z1, p.h.xi * vb * t.w);
        const Real vdtb = fma(Real(0.5) * t.rs, sqb, fma(Real(-0.5) * lev * lev, xb, -p.h.kappa * vb));
        vb = (t.vdt > Real(0)) ? fma(vdtb, p.h.dt, vb) : vb;
        if (inside) xb = fma(lb * p.l.inv_hx, ds, xb);
    }
    __device__ static void acc_end(Acc &a, Real vb_sum, const Par &p, const Shared &sh, double *wacc, int lane) {
        Hs::acc_end(a.h, vb_sum, p.h, typename Hs::Shared{}, wacc, lane);
        Lv::acc_end(a.l, vb_sum, p.l, sh, wacc + 5, lane);
    }
};

// ============================================================== kernels ====

// Dynamic chunk assignment: lane 0 takes the warp's next chunk from the queue.
__device__ __forceinline__ uint64_t take_chunk(unsigned long long *q, int lane) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(q, 1ull);
    return __shfl_sync(0xffffffffu, c, 0);
}
// After the block's last chunk (all threads): the last block of the grid to finish resets the
// queue for the next launch (every other block has stopped taking chunks by then).
__device__ __forceinline__ void queue_done(unsigned long long *q) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(q + 1, 1ull) == (unsigned long long)gridDim.x - 1) {
            q[0] = 0ull;
            q[1] = 0ull;
        }
    }
}

// 16-byte asynchronous global -> shared copies (L1 bypassed), grouped per
// segment; wait_group<N> returns when at most N of the thread's groups are
// still in flight (a hardware wait, no polling).
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// 16-byte vectors of the path precision (4 floats or 2 doubles).
template <typename Real>
struct Vec16;
template <>
struct Vec16<float> {
    using T = float4;
    __device__ static T make(const float *v) { return make_float4(v[0], v[1], v[2], v[3]); }
    __device__ static float get(const T &x, int k) { return k == 0 ? x.x : k == 1 ? x.y : k == 2 ? x.z : x.w; }
};
template <>
struct Vec16<double> {
    using T = double2;
    __device__ static T make(const double *v) { return make_double2(v[0], v[1]); }
    __device__ static double get(const T &x, int k) { return k == 0 ? x.x : x.y; }
};

// What the forward sweep leaves for the reverse sweep, in tiles of one warp
// chunk (32*PPT consecutive paths) and one segment.  Rows: first -- in the
// stored-normals variant -- the segment's normals, row (i*DZ + c)*PPT + q for
// step i, component c, path slot q, then the checkpoint (the state at the
// segment's start), row RZ + w*PPT + q for state word w, padded to whole
// groups of G = 16 / sizeof(Real) rows.  Within a tile, lane l's G rows of
// group g are one 16-byte vector at ((g * 32) + l) * G: the forward sweep
// writes a group with one vector store per lane (a warp writes 512
// contiguous bytes) and the reverse sweep reads it with one vector load.
// Tile (chunk, s) starts at (s * n_chunks + chunk) * Rp * 32 elements
// (n_chunks: the chunks the workspace holds; the warps of a sweep work on
// nearby segments, so their tiles are close together), and every store and
// load of the tile is a compile-time offset from one base.  The reverse sweep copies a
// warp's tile of segment s-1 into its half of a two-buffer shared staging
// area (same layout) while it works on segment s, so HBM latency is paid
// once per chunk instead of once per segment.
// kMode 2 (stored states) keeps instead the state before each of the segment's steps, row
// (i*SD + w)*PPT + q, and no checkpoint rows; the state after the last step goes to one extra
// tile (segment index n_seg).
template <class Md, int K, int PPT, int kMode>
struct SegTile {
    using Real = typename Md::Real;
    using V = Vec16<Real>;
    static constexpr bool kZ = kMode == 1;
    static constexpr int RZ = kZ ? K * Md::DZ * PPT : 0;                          // normals rows
    static constexpr int R = kMode == 2 ? K * Md::SD * PPT : RZ + Md::SD * PPT;    // + checkpoint rows
    static constexpr int kG = 16 / (int)sizeof(Real);               // rows per vector group
    static constexpr int Rp = (R + kG - 1) / kG * kG;               // rows padded to whole groups
    static constexpr int kElems = Rp * kWarp;                       // elements per tile
    static constexpr int kPieces = kElems * (int)sizeof(Real) / 16; // 16-byte pieces per tile
    static constexpr size_t kWarpBytes = 2 * (size_t)kElems * sizeof(Real);
    static constexpr size_t kBlockBytes = kWarpBytes * kWarpsPerBlock;
    __device__ static constexpr int zrow(int i, int c, int q) { return (i * Md::DZ + c) * PPT + q; }
    __device__ static constexpr int crow(int w, int q) { return RZ + w * PPT + q; }
    __device__ static constexpr int srow(int i, int w, int q) { return (i * Md::SD + w) * PPT + q; }
    // group g of this lane (tile or staging buffer base, lane)
    __device__ __forceinline__ static typename V::T *group(Real *t, int g, int lane) {
        return (typename V::T *)(t + ((size_t)g * kWarp + lane) * kG);
    }
    __device__ __forceinline__ static const typename V::T *group(const Real *t, int g, int lane) {
        return (const typename V::T *)(t + ((size_t)g * kWarp + lane) * kG);
    }
    // row r of this lane from a tile or staging buffer (the group is one vector load)
    __device__ __forceinline__ static Real row(const Real *t, int r, int lane) {
        return V::get(*group(t, r / kG, lane), r % kG);
    }
    __device__ __forceinline__ static Real *tile(void *base, uint64_t chunk, uint64_t n_chunks, int s) {
        return (Real *)base + ((size_t)s * n_chunks + chunk) * kElems;
    }
    // Copy tile (chunk, s) into staging buffer (s & 1).
    __device__ __forceinline__ static void issue(Real *stage, const void *base, uint64_t chunk, uint64_t n_chunks,
                                                 int s, int lane) {
        __syncwarp();  // every lane is done with this buffer's previous segment
        Real *buf = stage + (size_t)(s & 1) * kElems;
        const Real *src = tile(const_cast<void *>(base), chunk, n_chunks, s);
        constexpr int kPer = 16 / (int)sizeof(Real);
#pragma unroll
        for (int p0 = 0; p0 < kPieces; p0 += kWarp) {
            const int p = p0 + lane;
            if (kPieces % kWarp == 0 || p < kPieces) cp_async16(buf + p * kPer, src + p * kPer);
        }
        cp_async_commit();
    }
};

// Segments of n normals per path that together fill whole Philox blocks of four.
__host__ __device__ constexpr int philox_period_segments(int n) { return n % 4 == 0 ? 1 : n % 2 == 0 ? 2 : 4; }

template <class Md>
struct NormalSource {
    using Real = typename Md::Real;
    PathNormals<Real> gen;
    const double *table;
    __device__ __forceinline__ void init(const DevProblem &pb, const DevCall &cl, uint64_t p) {
        gen.init(p);
        table = nullptr;
        if constexpr (Md::kind == kGbm) {  // a normals table is accepted for GBM only
            if (pb.normals) table = pb.normals + (size_t)(p - pb.normals_path0) * pb.normals_stride;
        }
    }
    // Normals of step n.  first: the Philox block holding the step's first normal
    // may not be loaded -- a path's first step, or a segment's first step where
    // segments are visited out of order (the recompute of the reverse sweep); a
    // forward sweep reuses the block across its segments, which for segments
    // that do not start on a block boundary (local vol, K = 5) saves a block
    // per segment.
    __device__ __forceinline__ void get(int n, bool first, Real *z, const RoundKeys &rk) {
#pragma unroll
        for (int c = 0; c < Md::DZ; ++c) {
            const uint32_t j = (uint32_t)(n * Md::DZ + c);
            if (Md::kind == kGbm && table) {
                z[c] = (Real)table[j];
            } else {
                if ((first && c == 0) || (j & 3u) == 0u) gen.template fill<Md::kPhiloxWide>(j >> 2, rk);
                z[c] = gen.pick(j & 3u);
            }
        }
    }
};

template <class Md>
__device__ __forceinline__ void load_tables(unsigned char *base, const SmemPlan &sp,
                                            const DevProblem &pb, bool reverse, const DevCall &cl) {
    using Real = typename Md::Real;
    Real *strike = (Real *)(base + sp.strike);
    int *gseg = (int *)(base + sp.grp_seg);
    int *gbeg = (int *)(base + sp.grp_begin);
    for (int i = threadIdx.x; i < pb.m; i += blockDim.x) strike[i] = (Real)pb.strike[i];
    for (int g = threadIdx.x; g < pb.n_groups; g += blockDim.x) gseg[g] = pb.grp_seg[g];
    for (int g = threadIdx.x; g <= pb.n_groups; g += blockDim.x) gbeg[g] = pb.grp_begin[g];
    if (reverse) {
        Real *sw = (Real *)(base + sp.seed_w);
        // local vol: sqrt(dt) turns the adjoints of its premultiplied surface into d/d theta
        const double ss = Md::kind == kLv ? sqrt(pb.dt) : 1.0;
        for (int i = threadIdx.x; i < pb.m; i += blockDim.x) sw[i] = (Real)(cl.seed_w[i] * ss);
        double *wg = (double *)(base + sp.wacc_g);
        for (int q = threadIdx.x; q < kWarpsPerBlock * pb.M; q += blockDim.x) wg[q] = 0.0;
    } else {
        double *wy = (double *)(base + sp.wacc_y);
        for (int q = threadIdx.x; q < kWarpsPerBlock * pb.m; q += blockDim.x) wy[q] = 0.0;
    }
}

template <class Md, int K, int PPT, bool kStoreZ = false>
__global__ void __launch_bounds__(kBlock) path_forward_kernel(const DevProblem pb, const DevCall cl) {
    using Real = typename Md::Real;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n_steps = pb.n_seg * K;
    const SmemPlan sp(Md::kind, sizeof(Real), pb.m, pb.n_groups, pb.M, n_steps, pb.nx, false);
    load_tables<Md>(smem, sp, pb, false, cl);
    typename Md::Shared sh;
    typename Md::Par par;
    Md::setup(smem, sp, pb, cl.theta, n_steps, sh, par);
    __syncthreads();

    const Real *strike = (const Real *)(smem + sp.strike);
    const int *gseg = (const int *)(smem + sp.grp_seg);
    const int *gbeg = (const int *)(smem + sp.grp_begin);
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    double *wy = (double *)(smem + sp.wacc_y) + warp * pb.m;
    const Real S0 = (Real)pb.S0;
    using TL = SegTile<Md, K, PPT, kStoreZ>;
    // Philox round keys: from the kernel parameters (constant bank), or formed
    // once per thread into registers, whichever measured faster for the model
    const RoundKeys rk = Md::kKeysInRegisters ? philox_round_keys(cl.seed) : cl.rk;
    // The stored-normals variant always keeps its tiles: a compile-time
    // condition leaves each unrolled segment one branch-free block to schedule.
    const bool keep = kStoreZ || cl.keep_ckpt;

    constexpr uint64_t kChunk = (uint64_t)kWarp * PPT;
    const uint64_t n_chunks = (cl.n_paths + kChunk - 1) / kChunk;
    const bool dyn = cl.queue != nullptr;  // chunks from the queue, one partial row per chunk
    for (uint64_t ch = dyn ? take_chunk(cl.queue, lane) : (uint64_t)blockIdx.x * kWarpsPerBlock + warp; ch < n_chunks;
         ch = dyn ? take_chunk(cl.queue, lane) : ch + (uint64_t)gridDim.x * kWarpsPerBlock) {
        uint64_t local[PPT];
        bool active[PPT];
        NormalSource<Md> rng[PPT];
        typename Md::State st[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            local[q] = ch * kChunk + q * kWarp + lane;
            active[q] = local[q] < cl.n_paths;
            rng[q].init(pb, cl, cl.path0 + (active[q] ? local[q] : 0));
            st[q] = Md::init(par);
        }
        int g = 0;
        // Segments in groups of kPeriod whose normals fill whole Philox blocks, so
        // that each normal's block refill and lane are compile-time constants
        // (local vol, K = 5: four segments per 20 normals; Heston: one segment).
        constexpr int kPeriod = philox_period_segments(K * Md::DZ);
        for (int sg = 0; sg * kPeriod < pb.n_seg; ++sg) {
#pragma unroll
            for (int ss = 0; ss < kPeriod; ++ss) {
                const int s = sg * kPeriod + ss;
                if (kPeriod > 1 && s >= pb.n_seg) break;
                // the segment's normals first: its Philox blocks are independent of the state, so
                // the scheduler can overlap them; then the K dependent Euler steps.  The tile's
                // groups (normals when kept, checkpoint) go out as soon as all their rows exist.
                Real zs[K][PPT][Md::DZ];
                Real *tl = TL::tile(cl.ckpt, ch, cl.ckpt_stride / kChunk, s);
                auto store_group = [&](int g0) {
                    Real v[TL::kG];
#pragma unroll
                    for (int k = 0; k < TL::kG; ++k) {
                        const int r = g0 + k;
                        if (r < TL::RZ) {
                            v[k] = zs[r / (Md::DZ * PPT)][r % PPT][(r / PPT) % Md::DZ];
                        } else if (r < TL::R) {
                            const int w = (r - TL::RZ) / PPT, q = (r - TL::RZ) % PPT;
                            if constexpr (Md::SD == 2) v[k] = w == 0 ? st[q].x : st[q].v;
                            else v[k] = st[q].x;
                        } else {
                            v[k] = Real(0);
                        }
                    }
                    *TL::group(tl, g0 / TL::kG, lane) = TL::V::make(v);
                };
                if (keep) {
#pragma unroll
                    for (int g0 = 0; g0 < TL::Rp; g0 += TL::kG)
                        if (g0 >= TL::RZ) store_group(g0);  // checkpoint (and padding) only
                }
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    const int n = s * K + i;
#pragma unroll
                    for (int q = 0; q < PPT; ++q) rng[q].get(n, s == 0 && i == 0, zs[i][q], rk);
                    if (keep) {
#pragma unroll
                        for (int g0 = 0; g0 < TL::RZ; g0 += TL::kG)  // groups whose last normals row is step i's
                            if ((min(g0 + TL::kG, TL::RZ) - 1) / (Md::DZ * PPT) == i) store_group(g0);
                    }
                }
#pragma unroll
                for (int i = 0; i < K; ++i) {
#pragma unroll
                    for (int q = 0; q < PPT; ++q) Md::step(st[q], zs[i][q], s * K + i, par, sh, nullptr);
                }
                if (g < pb.n_groups && gseg[g] == s) {
                    Real S[PPT];
#pragma unroll
                    for (int q = 0; q < PPT; ++q) S[q] = S0 * exp_r<Real>(st[q].x);
                    for (int i0 = gbeg[g]; i0 < gbeg[g + 1]; i0 += kWarp) {
                        const int cnt = min(kWarp, gbeg[g + 1] - i0);
                        Real mine = Real(0);
                        for (int j = 0; j < cnt; ++j) {
                            Real pay = Real(0);
#pragma unroll
                            for (int q = 0; q < PPT; ++q)
                                pay += active[q] ? fmax(S[q] - strike[i0 + j], Real(0)) : Real(0);
                            const Real sum = warp_sum(pay);
                            mine = (lane == j) ? sum : mine;
                        }
                        if (lane < cnt) {
                            if (dyn) cl.part_y[ch * pb.m + i0 + lane] = (double)mine;
                            else wy[i0 + lane] += (double)mine;
                        }
                    }
                    ++g;
                }
            }
        }
    }
    if (dyn) {
        queue_done(cl.queue);
        return;
    }
    __syncthreads();
    const double *wall = (const double *)(smem + sp.wacc_y);
    for (int i = threadIdx.x; i < pb.m; i += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kWarpsPerBlock; ++w) s += wall[w * pb.m + i];
        cl.part_y[(size_t)blockIdx.x * pb.m + i] = s;
    }
}

// The reverse sweep's body; the kernels below differ only in the occupancy they are compiled for.
template <class Md, int K, int PPT, bool kLoadZ>
__device__ __forceinline__ void reverse_sweep(const DevProblem &pb, const DevCall &cl) {
    using Real = typename Md::Real;
    using ZS = SegTile<Md, K, PPT, kLoadZ>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n_steps = pb.n_seg * K;
    const SmemPlan sp(Md::kind, sizeof(Real), pb.m, pb.n_groups, pb.M, n_steps, pb.nx, true, ZS::kBlockBytes);
    load_tables<Md>(smem, sp, pb, true, cl);
    typename Md::Shared sh;
    typename Md::Par par;
    Md::setup(smem, sp, pb, cl.theta, n_steps, sh, par);
    __syncthreads();

    const Real *strike = (const Real *)(smem + sp.strike);
    const Real *sw = (const Real *)(smem + sp.seed_w);
    const int *gseg = (const int *)(smem + sp.grp_seg);
    const int *gbeg = (const int *)(smem + sp.grp_begin);
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    double *wg = (double *)(smem + sp.wacc_g) + warp * pb.M;
    const Real S0 = (Real)pb.S0;
    RoundKeys rk;
    if constexpr (!kLoadZ) rk = Md::kKeysInRegisters ? philox_round_keys(cl.seed) : cl.rk;
    Real *zstage = (Real *)(smem + sp.zstage) + (size_t)warp * 2 * ZS::kElems;

    constexpr uint64_t kChunk = (uint64_t)kWarp * PPT;
    const uint64_t n_chunks = (cl.n_paths + kChunk - 1) / kChunk;
    const bool dyn = cl.queue != nullptr;  // chunks from the queue, one partial row per chunk
    for (uint64_t ch = dyn ? take_chunk(cl.queue, lane) : (uint64_t)blockIdx.x * kWarpsPerBlock + warp; ch < n_chunks;
         ch = dyn ? take_chunk(cl.queue, lane) : ch + (uint64_t)gridDim.x * kWarpsPerBlock) {
        uint64_t local[PPT];
        bool active[PPT];
        NormalSource<Md> rng[PPT];
        Real xb[PPT], vb[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            local[q] = ch * kChunk + q * kWarp + lane;
            active[q] = local[q] < cl.n_paths;
            if constexpr (!kLoadZ) rng[q].init(pb, cl, cl.path0 + (active[q] ? local[q] : 0));
            xb[q] = Real(0);
            vb[q] = Real(0);
        }
        ZS::issue(zstage, cl.ckpt, ch, cl.ckpt_stride / kChunk, pb.n_seg - 1, lane);
        typename Md::Acc acc;
        Md::acc_begin(acc, n_steps, sh);
        int g = pb.n_groups - 1;
        for (int s = pb.n_seg - 1; s >= 0; --s) {
            if (s > 0) {
                ZS::issue(zstage, cl.ckpt, ch, cl.ckpt_stride / kChunk, s - 1, lane);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();  // the other lanes' copies of segment s are visible
            const Real *sbuf = zstage + (size_t)(s & 1) * ZS::kElems;
            typename Md::State st[PPT];
            typename Md::Tape tape[PPT][K];
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                st[q].x = ZS::row(sbuf, ZS::crow(0, q), lane);
                if constexpr (Md::SD == 2) st[q].v = ZS::row(sbuf, ZS::crow(1, q), lane);
            }
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int n = s * K + i;
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    Real z[Md::DZ];
                    if constexpr (kLoadZ) {
#pragma unroll
                        for (int c = 0; c < Md::DZ; ++c) z[c] = ZS::row(sbuf, ZS::zrow(i, c, q), lane);
                    } else {
                        rng[q].get(n, i == 0, z, rk);
                    }
                    Md::step(st[q], z, n, par, sh, &tape[q][i]);
                }
            }
            if (g >= 0 && gseg[g] == s) {
                Real S[PPT], seed[PPT];
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    S[q] = S0 * exp_r<Real>(st[q].x);
                    seed[q] = Real(0);
                }
                for (int i = gbeg[g]; i < gbeg[g + 1]; ++i) {  // each strike and weight read once
                    const Real k = strike[i], wgt = sw[i];
#pragma unroll
                    for (int q = 0; q < PPT; ++q) seed[q] = S[q] > k ? fma(wgt, S[q], seed[q]) : seed[q];
                }
#pragma unroll
                for (int q = 0; q < PPT; ++q)
                    if (active[q]) xb[q] += seed[q];
                --g;
            }
#pragma unroll
            for (int i = K - 1; i >= 0; --i) {
                const int n = s * K + i;
                Md::boundary(acc, n, sh, wg, lane);
#pragma unroll
                for (int q = 0; q < PPT; ++q) Md::adjoint(tape[q][i], n, xb[q], vb[q], acc, par, sh);
            }
        }
        Real vb_sum = Real(0);
#pragma unroll
        for (int q = 0; q < PPT; ++q) vb_sum += vb[q];
        Md::acc_end(acc, vb_sum, par, sh, wg, lane);
        if (dyn) {  // this chunk's sums to its own row; the warp's accumulators back to zero
            __syncwarp();
            for (int j = lane; j < pb.M; j += kWarp) {
                cl.part_g[ch * pb.M + j] = wg[j];
                wg[j] = 0.0;
            }
            __syncwarp();
        }
    }
    if (dyn) {
        queue_done(cl.queue);
        return;
    }
    __syncthreads();
    const double *wall = (const double *)(smem + sp.wacc_g);
    for (int j = threadIdx.x; j < pb.M; j += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kWarpsPerBlock; ++w) s += wall[w * pb.M + j];
        cl.part_g[(size_t)blockIdx.x * pb.M + j] = s;
    }
}

template <class Md, int K, int PPT, bool kLoadZ = false>
__global__ void __launch_bounds__(kBlock) path_reverse_kernel(const DevProblem pb, const DevCall cl) {
    reverse_sweep<Md, K, PPT, kLoadZ>(pb, cl);
}

// Long local-vol segments (K = 25, one path per thread: 25 steps unrolled with their tapes) take
// up to 253 registers and two blocks per SM when unbounded; compiled for three blocks (at most 168
// registers) they measured faster. Other models keep the unbounded kernel: a minimum of one block
// per SM still changes ptxas's allocation (stochastic local vol: 164 -> 188 registers, three ->
// two blocks per SM, 1.80 -> 2.21 ms).
template <class Md, int K, int PPT, bool kLoadZ = false>
__global__ void __launch_bounds__(kBlock, 3) path_reverse_kernel_b3(const DevProblem pb, const DevCall cl) {
    reverse_sweep<Md, K, PPT, kLoadZ>(pb, cl);
}

template <class Md, int K>
__host__ __device__ constexpr bool reverse_three_blocks() { return Md::kind == kLv && K >= 25; }

// ------------------------------------------------------ stored-states variant --
// The forward sweep stores the state before every step (SegTile mode 2: no normals, no
// checkpoints; the state after the last step in one extra tile), and the reverse sweep runs the
// adjoint alone: the model's adjoint_states takes a step's quantities from the states at both
// of its ends instead of re-running it (local vol: the step's increment gives sqrt(dt) z).

template <class Md, int K, int PPT>
__global__ void __launch_bounds__(kBlock) path_forward_states_kernel(const DevProblem pb, const DevCall cl) {
    using Real = typename Md::Real;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n_steps = pb.n_seg * K;
    const SmemPlan sp(Md::kind, sizeof(Real), pb.m, pb.n_groups, pb.M, n_steps, pb.nx, false);
    load_tables<Md>(smem, sp, pb, false, cl);
    typename Md::Shared sh;
    typename Md::Par par;
    Md::setup(smem, sp, pb, cl.theta, n_steps, sh, par);
    __syncthreads();

    const Real *strike = (const Real *)(smem + sp.strike);
    const int *gseg = (const int *)(smem + sp.grp_seg);
    const int *gbeg = (const int *)(smem + sp.grp_begin);
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    double *wy = (double *)(smem + sp.wacc_y) + warp * pb.m;
    const Real S0 = (Real)pb.S0;
    using TL = SegTile<Md, K, PPT, 2>;
    constexpr int kRowsPerStep = Md::SD * PPT;
    const RoundKeys rk = Md::kKeysInRegisters ? philox_round_keys(cl.seed) : cl.rk;

    constexpr uint64_t kChunk = (uint64_t)kWarp * PPT;
    const uint64_t n_chunks = (cl.n_paths + kChunk - 1) / kChunk;
    const uint64_t ws_chunks = cl.ckpt_stride / kChunk;
    const bool dyn = cl.queue != nullptr;  // chunks from the queue, one partial row per chunk
    for (uint64_t ch = dyn ? take_chunk(cl.queue, lane) : (uint64_t)blockIdx.x * kWarpsPerBlock + warp; ch < n_chunks;
         ch = dyn ? take_chunk(cl.queue, lane) : ch + (uint64_t)gridDim.x * kWarpsPerBlock) {
        uint64_t local[PPT];
        bool active[PPT];
        NormalSource<Md> rng[PPT];
        typename Md::State st[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            local[q] = ch * kChunk + q * kWarp + lane;
            active[q] = local[q] < cl.n_paths;
            rng[q].init(pb, cl, cl.path0 + (active[q] ? local[q] : 0));
            st[q] = Md::init(par);
        }
        int g = 0;
        constexpr int kPeriod = philox_period_segments(K * Md::DZ);
        for (int sg = 0; sg * kPeriod < pb.n_seg; ++sg) {
#pragma unroll
            for (int ss = 0; ss < kPeriod; ++ss) {
                const int s = sg * kPeriod + ss;
                if (kPeriod > 1 && s >= pb.n_seg) break;
                Real zs[K][PPT][Md::DZ];
                Real xs[K][PPT][Md::SD];  // the state before each step
                Real *tl = TL::tile(cl.ckpt, ch, ws_chunks, s);
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    const int n = s * K + i;
#pragma unroll
                    for (int q = 0; q < PPT; ++q) rng[q].get(n, s == 0 && i == 0, zs[i][q], rk);
                }
#pragma unroll
                for (int i = 0; i < K; ++i) {
#pragma unroll
                    for (int q = 0; q < PPT; ++q) {
                        xs[i][q][0] = st[q].x;
                        if constexpr (Md::SD == 2) xs[i][q][1] = st[q].v;
                    }
                    // groups whose last row is a state of step i go out now
#pragma unroll
                    for (int g0 = 0; g0 < TL::Rp; g0 += TL::kG) {
                        if ((min(g0 + TL::kG, TL::R) - 1) / kRowsPerStep != i) continue;
                        Real v[TL::kG];
#pragma unroll
                        for (int k = 0; k < TL::kG; ++k) {
                            const int r = g0 + k;
                            v[k] = r < TL::R ? xs[r / kRowsPerStep][r % PPT][(r / PPT) % Md::SD] : Real(0);
                        }
                        *TL::group(tl, g0 / TL::kG, lane) = TL::V::make(v);
                    }
#pragma unroll
                    for (int q = 0; q < PPT; ++q) Md::step(st[q], zs[i][q], s * K + i, par, sh, nullptr);
                }
                if (g < pb.n_groups && gseg[g] == s) {
                    Real S[PPT];
#pragma unroll
                    for (int q = 0; q < PPT; ++q) S[q] = S0 * exp_r<Real>(st[q].x);
                    for (int i0 = gbeg[g]; i0 < gbeg[g + 1]; i0 += kWarp) {
                        const int cnt = min(kWarp, gbeg[g + 1] - i0);
                        Real mine = Real(0);
                        for (int j = 0; j < cnt; ++j) {
                            Real pay = Real(0);
#pragma unroll
                            for (int q = 0; q < PPT; ++q)
                                pay += active[q] ? fmax(S[q] - strike[i0 + j], Real(0)) : Real(0);
                            const Real sum = warp_sum(pay);
                            mine = (lane == j) ? sum : mine;
                        }
                        if (lane < cnt) {
                            if (dyn) cl.part_y[ch * pb.m + i0 + lane] = (double)mine;
                            else wy[i0 + lane] += (double)mine;
                        }
                    }
                    ++g;
                }
            }
        }
        // the state after the last step: rows w*PPT + q of the extra tile
        Real *tf = TL::tile(cl.ckpt, ch, ws_chunks, pb.n_seg);
#pragma unroll
        for (int g0 = 0; g0 < kRowsPerStep; g0 += TL::kG) {
            Real v[TL::kG];
#pragma unroll
            for (int k = 0; k < TL::kG; ++k) {
                const int r = g0 + k;
                if (r < kRowsPerStep) {
                    const int w = r / PPT, q = r % PPT;
                    if constexpr (Md::SD == 2) v[k] = w == 0 ? st[q].x : st[q].v;
                    else v[k] = st[q].x;
                } else {
                    v[k] = Real(0);
                }
            }
            *TL::group(tf, g0 / TL::kG, lane) = TL::V::make(v);
        }
    }
    if (dyn) {
        queue_done(cl.queue);
        return;
    }
    __syncthreads();
    const double *wall = (const double *)(smem + sp.wacc_y);
    for (int i = threadIdx.x; i < pb.m; i += blockDim.x) {
        double sum = 0.0;
        for (int w = 0; w < kWarpsPerBlock; ++w) sum += wall[w * pb.m + i];
        cl.part_y[(size_t)blockIdx.x * pb.m + i] = sum;
    }
}

// Reverse sweep over stored states: per warp chunk, the extra tile gives the final states, then
// the segments from last to first, each staged (cp.async, two buffers, the next one in flight)
// while the previous runs: payoff seeds at the segment's end state, then the adjoints of its
// steps backwards from (state before, state after).
template <class Md, int K, int PPT>
// Compiled for five resident blocks per SM (96 registers, no spills); unbounded, the node caches
// take it to 121 registers and four blocks, measured slower (3.62 against 3.48 ms).
__global__ void __launch_bounds__(kBlock, 5) path_reverse_states_kernel(const DevProblem pb, const DevCall cl) {
    using Real = typename Md::Real;
    using ZS = SegTile<Md, K, PPT, 2>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n_steps = pb.n_seg * K;
    const SmemPlan sp(Md::kind, sizeof(Real), pb.m, pb.n_groups, pb.M, n_steps, pb.nx, true, ZS::kBlockBytes, true);
    load_tables<Md>(smem, sp, pb, true, cl);
    typename Md::Shared sh;
    typename Md::Par par;
    Md::setup(smem, sp, pb, cl.theta, n_steps, sh, par, true);
    __syncthreads();

    const Real *strike = (const Real *)(smem + sp.strike);
    const Real *sw = (const Real *)(smem + sp.seed_w);
    const int *gseg = (const int *)(smem + sp.grp_seg);
    const int *gbeg = (const int *)(smem + sp.grp_begin);
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    double *wg = (double *)(smem + sp.wacc_g) + warp * pb.M;
    const Real S0 = (Real)pb.S0;
    Real *zstage = (Real *)(smem + sp.zstage) + (size_t)warp * 2 * ZS::kElems;

    constexpr uint64_t kChunk = (uint64_t)kWarp * PPT;
    const uint64_t n_chunks = (cl.n_paths + kChunk - 1) / kChunk;
    const uint64_t ws_chunks = cl.ckpt_stride / kChunk;
    const bool dyn = cl.queue != nullptr;  // chunks from the queue, one partial row per chunk
    for (uint64_t ch = dyn ? take_chunk(cl.queue, lane) : (uint64_t)blockIdx.x * kWarpsPerBlock + warp; ch < n_chunks;
         ch = dyn ? take_chunk(cl.queue, lane) : ch + (uint64_t)gridDim.x * kWarpsPerBlock) {
        bool active[PPT];
        Real xb[PPT], vb[PPT];
        typename Md::State nx_[PPT];  // the state after the segment being processed
        typename Md::NodeCache ncache[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            active[q] = ch * kChunk + q * kWarp + lane < cl.n_paths;
            xb[q] = Real(0);
            vb[q] = Real(0);
            ncache[q].key = -1;
        }
        // the final states (extra tile, buffer n_seg & 1), and the last segment behind it
        ZS::issue(zstage, cl.ckpt, ch, ws_chunks, pb.n_seg, lane);
        ZS::issue(zstage, cl.ckpt, ch, ws_chunks, pb.n_seg - 1, lane);
        cp_async_wait<1>();
        __syncwarp();
        {
            const Real *fbuf = zstage + (size_t)(pb.n_seg & 1) * ZS::kElems;
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                nx_[q].x = ZS::row(fbuf, ZS::srow(0, 0, q), lane);
                if constexpr (Md::SD == 2) nx_[q].v = ZS::row(fbuf, ZS::srow(0, 1, q), lane);
            }
        }
        typename Md::Acc acc;
        Md::acc_begin(acc, n_steps, sh);
        int g = pb.n_groups - 1;
        for (int s = pb.n_seg - 1; s >= 0; --s) {
            if (s > 0) {
                ZS::issue(zstage, cl.ckpt, ch, ws_chunks, s - 1, lane);  // into the buffer of s + 1
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();  // the other lanes' copies of segment s are visible
            const Real *sbuf = zstage + (size_t)(s & 1) * ZS::kElems;
            // the lane's rows of the segment, one 16-byte load per group (conflict-free)
            typename ZS::V::T grp[ZS::Rp / ZS::kG];
#pragma unroll
            for (int k = 0; k < ZS::Rp / ZS::kG; ++k) grp[k] = *ZS::group(sbuf, k, lane);
            if (g >= 0 && gseg[g] == s) {
                Real S[PPT], seed[PPT];
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    S[q] = S0 * exp_r<Real>(nx_[q].x);
                    seed[q] = Real(0);
                }
                for (int i = gbeg[g]; i < gbeg[g + 1]; ++i) {  // each strike and weight read once
                    const Real k = strike[i], wgt = sw[i];
#pragma unroll
                    for (int q = 0; q < PPT; ++q) seed[q] = S[q] > k ? fma(wgt, S[q], seed[q]) : seed[q];
                }
#pragma unroll
                for (int q = 0; q < PPT; ++q)
                    if (active[q]) xb[q] += seed[q];
                --g;
            }
#pragma unroll
            for (int i = K - 1; i >= 0; --i) {
                const int n = s * K + i;
                Md::boundary(acc, n, sh, wg, lane);
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    typename Md::State cur;
                    constexpr int kG = ZS::kG;
                    cur.x = ZS::V::get(grp[ZS::srow(i, 0, q) / kG], ZS::srow(i, 0, q) % kG);
                    if constexpr (Md::SD == 2) cur.v = ZS::V::get(grp[ZS::srow(i, 1, q) / kG], ZS::srow(i, 1, q) % kG);
                    Md::adjoint_states_cached(cur, nx_[q], xb[q], acc, par, sh, ncache[q]);
                    nx_[q] = cur;
                }
            }
        }
        Real vb_sum = Real(0);
#pragma unroll
        for (int q = 0; q < PPT; ++q) vb_sum += vb[q];
        Md::acc_end(acc, vb_sum, par, sh, wg, lane);
        if (dyn) {  // this chunk's sums to its own row; the warp's accumulators back to zero
            __syncwarp();
            for (int j = lane; j < pb.M; j += kWarp) {
                cl.part_g[ch * pb.M + j] = wg[j];
                wg[j] = 0.0;
            }
            __syncwarp();
        }
    }
    if (dyn) {
        queue_done(cl.queue);
        return;
    }
    __syncthreads();
    const double *wall = (const double *)(smem + sp.wacc_g);
    for (int j = threadIdx.x; j < pb.M; j += blockDim.x) {
        double sum = 0.0;
        for (int w = 0; w < kWarpsPerBlock; ++w) sum += wall[w * pb.M + j];
        cl.part_g[(size_t)blockIdx.x * pb.M + j] = sum;
    }
}

// ------------------------------------------- recompute into shared memory --
// Checkpoint-and-recompute (the two-step algorithm's step 2 with only every K-th state kept) for
// local vol: per segment, last first, the reverse sweep re-runs the segment's K steps from its
// checkpoint, regenerating the normals, and keeps the states x_0..x_K of its PPT paths per
// thread in shared memory (per warp [K+1][PPT][32]) instead of a register tape; then it runs
// adjoint_states backwards over consecutive states, as the stored-states sweep does with states
// from HBM.  The registers no longer grow with K, so long segments keep several paths per thread.
template <class Md, int K, int PPT>
struct StateBuf {
    static constexpr size_t kElems = (size_t)(K + 1) * PPT * kWarp;  // per warp
    static constexpr size_t kBlockBytes = kElems * kWarpsPerBlock * sizeof(typename Md::Real);
    __device__ static constexpr int at(int i, int q, int lane) { return (i * PPT + q) * kWarp + lane; }
};

template <class Md, int K, int PPT>
__global__ void __launch_bounds__(kBlock) path_reverse_recompute_kernel(const DevProblem pb, const DevCall cl) {
    using Real = typename Md::Real;
    using SB = StateBuf<Md, K, PPT>;
    using TL = SegTile<Md, K, PPT, 0>;
    static_assert(Md::SD == 1, "one state word per path");
    extern __shared__ __align__(16) unsigned char smem[];
    const int n_steps = pb.n_seg * K;
    const SmemPlan sp(Md::kind, sizeof(Real), pb.m, pb.n_groups, pb.M, n_steps, pb.nx, true, SB::kBlockBytes, true);
    load_tables<Md>(smem, sp, pb, true, cl);
    typename Md::Shared sh;
    typename Md::Par par;
    Md::setup(smem, sp, pb, cl.theta, n_steps, sh, par, true);
    __syncthreads();

    const Real *strike = (const Real *)(smem + sp.strike);
    const Real *sw = (const Real *)(smem + sp.seed_w);
    const int *gseg = (const int *)(smem + sp.grp_seg);
    const int *gbeg = (const int *)(smem + sp.grp_begin);
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    double *wg = (double *)(smem + sp.wacc_g) + warp * pb.M;
    const Real S0 = (Real)pb.S0;
    Real *xs = (Real *)(smem + sp.zstage) + (size_t)warp * SB::kElems;
    const RoundKeys rk = Md::kKeysInRegisters ? philox_round_keys(cl.seed) : cl.rk;

    constexpr uint64_t kChunk = (uint64_t)kWarp * PPT;
    const uint64_t n_chunks = (cl.n_paths + kChunk - 1) / kChunk;
    const uint64_t ws_chunks = cl.ckpt_stride / kChunk;
    const bool dyn = cl.queue != nullptr;  // chunks from the queue, one partial row per chunk
    for (uint64_t ch = dyn ? take_chunk(cl.queue, lane) : (uint64_t)blockIdx.x * kWarpsPerBlock + warp; ch < n_chunks;
         ch = dyn ? take_chunk(cl.queue, lane) : ch + (uint64_t)gridDim.x * kWarpsPerBlock) {
        bool active[PPT];
        Real xb[PPT], vb[PPT];
        NormalSource<Md> rng[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const uint64_t local = ch * kChunk + q * kWarp + lane;
            active[q] = local < cl.n_paths;
            rng[q].init(pb, cl, cl.path0 + (active[q] ? local : 0));
            xb[q] = Real(0);
            vb[q] = Real(0);
        }
        typename Md::Acc acc;
        Md::acc_begin(acc, n_steps, sh);
        int g = pb.n_groups - 1;
        // the lane's checkpoint rows of the last segment (loaded one segment ahead)
        typename TL::V::T grp[TL::Rp / TL::kG];
        {
            const Real *tl = TL::tile(cl.ckpt, ch, ws_chunks, pb.n_seg - 1);
#pragma unroll
            for (int k = 0; k < TL::Rp / TL::kG; ++k) grp[k] = *TL::group(tl, k, lane);
        }
        for (int s = pb.n_seg - 1; s >= 0; --s) {
            typename Md::State st[PPT];
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                const int r = TL::crow(0, q);
                st[q].x = TL::V::get(grp[r / TL::kG], r % TL::kG);
                xs[SB::at(0, q, lane)] = st[q].x;
            }
            if (s > 0) {  // the next segment's checkpoint, in flight during this one
                const Real *tl = TL::tile(cl.ckpt, ch, ws_chunks, s - 1);
#pragma unroll
                for (int k = 0; k < TL::Rp / TL::kG; ++k) grp[k] = *TL::group(tl, k, lane);
            }
            // re-run the segment, keeping every state
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int n = s * K + i;
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    Real z[Md::DZ];
                    rng[q].get(n, i == 0, z, rk);
                    Md::step_nodes(st[q], z[0], n, par, sh);
                    xs[SB::at(i + 1, q, lane)] = st[q].x;
                }
            }
            if (g >= 0 && gseg[g] == s) {  // payoff seeds at the segment's end
                Real S[PPT], seed[PPT];
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    S[q] = S0 * exp_r<Real>(st[q].x);
                    seed[q] = Real(0);
                }
                for (int i = gbeg[g]; i < gbeg[g + 1]; ++i) {
                    const Real k = strike[i], wgt = sw[i];
#pragma unroll
                    for (int q = 0; q < PPT; ++q) seed[q] = S[q] > k ? fma(wgt, S[q], seed[q]) : seed[q];
                }
#pragma unroll
                for (int q = 0; q < PPT; ++q)
                    if (active[q]) xb[q] += seed[q];
                --g;
            }
            // the adjoint backwards over the kept states
#pragma unroll
            for (int i = K - 1; i >= 0; --i) {
                const int n = s * K + i;
                Md::boundary(acc, n, sh, wg, lane);
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    typename Md::State x0, x1;
                    x0.x = xs[SB::at(i, q, lane)];
                    x1.x = xs[SB::at(i + 1, q, lane)];
                    Md::adjoint_states(x0, x1, n, xb[q], vb[q], acc, par, sh);
                }
            }
        }
        Real vb_sum = Real(0);
#pragma unroll
        for (int q = 0; q < PPT; ++q) vb_sum += vb[q];
        Md::acc_end(acc, vb_sum, par, sh, wg, lane);
        if (dyn) {  // this chunk's sums to its own row; the warp's accumulators back to zero
            __syncwarp();
            for (int j = lane; j < pb.M; j += kWarp) {
                cl.part_g[ch * pb.M + j] = wg[j];
                wg[j] = 0.0;
            }
            __syncwarp();
        }
    }
    if (dyn) {
        queue_done(cl.queue);
        return;
    }
    __syncthreads();
    const double *wall = (const double *)(smem + sp.wacc_g);
    for (int j = threadIdx.x; j < pb.M; j += blockDim.x) {
        double sum = 0.0;
        for (int w = 0; w < kWarpsPerBlock; ++w) sum += wall[w * pb.M + j];
        cl.part_g[(size_t)blockIdx.x * pb.M + j] = sum;
    }
}

// ---------------------------------------------------- full-storage variant --
// The paper's branch for unconstrained memory (two-step algorithm, step 2:
// with the first step's intermediate values kept, the reverse sweep costs
// K_R Cost(F) alone): the forward sweep writes every step's tape (the model's
// Tape fields, SoA [step][field][path], coalesced) and x at each maturity; the
// reverse sweep streams them back and runs only the adjoint.

template <class Md, int K, int PPT>
__global__ void __launch_bounds__(kBlock) path_forward_store_kernel(const DevProblem pb, const DevCall cl) {
    using Real = typename Md::Real;
    using Tape = typename Md::Tape;
    constexpr int NF = sizeof(Tape) / sizeof(Real);
    extern __shared__ __align__(16) unsigned char smem[];
    const int n_steps = pb.n_seg * K;
    const SmemPlan sp(Md::kind, sizeof(Real), pb.m, pb.n_groups, pb.M, n_steps, pb.nx, false);
    load_tables<Md>(smem, sp, pb, false, cl);
    typename Md::Shared sh;
    typename Md::Par par;
    Md::setup(smem, sp, pb, cl.theta, n_steps, sh, par);
    __syncthreads();

    const Real *strike = (const Real *)(smem + sp.strike);
    const int *gseg = (const int *)(smem + sp.grp_seg);
    const int *gbeg = (const int *)(smem + sp.grp_begin);
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    double *wy = (double *)(smem + sp.wacc_y) + warp * pb.m;
    const Real S0 = (Real)pb.S0;
    Real *tp = (Real *)cl.tape;
    Real *xm = (Real *)cl.xmat;
    const uint64_t stride = cl.ckpt_stride;
    const RoundKeys rk = Md::kKeysInRegisters ? philox_round_keys(cl.seed) : cl.rk;

    constexpr uint64_t kChunk = (uint64_t)kWarp * PPT;
    const uint64_t n_chunks = (cl.n_paths + kChunk - 1) / kChunk;
    for (uint64_t ch = (uint64_t)blockIdx.x * kWarpsPerBlock + warp; ch < n_chunks;
         ch += (uint64_t)gridDim.x * kWarpsPerBlock) {
        uint64_t local[PPT];
        bool active[PPT];
        NormalSource<Md> rng[PPT];
        typename Md::State st[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            local[q] = ch * kChunk + q * kWarp + lane;
            active[q] = local[q] < cl.n_paths;
            rng[q].init(pb, cl, cl.path0 + (active[q] ? local[q] : 0));
            st[q] = Md::init(par);
        }
        int g = 0;
        for (int s = 0; s < pb.n_seg; ++s) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int n = s * K + i;
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    Real z[Md::DZ];
                    rng[q].get(n, s == 0 && i == 0, z, rk);
                    Tape t;
                    Md::step(st[q], z, n, par, sh, &t);
                    const Real *tf = (const Real *)&t;
#pragma unroll
                    for (int f = 0; f < NF; ++f) tp[((size_t)n * NF + f) * stride + local[q]] = tf[f];
                }
            }
            if (g < pb.n_groups && gseg[g] == s) {
                Real S[PPT];
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    xm[(size_t)g * stride + local[q]] = st[q].x;
                    S[q] = S0 * exp_r<Real>(st[q].x);
                }
                for (int i0 = gbeg[g]; i0 < gbeg[g + 1]; i0 += kWarp) {
                    const int cnt = min(kWarp, gbeg[g + 1] - i0);
                    Real mine = Real(0);
                    for (int j = 0; j < cnt; ++j) {
                        Real pay = Real(0);
#pragma unroll
                        for (int q = 0; q < PPT; ++q)
                            pay += active[q] ? fmax(S[q] - strike[i0 + j], Real(0)) : Real(0);
                        const Real sum = warp_sum(pay);
                        mine = (lane == j) ? sum : mine;
                    }
                    if (lane < cnt) wy[i0 + lane] += (double)mine;
                }
                ++g;
            }
        }
    }
    __syncthreads();
    const double *wall = (const double *)(smem + sp.wacc_y);
    for (int i = threadIdx.x; i < pb.m; i += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kWarpsPerBlock; ++w) s += wall[w * pb.m + i];
        cl.part_y[(size_t)blockIdx.x * pb.m + i] = s;
    }
}

template <class Md, int K, int PPT>
__global__ void __launch_bounds__(kBlock) path_reverse_tape_kernel(const DevProblem pb, const DevCall cl) {
    using Real = typename Md::Real;
    using Tape = typename Md::Tape;
    constexpr int NF = sizeof(Tape) / sizeof(Real);
    extern __shared__ __align__(16) unsigned char smem[];
    const int n_steps = pb.n_seg * K;
    const SmemPlan sp(Md::kind, sizeof(Real), pb.m, pb.n_groups, pb.M, n_steps, pb.nx, true);
    load_tables<Md>(smem, sp, pb, true, cl);
    typename Md::Shared sh;
    typename Md::Par par;
    Md::setup(smem, sp, pb, cl.theta, n_steps, sh, par);
    __syncthreads();

    const Real *strike = (const Real *)(smem + sp.strike);
    const Real *sw = (const Real *)(smem + sp.seed_w);
    const int *gseg = (const int *)(smem + sp.grp_seg);
    const int *gbeg = (const int *)(smem + sp.grp_begin);
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    double *wg = (double *)(smem + sp.wacc_g) + warp * pb.M;
    const Real S0 = (Real)pb.S0;
    const Real *tp = (const Real *)cl.tape;
    const Real *xm = (const Real *)cl.xmat;
    const uint64_t stride = cl.ckpt_stride;

    constexpr uint64_t kChunk = (uint64_t)kWarp * PPT;
    const uint64_t n_chunks = (cl.n_paths + kChunk - 1) / kChunk;
    for (uint64_t ch = (uint64_t)blockIdx.x * kWarpsPerBlock + warp; ch < n_chunks;
         ch += (uint64_t)gridDim.x * kWarpsPerBlock) {
        uint64_t local[PPT];
        bool active[PPT];
        Real xb[PPT], vb[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            local[q] = ch * kChunk + q * kWarp + lane;
            active[q] = local[q] < cl.n_paths;
            xb[q] = Real(0);
            vb[q] = Real(0);
        }
        typename Md::Acc acc;
        Md::acc_begin(acc, n_steps, sh);
        int g = pb.n_groups - 1;
        for (int s = pb.n_seg - 1; s >= 0; --s) {
            if (g >= 0 && gseg[g] == s) {
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    const Real S = S0 * exp_r<Real>(xm[(size_t)g * stride + local[q]]);
                    Real seed = Real(0);
                    for (int i = gbeg[g]; i < gbeg[g + 1]; ++i)
                        if (S > strike[i]) seed = fma(sw[i], S, seed);
                    if (active[q]) xb[q] += seed;
                }
                --g;
            }
#pragma unroll
            for (int i = K - 1; i >= 0; --i) {
                const int n = s * K + i;
                Md::boundary(acc, n, sh, wg, lane);
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    Tape t;
                    Real *tf = (Real *)&t;
#pragma unroll
                    for (int f = 0; f < NF; ++f) tf[f] = tp[((size_t)n * NF + f) * stride + local[q]];
                    Md::adjoint(t, n, xb[q], vb[q], acc, par, sh);
                }
            }
        }
        Real vb_sum = Real(0);
#pragma unroll
        for (int q = 0; q < PPT; ++q) vb_sum += vb[q];
        Md::acc_end(acc, vb_sum, par, sh, wg, lane);
    }
    __syncthreads();
    const double *wall = (const double *)(smem + sp.wacc_g);
    for (int j = threadIdx.x; j < pb.M; j += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kWarpsPerBlock; ++w) s += wall[w * pb.M + j];
        cl.part_g[(size_t)blockIdx.x * pb.M + j] = s;
    }
}

// Every variant of (model, K, PPT) for the host's kernel table.
template <class Md, int K, int PPT, class Table>
void set_kernels(Table *out) {
    out->fwd = (const void *)path_forward_kernel<Md, K, PPT>;
    if constexpr (reverse_three_blocks<Md, K>()) {
        out->rev = (const void *)path_reverse_kernel_b3<Md, K, PPT>;
        out->rev_z = (const void *)path_reverse_kernel_b3<Md, K, PPT, true>;
    } else {
        out->rev = (const void *)path_reverse_kernel<Md, K, PPT>;
        out->rev_z = (const void *)path_reverse_kernel<Md, K, PPT, true>;
    }
    out->fwd_store = (const void *)path_forward_store_kernel<Md, K, PPT>;
    out->rev_tape = (const void *)path_reverse_tape_kernel<Md, K, PPT>;
    out->fwd_z = (const void *)path_forward_kernel<Md, K, PPT, true>;
    out->stage_bytes_ckpt = SegTile<Md, K, PPT, false>::kBlockBytes;
    out->stage_bytes_z = SegTile<Md, K, PPT, true>::kBlockBytes;
    if constexpr (Md::kind == kLv) {  // stored states: local vol only
        // checkpoint-and-recompute re-runs each segment into shared memory
        out->rev = (const void *)path_reverse_recompute_kernel<Md, K, PPT>;
        out->stage_bytes_ckpt = StateBuf<Md, K, PPT>::kBlockBytes;
        out->rev_node_table = true;
        out->fwd_x = (const void *)path_forward_states_kernel<Md, K, PPT>;
        out->rev_x = (const void *)path_reverse_states_kernel<Md, K, PPT>;
        out->stage_bytes_x = SegTile<Md, K, PPT, 2>::kBlockBytes;
    }
}

}  // namespace mcaad
