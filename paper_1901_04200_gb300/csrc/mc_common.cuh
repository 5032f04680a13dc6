// mc_common.cuh -- device building blocks shared by the path kernels:
// Philox-4x32-10 (Salmon et al., SC'11), the uniform map, Box-Muller, warp
// sums, and the parameter blocks handed to every kernel by value.
#pragma once
#ifdef __CUDACC_RTC__
// compiled at run time (the tape compiler embeds this header): no system headers
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
typedef unsigned long size_t;
#else
#include <cuda_runtime.h>
#include <stdint.h>
#endif

namespace mcaad {

constexpr int kWarp = 32;
constexpr int kBlock = 128;             // threads per path-kernel block
constexpr int kWarpsPerBlock = kBlock / kWarp;
constexpr int kMaxInstruments = 1024;   // m limit (shared-memory tables)
constexpr int kMaxParams = 256;         // M limit

// ------------------------------------------------------------------ RNG ----

// Ten rounds of the Philox 4x32 bijection: each round multiplies words 0 and
// 2 by the two Philox constants, keeps the low halves as the new words 1 and
// 3, and xors the high halves with the other two words and the round key;
// the key advances by the Weyl increments between rounds.
// The round keys depend only on the seed: they are formed once on the host
// and travel in the kernel parameters (constant bank), so each round costs
// two 32 x 32 -> 64-bit products and two three-input xors.  kWide: each
// product from one wide multiply, else from a low and a high 32-bit multiply
// (the same bits; which issues faster depends on the surrounding kernel).
struct RoundKeys {
    uint32_t k[20];  // (k0, k1) of rounds 0..9
};
__host__ __device__ inline RoundKeys philox_round_keys(uint64_t seed) {
    RoundKeys rk;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        rk.k[2 * round] = k0;
        rk.k[2 * round + 1] = k1;
    }
    return rk;
}
template <bool kWide = true>
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys &rk) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        uint32_t lo0, hi0, lo1, hi1;
        if constexpr (kWide) {
            uint64_t p0, p1;
            asm("mul.wide.u32 %0, %1, %2;" : "=l"(p0) : "r"(c.x), "r"(0xD2511F53u));
            asm("mul.wide.u32 %0, %1, %2;" : "=l"(p1) : "r"(c.z), "r"(0xCD9E8D57u));
            lo0 = (uint32_t)p0;
            hi0 = (uint32_t)(p0 >> 32);
            lo1 = (uint32_t)p1;
            hi1 = (uint32_t)(p1 >> 32);
        } else {
            lo0 = c.x * 0xD2511F53u;
            hi0 = __umulhi(c.x, 0xD2511F53u);
            lo1 = c.z * 0xCD9E8D57u;
            hi1 = __umulhi(c.z, 0xCD9E8D57u);
        }
        c = make_uint4(hi1 ^ c.y ^ rk.k[2 * round], lo1, hi0 ^ c.w ^ rk.k[2 * round + 1], lo0);
    }
    return c;
}

// u(w) = ((w >> 9) + 0.5) * 2^-23.  In FP32: the float 1 + (w>>9)*2^-23 built
// from its bit pattern, minus (1 - 2^-24); the difference is representable,
// so the single rounded subtraction is exact.
__device__ __forceinline__ float uniform_f32(uint32_t w) {
    return __fsub_rn(__uint_as_float(0x3f800000u | (w >> 9)), 0.99999994f);
}
__device__ __forceinline__ double uniform_f64(uint32_t w) {
    return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

// The hardware approximations in their flush-to-zero forms: every argument
// they get on the path is a normal number (or zero), where the two forms agree,
// and the flush-to-zero form needs no rescaling around the instruction.
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float log2_approx(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void sincos_approx(float x, float &s, float &c) {
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(x));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(x));
}

// Box-Muller on one pair of uniforms: rad = sqrt(-2 ln u_a),
// (za, zb) = rad (cos 2 pi u_b, sin 2 pi u_b).  The FP32 version evaluates the
// angle as 2 pi (u_b - 1/2) + pi, i.e. negates cos and sin of an argument in
// (-pi, pi), where the fast hardware sine/cosine are accurate; u_b - 1/2 is
// exact.  -2 ln u_a is clamped at 0 against the approximate log near u = 1.
// u_a >= 2^-24 is normal; the angle is 0 or at least 2 pi 2^-24 in magnitude.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float &za, float &zb) {
    const float ua = uniform_f32(a);
    const float ub = uniform_f32(b);
    const float rad = sqrt_approx(fmaxf(-1.38629436111989061f * log2_approx(ua), 0.0f));  // -2 ln u = (-2 ln 2) log2 u
    float s, c;
    sincos_approx(fmaf(6.28318530717958648f, ub, -3.14159265358979324f), s, c);  // 2 pi u_b - pi, one rounding
    za = -rad * c;
    zb = -rad * s;
}
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double &za, double &zb) {
    const double ua = uniform_f64(a);
    const double ub = uniform_f64(b);
    const double rad = sqrt(-2.0 * log(ua));
    double s, c;
    sincospi(2.0 * ub, &s, &c);
    za = rad * c;
    zb = rad * s;
}

// Normals of one path, one Philox block (4 normals) at a time.
template <typename Real>
struct PathNormals {
    uint32_t p_lo, p_hi;
    Real z0, z1, z2, z3;
    __device__ __forceinline__ void init(uint64_t path) {
        p_lo = (uint32_t)path;
        p_hi = (uint32_t)(path >> 32);
    }
    template <bool kWide = true>
    __device__ __forceinline__ void fill(uint32_t call, const RoundKeys &rk) {
        const uint4 o = philox4x32_10<kWide>(make_uint4(call, 0u, p_lo, p_hi), rk);
        box_muller(o.x, o.y, z0, z1);
        box_muller(o.z, o.w, z2, z3);
    }
    __device__ __forceinline__ Real pick(uint32_t q) const {
        return q == 0 ? z0 : (q == 1 ? z1 : (q == 2 ? z2 : z3));
    }
};

// ------------------------------------------------------------ reductions ----

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ----------------------------------------------------------- parameters ----

enum ModelKind { kGbm = 0, kHeston = 1, kLv = 2, kSlv = 3 };

// Problem tables fixed at context creation (device pointers into the
// context's workspace).  Instruments are kept sorted by maturity; maturity
// group g covers sorted instruments [grp_begin[g], grp_begin[g+1]) and pays at
// step (grp_seg[g] + 1) * K, the end of segment grp_seg[g].
struct DevProblem {
    int kind;
    int K;            // checkpoint interval = segment length
    int n_seg;        // segments up to the last maturity
    int m, M;
    int n_groups;
    double S0, r, dt;
    const double *strike;       // [m] sorted
    const double *disc;         // [m] sorted, exp(-r T_i)
    const int *perm;            // [m] sorted index -> caller index
    const int *grp_seg;         // [n_groups]
    const int *grp_begin;       // [n_groups + 1]
    const int *bucket_of_step;  // GBM [n_seg * K]
    const int *lv_jt;           // LV/SLV [n_seg * K] time cell of step n
    const double *lv_a;         // LV/SLV [n_seg * K] time weight of step n
    int nt, nx;
    double x_lo, hx;
    const double *normals;      // optional GBM table
    uint64_t normals_path0, normals_rows;
    int normals_stride;
};

// One evaluation.
struct DevCall {
    const double *theta;  // [M]
    uint64_t seed;
    RoundKeys rk;         // Philox round keys of seed
    uint64_t path0;       // first global path
    uint64_t n_paths;
    void *ckpt;           // per-(chunk, segment) tiles of checkpoints (+ normals): SegTile
    uint64_t ckpt_stride; // paths padded to a multiple of 64 (full-storage tape stride)
    int keep_ckpt;
    double *part_y;       // [gridDim.x][m] per-block payoff sums (sorted order)
    double *part_g;       // [gridDim.x][M] per-block gradient sums
    const double *seed_w; // [m] sorted: lambda_i * disc_i (reverse sweep seeds)
    void *tape;           // full storage: [n_steps][tape fields][ckpt_stride] of Real
    void *xmat;           // full storage: [n_groups][ckpt_stride] x at each maturity
    // Work queue of the path sweeps (null: static chunk assignment, per-block partial sums): [0]
    // the next warp chunk, [1] finished blocks; with it, part_y / part_g hold one row per chunk
    // and the last block to finish resets both words to zero.
    unsigned long long *queue;
};

}  // namespace mcaad
