// mlp.cu -- the pricing surrogate on the tensor cores: MLP 7 -> 256 x 4 -> 1
// with SiLU, BF16 operands, FP32 accumulation (tcgen05 GEMM of tc_gemm.cuh),
// trained with the differential loss
//     L = mean (out - y)^2 + alpha * mean sum_{j<5} (d out/d x_j - dy_j)^2
// whose labels come from the Monte Carlo method (E y and its pathwise
// Jacobian).  Every matrix product is one tensor-core GEMM whose epilogue
// applies the elementwise work of that stage (bias, SiLU and its first and
// second derivatives, the products of the double-backward chain) and stores
// the operands of the following products, row-major and transposed:
//
//   F1..F4   z_l = h_{l-1} W_l^T + b_l, h_l = silu(z_l); F4 also forms
//            out = h_4 . w5 + b5, out_bar = 2 (out - y)/B and p_4 = w5 silu'(z_4)
//   T4..T1   g_{l-1} = p_l W_l, p_{l-1} = g_{l-1} silu'(z_{l-1}); T1 forms
//            g0_bar = 2 alpha (g_0 - dy)/B on the theta columns
//   R1..R4   p_bar_l = g_bar_{l-1} W_l^T, g_bar_l = p_bar_l silu'(z_l),
//            z_bar_l(tangent) = p_bar_l g_l silu''(z_l); R4 also forms
//            z_bar_4 = out_bar w5 silu'(z_4) + z_bar_4(tangent)
//   D4..D2   h_bar_{l-1} = z_bar_l W_l, z_bar_{l-1} = h_bar_{l-1} silu'(z_{l-1}) + tangent part
//   G1..G4   dW_l = [p_l ; z_bar_l]^T [g_bar_{l-1} ; h_{l-1}]  (K = 2B, split over CTAs)
//
// then fixed-order reductions (split-K slices, bias and w5 column sums, the
// loss) and Adam on FP32 master parameters, which also refreshes the BF16
// weight copies (W_l and W_l^T) the GEMMs read.  MCAAD_MLP_CHAIN=1 runs a
// training step's F, T, R and D as one chain_kernel launch instead (each CTA
// the whole sequence for its 128 rows), 2 as one chain_cluster_kernel launch
// (a cluster of eight CTAs per 128 rows); both measured slower.
#include <cuda_bf16.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "mcaad.h"
#include "tc_gemm.cuh"

namespace mcaad {
namespace mlp {

using bf16 = __nv_bfloat16;
constexpr int H = 256, DIN = 7, NTH = 5, KX = 64, NX = 16;
constexpr int kSplit = 16;  // K slices of the weight-gradient GEMMs (at most; see k_split)
// K slices for a batch of B rows (a multiple of 128): the weight-gradient GEMMs run over
// K = 2B = B/32 k-blocks of 64, and each slice must be whole k-blocks, so the split is the
// largest of 16, 8, 4 dividing B/32 (a multiple of 4).
constexpr int k_split(int B) { return (B / 32) % 16 == 0 ? 16 : ((B / 32) % 8 == 0 ? 8 : 4); }
// Columns per CTA of the weight-gradient GEMMs: 128 (64 CTAs per layer at batch 4096) keeps the
// tensor pipe busy 13.7 % of each SM's active cycles against 6.9 % with 32 (256 CTAs), for a step
// 1.4 % slower (0.187 against 0.1845 ms).
constexpr int kWgradBN = 128;
// Tuning knobs, read when a context is created: MCAAD_MLP_WGRAD_SPLIT (4, 8 or 16, used when it
// divides B/32) and MCAAD_MLP_WGRAD_BN (columns per CTA of the weight-gradient GEMMs: 16..256, a
// multiple of 16).
static int env_knob(const char *name) {
    const char *v = getenv(name);
    return v ? atoi(v) : 0;
}

// flat FP32 parameter layout
constexpr long long oW1 = 0, ob1 = oW1 + H * DIN, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H,
                    ob3 = oW3 + H * H, oW4 = ob3 + H, ob4 = oW4 + H * H, ow5 = ob4 + H, ob5 = ow5 + H,
                    kParams = ob5 + 1;
__host__ __device__ constexpr long long oW(int l) { return l == 1 ? oW1 : (l == 2 ? oW2 : (l == 3 ? oW3 : oW4)); }
__host__ __device__ constexpr long long ob(int l) { return l == 1 ? ob1 : (l == 2 ? ob2 : (l == 3 ? ob3 : ob4)); }

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + __expf(-z)); }
__device__ __forceinline__ float silu(float z) { return z * sigm(z); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = sigm(z);
    return s * (1.0f + z * (1.0f - s));
}
__device__ __forceinline__ float d2silu(float z) {
    const float s = sigm(z);
    return s * (1.0f - s) * (2.0f + z * (1.0f - 2.0f * s));
}

struct Bufs {
    int B;
    bf16 *x0;            // [B][KX]
    float *z[5];         // [B][H], l = 1..4
    bf16 *h[5];          // [B][H], l = 1..4
    float *out, *obar, *loss_rows;  // [B]
    float *outp;         // [H / 32][B] partial dot products of F4, per 32-column piece
    bf16 *p[5];          // [B][H], l = 1..4
    float *g[5];         // [B][H], l = 1..3 ; g[0]: [B][NX]
    bf16 *gb0;           // [B][KX]
    bf16 *gb[5];         // [B][H], l = 1..3
    float *gb4f;         // [B][H]
    float *zbt[5];       // [B][H]
    float *zb[5];        // [B][H]
    bf16 *zbb[5];        // [B][H], l = 2..4
    bf16 *Aop[5];        // [H][2B]
    bf16 *Bop[5];        // l = 1: [NX][2B], else [H][2B]
    float *part[5];      // l = 1..4: [split][H][N_l] split-K partials of dW_l
    int split;           // k_split(B), or MCAAD_MLP_WGRAD_SPLIT
    int wgrad_bn;        // columns per CTA of the 256-column layers G2..G4 (kWgradBN or the knob)
    float *colpart;      // [B / 128][41 * 32] column-sum chunks
    bf16 *Wb[5], *Wt[5];  // W1b [H][KX], W1t [NX][H], Wlb/Wlt [H][H]
    float *lsum;         // [1] loss scratch
    float *Xin, *yin, *dyin;  // [B][7], [B], [B][5]: the batch of mlp_train_step (fixed addresses)
    int *err;            // [1] tensor-core wait expiry flag
};

// ------------------------------------------------------------ epilogues ----

// transposed BF16 store: T[col][off + row] for the 32 (or n) columns of this row
__device__ __forceinline__ void store_t(bf16 *T, long long ldt, long long off, long long row, int c0, const float *v,
                                        int n) {
    for (int i = 0; i < n; ++i) T[(long long)(c0 + i) * ldt + off + row] = __float2bfloat16_rn(v[i]);
}
__device__ __forceinline__ void store_row_bf16(bf16 *D, long long ld, long long row, int c0, const float *v, int n) {
    for (int i = 0; i < n; i += 2) {
        __nv_bfloat162 t;
        t.x = __float2bfloat16_rn(v[i]);
        t.y = __float2bfloat16_rn(v[i + 1]);
        *(__nv_bfloat162 *)(D + row * ld + c0 + i) = t;
    }
}
__device__ __forceinline__ void store_row_f32(float *D, long long ld, long long row, int c0, const float *v, int n) {
    for (int i = 0; i < n; i += 4) *(float4 *)(D + row * ld + c0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
}

// Column-per-lane helpers (tc::gemm_body with kColumns): lane j holds column `col` of the warp's
// rows row0..row0+31, u[r] for row row0 + r.
__device__ __forceinline__ void col_load(const float *S, long long ld, int row0, int col, float (&w)[32]) {
#pragma unroll
    for (int r = 0; r < 32; ++r) w[r] = S[(long long)(row0 + r) * ld + col];
}
__device__ __forceinline__ void col_store_f32(float *D, long long ld, int row0, int col, const float (&u)[32]) {
#pragma unroll
    for (int r = 0; r < 32; ++r) D[(long long)(row0 + r) * ld + col] = u[r];
}
__device__ __forceinline__ void col_store_bf16(bf16 *D, long long ld, int row0, int col, const float (&u)[32]) {
#pragma unroll
    for (int r = 0; r < 32; ++r) D[(long long)(row0 + r) * ld + col] = __float2bfloat16_rn(u[r]);
}
// transposed: T[col][off + row0 + r]; the lane's 32 values are 64 contiguous bytes (16-byte
// aligned: ldt, off and row0 are multiples of 8), written as four 16-byte vectors
__device__ __forceinline__ void col_store_t(bf16 *T, long long ldt, long long off, int row0, int col,
                                            const float (&u)[32]) {
    uint4 *dst = (uint4 *)(T + (long long)col * ldt + off + row0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        __nv_bfloat162 p[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) p[k] = __floats2bfloat162_rn(u[8 * q + 2 * k], u[8 * q + 2 * k + 1]);
        dst[q] = *(const uint4 *)p;
    }
}

// F1..F3: z = acc + b; h = silu(z)
struct EpiFwd {
    static constexpr bool kColumns = true;
    const float *bias;
    float *z;
    bf16 *h;
    bf16 *hT;  // Bop_{l+1}: [H][2B], column B + row
    long long B2, Boff;
    __device__ void apply_cols(int row0, int col, const float (&u)[32], bool valid, int, int) const {
        if (!valid) return;
        const float b = bias[col];
        float zz[32], hh[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            zz[r] = u[r] + b;
            hh[r] = silu(zz[r]);
        }
        col_store_f32(z, H, row0, col, zz);
        col_store_bf16(h, H, row0, col, hh);
        col_store_t(hT, B2, Boff, row0, col, hh);
    }
};

// F4: as F1..F3, plus the partial dot product h . w5 over this 32-column piece
// (outp[piece][row], summed by finish_out_kernel) and p_4 = w5 silu'(z_4).
struct EpiFwdLast {
    static constexpr bool kColumns = true;
    const float *bias, *w5;
    float *z, *outp;
    bf16 *h, *p4, *p4T;  // p4T = Aop_4, column row
    long long B2, B;
    __device__ void apply_cols(int row0, int col, const float (&u)[32], bool valid, int, int lane) const {
        const float b = valid ? bias[col] : 0.0f, w = valid ? w5[col] : 0.0f;
        float zz[32], hh[32], pp[32], dot[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            zz[r] = u[r] + b;
            hh[r] = silu(zz[r]);
            pp[r] = w * dsilu(zz[r]);
            dot[r] = hh[r] * w;
        }
        const float row_dot = tc::warp_sum_scatter(dot, lane);  // lane r: row row0 + r
        outp[(long long)((col - lane) / 32) * B + row0 + lane] = row_dot;
        if (!valid) return;
        col_store_f32(z, H, row0, col, zz);
        col_store_bf16(h, H, row0, col, hh);
        col_store_bf16(p4, H, row0, col, pp);
        col_store_t(p4T, B2, 0, row0, col, pp);
    }
};

// T4..T2: g = acc; p = g silu'(z_{l-1})
struct EpiTan {
    static constexpr bool kColumns = true;
    const float *zprev;
    float *g;
    bf16 *p, *pT;  // pT = Aop_{l-1}, column row
    long long B2;
    __device__ void apply_cols(int row0, int col, const float (&u)[32], bool valid, int, int) const {
        if (!valid) return;
        float zp[32], pp[32];
        col_load(zprev, H, row0, col, zp);
#pragma unroll
        for (int r = 0; r < 32; ++r) pp[r] = u[r] * dsilu(zp[r]);
        col_store_f32(g, H, row0, col, u);
        col_store_bf16(p, H, row0, col, pp);
        col_store_t(pT, B2, 0, row0, col, pp);
    }
};

// T1: g_0 = acc (16 columns, 7 valid); g0_bar on the theta columns; derivative loss
struct EpiTanIn {
    static constexpr bool kColumns = false;
    float *g0;
    const float *dy;  // [B][NTH] or null (inference)
    bf16 *gb0, *gb0T;  // gb0 [B][KX]; gb0T = Bop_1 [NX][2B], column row
    float *loss_rows;
    long long B2;
    float two_alpha_inv_b, alpha_inv_b;
    __device__ void apply(long long row, int c0, const float (&acc)[32], int n, int, float &) const {
        float gbar[32];
        float l = 0.0f;
        for (int i = 0; i < 32; ++i) gbar[i] = 0.0f;
        for (int i = 0; i < NX; ++i) g0[row * NX + i] = acc[i];
        if (dy) {
            for (int j = 0; j < NTH; ++j) {
                const float d = acc[j] - dy[row * NTH + j];
                gbar[j] = two_alpha_inv_b * d;
                l = fmaf(d * d, alpha_inv_b, l);
            }
            loss_rows[row] += l;
            store_row_bf16(gb0, KX, row, 0, gbar, NX);
            store_t(gb0T, B2, 0, row, 0, gbar, NX);
        }
        (void)c0;
        (void)n;
    }
};

// R1..R3: g_bar = acc silu'(z_l); z_bar(tangent) = acc g_l silu''(z_l)
struct EpiTbar {
    static constexpr bool kColumns = true;
    const float *zl, *gl;
    bf16 *gb, *gbT;  // gbT = Bop_{l+1}, column row
    float *zbt;
    long long B2;
    __device__ void apply_cols(int row0, int col, const float (&u)[32], bool valid, int, int) const {
        if (!valid) return;
        float zz[32], gg[32], a[32], t[32];
        col_load(zl, H, row0, col, zz);
        col_load(gl, H, row0, col, gg);
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            a[r] = u[r] * dsilu(zz[r]);
            t[r] = u[r] * gg[r] * d2silu(zz[r]);
        }
        col_store_bf16(gb, H, row0, col, a);
        col_store_t(gbT, B2, 0, row0, col, a);
        col_store_f32(zbt, H, row0, col, t);
    }
};

// R4: g_bar_4 (FP32, for dw5), and the full z_bar_4 = out_bar w5 silu'(z_4) + tangent part
struct EpiTbarLast {
    static constexpr bool kColumns = true;
    const float *z4, *w5, *obar;
    float *gb4f, *zb4;
    bf16 *zbb4, *zb4T;  // zb4T = Aop_4, column B + row
    long long B2, Boff;
    __device__ void apply_cols(int row0, int col, const float (&u)[32], bool valid, int, int) const {
        if (!valid) return;
        const float w = w5[col];
        float zz[32], a[32], zb[32];
        col_load(z4, H, row0, col, zz);
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            const float ds = dsilu(zz[r]);
            a[r] = u[r] * ds;
            const float t = u[r] * w * d2silu(zz[r]);
            zb[r] = fmaf(obar[row0 + r] * w, ds, t);
        }
        col_store_f32(gb4f, H, row0, col, a);
        col_store_f32(zb4, H, row0, col, zb);
        col_store_bf16(zbb4, H, row0, col, zb);
        col_store_t(zb4T, B2, Boff, row0, col, zb);
    }
};

// D4..D2: z_bar_{l-1} = acc silu'(z_{l-1}) + z_bar_{l-1}(tangent)
struct EpiDbar {
    static constexpr bool kColumns = true;
    const float *zprev, *zbt;
    float *zb;
    bf16 *zbb, *zbT;  // zbb may be null (layer 1); zbT = Aop_{l-1}, column B + row
    long long B2, Boff;
    __device__ void apply_cols(int row0, int col, const float (&u)[32], bool valid, int, int) const {
        if (!valid) return;
        float zp[32], tb[32], v[32];
        col_load(zprev, H, row0, col, zp);
        col_load(zbt, H, row0, col, tb);
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = fmaf(u[r], dsilu(zp[r]), tb[r]);
        col_store_f32(zb, H, row0, col, v);
        if (zbb) col_store_bf16(zbb, H, row0, col, v);
        col_store_t(zbT, B2, Boff, row0, col, v);
    }
};

// G1..G4: FP32 partial of K slice s
struct EpiPartial {
    static constexpr bool kColumns = true;
    float *part;
    int N;
    long long M;
    __device__ void apply_cols(int row0, int col, const float (&u)[32], bool valid, int ks, int) const {
        if (valid) col_store_f32(part + (long long)ks * M * N, N, row0, col, u);
    }
};

template <class Epi>
__global__ void __launch_bounds__(tc::kThreads) gemm_kernel(const __grid_constant__ tc::TensorMaps tm,
                                                            const tc::GemmShape g, const Epi e) {
    tc::gemm_body(tm, g, e);
}

// Columns per CTA for N >= 32: 32-column tiles give 256 CTAs (about two per SM) for the
// 4096 x 256 layers, so the epilogue's SiLU work has more warps to hide its latency
// (0.40 ms per training step, against 0.50 ms with 64-column tiles at one CTA per SM).
constexpr int kBN = 32;
__host__ __device__ constexpr int tile_n(int N) { return N >= kBN ? kBN : N; }

// Launch with programmatic stream serialization: the kernel may start while the previous kernel
// in the stream finishes; every kernel launched this way calls tc::pdl_wait before it reads what
// its predecessors wrote.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

template <class Epi>
cudaError_t gemm(const bf16 *A, long long lda, const bf16 *Bm, long long ldb, int M, int N, int K, int k_slice,
                 const Epi &e, int *err, cudaStream_t st, int bn = 0) {
    const int BN = bn ? bn : tile_n(N);
    // shapes the kernel handles: whole 128-row tiles, BN-column tiles (16..256, a multiple of
    // 16), K slices of whole 64-wide k-blocks (the epilogue also stages through the ring, so at
    // least one stage must exist)
    if (M % tc::kBM || BN < 16 || BN > 256 || BN % 16 || N % BN || k_slice < tc::kBK || k_slice % tc::kBK ||
        K % k_slice)
        return cudaErrorInvalidValue;
    tc::TensorMaps tm;
    cudaError_t r = tc::make_maps(&tm, A, lda, Bm, ldb, M, N, K, BN);
    if (r != cudaSuccess) return r;
    tc::GemmShape g{M, N, K, BN, k_slice, err};
    const int kb = (k_slice / tc::kBK) < tc::kStages ? (k_slice / tc::kBK) : tc::kStages;
    const size_t smem = tc::smem_bytes(BN, kb);
    // the largest tile any call uses (BN = 256, a full ring), set once per device
    static bool attr_set[64] = {false};
    int dev = 0;
    r = cudaGetDevice(&dev);
    if (r != cudaSuccess) return r;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        r = cudaFuncSetAttribute(gemm_kernel<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tc::smem_bytes(256, tc::kStages));
        if (r != cudaSuccess) return r;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    r = launch_pdl(gemm_kernel<Epi>, dim3(M / tc::kBM, N / BN, K / k_slice), dim3(tc::kThreads), smem, st, tm, g, e);
    if (r != cudaSuccess) return r;
    return cudaGetLastError();
}

// ------------------------------------------------------------ small kernels --

// X [n_rows][7] FP32 -> x0 [B][KX] BF16 (zero padding) and X^T into Bop_1 columns B + row.
__global__ void prep_input_kernel(const float *__restrict__ X, int n_rows, int B, bf16 *x0, bf16 *xT, long long B2) {
    tc::pdl_wait();
    tc::pdl_trigger();
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < B * DIN; q += gridDim.x * blockDim.x) {
        const int r = q / DIN, j = q - r * DIN;
        const float v = r < n_rows ? X[(long long)r * DIN + j] : 0.0f;
        const bf16 b = __float2bfloat16_rn(v);
        x0[(long long)r * KX + j] = b;
        if (xT) xT[(long long)j * B2 + B + r] = b;
    }
}

// FP32 parameters -> BF16 W_l (row-major, layer 1 padded to KX columns) and W_l^T.
__global__ void weights_to_bf16_kernel(const float *__restrict__ prm, bf16 *W1b, bf16 *W1t, bf16 *W2b, bf16 *W2t,
                                       bf16 *W3b, bf16 *W3t, bf16 *W4b, bf16 *W4t) {
    tc::pdl_wait();
    tc::pdl_trigger();
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 3 * H * H + H * DIN; q += gridDim.x * blockDim.x) {
        if (q < H * DIN) {
            const int n = q / DIN, k = q - n * DIN;
            const bf16 b = __float2bfloat16_rn(prm[oW1 + q]);
            W1b[n * KX + k] = b;
            W1t[k * H + n] = b;
        } else {
            const int r = q - H * DIN;
            const int l = 2 + r / (H * H);
            const int e = r % (H * H), n = e / H, k = e - n * H;
            const bf16 b = __float2bfloat16_rn(prm[oW(l) + e]);
            bf16 *Wb = l == 2 ? W2b : (l == 3 ? W3b : W4b);
            bf16 *Wt = l == 2 ? W2t : (l == 3 ? W3t : W4t);
            Wb[n * H + k] = b;
            Wt[k * H + n] = b;
        }
    }
}

// out = sum of the F4 partial dot products (tile order) + b5; with labels,
// out_bar = 2 (out - y)/B and the value part of the loss.
__global__ void finish_out_kernel(const float *__restrict__ outp, int ntile, int B, const float *__restrict__ b5,
                                  const float *__restrict__ y, float inv_b, float *out, float *obar,
                                  float *loss_rows) {
    tc::pdl_wait();
    tc::pdl_trigger();
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < B; r += gridDim.x * blockDim.x) {
        float o = b5[0];
        for (int t = 0; t < ntile; ++t) o += outp[(long long)t * B + r];
        out[r] = o;
        if (y) {
            const float d = o - y[r];
            obar[r] = 2.0f * d * inv_b;
            loss_rows[r] = d * d * inv_b;
        }
    }
}

// dW_l[i][k] = sum over K slices in order, all four layers in one launch (layer 1: k < 7 of the
// 16 computed columns).
struct Partials {
    const float *part[5];
    int split;
};
__global__ void reduce_split_kernel(const Partials pp, float *grads) {
    tc::pdl_wait();
    tc::pdl_trigger();
    constexpr long long n1 = (long long)H * DIN, nl = (long long)H * H;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n1 + 3 * nl;
         q += (long long)gridDim.x * blockDim.x) {
        const int l = q < n1 ? 1 : 2 + (int)((q - n1) / nl);
        const long long e = q < n1 ? q : (q - n1) % nl;
        const int ncopy = l == 1 ? DIN : H, N = l == 1 ? NX : H;
        const long long i = e / ncopy, k = e - i * ncopy;
        const float *part = pp.part[l];
        float s = 0.0f;
        for (int sl = 0; sl < pp.split; ++sl) s += part[((long long)sl * H + i) * N + k];
        grads[oW(l) + e] = s;
    }
}

// ------------------------------------------------------- the row chain --
// Every product of the step except G1..G4 is row-local: a row's F, T, R and D stages read only
// that row's earlier results.  chain_kernel runs them all for one 128-row block per CTA (tc::Chain:
// one ring and one 256-column accumulator for the whole sequence), with the input staging and
// the F4 output row sums in between, so the fifteen GEMMs, prep_input and finish_out become one
// launch.  Stage order and epilogues are those of run_forward and loss_grad_impl.  Measured at
// batch 4096 (32 CTAs): 0.47 ms per training step against 0.18 ms with one launch per GEMM -- the
// epilogues' row-major and transposed stores (about 20 MB per step) then run on 32 SMs with four
// warps each (13.8 % of issue slots busy, the tensor pipe 3 % of active cycles), where one launch
// per GEMM spreads them over 256 CTAs; so it is opt-in (MCAAD_MLP_CHAIN=1).
constexpr int kChainStages = 15;  // F1..F4, T4..T1, R1..R4, D4..D2
struct ChainParams {
    CUtensorMap a[kChainStages], b[kChainStages];  // each stage's A (the block's rows) and B (all N rows)
    EpiFwd f[3];      // F1..F3
    EpiFwdLast f4;
    EpiTan t[3];      // T4, T3, T2
    EpiTanIn t1;
    EpiTbar r[3];     // R1..R3
    EpiTbarLast r4;
    EpiDbar d[3];     // D4, D3, D2
    const float *X, *b5, *y, *outp;
    bf16 *x0, *xT;
    float *out, *obar, *loss_rows;
    float inv_b;
    int B;
    long long B2;
    int *err;
};

__global__ void __launch_bounds__(tc::kThreads, 1) chain_kernel(const __grid_constant__ ChainParams P) {
    tc::Chain c;
    tc::chain_setup(c);
    tc::pdl_wait();
    const int row0 = blockIdx.x * tc::kBM;
    // the block's input rows: x0 (BF16, K padded to KX; the padding stays zero) and X^T into Bop_1
    for (int q = threadIdx.x; q < tc::kBM * DIN; q += blockDim.x) {
        const int r = row0 + q / DIN, j = q % DIN;
        const bf16 v = __float2bfloat16_rn(P.X[(long long)r * DIN + j]);
        P.x0[(long long)r * KX + j] = v;
        P.xT[(long long)j * P.B2 + P.B + r] = v;
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    bool ok = true;
    int s = 0;
    for (int l = 0; l < 3 && ok; ++l, ++s) ok = tc::chain_stage(c, &P.a[s], &P.b[s], l == 0 ? KX : H, H, row0, P.f[l]);
    if (ok) ok = tc::chain_stage(c, &P.a[s], &P.b[s], H, H, row0, P.f4);
    ++s;
    if (ok) {  // out, out_bar and the value part of the loss for the block's rows
        const int r = row0 + threadIdx.x;
        float o = P.b5[0];
        for (int t = 0; t < H / 32; ++t) o += P.outp[(long long)t * P.B + r];
        P.out[r] = o;
        const float d = o - P.y[r];
        P.obar[r] = 2.0f * d * P.inv_b;
        P.loss_rows[r] = d * d * P.inv_b;
    }
    __syncthreads();
    for (int l = 0; l < 3 && ok; ++l, ++s) ok = tc::chain_stage(c, &P.a[s], &P.b[s], H, H, row0, P.t[l]);
    if (ok) ok = tc::chain_stage(c, &P.a[s], &P.b[s], H, NX, row0, P.t1);
    ++s;
    for (int l = 0; l < 3 && ok; ++l, ++s) ok = tc::chain_stage(c, &P.a[s], &P.b[s], l == 0 ? KX : H, H, row0, P.r[l]);
    if (ok) ok = tc::chain_stage(c, &P.a[s], &P.b[s], H, H, row0, P.r4);
    ++s;
    for (int l = 0; l < 3 && ok; ++l, ++s) ok = tc::chain_stage(c, &P.a[s], &P.b[s], H, H, row0, P.d[l]);
    tc::pdl_trigger();
    tc::chain_teardown(c);
    if (!ok && threadIdx.x == 0 && P.err) atomicExch(P.err, 1);
}

// The same chain with each stage's 256 columns spread over a cluster of eight CTAs (32 columns
// each, as the per-GEMM launches tile them): a stage's epilogue stores reach the next stage's
// loads in the other CTAs through a cluster barrier (release/acquire) instead of a kernel
// boundary.  Every CTA passes every barrier, computing or not (T1's 16 columns are rank 0's), so a
// failed stage stops no CTA early.  Measured at batch 4096: 0.193 ms per training step against
// 0.187 ms with one launch per GEMM (MCAAD_MLP_CHAIN=2 selects it): the kernel boundaries it
// removes were not what each stage waits for; each CTA's own chain of TMA, MMA and epilogue
// latencies is the same in both.
constexpr int kClusterCtas = H / 32;
constexpr int kClusterBN = 32;

__global__ void __launch_bounds__(tc::kThreads, 1) chain_cluster_kernel(const __grid_constant__ ChainParams P) {
    tc::Chain c;
    tc::chain_setup(c, kClusterBN);
    const int rank = (int)tc::cluster_rank();
    const int row0 = (int)(blockIdx.x / kClusterCtas) * tc::kBM;
    const int col0 = rank * kClusterBN;
    constexpr int kRowsPer = tc::kBM / kClusterCtas;  // rows of the block's row work per CTA
    tc::pdl_wait();
    for (int q = threadIdx.x; q < kRowsPer * DIN; q += blockDim.x) {
        const int r = row0 + rank * kRowsPer + q / DIN, j = q % DIN;
        const bf16 v = __float2bfloat16_rn(P.X[(long long)r * DIN + j]);
        P.x0[(long long)r * KX + j] = v;
        P.xT[(long long)j * P.B2 + P.B + r] = v;
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    tc::cluster_sync();
    bool ok = true;
    int s = 0;
    auto stage = [&](const auto &epi, int K, int N, bool mine, int cb) {
        if (ok && mine) ok = tc::chain_stage(c, &P.a[s], &P.b[s], K, N, row0, epi, cb);
        ++s;
        tc::cluster_sync();
    };
    for (int l = 0; l < 3; ++l) stage(P.f[l], l == 0 ? KX : H, kClusterBN, true, col0);
    stage(P.f4, H, kClusterBN, true, col0);
    if (ok && threadIdx.x < kRowsPer) {  // out, out_bar and the value part of the loss
        const int r = row0 + rank * kRowsPer + threadIdx.x;
        float o = P.b5[0];
        for (int t = 0; t < H / 32; ++t) o += P.outp[(long long)t * P.B + r];
        P.out[r] = o;
        const float d = o - P.y[r];
        P.obar[r] = 2.0f * d * P.inv_b;
        P.loss_rows[r] = d * d * P.inv_b;
    }
    tc::cluster_sync();
    for (int l = 0; l < 3; ++l) stage(P.t[l], H, kClusterBN, true, col0);
    stage(P.t1, H, NX, rank == 0, 0);
    for (int l = 0; l < 3; ++l) stage(P.r[l], l == 0 ? KX : H, kClusterBN, true, col0);
    stage(P.r4, H, kClusterBN, true, col0);
    for (int l = 0; l < 3; ++l) stage(P.d[l], H, kClusterBN, true, col0);
    tc::pdl_trigger();
    tc::chain_teardown(c);
    if (!ok && threadIdx.x == 0 && P.err) atomicExch(P.err, 1);
}

// Column sums in a fixed order, coalesced, in two passes.  Pass 1: block
// (q, c) covers 32 consecutive columns of one source over row chunk c of
// kColChunk rows; lane = column, the 8 warps take rows r0 + w, r0 + w + 8, ...
// and their sums are added in warp order into colpart[c][...].  Sources:
// q < 32: db_l = sum_rows z_bar_l (l = 1 + q/8); q < 40: dw5 = sum_rows
// (g_bar_4 + h_4 out_bar); q == 40: db5 = sum out_bar (column 0) and the loss
// (column 1).  Pass 2 adds the chunks in chunk order.
constexpr int kColChunk = 128;
constexpr int kColOut = 41 * 32;

__global__ void __launch_bounds__(256) colsum_kernel(const Bufs b, float *colpart) {
    tc::pdl_wait();
    tc::pdl_trigger();
    __shared__ float red[8][33];
    const int q = blockIdx.x, chunk = blockIdx.y, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = chunk * kColChunk, r1 = min(b.B, r0 + kColChunk);
    float s = 0.0f;
    if (q < 32) {
        const int l = 1 + q / 8, c = (q % 8) * 32 + lane;
        for (int r = r0 + w; r < r1; r += 8) s += b.zb[l][(long long)r * H + c];
    } else if (q < 40) {
        const int c = (q - 32) * 32 + lane;
        for (int r = r0 + w; r < r1; r += 8)
            s += b.gb4f[(long long)r * H + c] + __bfloat162float(b.h[4][(long long)r * H + c]) * b.obar[r];
    } else if (lane < 2) {
        for (int r = r0 + w; r < r1; r += 8) s += lane == 0 ? b.obar[r] : b.loss_rows[r];
    }
    red[w][lane] = s;
    __syncthreads();
    if (w == 0) {
        float t = 0.0f;
        for (int k = 0; k < 8; ++k) t += red[k][lane];
        colpart[(long long)chunk * kColOut + q * 32 + lane] = t;
    }
}

__global__ void colsum_finish_kernel(const float *__restrict__ colpart, int n_chunks, float *grads, float *loss_out) {
    tc::pdl_wait();
    tc::pdl_trigger();
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < kColOut; o += gridDim.x * blockDim.x) {
        float t = 0.0f;
        for (int c = 0; c < n_chunks; ++c) t += colpart[(long long)c * kColOut + o];
        const int q = o / 32, lane = o % 32;
        if (q < 32) grads[ob(1 + q / 8) + (q % 8) * 32 + lane] = t;
        else if (q < 40) grads[ow5 + (q - 32) * 32 + lane] = t;
        else if (lane == 0) grads[ob5] = t;
        else if (lane == 1 && loss_out) loss_out[0] = t;
    }
}

// The BF16 weight copies the GEMMs read (W_l row-major, layer 1 padded to KX columns, and W_l^T).
struct WCopies {
    bf16 *Wb[5], *Wt[5];
};
__device__ __forceinline__ void put_weight_bf16(const WCopies &w, long long q, float val) {
    if (q < oW1 + H * DIN) {
        const int n = (int)(q / DIN), k = (int)(q - (long long)n * DIN);
        const bf16 b = __float2bfloat16_rn(val);
        w.Wb[1][n * KX + k] = b;
        w.Wt[1][k * H + n] = b;
        return;
    }
    for (int l = 2; l <= 4; ++l) {
        const long long e = q - oW(l);
        if (e >= 0 && e < (long long)H * H) {
            const int n = (int)(e / H), k = (int)(e - (long long)n * H);
            const bf16 b = __float2bfloat16_rn(val);
            w.Wb[l][n * H + k] = b;
            w.Wt[l][k * H + n] = b;
            return;
        }
    }
}

// Adam (Kingma & Ba) on the FP32 master parameters (t counts from 1, c1 and c2 its bias
// corrections), and the BF16 copies of the updated weights.
__global__ void adam_kernel(float *prm, const float *__restrict__ g, float *m, float *v, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2, const WCopies w) {
    tc::pdl_wait();
    tc::pdl_trigger();
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const float gg = g[q];
        const float mm = fmaf(b1, m[q], (1.0f - b1) * gg);
        const float vv = fmaf(b2, v[q], (1.0f - b2) * gg * gg);
        m[q] = mm;
        v[q] = vv;
        const float p = prm[q] - lr * (mm * c1) / (sqrtf(vv * c2) + eps);
        prm[q] = p;
        put_weight_bf16(w, q, p);
    }
}

int grid_for(long long work) {
    long long g = (work + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace mlp
}  // namespace mcaad

using namespace mcaad;
using namespace mcaad::mlp;

// A captured training step (mlp_train_step): the graph of loss and gradient, Adam and the weight
// refresh for one set of caller buffers, and its Adam node (whose learning rate and bias
// corrections change every step).
struct TrainGraph {
    cudaStream_t cap = nullptr;  // private stream the step is captured on
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t adam = nullptr;
    const void *key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // params, grads, loss, m, v
    float alpha = 0, beta1 = 0, beta2 = 0, eps = 0;
};

struct mlp_ctx {
    int device = 0;
    int B = 0;
    Bufs b{};
    unsigned char *ws = nullptr;
    bool owns = false;
    TrainGraph tg;
};

namespace {

struct Carve {
    unsigned char *base;
    size_t off = 0;
    template <typename T>
    T *take(size_t n) {
        T *p = base ? (T *)(base + off) : nullptr;
        off = (off + n * sizeof(T) + 255) / 256 * 256;
        return p;
    }
};

size_t layout(unsigned char *base, int B, Bufs *out) {
    Carve c{base};
    Bufs b{};
    b.B = B;
    b.split = k_split(B);
    const int sp = env_knob("MCAAD_MLP_WGRAD_SPLIT"), bn = env_knob("MCAAD_MLP_WGRAD_BN");
    if ((sp == 4 || sp == 8 || sp == 16) && (B / 32) % sp == 0) b.split = sp;
    b.wgrad_bn = (bn >= 16 && bn <= 256 && bn % 16 == 0) ? bn : kWgradBN;
    const size_t BH = (size_t)B * H, B2 = 2 * (size_t)B;
    b.x0 = c.take<bf16>((size_t)B * KX);
    for (int l = 1; l <= 4; ++l) b.z[l] = c.take<float>(BH);
    for (int l = 1; l <= 4; ++l) b.h[l] = c.take<bf16>(BH);
    b.out = c.take<float>(B);
    b.obar = c.take<float>(B);
    b.loss_rows = c.take<float>(B);
    b.outp = c.take<float>((size_t)(H / 32) * B);
    for (int l = 1; l <= 4; ++l) b.p[l] = c.take<bf16>(BH);
    b.g[0] = c.take<float>((size_t)B * NX);
    for (int l = 1; l <= 3; ++l) b.g[l] = c.take<float>(BH);
    b.gb0 = c.take<bf16>((size_t)B * KX);
    for (int l = 1; l <= 3; ++l) b.gb[l] = c.take<bf16>(BH);
    b.gb4f = c.take<float>(BH);
    for (int l = 1; l <= 4; ++l) b.zbt[l] = c.take<float>(BH);
    for (int l = 1; l <= 4; ++l) b.zb[l] = c.take<float>(BH);
    for (int l = 2; l <= 4; ++l) b.zbb[l] = c.take<bf16>(BH);
    for (int l = 1; l <= 4; ++l) b.Aop[l] = c.take<bf16>(H * B2);
    b.Bop[1] = c.take<bf16>(NX * B2);
    for (int l = 2; l <= 4; ++l) b.Bop[l] = c.take<bf16>(H * B2);
    for (int l = 1; l <= 4; ++l) b.part[l] = c.take<float>((size_t)kSplit * H * (l == 1 ? NX : H));
    b.colpart = c.take<float>((size_t)(B / 128) * 41 * 32);
    b.Wb[1] = c.take<bf16>((size_t)H * KX);
    b.Wt[1] = c.take<bf16>((size_t)NX * H);
    for (int l = 2; l <= 4; ++l) {
        b.Wb[l] = c.take<bf16>((size_t)H * H);
        b.Wt[l] = c.take<bf16>((size_t)H * H);
    }
    b.lsum = c.take<float>(1);
    b.Xin = c.take<float>((size_t)B * DIN);
    b.yin = c.take<float>(B);
    b.dyin = c.take<float>((size_t)B * NTH);
    b.err = c.take<int>(1);
    if (out) *out = b;
    return c.off;
}

mc_status cuda_st(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return MC_OK;
    fprintf(stderr, "mlp: %s: %s\n", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MC_ERR_OOM : MC_ERR_CUDA;
}

// F1..F4 (+ T4..T1 when grad) for the batch already staged in x0.
cudaError_t run_forward(mlp_ctx *c, const float *prm, const float *y, const float *dy, float alpha, bool tangent,
                        cudaStream_t st) {
    Bufs &b = c->b;
    const int B = b.B;
    const long long B2 = 2LL * B;
    const float inv_b = 1.0f / (float)B;
    cudaError_t e;
    for (int l = 1; l <= 3; ++l) {
        EpiFwd ep{prm + ob(l), b.z[l], b.h[l], b.Bop[l + 1], B2, B};
        const bf16 *A = l == 1 ? b.x0 : b.h[l - 1];
        const int K = l == 1 ? KX : H;
        e = gemm(A, K, b.Wb[l], K, B, H, K, K, ep, b.err, st);
        if (e != cudaSuccess) return e;
    }
    {
        EpiFwdLast ep{prm + ob4, prm + ow5, b.z[4], b.outp, b.h[4], b.p[4], b.Aop[4], B2, B};
        e = gemm(b.h[3], H, b.Wb[4], H, B, H, H, H, ep, b.err, st);
        if (e != cudaSuccess) return e;
        e = launch_pdl(finish_out_kernel, dim3(grid_for(B)), dim3(256), 0, st, (const float *)b.outp, H / 32, B,
                       prm + ob5, y, inv_b, b.out, b.obar, b.loss_rows);
        if (e != cudaSuccess) return e;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (!tangent) return cudaSuccess;
    for (int l = 4; l >= 2; --l) {
        EpiTan ep{b.z[l - 1], b.g[l - 1], b.p[l - 1], b.Aop[l - 1], B2};
        e = gemm(b.p[l], H, b.Wt[l], H, B, H, H, H, ep, b.err, st);
        if (e != cudaSuccess) return e;
    }
    EpiTanIn ep{b.g[0], dy, b.gb0, b.Bop[1], b.loss_rows, B2, 2.0f * alpha * inv_b, alpha * inv_b};
    return gemm(b.p[1], H, b.Wt[1], H, B, NX, H, H, ep, b.err, st);
}

void drop_graph(TrainGraph &tg) {
    if (tg.exec) cudaGraphExecDestroy(tg.exec);
    if (tg.graph) cudaGraphDestroy(tg.graph);
    tg.exec = nullptr;
    tg.graph = nullptr;
    tg.adam = nullptr;
}

// The differential loss and its gradient for the batch (X, y, dy), all stream-ordered on st.
// The row chain of the training step (F1..F4, T4..T1, R1..R4, D4..D2 and their input and output
// row work) as one chain_kernel launch of B/128 CTAs.
cudaError_t chain_impl(mlp_ctx *c, const float *prm, const float *X, const float *y, const float *dy, float alpha,
                       cudaStream_t st, bool cluster) {
    Bufs &b = c->b;
    const int B = b.B;
    const long long B2 = 2LL * B;
    const float inv_b = 1.0f / (float)B;
    ChainParams P;
    memset(&P, 0, sizeof(P));
    cudaError_t e = cudaSuccess;
    int s = 0;
    auto stage_maps = [&](const bf16 *A, int K, const bf16 *Bw, int N) {
        if (e == cudaSuccess) e = tc::make_map(&P.a[s], A, K, K, B, tc::kBM);
        if (e == cudaSuccess) e = tc::make_map(&P.b[s], Bw, K, K, N, cluster && N > kClusterBN ? kClusterBN : N);
        ++s;
    };
    for (int l = 1; l <= 3; ++l) {
        P.f[l - 1] = EpiFwd{prm + ob(l), b.z[l], b.h[l], b.Bop[l + 1], B2, B};
        stage_maps(l == 1 ? b.x0 : b.h[l - 1], l == 1 ? KX : H, b.Wb[l], H);
    }
    P.f4 = EpiFwdLast{prm + ob4, prm + ow5, b.z[4], b.outp, b.h[4], b.p[4], b.Aop[4], B2, B};
    stage_maps(b.h[3], H, b.Wb[4], H);
    for (int l = 4; l >= 2; --l) {
        P.t[4 - l] = EpiTan{b.z[l - 1], b.g[l - 1], b.p[l - 1], b.Aop[l - 1], B2};
        stage_maps(b.p[l], H, b.Wt[l], H);
    }
    P.t1 = EpiTanIn{b.g[0], dy, b.gb0, b.Bop[1], b.loss_rows, B2, 2.0f * alpha * inv_b, alpha * inv_b};
    stage_maps(b.p[1], H, b.Wt[1], NX);
    for (int l = 1; l <= 3; ++l) {
        P.r[l - 1] = EpiTbar{b.z[l], b.g[l], b.gb[l], b.Bop[l + 1], b.zbt[l], B2};
        stage_maps(l == 1 ? b.gb0 : b.gb[l - 1], l == 1 ? KX : H, b.Wb[l], H);
    }
    P.r4 = EpiTbarLast{b.z[4], prm + ow5, b.obar, b.gb4f, b.zb[4], b.zbb[4], b.Aop[4], B2, B};
    stage_maps(b.gb[3], H, b.Wb[4], H);
    for (int l = 4; l >= 2; --l) {
        P.d[4 - l] = EpiDbar{b.z[l - 1], b.zbt[l - 1], b.zb[l - 1], l - 1 >= 2 ? b.zbb[l - 1] : nullptr, b.Aop[l - 1],
                             B2, B};
        stage_maps(b.zbb[l], H, b.Wt[l], H);
    }
    if (e != cudaSuccess) return e;
    if (s != kChainStages) return cudaErrorInvalidValue;
    P.X = X;
    P.b5 = prm + ob5;
    P.y = y;
    P.outp = b.outp;
    P.x0 = b.x0;
    P.xT = b.Bop[1];
    P.out = b.out;
    P.obar = b.obar;
    P.loss_rows = b.loss_rows;
    P.inv_b = inv_b;
    P.B = B;
    P.B2 = B2;
    P.err = b.err;
    static bool attr_set[2][64] = {{false}};
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const size_t smem = cluster ? tc::chain_smem_bytes(kClusterBN) : tc::chain_smem_bytes();
    if (dev < 0 || dev >= 64 || !attr_set[cluster][dev]) {
        e = cudaFuncSetAttribute(cluster ? chain_cluster_kernel : chain_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[cluster][dev] = true;
    }
    if (!cluster) {
        e = launch_pdl(chain_kernel, dim3(B / tc::kBM), dim3(tc::kThreads), smem, st, P);
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((B / tc::kBM) * kClusterCtas);
        cfg.blockDim = dim3(tc::kThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        at[1].id = cudaLaunchAttributeClusterDimension;
        at[1].val.clusterDim.x = kClusterCtas;
        at[1].val.clusterDim.y = 1;
        at[1].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 2;
        e = cudaLaunchKernelEx(&cfg, chain_cluster_kernel, P);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t loss_grad_impl(mlp_ctx *c, const float *params, const float *X, const float *y, const float *dy,
                           float alpha, float *loss_out, float *grads, cudaStream_t st) {
    Bufs &b = c->b;
    const int B = b.B;
    const long long B2 = 2LL * B;
    cudaError_t e = cudaSuccess;
    // MCAAD_MLP_CHAIN=1: the row chain as one chain_kernel launch (measured slower, see
    // chain_kernel); 2: as one chain_cluster_kernel launch
    const int chain_mode = env_knob("MCAAD_MLP_CHAIN");
    const bool chain = chain_mode == 1 || chain_mode == 2;
    if (chain) {
        e = chain_impl(c, params, X, y, dy, alpha, st, chain_mode == 2);
    } else {
        e = launch_pdl(prep_input_kernel, dim3(grid_for((long long)B * DIN)), dim3(256), 0, st, X, B, B, b.x0,
                       b.Bop[1], B2);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = run_forward(c, params, y, dy, alpha, true, st);
    }
    // R1..R4: up the tangent chain
    for (int l = 1; l <= 4 && e == cudaSuccess && !chain; ++l) {
        const bf16 *A = l == 1 ? b.gb0 : b.gb[l - 1];
        const int K = l == 1 ? KX : H;
        if (l < 4) {
            EpiTbar ep{b.z[l], b.g[l], b.gb[l], b.Bop[l + 1], b.zbt[l], B2};
            e = gemm(A, K, b.Wb[l], K, B, H, K, K, ep, b.err, st);
        } else {
            EpiTbarLast ep{b.z[4], params + ow5, b.obar, b.gb4f, b.zb[4], b.zbb[4], b.Aop[4], B2, B};
            e = gemm(A, K, b.Wb[4], K, B, H, K, K, ep, b.err, st);
        }
    }
    // D4..D2: down the forward chain
    for (int l = 4; l >= 2 && e == cudaSuccess && !chain; --l) {
        EpiDbar ep{b.z[l - 1], b.zbt[l - 1], b.zb[l - 1], l - 1 >= 2 ? b.zbb[l - 1] : nullptr, b.Aop[l - 1], B2, B};
        e = gemm(b.zbb[l], H, b.Wt[l], H, B, H, H, H, ep, b.err, st);
    }
    // G1..G4: weight gradients over the concatenated 2B rows, split along K (G2..G4 in tiles of
    // wgrad_bn columns, G1's 16 columns in one tile)
    for (int l = 1; l <= 4 && e == cudaSuccess; ++l) {
        const int N = l == 1 ? NX : H;
        EpiPartial ep{b.part[l], N, H};
        e = gemm(b.Aop[l], B2, b.Bop[l], B2, H, N, (int)B2, (int)(B2 / b.split), ep, b.err, st,
                 N >= b.wgrad_bn ? b.wgrad_bn : 0);
    }
    if (e == cudaSuccess) {
        e = launch_pdl(reduce_split_kernel, dim3(grid_for((long long)H * DIN + 3LL * H * H)), dim3(256), 0, st,
                       Partials{{nullptr, b.part[1], b.part[2], b.part[3], b.part[4]}, b.split}, grads);
    }
    if (e == cudaSuccess) {
        const int n_chunks = B / kColChunk;
        e = launch_pdl(colsum_kernel, dim3(41, n_chunks), dim3(256), 0, st, b, b.colpart);
        if (e == cudaSuccess)
            e = launch_pdl(colsum_finish_kernel, dim3(grid_for(kColOut)), dim3(256), 0, st, (const float *)b.colpart,
                           n_chunks, grads, loss_out);
    }
    return e;
}

WCopies wcopies(const Bufs &b) {
    WCopies w{};
    for (int l = 1; l <= 4; ++l) {
        w.Wb[l] = b.Wb[l];
        w.Wt[l] = b.Wt[l];
    }
    return w;
}

// Adam step t on the parameters and the BF16 weight copies (one kernel).
cudaError_t adam_impl(mlp_ctx *c, float *params, const float *grads, float *m, float *v, int t, float lr, float beta1,
                      float beta2, float eps, cudaStream_t st) {
    const float c1 = 1.0f / (1.0f - powf(beta1, (float)t));
    const float c2 = 1.0f / (1.0f - powf(beta2, (float)t));
    return launch_pdl(adam_kernel, dim3(grid_for(kParams)), dim3(256), 0, st, params, grads, m, v, (long long)kParams,
                      lr, beta1, beta2, eps, c1, c2, wcopies(c->b));
}

}  // namespace

extern "C" {

int64_t mlp_n_params(void) { return kParams; }

mc_status mlp_workspace_size(int32_t batch, size_t *bytes_out) {
    if (!bytes_out || batch < 128 || batch % 128) return MC_ERR_INVALID_ARG;
    *bytes_out = layout(nullptr, batch, nullptr);
    return MC_OK;
}

mc_status mlp_create(int device, int32_t batch, void *workspace, size_t workspace_bytes, mlp_ctx **out) {
    if (!out || batch < 128 || batch % 128) return MC_ERR_INVALID_ARG;
    *out = nullptr;
    const size_t need = layout(nullptr, batch, nullptr);
    mc_status s = cuda_st(cudaSetDevice(device), "cudaSetDevice");
    if (s != MC_OK) return s;
    mlp_ctx *c = new (std::nothrow) mlp_ctx();
    if (!c) return MC_ERR_OOM;
    c->device = device;
    c->B = batch;
    if (workspace) {
        if (workspace_bytes < need || ((uintptr_t)workspace & 255u)) {
            delete c;
            return MC_ERR_INVALID_ARG;
        }
        c->ws = (unsigned char *)workspace;
    } else {
        s = cuda_st(cudaMalloc((void **)&c->ws, need), "cudaMalloc");
        if (s != MC_OK) {
            delete c;
            return s;
        }
        c->owns = true;
    }
    layout(c->ws, batch, &c->b);
    // padding columns and rows that no kernel writes must read as zero
    s = cuda_st(cudaMemset(c->ws, 0, need), "cudaMemset");
    if (s != MC_OK) {
        if (c->owns) cudaFree(c->ws);
        delete c;
        return s;
    }
    *out = c;
    return MC_OK;
}

void mlp_destroy(mlp_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    drop_graph(c->tg);
    if (c->tg.cap) cudaStreamDestroy(c->tg.cap);
    if (c->owns && c->ws) {
        cudaSetDevice(c->device);
        cudaFree(c->ws);
    }
    delete c;
}

mc_status mlp_set_weights(mlp_ctx *c, const float *params, void *stream) {
    if (!c || !params) return MC_ERR_INVALID_ARG;
    Bufs &b = c->b;
    weights_to_bf16_kernel<<<grid_for(3LL * H * H + H * DIN), 256, 0, (cudaStream_t)stream>>>(
        params, b.Wb[1], b.Wt[1], b.Wb[2], b.Wt[2], b.Wb[3], b.Wt[3], b.Wb[4], b.Wt[4]);
    return cuda_st(cudaGetLastError(), "weights_to_bf16");
}

mc_status mlp_forward(mlp_ctx *c, const float *params, const float *X, int32_t n_rows, float *out, float *dout_dx,
                      void *stream) {
    if (!c || !params || !X || !out || n_rows < 1 || n_rows > c->B) return MC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Bufs &b = c->b;
    prep_input_kernel<<<grid_for((long long)c->B * DIN), 256, 0, st>>>(X, n_rows, c->B, b.x0, nullptr, 0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = run_forward(c, params, nullptr, nullptr, 0.0f, dout_dx != nullptr, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, b.out, sizeof(float) * n_rows, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && dout_dx)
        e = cudaMemcpy2DAsync(dout_dx, sizeof(float) * DIN, b.g[0], sizeof(float) * NX, sizeof(float) * DIN, n_rows,
                              cudaMemcpyDeviceToDevice, st);
    return cuda_st(e, "mlp_forward");
}

mc_status mlp_loss_grad(mlp_ctx *c, const float *params, const float *X, const float *y, const float *dy, float alpha,
                        float *loss_out, float *grads, void *stream) {
    if (!c || !params || !X || !y || !dy || !grads) return MC_ERR_INVALID_ARG;
    return cuda_st(loss_grad_impl(c, params, X, y, dy, alpha, loss_out, grads, (cudaStream_t)stream), "mlp_loss_grad");
}

mc_status mlp_adam_step(mlp_ctx *c, float *params, const float *grads, float *m, float *v, int32_t t, float lr,
                        float beta1, float beta2, float eps, void *stream) {
    if (!c || !params || !grads || !m || !v || t < 1) return MC_ERR_INVALID_ARG;
    return cuda_st(adam_impl(c, params, grads, m, v, t, lr, beta1, beta2, eps, (cudaStream_t)stream), "adam");
}

}  // extern "C"

namespace {

// Capture loss and gradient, Adam and the weight refresh of the context's own batch buffers into
// a graph (on the context's private stream: capture is not possible on the legacy default
// stream), and find the Adam node.
cudaError_t capture_step(mlp_ctx *c, float *params, float *grads, float *loss_out, float *m, float *v, float alpha,
                         float beta1, float beta2, float eps) {
    TrainGraph &tg = c->tg;
    drop_graph(tg);
    cudaError_t e = cudaSuccess;
    if (!tg.cap) e = cudaStreamCreateWithFlags(&tg.cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(tg.cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    Bufs &b = c->b;
    cudaError_t e1 = loss_grad_impl(c, params, b.Xin, b.yin, b.dyin, alpha, loss_out, grads, tg.cap);
    if (e1 == cudaSuccess) e1 = adam_impl(c, params, grads, m, v, 1, 1e-3f, beta1, beta2, eps, tg.cap);
    e = cudaStreamEndCapture(tg.cap, &tg.graph);
    if (e1 != cudaSuccess) e = e1;
    if (e != cudaSuccess) {
        drop_graph(tg);
        return e;
    }
    size_t n = 0;
    e = cudaGraphGetNodes(tg.graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess && n) e = cudaGraphGetNodes(tg.graph, nodes.data(), &n);
    for (size_t i = 0; e == cudaSuccess && i < n && !tg.adam; ++i) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nodes[i], &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        if (cudaGraphKernelNodeGetParams(nodes[i], &kp) == cudaSuccess && kp.func == (void *)adam_kernel)
            tg.adam = nodes[i];
    }
    if (e == cudaSuccess && !tg.adam) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&tg.exec, tg.graph, 0);
    if (e != cudaSuccess) {
        drop_graph(tg);
        return e;
    }
    const void *key[5] = {params, grads, loss_out, m, v};
    for (int i = 0; i < 5; ++i) tg.key[i] = key[i];
    tg.alpha = alpha;
    tg.beta1 = beta1;
    tg.beta2 = beta2;
    tg.eps = eps;
    return cudaSuccess;
}

}  // namespace

extern "C" {

mc_status mlp_train_step(mlp_ctx *c, float *params, const float *X, const float *y, const float *dy, float alpha,
                         float *grads, float *loss_out, float *m, float *v, int32_t t, float lr, float beta1,
                         float beta2, float eps, void *stream) {
    if (!c || !params || !X || !y || !dy || !grads || !m || !v || t < 1) return MC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Bufs &b = c->b;
    const int B = b.B;
    cudaError_t e = cudaMemcpyAsync(b.Xin, X, sizeof(float) * B * DIN, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.yin, y, sizeof(float) * B, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.dyin, dy, sizeof(float) * B * NTH, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_st(e, "mlp_train_step");
    TrainGraph &tg = c->tg;
    const void *key[5] = {params, grads, loss_out, m, v};
    bool same = tg.exec && tg.alpha == alpha && tg.beta1 == beta1 && tg.beta2 == beta2 && tg.eps == eps;
    for (int i = 0; i < 5; ++i) same = same && tg.key[i] == key[i];
    if (!same) {
        // this step runs eagerly (it also sets every kernel's launch attributes); the graph is
        // captured for the following steps with these buffers
        e = loss_grad_impl(c, params, b.Xin, b.yin, b.dyin, alpha, loss_out, grads, st);
        if (e == cudaSuccess) e = adam_impl(c, params, grads, m, v, t, lr, beta1, beta2, eps, st);
        if (e == cudaSuccess) e = capture_step(c, params, grads, loss_out, m, v, alpha, beta1, beta2, eps);
        return cuda_st(e, "mlp_train_step");
    }
    // the Adam node's learning rate and bias corrections for step t
    float lr_ = lr, b1 = beta1, b2 = beta2, ep = eps;
    float c1 = 1.0f / (1.0f - powf(beta1, (float)t)), c2 = 1.0f / (1.0f - powf(beta2, (float)t));
    long long n = kParams;
    float *prm = params, *mm = m, *vv = v;
    const float *g = grads;
    WCopies wc = wcopies(b);
    void *args[12] = {&prm, &g, &mm, &vv, &n, &lr_, &b1, &b2, &ep, &c1, &c2, &wc};
    cudaKernelNodeParams kp;
    e = cudaGraphKernelNodeGetParams(tg.adam, &kp);
    if (e == cudaSuccess) {
        kp.kernelParams = args;
        kp.extra = nullptr;
        e = cudaGraphExecKernelNodeSetParams(tg.exec, tg.adam, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(tg.exec, st);
    return cuda_st(e, "mlp_train_step");
}

mc_status mlp_error_flag(mlp_ctx *c, int32_t *flag_host) {
    if (!c || !flag_host) return MC_ERR_INVALID_ARG;
    return cuda_st(cudaMemcpy(flag_host, c->b.err, sizeof(int), cudaMemcpyDeviceToHost), "error flag");
}

}  // extern "C"
