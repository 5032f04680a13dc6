// tc_gemm.cuh -- BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory), D[M x N] = A[M x K] B[N x K]^T,
// with both operands K-major ("row-major, K contiguous") in global memory.
//
// One CTA of 128 threads computes a 128 x BN tile (BN <= 256, a multiple of
// 16) of D: blockIdx.x picks the 128 rows, blockIdx.y the BN columns and
// blockIdx.z the K slice when K is split.  Operand
// k-blocks of 64 elements (128 bytes per row) are copied to shared memory with
// 16-byte cp.async in the 128-byte-swizzle K-major layout (row r at r*128 B,
// 16-byte chunk c stored at chunk c ^ (r & 7), tiles 1024-byte aligned), up to
// four k-blocks per round; thread 0 issues four m128 x nN x k16 MMAs per
// k-block and commits them to an mbarrier; the epilogue reads each warp's 32
// accumulator rows (TMEM lanes 32w..32w+31) in 32-column pieces with
// tcgen05.ld and hands them to the epilogue functor.  Every wait on the
// mbarrier has an iteration limit; on expiry the kernel records an error code
// and returns after freeing its tensor memory.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mcaad {
namespace tc {

constexpr int kThreads = 128;
constexpr int kBM = 128;       // rows per CTA (one TMEM lane per row)
constexpr int kBK = 64;        // k-block: 64 BF16 = 128 bytes per row
constexpr int kMaxKB = 4;      // k-blocks per load round
constexpr uint32_t kWaitLimit = 1u << 22;

__host__ __device__ constexpr size_t tile_a_bytes() { return (size_t)kBM * kBK * 2; }
__host__ __device__ constexpr size_t tile_b_bytes(int n) { return (size_t)n * kBK * 2; }
// dynamic shared memory: 1024 B alignment slack + KB rounds of A and B tiles + barrier words
__host__ __device__ constexpr size_t smem_bytes(int n, int kb) {
    return 1024 + (size_t)kb * (tile_a_bytes() + tile_b_bytes(n)) + 64;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading byte offset (unused
// for swizzled K-major tiles), stride byte offset 1024 (eight 128-byte rows),
// descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's row.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive columns (for N = 16 tiles).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[32]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
#pragma unroll
    for (int i = 16; i < 32; ++i) v[i] = 0.f;
}

struct GemmShape {
    const __nv_bfloat16 *A;
    long long lda;  // elements between rows of A (>= K, multiple of 8)
    const __nv_bfloat16 *B;
    long long ldb;
    int M, N, K;    // M % 128 == 0, N % BN == 0, K % 64 == 0
    int BN;         // columns per CTA: a multiple of 16, at most 256; gridDim.y = N / BN
    int k_slice;    // K per CTA (a multiple of 64); gridDim.z = K / k_slice
    int *err;       // set to 1 if an mbarrier wait expired
};

// The GEMM body; Epi::apply(row, col0, v[32], ncols, kslice, state) consumes
// the accumulator columns col0..col0+ncols-1 (global column indices) of
// global row `row`, in increasing col0 within this CTA's BN columns; `state`
// is a per-thread float the epilogue may carry from one piece of its row to
// the next (it starts at 0).
template <class Epi>
__device__ __forceinline__ void gemm_body(const GemmShape &g, const Epi &epi) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int N = g.BN;
    const int kb_total = g.k_slice / kBK;
    const int kb_round = kb_total < kMaxKB ? kb_total : kMaxKB;
    unsigned char *tA = base;
    unsigned char *tB = base + (size_t)kb_round * tile_a_bytes();
    uint64_t *bar = (uint64_t *)(tB + (size_t)kb_round * tile_b_bytes(N));
    uint32_t *tslot = (uint32_t *)(bar + 1);
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const uint32_t ncols = N <= 32 ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u));

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t bar_s = smem_u32(bar);
    const uint32_t idesc = idesc_bf16(kBM, N);
    const long long row0 = (long long)blockIdx.x * kBM;
    const long long col_base = (long long)blockIdx.y * g.BN;
    const long long kbase = (long long)blockIdx.z * g.k_slice;
    uint32_t phase = 0;
    bool ok = true;

    for (int kb0 = 0; kb0 < kb_total && ok; kb0 += kb_round) {
        const int nkb = (kb_total - kb0) < kb_round ? (kb_total - kb0) : kb_round;
        // A: 128 rows x 8 chunks per k-block; B: N rows x 8 chunks per k-block
        for (int q = tid; q < nkb * kBM * 8; q += kThreads) {
            const int kb = q / (kBM * 8), rem = q - kb * (kBM * 8), r = rem >> 3, c = rem & 7;
            const __nv_bfloat16 *src = g.A + (row0 + r) * g.lda + kbase + (long long)(kb0 + kb) * kBK + c * 8;
            cp_async16(smem_u32(tA + kb * tile_a_bytes() + r * 128 + ((c ^ (r & 7)) << 4)), src);
        }
        for (int q = tid; q < nkb * N * 8; q += kThreads) {
            const int kb = q / (N * 8), rem = q - kb * (N * 8), r = rem >> 3, c = rem & 7;
            const __nv_bfloat16 *src = g.B + (col_base + r) * g.ldb + kbase + (long long)(kb0 + kb) * kBK + c * 8;
            cp_async16(smem_u32(tB + kb * tile_b_bytes(N) + r * 128 + ((c ^ (r & 7)) << 4)), src);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int kb = 0; kb < nkb; ++kb) {
                const uint32_t a0 = smem_u32(tA + kb * tile_a_bytes());
                const uint32_t b0 = smem_u32(tB + kb * tile_b_bytes(N));
#pragma unroll
                for (int k = 0; k < kBK / 16; ++k) {
                    mma_bf16(tmem, desc_sw128(a0 + k * 32), desc_sw128(b0 + k * 32), idesc,
                             (kb0 + kb + k) > 0 ? 1u : 0u);
                }
            }
            mma_commit(bar_s);
        }
        ok = mbar_wait(bar_s, phase);
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (!ok) {
        if (tid == 0 && g.err) atomicExch(g.err, 1);
    } else {
        const long long row = row0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        float state = 0.0f;
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            if (N - c0 >= 32) tmem_ld32(trow + (uint32_t)c0, v);
            else tmem_ld16(trow + (uint32_t)c0, v);
            epi.apply(row, (int)col_base + c0, v, (N - c0) < 32 ? (N - c0) : 32, blockIdx.z, state);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    }
}

}  // namespace tc
}  // namespace mcaad
