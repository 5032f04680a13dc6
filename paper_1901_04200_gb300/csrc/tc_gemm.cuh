// tc_gemm.cuh -- BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory), D[M x N] = A[M x K] B[N x K]^T,
// with both operands K-major ("row-major, K contiguous") in global memory.
//
// One CTA of 128 threads computes a 128 x BN tile (BN <= 256, a multiple of
// 16) of D: blockIdx.x picks the 128 rows, blockIdx.y the BN columns and
// blockIdx.z the K slice when K is split.  Operand k-blocks of 64 elements
// (128 bytes per row) arrive in shared memory by TMA (cp.async.bulk.tensor,
// 128-byte swizzle: row r at r*128 B, 16-byte chunk c at chunk c ^ (r & 7),
// tiles 1024-byte aligned) into a ring of up to kStages stages:
//   lane 0 of warp 0 (producer) waits until a stage is free (its "empty"
//     mbarrier), arms its "full" mbarrier with the stage's byte count and
//     issues the A and B tile loads;
//   lane 0 of warp 1 (MMA issuer) waits for a stage's "full" mbarrier, issues
//     four m128 x nN x k16 MMAs and commits them to the stage's "empty"
//     mbarrier, which the tensor cores arrive on once they have read the
//     stage -- so the loads of later k-blocks overlap the MMAs of earlier
//     ones; after the last k-block it commits to the "done" mbarrier;
//   all four warps wait for "done" and run the epilogue: each warp reads its
//     32 accumulator rows (TMEM lanes 32w..32w+31) in 32-column pieces with
//     tcgen05.ld and hands them to the epilogue functor.
// Every mbarrier wait has an iteration limit; on expiry the kernel records an
// error code, waits (again with a limit) for the loads it issued, frees its
// tensor memory and returns.  The same pieces also run a chain of GEMMs in one
// CTA (tc::Chain, below).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mcaad {
namespace tc {

constexpr int kThreads = 128;
constexpr int kBM = 128;       // rows per CTA (one TMEM lane per row)
constexpr int kBK = 64;        // k-block: 64 BF16 = 128 bytes per row
constexpr int kStages = 4;     // shared-memory ring depth
constexpr uint32_t kWaitLimit = 1u << 22;

__host__ __device__ constexpr size_t tile_a_bytes() { return (size_t)kBM * kBK * 2; }
__host__ __device__ constexpr size_t tile_b_bytes(int n) { return (size_t)n * kBK * 2; }
// dynamic shared memory: 1024 B alignment slack + `stages` ring stages of A and B tiles +
// barrier words (full[kStages], empty[kStages], done) and the TMEM address slot
__host__ __device__ constexpr size_t smem_bytes(int n, int stages) {
    return 1024 + (size_t)stages * (tile_a_bytes() + tile_b_bytes(n)) + 8 * (2 * kStages + 1) + 8;
}

// The two operands' TMA descriptors (built on the host by make_tensor_maps), passed by value
// as one __grid_constant__ kernel parameter so that their addresses are valid for TMA.
struct TensorMaps {
    CUtensorMap a, b;
};

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

// The mbarrier at `bar` receives one arrival when all previously issued MMAs of this thread
// have completed (and so have finished reading their shared-memory operands).
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

// Arrive on `bar` and add `bytes` to the transaction count its current phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the completion of the phase with parity `phase`; false once the limit
// expires.
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

// Programmatic dependent launch: pdl_wait blocks until the grids this one depends on have
// completed and their memory is visible (a no-op without such a dependency); pdl_trigger lets
// the dependent grid start launching (its blocks then run their prologue and wait in pdl_wait).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// TMA: the box at coordinates (x = k element, y = row) of the 2-D tensor map into shared
// memory at `dst`, completing `bytes` of the transaction count of mbarrier `bar`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
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
    int M, N, K;    // M % 128 == 0, N % BN == 0, K % 64 == 0
    int BN;         // columns per CTA: a multiple of 16, at most 256; gridDim.y = N / BN
    int k_slice;    // K per CTA (a multiple of 64); gridDim.z = K / k_slice
    int *err;       // set to 1 if an mbarrier wait expired
};

// Warp reduce-scatter: lane r returns the sum over the 32 lanes of their x[r] (a butterfly that
// halves the values each step: 31 shuffles for 32 sums).
__device__ __forceinline__ float warp_sum_scatter(float (&x)[32], int lane) {
#pragma unroll
    for (int o = 16, n = 32; o >= 1; o >>= 1, n >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < n / 2; ++j) {
            const float keep = up ? x[j + n / 2] : x[j];
            const float send = up ? x[j] : x[j + n / 2];
            x[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return x[0];
}

// The GEMM body.  With Epi::kColumns false, Epi::apply(row, col0, v[32], ncols, kslice, state) consumes
// the accumulator columns col0..col0+ncols-1 (global column indices) of
// global row `row`, in increasing col0 within this CTA's BN columns; `state`
// is a per-thread float the epilogue may carry from one piece of its row to
// the next (it starts at 0).  With Epi::kColumns true, Epi::apply_cols(row0, col, u[32], valid,
// kslice, lane) receives in lane j the column col = col0 + j of the warp's 32 rows row0..row0+31
// (u[r] for row row0 + r; valid is false for columns beyond N).  tm.a maps A as a 2-D tensor (K contiguous, M
// rows) with a 64 x 128 box, tm.b maps B (K contiguous, N rows) with a
// 64 x BN box, both 128-byte swizzled.
template <class Epi>
__device__ __forceinline__ void gemm_body(const TensorMaps &tm, const GemmShape &g, const Epi &epi) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int N = g.BN;
    const int kb_total = g.k_slice / kBK;
    const int S = kb_total < kStages ? kb_total : kStages;
    unsigned char *tA = base;
    unsigned char *tB = base + (size_t)S * tile_a_bytes();
    uint64_t *bars = (uint64_t *)(tB + (size_t)S * tile_b_bytes(N));  // full[kStages], empty[kStages], done
    uint32_t *tslot = (uint32_t *)(bars + 2 * kStages + 1);
    volatile int *fail = (volatile int *)(tslot + 1);  // set by the producer or MMA lane on an expired wait
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const uint32_t ncols = N <= 32 ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u));
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kStages), done = smem_u32(bars + 2 * kStages);
    const uint32_t stage_bytes = (uint32_t)(tile_a_bytes() + tile_b_bytes(N));

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        *fail = 0;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm.a) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm.b) : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    // everything above (tensor memory, barriers, descriptor prefetch) overlaps the previous
    // kernel; the operands and the epilogue's inputs are its outputs
    pdl_wait();
    const int row0 = blockIdx.x * kBM;
    const int col_base = blockIdx.y * g.BN;
    const int kbase = blockIdx.z * g.k_slice;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            // producer: k-block kb goes to stage kb % S; from the second round on, the stage is
            // reused once the MMAs that read it have completed (its empty barrier's phase)
            int issued = 0;
            for (int kb = 0; kb < kb_total; ++kb) {
                const int s = kb % S;
                if (kb >= S && !mbar_wait(empty0 + 8 * s, (uint32_t)((kb / S - 1) & 1))) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(full0 + 8 * s, stage_bytes);
                tma_load_2d(smem_u32(tA + (size_t)s * tile_a_bytes()), &tm.a, kbase + kb * kBK, row0, full0 + 8 * s);
                tma_load_2d(smem_u32(tB + (size_t)s * tile_b_bytes(N)), &tm.b, kbase + kb * kBK, col_base,
                            full0 + 8 * s);
                ++issued;
            }
            // before anything can leave: the loads of the last round have landed (bounded)
            for (int kb = issued - S < 0 ? 0 : issued - S; kb < issued; ++kb)
                if (!mbar_wait(full0 + 8 * (kb % S), (uint32_t)((kb / S) & 1))) ok = false;
            if (!ok) *fail = 1;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            const uint32_t idesc = idesc_bf16(kBM, N);
            for (int kb = 0; kb < kb_total; ++kb) {
                const int s = kb % S;
                if (!mbar_wait(full0 + 8 * s, (uint32_t)((kb / S) & 1))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = smem_u32(tA + (size_t)s * tile_a_bytes());
                const uint32_t b0 = smem_u32(tB + (size_t)s * tile_b_bytes(N));
#pragma unroll
                for (int k = 0; k < kBK / 16; ++k)
                    mma_bf16(tmem, desc_sw128(a0 + k * 32), desc_sw128(b0 + k * 32), idesc, (kb + k) > 0 ? 1u : 0u);
                mma_commit(empty0 + 8 * s);
            }
            // "done" arrives when every MMA issued above has completed (also after an expired
            // wait, so that no MMA is still running when the tensor memory is freed)
            mma_commit(done);
            if (!ok) *fail = 1;
        }
        __syncwarp();
    }
    ok = mbar_wait(done, 0u) && ok;
    if (!ok) *fail = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    pdl_trigger();  // the next kernel may start its prologue during this epilogue
    if (*fail) {
        if (tid == 0 && g.err) atomicExch(g.err, 1);
    } else if constexpr (Epi::kColumns) {
        // column-per-lane epilogue: each 32 x 32 piece of the warp's rows goes through shared
        // memory (the drained ring; pitch 33 floats, conflict-free both ways), so that lane j
        // holds column col_base + c0 + j of the warp's 32 rows and the functor's loads and
        // row-major stores are coalesced across lanes
        float *stage = (float *)base + warp * 32 * 33;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            if (N - c0 >= 32) tmem_ld32(trow + (uint32_t)c0, v);
            else tmem_ld16(trow + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) stage[lane * 33 + i] = v[i];
            __syncwarp();
            float u[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) u[r] = stage[r * 33 + lane];
            __syncwarp();
            epi.apply_cols(row0 + warp * 32, col_base + c0 + lane, u, lane < N - c0, (int)blockIdx.z, lane);
        }
    } else {
        const int row = row0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        float state = 0.0f;
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            if (N - c0 >= 32) tmem_ld32(trow + (uint32_t)c0, v);
            else tmem_ld16(trow + (uint32_t)c0, v);
            epi.apply((long long)row, col_base + c0, v, (N - c0) < 32 ? (N - c0) : 32, blockIdx.z, state);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    }
}

// ---------------------------------------------------------------- chains --
// A CTA that runs a sequence of GEMMs over its own 128 rows (D_s[128 x N_s] = A_s B_s^T, each
// stage one tile of at most the chain's `bn` columns, from column col0), each stage's epilogue
// writing what later stages read: the ring, its barriers and the tensor memory are set up once,
// and the ring's slot and phase run on across stages (k-block g of the chain uses slot
// g % kStages).  Between stages the CTA waits for
// the epilogue's stores (generic proxy) to be visible to the next stage's TMA loads (async proxy).
// A chain whose stages are at most `bn` columns wide (the B tile's rows; 256 when one CTA takes a
// whole layer, 32 when a cluster of CTAs splits its columns) needs chain_smem_bytes(bn) of shared
// memory.  A stage with an expired wait sets `fail`; the caller stops running stages (every thread
// sees the flag after the stage's closing barrier).
constexpr int kChainBN = 256;
__host__ __device__ constexpr size_t chain_smem_bytes(int bn = kChainBN) { return smem_bytes(bn, kStages); }

struct Chain {
    unsigned char *base, *tA, *tB;
    uint32_t full0, empty0, done, tmem;
    volatile int *fail;
    int bn;      // the widest stage: B slot rows and tensor-memory columns
    int kbg;     // k-blocks issued by earlier stages
    int stages;  // stages run (the done barrier's phase)
};

__host__ __device__ constexpr uint32_t tmem_cols(int bn) { return bn <= 32 ? 32u : (bn <= 64 ? 64u : (bn <= 128 ? 128u : 256u)); }

// All threads: carve the ring, initialise the barriers, allocate the tensor memory.
__device__ __forceinline__ void chain_setup(Chain &c, int bn = kChainBN) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    c.bn = bn;
    c.base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    c.tA = c.base;
    c.tB = c.base + (size_t)kStages * tile_a_bytes();
    uint64_t *bars = (uint64_t *)(c.tB + (size_t)kStages * tile_b_bytes(bn));
    uint32_t *tslot = (uint32_t *)(bars + 2 * kStages + 1);
    c.fail = (volatile int *)(tslot + 1);
    c.full0 = smem_u32(bars);
    c.empty0 = smem_u32(bars + kStages);
    c.done = smem_u32(bars + 2 * kStages);
    c.kbg = 0;
    c.stages = 0;
    const int tid = threadIdx.x;
    if (tid / 32 == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(tmem_cols(bn)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        *c.fail = 0;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(c.full0 + 8 * s, 1);
            mbar_init(c.empty0 + 8 * s, 1);
        }
        mbar_init(c.done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    c.tmem = *tslot;
}

// One stage: D[row0 .. row0+127][col0 .. col0+N) = A[rows][0 .. K) B[col0 .. col0+N)[0 .. K)^T (K a
// multiple of 64, at most kStages * 64 = 256; N a multiple of 16, at most the chain's bn; the B
// map's box is N rows), then the epilogue as in gemm_body (Epi::kColumns: lane j
// of a warp gets column c0 + j of the warp's 32 rows; else each thread its row).  Returns false
// (and sets the chain's fail flag) if a wait expired.
template <class Epi>
__device__ __forceinline__ bool chain_stage(Chain &c, const CUtensorMap *ma, const CUtensorMap *mb, int K, int N,
                                            int row0, const Epi &epi, int col0 = 0) {
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int kbt = K / kBK;
    const uint32_t stage_bytes = (uint32_t)(tile_a_bytes() + tile_b_bytes(N));
    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {  // producer
            int issued = 0;
            for (int kb = 0; kb < kbt; ++kb) {
                const int g = c.kbg + kb, s = g % kStages;
                if (g >= kStages && !mbar_wait(c.empty0 + 8 * s, (uint32_t)((g / kStages - 1) & 1))) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(c.full0 + 8 * s, stage_bytes);
                tma_load_2d(smem_u32(c.tA + (size_t)s * tile_a_bytes()), ma, kb * kBK, row0, c.full0 + 8 * s);
                tma_load_2d(smem_u32(c.tB + (size_t)s * tile_b_bytes(c.bn)), mb, kb * kBK, col0, c.full0 + 8 * s);
                ++issued;
            }
            // no load in flight when the stage ends (bounded; K <= kStages * kBK, so each slot holds
            // one k-block of this stage and its phase is the one armed above)
            for (int kb = 0; kb < issued; ++kb) {
                const int g = c.kbg + kb;
                if (!mbar_wait(c.full0 + 8 * (g % kStages), (uint32_t)((g / kStages) & 1))) ok = false;
            }
            if (!ok) *c.fail = 1;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            const uint32_t idesc = idesc_bf16(kBM, N);
            for (int kb = 0; kb < kbt; ++kb) {
                const int g = c.kbg + kb, s = g % kStages;
                if (!mbar_wait(c.full0 + 8 * s, (uint32_t)((g / kStages) & 1))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = smem_u32(c.tA + (size_t)s * tile_a_bytes());
                const uint32_t b0 = smem_u32(c.tB + (size_t)s * tile_b_bytes(c.bn));
#pragma unroll
                for (int k = 0; k < kBK / 16; ++k)
                    mma_bf16(c.tmem, desc_sw128(a0 + k * 32), desc_sw128(b0 + k * 32), idesc,
                             (kb + k) > 0 ? 1u : 0u);
                mma_commit(c.empty0 + 8 * s);
            }
            mma_commit(c.done);  // also after an expired wait: no MMA runs past the stage
            if (!ok) *c.fail = 1;
        }
        __syncwarp();
    }
    ok = mbar_wait(c.done, (uint32_t)(c.stages & 1)) && ok;
    if (!ok) *c.fail = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (!*c.fail) {
        const uint32_t trow = c.tmem + ((uint32_t)(warp * 32) << 16);
        if constexpr (Epi::kColumns) {
            float *stage = (float *)c.base + warp * 32 * 33;  // the drained ring
            for (int c0 = 0; c0 < N; c0 += 32) {
                float v[32];
                if (N - c0 >= 32) tmem_ld32(trow + (uint32_t)c0, v);
                else tmem_ld16(trow + (uint32_t)c0, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) stage[lane * 33 + i] = v[i];
                __syncwarp();
                float u[32];
#pragma unroll
                for (int r = 0; r < 32; ++r) u[r] = stage[r * 33 + lane];
                __syncwarp();
                epi.apply_cols(row0 + warp * 32, col0 + c0 + lane, u, lane < N - c0, 0, lane);
            }
        } else {
            const int row = row0 + warp * 32 + lane;
            float state = 0.0f;
            for (int c0 = 0; c0 < N; c0 += 32) {
                float v[32];
                if (N - c0 >= 32) tmem_ld32(trow + (uint32_t)c0, v);
                else tmem_ld16(trow + (uint32_t)c0, v);
                epi.apply((long long)row, col0 + c0, v, (N - c0) < 32 ? (N - c0) : 32, 0, state);
            }
        }
    }
    // the stores reach the next stage's TMA loads; tensor memory is free for its MMAs
    asm volatile("fence.proxy.async.global;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    c.kbg += kbt;
    ++c.stages;
    return !*c.fail;
}

// All threads, after the last stage: free the tensor memory.
__device__ __forceinline__ void chain_teardown(Chain &c) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x / 32 == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.tmem), "r"(tmem_cols(c.bn)));
    }
}

// All threads of every CTA of the cluster: a barrier that also orders memory (release before
// arriving, acquire after waiting), then the acquired global data made visible to this thread's
// later TMA loads.  Every CTA of a cluster must call it the same number of times.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Host: the TMA descriptor of a BF16 operand stored as `rows` rows of `cols` elements (K
// contiguous) with a row pitch of `ld` elements, loaded in boxes of 64 elements x `box_rows`
// rows with the 128-byte swizzle the MMA descriptors expect.  The encoder comes from the driver
// through the runtime's entry-point query (no link against the driver library).  The base address
// and the pitch must be multiples of 16 bytes (checked by the encoder).
inline cudaError_t make_map(CUtensorMap *map, const void *ptr, long long ld, long long cols, long long rows,
                            int box_rows) {
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }();
    if (!encode) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Host: both descriptors of D[M x N] = A[M x K] B[N x K]^T with N-tiles of BN columns.
inline cudaError_t make_maps(TensorMaps *tm, const void *A, long long lda, const void *B, long long ldb, int M, int N,
                             int K, int BN) {
    cudaError_t e = make_map(&tm->a, A, lda, K, M, kBM);
    if (e == cudaSuccess) e = make_map(&tm->b, B, ldb, K, N, BN);
    return e;
}

}  // namespace tc
}  // namespace mcaad
