// tc_gemm_test.cu -- the plain tensor-core GEMM (FP32 result stored
// row-major, one slice per K split) behind the mc_tc_gemm_bf16 entry point.
#include "mcaad.h"
#include "tc_gemm.cuh"

namespace mcaad {
namespace tc {

struct StoreEpi {
    static constexpr bool kColumns = true;
    float *D;
    long long ldd;
    long long slice_stride;  // elements between K-slice outputs
    __device__ __forceinline__ void apply_cols(int row0, int col, const float (&u)[32], bool valid, int ks,
                                               int) const {
        if (!valid) return;
        float *o = D + ks * slice_stride + col;
#pragma unroll
        for (int r = 0; r < 32; ++r) o[(long long)(row0 + r) * ldd] = u[r];
    }
};

__global__ void __launch_bounds__(kThreads) gemm_store_kernel(const __grid_constant__ TensorMaps tm,
                                                               const GemmShape g, const StoreEpi e) {
    gemm_body(tm, g, e);
}

}  // namespace tc
}  // namespace mcaad

using namespace mcaad;

extern "C" mc_status mc_tc_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, int32_t M, int32_t N,
                                     int32_t K, int32_t k_slice, float *D, int64_t ldd, int32_t *err,
                                     void *stream) {
    if (!A || !B || !D || M <= 0 || N <= 0 || K <= 0) return MC_ERR_INVALID_ARG;
    if (M % tc::kBM || N % 16 || N > 256 || K % tc::kBK || k_slice <= 0 || k_slice % tc::kBK || K % k_slice)
        return MC_ERR_INVALID_ARG;
    if (lda < K || ldb < K || lda % 8 || ldb % 8 || ldd < N) return MC_ERR_INVALID_ARG;
    if (((uintptr_t)A & 15u) || ((uintptr_t)B & 15u)) return MC_ERR_INVALID_ARG;
    const int BN = N >= 64 && N % 64 == 0 ? 64 : N;
    tc::TensorMaps tm;
    if (tc::make_maps(&tm, A, lda, B, ldb, M, N, K, BN) != cudaSuccess) return MC_ERR_INVALID_ARG;
    tc::GemmShape g{M, N, K, BN, k_slice, err};
    tc::StoreEpi e{D, ldd, (long long)M * ldd};
    const int kb = (k_slice / tc::kBK) < tc::kStages ? (k_slice / tc::kBK) : tc::kStages;
    const size_t smem = tc::smem_bytes(BN, kb);
    cudaError_t st = cudaFuncSetAttribute(tc::gemm_store_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)tc::smem_bytes(256, tc::kStages));
    if (st != cudaSuccess) return MC_ERR_CUDA;
    tc::gemm_store_kernel<<<dim3(M / tc::kBM, N / BN, K / k_slice), tc::kThreads, smem, (cudaStream_t)stream>>>(tm, g,
                                                                                                                e);
    return cudaGetLastError() == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}
