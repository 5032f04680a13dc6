// mc_internal.h -- declarations shared by the host API and the kernel
// translation units of libmcaad (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mc_common.cuh"

namespace mcaad {

struct KernelPair {
    const void *fwd = nullptr;        // forward sweep, checkpoints every K steps
    const void *rev = nullptr;        // reverse sweep, recompute from checkpoints
    const void *fwd_store = nullptr;  // forward sweep storing the whole tape
    const void *rev_tape = nullptr;   // reverse sweep reading the stored tape
    const void *fwd_z = nullptr;      // forward sweep with checkpoints that also stores its normals
    const void *rev_z = nullptr;      // reverse sweep recomputing from checkpoints on the stored normals
    size_t stage_bytes_ckpt = 0;      // rev's shared staging buffers per block
    bool rev_node_table = false;      // rev reads the surface as per-time-cell node pairs
    size_t stage_bytes_z = 0;         // rev_z's shared staging buffers per block
    const void *fwd_x = nullptr;      // forward sweep storing the state before every step (local vol)
    const void *rev_x = nullptr;      // reverse sweep running the adjoint from the stored states
    size_t stage_bytes_x = 0;         // rev_x's shared staging buffers per block
};

// Path kernels of (kind, precision, segment length K, paths per thread);
// false if that combination is not instantiated.
bool gbm_kernels(int precision, int K, int ppt, KernelPair *out);
bool heston_kernels(int precision, int K, int ppt, KernelPair *out);
bool lv_kernels(int precision, int K, int ppt, KernelPair *out);
bool lv_kernels_fp64(int K, int ppt, KernelPair *out);
bool slv_kernels(int precision, int K, int ppt, KernelPair *out);

// Small kernels (mc_aux.cu).
// Partial rows per block of the first level of a two-level finalize (launch_finalize_* with a
// scratch buffer of ceil(rows / kRowsPerBlock) rows).
constexpr int kRowsPerBlock = 64;
// Kernels one launch_finalize_* call issues for nb partial rows: two when it folds them first.
inline int finalize_kernels(int nb, const double *scratch) { return (scratch && nb > 2 * kRowsPerBlock) ? 2 : 1; }
cudaError_t launch_finalize_forward(const double *part_y, int nb, int m, double inv_n,
                                    const double *disc, const int *perm, const double *C,
                                    double *Ey_out, double *seed_w, double *lam2,
                                    unsigned int *ticket, double *G_out, cudaStream_t st,
                                    double *scratch = nullptr);
cudaError_t launch_seed_from_ybar(const double *ybar, const int *perm, const double *disc, int m,
                                  double *seed_w, cudaStream_t st);
cudaError_t launch_finalize_grad(const double *part_g, int nb, int M, double inv_n, double *grad,
                                 cudaStream_t st, double *scratch = nullptr);
cudaError_t launch_philox_fill(uint64_t seed, uint64_t path0, uint32_t n_paths, uint32_t n_calls,
                               uint32_t *out, cudaStream_t st);
cudaError_t launch_normals_fill(uint64_t seed, uint64_t path0, uint32_t n_paths,
                                uint32_t n_per_path, int precision, void *out, cudaStream_t st);

// Forward-mode Jacobian (mc_jacobian.cu).
size_t jacobian_smem_bytes(int m, int n_groups, int precision);
const void *jacobian_kernel(int precision);
int jacobian_ppt(int precision);  // paths per thread of jacobian_kernel
cudaError_t launch_jacobian(const DevProblem &pb, int precision, const double *thetas, const double *strikes_t,
                            int n_theta, uint64_t seed, uint64_t path0, uint64_t n_paths, int bpt, size_t smem,
                            double *part, const double *disc, const int *perm, double *Ey_out,
                            double *J_out, cudaStream_t st);
cudaError_t launch_tangent_finalize(const double *Ey, const double *J, const double *C, int m, double *G_out,
                                    double *grad_out, cudaStream_t st);

}  // namespace mcaad
