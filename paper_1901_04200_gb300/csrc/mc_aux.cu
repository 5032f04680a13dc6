// mc_aux.cu -- the small kernels around the path sweeps: the fixed-order
// finalisation of E y, lambda and G (two-step algorithm, step 1 and the
// seeds of step 2), the reverse-sweep seeds of a vector-Jacobian product, the
// fixed-order finalisation of grad G (step 3), and the generator test fills.
#include "mc_internal.h"

namespace mcaad {

constexpr int kFinBlock = 256;

// E y_i = disc_i * (sum over blocks, in block order) / P  (caller order via
// perm); with targets C: lambda_i = E y_i - C_i, seed_i = lambda_i disc_i and
// G = 1/2 sum_i lambda_i^2 summed in sorted-instrument order by one thread.
__global__ void __launch_bounds__(kFinBlock)
finalize_forward_kernel(const double *__restrict__ part_y, int nb, int m, double inv_n,
                        const double *__restrict__ disc, const int *__restrict__ perm,
                        const double *__restrict__ C, double *Ey_out, double *seed_w,
                        double *G_out) {
    extern __shared__ double lam2[];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part_y[(size_t)b * m + i];
        const double ey = disc[i] * (s * inv_n);
        const int ci = perm[i];
        if (Ey_out) Ey_out[ci] = ey;
        if (C) {
            const double lam = ey - C[ci];
            seed_w[i] = lam * disc[i];
            lam2[i] = lam * lam;
        }
    }
    __syncthreads();
    if (C && threadIdx.x == 0) {
        double g = 0.0;
        for (int i = 0; i < m; ++i) g += lam2[i];
        *G_out = 0.5 * g;
    }
}

__global__ void seed_from_ybar_kernel(const double *__restrict__ ybar, const int *__restrict__ perm,
                                      const double *__restrict__ disc, int m, double *seed_w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        seed_w[i] = ybar[perm[i]] * disc[i];
}

__global__ void __launch_bounds__(kFinBlock)
finalize_grad_kernel(const double *__restrict__ part_g, int nb, int M, double inv_n, double *grad) {
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part_g[(size_t)b * M + j];
        grad[j] = s * inv_n;
    }
}

__global__ void philox_fill_kernel(uint64_t seed, uint64_t path0, uint32_t n_paths, uint32_t n_calls,
                                   uint4 *out) {
    const uint64_t total = (uint64_t)n_paths * n_calls;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = q / n_calls;
        const uint32_t c = (uint32_t)(q - i * n_calls);
        const uint64_t p = path0 + i;
        out[q] = philox4x32_10(make_uint4(c, 0u, (uint32_t)p, (uint32_t)(p >> 32)), (uint32_t)seed,
                               (uint32_t)(seed >> 32));
    }
}

template <typename Real>
__global__ void normals_fill_kernel(uint64_t seed, uint64_t path0, uint32_t n_paths,
                                    uint32_t n_per_path, Real *out) {
    const uint32_t n_calls = (n_per_path + 3) / 4;
    const uint64_t total = (uint64_t)n_paths * n_calls;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = q / n_calls;
        const uint32_t c = (uint32_t)(q - i * n_calls);
        PathNormals<Real> g;
        g.init(seed, path0 + i);
        g.fill(c);
        Real *o = out + i * n_per_path;
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t j = 4 * c + k;
            if (j < n_per_path) o[j] = g.pick(k);
        }
    }
}

static int grid_for(uint64_t work, int block) {
    uint64_t g = (work + block - 1) / block;
    if (g > 65536) g = 65536;
    return (int)(g ? g : 1);
}

cudaError_t launch_finalize_forward(const double *part_y, int nb, int m, double inv_n,
                                    const double *disc, const int *perm, const double *C,
                                    double *Ey_out, double *seed_w, double *G_out,
                                    cudaStream_t st) {
    finalize_forward_kernel<<<1, kFinBlock, (size_t)m * sizeof(double), st>>>(
        part_y, nb, m, inv_n, disc, perm, C, Ey_out, seed_w, G_out);
    return cudaGetLastError();
}

cudaError_t launch_seed_from_ybar(const double *ybar, const int *perm, const double *disc, int m,
                                  double *seed_w, cudaStream_t st) {
    seed_from_ybar_kernel<<<grid_for(m, 256), 256, 0, st>>>(ybar, perm, disc, m, seed_w);
    return cudaGetLastError();
}

cudaError_t launch_finalize_grad(const double *part_g, int nb, int M, double inv_n, double *grad,
                                 cudaStream_t st) {
    finalize_grad_kernel<<<1, kFinBlock, 0, st>>>(part_g, nb, M, inv_n, grad);
    return cudaGetLastError();
}

cudaError_t launch_philox_fill(uint64_t seed, uint64_t path0, uint32_t n_paths, uint32_t n_calls,
                               uint32_t *out, cudaStream_t st) {
    philox_fill_kernel<<<grid_for((uint64_t)n_paths * n_calls, 256), 256, 0, st>>>(
        seed, path0, n_paths, n_calls, (uint4 *)out);
    return cudaGetLastError();
}

cudaError_t launch_normals_fill(uint64_t seed, uint64_t path0, uint32_t n_paths,
                                uint32_t n_per_path, int precision, void *out, cudaStream_t st) {
    const uint64_t work = (uint64_t)n_paths * ((n_per_path + 3) / 4);
    if (precision == 0)
        normals_fill_kernel<double><<<grid_for(work, 256), 256, 0, st>>>(seed, path0, n_paths,
                                                                        n_per_path, (double *)out);
    else
        normals_fill_kernel<float><<<grid_for(work, 256), 256, 0, st>>>(seed, path0, n_paths,
                                                                       n_per_path, (float *)out);
    return cudaGetLastError();
}

}  // namespace mcaad
