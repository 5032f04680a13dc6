// mc_aux.cu -- the small kernels around the path sweeps: the fixed-order
// finalisation of E y, lambda and G (two-step algorithm, step 1 and the
// seeds of step 2), the reverse-sweep seeds of a vector-Jacobian product, the
// fixed-order finalisation of grad G (step 3), and the generator test fills.
#include "mc_internal.h"

namespace mcaad {

constexpr int kFinBlock = 256;

// Fixed-order sum of v[0], v[stride], ... v[(n-1)*stride] by one block: each
// thread adds its strided subsequence in order, then a fixed tree over the
// threads.  Deterministic for a given n.
__device__ double block_ordered_sum(const double *__restrict__ v, int n, size_t stride, double *red) {
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) s += v[(size_t)b * stride];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    return red[0];
}

// One block per instrument i (sorted order): E y_i = disc_i * (sum over the
// forward sweep's blocks) / P, written in caller order via perm.  With
// targets C: lambda_i = E y_i - C_i, seed_i = lambda_i disc_i, and the last
// block to finish (atomic ticket, no waiting) forms G = 1/2 sum_i lambda_i^2 in
// instrument order and resets the ticket.
__global__ void __launch_bounds__(kFinBlock)
finalize_forward_kernel(const double *__restrict__ part_y, int nb, int m, double inv_n,
                        const double *__restrict__ disc, const int *__restrict__ perm,
                        const double *__restrict__ C, double *Ey_out, double *seed_w,
                        double *lam2, unsigned int *ticket, double *G_out) {
    __shared__ double red[kFinBlock];
    __shared__ bool last;
    const int i = blockIdx.x;
    const double s = block_ordered_sum(part_y + i, nb, (size_t)m, red);
    if (threadIdx.x == 0) {
        const double ey = disc[i] * (s * inv_n);
        const int ci = perm[i];
        if (Ey_out) Ey_out[ci] = ey;
        last = false;
        if (C) {
            const double lam = ey - C[ci];
            seed_w[i] = lam * disc[i];
            lam2[i] = lam * lam;
            __threadfence();
            last = atomicAdd(ticket, 1u) == (unsigned)(m - 1);
        }
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double g = 0.0;
        for (int q = 0; q < m; ++q) g += ((volatile double *)lam2)[q];
        *G_out = 0.5 * g;
        *ticket = 0u;
    }
}

__global__ void seed_from_ybar_kernel(const double *__restrict__ ybar, const int *__restrict__ perm,
                                      const double *__restrict__ disc, int m, double *seed_w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        seed_w[i] = ybar[perm[i]] * disc[i];
}

// One block per parameter j: grad_j = (sum over the reverse sweep's blocks) / P.
__global__ void __launch_bounds__(kFinBlock)
finalize_grad_kernel(const double *__restrict__ part_g, int nb, int M, double inv_n, double *grad) {
    __shared__ double red[kFinBlock];
    const int j = blockIdx.x;
    const double s = block_ordered_sum(part_g + j, nb, (size_t)M, red);
    if (threadIdx.x == 0) grad[j] = s * inv_n;
}

__global__ void philox_fill_kernel(const RoundKeys rk, uint64_t path0, uint32_t n_paths, uint32_t n_calls,
                                   uint4 *out) {
    const uint64_t total = (uint64_t)n_paths * n_calls;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = q / n_calls;
        const uint32_t c = (uint32_t)(q - i * n_calls);
        const uint64_t p = path0 + i;
        out[q] = philox4x32_10(make_uint4(c, 0u, (uint32_t)p, (uint32_t)(p >> 32)), rk);
    }
}

template <typename Real>
__global__ void normals_fill_kernel(const RoundKeys rk, uint64_t path0, uint32_t n_paths,
                                    uint32_t n_per_path, Real *out) {
    const uint32_t n_calls = (n_per_path + 3) / 4;
    const uint64_t total = (uint64_t)n_paths * n_calls;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = q / n_calls;
        const uint32_t c = (uint32_t)(q - i * n_calls);
        PathNormals<Real> g;
        g.init(path0 + i);
        g.fill(c, rk);
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

// First level of a two-level fixed-order sum over many partial rows: block b adds rows
// [b*R, (b+1)*R) in order, one thread per column (reads of a row are coalesced), into row b of out.
__global__ void __launch_bounds__(kFinBlock)
reduce_rows_kernel(const double *__restrict__ part, int rows, int width, int R, double *__restrict__ out) {
    const int r0 = blockIdx.x * R, r1 = min(rows, r0 + R);
    for (int c = threadIdx.x; c < width; c += blockDim.x) {
        double s = 0.0;
        for (int r = r0; r < r1; ++r) s += part[(size_t)r * width + c];
        out[(size_t)blockIdx.x * width + c] = s;
    }
}

// Many rows (one per warp chunk) and a scratch buffer of ceil(rows / kRowsPerBlock) rows: sum them
// in two fixed-order levels; returns the rows the per-column finalize then adds.
static cudaError_t fold_rows(const double *&part, int &nb, int width, double *scratch, cudaStream_t st) {
    if (finalize_kernels(nb, scratch) == 1) return cudaSuccess;
    const int nb1 = (nb + kRowsPerBlock - 1) / kRowsPerBlock;
    reduce_rows_kernel<<<nb1, kFinBlock, 0, st>>>(part, nb, width, kRowsPerBlock, scratch);
    part = scratch;
    nb = nb1;
    return cudaGetLastError();
}

cudaError_t launch_finalize_forward(const double *part_y, int nb, int m, double inv_n,
                                    const double *disc, const int *perm, const double *C,
                                    double *Ey_out, double *seed_w, double *lam2,
                                    unsigned int *ticket, double *G_out, cudaStream_t st, double *scratch) {
    cudaError_t e = fold_rows(part_y, nb, m, scratch, st);
    if (e != cudaSuccess) return e;
    finalize_forward_kernel<<<m, kFinBlock, 0, st>>>(part_y, nb, m, inv_n, disc, perm, C, Ey_out,
                                                      seed_w, lam2, ticket, G_out);
    return cudaGetLastError();
}

cudaError_t launch_seed_from_ybar(const double *ybar, const int *perm, const double *disc, int m,
                                  double *seed_w, cudaStream_t st) {
    seed_from_ybar_kernel<<<grid_for(m, 256), 256, 0, st>>>(ybar, perm, disc, m, seed_w);
    return cudaGetLastError();
}

cudaError_t launch_finalize_grad(const double *part_g, int nb, int M, double inv_n, double *grad,
                                 cudaStream_t st, double *scratch) {
    cudaError_t e = fold_rows(part_g, nb, M, scratch, st);
    if (e != cudaSuccess) return e;
    finalize_grad_kernel<<<M, kFinBlock, 0, st>>>(part_g, nb, M, inv_n, grad);
    return cudaGetLastError();
}

cudaError_t launch_philox_fill(uint64_t seed, uint64_t path0, uint32_t n_paths, uint32_t n_calls,
                               uint32_t *out, cudaStream_t st) {
    philox_fill_kernel<<<grid_for((uint64_t)n_paths * n_calls, 256), 256, 0, st>>>(
        philox_round_keys(seed), path0, n_paths, n_calls, (uint4 *)out);
    return cudaGetLastError();
}

cudaError_t launch_normals_fill(uint64_t seed, uint64_t path0, uint32_t n_paths,
                                uint32_t n_per_path, int precision, void *out, cudaStream_t st) {
    const uint64_t work = (uint64_t)n_paths * ((n_per_path + 3) / 4);
    const RoundKeys rk = philox_round_keys(seed);
    if (precision == 0)
        normals_fill_kernel<double><<<grid_for(work, 256), 256, 0, st>>>(rk, path0, n_paths, n_per_path,
                                                                        (double *)out);
    else
        normals_fill_kernel<float><<<grid_for(work, 256), 256, 0, st>>>(rk, path0, n_paths, n_per_path,
                                                                       (float *)out);
    return cudaGetLastError();
}

}  // namespace mcaad
