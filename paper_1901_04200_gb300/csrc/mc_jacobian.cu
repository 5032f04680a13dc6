// mc_jacobian.cu -- forward-mode Jacobian of E y for many Heston parameter
// vectors at once: E y_i(theta_t) and d E y_i / d theta_j (t = 0..n_theta-1),
// the labels of the pricing surrogate.
//
// The gradient identity of the paper (dG/dx_j = E(sum_i (E y_i - C_i)
// dy_i/dx_j)) needs the pathwise derivative dy_i/dtheta_j inside the
// expectation; with M = 5 parameters one forward sweep that carries the five
// tangents (dx/dtheta_j, dv/dtheta_j) along each path gives every
// d E y_i/d theta_j at once, at about the cost of the reverse sweep and with
// no checkpoints.  The kink conventions are those of the reverse sweep:
// d max(v,0)/dv = 1{v > 0}, the tangent of sqrt(v+ dt) is 0 when v <= 0, the
// payoff derivative is 1{S > K}.
//
// Paths of parameter vector t are the global paths path0 + [t P, (t+1) P)
// with the call's seed, so different t draw independent normals.  Grid (bpt, n_theta):
// block (b, t) walks warps over chunks of 32 * PPT paths of its slice of
// theta t's paths (PPT independent recursions per thread: two in FP32, one in
// FP64) and leaves FP64 sums of y_i and of dy_i/dtheta_j per block (per-thread
// sums over its paths and warp sums in the path precision, FP64 above the
// warp, no atomics).
#include "mc_internal.h"
#include "mc_paths.cuh"

namespace mcaad {

constexpr int kJacM = 5;  // Heston parameters (kappa, theta_h, xi, rho, v0)

template <typename Real, int PPT>
__global__ void __launch_bounds__(kBlock)
heston_jacobian_kernel(const DevProblem pb, const double *__restrict__ thetas,
                       const double *__restrict__ strikes_t, const RoundKeys rk, uint64_t path0,
                       uint64_t n_paths, int bpt, double *__restrict__ out) {
    // out: [n_theta][bpt][m][1 + M] sums (y, then dy/dtheta_j)
    extern __shared__ __align__(16) unsigned char smem[];
    const int m = pb.m;
    const int t = blockIdx.y;
    Real *strike = (Real *)smem;
    int *gseg = (int *)(smem + align_up((size_t)m * sizeof(Real), 16));
    int *gbeg = gseg + pb.n_groups;
    double *wacc = (double *)(smem + align_up(align_up((size_t)m * sizeof(Real), 16) +
                                              (size_t)(2 * pb.n_groups + 1) * 4, 16));
    const int W = (1 + kJacM) * m;  // values per warp
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        strike[i] = (Real)(strikes_t ? strikes_t[(size_t)t * m + pb.perm[i]] : pb.strike[i]);
    for (int g = threadIdx.x; g < pb.n_groups; g += blockDim.x) gseg[g] = pb.grp_seg[g];
    for (int g = threadIdx.x; g <= pb.n_groups; g += blockDim.x) gbeg[g] = pb.grp_begin[g];
    for (int q = threadIdx.x; q < kWarpsPerBlock * W; q += blockDim.x) wacc[q] = 0.0;
    const double *th = thetas + (size_t)t * kJacM;
    const double kappa_d = th[0], thh_d = th[1], xi_d = th[2], rho_d = th[3];
    const Real kappa = (Real)kappa_d, xi = (Real)xi_d, rho = (Real)rho_d;
    const Real rhob = (Real)sqrt(1.0 - rho_d * rho_d);
    const Real rho_over_rhob = (Real)(rho_d / sqrt(1.0 - rho_d * rho_d));
    const Real v0 = (Real)th[4];
    const Real dt = (Real)pb.dt, rdt = (Real)(pb.r * pb.dt), kthdt = (Real)(kappa_d * thh_d * pb.dt);
    const Real thdt = (Real)(thh_d * pb.dt), kdt = (Real)(kappa_d * pb.dt);
    const Real S0 = (Real)pb.S0;
    __syncthreads();

    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    double *wrow = wacc + warp * W;
    const int K = pb.K;
    constexpr uint64_t kChunk = (uint64_t)kWarp * PPT;  // lane l carries paths chunk*kChunk + q*32 + l
    const uint64_t chunks = (n_paths + kChunk - 1) / kChunk;
    for (uint64_t ch = (uint64_t)blockIdx.x * kWarpsPerBlock + warp; ch < chunks;
         ch += (uint64_t)bpt * kWarpsPerBlock) {
        bool active[PPT];
        PathNormals<Real> rng[PPT];
        Real x[PPT], v[PPT], dx[PPT][kJacM], dv[PPT][kJacM];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const uint64_t local = ch * kChunk + q * kWarp + lane;
            active[q] = local < n_paths;
            rng[q].init(path0 + (uint64_t)t * n_paths + (active[q] ? local : 0));
            x[q] = Real(0);
            v[q] = v0;
#pragma unroll
            for (int j = 0; j < kJacM; ++j) {
                dx[q][j] = Real(0);
                dv[q][j] = (j == 4) ? Real(1) : Real(0);
            }
        }
        int g = 0;
        for (int s = 0; s < pb.n_seg; ++s) {
            for (int i = 0; i < K; ++i) {
                const int n = s * K + i;
                const uint32_t j0 = (uint32_t)(2 * n);
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    if ((j0 & 3u) == 0u) rng[q].fill(j0 >> 2, rk);
                    const Real z1 = rng[q].pick(j0 & 3u), z2 = rng[q].pick((j0 + 1) & 3u);
                    const bool pos = v[q] > Real(0);
                    const Real vdt = fmax(v[q], Real(0)) * dt;
                    const Real rs = rsqrt_r<Real>(fmax(vdt, tiny_r<Real>()));
                    const Real sq = vdt * rs;
                    const Real w = fma(rho, z1, rhob * z2);
                    // tangents: d vdt = 1{v>0} dt dv; d sq = rs/2 d vdt
                    const Real dts = pos ? dt : Real(0);
                    const Real cx = Real(0.5) * fma(rs, z1, Real(-1));   // dx'/d vdt
                    const Real cv = fma(Real(0.5) * xi * rs, w, -kappa);  // dv'/d vdt
                    const Real e_kappa = thdt - vdt, e_th = kdt, e_xi = sq * w;
                    const Real e_rho = xi * sq * fma(-rho_over_rhob, z2, z1);
#pragma unroll
                    for (int j = 0; j < kJacM; ++j) {
                        const Real dvdt = dts * dv[q][j];
                        dx[q][j] = fma(cx, dvdt, dx[q][j]);
                        Real e = Real(0);
                        if (j == 0) e = e_kappa;
                        if (j == 1) e = e_th;
                        if (j == 2) e = e_xi;
                        if (j == 3) e = e_rho;
                        dv[q][j] = fma(cv, dvdt, dv[q][j]) + e;
                    }
                    x[q] = x[q] + fma(sq, z1, fma(Real(-0.5), vdt, rdt));
                    v[q] = v[q] + fma(xi * sq, w, fma(-kappa, vdt, kthdt));
                }
            }
            if (g < pb.n_groups && gseg[g] == s) {
                Real S[PPT];
#pragma unroll
                for (int q = 0; q < PPT; ++q) S[q] = S0 * exp_r<Real>(x[q]);
                for (int i = gbeg[g]; i < gbeg[g + 1]; ++i) {
                    Real vals[1 + kJacM];
#pragma unroll
                    for (int k = 0; k <= kJacM; ++k) vals[k] = Real(0);
#pragma unroll
                    for (int q = 0; q < PPT; ++q) {
                        const bool itm = active[q] && S[q] > strike[i];
                        vals[0] += itm ? S[q] - strike[i] : Real(0);
#pragma unroll
                        for (int j = 0; j < kJacM; ++j) vals[1 + j] += itm ? S[q] * dx[q][j] : Real(0);
                    }
                    warp_flush_n(wrow, i * (1 + kJacM), vals, lane);
                }
                ++g;
            }
        }
    }
    __syncthreads();
    double *o = out + ((size_t)t * bpt + blockIdx.x) * W;
    for (int q = threadIdx.x; q < W; q += blockDim.x) {
        double s = 0.0;
        for (int w2 = 0; w2 < kWarpsPerBlock; ++w2) s += wacc[w2 * W + q];
        o[q] = s;
    }
}

// (E y, J) of theta t from its bpt block sums, in caller instrument order.
__global__ void jacobian_finalize_kernel(const double *__restrict__ part, int n_theta, int bpt, int m,
                                         const double *__restrict__ disc, const int *__restrict__ perm,
                                         double inv_n, double *Ey_out, double *J_out) {
    const int W = (1 + kJacM) * m;
    const uint64_t total = (uint64_t)n_theta * W;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const int t = (int)(q / W);
        const int r = (int)(q - (uint64_t)t * W);
        const int i = r / (1 + kJacM), c = r - i * (1 + kJacM);
        double s = 0.0;
        for (int b = 0; b < bpt; ++b) s += part[((size_t)t * bpt + b) * W + r];
        const double val = disc[i] * s * inv_n;
        const int ci = perm[i];
        if (c == 0) {
            if (Ey_out) Ey_out[(size_t)t * m + ci] = val;
        } else {
            J_out[((size_t)t * m + ci) * kJacM + (c - 1)] = val;
        }
    }
}

size_t jacobian_smem_bytes(int m, int n_groups, int precision) {
    const size_t real = precision == 0 ? 8 : 4;
    size_t o = align_up((size_t)m * real, 16);
    o = align_up(o + (size_t)(2 * n_groups + 1) * 4, 16);
    return o + (size_t)kWarpsPerBlock * (1 + kJacM) * m * 8;
}

// Paths per thread of the forward-mode kernel: two independent recursions in
// FP32 (as the path sweeps), one in FP64.
int jacobian_ppt(int precision) { return precision == 0 ? 1 : 2; }

const void *jacobian_kernel(int precision) {
    return precision == 0 ? (const void *)heston_jacobian_kernel<double, 1>
                          : (const void *)heston_jacobian_kernel<float, 2>;
}

cudaError_t launch_jacobian(const DevProblem &pb, int precision, const double *thetas, const double *strikes_t,
                            int n_theta, uint64_t seed, uint64_t path0, uint64_t n_paths, int bpt, size_t smem,
                            double *part, const double *disc, const int *perm, double *Ey_out,
                            double *J_out, cudaStream_t st) {
    const void *fn = jacobian_kernel(precision);
    const RoundKeys rk = philox_round_keys(seed);
    void *args[] = {(void *)&pb, (void *)&thetas, (void *)&strikes_t, (void *)&rk, (void *)&path0,
                    (void *)&n_paths, (void *)&bpt, (void *)&part};
    cudaError_t e = cudaLaunchKernel(fn, dim3(bpt, n_theta), dim3(kBlock), args, smem, st);
    if (e != cudaSuccess) return e;
    const uint64_t total = (uint64_t)n_theta * (1 + kJacM) * pb.m;
    int grid = (int)((total + 255) / 256);
    if (grid > 65536) grid = 65536;
    jacobian_finalize_kernel<<<grid, 256, 0, st>>>(part, n_theta, bpt, pb.m, disc, perm, 1.0 / (double)n_paths,
                                                  Ey_out, J_out);
    return cudaGetLastError();
}

// G and its gradient from E y and the Jacobian of one parameter vector (the
// gradient identity with the expectation taken per instrument first):
// lambda_i = E y_i - C_i, G = 1/2 sum_i lambda_i^2 (eq. 241118A),
// dG/dtheta_j = sum_i lambda_i dE y_i/dtheta_j.  One warp; each sum runs over
// i in order.
__global__ void tangent_finalize_kernel(const double *__restrict__ Ey, const double *__restrict__ J,
                                        const double *__restrict__ C, int m, double *G_out, double *grad_out) {
    const int j = threadIdx.x;
    if (j < kJacM) {
        double g = 0.0;
        for (int i = 0; i < m; ++i) g += (Ey[i] - C[i]) * J[(size_t)i * kJacM + j];
        grad_out[j] = g;
    } else if (j == kJacM) {
        double G = 0.0;
        for (int i = 0; i < m; ++i) {
            const double l = Ey[i] - C[i];
            G += l * l;
        }
        *G_out = 0.5 * G;
    }
}

cudaError_t launch_tangent_finalize(const double *Ey, const double *J, const double *C, int m, double *G_out,
                                    double *grad_out, cudaStream_t st) {
    tangent_finalize_kernel<<<1, kWarp, 0, st>>>(Ey, J, C, m, G_out, grad_out);
    return cudaGetLastError();
}

}  // namespace mcaad
