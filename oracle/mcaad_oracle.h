/*
 * mcaad_oracle.h -- FP64 CPU oracle for G = 1/2 sum_i (E y_i - C_i)^2 and its
 * gradient (arXiv 1901.04200, eq. 241118A and the two-step algorithm).
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; the CUDA library never includes or links it.
 */
#ifndef MCAAD_ORACLE_H
#define MCAAD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ERR = 1 };
enum { ORC_GBM_PWC = 0, ORC_HESTON_FT = 1, ORC_LV_BILINEAR = 2, ORC_HESTON_SLV = 3 };

/* One calibration problem.  All arrays are host memory owned by the caller.
 * State x = ln(S/S0) starts at 0; Heston's v starts at theta[4].
 *   GBM_PWC:      theta[b] = volatility of bucket b; step n lies in the first
 *                 bucket b with n < bucket_end[b].
 *   HESTON_FT:    theta = (kappa, theta_h, xi, rho, v0).
 *   LV_BILINEAR:  theta[j*nx + c] = sigma at time t_j = j*t_max/(nt-1) and
 *                 log-moneyness x_c = x_lo + c*(x_hi-x_lo)/(nx-1).
 *   HESTON_SLV:   theta = (kappa, theta_h, xi, rho, v0, L[0..nt*nx)) with the
 *                 leverage L on the same node grid as LV_BILINEAR.
 * Instrument i is a call with strike K[i] paying at step mat_step[i]
 * (time mat_step[i]*dt), discounted at rate r.
 * normals: optional [P][n_steps*normals_per_step] table for global paths
 * normals_path0 .. normals_path0+P-1; NULL means Philox with key = seed. */
typedef struct {
    int kind;
    double S0, r, dt;
    int n_steps;
    int n_buckets;
    const int *bucket_end;
    int nt, nx;
    double t_max, x_lo, x_hi;
    int m;
    const double *K;
    const int *mat_step;
    const double *normals;
    uint64_t normals_path0;
    uint64_t seed;
} orc_problem;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_philox_fill(uint64_t seed, uint64_t path0, uint32_t n_paths, uint32_t n_calls, uint32_t *out);
double orc_uniform(uint32_t w);
double orc_normal(uint64_t seed, uint64_t path, uint64_t j);
void orc_normals_fill(uint64_t seed, uint64_t path0, uint32_t n_paths, uint32_t n_per_path, double *out);

int orc_state_dim(const orc_problem *pb);
int orc_normals_per_step(const orc_problem *pb);
int orc_n_params(const orc_problem *pb);
int orc_last_step(const orc_problem *pb);
int orc_check(const orc_problem *pb, const double *theta);

int orc_path_forward(const orc_problem *pb, const double *theta, uint64_t p,
                     double *states, double *z, double *y);
int orc_path_adjoint(const orc_problem *pb, const double *theta, const double *states,
                     const double *z, const double *lambda, double *g);

int orc_forward(const orc_problem *pb, const double *theta, uint64_t path0, uint64_t n_paths,
                int n_threads, double *Ey);
int orc_vjp(const orc_problem *pb, const double *theta, const double *ybar, uint64_t path0,
            uint64_t n_paths, int n_threads, double *theta_bar);
int orc_value_and_grad(const orc_problem *pb, const double *theta, const double *C,
                       uint64_t path0, uint64_t n_paths, int n_threads,
                       double *Ey, double *G, double *grad);
int orc_states_at(const orc_problem *pb, const double *theta, uint64_t path0, uint64_t n_paths,
                  int step, int n_threads, double *out);

#ifdef __cplusplus
}
#endif
#endif
