/*
 * mcaad_oracle.c -- plain, slow FP64 CPU oracle for the value and adjoint
 * gradient of the calibration objective G = 1/2 sum_i (E y_i - C_i)^2
 * (Goloubentsev & Lakshtanov, arXiv 1901.04200, eq. 241118A).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA library.
 *
 * What it computes, in the paper's order:
 *   forward algorithm F (paper, definition of F: M parameters plus N random
 *     variables -> m payoffs of one path) for three SDE discretisations
 *     (paper, Heston SLV model paragraph: an Euler scheme):
 *       GBM with piecewise-constant volatility (log-Euler),
 *       Heston with full-truncation Euler,
 *       local volatility on a bilinear node surface (log-Euler),
 *       Heston stochastic local volatility (the paper's test model: the
 *       Heston variance process times a leverage surface L(t, S) on fixed
 *       nodes, interpolated bilinearly; full-truncation Euler);
 *     every state of a path is stored (no checkpointing);
 *   Monte Carlo mean E y_i = (1/P) sum_p y_i(omega_p) (paper, Monte-Carlo
 *     remarks);
 *   lambda_i = E y_i - C_i and G (eq. 241118A; two-step algorithm, step 2);
 *   per path, the reverse algorithm R seeded with lambda (eq. 0711A), written
 *     by hand backwards over the stored states, and the sum over paths
 *     (two-step algorithm, steps 2 and 3; the gradient identity
 *     dG/dx_j = E(sum_i (E y_i - C_i) dy_i/dx_j)).
 *
 * Random numbers (the paper names no generator): Philox-4x32-10 from
 * Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3"
 * (SC'11), and the Box-Muller transform.  Normal j of global path p comes
 * from the Philox block with counter (j>>2 as a 64-bit number in words 0-1,
 * p as a 64-bit number in words 2-3) and key (seed low word, seed high
 * word).  Block words (o0,o1) make normals j&3 = 0,1 and (o2,o3) make 2,3:
 *   u(w) = ((w >> 9) + 0.5) * 2^-23,  rad = sqrt(-2 ln u(o_{2q})),
 *   z_{2q} = rad cos(2 pi u(o_{2q+1})),  z_{2q+1} = rad sin(2 pi u(o_{2q+1})).
 *
 * Sums over paths run in fixed chunks of ORC_CHUNK paths, each summed in path
 * order; chunk sums are added in chunk order, so results do not depend on the
 * number of threads.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "mcaad_oracle.h"

#define ORC_CHUNK 1024

static const double ORC_TWO_PI = 6.283185307179586476925286766559;

/* ---------------------------------------------------------------- Philox */

/* One Philox-4x32-10 block (SC'11: ten rounds of the 4x32 S-box with
 * multipliers 0xD2511F53, 0xCD9E8D57 and the Weyl key schedule
 * 0x9E3779B9, 0xBB67AE85, the key being bumped between rounds). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox_fill(uint64_t seed, uint64_t path0, uint32_t n_paths, uint32_t n_calls,
                     uint32_t *out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t i = 0; i < n_paths; ++i) {
        uint64_t p = path0 + i;
        for (uint32_t c = 0; c < n_calls; ++c) {
            uint32_t ctr[4] = {c, 0u, (uint32_t)p, (uint32_t)(p >> 32)};
            orc_philox4x32_10(ctr, key, out + ((size_t)i * n_calls + c) * 4);
        }
    }
}

double orc_uniform(uint32_t w)
{
    return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Normal number j of global path p (the counter layout in the file header). */
double orc_normal(uint64_t seed, uint64_t p, uint64_t j)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t call = j >> 2;
    uint32_t ctr[4] = {(uint32_t)call, (uint32_t)(call >> 32), (uint32_t)p, (uint32_t)(p >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    int q = (int)((j & 3) >> 1);
    double ua = orc_uniform(o[2 * q]);
    double ub = orc_uniform(o[2 * q + 1]);
    double rad = sqrt(-2.0 * log(ua));
    return (j & 1) ? rad * sin(ORC_TWO_PI * ub) : rad * cos(ORC_TWO_PI * ub);
}

void orc_normals_fill(uint64_t seed, uint64_t path0, uint32_t n_paths, uint32_t n_per_path,
                      double *out)
{
    for (uint32_t i = 0; i < n_paths; ++i)
        for (uint32_t j = 0; j < n_per_path; ++j)
            out[(size_t)i * n_per_path + j] = orc_normal(seed, path0 + i, j);
}

/* ------------------------------------------------------- problem helpers */

static int has_variance(const orc_problem *pb)
{
    return pb->kind == ORC_HESTON_FT || pb->kind == ORC_HESTON_SLV;
}
int orc_state_dim(const orc_problem *pb) { return has_variance(pb) ? 2 : 1; }
int orc_normals_per_step(const orc_problem *pb) { return has_variance(pb) ? 2 : 1; }

int orc_n_params(const orc_problem *pb)
{
    switch (pb->kind) {
    case ORC_GBM_PWC: return pb->n_buckets;
    case ORC_HESTON_FT: return 5;
    case ORC_LV_BILINEAR: return pb->nt * pb->nx;
    case ORC_HESTON_SLV: return 5 + pb->nt * pb->nx;
    }
    return -1;
}

/* The last step any payoff needs: steps after it change no y_i. */
int orc_last_step(const orc_problem *pb)
{
    int n = 0;
    for (int i = 0; i < pb->m; ++i)
        if (pb->mat_step[i] > n) n = pb->mat_step[i];
    return n;
}

int orc_check(const orc_problem *pb, const double *theta)
{
    if (pb->kind < 0 || pb->kind > 3) return ORC_ERR;
    if (pb->m < 1 || pb->n_steps < 1 || !(pb->dt > 0.0)) return ORC_ERR;
    for (int i = 0; i < pb->m; ++i)
        if (pb->mat_step[i] < 1 || pb->mat_step[i] > pb->n_steps) return ORC_ERR;
    if (pb->kind == ORC_GBM_PWC) {
        if (pb->n_buckets < 1) return ORC_ERR;
        for (int b = 0; b < pb->n_buckets; ++b) {
            int prev = b ? pb->bucket_end[b - 1] : 0;
            if (pb->bucket_end[b] <= prev) return ORC_ERR;
        }
        if (pb->bucket_end[pb->n_buckets - 1] < orc_last_step(pb)) return ORC_ERR;
    }
    if (has_variance(pb) && theta) {
        if (!(fabs(theta[3]) < 1.0)) return ORC_ERR;
    }
    if (pb->kind == ORC_LV_BILINEAR || pb->kind == ORC_HESTON_SLV) {
        if (pb->nt < 2 || pb->nx < 2 || !(pb->t_max > 0.0) || !(pb->x_hi > pb->x_lo)) return ORC_ERR;
    }
    return ORC_OK;
}

/* Normal number j of path p: from the caller's table when it gives one,
 * otherwise from Philox. */
static double path_normal(const orc_problem *pb, uint64_t p, uint64_t j)
{
    if (pb->normals) {
        size_t per_path = (size_t)pb->n_steps * orc_normals_per_step(pb);
        return pb->normals[(size_t)(p - pb->normals_path0) * per_path + j];
    }
    return orc_normal(pb->seed, p, j);
}

/* GBM bucket of step n: the first bucket whose end step exceeds n. */
static int gbm_bucket(const orc_problem *pb, int n)
{
    int b = 0;
    while (n >= pb->bucket_end[b]) ++b;
    return b;
}

/* Bilinear local volatility with flat extrapolation; also returns the four
 * node indices and weights, and d sigma / d x (zero where x is clamped). */
typedef struct {
    double sigma, dsdx;
    int node[4];
    double wgt[4];
} lv_eval;

static lv_eval lv_sigma(const orc_problem *pb, const double *theta, int n, double x)
{
    lv_eval e;
    double ht = pb->t_max / (double)(pb->nt - 1);
    double hx = (pb->x_hi - pb->x_lo) / (double)(pb->nx - 1);
    double ut = ((double)n * pb->dt) / ht;
    int jt = (int)floor(ut);
    if (jt < 0) jt = 0;
    if (jt > pb->nt - 2) jt = pb->nt - 2;
    double a = ut - (double)jt;
    if (a < 0.0) a = 0.0;
    if (a > 1.0) a = 1.0;
    double ux = (x - pb->x_lo) / hx;
    double fl = floor(ux);
    int c;
    if (fl < 0.0) c = 0;
    else if (fl > (double)(pb->nx - 2)) c = pb->nx - 2;
    else c = (int)fl;
    double b = ux - (double)c;
    int inside = 1;
    if (b < 0.0) { b = 0.0; inside = 0; }
    if (b > 1.0) { b = 1.0; inside = 0; }
    int nx = pb->nx;
    double s00 = theta[jt * nx + c], s01 = theta[jt * nx + c + 1];
    double s10 = theta[(jt + 1) * nx + c], s11 = theta[(jt + 1) * nx + c + 1];
    e.sigma = (1.0 - a) * ((1.0 - b) * s00 + b * s01) + a * ((1.0 - b) * s10 + b * s11);
    e.dsdx = inside ? ((1.0 - a) * (s01 - s00) + a * (s11 - s10)) / hx : 0.0;
    e.node[0] = jt * nx + c;            e.wgt[0] = (1.0 - a) * (1.0 - b);
    e.node[1] = jt * nx + c + 1;        e.wgt[1] = (1.0 - a) * b;
    e.node[2] = (jt + 1) * nx + c;      e.wgt[2] = a * (1.0 - b);
    e.node[3] = (jt + 1) * nx + c + 1;  e.wgt[3] = a * b;
    return e;
}

/* --------------------------------------------------- forward algorithm F */

/* One path of F.  states: [(n_last+1) * state_dim], state after n steps at
 * row n (x = ln(S/S0), and v for Heston); z: [n_last * normals_per_step];
 * y: [m] discounted payoffs.  Returns ORC_OK. */
int orc_path_forward(const orc_problem *pb, const double *theta, uint64_t p,
                     double *states, double *z, double *y)
{
    int nl = orc_last_step(pb);
    int sd = orc_state_dim(pb), dz = orc_normals_per_step(pb);
    double dt = pb->dt, sdt = sqrt(pb->dt), r = pb->r;
    states[0] = 0.0;
    if (has_variance(pb)) states[1] = theta[4];
    for (int n = 0; n < nl; ++n) {
        for (int c = 0; c < dz; ++c) z[n * dz + c] = path_normal(pb, p, (uint64_t)n * dz + c);
        const double *s = states + (size_t)n * sd;
        double *s1 = states + (size_t)(n + 1) * sd;
        if (pb->kind == ORC_GBM_PWC) {
            double vol = theta[gbm_bucket(pb, n)];
            s1[0] = s[0] + (r - 0.5 * vol * vol) * dt + vol * sdt * z[n];
        } else if (pb->kind == ORC_HESTON_FT) {
            double kappa = theta[0], th = theta[1], xi = theta[2], rho = theta[3];
            double x = s[0], v = s[1];
            double vp = v > 0.0 ? v : 0.0;
            double sq = sqrt(vp * dt);
            double z1 = z[2 * n], z2 = z[2 * n + 1];
            double w = rho * z1 + sqrt(1.0 - rho * rho) * z2;
            s1[0] = x + (r - 0.5 * vp) * dt + sq * z1;
            s1[1] = v + kappa * (th - vp) * dt + xi * sq * w;
        } else if (pb->kind == ORC_HESTON_SLV) {
            double kappa = theta[0], th = theta[1], xi = theta[2], rho = theta[3];
            double x = s[0], v = s[1];
            double vp = v > 0.0 ? v : 0.0;
            double sq = sqrt(vp * dt);
            double lev = lv_sigma(pb, theta + 5, n, x).sigma;
            double z1 = z[2 * n], z2 = z[2 * n + 1];
            double w = rho * z1 + sqrt(1.0 - rho * rho) * z2;
            s1[0] = x + (r - 0.5 * lev * lev * vp) * dt + lev * sq * z1;
            s1[1] = v + kappa * (th - vp) * dt + xi * sq * w;
        } else {
            lv_eval e = lv_sigma(pb, theta, n, s[0]);
            s1[0] = s[0] + (r - 0.5 * e.sigma * e.sigma) * dt + e.sigma * sdt * z[n];
        }
    }
    for (int i = 0; i < pb->m; ++i) {
        int ni = pb->mat_step[i];
        double S = pb->S0 * exp(states[(size_t)ni * sd]);
        double disc = exp(-r * (double)ni * dt);
        y[i] = disc * (S > pb->K[i] ? S - pb->K[i] : 0.0);
    }
    return ORC_OK;
}

/* ---------------------------------------------------- reverse algorithm R */

/* One path of R (eq. 0711A with seed lambda): g[j] = sum_i lambda_i dy_i/dtheta_j,
 * by hand backwards over the states F stored.  Kink conventions: the call
 * payoff has derivative 1{S > K}; max(v, 0) has derivative 1{v > 0}; the
 * local-vol surface has d sigma/dx = 0 where x is clamped. */
int orc_path_adjoint(const orc_problem *pb, const double *theta, const double *states,
                     const double *z, const double *lambda, double *g)
{
    int nl = orc_last_step(pb);
    int sd = orc_state_dim(pb);
    int M = orc_n_params(pb);
    double dt = pb->dt, sdt = sqrt(pb->dt), r = pb->r;
    for (int j = 0; j < M; ++j) g[j] = 0.0;
    double xb = 0.0, vb = 0.0; /* adjoints of the state after step n */
    for (int n = nl; n >= 0; --n) {
        /* payoffs read the state after n steps */
        for (int i = 0; i < pb->m; ++i) {
            if (pb->mat_step[i] != n) continue;
            double S = pb->S0 * exp(states[(size_t)n * sd]);
            double disc = exp(-r * (double)n * dt);
            if (S > pb->K[i]) xb += lambda[i] * disc * S;
        }
        if (n == 0) break;
        int k = n - 1; /* step k maps state k to state n */
        const double *s = states + (size_t)k * sd;
        if (pb->kind == ORC_GBM_PWC) {
            int b = gbm_bucket(pb, k);
            double vol = theta[b];
            g[b] += xb * (-vol * dt + sdt * z[k]);
            /* x_k enters x_n with coefficient 1 */
        } else if (pb->kind == ORC_HESTON_FT) {
            double kappa = theta[0], th = theta[1], xi = theta[2], rho = theta[3];
            double v = s[1];
            double vp = v > 0.0 ? v : 0.0;
            double sq = sqrt(vp * dt);
            double z1 = z[2 * k], z2 = z[2 * k + 1];
            double rhob = sqrt(1.0 - rho * rho);
            double w = rho * z1 + rhob * z2;
            g[0] += vb * (th - vp) * dt;
            g[1] += vb * kappa * dt;
            g[2] += vb * sq * w;
            g[3] += vb * xi * sq * (z1 - rho / rhob * z2);
            double vpb = xb * (-0.5 * dt) + vb * (-kappa * dt);
            if (vp > 0.0) vpb += (xb * z1 + vb * xi * w) * dt / (2.0 * sq);
            double vb_new = vb + (v > 0.0 ? vpb : 0.0);
            vb = vb_new;
            /* xb unchanged: x_k enters x_n with coefficient 1 */
        } else if (pb->kind == ORC_HESTON_SLV) {
            double kappa = theta[0], th = theta[1], xi = theta[2], rho = theta[3];
            double v = s[1];
            double vp = v > 0.0 ? v : 0.0;
            double sq = sqrt(vp * dt);
            lv_eval e = lv_sigma(pb, theta + 5, k, s[0]);
            double lev = e.sigma;
            double z1 = z[2 * k], z2 = z[2 * k + 1];
            double rhob = sqrt(1.0 - rho * rho);
            double w = rho * z1 + rhob * z2;
            /* leverage: x_n depends on lev through -lev^2 vp dt / 2 + lev sq z1 */
            double levb = xb * (-lev * vp * dt + sq * z1);
            for (int q = 0; q < 4; ++q) g[5 + e.node[q]] += levb * e.wgt[q];
            g[0] += vb * (th - vp) * dt;
            g[1] += vb * kappa * dt;
            g[2] += vb * sq * w;
            g[3] += vb * xi * sq * (z1 - rho / rhob * z2);
            double vpb = xb * (-0.5 * lev * lev * dt) + vb * (-kappa * dt);
            if (vp > 0.0) vpb += (xb * lev * z1 + vb * xi * w) * dt / (2.0 * sq);
            vb = vb + (v > 0.0 ? vpb : 0.0);
            xb = xb + levb * e.dsdx;
        } else {
            lv_eval e = lv_sigma(pb, theta, k, s[0]);
            double sb = xb * (-e.sigma * dt + sdt * z[k]);
            for (int q = 0; q < 4; ++q) g[e.node[q]] += sb * e.wgt[q];
            xb = xb + sb * e.dsdx;
        }
    }
    if (has_variance(pb)) g[4] += vb;
    return ORC_OK;
}

/* ---------------------------------------------------- path-sum machinery */

typedef struct {
    const orc_problem *pb;
    const double *theta;
    const double *lambda; /* NULL: forward pass (sum y); else adjoint pass (sum g) */
    uint64_t path0, n_paths;
    int width;            /* m or M */
    double *chunk_sums;   /* [n_chunks][width] */
    uint64_t n_chunks;
    uint64_t next_chunk;
    pthread_mutex_t lock;
} sum_job;

static void *sum_worker(void *arg)
{
    sum_job *jb = (sum_job *)arg;
    const orc_problem *pb = jb->pb;
    int nl = orc_last_step(pb);
    int sd = orc_state_dim(pb), dz = orc_normals_per_step(pb);
    int m = pb->m, M = orc_n_params(pb);
    double *states = (double *)malloc(sizeof(double) * (size_t)(nl + 1) * sd);
    double *z = (double *)malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1) * dz);
    double *y = (double *)malloc(sizeof(double) * (size_t)m);
    double *g = (double *)malloc(sizeof(double) * (size_t)M);
    for (;;) {
        pthread_mutex_lock(&jb->lock);
        uint64_t ch = jb->next_chunk++;
        pthread_mutex_unlock(&jb->lock);
        if (ch >= jb->n_chunks) break;
        double *acc = jb->chunk_sums + ch * (uint64_t)jb->width;
        for (int j = 0; j < jb->width; ++j) acc[j] = 0.0;
        uint64_t a = ch * ORC_CHUNK;
        uint64_t b = a + ORC_CHUNK;
        if (b > jb->n_paths) b = jb->n_paths;
        for (uint64_t q = a; q < b; ++q) {
            uint64_t p = jb->path0 + q;
            orc_path_forward(pb, jb->theta, p, states, z, y);
            if (!jb->lambda) {
                for (int i = 0; i < m; ++i) acc[i] += y[i];
            } else {
                orc_path_adjoint(pb, jb->theta, states, z, jb->lambda, g);
                for (int j = 0; j < M; ++j) acc[j] += g[j];
            }
        }
    }
    free(states); free(z); free(y); free(g);
    return NULL;
}

/* Mean over paths [path0, path0+n_paths) of y (lambda == NULL) or of the
 * per-path R result g (lambda given); out has width m or M. */
static int path_mean(const orc_problem *pb, const double *theta, const double *lambda,
                     uint64_t path0, uint64_t n_paths, int n_threads, double *out)
{
    int width = lambda ? orc_n_params(pb) : pb->m;
    sum_job jb;
    memset(&jb, 0, sizeof(jb));
    jb.pb = pb; jb.theta = theta; jb.lambda = lambda;
    jb.path0 = path0; jb.n_paths = n_paths; jb.width = width;
    jb.n_chunks = (n_paths + ORC_CHUNK - 1) / ORC_CHUNK;
    jb.chunk_sums = (double *)calloc((size_t)(jb.n_chunks ? jb.n_chunks : 1) * width, sizeof(double));
    if (!jb.chunk_sums) return ORC_ERR;
    pthread_mutex_init(&jb.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if ((uint64_t)n_threads > jb.n_chunks) n_threads = (int)(jb.n_chunks ? jb.n_chunks : 1);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, sum_worker, &jb);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&jb.lock);
    for (int j = 0; j < width; ++j) {
        double s = 0.0;
        for (uint64_t ch = 0; ch < jb.n_chunks; ++ch) s += jb.chunk_sums[ch * width + j];
        out[j] = s / (double)n_paths;
    }
    free(jb.chunk_sums);
    return ORC_OK;
}

/* ------------------------------------------------------------ public API */

int orc_forward(const orc_problem *pb, const double *theta, uint64_t path0, uint64_t n_paths,
                int n_threads, double *Ey)
{
    if (orc_check(pb, theta) || n_paths == 0) return ORC_ERR;
    return path_mean(pb, theta, NULL, path0, n_paths, n_threads, Ey);
}

int orc_vjp(const orc_problem *pb, const double *theta, const double *ybar, uint64_t path0,
            uint64_t n_paths, int n_threads, double *theta_bar)
{
    if (orc_check(pb, theta) || n_paths == 0) return ORC_ERR;
    return path_mean(pb, theta, ybar, path0, n_paths, n_threads, theta_bar);
}

/* The two-step algorithm: step 1 gives E y; lambda = E y - C and G; steps 2-3
 * give grad G = (1/P) sum_p sum_i lambda_i dy_i(omega_p)/dtheta. */
int orc_value_and_grad(const orc_problem *pb, const double *theta, const double *C,
                       uint64_t path0, uint64_t n_paths, int n_threads,
                       double *Ey, double *G, double *grad)
{
    if (orc_check(pb, theta) || n_paths == 0) return ORC_ERR;
    int m = pb->m;
    if (path_mean(pb, theta, NULL, path0, n_paths, n_threads, Ey)) return ORC_ERR;
    double *lambda = (double *)malloc(sizeof(double) * (size_t)m);
    double g2 = 0.0;
    for (int i = 0; i < m; ++i) {
        lambda[i] = Ey[i] - C[i];
        g2 += lambda[i] * lambda[i];
    }
    *G = 0.5 * g2;
    int rc = path_mean(pb, theta, lambda, path0, n_paths, n_threads, grad);
    free(lambda);
    return rc;
}

/* State after `step` steps of each path in [path0, path0+n_paths): out is
 * [n_paths][state_dim] (x = ln(S/S0), and v for the variance models).  Plain
 * read-out of F's stored states, for pins of the one-step dynamics. */
typedef struct {
    const orc_problem *pb;
    const double *theta;
    uint64_t path0, n_paths;
    int step;
    double *out;
    uint64_t next;
    pthread_mutex_t lock;
} states_job;

static void *states_worker(void *arg)
{
    states_job *jb = (states_job *)arg;
    const orc_problem *pb = jb->pb;
    int nl = orc_last_step(pb);
    int sd = orc_state_dim(pb), dz = orc_normals_per_step(pb);
    double *states = (double *)malloc(sizeof(double) * (size_t)(nl + 1) * sd);
    double *z = (double *)malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1) * dz);
    double *y = (double *)malloc(sizeof(double) * (size_t)pb->m);
    for (;;) {
        pthread_mutex_lock(&jb->lock);
        uint64_t ch = jb->next++;
        pthread_mutex_unlock(&jb->lock);
        uint64_t a = ch * ORC_CHUNK;
        if (a >= jb->n_paths) break;
        uint64_t b = a + ORC_CHUNK;
        if (b > jb->n_paths) b = jb->n_paths;
        for (uint64_t q = a; q < b; ++q) {
            orc_path_forward(pb, jb->theta, jb->path0 + q, states, z, y);
            for (int c = 0; c < sd; ++c)
                jb->out[q * (uint64_t)sd + c] = states[(size_t)jb->step * sd + c];
        }
    }
    free(states); free(z); free(y);
    return NULL;
}

int orc_states_at(const orc_problem *pb, const double *theta, uint64_t path0, uint64_t n_paths,
                  int step, int n_threads, double *out)
{
    if (orc_check(pb, theta) || n_paths == 0) return ORC_ERR;
    if (step < 0 || step > orc_last_step(pb)) return ORC_ERR;
    states_job jb;
    memset(&jb, 0, sizeof(jb));
    jb.pb = pb; jb.theta = theta; jb.path0 = path0; jb.n_paths = n_paths;
    jb.step = step; jb.out = out;
    pthread_mutex_init(&jb.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, states_worker, &jb);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&jb.lock);
    return ORC_OK;
}
