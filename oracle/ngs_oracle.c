/*
 * NanoGS FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (tests, smoke check and
 * the benchmark's CPU-baseline leg).  Plain double-precision loops that follow
 * the method's definitions in the paper's order; no blocking or fusion.
 *
 * Sections cited: Sec. 3.1 (kNN merge graph), Sec. 3.2 (merge cost,
 * Eqs. unnormalized_splats, norm_mixture, Dmerge_main, Equ:cost), Sec. 3.3
 * (MPMM, Eqs. vm_weights, vm_cov, vm_alpha), Sec. 3.4 (progressive batched
 * merging), App. A (Monte Carlo estimator Eq. mc_kl_estimator and the closed
 * Gaussian I-divergence), App. B Algorithm 1 (the driver loop).
 *
 * Readings where the paper is silent:
 *   - quaternion order (w,x,y,z), normalised before use;
 *   - median = lower median sorted[(n-1)/2];
 *   - ties: kNN by (d^2, index), greedy by (cost, lo, hi), NaN cost last;
 *   - sampling: x = mu_c + Sigma_c^{1/2} z (symmetric square root), common z
 *     per pass from SplitMix64 + Box-Muller; mode 0 integrates the component
 *     draw out (pi g(x_i) + (1-pi) g(x_j)), mode 1 draws it with u < pi;
 *   - mode 2 keeps mode 0's draws but replaces the sampled -log q_m(x) by its
 *     exact mean under p~, 1/2 log det(2 pi Sigma_m) + 3/2 (q_m carries p~'s
 *     own mean and covariance, App. A), so only the entropy of p~ is sampled;
 *   - mode 3 is the MSE surrogate of the Sec. 4 ablation, chosen here as
 *     |mu_i - mu_j|^2 + ||Sigma_i - Sigma_j||_F^2 (deterministic);
 *   - merged splat at slot min(i,j), stable order otherwise;
 *   - merged covariance -> (log-scale, quaternion) by cyclic Jacobi, eigen-
 *     values floored at eig_floor, canonical eigenvector signs, w >= 0;
 *   - merged opacity written as a logit in the log-transmittance form.
 */
#include "ngs_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559
#define LOG_2PI 1.8378770664093454835606594728112

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the later parallel loops started from the calling thread (t > 0);
   returns the count in effect.  Timing only: results do not depend on it. */
int orc_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#endif
    return orc_num_threads();
}

/* softplus(x) = log(1 + e^x), written to avoid overflow. */
static double softplus(double x) {
    return x > 0 ? x + log1p(exp(-x)) : log1p(exp(x));
}

/* ------------------------------------------------------------------------ */
/* Conversions (3DGS parameterisation).                                       */

void orc_quat_to_R(const double *q, double *R) {
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* One splat as a Gaussian: Sigma = R diag(s^2) R^T, mass w (Eq. unnormalized_splats). */
typedef struct {
    double mu[3], R[9], s[3], Sig[9], logdet, logw, logit;
} gauss_t;

static void splat_gauss(const double *xyz, const double *ls, const double *rot, double logit,
                        gauss_t *g) {
    for (int a = 0; a < 3; a++) g->mu[a] = xyz[a];
    orc_quat_to_R(rot, g->R);
    for (int a = 0; a < 3; a++) g->s[a] = exp(ls[a]);
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += g->R[r * 3 + k] * g->s[k] * g->s[k] * g->R[c * 3 + k];
            g->Sig[r * 3 + c] = acc;
        }
    g->logdet = 2.0 * (ls[0] + ls[1] + ls[2]);
    /* log w = 1.5 log(2 pi) + log alpha + sum_k log s_k, log alpha = -softplus(-logit) */
    g->logw = 1.5 * LOG_2PI - softplus(-logit) + ls[0] + ls[1] + ls[2];
    g->logit = logit;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: opacity pre-filter.                                           */

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

int64_t orc_prefilter(int64_t n, const double *logit, double tau, uint8_t *keep) {
    if (n <= 0) return 0;
    double *alpha = (double *)malloc(sizeof(double) * n);
    double *sorted = (double *)malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; i++) alpha[i] = 1.0 / (1.0 + exp(-logit[i]));
    memcpy(sorted, alpha, sizeof(double) * n);
    qsort(sorted, n, sizeof(double), cmp_double);
    double med = sorted[(n - 1) / 2];
    double taup = tau < med ? tau : med;
    int64_t kept = 0;
    for (int64_t i = 0; i < n; i++) {
        keep[i] = alpha[i] >= taup;
        kept += keep[i];
    }
    free(alpha);
    free(sorted);
    return kept;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: k nearest neighbours.                                            */

typedef struct { double d2; int32_t j; } cand_t;

static int cand_less(const cand_t *a, const cand_t *b) {
    return a->d2 < b->d2 || (a->d2 == b->d2 && a->j < b->j);
}

static double dist2(const double *a, const double *b) {
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return (dx * dx + dy * dy) + dz * dz;
}

/* keep the kk smallest candidates, sorted ascending, by insertion */
static void topk_insert(cand_t *list, int *cnt, int kk, cand_t c) {
    if (*cnt == kk && !cand_less(&c, &list[kk - 1])) return;
    int p = *cnt < kk ? (*cnt)++ : kk - 1;
    while (p > 0 && cand_less(&c, &list[p - 1])) {
        list[p] = list[p - 1];
        p--;
    }
    list[p] = c;
}

static int k_effective(int64_t n, int k) {
    int ke = k < 1 ? 1 : k;
    if ((int64_t)ke > n - 1) ke = (int)(n - 1);
    return ke;
}

int orc_knn_brute_queries(int64_t n, const double *xyz, int k, int64_t nq,
                          const int64_t *queries, int32_t *nbr) {
    int ke = k_effective(n, k);
    if (ke <= 0) return 0;
#pragma omp parallel
    {
        cand_t *list = (cand_t *)malloc(sizeof(cand_t) * ke);
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < nq; t++) {
            int64_t i = queries ? queries[t] : t;
            int cnt = 0;
            for (int64_t j = 0; j < n; j++) {
                if (j == i) continue;
                cand_t c = {dist2(xyz + 3 * i, xyz + 3 * j), (int32_t)j};
                topk_insert(list, &cnt, ke, c);
            }
            for (int a = 0; a < ke; a++) nbr[t * ke + a] = list[a].j;
        }
        free(list);
    }
    return ke;
}

int orc_knn_brute(int64_t n, const double *xyz, int k, int32_t *nbr) {
    return orc_knn_brute_queries(n, xyz, k, n, NULL, nbr);
}

/* Uniform grid over the bounding box; each query scans cubic shells of cells
 * around its own cell until every point outside the scanned cube is strictly
 * farther than the current k-th candidate (then no outside point can enter or
 * tie).  Same output definition as the brute force. */
int orc_knn_grid(int64_t n, const double *xyz, int k, int32_t *nbr) {
    int ke = k_effective(n, k);
    if (ke <= 0) return 0;
    double lo[3], hi[3];
    for (int a = 0; a < 3; a++) { lo[a] = xyz[a]; hi[a] = xyz[a]; }
    for (int64_t i = 1; i < n; i++)
        for (int a = 0; a < 3; a++) {
            if (xyz[3 * i + a] < lo[a]) lo[a] = xyz[3 * i + a];
            if (xyz[3 * i + a] > hi[a]) hi[a] = xyz[3 * i + a];
        }
    double side = 0;
    for (int a = 0; a < 3; a++) if (hi[a] - lo[a] > side) side = hi[a] - lo[a];
    if (side <= 0) side = 1;
    int64_t G = (int64_t)ceil(cbrt((double)n / 2.0));
    if (G < 1) G = 1;
    if (G > 1024) G = 1024;
    double h = side / (double)G * (1.0 + 1e-12);
    int64_t ncell = G * G * G;
    int64_t *cstart = (int64_t *)calloc(ncell + 1, sizeof(int64_t));
    int64_t *pcell = (int64_t *)malloc(sizeof(int64_t) * n);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * n);
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (ncell + 1));
    for (int64_t i = 0; i < n; i++) {
        int64_t c[3];
        for (int a = 0; a < 3; a++) {
            c[a] = (int64_t)floor((xyz[3 * i + a] - lo[a]) / h);
            if (c[a] < 0) c[a] = 0;
            if (c[a] >= G) c[a] = G - 1;
        }
        pcell[i] = (c[0] * G + c[1]) * G + c[2];
        cstart[pcell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) cstart[c + 1] += cstart[c];
    memcpy(fill, cstart, sizeof(int64_t) * (ncell + 1));
    for (int64_t i = 0; i < n; i++) order[fill[pcell[i]]++] = (int32_t)i;
#pragma omp parallel
    {
        cand_t *list = (cand_t *)malloc(sizeof(cand_t) * ke);
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; i++) {
            const double *q = xyz + 3 * i;
            int64_t qc[3];
            for (int a = 0; a < 3; a++) {
                qc[a] = (int64_t)floor((q[a] - lo[a]) / h);
                if (qc[a] < 0) qc[a] = 0;
                if (qc[a] >= G) qc[a] = G - 1;
            }
            int cnt = 0;
            for (int64_t r = 0;; r++) {
                /* visit cells at Chebyshev distance exactly r from qc */
                for (int64_t cx = qc[0] - r; cx <= qc[0] + r; cx++) {
                    if (cx < 0 || cx >= G) continue;
                    for (int64_t cy = qc[1] - r; cy <= qc[1] + r; cy++) {
                        if (cy < 0 || cy >= G) continue;
                        for (int64_t cz = qc[2] - r; cz <= qc[2] + r; cz++) {
                            if (cz < 0 || cz >= G) continue;
                            int64_t ch = llabs(cx - qc[0]);
                            if (llabs(cy - qc[1]) > ch) ch = llabs(cy - qc[1]);
                            if (llabs(cz - qc[2]) > ch) ch = llabs(cz - qc[2]);
                            if (ch != r) continue;
                            int64_t cell = (cx * G + cy) * G + cz;
                            for (int64_t p = cstart[cell]; p < cstart[cell + 1]; p++) {
                                int32_t j = order[p];
                                if (j == i) continue;
                                cand_t c = {dist2(q, xyz + 3 * (int64_t)j), j};
                                topk_insert(list, &cnt, ke, c);
                            }
                        }
                    }
                }
                /* distance from q to the outside of the scanned cube; a face on
                 * the grid boundary has nothing beyond it */
                double g = INFINITY;
                int covers_all = 1;
                for (int a = 0; a < 3; a++) {
                    if (qc[a] - r > 0) {
                        double d = q[a] - (lo[a] + (double)(qc[a] - r) * h);
                        if (d < g) g = d;
                        covers_all = 0;
                    }
                    if (qc[a] + r < G - 1) {
                        double d = (lo[a] + (double)(qc[a] + r + 1) * h) - q[a];
                        if (d < g) g = d;
                        covers_all = 0;
                    }
                }
                if (covers_all) break;
                if (cnt == ke && list[ke - 1].d2 < g * g) break;
            }
            for (int a = 0; a < ke; a++) nbr[i * ke + a] = list[a].j;
        }
        free(list);
    }
    free(cstart); free(pcell); free(order); free(fill);
    return ke;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: undirected union of the directed kNN lists.                  */

static int cmp_edge64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

int64_t orc_union_edges(int64_t n, int k_eff, const int32_t *nbr, int32_t *lo, int32_t *hi) {
    int64_t m = n * (int64_t)k_eff;
    if (m <= 0) return 0;
    uint64_t *e = (uint64_t *)malloc(sizeof(uint64_t) * m);
    for (int64_t i = 0; i < n; i++)
        for (int a = 0; a < k_eff; a++) {
            uint64_t j = (uint64_t)nbr[i * k_eff + a];
            uint64_t u = (uint64_t)i < j ? (uint64_t)i : j, v = (uint64_t)i < j ? j : (uint64_t)i;
            e[i * k_eff + a] = (u << 32) | v;
        }
    qsort(e, m, sizeof(uint64_t), cmp_edge64);
    int64_t cnt = 0;
    for (int64_t t = 0; t < m; t++) {
        if (t > 0 && e[t] == e[t - 1]) continue;
        lo[cnt] = (int32_t)(e[t] >> 32);
        hi[cnt] = (int32_t)(e[t] & 0xffffffffu);
        cnt++;
    }
    free(e);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Common random numbers (App. A): SplitMix64 (Steele, Lea & Flood 2014) and  */
/* the Box-Muller transform (Box & Muller 1958).                              */

static uint64_t splitmix64(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform in (0, 1] from the top 53 bits */
static double uniform01(uint64_t *state) {
    return (double)((splitmix64(state) >> 11) + 1) * (1.0 / 9007199254740992.0);
}

void orc_mc_draws(uint64_t seed, uint32_t pass, int S, float *z, float *u) {
    uint64_t state = seed ^ ((uint64_t)pass * 0xD1B54A32D192ED03ULL);
    for (int s = 0; s < S; s++) {
        double u1 = uniform01(&state), u2 = uniform01(&state);
        double u3 = uniform01(&state), u4 = uniform01(&state);
        double r1 = sqrt(-2.0 * log(u1)), r2 = sqrt(-2.0 * log(u3));
        z[3 * s + 0] = (float)(r1 * cos(TWO_PI * u2));
        z[3 * s + 1] = (float)(r1 * sin(TWO_PI * u2));
        z[3 * s + 2] = (float)(r2 * cos(TWO_PI * u4));
        u[s] = (float)uniform01(&state);
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3 MPMM on moments.                                                  */

void orc_mpmm_moments(double wi, const double *mui, const double *Si, const double *fi,
                      double wj, const double *muj, const double *Sj, const double *fj, int F,
                      double *mum, double *Sm, double *fm) {
    double W = wi + wj;
    for (int a = 0; a < 3; a++) mum[a] = (wi * mui[a] + wj * muj[a]) / W;
    double di[3], dj[3];
    for (int a = 0; a < 3; a++) { di[a] = mui[a] - mum[a]; dj[a] = muj[a] - mum[a]; }
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++)
            Sm[r * 3 + c] = (wi * (Si[r * 3 + c] + di[r] * di[c]) +
                             wj * (Sj[r * 3 + c] + dj[r] * dj[c])) / W;
    if (fm)
        for (int t = 0; t < F; t++) fm[t] = (wi * fi[t] + wj * fj[t]) / W;
}

/* MPMM with the mass ratio given in log space: pi = w_i / W = sigmoid(log w_i
 * - log w_j).  Same equations as orc_mpmm_moments, without forming w (which
 * under/overflows for tiny splats). */
static void mpmm_pi(double pi, double pj, const gauss_t *gi, const gauss_t *gj,
                    double *mum, double *Sm) {
    for (int a = 0; a < 3; a++) mum[a] = pi * gi->mu[a] + pj * gj->mu[a];
    double di[3], dj[3];
    for (int a = 0; a < 3; a++) { di[a] = gi->mu[a] - mum[a]; dj[a] = gj->mu[a] - mum[a]; }
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++)
            Sm[r * 3 + c] = pi * (gi->Sig[r * 3 + c] + di[r] * di[c]) +
                            pj * (gj->Sig[r * 3 + c] + dj[r] * dj[c]);
}

static void mass_ratio(const gauss_t *gi, const gauss_t *gj, double *pi, double *pj,
                       double *logpi, double *logpj) {
    *logpi = -softplus(gj->logw - gi->logw);
    *logpj = -softplus(gi->logw - gj->logw);
    *pi = exp(*logpi);
    *pj = exp(*logpj);
}

/* ------------------------------------------------------------------------ */
/* Gaussian log densities (the -1.5 log 2 pi term cancels in every use).     */

/* h(x) = -1/2 log det Sigma - 1/2 (x-mu)^T Sigma^{-1} (x-mu), Sigma^{-1} applied
 * in the splat's own frame: y = diag(1/s) R^T (x - mu). */
static double h_splat(const gauss_t *g, const double *x) {
    double d[3] = {x[0] - g->mu[0], x[1] - g->mu[1], x[2] - g->mu[2]};
    double q = 0;
    for (int k = 0; k < 3; k++) {
        double y = (g->R[0 * 3 + k] * d[0] + g->R[1 * 3 + k] * d[1] + g->R[2 * 3 + k] * d[2]) / g->s[k];
        q += y * y;
    }
    return -0.5 * g->logdet - 0.5 * q;
}

/* Cholesky of a 3x3 SPD matrix (lower L, row-major); returns 0 if not SPD. */
static int chol3(const double *A, double *L) {
    memset(L, 0, sizeof(double) * 9);
    for (int j = 0; j < 3; j++) {
        double s = A[j * 3 + j];
        for (int k = 0; k < j; k++) s -= L[j * 3 + k] * L[j * 3 + k];
        if (!(s > 0)) return 0;
        L[j * 3 + j] = sqrt(s);
        for (int i = j + 1; i < 3; i++) {
            double t = A[i * 3 + j];
            for (int k = 0; k < j; k++) t -= L[i * 3 + k] * L[j * 3 + k];
            L[i * 3 + j] = t / L[j * 3 + j];
        }
    }
    return 1;
}

/* h for the merged Gaussian through its Cholesky factor: |L^{-1}(x-mu)|^2. */
static double h_chol(const double *mu, const double *L, double logdet, const double *x) {
    double d[3] = {x[0] - mu[0], x[1] - mu[1], x[2] - mu[2]};
    double y[3];
    for (int i = 0; i < 3; i++) {
        double t = d[i];
        for (int k = 0; k < i; k++) t -= L[i * 3 + k] * y[k];
        y[i] = t / L[i * 3 + i];
    }
    return -0.5 * logdet - 0.5 * (y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
}

static double logsumexp2(double a, double b) {
    double m = a > b ? a : b;
    if (m == -INFINITY) return -INFINITY;
    return m + log(exp(a - m) + exp(b - m));
}

/* x = mu + Sigma^{1/2} z with the symmetric square root R diag(s) R^T. */
static void sample_point(const gauss_t *g, const float *z, double *x) {
    double t[3];
    for (int k = 0; k < 3; k++)
        t[k] = g->s[k] * (g->R[0 * 3 + k] * z[0] + g->R[1 * 3 + k] * z[1] + g->R[2 * 3 + k] * z[2]);
    for (int a = 0; a < 3; a++)
        x[a] = g->mu[a] + g->R[a * 3 + 0] * t[0] + g->R[a * 3 + 1] * t[1] + g->R[a * 3 + 2] * t[2];
}

/* MSE geometric surrogate (the "w/o I-divergence" ablation of Sec. 4): squared
 * distance of the centres plus the squared Frobenius norm of the covariance
 * difference. */
static double dgeo_mse(const gauss_t *gi, const gauss_t *gj) {
    double r = 0;
    for (int a = 0; a < 3; a++) {
        double d = gi->mu[a] - gj->mu[a];
        r += d * d;
    }
    for (int t = 0; t < 9; t++) {
        double d = gi->Sig[t] - gj->Sig[t];
        r += d * d;
    }
    return r;
}

/* Eq. mc_kl_estimator for one pair: KL(p~_ij || q_m) estimated with S common
 * samples (modes 0-2), or the MSE surrogate (mode 3).  Returns +inf if the
 * merged covariance is not positive definite (modes 0-2). */
static double dgeo_gauss(const gauss_t *gi, const gauss_t *gj, int S, const float *z,
                         const float *u, int mode) {
    if (mode == 3) return dgeo_mse(gi, gj);
    double pi, pj, lpi, lpj;
    mass_ratio(gi, gj, &pi, &pj, &lpi, &lpj);
    double mum[3], Sm[9], L[9];
    mpmm_pi(pi, pj, gi, gj, mum, Sm);
    if (!chol3(Sm, L)) return INFINITY;
    double logdet_m = 2.0 * (log(L[0]) + log(L[4]) + log(L[8]));
    double acc = 0;
    for (int s = 0; s < S; s++) {
        const float *zs = z + 3 * s;
        double xi[3], xj[3];
        if (mode == 0 || mode == 2) {
            sample_point(gi, zs, xi);
            sample_point(gj, zs, xj);
            /* -E_p~[log q_m] in closed form: the expected Mahalanobis term of a
             * Gaussian under its own moments is 3 (three dimensions) */
            double hmi = mode == 0 ? h_chol(mum, L, logdet_m, xi) : -0.5 * logdet_m - 1.5;
            double hmj = mode == 0 ? h_chol(mum, L, logdet_m, xj) : -0.5 * logdet_m - 1.5;
            double gxi = logsumexp2(lpi + h_splat(gi, xi), lpj + h_splat(gj, xi)) - hmi;
            double gxj = logsumexp2(lpi + h_splat(gi, xj), lpj + h_splat(gj, xj)) - hmj;
            acc += pi * gxi + pj * gxj;
        } else {
            const gauss_t *gc = ((double)u[s] < pi) ? gi : gj;
            sample_point(gc, zs, xi);
            acc += logsumexp2(lpi + h_splat(gi, xi), lpj + h_splat(gj, xi)) -
                   h_chol(mum, L, logdet_m, xi);
        }
    }
    return acc / (double)S;
}

double orc_dgeo_pair(const double *xyz_i, const double *ls_i, const double *rot_i, double logit_i,
                     const double *xyz_j, const double *ls_j, const double *rot_j, double logit_j,
                     int S, const float *z, const float *u, int mode) {
    gauss_t gi, gj;
    splat_gauss(xyz_i, ls_i, rot_i, logit_i, &gi);
    splat_gauss(xyz_j, ls_j, rot_j, logit_j, &gj);
    return dgeo_gauss(&gi, &gj, S, z, u, mode);
}

void orc_edge_costs(int64_t n, const double *xyz, const double *log_scale, const double *rot,
                    const double *logit, const double *sh, int F,
                    int64_t m, const int32_t *lo, const int32_t *hi,
                    int S, const float *z, const float *u, int mode,
                    double lambda_geo, double lambda_app,
                    double *cost, double *dgeo, double *dapp) {
    (void)n;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        int64_t i = lo[e], j = hi[e];
        gauss_t gi, gj;
        splat_gauss(xyz + 3 * i, log_scale + 3 * i, rot + 4 * i, logit[i], &gi);
        splat_gauss(xyz + 3 * j, log_scale + 3 * j, rot + 4 * j, logit[j], &gj);
        double dg = dgeo_gauss(&gi, &gj, S, z, u, mode);
        double da = 0;
        for (int t = 0; t < F; t++) {
            double d = sh[i * F + t] - sh[j * F + t];
            da += d * d;
        }
        cost[e] = lambda_geo * dg + lambda_app * da;
        if (dgeo) dgeo[e] = dg;
        if (dapp) dapp[e] = da;
    }
}

/* ------------------------------------------------------------------------ */
/* Closed forms (App. A): KL between Gaussians and the I-divergence of two   */
/* unnormalised Gaussians.                                                    */

static int inv3(const double *A, double *Ai, double *det) {
    double d = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
               A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (d == 0) return 0;
    Ai[0] = (A[4] * A[8] - A[5] * A[7]) / d; Ai[1] = (A[2] * A[7] - A[1] * A[8]) / d;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) / d; Ai[3] = (A[5] * A[6] - A[3] * A[8]) / d;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) / d; Ai[5] = (A[2] * A[3] - A[0] * A[5]) / d;
    Ai[6] = (A[3] * A[7] - A[4] * A[6]) / d; Ai[7] = (A[1] * A[6] - A[0] * A[7]) / d;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) / d;
    *det = d;
    return 1;
}

double orc_kl_gauss(const double *mui, const double *Si, const double *muj, const double *Sj) {
    double Sji[9], detj, deti, tmp[9];
    if (!inv3(Sj, Sji, &detj) || !inv3(Si, tmp, &deti)) return NAN;
    double tr = 0;
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) tr += Sji[r * 3 + c] * Si[c * 3 + r];
    double d[3] = {muj[0] - mui[0], muj[1] - mui[1], muj[2] - mui[2]};
    double quad = 0;
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) quad += d[r] * Sji[r * 3 + c] * d[c];
    return 0.5 * (tr + quad - 3.0 + log(detj / deti));
}

double orc_idiv_gauss(double mi, const double *mui, const double *Si,
                      double mj, const double *muj, const double *Sj) {
    return mi * (log(mi / mj) + orc_kl_gauss(mui, Si, muj, Sj)) - mi + mj;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.4 / Algorithm 1: greedy disjoint pairs.                             */

typedef struct { double c; int32_t lo, hi; } ekey_t;

static int cmp_ekey(const void *a, const void *b) {
    const ekey_t *x = (const ekey_t *)a, *y = (const ekey_t *)b;
    if (x->c < y->c) return -1;
    if (x->c > y->c) return 1;
    if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
    if (x->hi != y->hi) return x->hi < y->hi ? -1 : 1;
    return 0;
}

int64_t orc_greedy(int64_t n, int64_t m, const int32_t *lo, const int32_t *hi,
                   const double *cost, int64_t P, int32_t *pair_lo, int32_t *pair_hi) {
    if (n <= 0 || m <= 0 || P <= 0) return 0;
    ekey_t *k = (ekey_t *)malloc(sizeof(ekey_t) * m);
    for (int64_t e = 0; e < m; e++) {
        double c = cost[e];
        if (isnan(c)) c = INFINITY; /* NaN ranks with +inf */
        if (c == 0) c = 0.0;        /* -0 ranks with +0 */
        k[e].c = c; k[e].lo = lo[e]; k[e].hi = hi[e];
    }
    qsort(k, m, sizeof(ekey_t), cmp_ekey);
    uint8_t *used = (uint8_t *)calloc(n, 1);
    int64_t cnt = 0;
    for (int64_t t = 0; t < m && cnt < P; t++) {
        if (used[k[t].lo] || used[k[t].hi]) continue;
        used[k[t].lo] = used[k[t].hi] = 1;
        pair_lo[cnt] = k[t].lo;
        pair_hi[cnt] = k[t].hi;
        cnt++;
    }
    free(k);
    free(used);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Merged covariance -> scale + rotation: cyclic Jacobi (Golub & Van Loan,   */
/* Sec. 8.5) with a canonical form.                                           */

int orc_eig3(const double *Ain, double *lam, double *V) {
    double A[9];
    memcpy(A, Ain, sizeof(A));
    for (int i = 0; i < 9; i++) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
    double fro = 0;
    for (int i = 0; i < 9; i++) fro += A[i] * A[i];
    fro = sqrt(fro);
    int sweep = 0;
    for (; sweep < 64; sweep++) {
        double off = sqrt(2.0 * (A[1] * A[1] + A[2] * A[2] + A[5] * A[5]));
        if (off <= 1e-15 * fro || off == 0) break;
        for (int p = 0; p < 2; p++)
            for (int q = p + 1; q < 3; q++) {
                double apq = A[p * 3 + q];
                if (apq == 0) continue;
                /* 2x2 symmetric Schur: zero A[p][q] with a rotation (c, s) */
                double tau = (A[q * 3 + q] - A[p * 3 + p]) / (2.0 * apq);
                double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- J^T A J, J = identity with J[p][p]=c, J[p][q]=s, J[q][p]=-s, J[q][q]=c */
                for (int k = 0; k < 3; k++) {
                    double akp = A[k * 3 + p], akq = A[k * 3 + q];
                    A[k * 3 + p] = c * akp - s * akq;
                    A[k * 3 + q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; k++) {
                    double apk = A[p * 3 + k], aqk = A[q * 3 + k];
                    A[p * 3 + k] = c * apk - s * aqk;
                    A[q * 3 + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; k++) {
                    double vkp = V[k * 3 + p], vkq = V[k * 3 + q];
                    V[k * 3 + p] = c * vkp - s * vkq;
                    V[k * 3 + q] = s * vkp + c * vkq;
                }
            }
    }
    double l[3] = {A[0], A[4], A[8]};
    /* sort eigenpairs descending */
    int idx[3] = {0, 1, 2};
    for (int a = 0; a < 3; a++)
        for (int b = a + 1; b < 3; b++)
            if (l[idx[b]] > l[idx[a]]) { int t = idx[a]; idx[a] = idx[b]; idx[b] = t; }
    double W[9];
    for (int c = 0; c < 3; c++) {
        lam[c] = l[idx[c]];
        for (int r = 0; r < 3; r++) W[r * 3 + c] = V[r * 3 + idx[c]];
    }
    /* each column's largest-magnitude component positive (first one on ties) */
    for (int c = 0; c < 3; c++) {
        int best = 0;
        for (int r = 1; r < 3; r++)
            if (fabs(W[r * 3 + c]) > fabs(W[best * 3 + c])) best = r;
        if (W[best * 3 + c] < 0)
            for (int r = 0; r < 3; r++) W[r * 3 + c] = -W[r * 3 + c];
    }
    double det = W[0] * (W[4] * W[8] - W[5] * W[7]) - W[1] * (W[3] * W[8] - W[5] * W[6]) +
                 W[2] * (W[3] * W[7] - W[4] * W[6]);
    if (det < 0)
        for (int r = 0; r < 3; r++) W[r * 3 + 2] = -W[r * 3 + 2];
    memcpy(V, W, sizeof(W));
    return sweep;
}

/* Shepperd (1978): pick the largest of (trace, R00, R11, R22) as the pivot. */
void orc_R_to_quat(const double *R, double *q) {
    double tr = R[0] + R[4] + R[8];
    double w, x, y, z;
    if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
        double r = sqrt(1.0 + tr);
        w = 0.5 * r;
        x = (R[7] - R[5]) / (2.0 * r);
        y = (R[2] - R[6]) / (2.0 * r);
        z = (R[3] - R[1]) / (2.0 * r);
    } else if (R[0] >= R[4] && R[0] >= R[8]) {
        double r = sqrt(1.0 + R[0] - R[4] - R[8]);
        x = 0.5 * r;
        w = (R[7] - R[5]) / (2.0 * r);
        y = (R[1] + R[3]) / (2.0 * r);
        z = (R[2] + R[6]) / (2.0 * r);
    } else if (R[4] >= R[8]) {
        double r = sqrt(1.0 - R[0] + R[4] - R[8]);
        y = 0.5 * r;
        w = (R[2] - R[6]) / (2.0 * r);
        x = (R[1] + R[3]) / (2.0 * r);
        z = (R[5] + R[7]) / (2.0 * r);
    } else {
        double r = sqrt(1.0 - R[0] - R[4] + R[8]);
        z = 0.5 * r;
        w = (R[3] - R[1]) / (2.0 * r);
        x = (R[2] + R[6]) / (2.0 * r);
        y = (R[5] + R[7]) / (2.0 * r);
    }
    if (w < 0) { w = -w; x = -x; y = -y; z = -z; }
    double nn = sqrt(w * w + x * x + y * y + z * z);
    q[0] = w / nn; q[1] = x / nn; q[2] = y / nn; q[3] = z / nn;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3: merge one pair (lo, hi) into (xyz, log_scale, rot, logit, sh).  */

static void merge_pair(const double *xyz, const double *log_scale, const double *rot,
                       const double *logit, const double *sh, int F, int64_t i, int64_t j,
                       double eig_floor, double *oxyz, double *ols, double *orot,
                       double *ologit, double *osh) {
    gauss_t gi, gj;
    splat_gauss(xyz + 3 * i, log_scale + 3 * i, rot + 4 * i, logit[i], &gi);
    splat_gauss(xyz + 3 * j, log_scale + 3 * j, rot + 4 * j, logit[j], &gj);
    double pi, pj, lpi, lpj;
    mass_ratio(&gi, &gj, &pi, &pj, &lpi, &lpj);
    double mum[3], Sm[9];
    mpmm_pi(pi, pj, &gi, &gj, mum, Sm);
    for (int a = 0; a < 3; a++) oxyz[a] = mum[a];
    for (int t = 0; t < F; t++) osh[t] = pi * sh[i * F + t] + pj * sh[j * F + t];
    /* Eq. vm_alpha: alpha_m = 1 - (1-alpha_i)(1-alpha_j), via log T */
    double logT = -softplus(logit[i]) - softplus(logit[j]);
    *ologit = log(-expm1(logT)) - logT;
    double lam[3], V[9];
    orc_eig3(Sm, lam, V);
    for (int a = 0; a < 3; a++) {
        double l = lam[a] > eig_floor ? lam[a] : eig_floor;
        ols[a] = 0.5 * log(l);
    }
    orc_R_to_quat(V, orot);
}

int64_t orc_merge_compact(int64_t n, const double *xyz, const double *log_scale,
                          const double *rot, const double *logit, const double *sh, int F,
                          int64_t npairs, const int32_t *pair_lo, const int32_t *pair_hi,
                          double eig_floor,
                          double *oxyz, double *olog_scale, double *orot, double *ologit,
                          double *osh) {
    int32_t *role = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) role[i] = -1; /* -1 unmatched, -2 dropped, >=0 partner */
    for (int64_t p = 0; p < npairs; p++) {
        int64_t a = pair_lo[p], b = pair_hi[p];
        if (a < 0 || b >= n || a >= b || role[a] != -1 || role[b] != -1) { free(role); return -1; }
        role[a] = (int32_t)b;
        role[b] = -2;
    }
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int64_t out = 0;
    for (int64_t i = 0; i < n; i++) pos[i] = role[i] == -2 ? -1 : out++;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int64_t o = pos[i];
        if (o < 0) continue;
        if (role[i] >= 0) {
            merge_pair(xyz, log_scale, rot, logit, sh, F, i, role[i], eig_floor, oxyz + 3 * o,
                       olog_scale + 3 * o, orot + 4 * o, ologit + o, osh + o * F);
        } else {
            memcpy(oxyz + 3 * o, xyz + 3 * i, 3 * sizeof(double));
            memcpy(olog_scale + 3 * o, log_scale + 3 * i, 3 * sizeof(double));
            memcpy(orot + 4 * o, rot + 4 * i, 4 * sizeof(double));
            ologit[o] = logit[i];
            memcpy(osh + o * F, sh + i * F, F * sizeof(double));
        }
    }
    free(role);
    free(pos);
    return out;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.4, local neighbourhood refresh: the lists of the pass after a merge */
/* from the lists before it; only the new splats are queried again.          */

/* Row order after a merge (merged splat at the lower row, the higher row
   removed, the others in order): new id of every old row, the removed row
   taking its partner's. */
static void merge_id_map(int64_t n_old, int64_t np, const int32_t *plo, const int32_t *phi,
                         int32_t *map_old) {
    uint8_t *gone = (uint8_t *)calloc((size_t)(n_old > 0 ? n_old : 1), 1);
    for (int64_t t = 0; t < np; t++) gone[phi[t]] = 1;
    int32_t r = 0;
    for (int64_t o = 0; o < n_old; o++) map_old[o] = gone[o] ? -1 : r++;
    for (int64_t t = 0; t < np; t++) map_old[phi[t]] = map_old[plo[t]];
    free(gone);
}

int64_t orc_refresh_lists(int64_t n_old, int k_old, const int32_t *prev, int64_t np,
                          const int32_t *plo, const int32_t *phi, int64_t n_new,
                          const double *xyz, int k, int32_t *nbr, uint8_t *requery) {
    int ke = k_effective(n_new, k);
    if (ke <= 0) return 0;
    int32_t *map_old = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_old > 0 ? n_old : 1));
    int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_new);
    merge_id_map(n_old, np, plo, phi, map_old);
    for (int64_t r = 0; r < n_new; r++) src[r] = -1;
    uint8_t *merged = (uint8_t *)calloc((size_t)n_old, 1);
    for (int64_t t = 0; t < np; t++) merged[plo[t]] = merged[phi[t]] = 1;
    for (int64_t o = 0; o < n_old; o++)
        if (!merged[o]) src[map_old[o]] = (int32_t)o;   /* kept rows; new splats stay -1 */
    int64_t nq = 0;
    cand_t *list = (cand_t *)malloc(sizeof(cand_t) * (size_t)(k_old > 0 ? k_old : 1));
    for (int64_t r = 0; r < n_new; r++) {
        int rq = src[r] < 0 || k_old != ke;
        int cnt = 0;
        for (int t = 0; !rq && t < k_old; t++) {
            int32_t m = map_old[prev[(int64_t)src[r] * k_old + t]];
            if (m == r) { rq = 1; break; }
            for (int a = 0; a < cnt; a++)
                if (list[a].j == m) { rq = 1; break; }
            if (rq) break;
            cand_t c = {dist2(xyz + 3 * r, xyz + 3 * (int64_t)m), m};
            topk_insert(list, &cnt, ke, c);
        }
        requery[r] = (uint8_t)rq;
        if (rq) { nq++; continue; }
        for (int a = 0; a < ke; a++) nbr[r * ke + a] = list[a].j;   /* sorted by (d^2, id) */
    }
    if (nq > 0) {
        int64_t *q = (int64_t *)malloc(sizeof(int64_t) * (size_t)nq);
        int32_t *out = (int32_t *)malloc(sizeof(int32_t) * (size_t)nq * ke);
        int64_t t = 0;
        for (int64_t r = 0; r < n_new; r++)
            if (requery[r]) q[t++] = r;
        orc_knn_brute_queries(n_new, xyz, k, nq, q, out);
        for (t = 0; t < nq; t++)
            memcpy(nbr + q[t] * ke, out + t * ke, sizeof(int32_t) * ke);
        free(q);
        free(out);
    }
    free(list);
    free(merged);
    free(src);
    free(map_old);
    return nq;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 end to end.                                                    */

static void select_rows(int64_t n, const uint8_t *keep, double *a, int w) {
    int64_t o = 0;
    for (int64_t i = 0; i < n; i++)
        if (keep[i]) {
            if (o != i) memmove(a + o * w, a + i * w, sizeof(double) * w);
            o++;
        }
}

int64_t orc_simplify(int64_t n0, double *xyz, double *log_scale, double *rot, double *logit,
                     double *sh, int F, int64_t target, int k, double tau, int prefilter,
                     int S, int mode, double lambda_geo, double lambda_app, uint64_t seed,
                     double eig_floor, int max_passes, int use_grid, int refresh_period,
                     int32_t *passes, int64_t *pass_n, int64_t *pass_e, int64_t *pass_m,
                     int64_t *pass_rq) {
    int64_t n = n0;
    if (passes) *passes = 0;
    if (n <= 0) return 0;
    if (prefilter) {
        uint8_t *keep = (uint8_t *)malloc(n);
        int64_t kept = orc_prefilter(n, logit, tau, keep);
        select_rows(n, keep, xyz, 3);
        select_rows(n, keep, log_scale, 3);
        select_rows(n, keep, rot, 4);
        select_rows(n, keep, logit, 1);
        select_rows(n, keep, sh, F);
        free(keep);
        n = kept;
    }
    double *b_xyz = (double *)malloc(sizeof(double) * 3 * n0);
    double *b_ls = (double *)malloc(sizeof(double) * 3 * n0);
    double *b_rot = (double *)malloc(sizeof(double) * 4 * n0);
    double *b_logit = (double *)malloc(sizeof(double) * n0);
    double *b_sh = (double *)malloc(sizeof(double) * (size_t)F * n0);
    int32_t *nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)n0 * (k > 0 ? k : 1));
    int32_t *elo = (int32_t *)malloc(sizeof(int32_t) * (size_t)n0 * (k > 0 ? k : 1));
    int32_t *ehi = (int32_t *)malloc(sizeof(int32_t) * (size_t)n0 * (k > 0 ? k : 1));
    double *cost = (double *)malloc(sizeof(double) * (size_t)n0 * (k > 0 ? k : 1));
    int32_t *plo = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n0 / 2 + 1));
    int32_t *phi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n0 / 2 + 1));
    float *z = (float *)malloc(sizeof(float) * 3 * (S > 0 ? S : 1));
    float *u = (float *)malloc(sizeof(float) * (S > 0 ? S : 1));
    int32_t *prev = (int32_t *)malloc(sizeof(int32_t) * (size_t)n0 * (k > 0 ? k : 1));
    uint8_t *rqf = (uint8_t *)malloc((size_t)(n0 > 0 ? n0 : 1));
    int64_t n_prev = 0, mm_prev = 0;
    int ke_prev = 0;
    int p = 0;
    while (n > target && n > 1 && p < max_passes) {
        int ke;
        int64_t rq = n;
        if (refresh_period > 1 && p % refresh_period != 0) {
            /* the previous pass's lists carried through its merge */
            memcpy(prev, nbr, sizeof(int32_t) * (size_t)n_prev * ke_prev);
            rq = orc_refresh_lists(n_prev, ke_prev, prev, mm_prev, plo, phi, n, xyz, k, nbr, rqf);
            ke = k_effective(n, k);
        } else {
            ke = use_grid ? orc_knn_grid(n, xyz, k, nbr) : orc_knn_brute(n, xyz, k, nbr);
        }
        if (pass_rq) pass_rq[p] = rq;
        int64_t m = orc_union_edges(n, ke, nbr, elo, ehi);
        orc_mc_draws(seed, (uint32_t)p, S, z, u);
        orc_edge_costs(n, xyz, log_scale, rot, logit, sh, F, m, elo, ehi, S, z, u, mode,
                       lambda_geo, lambda_app, cost, NULL, NULL);
        int64_t P = n - target;
        int64_t mm = orc_greedy(n, m, elo, ehi, cost, P, plo, phi);
        if (pass_n) pass_n[p] = n;
        if (pass_e) pass_e[p] = m;
        if (pass_m) pass_m[p] = mm;
        p++;
        if (mm == 0) break;
        n_prev = n;
        ke_prev = ke;
        mm_prev = mm;
        int64_t nn = orc_merge_compact(n, xyz, log_scale, rot, logit, sh, F, mm, plo, phi,
                                       eig_floor, b_xyz, b_ls, b_rot, b_logit, b_sh);
        memcpy(xyz, b_xyz, sizeof(double) * 3 * nn);
        memcpy(log_scale, b_ls, sizeof(double) * 3 * nn);
        memcpy(rot, b_rot, sizeof(double) * 4 * nn);
        memcpy(logit, b_logit, sizeof(double) * nn);
        memcpy(sh, b_sh, sizeof(double) * (size_t)F * nn);
        n = nn;
    }
    if (passes) *passes = p;
    free(b_xyz); free(b_ls); free(b_rot); free(b_logit); free(b_sh);
    free(nbr); free(elo); free(ehi); free(cost); free(plo); free(phi); free(z); free(u);
    free(prev); free(rqf);
    return n;
}
