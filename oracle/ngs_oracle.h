/*
 * NanoGS FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct restatement of the simplification method
 * (NanoGS, Sec. 3 and Algorithm 1) in double precision.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never calls it and shares no code with it.
 *
 * Conventions shared with the callers (not with the CUDA path):
 *   splat arrays are double, SoA, row-major per splat:
 *     xyz[n*3], log_scale[n*3], rot[n*4] (w,x,y,z), logit[n], sh[n*F]
 *   edges are (lo, hi) index pairs with lo < hi.
 *
 * Parity status per function is stated beside each declaration; every
 * function is pinned by a "not gpu" test against something other than itself.
 */
#ifndef NGS_ORACLE_H
#define NGS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int orc_num_threads(void);
int orc_set_num_threads(int t);

/* Algorithm 1, opacity pre-filter: tau' = min(tau, lower median alpha); keep
 * alpha >= tau'.  keep[i] is set to 0/1; returns the kept count. */
int64_t orc_prefilter(int64_t n, const double *logit, double tau, uint8_t *keep);

/* Sec. 3.1 / Algorithm 1: directed kNN, k_eff = min(max(1,k), n-1) nearest
 * other centres by squared Euclidean distance, ordered by (d^2, index).
 * nbr is n*k_eff.  Brute force over all pairs. */
int orc_knn_brute(int64_t n, const double *xyz, int k, int32_t *nbr);
/* Same definition for a subset of queries: nbr is nq*k_eff. */
int orc_knn_brute_queries(int64_t n, const double *xyz, int k, int64_t nq,
                          const int64_t *queries, int32_t *nbr);
/* Same definition, uniform-grid search with exact shell termination. */
int orc_knn_grid(int64_t n, const double *xyz, int k, int32_t *nbr);

/* Algorithm 1 UndirectedUnionEdges: unique {i,j}, i<j, lexicographic order.
 * Returns |E| (lo/hi must hold n*k_eff entries). */
int64_t orc_union_edges(int64_t n, int k_eff, const int32_t *nbr, int32_t *lo, int32_t *hi);

/* Common random numbers for the Monte Carlo estimator (App. A): S standard
 * normal 3-vectors z and S uniforms u for pass `pass`, drawn from a
 * SplitMix64 stream and Box-Muller, rounded to float. */
void orc_mc_draws(uint64_t seed, uint32_t pass, int S, float *z, float *u);

/* Sec. 3.2 merge cost C = lambda_geo * D_geo + lambda_app * D_app per edge.
 * mode 0: component-stratified CRN estimator; mode 1: literal mixture draw;
 * mode 2: mode 0 with the cross-entropy term in closed form; mode 3: MSE
 * surrogate |mu_i - mu_j|^2 + ||Sigma_i - Sigma_j||_F^2.
 * dgeo/dapp may be NULL. */
void orc_edge_costs(int64_t n, const double *xyz, const double *log_scale, const double *rot,
                    const double *logit, const double *sh, int F,
                    int64_t m, const int32_t *lo, const int32_t *hi,
                    int S, const float *z, const float *u, int mode,
                    double lambda_geo, double lambda_app,
                    double *cost, double *dgeo, double *dapp);

/* Sec. 3.4 / Algorithm 1 GreedyDisjointPairs: sort by (cost, lo, hi), NaN
 * last, take an edge if both endpoints are free, stop after P picks.  Pairs
 * are returned in pick order; returns the count. */
int64_t orc_greedy(int64_t n, int64_t m, const int32_t *lo, const int32_t *hi,
                   const double *cost, int64_t P, int32_t *pair_lo, int32_t *pair_hi);

/* Sec. 3.3 MPMM merge of every pair (lo<hi), written to slot lo; slot hi is
 * dropped; every other splat keeps its relative order.  Outputs must hold n
 * splats; returns the new count (-1 on bad input). */
int64_t orc_merge_compact(int64_t n, const double *xyz, const double *log_scale,
                          const double *rot, const double *logit, const double *sh, int F,
                          int64_t npairs, const int32_t *pair_lo, const int32_t *pair_hi,
                          double eig_floor,
                          double *oxyz, double *olog_scale, double *orot, double *ologit,
                          double *osh);

/* Algorithm 1 end to end (in place, arrays hold n0 splats).  Returns the final
 * count; per-pass counts go to pass_n / pass_e / pass_m (may be NULL, at most
 * max_passes entries) and the pass count to *passes. */
int64_t orc_simplify(int64_t n0, double *xyz, double *log_scale, double *rot, double *logit,
                     double *sh, int F, int64_t target, int k, double tau, int prefilter,
                     int S, int mode, double lambda_geo, double lambda_app, uint64_t seed,
                     double eig_floor, int max_passes, int use_grid, int refresh_period,
                     int32_t *passes, int64_t *pass_n, int64_t *pass_e, int64_t *pass_m,
                     int64_t *pass_rq);
/* Sec. 3.4 local neighbourhood refresh: the kNN lists after a merge from the
   lists before it.  prev: n_old x k_old lists; (plo[t], phi[t]) the merged
   pairs (old ids, plo < phi); xyz: the n_new centres after the merge (merged
   splat at the lower row, the higher row removed, others in order).  A new
   row is re-queried (exact k_eff nearest, brute force) when it holds a merged
   splat, when k_eff changed, or when its old list maps to an id repeated or
   equal to itself; otherwise its list is the mapped old list sorted by
   (d^2, id).  requery[r] records the decision; returns the re-queried count. */
int64_t orc_refresh_lists(int64_t n_old, int k_old, const int32_t *prev, int64_t np,
                          const int32_t *plo, const int32_t *phi, int64_t n_new,
                          const double *xyz, int k, int32_t *nbr, uint8_t *requery);

/* ---- single-pair helpers, exposed for the pins ---- */
/* Unit quaternion (w,x,y,z) -> row-major rotation matrix (normalises q). */
void orc_quat_to_R(const double *q, double *R);
/* Cyclic Jacobi eigendecomposition of a symmetric 3x3 (row-major) with the
 * canonical form: eigenvalues descending, each eigenvector's largest-magnitude
 * component positive, det(V) = +1 (V columns are eigenvectors). Returns sweeps. */
int orc_eig3(const double *A, double *lam, double *V);
/* Rotation matrix -> quaternion (Shepperd), w >= 0. */
void orc_R_to_quat(const double *R, double *q);
/* MPMM on the moment form (Eqs. vm_weights..vm_cov): inputs w, mu, Sigma(3x3),
 * f; outputs pi, mu_m, Sigma_m(3x3), f_m. */
void orc_mpmm_moments(double wi, const double *mui, const double *Si, const double *fi,
                      double wj, const double *muj, const double *Sj, const double *fj, int F,
                      double *mum, double *Sm, double *fm);
/* Closed-form KL(N_i || N_j) and I-divergence of unnormalised Gaussians (App. A). */
double orc_kl_gauss(const double *mui, const double *Si, const double *muj, const double *Sj);
double orc_idiv_gauss(double mi, const double *mui, const double *Si,
                      double mj, const double *muj, const double *Sj);
/* D_geo of one pair given splat parameters (mode 0..3), S samples z,u. */
double orc_dgeo_pair(const double *xyz_i, const double *ls_i, const double *rot_i, double logit_i,
                     const double *xyz_j, const double *ls_j, const double *rot_j, double logit_j,
                     int S, const float *z, const float *u, int mode);

#ifdef __cplusplus
}
#endif
#endif
