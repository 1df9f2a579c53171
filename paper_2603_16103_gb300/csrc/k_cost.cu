// Merge cost of every candidate edge (Sec. 3.2, Eq. Equ:cost; App. A).
//
// C(i,j) = lambda_geo * D_geo + lambda_app * D_app with
//   D_app = || f_i - f_j ||^2 over all SH coefficients,
//   D_geo = KL( pi N_i + (1-pi) N_j || N(mu_m, Sigma_m) ) estimated with S
//           common standard-normal draws z_s shared by all edges of a pass,
//   pi = w_i / (w_i + w_j), w = (2 pi)^{3/2} alpha prod s (Eq. vm_weights),
//   (mu_m, Sigma_m) the MPMM moments (Eq. vm_cov).
// Sample points use the symmetric square root, x_c = mu_c + Sigma_c^{1/2} z.
// Writing every log-density relative to the merged Gaussian,
//   g(x) = logsumexp(log pi + a_i - q_i(x)/2, log(1-pi) + a_j - q_j(x)/2) + q_m(x)/2,
//   a_c  = log sqrt(det Sigma_m / det Sigma_c),  q_c = Mahalanobis^2 under c,
// keeps FP32 cancellation small; q_c(x_c) = |z|^2 exactly.
// Mode 0 averages pi g(x_i) + (1-pi) g(x_j) (the component draw integrated
// out); mode 1 takes g(x_i) if u_s < pi else g(x_j).  Mode 2 is mode 0 with
// the cross-entropy term in closed form: -E[log q_m] = 1/2 log det(2 pi Sigma_m)
// + 3/2, so q_m(x)/2 above becomes 3/2 and only the entropy is sampled.
// Mode 3 is the MSE surrogate |mu_i - mu_j|^2 + ||Sigma_i - Sigma_j||_F^2
// (the Sec. 4 ablation), evaluated in FP32 with no FP64 path.
// A merged covariance whose FP32 Cholesky pivots fall below 1e-2 of the
// matching diagonal entries (near-degenerate) is redone entirely in FP64.
//
// Accuracy contract (cost_tol = tau_c > 0): the FP32 kernel carries a
// first-order running estimate E of its own rounding error (each Mahalanobis
// term, log-determinant, log-sum-exp and sum, weighted by how much it enters
// the result) and sends an edge to the FP64 path when 2 E exceeds
// tau_c max(|C|, 1); every cost it keeps is then within tau_c max(|C|, 1) of
// the FP64 value.  After the costs, each vertex compares the costs of its
// adjacent edges: two whose costs lie within tau_c (max(|C_e|,1) +
// max(|C_f|,1)) of each other are both recomputed in FP64 (D_geo and D_app)
// and stored rounded to FP32.  Every comparison the greedy rule of Sec. 3.4
// makes is between adjacent edges, so the pair set then follows the FP64
// costs except where two FP64 costs round to the same FP32 value.
#include "ffmath.cuh"
#include "ngs_device.cuh"
#include "ngs_internal.h"

namespace {

constexpr float LOG_2PI_F = 1.8378770664093453f;
constexpr int REC = 16;  // floats per per-splat record

// record layout: (mu, log w), R row-major, 1 / s.  The edge kernel derives
// s, Sigma and Sigma^{1/2} z from these (fewer bytes through L1 per edge).
enum { R_MU = 0, R_LW = 3, R_R = 4, R_INVS = 13 };

__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float *R) {
    float inv = rsqrtf(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

// y = R diag(s) R^T z, with s = 1 / invs (the same rounding as a stored s)
__device__ __forceinline__ void sym_sqrt_apply(const float *R, const float *invs, const float *z,
                                               float *y) {
    float t[3];
#pragma unroll
    for (int k = 0; k < 3; k++)
        t[k] = (1.0f / invs[k]) * (R[k] * z[0] + R[3 + k] * z[1] + R[6 + k] * z[2]);
#pragma unroll
    for (int a = 0; a < 3; a++) y[a] = R[3 * a] * t[0] + R[3 * a + 1] * t[1] + R[3 * a + 2] * t[2];
}

__global__ void k_prep(const float *__restrict__ xyz, const float *__restrict__ ls,
                       const float *__restrict__ rot, const float *__restrict__ logit, int64_t n,
                       float *__restrict__ rec) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        float r[REC];
        float R[9], sc[3], l[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            r[R_MU + a] = xyz[3 * v + a];
            l[a] = ls[3 * v + a];
            sc[a] = expf(l[a]);
        }
        quat_rot(rot[4 * v], rot[4 * v + 1], rot[4 * v + 2], rot[4 * v + 3], R);
        r[R_LW] = 1.5f * LOG_2PI_F - softplusf(-logit[v]) + (l[0] + l[1] + l[2]);
#pragma unroll
        for (int k = 0; k < 9; k++) r[R_R + k] = R[k];
#pragma unroll
        for (int a = 0; a < 3; a++) r[R_INVS + a] = 1.0f / sc[a];
        float4 *dst = (float4 *)(rec + (int64_t)v * REC);
#pragma unroll
        for (int k = 0; k < REC / 4; k++) dst[k] = make_float4(r[4 * k], r[4 * k + 1], r[4 * k + 2], r[4 * k + 3]);
    }
}

// log(e^a + e^b), and wa = the weight of a in it (e^(a - lse))
__device__ __forceinline__ float lse2w(float a, float b, float &wa) {
    const float m = fmaxf(a, b);
    const float e = __expf(-fabsf(a - b));
    const float ws = __fdividef(e, 1.0f + e);  // weight of the smaller argument
    wa = a >= b ? 1.0f - ws : ws;
    return m + log1pf(e);
}
// square root of q >= 0 for the error estimate (approximate; 0 at 0)
__device__ __forceinline__ float sqrt_nn(float q) { return q * rsqrtf(fmaxf(q, 1e-30f)); }
__device__ __forceinline__ float absmax3(const float *v) {
    return fmaxf(fmaxf(fabsf(v[0]), fabsf(v[1])), fabsf(v[2]));
}
constexpr float U32 = 5.9604645e-8f;  // unit roundoff of FP32, 2^-24

// |diag(inv_s) R^T v|^2
__device__ __forceinline__ float maha_splat(const float *R, const float *invs, const float *v) {
    float q = 0.f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        float t = (R[k] * v[0] + R[3 + k] * v[1] + R[6 + k] * v[2]) * invs[k];
        q += t * t;
    }
    return q;
}

// |L^{-1} v|^2 with L lower (l00, l10, l11, l20, l21, l22) and inverse diagonal
__device__ __forceinline__ float maha_chol(const float *L, const float *il, const float *v) {
    float y0 = v[0] * il[0];
    float y1 = (v[1] - L[1] * y0) * il[1];
    float y2 = (v[2] - L[3] * y0 - L[4] * y1) * il[2];
    return y0 * y0 + y1 * y1 + y2 * y2;
}

// ---------------------------------------------------------------- FP64 path
struct G64 {
    double mu[3], R[9], s[3], Sig[6], sum_ls, lw;
};

__device__ void splat64(const float *xyz, const float *ls, const float *rot, const float *logit,
                        int64_t v, G64 &g) {
    double w = rot[4 * v], x = rot[4 * v + 1], y = rot[4 * v + 2], z = rot[4 * v + 3];
    double nn = w * w + x * x + y * y + z * z;
    double inv = 1.0 / sqrt(nn);
    w *= inv; x *= inv; y *= inv; z *= inv;
    double *R = g.R;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
    g.sum_ls = 0;
    for (int a = 0; a < 3; a++) {
        g.mu[a] = xyz[3 * v + a];
        g.s[a] = exp((double)ls[3 * v + a]);
        g.sum_ls += (double)ls[3 * v + a];
    }
    int idx = 0;
    for (int a = 0; a < 3; a++)
        for (int b = a; b < 3; b++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += R[3 * a + k] * g.s[k] * g.s[k] * R[3 * b + k];
            g.Sig[idx++] = acc;
        }
    g.lw = 1.5 * 1.8378770664093454835606594728112 - softplus_d(-(double)logit[v]) + g.sum_ls;
}

__device__ double maha64_splat(const G64 &g, const double *v) {
    double q = 0;
    for (int k = 0; k < 3; k++) {
        double t = (g.R[k] * v[0] + g.R[3 + k] * v[1] + g.R[6 + k] * v[2]) / g.s[k];
        q += t * t;
    }
    return q;
}

__device__ double lse2_d(double a, double b) {
    double m = fmax(a, b);
    return m + log1p(exp(-fabs(a - b)));
}

__device__ __noinline__ double dgeo_fp64(const float *xyz, const float *ls, const float *rot,
                            const float *logit, int64_t i, int64_t j, int S,
                            const float *__restrict__ zs, const float *__restrict__ us, int mode) {
    G64 gi, gj;
    splat64(xyz, ls, rot, logit, i, gi);
    splat64(xyz, ls, rot, logit, j, gj);
    if (mode == 3) {
        double r = 0;
        for (int a = 0; a < 3; a++) r += (gi.mu[a] - gj.mu[a]) * (gi.mu[a] - gj.mu[a]);
        for (int t = 0; t < 6; t++) {
            const double dd = gi.Sig[t] - gj.Sig[t];
            r += (t == 0 || t == 3 || t == 5 ? 1.0 : 2.0) * dd * dd;
        }
        return r;
    }
    // pi = sigmoid(ld) and its complement share t = e^{-|ld|}
    const double ld = gi.lw - gj.lw;
    const double t = exp(-fabs(ld)), l1t = log1p(t);
    const double lpi = -(fmax(-ld, 0.0) + l1t), lpj = -(fmax(ld, 0.0) + l1t);
    const double big = 1.0 / (1.0 + t), small = t * big;
    const double pi = ld >= 0 ? big : small, pj = ld >= 0 ? small : big;
    double d[3] = {gi.mu[0] - gj.mu[0], gi.mu[1] - gj.mu[1], gi.mu[2] - gj.mu[2]};
    double Sm[6];
    int idx = 0;
    for (int a = 0; a < 3; a++)
        for (int b = a; b < 3; b++, idx++) Sm[idx] = pi * gi.Sig[idx] + pj * gj.Sig[idx] + pi * pj * d[a] * d[b];
    // Sm = (00 01 02 11 12 22)
    double l00 = sqrt(Sm[0]);
    double l10 = Sm[1] / l00, l20 = Sm[2] / l00;
    double t11 = Sm[3] - l10 * l10;
    if (!(t11 > 0)) return INFINITY;
    double l11 = sqrt(t11);
    double l21 = (Sm[4] - l20 * l10) / l11;
    double t22 = Sm[5] - l20 * l20 - l21 * l21;
    if (!(t22 > 0)) return INFINITY;
    double l22 = sqrt(t22);
    double half_ldm = 0.5 * log(Sm[0] * t11 * t22);  // log(l00 l11 l22)
    double ai = half_ldm - gi.sum_ls, aj = half_ldm - gj.sum_ls;
    double acc = 0;
    for (int s = 0; s < S; s++) {
        double z[3] = {zs[3 * s], zs[3 * s + 1], zs[3 * s + 2]};
        double zz = z[0] * z[0] + z[1] * z[1] + z[2] * z[2];
        double yi[3], yj[3];
        for (int pass = 0; pass < 2; pass++) {
            const G64 &g = pass == 0 ? gi : gj;
            double *y = pass == 0 ? yi : yj;
            double t[3];
            for (int k = 0; k < 3; k++) t[k] = g.s[k] * (g.R[k] * z[0] + g.R[3 + k] * z[1] + g.R[6 + k] * z[2]);
            for (int a = 0; a < 3; a++) y[a] = g.R[3 * a] * t[0] + g.R[3 * a + 1] * t[1] + g.R[3 * a + 2] * t[2];
        }
        double gvals[2];
        for (int side = 0; side < 2; side++) {
            // side 0: x = x_i, side 1: x = x_j ; offsets from each mean
            double vi[3], vj[3], vm[3];
            for (int a = 0; a < 3; a++) {
                if (side == 0) {
                    vi[a] = yi[a];
                    vj[a] = d[a] + yi[a];
                    vm[a] = pj * d[a] + yi[a];
                } else {
                    vi[a] = yj[a] - d[a];
                    vj[a] = yj[a];
                    vm[a] = yj[a] - pi * d[a];
                }
            }
            double qi = side == 0 ? zz : maha64_splat(gi, vi);
            double qj = side == 1 ? zz : maha64_splat(gj, vj);
            double y0 = vm[0] / l00, y1 = (vm[1] - l10 * y0) / l11, y2 = (vm[2] - l20 * y0 - l21 * y1) / l22;
            double qm = y0 * y0 + y1 * y1 + y2 * y2;
            gvals[side] = lse2_d(lpi + ai - 0.5 * qi, lpj + aj - 0.5 * qj) + (mode == 2 ? 1.5 : 0.5 * qm);
        }
        if (mode != 1) acc += pi * gvals[0] + pj * gvals[1];
        else acc += ((double)us[s] < pi) ? gvals[0] : gvals[1];
    }
    return acc / S;
}

// D_app = sum over the F coefficients of (f_i - f_j)^2 in FP64
__device__ double dapp_fp64(const float *sh, int F, int64_t i, int64_t j) {
    double a = 0;
    for (int t = 0; t < F; t++) {
        const double d = (double)sh[i * F + t] - (double)sh[j * F + t];
        a += d * d;
    }
    return a;
}

// ---------------------------------------------------------------- float-float path
// The same evaluation as the FP64 path, step for step, in float-float
// arithmetic on the FP32 pipes (ffmath.cuh): about 48 significant bits, so
// the cost rounds to the same float as the FP64 evaluation except within a
// few units of 2^-48 of a rounding boundary.  GB300 runs FP64 at about 1/64
// of the FP32 rate; this path is the default for the edges the accuracy
// contract refines, FP64 the option (fp64_policy 3).
struct Gff {
    float mu[3];
    ff R[9], s[3], is[3], Sig[6], sum_ls, lw;
};

constexpr float FF_HLOG2PI_H = 0x1.60df56p+1f;   // 1.5 log(2 pi), head
constexpr float FF_HLOG2PI_L = -0x1.368e2p-24f;  // and tail

__device__ __forceinline__ ff ff_twice(ff a) { return {__fmul_rn(a.h, 2.f), __fmul_rn(a.l, 2.f)}; }

__device__ __noinline__ void splat_ff(const float *xyz, const float *ls, const float *rot,
                                      const float *logit, int64_t v, Gff &g) {
    const float qw = rot[4 * v], qx = rot[4 * v + 1], qy = rot[4 * v + 2], qz = rot[4 * v + 3];
    const ff nn = ff_add(ff_add(ff_prod(qw, qw), ff_prod(qx, qx)), ff_add(ff_prod(qy, qy), ff_prod(qz, qz)));
    const ff inv = ff_div(ff_of(1.f), ff_sqrt(nn));
    const ff w = ff_mulf(inv, qw), x = ff_mulf(inv, qx), y = ff_mulf(inv, qy), z = ff_mulf(inv, qz);
    const ff xx = ff_sqr(x), yy = ff_sqr(y), zz = ff_sqr(z);
    const ff xy = ff_mul(x, y), xz = ff_mul(x, z), yz = ff_mul(y, z);
    const ff wx = ff_mul(w, x), wy = ff_mul(w, y), wz = ff_mul(w, z);
    const ff one = ff_of(1.f);
    g.R[0] = ff_sub(one, ff_twice(ff_add(yy, zz)));
    g.R[1] = ff_twice(ff_sub(xy, wz));
    g.R[2] = ff_twice(ff_add(xz, wy));
    g.R[3] = ff_twice(ff_add(xy, wz));
    g.R[4] = ff_sub(one, ff_twice(ff_add(xx, zz)));
    g.R[5] = ff_twice(ff_sub(yz, wx));
    g.R[6] = ff_twice(ff_sub(xz, wy));
    g.R[7] = ff_twice(ff_add(yz, wx));
    g.R[8] = ff_sub(one, ff_twice(ff_add(xx, yy)));
    ff s2[3];
    for (int a = 0; a < 3; a++) {
        g.mu[a] = xyz[3 * v + a];
        g.s[a] = ff_exp(ff_of(ls[3 * v + a]));
        g.is[a] = ff_div(one, g.s[a]);
        s2[a] = ff_sqr(g.s[a]);
    }
    g.sum_ls = ff_add_acc(ff_two_sum(ls[3 * v], ls[3 * v + 1]), ff_of(ls[3 * v + 2]));
    int idx = 0;
    for (int a = 0; a < 3; a++)
        for (int b = a; b < 3; b++) {
            ff acc = ff_of(0.f);
            for (int k = 0; k < 3; k++) acc = ff_add(acc, ff_mul(ff_mul(g.R[3 * a + k], s2[k]), g.R[3 * b + k]));
            g.Sig[idx++] = acc;
        }
    g.lw = ff_add(ff_sub(ff{FF_HLOG2PI_H, FF_HLOG2PI_L}, ff_softplus(ff_of(-logit[v]))), g.sum_ls);
}

__device__ __forceinline__ ff maha_ff(const Gff &g, const ff *v) {
    ff q = ff_of(0.f);
    for (int k = 0; k < 3; k++) {
        const ff t = ff_mul(ff_add(ff_add(ff_mul(g.R[k], v[0]), ff_mul(g.R[3 + k], v[1])), ff_mul(g.R[6 + k], v[2])),
                            g.is[k]);
        q = ff_add(q, ff_sqr(t));
    }
    return q;
}

// log(a b c) for a, b, c > 0, without forming a product that could leave the
// float range: the factors' binary exponents are taken out first
__device__ __forceinline__ ff ff_log_prod3(ff a, ff b, ff c) {
    int ea, eb, ec;
    frexpf(a.h, &ea);
    frexpf(b.h, &eb);
    frexpf(c.h, &ec);
    const ff m = ff_mul(ff_mul(ff_ldexp(a, -ea), ff_ldexp(b, -eb)), ff_ldexp(c, -ec));
    ff y = ff_log(m);
    const float ef = (float)(ea + eb + ec);
    y = ff_add_acc(y, ff_prod(ef, FF_LN2_H));
    y = ff_add_acc(y, ff_prod(ef, FF_LN2_M));
    return ff_add(y, ff_of(__fmul_rn(ef, FF_LN2_L)));
}

__device__ __noinline__ ff dgeo_ff(const float *xyz, const float *ls, const float *rot,
                                   const float *logit, int64_t i, int64_t j, int S,
                                   const float *__restrict__ zs, const float *__restrict__ us, int mode) {
    Gff gi, gj;
    splat_ff(xyz, ls, rot, logit, i, gi);
    splat_ff(xyz, ls, rot, logit, j, gj);
    if (mode == 3) {
        ff r = ff_of(0.f);
        for (int a = 0; a < 3; a++) r = ff_add(r, ff_sqr(ff_two_sum(gi.mu[a], -gj.mu[a])));
        for (int t = 0; t < 6; t++) {
            const ff dd = ff_sub_acc(gi.Sig[t], gj.Sig[t]);
            const ff e2 = ff_sqr(dd);
            r = ff_add(r, (t == 0 || t == 3 || t == 5) ? e2 : ff_twice(e2));
        }
        return r;
    }
    const ff inf = ff_of(__int_as_float(0x7f800000));
    // pi = sigmoid(ld) and its complement share t = e^{-|ld|}
    const ff ld = ff_sub_acc(gi.lw, gj.lw);
    const bool ldpos = !(ld.h < 0.f);
    const ff t = ff_exp(ff_neg(ff_abs(ld))), l1t = ff_log1p(t);
    const ff zero = ff_of(0.f);
    const ff lpi = ff_neg(ff_add(ldpos ? zero : ff_neg(ld), l1t));
    const ff lpj = ff_neg(ff_add(ldpos ? ld : zero, l1t));
    const ff big = ff_div(ff_of(1.f), ff_add_acc(ff_of(1.f), t)), small = ff_mul(t, big);
    const ff pi = ldpos ? big : small, pj = ldpos ? small : big;
    const ff pp = ff_mul(pi, pj);
    ff d[3];
    for (int a = 0; a < 3; a++) d[a] = ff_two_sum(gi.mu[a], -gj.mu[a]);
    ff Sm[6];
    int idx = 0;
    for (int a = 0; a < 3; a++)
        for (int b = a; b < 3; b++, idx++)
            Sm[idx] = ff_add(ff_add(ff_mul(pi, gi.Sig[idx]), ff_mul(pj, gj.Sig[idx])),
                             ff_mul(ff_mul(pp, d[a]), d[b]));
    // Sm = (00 01 02 11 12 22)
    const ff l00 = ff_sqrt(Sm[0]);
    const ff l10 = ff_div(Sm[1], l00), l20 = ff_div(Sm[2], l00);
    const ff t11 = ff_sub_acc(Sm[3], ff_sqr(l10));
    if (!ff_pos(t11)) return inf;
    const ff l11 = ff_sqrt(t11);
    const ff l21 = ff_div(ff_sub_acc(Sm[4], ff_mul(l20, l10)), l11);
    const ff t22 = ff_sub_acc(ff_sub_acc(Sm[5], ff_sqr(l20)), ff_sqr(l21));
    if (!ff_pos(t22)) return inf;
    const ff l22 = ff_sqrt(t22);
    const ff half_ldm = ff_mulf(ff_log_prod3(Sm[0], t11, t22), 0.5f);  // log(l00 l11 l22)
    const ff ai = ff_sub_acc(half_ldm, gi.sum_ls), aj = ff_sub_acc(half_ldm, gj.sum_ls);
    const ff ci = ff_add(lpi, ai), cj = ff_add(lpj, aj);
    ff acc = zero;
    for (int s = 0; s < S; s++) {
        const float z[3] = {zs[3 * s], zs[3 * s + 1], zs[3 * s + 2]};
        const ff zz = ff_add(ff_add(ff_prod(z[0], z[0]), ff_prod(z[1], z[1])), ff_prod(z[2], z[2]));
        ff yi[3], yj[3];
        for (int pass = 0; pass < 2; pass++) {
            const Gff &g = pass == 0 ? gi : gj;
            ff *y = pass == 0 ? yi : yj;
            ff tt[3];
            for (int k = 0; k < 3; k++)
                tt[k] = ff_mul(g.s[k], ff_add(ff_add(ff_mulf(g.R[k], z[0]), ff_mulf(g.R[3 + k], z[1])),
                                              ff_mulf(g.R[6 + k], z[2])));
            for (int a = 0; a < 3; a++)
                y[a] = ff_add(ff_add(ff_mul(g.R[3 * a], tt[0]), ff_mul(g.R[3 * a + 1], tt[1])),
                              ff_mul(g.R[3 * a + 2], tt[2]));
        }
        ff gv[2];
        for (int side = 0; side < 2; side++) {
            // side 0: x = x_i, side 1: x = x_j; offsets from each mean
            ff vi[3], vj[3], vm[3];
            for (int a = 0; a < 3; a++) {
                if (side == 0) {
                    vi[a] = yi[a];
                    vj[a] = ff_add(d[a], yi[a]);
                    vm[a] = ff_add(ff_mul(pj, d[a]), yi[a]);
                } else {
                    vi[a] = ff_sub(yj[a], d[a]);
                    vj[a] = yj[a];
                    vm[a] = ff_sub(yj[a], ff_mul(pi, d[a]));
                }
            }
            const ff qi = side == 0 ? zz : maha_ff(gi, vi);
            const ff qj = side == 1 ? zz : maha_ff(gj, vj);
            const ff y0 = ff_div(vm[0], l00);
            const ff y1 = ff_div(ff_sub(vm[1], ff_mul(l10, y0)), l11);
            const ff y2 = ff_div(ff_sub(ff_sub(vm[2], ff_mul(l20, y0)), ff_mul(l21, y1)), l22);
            const ff qm = ff_add(ff_add(ff_sqr(y0), ff_sqr(y1)), ff_sqr(y2));
            const ff l = ff_lse2(ff_sub(ci, ff_mulf(qi, 0.5f)), ff_sub(cj, ff_mulf(qj, 0.5f)));
            gv[side] = ff_add(l, mode == 2 ? ff_of(1.5f) : ff_mulf(qm, 0.5f));
        }
        if (mode != 1) {
            acc = ff_add(acc, ff_add(ff_mul(pi, gv[0]), ff_mul(pj, gv[1])));
        } else {
            // u_s < pi, decided exactly
            const bool first = ff_pos(ff_sub_acc(pi, ff_of(us[s])));
            acc = ff_add(acc, first ? gv[0] : gv[1]);
        }
    }
    return ff_div(acc, ff_of((float)S));
}

// D_app = sum over the F coefficients of (f_i - f_j)^2 (each difference exact)
__device__ ff dapp_ff(const float *sh, int F, int64_t i, int64_t j) {
    ff a = ff_of(0.f);
    for (int t = 0; t < F; t++) a = ff_add(a, ff_sqr(ff_two_sum(sh[i * F + t], -sh[j * F + t])));
    return a;
}

// the whole cost in float-float, rounded once to FP32 (i = lower canonical id)
__device__ float cost_ff(const float *xyz, const float *ls, const float *rot, const float *logit,
                         const float *sh, int F, int64_t i, int64_t j, int S,
                         const float *zs, const float *us, int mode, float lg, float la) {
    const ff dg = dgeo_ff(xyz, ls, rot, logit, i, j, S, zs, us, mode);
    if (!(dg.h < __int_as_float(0x7f800000))) return dg.h;
    return ff_to_float(ff_add(ff_mulf(dg, lg), ff_mulf(dapp_ff(sh, F, i, j), la)));
}

// the whole cost in FP64, rounded once to FP32 (i = lower canonical id)
__device__ float cost_fp64(const float *xyz, const float *ls, const float *rot, const float *logit,
                           const float *sh, int F, int64_t i, int64_t j, int S,
                           const float *zs, const float *us, int mode, float lg, float la) {
    const double dg = dgeo_fp64(xyz, ls, rot, logit, i, j, S, zs, us, mode);
    return (float)((double)lg * dg + (double)la * dapp_fp64(sh, F, i, j));
}

// ---------------------------------------------------------------- edge kernel
// Record layout in float4 groups: G0 = (mu, log w), G1..G3 = R (row-major)
// then inv_s in G3.yzw.

// Sigma = R diag(s^2) R^T, upper triangle (00 01 02 11 12 22)
__device__ __forceinline__ void cov6(const float *R, const float *s, float *S6) {
    const float s2[3] = {s[0] * s[0], s[1] * s[1], s[2] * s[2]};
    int idx = 0;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = a; b < 3; b++)
            S6[idx++] = R[3 * a] * s2[0] * R[3 * b] + R[3 * a + 1] * s2[1] * R[3 * b + 1] +
                        R[3 * a + 2] * s2[2] * R[3 * b + 2];
}
// 32 bytes through the read-only path in one load (p 32-byte aligned)
__device__ __forceinline__ void ldg_v8(const float *p, float *r) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
        : "l"(p));
}

template <int MODE>
__global__ void __launch_bounds__(256, 3)
    k_edge_cost(const int4 *__restrict__ erec, int64_t m, const float *__restrict__ rec,
                const float *__restrict__ sh, int F,
                const float *__restrict__ zs, const float *__restrict__ us, int S,
                float lg, float la, int policy, const float *__restrict__ xyz,
                const float *__restrict__ ls, const float *__restrict__ rot,
                const float *__restrict__ logit, float *__restrict__ cost_slot,
                float *__restrict__ revcost, float *__restrict__ cost_out,
                unsigned long long *fp64_count, int32_t *__restrict__ fp64_list, float tol) {
    const int lane = threadIdx.x & 31;
    const int F4 = F >> 2;
    const float4 *sh4 = (const float4 *)sh;
    // Warp-uniform loop over 32-edge chunks.  The appearance term is summed by
    // 4 lanes per edge, each a quarter of the float4 chunks of both SH rows,
    // so a load instruction reads 8 rows x 64 contiguous bytes instead of 32
    // rows x 16 bytes (the gathers are bound by the L1 data pipe); each lane
    // then evaluates its own edge's geometric term.
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = base + threadIdx.x;
        const bool valid = e < m;
        // i = lower canonical id: the arithmetic is then independent of row order
        const int4 er = valid ? __ldg(erec + e) : make_int4(-1, 0, 0, -1);
        float dapp = 0.f;
        if ((F & 3) == 0) {
            const int64_t wb = base + (threadIdx.x & ~31);
            float dpart[4];
#pragma unroll
            for (int qd = 0; qd < 4; qd++) {
                const int el = qd * 8 + (lane >> 2), sub = lane & 3;
                const int32_t ii = __shfl_sync(FULL_MASK, er.y, el), jj = __shfl_sync(FULL_MASK, er.z, el);
                float acc = 0.f;
                if (wb + el < m) {
                    const float4 *fi = sh4 + (int64_t)ii * F4, *fj = sh4 + (int64_t)jj * F4;
                    if (F4 <= 12) {
                        // up to 3 chunks of each row, all loads in flight together
                        float4 a[3], b[3];
#pragma unroll
                        for (int u = 0; u < 3; u++) {
                            const int t = sub + 4 * u;
                            a[u] = t < F4 ? __ldg(fi + t) : make_float4(0.f, 0.f, 0.f, 0.f);
                            b[u] = t < F4 ? __ldg(fj + t) : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < 3; u++) {
                            const float dx = a[u].x - b[u].x, dy = a[u].y - b[u].y;
                            const float dz = a[u].z - b[u].z, dw = a[u].w - b[u].w;
                            acc += dx * dx + dy * dy + dz * dz + dw * dw;
                        }
                    } else {
                        for (int t = sub; t < F4; t += 4) {
                            const float4 a = __ldg(fi + t), b = __ldg(fj + t);
                            const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
                            acc += dx * dx + dy * dy + dz * dz + dw * dw;
                        }
                    }
                }
                acc += __shfl_xor_sync(FULL_MASK, acc, 1);
                acc += __shfl_xor_sync(FULL_MASK, acc, 2);
                dpart[qd] = acc;
            }
            const int src = (lane & 7) * 4;
            const float d0 = __shfl_sync(FULL_MASK, dpart[0], src), d1 = __shfl_sync(FULL_MASK, dpart[1], src);
            const float d2 = __shfl_sync(FULL_MASK, dpart[2], src), d3 = __shfl_sync(FULL_MASK, dpart[3], src);
            const int qd = lane >> 3;
            dapp = qd == 0 ? d0 : (qd == 1 ? d1 : (qd == 2 ? d2 : d3));
        } else if (valid) {
            for (int t = 0; t < F; t++) {
                float df = sh[(int64_t)er.y * F + t] - sh[(int64_t)er.z * F + t];
                dapp += df * df;
            }
        }
        if (!valid) continue;
        const int32_t sl = er.x;
        const int64_t i = er.y, j = er.z;
        float ri[16], rj[16];
        ldg_v8(rec + i * REC, ri);
        ldg_v8(rec + i * REC + 8, ri + 8);
        ldg_v8(rec + j * REC, rj);
        ldg_v8(rec + j * REC + 8, rj + 8);
        const float4 i0 = make_float4(ri[0], ri[1], ri[2], ri[3]);
        const float4 j0 = make_float4(rj[0], rj[1], rj[2], rj[3]);
        float Rm[9], invs_i[3], Rn[9], invs_j[3];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            Rm[k] = ri[R_R + k];
            Rn[k] = rj[R_R + k];
        }
#pragma unroll
        for (int a = 0; a < 3; a++) {
            invs_i[a] = ri[R_INVS + a];
            invs_j[a] = rj[R_INVS + a];
        }
        float si[3], sj[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            si[a] = 1.0f / invs_i[a];
            sj[a] = 1.0f / invs_j[a];
        }
        const float d[3] = {i0.x - j0.x, i0.y - j0.y, i0.z - j0.z};
        if (MODE == 3) {
            float Si[6], Sj[6];
            cov6(Rm, si, Si);
            cov6(Rn, sj, Sj);
            // Sigma (00 01 02 11 12 22): off-diagonal entries count twice
            float dgeo = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
#pragma unroll
            for (int t = 0; t < 6; t++) {
                const float e = Si[t] - Sj[t];
                dgeo += (t == 0 || t == 3 || t == 5 ? 1.f : 2.f) * e * e;
            }
            const float c = lg * dgeo + la * dapp;
            cost_slot[sl] = c;
            if (er.w >= 0) cost_slot[er.w] = c;
        else if (er.w <= -2) revcost[-2 - er.w] = c;
            if (cost_out) cost_out[e] = c;
            continue;
        }
        // ---- MPMM moments (Eqs. vm_weights, vm_cov)
        const float ld = i0.w - j0.w;
        const float lpi = -softplusf(-ld), lpj = -softplusf(ld);
        const float pi = __expf(lpi), pj = __expf(lpj);
        const float ppd = pi * pj;
        float Sm[6];
        {
            float Si[6], Sj[6];
            cov6(Rm, si, Si);
            cov6(Rn, sj, Sj);
            int idx = 0;
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = a; b < 3; b++, idx++)
                    Sm[idx] = pi * Si[idx] + pj * Sj[idx] + ppd * d[a] * d[b];
        }
        // ---- Cholesky of Sigma_m (00 01 02 11 12 22)
        float L[6], il[3];
        L[0] = sqrtf(Sm[0]);
        il[0] = 1.0f / L[0];
        L[1] = Sm[1] * il[0];
        L[3] = Sm[2] * il[0];
        const float t11 = Sm[3] - L[1] * L[1];
        L[2] = sqrtf(fmaxf(t11, 0.f));
        il[1] = 1.0f / L[2];
        L[4] = (Sm[4] - L[3] * L[1]) * il[1];
        const float t22 = Sm[5] - L[3] * L[3] - L[4] * L[4];
        L[5] = sqrtf(fmaxf(t22, 0.f));
        il[2] = 1.0f / L[5];
        // FP32 loses about eps32 / (pivot / diagonal) of the log-determinant: a
        // ratio below 1e-2 (error above ~6e-6) sends the edge to FP64
        bool flag = !(Sm[0] > 0.f) || !(t11 > 1e-2f * Sm[3]) || !(t22 > 1e-2f * Sm[5]);
        if (policy == 1) {
            // smallest / largest scale of either endpoint below 1e-3
            const float ri = fminf(fminf(invs_i[0], invs_i[1]), invs_i[2]) /
                             fmaxf(fmaxf(invs_i[0], invs_i[1]), invs_i[2]);
            const float rj = fminf(fminf(invs_j[0], invs_j[1]), invs_j[2]) /
                             fmaxf(fmaxf(invs_j[0], invs_j[1]), invs_j[2]);
            flag = flag || ri < 1e-3f || rj < 1e-3f;
        }
        // running error estimate of dgeo:
        //   (eg + u gw + e_gmul gsum) / S + e_const
        float dgeo, eg = 0.f, gw = 0.f, gsum = 0.f, e_const = 0.f, e_gmul = 0.f;
        bool tie = false;      // mode 1: u_s within FP32 reach of pi
        if (!flag) {
            // a_c = log sqrt(det Sm / det Sigma_c) as a product of O(1) ratios
            const float ai = logf((L[0] * invs_i[0]) * (L[2] * invs_i[1]) * (L[5] * invs_i[2]));
            const float aj = logf((L[0] * invs_j[0]) * (L[2] * invs_j[1]) * (L[5] * invs_j[2]));
            const float ci = lpi + ai, cj = lpj + aj;
            // error scales of the estimate: log-determinant (Cholesky pivot
            // ratios Sm_kk / L_kk^2), the c terms, log w, the inverse scales
            const float r1 = Sm[3] * il[1] * il[1], r2 = Sm[5] * il[2] * il[2];
            const float rmax = fmaxf(1.f, fmaxf(r1, r2));
            // terms of the estimate that do not depend on the sample, added
            // after the loop: the c terms (one bound for both; every sample
            // weighs them by pi + (1 - pi) = 1), and the log-weight
            // difference through pi (1 - pi), which multiplies |g|
            e_const = U32 * (12.f + 4.f * (r1 + r2) + fabsf(lpi) + fabsf(ai) + fabsf(lpj) + fabsf(aj));
            if (MODE != 1) {
                const float e_ld = 2.f * U32 * (fabsf(i0.w) + fabsf(j0.w));
                e_const += 2.f * ppd * e_ld;
                e_gmul = ppd * e_ld;
            }
            float acc = 0.f;
            const bool est = tol > 0.f;
            for (int s = 0; s < S; s++) {
                const float z[3] = {zs[3 * s], zs[3 * s + 1], zs[3 * s + 2]};
                const float zz = z[0] * z[0] + z[1] * z[1] + z[2] * z[2];
                // x = x_i.  Error terms are formed as soon as their inputs
                // exist (first-order rounding of each Mahalanobis term:
                // offsets of size |d| + |y| through 1/s or 1/L, and q itself;
                // each entering its log-sum-exp by its weight)
                float gi, e_gi = 0.f;
                {
                    float yi[3];
                    sym_sqrt_apply(Rm, invs_i, z, yi);
                    const float vi = absmax3(d) + absmax3(yi);
                    float v1[3] = {d[0] + yi[0], d[1] + yi[1], d[2] + yi[2]};
                    float v2[3] = {pj * d[0] + yi[0], pj * d[1] + yi[1], pj * d[2] + yi[2]};
                    const float qj = maha_splat(Rn, invs_j, v1);
                    const float qmi = MODE == 2 ? 0.f : maha_chol(L, il, v2);
                    const float A1 = ci - 0.5f * zz, B1 = cj - 0.5f * qj;
                    float wa1;
                    const float l1 = lse2w(A1, B1, wa1);
                    gi = l1 + (MODE == 2 ? 1.5f : 0.5f * qmi);
                    if (est) {
                        const float imx_j = fmaxf(fmaxf(invs_j[0], invs_j[1]), invs_j[2]);
                        const float e_qj = 8.f * U32 * sqrt_nn(qj) * vi * imx_j + 2.f * U32 * qj;
                        const float ilmx = fmaxf(fmaxf(il[0], il[1]), il[2]);
                        const float e_qm = MODE == 2 ? 0.f : 8.f * U32 * sqrt_nn(qmi) * vi * ilmx + 4.f * U32 * rmax * qmi;
                        // rounding of the log-sum-exp inputs, weighted, is within
                        // |l| + 1 (l = lse >= the larger input), its output within |l|
                        e_gi = (1.f - wa1) * 0.5f * e_qj + 0.5f * e_qm + U32 * (2.f * fabsf(l1) + 1.f + qmi);
                    }
                }
                // x = x_j
                float gj, e_gj = 0.f;
                {
                    float yj[3];
                    sym_sqrt_apply(Rn, invs_j, z, yj);
                    const float vj = absmax3(d) + absmax3(yj);
                    float w1[3] = {yj[0] - d[0], yj[1] - d[1], yj[2] - d[2]};
                    float w2[3] = {yj[0] - pi * d[0], yj[1] - pi * d[1], yj[2] - pi * d[2]};
                    const float qi = maha_splat(Rm, invs_i, w1);
                    const float qmj = MODE == 2 ? 0.f : maha_chol(L, il, w2);
                    const float A2 = ci - 0.5f * qi, B2 = cj - 0.5f * zz;
                    float wa2;
                    const float l2 = lse2w(A2, B2, wa2);
                    gj = l2 + (MODE == 2 ? 1.5f : 0.5f * qmj);
                    if (est) {
                        const float imx_i = fmaxf(fmaxf(invs_i[0], invs_i[1]), invs_i[2]);
                        const float e_qi = 8.f * U32 * sqrt_nn(qi) * vj * imx_i + 2.f * U32 * qi;
                        const float ilmx = fmaxf(fmaxf(il[0], il[1]), il[2]);
                        const float e_qm = MODE == 2 ? 0.f : 8.f * U32 * sqrt_nn(qmj) * vj * ilmx + 4.f * U32 * rmax * qmj;
                        e_gj = wa2 * 0.5f * e_qi + 0.5f * e_qm + U32 * (2.f * fabsf(l2) + 1.f + qmj);
                    }
                }
                acc += MODE != 1 ? (pi * gi + pj * gj) : (us[s] < pi ? gi : gj);
                if (est) {
                    if (MODE != 1) {
                        eg += pi * e_gi + pj * e_gj;
                        gw += pi * fabsf(gi) + pj * fabsf(gj);
                        gsum += fabsf(gi) + fabsf(gj);
                    } else {
                        const bool first = us[s] < pi;
                        eg += first ? e_gi : e_gj;
                        gw += fabsf(first ? gi : gj);
                        tie = tie || fabsf(us[s] - pi) <= 1e-5f;
                    }
                }
            }
            dgeo = acc / (float)S;
        } else {
            dgeo = 0.f;  // evaluated in FP64 by k_edge_cost64 from the list below
        }
        const float c = lg * dgeo + la * dapp;
        if (tol > 0.f && !flag) {
            // keep the FP32 cost only when twice its error estimate is within
            // tol max(|C|, 1); D_app: F/4 + 4 roundings per lane sum, 16 in all
            const float E = lg * ((eg + U32 * gw + e_gmul * gsum) / (float)S + e_const) + la * 16.f * U32 * dapp +
                            U32 * fabsf(c);
            flag = tie || !(2.f * E <= tol * fmaxf(fabsf(c), 1.f));
        }
        // flagged edges go to the FP64 list (one atomic per warp)
        const unsigned am = __activemask();
        const unsigned fm = __ballot_sync(am, flag);
        if (fm) {
            const int first = __ffs(fm) - 1;
            unsigned long long at = 0;
            if (lane == first) at = atomicAdd(fp64_count, (unsigned long long)__popc(fm));
            at = __shfl_sync(am, at, first);
            if (flag) fp64_list[at + __popc(fm & ((1u << lane) - 1u))] = (int32_t)e;
        }
        if (flag) continue;
        cost_slot[sl] = c;
        if (er.w >= 0) cost_slot[er.w] = c;
        else if (er.w <= -2) revcost[-2 - er.w] = c;
        if (cost_out) cost_out[e] = c;
    }
}

// FP64 evaluation of the flagged edges: D_geo and D_app in FP64, the cost
// rounded once to FP32.
template <bool F64>
__global__ void k_edge_cost_x(const int32_t *__restrict__ list, const unsigned long long *__restrict__ count,
                              const int4 *__restrict__ erec, const float *__restrict__ zs,
                              const float *__restrict__ us, int S, int mode, float lg, float la,
                              const float *__restrict__ xyz, const float *__restrict__ ls,
                              const float *__restrict__ rot, const float *__restrict__ logit,
                              const float *__restrict__ sh, int F,
                              float *__restrict__ cost_slot, float *__restrict__ revcost,
                              float *__restrict__ cost_out) {
    const int64_t cnt = (int64_t)*count;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = list[t];
        const int4 er = erec[e];
        const float c = F64 ? cost_fp64(xyz, ls, rot, logit, sh, F, er.y, er.z, S, zs, us, mode, lg, la)
                            : cost_ff(xyz, ls, rot, logit, sh, F, er.y, er.z, S, zs, us, mode, lg, la);
        cost_slot[er.x] = c;
        if (er.w >= 0) cost_slot[er.w] = c;
        else if (er.w <= -2) revcost[-2 - er.w] = c;
        if (cost_out) cost_out[e] = c;
    }
}

// ---------------------------------------------------------------- near ties
// Two adjacent edges whose costs are within the accuracy contract of each
// other (see the file header) are both recomputed in FP64.
__device__ __forceinline__ bool near_tie(float a, float b, float tol) {
    return fabsf(a - b) <= tol * (fmaxf(fabsf(a), 1.f) + fmaxf(fabsf(b), 1.f));
}

// mark slot s; a slot marked for the first time goes to the refine list
__device__ __forceinline__ void mark_slot(uint32_t *bits, int32_t s, int32_t *list,
                                          unsigned long long *cnt) {
    const uint32_t bit = 1u << (s & 31);
    const uint32_t old = atomicOr(bits + (s >> 5), bit);
    if (!(old & bit)) list[atomicAdd(cnt, 1ull)] = s;
}

// Ascending sort of N register keys by a bitonic network (static indices).
template <int N>
__device__ __forceinline__ void sort_asc_u32(uint32_t (&a)[N]) {
#pragma unroll
    for (int k = 2; k <= N; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < N; i++) {
                const int l = i ^ j;
                if (l > i) {
                    const uint32_t x = a[i], y = a[l];
                    const bool up = (i & k) == 0;
                    a[i] = up ? min(x, y) : max(x, y);
                    a[l] = up ? max(x, y) : min(x, y);
                }
            }
}

// Exact pairwise marks of one vertex (any slot width, any number of in-slots).
template <int KM>
__device__ __forceinline__ void near_ties_pairwise(const float (&c)[KM], int64_t base, int32_t r0,
                                                   int32_t r1, const float *__restrict__ revcost,
                                                   const int32_t *__restrict__ rev, float tol,
                                                   uint32_t *bits, int32_t *list,
                                                   unsigned long long *cnt) {
    uint32_t own = 0;  // own slots to mark
#pragma unroll
    for (int a = 0; a < KM; a++)
#pragma unroll
        for (int b = a + 1; b < KM; b++)
            if (near_tie(c[a], c[b], tol)) own |= (1u << a) | (1u << b);
    for (int32_t r = r0; r < r1; r++) {
        const float cr = __ldg(revcost + r);
        bool hit = false;
#pragma unroll
        for (int a = 0; a < KM; a++)
            if (near_tie(c[a], cr, tol)) {
                own |= 1u << a;
                hit = true;
            }
        for (int32_t r2 = r + 1; r2 < r1; r2++) {
            if (near_tie(cr, __ldg(revcost + r2), tol)) {
                hit = true;
                mark_slot(bits, __ldg(rev + r2), list, cnt);
            }
        }
        if (hit) mark_slot(bits, __ldg(rev + r), list, cnt);
    }
    while (own) {
        const int a = __ffs(own) - 1;
        own &= own - 1;
        mark_slot(bits, (int32_t)(base + a), list, cnt);
    }
}

// decoded value of a packed sort key (low bits hold a slot index)
template <int K>
__device__ __forceinline__ float key_value(uint32_t k) {
    return order_bits_float(k & ~(uint32_t)(K - 1));
}

// One thread per vertex v: the costs of its K slots and of its in-slots
// (non-mutual edges of other vertices that point at v) are compared.
// For K in {4, 8, 16, 32} the K own costs are sorted (slot index packed into
// the low log2(K) bits of the orderable key, which moves a value by under K
// ulp) and only sorted neighbours are compared, with the threshold widened
// by 1e-3 of itself and by 2K ulp.  Sorted neighbours suffice: if two costs
// a < c are in near tie, every cost b between them is within the same
// distance of a and of c, and with tol <= 1e-4 all of m_a, m_b, m_c =
// max(|.|, 1) lie within 3 tol (< 1e-3) of each other, so each consecutive pair of the
// chain passes the widened test (marking a superset).  An in-slot cost is
// placed into the sorted own costs (binary search over shared memory) and
// compared with its two neighbours there, by the same chain argument; in-slot
// pairs are compared directly.  Other K: every pair is compared.
template <int K>
__global__ void __launch_bounds__(128)
    k_near_ties(int64_t n, int kk, const float *__restrict__ cost_slot,
                const int32_t *__restrict__ rev_ptr, const int32_t *__restrict__ rev,
                const float *__restrict__ revcost, float tol, uint32_t *bits, int32_t *list,
                unsigned long long *cnt) {
    constexpr int KM = K > 0 ? K : NGS_MAX_K;
    constexpr int KS = K > 0 ? K : 1;
    constexpr uint32_t IMASK = K > 0 ? (uint32_t)K - 1u : 0u;
    __shared__ uint32_t skey[KS][128];  // sorted own keys, one column per thread
    const float tw = tol * 1.001f;
    const float ulps = 2.f * KM * 1.2e-7f;
    auto close = [&](float x, float y) {  // widened near-tie test
        const float mx = fmaxf(fabsf(x), 1.f), my = fmaxf(fabsf(y), 1.f);
        return fabsf(x - y) <= tw * (mx + my) + ulps * fmaxf(mx, my);
    };
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t base = v * kk;
        const int32_t r0 = rev_ptr[v], r1 = rev_ptr[v + 1];
        if (K == 0) {
            float c[KM];
#pragma unroll
            for (int t = 0; t < KM; t++) c[t] = t < kk ? cost_slot[base + t] : NAN;
            near_ties_pairwise<KM>(c, base, r0, r1, revcost, rev, tol, bits, list, cnt);
            continue;
        }
        uint32_t key[KS];
        {
            const float4 *c4 = (const float4 *)(cost_slot + base);
#pragma unroll
            for (int t = 0; t < KS / 4; t++) {
                const float4 x = __ldg(c4 + t);
                key[4 * t] = (cost_order_bits(x.x) & ~IMASK) | (uint32_t)(4 * t);
                key[4 * t + 1] = (cost_order_bits(x.y) & ~IMASK) | (uint32_t)(4 * t + 1);
                key[4 * t + 2] = (cost_order_bits(x.z) & ~IMASK) | (uint32_t)(4 * t + 2);
                key[4 * t + 3] = (cost_order_bits(x.w) & ~IMASK) | (uint32_t)(4 * t + 3);
            }
        }
        sort_asc_u32<KS>(key);
        uint32_t own = 0;  // own slots to mark
        float prev = key_value<KS>(key[0]);
#pragma unroll
        for (int a = 0; a + 1 < KS; a++) {
            const float cur = key_value<KS>(key[a + 1]);
            if (close(prev, cur)) own |= (1u << (key[a] & IMASK)) | (1u << (key[a + 1] & IMASK));
            prev = cur;
        }
        if (r1 > r0) {
#pragma unroll
            for (int a = 0; a < KS; a++) skey[a][threadIdx.x] = key[a];
            for (int32_t r = r0; r < r1; r++) {
                const float cr = __ldg(revcost + r);
                const uint32_t kr = cost_order_bits(cr);
                // first sorted own key above kr, then its two neighbours
                int lo = 0, hi = KS;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (skey[mid][threadIdx.x] <= kr) lo = mid + 1; else hi = mid;
                }
                bool hit = false;
                if (lo > 0) {
                    const uint32_t kb = skey[lo - 1][threadIdx.x];
                    if (close(key_value<KS>(kb), cr)) { own |= 1u << (kb & IMASK); hit = true; }
                }
                if (lo < KS) {
                    const uint32_t ka = skey[lo][threadIdx.x];
                    if (close(key_value<KS>(ka), cr)) { own |= 1u << (ka & IMASK); hit = true; }
                }
                for (int32_t r2 = r + 1; r2 < r1; r2++) {
                    if (near_tie(cr, __ldg(revcost + r2), tol)) {
                        hit = true;
                        mark_slot(bits, __ldg(rev + r2), list, cnt);
                    }
                }
                if (hit) mark_slot(bits, __ldg(rev + r), list, cnt);
            }
        }
        while (own) {
            const int a = __ffs(own) - 1;
            own &= own - 1;
            mark_slot(bits, (int32_t)(base + a), list, cnt);
        }
    }
}

__device__ __forceinline__ uint32_t cid_at(const int32_t *cid, int64_t v) {
    return cid ? (uint32_t)cid[v] : (uint32_t)v;
}

// FP64 cost of the edge of each listed slot, into both slots of a mutual
// edge and, for the C-ABI view, into its lexicographic position.
template <bool F64>
__global__ void k_refine_costs(const int32_t *__restrict__ list, const unsigned long long *__restrict__ count,
                               int kk, const int32_t *__restrict__ nbr, const int32_t *__restrict__ cid,
                               const float *__restrict__ zs, const float *__restrict__ us, int S,
                               int mode, float lg, float la, const float *__restrict__ xyz,
                               const float *__restrict__ ls, const float *__restrict__ rot,
                               const float *__restrict__ logit, const float *__restrict__ sh, int F,
                               float *cost_slot, const int32_t *__restrict__ rev_ptr,
                               const int32_t *__restrict__ rev, float *revcost,
                               const int32_t *__restrict__ elo,
                               const int32_t *__restrict__ ehi, int64_t m, float *cost_out) {
    const int64_t cnt = (int64_t)*count;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = list[t];
        const int64_t a = s / kk, b = nbr[s];
        const uint32_t ca = cid_at(cid, a), cb = cid_at(cid, b);
        const int64_t lo = ca < cb ? a : b, hi = ca < cb ? b : a;
        const float c = F64 ? cost_fp64(xyz, ls, rot, logit, sh, F, lo, hi, S, zs, us, mode, lg, la)
                            : cost_ff(xyz, ls, rot, logit, sh, F, lo, hi, S, zs, us, mode, lg, la);
        cost_slot[s] = c;
        bool mutual = false;
        for (int q = 0; q < kk; q++)  // the mirror slot of a mutual edge
            if (nbr[b * kk + q] == (int32_t)a) {
                cost_slot[b * kk + q] = c;
                mutual = true;
            }
        if (!mutual)  // the in-edge entry of b
            for (int32_t r = rev_ptr[b]; r < rev_ptr[b + 1]; r++)
                if (rev[r] == s) revcost[r] = c;
        if (cost_out) {
            // lexicographic position of (lo, hi) in canonical ids
            const uint64_t key = ((uint64_t)(ca < cb ? ca : cb) << 32) | (ca < cb ? cb : ca);
            int64_t x = 0, y = m;
            while (x < y) {
                const int64_t mid = (x + y) >> 1;
                const uint64_t km = ((uint64_t)(uint32_t)elo[mid] << 32) | (uint32_t)ehi[mid];
                if (km < key) x = mid + 1; else y = mid;
            }
            if (x < m) cost_out[x] = c;
        }
    }
}

__global__ void k_costs_to_slots(const int4 *__restrict__ erec_lex, int64_t m,
                                 const float *__restrict__ cost, float *cost_slot,
                                 float *revcost) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int4 r = erec_lex[e];
        const float c = cost[e];
        cost_slot[r.x] = c;
        if (r.w >= 0) cost_slot[r.w] = c;
        else if (r.w <= -2) revcost[-2 - r.w] = c;
    }
}

__device__ __forceinline__ ff ff_from_double(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__global__ void k_ff_selftest(int op, const double *__restrict__ x, const double *__restrict__ y,
                              int64_t n, double *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const ff a = ff_from_double(x[i]), b = y ? ff_from_double(y[i]) : ff_of(0.f);
        ff r;
        switch (op) {
            case 0: r = ff_exp(a); break;
            case 1: r = ff_log(a); break;
            case 2: r = ff_log1p(a); break;
            case 3: r = ff_sqrt(a); break;
            case 4: r = ff_div(a, b); break;
            case 5: r = ff_softplus(a); break;
            case 6: r = ff_lse2(a, b); break;
            default: r = ff_mul(a, b); break;
        }
        out[i] = ff_to_double(r);
    }
}

}  // namespace

void ff_selftest(ngs_ctx *c, int op, const double *x, const double *y, int64_t n, double *out) {
    if (n <= 0) return;
    double *d = (double *)ws<uint8_t>(c, c->b_tielist, 8 * (size_t)n * 3);  // edge-cost scratch
    NGS_CHECK_CUDA(cudaMemcpyAsync(d, x, 8 * n, cudaMemcpyHostToDevice, c->st));
    if (y) NGS_CHECK_CUDA(cudaMemcpyAsync(d + n, y, 8 * n, cudaMemcpyHostToDevice, c->st));
    launch(c, "ff_selftest", dim3(grid_stride_blocks(c, n, 128, 4)), dim3(128), 0, k_ff_selftest, op,
           (const double *)d, y ? (const double *)(d + n) : (const double *)nullptr, n, d + 2 * n);
    NGS_CHECK_CUDA(cudaMemcpyAsync(out, d + 2 * n, 8 * n, cudaMemcpyDeviceToHost, c->st));
    sync_stream(c);
}

void edge_costs(ngs_ctx *c, const SplatView &s, GraphDev &g, uint32_t pass, bool lex,
                float *cost_out) {
    const int64_t m = g.n_edges;
    const int S = c->prm.mc_samples;
    c->h_pin[1] = 0;  // edges sent to FP64 by their error estimate (filled below)
    c->h_pin[5] = 0;  // slots recomputed in FP64 as near ties
    if (m <= 0) return;
    // the host buffer may go out of scope on return (put_small stages it)
    std::vector<float> h(4 * (size_t)S);
    host_mc_draws(c->prm.seed, pass, S, h.data(), h.data() + 3 * S);
    float *zs = ws<float>(c, c->b_rng, 4 * S);
    put_small(c, zs, h.data(), sizeof(float) * 4 * (size_t)S);
    const float *us = zs + 3 * S;
    float *rec = ws<float>(c, c->b_rec, s.n * REC);
    // the edge-cost kernel reads each 64-byte record as two 32-byte loads
    if ((uintptr_t)rec & 31) NGS_FAIL(NGS_ERR_CUDA, "edge_costs: record buffer not 32-byte aligned");
    launch(c, "cost_prep", dim3(grid_stride_blocks(c, s.n, 256, 8)), dim3(256), 0, k_prep, s.xyz,
           s.ls, s.rot, s.logit, s.n, rec);
    // [0] edges on the FP64 list, [1] slots on the near-tie list
    unsigned long long *cnt = (unsigned long long *)ws<uint8_t>(c, c->b_status, 64);
    int32_t *list = ws<int32_t>(c, c->b_fp64list, m);
    NGS_CHECK_CUDA(cudaMemsetAsync(cnt, 0, 16, c->st));
    const int mode = c->prm.cost_mode;
    const float tol = (float)c->prm.cost_tol;
    const float lg = c->prm.lambda_geo, la = c->prm.lambda_app;
    const int4 *er = lex ? g.erec_lex : g.erec;
    float *cout = lex ? cost_out : nullptr;
    auto kern = mode == 1 ? k_edge_cost<1> : mode == 2 ? k_edge_cost<2> : mode == 3 ? k_edge_cost<3>
                                                                                    : k_edge_cost<0>;
    launch(c, "edge_cost", dim3(grid_stride_blocks(c, m, 256, c->tune.cost_blocks_per_sm)), dim3(256), 0,
           kern, er, m, (const float *)rec, (const float *)s.sh, s.F, (const float *)zs, us, S, lg,
           la, c->prm.fp64_policy, (const float *)s.xyz, (const float *)s.ls, (const float *)s.rot,
           (const float *)s.logit, g.cost_slot, g.revcost, cout, cnt, list, tol);
    // the flagged edges (few) in extended precision, three 128-thread blocks
    // per SM (the register limit); the grid covers the worst case, threads
    // past the device count exit at once
    const bool f64 = c->prm.fp64_policy == 3;
    launch(c, "edge_cost_x", dim3(grid_stride_blocks(c, m, 128, 3)), dim3(128), 0,
           f64 ? k_edge_cost_x<true> : k_edge_cost_x<false>,
           (const int32_t *)list, (const unsigned long long *)cnt, er, (const float *)zs, us, S, mode,
           lg, la, (const float *)s.xyz, (const float *)s.ls, (const float *)s.rot,
           (const float *)s.logit, (const float *)s.sh, s.F, g.cost_slot, g.revcost, cout);
    if (tol > 0.f) {
        const int64_t ns = g.n * g.k_eff;
        uint32_t *bits = ws<uint32_t>(c, c->b_tiebits, (ns + 31) / 32);
        NGS_CHECK_CUDA(cudaMemsetAsync(bits, 0, 4 * ((ns + 31) / 32), c->st));
        int32_t *tl = ws<int32_t>(c, c->b_tielist, ns);
        const dim3 gr(grid_stride_blocks(c, g.n, 128, 16)), bl(128);
        auto nt = g.k_eff == 4 ? k_near_ties<4> : g.k_eff == 8 ? k_near_ties<8>
                : g.k_eff == 16 ? k_near_ties<16> : g.k_eff == 32 ? k_near_ties<32> : k_near_ties<0>;
        launch(c, "near_ties", gr, bl, 0, nt, g.n, g.k_eff, (const float *)g.cost_slot,
               (const int32_t *)g.rev_ptr, (const int32_t *)g.rev, (const float *)g.revcost, tol,
               bits, tl, cnt + 1);
        launch(c, "refine_costs", dim3(grid_stride_blocks(c, ns, 128, 4)), dim3(128), 0,
               f64 ? k_refine_costs<true> : k_refine_costs<false>, (const int32_t *)tl,
               (const unsigned long long *)(cnt + 1), g.k_eff,
               g.nbr, g.cid, (const float *)zs, us, S, mode, lg, la, (const float *)s.xyz,
               (const float *)s.ls, (const float *)s.rot, (const float *)s.logit,
               (const float *)s.sh, s.F, g.cost_slot, (const int32_t *)g.rev_ptr,
               (const int32_t *)g.rev, g.revcost, lex ? (const int32_t *)g.elo : nullptr,
               lex ? (const int32_t *)g.ehi : nullptr, m, cout);
    }
    get_small(c, c->h_pin + 1, cnt, 8);
    get_small(c, c->h_pin + 5, cnt + 1, 8);
}

void costs_to_slots(ngs_ctx *c, GraphDev &g, const float *cost_lex) {
    const int64_t m = g.n_edges;
    if (m <= 0) return;
    launch(c, "costs_to_slots", dim3(grid_stride_blocks(c, m, 256, 8)), dim3(256), 0,
           k_costs_to_slots, (const int4 *)g.erec_lex, m, cost_lex, g.cost_slot, g.revcost);
}
