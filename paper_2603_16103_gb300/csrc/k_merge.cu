// MPMM merge of selected pairs (Sec. 3.3) with stream compaction, the
// opacity pre-filter (Algorithm 1) and row permutations.
//
// Merge of (i, j), i the lower canonical id, written to i's output row:
//   pi = w_i / (w_i + w_j), w = (2 pi)^{3/2} alpha prod s   (Eq. vm_weights)
//   mu_m = pi mu_i + (1-pi) mu_j,  f_m = pi f_i + (1-pi) f_j
//   Sigma_m = pi Sigma_i + (1-pi) Sigma_j + pi (1-pi) d d^T,  d = mu_i - mu_j
//             (Eq. vm_cov; the dispersion term of Eq. vm_cov_decomp_short)
//   alpha_m = 1 - (1-alpha_i)(1-alpha_j)                    (Eq. vm_alpha)
//             stored as logit = log(-expm1(log T)) - log T,
//             log T = -softplus(l_i) - softplus(l_j)
//   Sigma_m = V diag(lambda) V^T -> log-scale = log(max(lambda, floor)) / 2,
//             rotation = V as a unit quaternion.
// The eigendecomposition starts with an FP32 cyclic Jacobi and is finished
// in FP64 (Sigma_m assembled in FP64, one FP64 Jacobi sweep warm-started
// from the re-orthonormalised FP32 eigenvectors).  Canonical form: eigenvalues descending,
// each eigenvector's largest-magnitude component positive, det V = +1,
// quaternion with w >= 0.
#include "ngs_device.cuh"
#include "ngs_internal.h"

namespace {

constexpr float LOG_2PI_F = 1.8378770664093453f;

template <class T>
__device__ __forceinline__ void quat_to_rot(const float *q, T *R) {
    T w = q[0], x = q[1], y = q[2], z = q[3];
    T inv = (T)1 / sqrt(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

// Sigma = R diag(s2) R^T as a full symmetric 3x3 (row-major)
template <class T>
__device__ __forceinline__ void rot_cov(const T *R, const T *s2, T *S) {
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = a; b < 3; b++) {
            T v = R[3 * a] * s2[0] * R[3 * b] + R[3 * a + 1] * s2[1] * R[3 * b + 1] +
                  R[3 * a + 2] * s2[2] * R[3 * b + 2];
            S[3 * a + b] = v;
            S[3 * b + a] = v;
        }
}

// One cyclic sweep of Jacobi rotations on symmetric A (row-major), V <- V J.
template <class T>
__device__ __forceinline__ void jacobi_sweep(T *A, T *V) {
#pragma unroll
    for (int pq = 0; pq < 3; pq++) {
        const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
        T apq = A[3 * p + q];
        if (apq == (T)0) continue;
        T app = A[3 * p + p], aqq = A[3 * q + q];
        T tau = (aqq - app) / (2 * apq);
        T t = (tau >= 0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
        T cth = (T)1 / sqrt((T)1 + t * t), sth = t * cth;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            T akp = A[3 * k + p], akq = A[3 * k + q];
            A[3 * k + p] = cth * akp - sth * akq;
            A[3 * k + q] = sth * akp + cth * akq;
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            T apk = A[3 * p + k], aqk = A[3 * q + k];
            A[3 * p + k] = cth * apk - sth * aqk;
            A[3 * q + k] = sth * apk + cth * aqk;
        }
        A[3 * p + q] = A[3 * q + p] = 0;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            T vkp = V[3 * k + p], vkq = V[3 * k + q];
            V[3 * k + p] = cth * vkp - sth * vkq;
            V[3 * k + q] = sth * vkp + cth * vkq;
        }
    }
}

template <class T>
__device__ __forceinline__ T offdiag2(const T *A) {
    return A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
}
template <class T>
__device__ __forceinline__ T diag2(const T *A) {
    return A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
}

// 1/sqrt(x) for x of order one (a squared norm of a nearly unit vector): an
// FP32 estimate (relative error below 2^-22) refined by one FP64 Newton step,
// which leaves a relative error below 1e-13.
__device__ __forceinline__ double rsqrt64(double x) {
    const double y = (double)rsqrtf((float)x);
    return y * (1.5 - 0.5 * x * y * y);
}

__device__ __forceinline__ void quat_rot64(const float *q, double *R) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    const double inv = rsqrt64(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

// One FP64 Jacobi sweep on a nearly diagonal symmetric B (upper triangle
// b[0..5] = 00 01 02 11 12 22), V <- V J, B <- J^T B J.  When the
// off-diagonal entry is tiny against the diagonal gap the rotation is the
// small-angle one, t = b_pq / (b_qq - b_pp) (in FP32: its relative error only
// scales the residual), c = 1 - t^2/2, s = t c, orthogonal to O(t^4); other
// rotations use the exact formula in FP64.  Only the entries the rotation
// changes are updated: b_pp, b_qq, b_rp, b_rq (r the third index).
__device__ __forceinline__ void refine_sweep64(double *b, double *V) {
#pragma unroll
    for (int pq = 0; pq < 3; pq++) {
        const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
        // upper-triangle slots of (p,p), (q,q), (p,q), (r,p), (r,q), r = 3 - p - q
        const int ipp = p == 0 ? 0 : 3, iqq = q == 1 ? 3 : 5;
        const int ipq = pq == 0 ? 1 : (pq == 1 ? 2 : 4);
        const int irp = pq == 0 ? 2 : 1;  // (2,0) / (1,0) / (0,1)
        const int irq = pq == 2 ? 2 : 4;  // (2,1) / (1,2) / (0,2)
        const double apq = b[ipq];
        if (apq == 0.0) continue;
        const double app = b[ipp], aqq = b[iqq];
        const double diff = aqq - app;
        double c, s;
        if (fabs(apq) < 1e-4 * fabs(diff)) {
            const double t = (double)((float)apq / (float)diff);
            c = 1.0 - 0.5 * t * t;
            s = t * c;
        } else {
            const double tau = diff / (2.0 * apq);
            const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
        }
        const double cc = c * c, ss = s * s, cs2 = 2.0 * c * s;
        const double arp = b[irp], arq = b[irq];
        b[ipp] = cc * app - cs2 * apq + ss * aqq;
        b[iqq] = ss * app + cs2 * apq + cc * aqq;
        b[ipq] = 0.0;
        b[irp] = c * arp - s * arq;
        b[irq] = s * arp + c * arq;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const double vkp = V[3 * k + p], vkq = V[3 * k + q];
            V[3 * k + p] = c * vkp - s * vkq;
            V[3 * k + q] = s * vkp + c * vkq;
        }
    }
}

// Sigma = R diag(s2) R^T in FP64 from an FP64 rotation and FP32 squared
// scales, upper triangle (00 01 02 11 12 22)
__device__ __forceinline__ void rot_cov6_64(const double *R, const float *s2, double *S6) {
    double Rs[9];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int k = 0; k < 3; k++) Rs[3 * a + k] = R[3 * a + k] * (double)s2[k];
    int idx = 0;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = a; b < 3; b++, idx++)
            S6[idx] = Rs[3 * a] * R[3 * b] + Rs[3 * a + 1] * R[3 * b + 1] + Rs[3 * a + 2] * R[3 * b + 2];
}

// canonical eigen form + quaternion (w >= 0)
__device__ void canonical_quat(double *lam, double *V, float *q_out) {
    // sort descending (3-element network), permuting columns
#define SWAPC(a, b)                                                           \
    if (lam[b] > lam[a]) {                                                    \
        double t = lam[a]; lam[a] = lam[b]; lam[b] = t;                       \
        for (int r = 0; r < 3; r++) {                                         \
            double u = V[3 * r + a]; V[3 * r + a] = V[3 * r + b]; V[3 * r + b] = u; \
        }                                                                     \
    }
    SWAPC(0, 1)
    SWAPC(0, 2)
    SWAPC(1, 2)
#undef SWAPC
    for (int cidx = 0; cidx < 3; cidx++) {
        int best = 0;
        for (int r = 1; r < 3; r++)
            if (fabs(V[3 * r + cidx]) > fabs(V[3 * best + cidx])) best = r;
        if (V[3 * best + cidx] < 0)
            for (int r = 0; r < 3; r++) V[3 * r + cidx] = -V[3 * r + cidx];
    }
    // det V = +-1: its sign in FP32
    float Vf[9];
#pragma unroll
    for (int k = 0; k < 9; k++) Vf[k] = (float)V[k];
    const float det = Vf[0] * (Vf[4] * Vf[8] - Vf[5] * Vf[7]) - Vf[1] * (Vf[3] * Vf[8] - Vf[5] * Vf[6]) +
                      Vf[2] * (Vf[3] * Vf[7] - Vf[4] * Vf[6]);
    if (det < 0.f)
        for (int r = 0; r < 3; r++) V[3 * r + 2] = -V[3 * r + 2];
    // rotation matrix -> quaternion (FP32), pivot on the largest of trace and diagonal
    float R[9];
#pragma unroll
    for (int k = 0; k < 9; k++) R[k] = (float)V[k];
    const float tr = R[0] + R[4] + R[8];
    float w, x, y, z;
    if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
        const float r = sqrtf(1.0f + tr), h = 0.5f / r;
        w = 0.5f * r; x = (R[7] - R[5]) * h; y = (R[2] - R[6]) * h; z = (R[3] - R[1]) * h;
    } else if (R[0] >= R[4] && R[0] >= R[8]) {
        const float r = sqrtf(1.0f + R[0] - R[4] - R[8]), h = 0.5f / r;
        x = 0.5f * r; w = (R[7] - R[5]) * h; y = (R[1] + R[3]) * h; z = (R[2] + R[6]) * h;
    } else if (R[4] >= R[8]) {
        const float r = sqrtf(1.0f - R[0] + R[4] - R[8]), h = 0.5f / r;
        y = 0.5f * r; w = (R[2] - R[6]) * h; x = (R[1] + R[3]) * h; z = (R[5] + R[7]) * h;
    } else {
        const float r = sqrtf(1.0f - R[0] - R[4] + R[8]), h = 0.5f / r;
        z = 0.5f * r; w = (R[3] - R[1]) * h; x = (R[2] + R[6]) * h; y = (R[5] + R[7]) * h;
    }
    if (w < 0.f) { w = -w; x = -x; y = -y; z = -z; }
    const float inv = rsqrtf(w * w + x * x + y * y + z * z);
    q_out[0] = w * inv; q_out[1] = x * inv;
    q_out[2] = y * inv; q_out[3] = z * inv;
}

struct Rows {
    const float *xyz, *ls, *rot, *logit, *sh;
};
struct WRows {
    float *xyz, *ls, *rot, *logit, *sh;
};

__device__ __forceinline__ void copy_row(const Rows &in, int64_t a, const WRows &out, int64_t b,
                                         int F) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
        out.xyz[3 * b + k] = in.xyz[3 * a + k];
        out.ls[3 * b + k] = in.ls[3 * a + k];
    }
#pragma unroll
    for (int k = 0; k < 4; k++) out.rot[4 * b + k] = in.rot[4 * a + k];
    out.logit[b] = in.logit[a];
    if ((F & 3) == 0) {
        const float4 *s = (const float4 *)(in.sh + a * F);
        float4 *d = (float4 *)(out.sh + b * F);
        for (int t = 0; t < F / 4; t++) d[t] = s[t];
    } else {
        for (int t = 0; t < F; t++) out.sh[b * F + t] = in.sh[a * F + t];
    }
}

// Row moves with one thread per 16-byte SH chunk plus one thread for the 11
// scalar fields, so each row's SH is read and written by consecutive lanes.
// mode 0: out[pos[v]] = in[v] where keep[v]; 1: out[dst[v]] = in[v];
// 2: out[v] = in[src[v]].
__device__ __forceinline__ void move_chunk(const Rows &in, int64_t a, const WRows &out, int64_t b,
                                           int F, int ch) {
    const int nch = F >> 2;
    if (ch < nch) {
        ((float4 *)(out.sh + b * F))[ch] = __ldg((const float4 *)(in.sh + a * F) + ch);
    } else {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            out.xyz[3 * b + k] = in.xyz[3 * a + k];
            out.ls[3 * b + k] = in.ls[3 * a + k];
        }
        *(float4 *)(out.rot + 4 * b) = *(const float4 *)(in.rot + 4 * a);
        out.logit[b] = in.logit[a];
    }
}

// merge rows i and j of `in` into row o of `out`; returns 1 if an eigenvalue
// was raised to the floor
__device__ int merge_pair(const Rows &in, int64_t i, int64_t j, const WRows &out, int64_t o, int F,
                          double eig_floor, int policy) {
    float li = in.logit[i], lj = in.logit[j];
    float lsi[3], lsj[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        lsi[a] = in.ls[3 * i + a];
        lsj[a] = in.ls[3 * j + a];
    }
    const float lwi = 1.5f * LOG_2PI_F - softplusf(-li) + (lsi[0] + lsi[1] + lsi[2]);
    const float lwj = 1.5f * LOG_2PI_F - softplusf(-lj) + (lsj[0] + lsj[1] + lsj[2]);
    const float ld = lwi - lwj;
    const float pi = expf(-softplusf(-ld)), pj = expf(-softplusf(ld));
    float mi[3], mj[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        mi[a] = in.xyz[3 * i + a];
        mj[a] = in.xyz[3 * j + a];
        out.xyz[3 * o + a] = pi * mi[a] + pj * mj[a];
    }
    // appearance
    if ((F & 3) == 0) {
        const float4 *fi = (const float4 *)(in.sh + i * F), *fj = (const float4 *)(in.sh + j * F);
        float4 *fo = (float4 *)(out.sh + o * F);
        for (int t = 0; t < F / 4; t++) {
            float4 a = fi[t], b = fj[t];
            fo[t] = make_float4(pi * a.x + pj * b.x, pi * a.y + pj * b.y, pi * a.z + pj * b.z,
                                pi * a.w + pj * b.w);
        }
    } else {
        for (int t = 0; t < F; t++) out.sh[o * F + t] = pi * in.sh[i * F + t] + pj * in.sh[j * F + t];
    }
    // opacity union in the log-transmittance form
    const float logT = -softplusf(li) - softplusf(lj);
    out.logit[o] = logf(-expm1f(logT)) - logT;
    // covariance: FP32 pass
    float qi[4], qj[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        qi[k] = in.rot[4 * i + k];
        qj[k] = in.rot[4 * j + k];
    }
    float Ri[9], Rj[9], s2i[3], s2j[3], Si[9], Sj[9], A[9], V[9];
    quat_to_rot<float>(qi, Ri);
    quat_to_rot<float>(qj, Rj);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        s2i[a] = expf(2.f * lsi[a]);
        s2j[a] = expf(2.f * lsj[a]);
    }
    rot_cov<float>(Ri, s2i, Si);
    rot_cov<float>(Rj, s2j, Sj);
    const float d[3] = {mi[0] - mj[0], mi[1] - mj[1], mi[2] - mj[2]};
    const float ppd = pi * pj;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) A[3 * a + b] = pi * Si[3 * a + b] + pj * Sj[3 * a + b] + ppd * d[a] * d[b];
#pragma unroll
    for (int k = 0; k < 9; k++) V[k] = (k % 4 == 0) ? 1.f : 0.f;
    for (int sw = 0; sw < 6; sw++) {
        if (offdiag2(A) <= 1e-14f * diag2(A)) break;
        jacobi_sweep<float>(A, V);
    }
    double lam[3], V64[9];
    const float lmin = fminf(fminf(A[0], A[4]), A[8]), lmax = fmaxf(fmaxf(A[0], A[4]), A[8]);
    const bool fp64 = policy != 2 || !(lmin > 1e-4f * lmax);
    if (fp64) {
        // FP64 finish: Sigma_m assembled in FP64 (rotations normalised in FP64,
        // s^2 and pi taken from their FP32 values), rotated into the
        // re-orthonormalised FP32 eigenbasis, then one FP64 Jacobi sweep.
        double Ri64[9], Rj64[9], Si6[6], Sj6[6], S64[9];
        quat_rot64(qi, Ri64);
        quat_rot64(qj, Rj64);
        rot_cov6_64(Ri64, s2i, Si6);
        rot_cov6_64(Rj64, s2j, Sj6);
        const double pid = (double)pi, pjd = (double)pj, ppd64 = pid * pjd;
        const double dd[3] = {(double)mi[0] - mj[0], (double)mi[1] - mj[1], (double)mi[2] - mj[2]};
        {
            int idx = 0;
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = a; b < 3; b++, idx++) {
                    const double v = pid * Si6[idx] + pjd * Sj6[idx] + ppd64 * dd[a] * dd[b];
                    S64[3 * a + b] = v;
                    S64[3 * b + a] = v;
                }
        }
        // Gram-Schmidt of the FP32 eigenvectors (columns of V)
        double Q[9];
#pragma unroll
        for (int k = 0; k < 9; k++) Q[k] = V[k];
        {
            const double n0 = rsqrt64(Q[0] * Q[0] + Q[3] * Q[3] + Q[6] * Q[6]);
            Q[0] *= n0; Q[3] *= n0; Q[6] *= n0;
            const double dp = Q[0] * Q[1] + Q[3] * Q[4] + Q[6] * Q[7];
            Q[1] -= dp * Q[0]; Q[4] -= dp * Q[3]; Q[7] -= dp * Q[6];
            const double n1 = rsqrt64(Q[1] * Q[1] + Q[4] * Q[4] + Q[7] * Q[7]);
            Q[1] *= n1; Q[4] *= n1; Q[7] *= n1;
            Q[2] = Q[3] * Q[7] - Q[6] * Q[4];
            Q[5] = Q[6] * Q[1] - Q[0] * Q[7];
            Q[8] = Q[0] * Q[4] - Q[3] * Q[1];
        }
        // B = Q^T S64 Q (nearly diagonal), upper triangle
        double T[9], B[6];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++)
                T[3 * a + b] = S64[3 * a] * Q[b] + S64[3 * a + 1] * Q[3 + b] + S64[3 * a + 2] * Q[6 + b];
        {
            int idx = 0;
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = a; b < 3; b++, idx++)
                    B[idx] = Q[a] * T[b] + Q[3 + a] * T[3 + b] + Q[6 + a] * T[6 + b];
        }
        refine_sweep64(B, Q);
        lam[0] = B[0]; lam[1] = B[3]; lam[2] = B[5];
#pragma unroll
        for (int k = 0; k < 9; k++) V64[k] = Q[k];
    } else {
        lam[0] = A[0]; lam[1] = A[4]; lam[2] = A[8];
#pragma unroll
        for (int k = 0; k < 9; k++) V64[k] = V[k];
    }
    float q[4];
    canonical_quat(lam, V64, q);
    int hits = 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        double l = lam[a];
        if (!(l > eig_floor)) {
            l = eig_floor;
            hits = 1;
        }
        out.ls[3 * o + a] = 0.5f * logf((float)l);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) out.rot[4 * o + k] = q[k];
    return hits;
}

__global__ void k_keep_flags(int64_t n, const int32_t *__restrict__ role, int32_t *keep,
                             int32_t *mflag) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = role[v];
        keep[v] = r != -2;
        mflag[v] = r >= 0;
    }
}

__global__ void k_copy_kept(Rows in, WRows out, int64_t n, int F, const int32_t *__restrict__ role,
                            const int32_t *__restrict__ pos) {
    if ((F & 3) == 0) {
        const int per = (F >> 2) + 1;
        const int64_t total = n * per;
        for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
             t += (int64_t)gridDim.x * blockDim.x) {
            const int64_t v = t / per;
            if (role[v] == -1) move_chunk(in, v, out, pos[v], F, (int)(t - v * per));
        }
    } else {
        for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
             v += (int64_t)gridDim.x * blockDim.x)
            if (role[v] == -1) copy_row(in, v, out, pos[v], F);
    }
}

__global__ void k_list_merges(int64_t n, const int32_t *__restrict__ mflag,
                              const int32_t *__restrict__ mpos, int32_t *list) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (mflag[v]) list[mpos[v]] = (int32_t)v;
}

__global__ void k_merge(Rows in, WRows out, const int32_t *__restrict__ list, int64_t npairs, int F,
                        const int32_t *__restrict__ role, const int32_t *__restrict__ pos,
                        double eig_floor, int policy, unsigned long long *floor_hits) {
    int hits = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < npairs;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = list[t];
        hits += merge_pair(in, i, role[i], out, pos[i], F, eig_floor, policy);
    }
    if (hits) atomicAdd(floor_hits, (unsigned long long)hits);
}

__global__ void k_cid_flags(int64_t n, const int32_t *__restrict__ cid,
                            const int32_t *__restrict__ keep, int32_t *cflag) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        cflag[cid[v]] = keep[v];
}

__global__ void k_cid_update(int64_t n, const int32_t *__restrict__ cid,
                             const int32_t *__restrict__ keep, const int32_t *__restrict__ pos,
                             const int32_t *__restrict__ cscan, int32_t *cid_out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (keep[v]) cid_out[pos[v]] = cscan[cid[v]];
}

__global__ void k_pairs_role(const int32_t *__restrict__ pairs, int64_t np, int64_t n,
                             int32_t *role, int32_t *err) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = pairs[2 * p], hi = pairs[2 * p + 1];
        if (lo < 0 || hi >= n || lo >= hi) {
            atomicOr(err, 1);
            continue;
        }
        if (atomicCAS(&role[lo], -1, hi) != -1) atomicOr(err, 2);
        if (atomicCAS(&role[hi], -1, -2) != -1) atomicOr(err, 2);
    }
}

__global__ void k_partner_role(int64_t n, const int32_t *__restrict__ partner,
                               const int32_t *__restrict__ cid, int32_t *role) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = partner[v];
        int32_t r = -1;
        if (u >= 0) {
            uint32_t cv = cid ? (uint32_t)cid[v] : (uint32_t)v;
            uint32_t cu = cid ? (uint32_t)cid[u] : (uint32_t)u;
            r = cv < cu ? u : -2;
        }
        role[v] = r;
    }
}

__global__ void k_logit_keys(const float *__restrict__ logit, int64_t n, uint32_t *keys) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        keys[v] = float_order_bits(logit[v]);
}

__global__ void k_prefilter_flags(const float *__restrict__ logit, int64_t n,
                                  const uint32_t *__restrict__ med_bits, double l_tau,
                                  int32_t *keep) {
    // alpha_i >= min(tau, alpha_med)  <=>  logit_i >= min(logit(tau), logit_med)
    const double thr = fmin((double)order_bits_float(*med_bits), l_tau);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        keep[v] = (double)logit[v] >= thr;
}

// chunks [ch0, ch0 + per) of each row: F/4 SH chunks, then the scalar fields
__global__ void k_move_rows(Rows in, WRows out, int64_t n, int F, int mode,
                            const int32_t *__restrict__ keep, const int32_t *__restrict__ idx,
                            int ch0, int per) {
    const int64_t total = n * per;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = t / per;
        const int ch = ch0 + (int)(t - v * per);
        if (mode == 0) {
            if (keep[v]) move_chunk(in, v, out, idx[v], F, ch);
        } else if (mode == 1) {
            move_chunk(in, v, out, idx[v], F, ch);
        } else {
            move_chunk(in, idx[v], out, v, F, ch);
        }
    }
}

__global__ void k_compact(Rows in, WRows out, int64_t n, int F, const int32_t *__restrict__ keep,
                          const int32_t *__restrict__ pos) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (keep[v]) copy_row(in, v, out, pos[v], F);
}

__global__ void k_scatter(Rows in, WRows out, int64_t n, int F, const int32_t *__restrict__ dst) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        copy_row(in, v, out, dst[v], F);
}

__global__ void k_gather(Rows in, WRows out, int64_t n, int F, const uint32_t *__restrict__ src) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        copy_row(in, src[v], out, v, F);
}

Rows rows_of(const SplatView &s) { return Rows{s.xyz, s.ls, s.rot, s.logit, s.sh}; }
WRows wrows_of(SplatView &s) { return WRows{s.xyz, s.ls, s.rot, s.logit, s.sh}; }

}  // namespace

int64_t merge_compact(ngs_ctx *c, const SplatView &in, const int32_t *role, SplatView &out,
                      const int32_t *cid, int32_t *cid_out) {
    const int64_t n = in.n;
    out.F = in.F;
    if (n <= 0) {
        out.n = 0;
        return 0;
    }
    int32_t *keep = ws<int32_t>(c, c->b_keep, n + 1);
    int32_t *pos = ws<int32_t>(c, c->b_pos, n + 1);
    int32_t *mflag = ws<int32_t>(c, c->b_flag, 2 * (n + 1));
    int32_t *mpos = mflag + (n + 1);
    const unsigned grid = grid_stride_blocks(c, n, 256, 8);
    launch(c, "keep_flags", dim3(grid), dim3(256), 0, k_keep_flags, n, role, keep, mflag);
    scan_i32(c, keep, pos, n);
    scan_i32(c, mflag, mpos, n);
    NGS_CHECK_CUDA(cudaMemcpyAsync(c->h_pin, pos + n, 4, cudaMemcpyDeviceToHost, c->st));
    NGS_CHECK_CUDA(cudaMemcpyAsync((int32_t *)c->h_pin + 1, mpos + n, 4, cudaMemcpyDeviceToHost, c->st));
    sync_stream(c);
    const int64_t nout = ((int32_t *)c->h_pin)[0];
    const int64_t npairs = ((int32_t *)c->h_pin)[1];
    int32_t *list = ws<int32_t>(c, c->b_pairs, npairs);
    launch(c, "list_merges", dim3(grid), dim3(256), 0, k_list_merges, n, (const int32_t *)mflag,
           (const int32_t *)mpos, list);
    Rows ri = rows_of(in);
    WRows wo = wrows_of(out);
    launch(c, "copy_kept", dim3(grid_stride_blocks(c, n * ((in.F >> 2) + 1), 256, 16)), dim3(256),
           0, k_copy_kept, ri, wo, n, in.F, role, (const int32_t *)pos);
    unsigned long long *hits = (unsigned long long *)ws<uint8_t>(c, c->b_status, 64) + 1;
    NGS_CHECK_CUDA(cudaMemsetAsync(hits, 0, 8, c->st));
    if (npairs > 0)
        launch(c, "merge", dim3(grid_stride_blocks(c, npairs, 128, 16)), dim3(128), 0, k_merge, ri,
               wo, (const int32_t *)list, npairs, in.F, role, (const int32_t *)pos,
               c->prm.eig_floor, c->prm.fp64_policy, hits);
    NGS_CHECK_CUDA(cudaMemcpyAsync(c->h_pin + 2, hits, 8, cudaMemcpyDeviceToHost, c->st));
    if (cid) {
        int32_t *cflag = ws<int32_t>(c, c->b_cflag, n + 1);
        int32_t *cscan = ws<int32_t>(c, c->b_cscan, n + 1);
        launch(c, "cid_flags", dim3(grid), dim3(256), 0, k_cid_flags, n, cid, (const int32_t *)keep,
               cflag);
        scan_i32(c, cflag, cscan, n);
        launch(c, "cid_update", dim3(grid), dim3(256), 0, k_cid_update, n, cid,
               (const int32_t *)keep, (const int32_t *)pos, (const int32_t *)cscan, cid_out);
    }
    sync_stream(c);
    c->floor_hits += (int64_t)c->h_pin[2];
    out.n = nout;
    return nout;
}

bool pairs_to_role(ngs_ctx *c, const int32_t *pairs, int64_t npairs, int64_t n, int32_t *role) {
    NGS_CHECK_CUDA(cudaMemsetAsync(role, 0xff, sizeof(int32_t) * n, c->st));  // -1
    int32_t *err = (int32_t *)ws<uint8_t>(c, c->b_status, 64) + 8;
    NGS_CHECK_CUDA(cudaMemsetAsync(err, 0, 4, c->st));
    if (npairs > 0)
        launch(c, "pairs_role", dim3(grid_stride_blocks(c, npairs, 256, 8)), dim3(256), 0,
               k_pairs_role, pairs, npairs, n, role, err);
    NGS_CHECK_CUDA(cudaMemcpyAsync(c->h_pin + 3, err, 4, cudaMemcpyDeviceToHost, c->st));
    sync_stream(c);
    return *(int32_t *)(c->h_pin + 3) == 0;
}

void partner_to_role(ngs_ctx *c, const int32_t *partner, const int32_t *cid, int64_t n,
                     int32_t *role) {
    launch(c, "partner_role", dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0, k_partner_role,
           n, partner, cid, role);
}

int64_t prefilter_flags(ngs_ctx *c, const float *logit, int64_t n, double tau, int32_t *keep) {
    if (n <= 0) return 0;
    uint32_t *keys = ws<uint32_t>(c, c->b_codes, n);
    uint32_t *med = (uint32_t *)ws<uint8_t>(c, c->b_sel, 64);
    const unsigned grid = grid_stride_blocks(c, n, 256, 8);
    launch(c, "logit_keys", dim3(grid), dim3(256), 0, k_logit_keys, logit, n, keys);
    radix_select_u32(c, keys, n, (n - 1) / 2, med);
    const double l_tau = log(tau / (1.0 - tau));
    launch(c, "prefilter_flags", dim3(grid), dim3(256), 0, k_prefilter_flags, logit, n,
           (const uint32_t *)med, l_tau, keep);
    int32_t *pos = ws<int32_t>(c, c->b_pos, n + 1);
    scan_i32(c, keep, pos, n);
    NGS_CHECK_CUDA(cudaMemcpyAsync(c->h_pin, pos + n, 4, cudaMemcpyDeviceToHost, c->st));
    sync_stream(c);
    return *(int32_t *)c->h_pin;
}

static void move_rows(ngs_ctx *c, const SplatView &in, SplatView &out, int64_t n, int mode,
                      const int32_t *keep, const int32_t *idx, const char *name) {
    if (n <= 0) return;
    WRows wo = wrows_of(out);
    if ((in.F & 3) == 0 && in.F <= 64) {
        const int per = (in.F >> 2) + 1;
        launch(c, name, dim3(grid_stride_blocks(c, n * per, 256, 16)), dim3(256), 0, k_move_rows,
               rows_of(in), wo, n, in.F, mode, keep, idx, 0, per);
    } else if (mode == 0) {
        launch(c, name, dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0, k_compact, rows_of(in),
               wo, n, in.F, keep, idx);
    } else if (mode == 1) {
        launch(c, name, dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0, k_scatter, rows_of(in),
               wo, n, in.F, idx);
    } else {
        launch(c, name, dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0, k_gather, rows_of(in),
               wo, n, in.F, (const uint32_t *)idx);
    }
}

void compact_rows(ngs_ctx *c, const SplatView &in, const int32_t *keep, const int32_t *pos,
                  SplatView &out) {
    move_rows(c, in, out, in.n, 0, keep, pos, "compact_rows");
}

void scatter_rows(ngs_ctx *c, const SplatView &in, const int32_t *dst, SplatView &out) {
    move_rows(c, in, out, in.n, 1, nullptr, dst, "scatter_rows");
}

void gather_rows(ngs_ctx *c, const SplatView &in, const uint32_t *src, SplatView &out) {
    move_rows(c, in, out, out.n, 2, nullptr, (const int32_t *)src, "gather_rows");
}

void gather_rows_part(ngs_ctx *c, const SplatView &in, const uint32_t *src, SplatView &out,
                      bool sh) {
    const int64_t n = out.n;
    if (n <= 0) return;
    const int nch = in.F >> 2;
    const int ch0 = sh ? 0 : nch, per = sh ? nch : 1;
    launch(c, sh ? "gather_rows_sh" : "gather_rows", dim3(grid_stride_blocks(c, n * per, 256, 16)),
           dim3(256), 0, k_move_rows, rows_of(in), wrows_of(out), n, in.F, 2,
           (const int32_t *)nullptr, (const int32_t *)src, ch0, per);
}
