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
// in float-float arithmetic (Sigma_m assembled in float-float, one Jacobi
// sweep warm-started from the re-orthonormalised FP32 eigenvectors; see
// finish_ff), or in FP64 under fp64_policy 3 (finish_fp64).  Canonical form: eigenvalues descending,
// each eigenvector's largest-magnitude component positive, det V = +1,
// quaternion with w >= 0.
#include "ffmath.cuh"
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

// ---------------------------------------------------------------- float-float
// Extended precision (float-float) arithmetic: ffmath.cuh.

// Extended-precision finish of the eigendecomposition of Sigma_m.
//   * Q: the FP32 Jacobi eigenvectors, re-orthonormalised by Gram-Schmidt in
//     FP32, so Q^T Q = I + E with |E| ~ 1e-7.
//   * Sigma_m assembled in float-float from the FP32 inputs (rotations, s^2,
//     pi, and the exact centre difference), B = Q^T Sigma_m Q in float-float.
//   * One Jacobi sweep on the nearly diagonal B: rotation angles in FP32, the
//     updates of B in float-float, V = Q J in FP32.
// The congruence with a nearly orthonormal Q moves every eigenvalue by a
// relative |E| at most (Ostrowski's theorem), so small eigenvalues keep about
// FP32 relative accuracy however ill-conditioned Sigma_m is; the float-float
// assembly and rotation are what remove the cancellation of the FP32 pass.
__device__ __forceinline__ void finish_ff(const float *Ri, const float *Rj, const float *s2i,
                                          const float *s2j, float pi, float pj, const float *mi,
                                          const float *mj, float *V, ff *lam) {
    // Gram-Schmidt of the columns of V
    float Q[9];
    {
        const float n0 = rsqrtf(V[0] * V[0] + V[3] * V[3] + V[6] * V[6]);
        Q[0] = V[0] * n0; Q[3] = V[3] * n0; Q[6] = V[6] * n0;
        const float dp = Q[0] * V[1] + Q[3] * V[4] + Q[6] * V[7];
        float c1[3] = {V[1] - dp * Q[0], V[4] - dp * Q[3], V[7] - dp * Q[6]};
        const float n1 = rsqrtf(c1[0] * c1[0] + c1[1] * c1[1] + c1[2] * c1[2]);
        Q[1] = c1[0] * n1; Q[4] = c1[1] * n1; Q[7] = c1[2] * n1;
        Q[2] = Q[3] * Q[7] - Q[6] * Q[4];
        Q[5] = Q[6] * Q[1] - Q[0] * Q[7];
        Q[8] = Q[0] * Q[4] - Q[3] * Q[1];
    }
    // Sigma_m, upper triangle (00 01 02 11 12 22)
    ff d[3];
#pragma unroll
    for (int a = 0; a < 3; a++) d[a] = ff_two_sum(mi[a], -mj[a]);
    const ff pp = ff_prod(pi, pj);
    ff S[6];
    {
        int idx = 0;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = a; b < 3; b++, idx++) {
                ff si = ff_mulf(ff_prod(Ri[3 * a], s2i[0]), Ri[3 * b]);
                ff sj = ff_mulf(ff_prod(Rj[3 * a], s2j[0]), Rj[3 * b]);
#pragma unroll
                for (int k = 1; k < 3; k++) {
                    si = ff_add(si, ff_mulf(ff_prod(Ri[3 * a + k], s2i[k]), Ri[3 * b + k]));
                    sj = ff_add(sj, ff_mulf(ff_prod(Rj[3 * a + k], s2j[k]), Rj[3 * b + k]));
                }
                ff v = ff_add(ff_mulf(si, pi), ff_mulf(sj, pj));
                S[idx] = ff_add(v, ff_mul(ff_mul(pp, d[a]), d[b]));
            }
    }
    // T = Sigma_m Q, B = Q^T T (upper triangle)
    const int sym[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
    ff T[9], B[6];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            ff t = ff_mulf(S[sym[3 * a]], Q[b]);
            t = ff_add(t, ff_mulf(S[sym[3 * a + 1]], Q[3 + b]));
            T[3 * a + b] = ff_add(t, ff_mulf(S[sym[3 * a + 2]], Q[6 + b]));
        }
    {
        int idx = 0;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = a; b < 3; b++, idx++) {
                ff t = ff_mulf(T[b], Q[a]);
                t = ff_add(t, ff_mulf(T[3 + b], Q[3 + a]));
                B[idx] = ff_add(t, ff_mulf(T[6 + b], Q[6 + a]));
            }
    }
    // one sweep, V <- Q J
#pragma unroll
    for (int k = 0; k < 9; k++) V[k] = Q[k];
#pragma unroll
    for (int pq = 0; pq < 3; pq++) {
        const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
        // upper-triangle slots of (p,p), (q,q), (p,q), (r,p), (r,q), r = 3 - p - q
        const int ipp = p == 0 ? 0 : 3, iqq = q == 1 ? 3 : 5;
        const int ipq = pq == 0 ? 1 : (pq == 1 ? 2 : 4);
        const int irp = pq == 0 ? 2 : 1;
        const int irq = pq == 2 ? 2 : 4;
        const ff apq = B[ipq];
        if (apq.h == 0.f) continue;
        const ff app = B[ipp], aqq = B[iqq];
        const float diff = ff_add(aqq, {-app.h, -app.l}).h;
        float c, s;
        if (fabsf(apq.h) < 1e-4f * fabsf(diff)) {
            // small angle: t = b_pq / (b_qq - b_pp), c = 1 - t^2/2, s = t c
            const float t = apq.h / diff;
            c = 1.0f - 0.5f * t * t;
            s = t * c;
        } else {
            const float tau = diff / (2.0f * apq.h);
            const float t = (tau >= 0.f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
            c = rsqrtf(1.0f + t * t);
            s = t * c;
        }
        const ff cc = ff_prod(c, c), ss = ff_prod(s, s), cs2 = ff_prod(2.0f * c, s);
        const ff arp = B[irp], arq = B[irq];
        const ff mid = ff_mul(cs2, apq);
        B[ipp] = ff_add(ff_add(ff_mul(cc, app), {-mid.h, -mid.l}), ff_mul(ss, aqq));
        B[iqq] = ff_add(ff_add(ff_mul(ss, app), mid), ff_mul(cc, aqq));
        B[ipq] = {0.f, 0.f};
        B[irp] = ff_add(ff_mulf(arp, c), ff_mulf(arq, -s));
        B[irq] = ff_add(ff_mulf(arp, s), ff_mulf(arq, c));
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float vkp = V[3 * k + p], vkq = V[3 * k + q];
            V[3 * k + p] = c * vkp - s * vkq;
            V[3 * k + q] = s * vkp + c * vkq;
        }
    }
    lam[0] = B[0];
    lam[1] = B[3];
    lam[2] = B[5];
}

// FP64 finish of the eigendecomposition (fp64_policy 3): Sigma_m assembled
// in FP64 from the inputs (rotation from the quaternion, s^2 = e^{2 log s},
// pi from the weights, the centre difference), rotated into the FP32
// eigenvectors V and diagonalised by FP64 Jacobi sweeps; eigenvalues and
// eigenvectors are handed to the canonical form as float-float and FP32.
__device__ __forceinline__ void finish_fp64(const float *qi, const float *qj, const float *lsi,
                                            const float *lsj, float li, float lj, const float *mi,
                                            const float *mj, float *V, ff *lam) {
    double Ri[9], Rj[9], s2i[3], s2j[3], Si[9], Sj[9], S[9];
    quat_to_rot<double>(qi, Ri);
    quat_to_rot<double>(qj, Rj);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        s2i[a] = exp(2.0 * (double)lsi[a]);
        s2j[a] = exp(2.0 * (double)lsj[a]);
    }
    rot_cov<double>(Ri, s2i, Si);
    rot_cov<double>(Rj, s2j, Sj);
    const double lwi = -softplus_d(-(double)li) + ((double)lsi[0] + (double)lsi[1] + (double)lsi[2]);
    const double lwj = -softplus_d(-(double)lj) + ((double)lsj[0] + (double)lsj[1] + (double)lsj[2]);
    const double ld = lwi - lwj, t = exp(-fabs(ld));
    const double big = 1.0 / (1.0 + t), small = t * big;
    const double pi = ld >= 0 ? big : small, pj = ld >= 0 ? small : big;
    double d[3];
#pragma unroll
    for (int a = 0; a < 3; a++) d[a] = (double)mi[a] - (double)mj[a];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++)
            S[3 * a + b] = pi * Si[3 * a + b] + pj * Sj[3 * a + b] + pi * pj * d[a] * d[b];
    // A = Q^T S Q with Q = V (FP32 eigenvectors), then Jacobi in FP64
    double Q[9], T[9], A[9];
#pragma unroll
    for (int k = 0; k < 9; k++) Q[k] = V[k];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++)
            T[3 * a + b] = S[3 * a] * Q[b] + S[3 * a + 1] * Q[3 + b] + S[3 * a + 2] * Q[6 + b];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++)
            A[3 * a + b] = Q[a] * T[b] + Q[3 + a] * T[3 + b] + Q[6 + a] * T[6 + b];
    for (int sw = 0; sw < 8; sw++) {
        if (offdiag2(A) <= 1e-30 * diag2(A)) break;
        jacobi_sweep<double>(A, Q);
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double l = A[4 * k];
        const float h = (float)l;
        lam[k] = {h, (float)(l - (double)h)};
    }
#pragma unroll
    for (int k = 0; k < 9; k++) V[k] = (float)Q[k];
}

// canonical eigen form + quaternion (w >= 0)
__device__ void canonical_quat(ff *lam, float *V, float *q_out) {
    // sort descending (3-element network), permuting columns
#define SWAPC(a, b)                                                           \
    if (ff_gt(lam[b], lam[a])) {                                              \
        const ff t = lam[a]; lam[a] = lam[b]; lam[b] = t;                     \
        for (int r = 0; r < 3; r++) {                                         \
            float u = V[3 * r + a]; V[3 * r + a] = V[3 * r + b]; V[3 * r + b] = u; \
        }                                                                     \
    }
    SWAPC(0, 1)
    SWAPC(0, 2)
    SWAPC(1, 2)
#undef SWAPC
    for (int cidx = 0; cidx < 3; cidx++) {
        int best = 0;
        for (int r = 1; r < 3; r++)
            if (fabsf(V[3 * r + cidx]) > fabsf(V[3 * best + cidx])) best = r;
        if (V[3 * best + cidx] < 0)
            for (int r = 0; r < 3; r++) V[3 * r + cidx] = -V[3 * r + cidx];
    }
    // det V = +-1: its sign in FP32
    const float *Vf = V;
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
        out.xyz[3 * b + k] = __ldg(in.xyz + 3 * a + k);
        out.ls[3 * b + k] = __ldg(in.ls + 3 * a + k);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) out.rot[4 * b + k] = __ldg(in.rot + 4 * a + k);
    out.logit[b] = __ldg(in.logit + a);
    if ((F & 3) == 0) {
        const float4 *s = (const float4 *)(in.sh + a * F);
        float4 *d = (float4 *)(out.sh + b * F);
        for (int t = 0; t < F / 4; t++) d[t] = __ldg(s + t);
    } else {
        for (int t = 0; t < F; t++) out.sh[b * F + t] = __ldg(in.sh + a * F + t);
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
        // read-only loads first, so the eleven fields are in flight together
        float x[3], l[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            x[k] = __ldg(in.xyz + 3 * a + k);
            l[k] = __ldg(in.ls + 3 * a + k);
        }
        const float4 r = __ldg((const float4 *)(in.rot + 4 * a));
        const float o = __ldg(in.logit + a);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            out.xyz[3 * b + k] = x[k];
            out.ls[3 * b + k] = l[k];
        }
        *(float4 *)(out.rot + 4 * b) = r;
        out.logit[b] = o;
    }
}

// 32 bytes in one load (read-only path) or one store; p 32-byte aligned
__device__ __forceinline__ void ldg_v8m(const float *p, float *r) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
        : "l"(p));
}
__device__ __forceinline__ void stg_v8m(float *p, const float *r) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "l"(p), "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7]));
}
// merge rows i and j of `in` into row o of `out`; returns 1 if an eigenvalue
// was raised to the floor.  F64: the FP64 eigen finish (fp64_policy 3).
template <bool F64>
__device__ int merge_pair(const Rows &in, int64_t i, int64_t j, const WRows &out, int64_t o, int F, int sh8,
                          double eig_floor, int policy) {
    // every input field through the read-only path, so no load waits behind
    // an output store
    float li = __ldg(in.logit + i), lj = __ldg(in.logit + j);
    float lsi[3], lsj[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        lsi[a] = __ldg(in.ls + 3 * i + a);
        lsj[a] = __ldg(in.ls + 3 * j + a);
    }
    const float lwi = 1.5f * LOG_2PI_F - softplusf(-li) + (lsi[0] + lsi[1] + lsi[2]);
    const float lwj = 1.5f * LOG_2PI_F - softplusf(-lj) + (lsj[0] + lsj[1] + lsj[2]);
    const float ld = lwi - lwj;
    const float pi = expf(-softplusf(-ld)), pj = expf(-softplusf(ld));
    float mi[3], mj[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        mi[a] = __ldg(in.xyz + 3 * i + a);
        mj[a] = __ldg(in.xyz + 3 * j + a);
        out.xyz[3 * o + a] = pi * mi[a] + pj * mj[a];
    }
    // appearance: 32-byte chunks when F % 8 == 0 and both arrays are 32-byte
    // aligned (sh8), else 16-byte chunks, else scalars
    if (sh8) {
        for (int t = 0; t < F / 8; t++) {
            float a[8], b[8], r[8];
            ldg_v8m(in.sh + i * F + 8 * t, a);
            ldg_v8m(in.sh + j * F + 8 * t, b);
#pragma unroll
            for (int q = 0; q < 8; q++) r[q] = pi * a[q] + pj * b[q];
            stg_v8m(out.sh + o * F + 8 * t, r);
        }
    } else if ((F & 3) == 0) {
        const float4 *fi = (const float4 *)(in.sh + i * F), *fj = (const float4 *)(in.sh + j * F);
        float4 *fo = (float4 *)(out.sh + o * F);
        // read-only loads: the compiler may issue them ahead of the stores
        for (int t = 0; t < F / 4; t++) {
            const float4 a = __ldg(fi + t), b = __ldg(fj + t);
            fo[t] = make_float4(pi * a.x + pj * b.x, pi * a.y + pj * b.y, pi * a.z + pj * b.z,
                                pi * a.w + pj * b.w);
        }
    } else {
        for (int t = 0; t < F; t++)
            out.sh[o * F + t] = pi * __ldg(in.sh + i * F + t) + pj * __ldg(in.sh + j * F + t);
    }
    // opacity union in the log-transmittance form
    const float logT = -softplusf(li) - softplusf(lj);
    out.logit[o] = logf(-expm1f(logT)) - logT;
    // covariance: FP32 pass
    float qi[4], qj[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        qi[k] = __ldg(in.rot + 4 * i + k);
        qj[k] = __ldg(in.rot + 4 * j + k);
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
    ff lam[3];
    const float lmin = fminf(fminf(A[0], A[4]), A[8]), lmax = fmaxf(fmaxf(A[0], A[4]), A[8]);
    if (F64) {
        finish_fp64(qi, qj, lsi, lsj, li, lj, mi, mj, V, lam);
    } else if (policy != 2 || !(lmin > 1e-4f * lmax)) {
        finish_ff(Ri, Rj, s2i, s2j, pi, pj, mi, mj, V, lam);
    } else {
        lam[0] = {A[0], 0.f};
        lam[1] = {A[4], 0.f};
        lam[2] = {A[8], 0.f};
    }
    float q[4];
    canonical_quat(lam, V, q);
    const float floor_f = (float)eig_floor;
    int hits = 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float l = lam[a].h + lam[a].l;
        if (!(l > floor_f)) {
            l = floor_f;
            hits = 1;
        }
        out.ls[3 * o + a] = 0.5f * logf(l);
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

template <bool F64>
__global__ void k_merge(Rows in, WRows out, const int32_t *__restrict__ list, int64_t npairs, int F, int sh8,
                        const int32_t *__restrict__ role, const int32_t *__restrict__ pos,
                        double eig_floor, int policy, unsigned long long *floor_hits) {
    int hits = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < npairs;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = list[t];
        hits += merge_pair<F64>(in, i, role[i], out, pos[i], F, sh8, eig_floor, policy);
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
    int32_t *mflag = ws<int32_t>(c, c->b_flag, 2 * (n + 4));
    int32_t *mpos = mflag + ((n + 4) & ~(int64_t)3);  // 16-byte aligned for the vector scan
    const unsigned grid = grid_stride_blocks(c, n, 256, 8);
    launch(c, "keep_flags", dim3(grid), dim3(256), 0, k_keep_flags, n, role, keep, mflag);
    scan_i32(c, keep, pos, n);
    scan_i32(c, mflag, mpos, n);
    get_small(c, c->h_pin, pos + n, 4);
    get_small(c, (int32_t *)c->h_pin + 1, mpos + n, 4);
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
        launch(c, "merge", dim3(grid_stride_blocks(c, npairs, 128, 16)), dim3(128), 0,
               c->prm.fp64_policy == 3 ? k_merge<true> : k_merge<false>, ri,
               wo, (const int32_t *)list, npairs, in.F,
               (in.F % 8 == 0 && ((uintptr_t)ri.sh & 31) == 0 && ((uintptr_t)wo.sh & 31) == 0) ? 1 : 0,
               role, (const int32_t *)pos,
               c->prm.eig_floor, c->prm.fp64_policy, hits);
    get_small(c, c->h_pin + 2, hits, 8);
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
    get_small(c, c->h_pin + 3, err, 4);
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
    get_small(c, c->h_pin, pos + n, 4);
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
