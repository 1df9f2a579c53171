// Algorithm 1 for one or many scenes at once.
//
// All scenes' splats are concatenated into one working set, grouped by scene
// and kept in Morton order inside each scene; every stage of a pass (kNN,
// edges, costs, matching rounds, merge + compaction) runs as one launch over
// all scenes together.  Per scene:
//   * canonical ids are the ranks of its pre-filter survivors in its input
//     order (dense and contiguous per scene in the working set);
//   * the pre-filter median, the Morton frame, the cell table, the pair cap
//     P = n - target and the stop rule (n <= target, or no pair found) are
//     its own;
//   * the per-pass random numbers are those of pass p, identical for every
//     scene, so each scene's result equals ngs_simplify on it alone.
// A scene that stops is written back (canonical order) to its own arrays and
// removed from the working set before the next pass.
#include <string.h>

#include <algorithm>
#include <vector>

#include "ngs_device.cuh"
#include "ngs_internal.h"

namespace {

// scratch slots in ngs_ctx::b_eng
enum EngBuf {
    E_P, E_CNT, E_KHI, E_KLO, E_KS, E_ORD, E_ORD2, E_POS2, E_SEG, E_SHIFT, E_SID,
    E_SIDW, E_SRC, E_SSID, E_START, E_STOP, E_T1, E_T2, E_T3, E_THR, E_TMP, E_WS,
    E_COUNT
};
static_assert(E_COUNT <= 32, "ngs_ctx::b_eng has 32 slots");

struct SrcRows {
    float *xyz, *ls, *rot, *logit, *sh;
};

__device__ __forceinline__ int scene_of(const int64_t *__restrict__ start, int S, int64_t row) {
    int lo = 0, hi = S - 1;  // last scene with start <= row
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= row) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// A row moves as parts_of(F) independent parts: one per 16-byte SH chunk and
// one for the 11 scalar fields, when F is a multiple of 4 (the caller's sh is
// then 16-byte aligned); otherwise as one part.
__host__ __device__ __forceinline__ int parts_of(int F) { return (F & 3) ? 1 : (F >> 2) + 1; }

__device__ __forceinline__ void move_part(const SrcRows &a, int64_t ra, const SrcRows &b, int64_t rb,
                                          int F, int ch) {
    // source and destination never overlap: read-only loads, issued before
    // the stores
    if ((F & 3) == 0 && ch < (F >> 2)) {
        ((float4 *)(b.sh + rb * F))[ch] = __ldg((const float4 *)(a.sh + ra * F) + ch);
    } else {
        float x[3], l[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            x[k] = __ldg(a.xyz + 3 * ra + k);
            l[k] = __ldg(a.ls + 3 * ra + k);
        }
        const float4 r = __ldg((const float4 *)(a.rot + 4 * ra));
        const float o = __ldg(a.logit + ra);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            b.xyz[3 * rb + k] = x[k];
            b.ls[3 * rb + k] = l[k];
        }
        *(float4 *)(b.rot + 4 * rb) = r;
        b.logit[rb] = o;
        if (F & 3)
            for (int t = 0; t < F; t++) b.sh[rb * F + t] = __ldg(a.sh + ra * F + t);
    }
}

// concatenate the scenes' caller arrays into one working input
__global__ void k_gather_scenes(const SrcRows *__restrict__ src, const int64_t *__restrict__ start,
                                int S, int64_t n, int F, SrcRows dst) {
    const int per = parts_of(F);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * per;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / per;
        const int s = scene_of(start, S, row);
        move_part(src[s], row - start[s], dst, row, F, (int)(t - row * per));
    }
}

// write rows of stopped scenes back to their caller arrays (row = cid - base)
__global__ void k_extract(SrcRows a, int64_t n, int F, const int32_t *__restrict__ sid,
                          const int32_t *__restrict__ cid, const uint8_t *__restrict__ stop,
                          const int64_t *__restrict__ base, const SrcRows *__restrict__ out) {
    const int per = parts_of(F);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * per;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / per;
        const int s = sid[row];
        if (!stop[s]) continue;
        move_part(a, row, out[s], (int64_t)cid[row] - base[s], F, (int)(t - row * per));
    }
}

// keep rows of running scenes; their canonical ids move down by the rows of
// stopped scenes before them
__global__ void k_running_flags(int64_t n, const int32_t *__restrict__ sid,
                                const uint8_t *__restrict__ stop, int32_t *keep) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        keep[v] = stop[sid[v]] ? 0 : 1;
}

__global__ void k_compact_running(SrcRows a, SrcRows b, int64_t n, int F,
                                  const int32_t *__restrict__ keep, const int32_t *__restrict__ pos,
                                  const int32_t *__restrict__ sid, const int32_t *__restrict__ cid,
                                  const int64_t *__restrict__ shift, int32_t *cid_out) {
    const int per = parts_of(F);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * per;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / per;
        if (!keep[row]) continue;
        const int ch = (int)(t - row * per);
        move_part(a, row, b, pos[row], F, ch);
        if (ch == 0) cid_out[pos[row]] = cid[row] - (int32_t)shift[sid[row]];
    }
}

// hdst[s] = pos[at[s]] into pinned host memory (read after a stream sync)
__global__ void k_pos_at(const int32_t *__restrict__ pos, const int64_t *__restrict__ at, int m,
                         int32_t *hdst) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < m) hdst[s] = pos[at[s]];
}

__global__ void k_fill_sid(const int64_t *__restrict__ start, int S, int64_t n, int32_t *sid) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        sid[v] = scene_of(start, S, v);
}

// ---- pre-filter with one median per scene
__global__ void k_logit_keys_rows(const float *__restrict__ logit, int64_t n, uint32_t *keys,
                                  uint32_t *keys_copy, uint32_t *vals) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = float_order_bits(logit[v]);
        keys[v] = k;
        keys_copy[v] = k;
        vals[v] = (uint32_t)v;
    }
}

__global__ void k_gather_sid(const int32_t *__restrict__ sid, const uint32_t *__restrict__ vals,
                             int64_t n, int S, const int32_t *__restrict__ keep, uint32_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = vals[i];
        out[i] = keep && !keep[r] ? (uint32_t)S : (uint32_t)sid[r];
    }
}

// alpha >= min(tau, alpha_med)  <=>  logit >= min(logit(tau), logit_med), per scene
__global__ void k_scene_thr(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ order,
                            const int64_t *__restrict__ start, int S, double l_tau, double *thr) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int64_t n = start[s + 1] - start[s];
    if (n <= 0) {
        thr[s] = l_tau;
        return;
    }
    const uint32_t med = keys[order[start[s] + (n - 1) / 2]];
    thr[s] = fmin((double)order_bits_float(med), l_tau);
}

__global__ void k_prefilter_rows(const float *__restrict__ logit, const int32_t *__restrict__ sid,
                                 int64_t n, const double *__restrict__ thr, int32_t *keep) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        keep[v] = (double)logit[v] >= thr[sid[v]];
}

__global__ void k_fill_ones(int32_t *a, int64_t n) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        a[v] = 1;
}

// ---- per-scene Morton frames
__global__ void k_frames_init(uint32_t *acc, int S) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8 * S) return;
    const int f = t & 7;
    acc[t] = f < 3 ? 0xffffffffu : 0u;
}

// each warp scans one contiguous run of rows (scenes are contiguous, so a run
// meets few scene boundaries) and flushes its bounds once per scene it meets
__device__ __forceinline__ void frames_flush(uint32_t *acc, int s, float mn[3], float mx[3],
                                             uint32_t &bad) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        mn[a] = warp_min(mn[a]);
        mx[a] = warp_max(mx[a]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(FULL_MASK, bad, o);
    if ((threadIdx.x & 31) == 0 && s >= 0) {
        uint32_t *a8 = acc + 8 * s;
#pragma unroll
        for (int a = 0; a < 3; a++)
            if (mn[a] <= mx[a]) {
                atomicMin(&a8[a], float_order_bits(mn[a]));
                atomicMax(&a8[3 + a], float_order_bits(mx[a]));
            }
        if (bad) atomicAdd(&a8[6], bad);
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        mn[a] = INFINITY;
        mx[a] = -INFINITY;
    }
    bad = 0;
}

__global__ void k_frames_reduce(const float *__restrict__ xyz, const int32_t *__restrict__ sid,
                                int64_t n, uint32_t *acc) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t per = ((n + nwarps - 1) / nwarps + 31) & ~(int64_t)31;
    const int64_t r0 = w * per, r1 = r0 + per < n ? r0 + per : n;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    uint32_t bad = 0;
    int cur = -1;  // scene of the accumulated rows (warp-uniform)
    for (int64_t base = r0; base < r1; base += 32) {
        const int64_t i = base + lane;
        const int s = i < r1 ? sid[i] : -1;
        const int s_first = __shfl_sync(FULL_MASK, s, 0);
        const int64_t last = r1 - 1 - base;
        const int s_last = __shfl_sync(FULL_MASK, s, last < 31 ? (int)last : 31);
        if (s_first != cur || s_last != cur) {
            frames_flush(acc, cur, mn, mx, bad);
            cur = s_first;
        }
        if (s_first == s_last) {
            if (i < r1) {
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const float v = xyz[3 * i + a];
                    if (!isfinite(v)) {
                        bad++;
                        continue;
                    }
                    mn[a] = fminf(mn[a], v);
                    mx[a] = fmaxf(mx[a], v);
                }
            }
        } else if (i < r1) {  // a scene boundary inside these 32 rows
            uint32_t *a8 = acc + 8 * s;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float v = xyz[3 * i + a];
                if (!isfinite(v)) {
                    atomicAdd(&a8[6], 1u);
                    continue;
                }
                atomicMin(&a8[a], float_order_bits(v));
                atomicMax(&a8[3 + a], float_order_bits(v));
            }
        }
    }
    frames_flush(acc, cur, mn, mx, bad);
}

__global__ void k_frames_final(const uint32_t *__restrict__ acc, int S, float *frames,
                               uint32_t *bad) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const uint32_t *a = acc + 8 * s;
    float lo[3], side = 0.0f;
    for (int k = 0; k < 3; k++) {
        if (a[k] == 0xffffffffu) {
            lo[k] = 0.0f;
            continue;
        }
        lo[k] = order_bits_float(a[k]);
        side = fmaxf(side, order_bits_float(a[3 + k]) - lo[k]);
    }
    if (!(side > 0.0f)) side = 1.0f;
    float *f = frames + 8 * s;
    f[0] = lo[0];
    f[1] = lo[1];
    f[2] = lo[2];
    f[3] = 1024.0f / (side * 1.0001f);
    f[4] = 0.f;
    if (a[6]) atomicAdd(bad, a[6]);
}

__device__ __forceinline__ uint32_t spread10e(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// 30-bit Morton code of each row in its scene's frame (same quantisation as
// the single-frame kernel); with `keep`, dropped rows get bit 30 so that
// they sort after every kept row
__global__ void k_morton_rows(const float *__restrict__ xyz, const int32_t *__restrict__ sid,
                              int64_t n, const float *__restrict__ frames,
                              const int32_t *__restrict__ keep, uint32_t *keys, uint32_t *vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float *f = frames + 8 * (sid ? sid[i] : 0);
        const float q[3] = {(xyz[3 * i] - f[0]) * f[3], (xyz[3 * i + 1] - f[1]) * f[3],
                            (xyz[3 * i + 2] - f[2]) * f[3]};
        uint32_t cc[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const float v = q[a];
            cc[a] = (v >= 1023.0f) ? 1023u : (v > 0.0f ? (uint32_t)v : 0u);
        }
        keys[i] = spread10e(cc[0]) | (spread10e(cc[1]) << 1) | (spread10e(cc[2]) << 2) |
                  (keep && !keep[i] ? 1u << 30 : 0u);
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_gather_cid(const uint32_t *__restrict__ order, const int32_t *__restrict__ pos,
                             int64_t n, int32_t *cid) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        cid[p] = pos[order[p]];
}

// ---- per-scene pair counts and caps
// Rows of a scene are contiguous, so the lanes of a warp mostly share one
// scene: one atomic per scene present in the warp.
__global__ void k_scene_pairs(int64_t n, const int32_t *__restrict__ mate,
                              const int32_t *__restrict__ cid, const int32_t *__restrict__ sid,
                              int32_t *cnt) {
    const int lane = threadIdx.x & 31;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = b + threadIdx.x;
        bool has = false;
        int32_t s = 0;
        if (v < n) {
            const int32_t u = mate[v];
            has = u >= 0 && cid[v] < cid[u];
            s = sid[v];
        }
        const unsigned peers = __match_any_sync(FULL_MASK, has ? s : -1 - lane);
        if (has && lane == __ffs(peers) - 1) atomicAdd(&cnt[s], __popc(peers));
    }
}

// one sortable record per matched pair (at its lower-cid endpoint)
__global__ void k_pair_list(int64_t n, const uint64_t *__restrict__ keys,
                            const int32_t *__restrict__ flagpos, const int32_t *__restrict__ sid,
                            uint32_t *klo, uint32_t *khi, uint32_t *ksid) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[v];
        if (k == ~0ull) continue;
        const int32_t p = flagpos[v];
        klo[p] = (uint32_t)(k & 0xffffffffu);
        khi[p] = (uint32_t)(k >> 32);
        ksid[p] = (uint32_t)sid[v];
    }
}

__global__ void k_key_flags(int64_t n, const uint64_t *__restrict__ keys, int32_t *flag) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        flag[v] = keys[v] != ~0ull;
}

// threshold of scene s = its (P_s)-th smallest pair key, or UINT64_MAX when
// the scene matched at most P_s pairs.  The records are sorted by (scene,
// cost bits, lower id): khi = cost bits in that order, klo[order[i]] = the
// lower id of record i.
__global__ void k_scene_caps(const uint32_t *__restrict__ khi, const uint32_t *__restrict__ klo,
                             const uint32_t *__restrict__ order, const int64_t *__restrict__ seg,
                             const int64_t *__restrict__ P, int S, uint64_t *thr) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int64_t m = seg[s + 1] - seg[s];
    if (P[s] >= m) {
        thr[s] = ~0ull;
    } else if (P[s] <= 0) {
        thr[s] = 0ull;  // below every key: no pair of this scene merges
    } else {
        const int64_t i = seg[s] + P[s] - 1;
        thr[s] = ((uint64_t)khi[i] << 32) | klo[order[i]];
    }
}

int bits_for(int S) {
    int b = 1;
    while ((1 << b) <= S) b++;
    return b;
}

SplatView scratch(ngs_ctx *c, DevBuf *b, int64_t n, int F) {
    SplatView v;
    v.xyz = ws<float>(c, b[0], 3 * n);
    v.ls = ws<float>(c, b[1], 3 * n);
    v.rot = ws<float>(c, b[2], 4 * n);
    v.logit = ws<float>(c, b[3], n);
    v.sh = ws<float>(c, b[4], (int64_t)F * n);
    v.n = n;
    v.F = F;
    return v;
}

SrcRows rows(const SplatView &v) { return SrcRows{v.xyz, v.ls, v.rot, v.logit, v.sh}; }

template <class T>
T *upload(ngs_ctx *c, DevBuf &b, const T *h, size_t count) {
    T *d = (T *)ws_get(c, b, sizeof(T) * (count ? count : 1));
    put_small(c, d, h, sizeof(T) * count);
    return d;
}

template <class T>
void download(ngs_ctx *c, T *h, const T *d, size_t count) {
    if (count) NGS_CHECK_CUDA(cudaMemcpyAsync(h, d, sizeof(T) * count, cudaMemcpyDeviceToHost, c->st));
}

}  // namespace

void engine_simplify(ngs_ctx *c, ngs_splats *sc, const int64_t *targets, int S, ngs_stats *st) {
    const int F = sc[0].sh_dim;
    const int64_t launches0 = c->launches, syncs0 = c->syncs;
    c->fp64_edges = 0;
    c->floor_hits = 0;
    std::vector<int64_t> in0(S + 1, 0);
    for (int s = 0; s < S; s++) in0[s + 1] = in0[s] + sc[s].n;
    const int64_t N0 = in0[S];
    if (st) {
        memset(st, 0, sizeof(*st));
        st->n_input = N0;
    }
    if (N0 > NGS_MAX_N)
        NGS_FAIL(NGS_ERR_INVALID_ARG, "total splats %lld above %lld", (long long)N0,
                 (long long)NGS_MAX_N);
    check_slots(N0, c->prm.k, S > 1 ? "ngs_batch_simplify" : "ngs_simplify");
    if (N0 <= 0) return;
    const bool multi = S > 1;
    if (multi)
        for (int s = 0; s < S; s++)
            if (targets[s] <= k_eff_of(INT64_MAX, c->prm.k))
                NGS_FAIL(NGS_ERR_INVALID_ARG, "scene %d: target %lld too small to batch", s,
                         (long long)targets[s]);
    std::vector<SrcRows> hsrc(S);
    for (int s = 0; s < S; s++)
        hsrc[s] = SrcRows{sc[s].xyz, sc[s].log_scale, sc[s].rot, sc[s].opacity_logit, sc[s].sh};
    const SrcRows *dsrc = upload(c, c->b_eng[E_SRC], hsrc.data(), S);
    const int64_t *din0 = upload(c, c->b_eng[E_START], in0.data(), S + 1);

    // ---- working input: the caller's arrays (one scene) or their concatenation
    SplatView IN;
    if (!multi) {
        IN = SplatView{sc[0].xyz, sc[0].log_scale, sc[0].rot, sc[0].opacity_logit, sc[0].sh, N0, F};
    } else {
        IN = scratch(c, c->b_sB, N0, F);
        launch(c, "gather_scenes", dim3(grid_stride_blocks(c, N0 * parts_of(F), 256, 16)),
               dim3(256), 0, k_gather_scenes, dsrc, din0, S, N0, F, rows(IN));
    }
    const unsigned g0 = grid_stride_blocks(c, N0, 256, 8);
    int32_t *sid_in = ws<int32_t>(c, c->b_eng[E_SID], N0);
    if (multi) launch(c, "fill_sid", dim3(g0), dim3(256), 0, k_fill_sid, din0, S, N0, sid_in);
    else NGS_CHECK_CUDA(cudaMemsetAsync(sid_in, 0, 4 * N0, c->st));

    // ---- pre-filter (Algorithm 1), one median per scene
    int32_t *keep = ws<int32_t>(c, c->b_role, N0 + 1);
    int32_t *pos = ws<int32_t>(c, c->b_pos, N0 + 1);
    if (!c->prm.prefilter) {
        launch(c, "fill_ones", dim3(g0), dim3(256), 0, k_fill_ones, keep, N0);
        scan_i32(c, keep, pos, N0);
    } else if (!multi) {
        prefilter_flags(c, IN.logit, N0, c->prm.tau, keep);  // leaves its scan in b_pos
    } else {
        uint32_t *k0 = ws<uint32_t>(c, c->b_codes, N0), *kc = ws<uint32_t>(c, c->b_codes2, N0);
        uint32_t *vals = ws<uint32_t>(c, c->b_vals, N0), *v2 = ws<uint32_t>(c, c->b_vals2, N0);
        uint32_t *kt = ws<uint32_t>(c, c->b_eng[E_TMP], N0);
        launch(c, "logit_keys", dim3(g0), dim3(256), 0, k_logit_keys_rows, IN.logit, N0, k0, kc,
               vals);
        radix_sort_u32(c, kc, vals, kt, v2, N0, 32);
        launch(c, "gather_sid", dim3(g0), dim3(256), 0, k_gather_sid, (const int32_t *)sid_in,
               (const uint32_t *)vals, N0, S, (const int32_t *)nullptr, kc);
        radix_sort_u32(c, kc, vals, kt, v2, N0, bits_for(S));
        double *thr = (double *)ws<uint8_t>(c, c->b_eng[E_THR], 8 * (S + 1));
        launch(c, "scene_thr", dim3(blocks_for(S, 128)), dim3(128), 0, k_scene_thr,
               (const uint32_t *)k0, (const uint32_t *)vals, din0, S,
               log(c->prm.tau / (1.0 - c->prm.tau)), thr);
        launch(c, "prefilter_rows", dim3(g0), dim3(256), 0, k_prefilter_rows, IN.logit,
               (const int32_t *)sid_in, N0, (const double *)thr, keep);
        scan_i32(c, keep, pos, N0);
    }
    // kept rows per scene: scene s keeps [pos[in0[s]], pos[in0[s+1]])
    std::vector<int64_t> kin(S + 1);
    {
        int32_t *hp = (int32_t *)(c->h_pin + 64);  // pinned, S + 1 <= 4097 entries
        launch(c, "kept_counts", dim3(blocks_for(S + 1, 256)), dim3(256), 0, k_pos_at,
               (const int32_t *)pos, din0, S + 1, hp);
        sync_stream(c);
        for (int s = 0; s <= S; s++) kin[s] = hp[s];
    }
    const int64_t nf = kin[S];
    if (st) st->n_filtered = nf;

    // ---- Morton frames per scene (over all input rows)
    float *frames = ws<float>(c, c->b_frame, 8 * S);
    {
        uint32_t *acc = ws<uint32_t>(c, c->b_bbox, 8 * S + 8);
        uint32_t *bad = acc + 8 * S;
        NGS_CHECK_CUDA(cudaMemsetAsync(bad, 0, 4, c->st));
        if (!multi) {
            morton_frame(c, IN.xyz, N0, frames);
            NGS_CHECK_CUDA(cudaMemcpyAsync(bad, frames + 4, 4, cudaMemcpyDeviceToDevice, c->st));
        } else {
            launch(c, "frames_init", dim3(blocks_for(8 * S, 256)), dim3(256), 0, k_frames_init,
                   acc, S);
            launch(c, "frames_reduce", dim3(g0), dim3(256), 0, k_frames_reduce, IN.xyz,
                   (const int32_t *)sid_in, N0, acc);
            launch(c, "frames_final", dim3(blocks_for(S, 128)), dim3(128), 0, k_frames_final,
                   (const uint32_t *)acc, S, frames, bad);
        }
        get_small(c, c->h_pin + 4, bad, 4);
        sync_stream(c);
        const uint32_t nbad = *(uint32_t *)(c->h_pin + 4);
        if (nbad) NGS_FAIL(NGS_ERR_INVALID_ARG, "%u non-finite centre coordinates", nbad);
    }

    // ---- survivors into Morton order within each scene (working set A)
    // A single scene whose SH array is still being uploaded (ngs_simplify_host)
    // gathers its SH rows only when first needed: before the first edge costs
    // or write-back, so the upload overlaps the first graph stages.
    bool defer_sh = !multi && c->sh_wait && (F & 3) == 0 && F <= 64;
    uint32_t *order0 = nullptr;
    SplatView A, B;
    int32_t *cidA = nullptr, *cidB = nullptr;
    {
        uint32_t *keys = ws<uint32_t>(c, c->b_codes, N0), *order = ws<uint32_t>(c, c->b_vals, N0);
        uint32_t *k2 = ws<uint32_t>(c, c->b_codes2, N0), *v2 = ws<uint32_t>(c, c->b_vals2, N0);
        if (!multi) {  // (dropped, code) in one 31-bit sort
            launch(c, "morton", dim3(g0), dim3(256), 0, k_morton_rows, IN.xyz,
                   (const int32_t *)nullptr, N0, (const float *)frames, (const int32_t *)keep,
                   keys, order);
            radix_sort_u32(c, keys, order, k2, v2, N0, 31);
        } else {
            launch(c, "morton", dim3(g0), dim3(256), 0, k_morton_rows, IN.xyz,
                   (const int32_t *)sid_in, N0, (const float *)frames, (const int32_t *)nullptr,
                   keys, order);
            radix_sort_u32(c, keys, order, k2, v2, N0, 30);
            // stable by scene; pre-filtered rows (scene S) last
            launch(c, "gather_sid", dim3(g0), dim3(256), 0, k_gather_sid,
                   (const int32_t *)sid_in, (const uint32_t *)order, N0, S,
                   (const int32_t *)keep, keys);
            radix_sort_u32(c, keys, order, k2, v2, N0, bits_for(S));
        }
        A = scratch(c, c->b_sA, nf, F);
        B = multi ? scratch(c, c->b_sC, nf, F) : scratch(c, c->b_sB, nf, F);
        // the rows' scales and rotations may still be uploading (ngs_simplify_host)
        if (c->rest_wait) NGS_CHECK_CUDA(cudaStreamWaitEvent(c->st, c->rest_wait, 0));
        if (defer_sh) {
            // the SH rows follow once their upload has finished (ensure_sh)
            gather_rows_part(c, IN, order, A, false);
            order0 = ws<uint32_t>(c, c->b_order0, nf);
            NGS_CHECK_CUDA(cudaMemcpyAsync(order0, order, 4 * nf, cudaMemcpyDeviceToDevice, c->st));
        } else {
            if (c->sh_wait) NGS_CHECK_CUDA(cudaStreamWaitEvent(c->st, c->sh_wait, 0));
            gather_rows(c, IN, order, A);
        }
        cidA = ws<int32_t>(c, c->b_cid, nf + 1);
        cidB = ws<int32_t>(c, c->b_cid2, nf + 1);
        launch(c, "gather_cid", dim3(grid_stride_blocks(c, nf, 256, 8)), dim3(256), 0,
               k_gather_cid, (const uint32_t *)order, (const int32_t *)pos, nf, cidA);
    }

    // ---- per-scene state (host)
    std::vector<int64_t> n(S), tgt(S), wstart(S + 1), pairs_s(S), P(S);
    std::vector<uint8_t> running(S), out_done(S, 0), stop(S);
    for (int s = 0; s < S; s++) {
        n[s] = kin[s + 1] - kin[s];
        tgt[s] = targets[s];
        running[s] = n[s] > tgt[s] && n[s] > 1;
    }
    for (int s = 0; s <= S; s++) wstart[s] = kin[s];
    int32_t *sidA = ws<int32_t>(c, c->b_eng[E_SIDW], nf + 1);

    auto ensure_sh = [&]() {
        if (!defer_sh) return;
        NGS_CHECK_CUDA(cudaStreamWaitEvent(c->st, c->sh_wait, 0));
        gather_rows_part(c, IN, order0, A, true);
        defer_sh = false;
    };
    // write stopped scenes back (canonical order) and drop them from A
    auto extract = [&](bool all) {
        bool any = false, left = false;
        for (int s = 0; s < S; s++) {
            stop[s] = !out_done[s] && (all || !running[s]);
            any = any || stop[s];
            left = left || (!out_done[s] && !stop[s]);
        }
        if (!any) return;
        ensure_sh();
        const int64_t nA = A.n;
        if (nA > 0) {
            const int64_t *dws = upload(c, c->b_eng[E_WS], wstart.data(), S + 1);
            if (multi) launch(c, "fill_sid", dim3(grid_stride_blocks(c, nA, 256, 8)), dim3(256), 0,
                              k_fill_sid, dws, S, nA, sidA);
            else NGS_CHECK_CUDA(cudaMemsetAsync(sidA, 0, 4 * nA, c->st));
            const uint8_t *dstop = upload(c, c->b_eng[E_STOP], stop.data(), S);
            launch(c, "extract", dim3(grid_stride_blocks(c, nA * parts_of(F), 256, 16)),
                   dim3(256), 0, k_extract, rows(A), nA, F, (const int32_t *)sidA,
                   (const int32_t *)cidA, dstop, dws, dsrc);
            if (left) {
                std::vector<int64_t> shift(S, 0);
                int64_t removed = 0;
                for (int s = 0; s < S; s++) {
                    shift[s] = removed;
                    if (stop[s]) removed += n[s];
                }
                const int64_t *dshift = upload(c, c->b_eng[E_SHIFT], shift.data(), S);
                int32_t *kp = ws<int32_t>(c, c->b_keep, nA + 1);
                int32_t *pp = ws<int32_t>(c, c->b_eng[E_POS2], nA + 1);
                launch(c, "running_flags", dim3(grid_stride_blocks(c, nA, 256, 8)), dim3(256), 0,
                       k_running_flags, nA, (const int32_t *)sidA, dstop, kp);
                scan_i32(c, kp, pp, nA);
                launch(c, "compact_running",
                       dim3(grid_stride_blocks(c, nA * parts_of(F), 256, 16)), dim3(256), 0,
                       k_compact_running, rows(A), rows(B), nA, F, (const int32_t *)kp,
                       (const int32_t *)pp, (const int32_t *)sidA, (const int32_t *)cidA, dshift,
                       cidB);
                std::swap(A, B);
                std::swap(cidA, cidB);
            }
            sync_stream(c);  // the uploads above read host vectors
        }
        int64_t cur = 0;
        for (int s = 0; s < S; s++) {
            if (stop[s]) {
                sc[s].n = n[s];
                out_done[s] = 1;
            }
            wstart[s] = cur;
            if (!out_done[s]) cur += n[s];
        }
        wstart[S] = cur;
        A.n = cur;
    };

    int pass = 0;
    int64_t fp64_total = 0, tie_total = 0, requeried_total = 0;
    // local neighbourhood refresh (Sec. 3.4), one scene: on passes p with
    // p % refresh_period != 0 the previous lists are carried through the merge
    const int R = multi ? 1 : c->prm.refresh_period;
    bool have_prev = false;
    bool rows_sorted = true;  // A in (scene, Morton code) order (no merge yet)
    int64_t n_prev = 0;
    int k_prev = 0;
    while (pass < c->prm.max_passes) {
        extract(false);
        if (A.n <= 0) break;
        const int64_t nA = A.n;
        // per-row scene ids of the running scenes
        const int64_t *dws = upload(c, c->b_eng[E_WS], wstart.data(), S + 1);
        if (multi) launch(c, "fill_sid", dim3(grid_stride_blocks(c, nA, 256, 8)), dim3(256), 0,
                          k_fill_sid, dws, S, nA, sidA);
        GraphDev &g = c->g;
        g = GraphDev{};
        g.n = nA;
        g.k_eff = k_eff_of(nA, c->prm.k);
        for (int s = 0; s < S; s++)  // equal for all running scenes (checked on entry)
            if (!out_done[s] && k_eff_of(n[s], c->prm.k) != g.k_eff)
                NGS_FAIL(NGS_ERR_STATE, "scene %d: k_eff differs within a batch", s);
        g.cid = cidA;
        // exact Morton order of this pass, grouped by scene
        uint32_t *pk = ws<uint32_t>(c, c->b_codes, nA), *pv = ws<uint32_t>(c, c->b_vals, nA);
        uint32_t *pk2 = ws<uint32_t>(c, c->b_codes2, nA), *pv2 = ws<uint32_t>(c, c->b_vals2, nA);
        uint32_t *code_row = ws<uint32_t>(c, c->b_eng[E_TMP], nA);
        int32_t *ssid = nullptr;
        launch(c, "morton", dim3(grid_stride_blocks(c, nA, 256, 8)), dim3(256), 0, k_morton_rows,
               (const float *)A.xyz, multi ? (const int32_t *)sidA : (const int32_t *)nullptr, nA,
               (const float *)frames, (const int32_t *)nullptr, pk, pv);
        // Until the first merge the rows are still in the order of the initial
        // sort, (scene, Morton code) under the same frames: the sorts below
        // would return the identity, so they are skipped.
        if (multi) {
            uint32_t *sk = ws<uint32_t>(c, c->b_eng[E_SSID], nA);
            if (rows_sorted) {
                NGS_CHECK_CUDA(cudaMemcpyAsync(sk, sidA, 4 * nA, cudaMemcpyDeviceToDevice, c->st));
            } else {
                NGS_CHECK_CUDA(cudaMemcpyAsync(code_row, pk, 4 * nA, cudaMemcpyDeviceToDevice, c->st));
                radix_sort_u32(c, pk, pv, pk2, pv2, nA, 30);
                launch(c, "gather_sid", dim3(grid_stride_blocks(c, nA, 256, 8)), dim3(256), 0,
                       k_gather_sid, (const int32_t *)sidA, (const uint32_t *)pv, nA, S,
                       (const int32_t *)nullptr, sk);
                radix_sort_u32(c, sk, pv, pk2, pv2, nA, bits_for(S));
                gather_u32(c, code_row, pv, nA, pk);
            }
            ssid = (int32_t *)sk;
        } else if (!rows_sorted) {
            radix_sort_u32(c, pk, pv, pk2, pv2, nA, 30);
        }
        float4 *pts = ws<float4>(c, c->b_pts, nA);
        gather_points(c, A.xyz, cidA, pv, nA, pts);
        int32_t *nbr = ws<int32_t>(c, c->b_nbr, nA * g.k_eff);
        std::vector<int64_t> scene_n(S);
        for (int s = 0; s < S; s++) scene_n[s] = out_done[s] ? 0 : n[s];
        if (R > 1 && have_prev && pass % R != 0) {
            int32_t *qlist = ws<int32_t>(c, c->b_qlist, nA + 1);
            const int64_t nq = refresh_rows(c, nA, g.k_eff, k_prev, n_prev, (const int32_t *)c->b_rsrc.p,
                                            (const int32_t *)c->b_prevnbr.p, (const int32_t *)c->b_rmap.p,
                                            A.xyz, cidA, pv, nbr, qlist);
            knn_search(c, KnnInput{pts, pk, pv, ssid, frames, scene_n.data(), S, nA, 0, cidA, qlist, nq},
                       g.k_eff, nbr);
            requeried_total += nq;
        } else {
            knn_search(c, KnnInput{pts, pk, pv, ssid, frames, scene_n.data(), S, nA, 0, cidA},
                       g.k_eff, nbr);
            requeried_total += nA;
        }
        have_prev = false;
        build_edges(c, nbr, g);
        ensure_sh();
        edge_costs(c, A, g, (uint32_t)pass, false, nullptr);
        int32_t *partner = ws<int32_t>(c, c->b_partner, nA);
        int64_t np = 0;
        if (!multi) {
            P[0] = n[0] - tgt[0];
            np = select_pairs(c, g, P[0], partner);
            pairs_s[0] = np;
        } else {
            const int64_t matched = match_rounds(c, g);
            std::vector<int32_t> cnt(S, 0);
            int32_t *dcnt = ws<int32_t>(c, c->b_eng[E_CNT], S + 1);
            NGS_CHECK_CUDA(cudaMemsetAsync(dcnt, 0, 4 * S, c->st));
            if (matched > 0)
                launch(c, "scene_pairs", dim3(grid_stride_blocks(c, nA, 256, 8)), dim3(256), 0,
                       k_scene_pairs, nA, (const int32_t *)c->b_mate.p, (const int32_t *)cidA,
                       (const int32_t *)sidA, dcnt);
            download(c, cnt.data(), dcnt, S);
            sync_stream(c);
            bool capped = false;
            std::vector<int64_t> seg(S + 1, 0);
            for (int s = 0; s < S; s++) {
                P[s] = out_done[s] ? 0 : n[s] - tgt[s];
                pairs_s[s] = std::min<int64_t>(cnt[s], P[s]);
                np += pairs_s[s];
                capped = capped || cnt[s] > P[s];
                seg[s + 1] = seg[s] + cnt[s];
            }
            uint64_t *thr = (uint64_t *)ws<uint8_t>(c, c->b_eng[E_THR], 8 * (S + 1));
            if (capped) {
                // per-scene thresholds: pair keys sorted by (scene, cost, lo id)
                uint64_t *keys = (uint64_t *)ws<uint8_t>(c, c->b_flag, 8 * nA);
                pair_keys(c, g, keys);
                int32_t *fl = ws<int32_t>(c, c->b_keep, nA + 1), *fp = ws<int32_t>(c, c->b_eng[E_POS2], nA + 1);
                launch(c, "key_flags", dim3(grid_stride_blocks(c, nA, 256, 8)), dim3(256), 0,
                       k_key_flags, nA, (const uint64_t *)keys, fl);
                scan_i32(c, fl, fp, nA);
                const int64_t m = seg[S];
                uint32_t *klo = ws<uint32_t>(c, c->b_eng[E_KLO], m), *khi = ws<uint32_t>(c, c->b_eng[E_KHI], m);
                uint32_t *ks = ws<uint32_t>(c, c->b_eng[E_KS], m), *ord = ws<uint32_t>(c, c->b_eng[E_ORD], m);
                uint32_t *t1 = ws<uint32_t>(c, c->b_eng[E_T1], m), *t2 = ws<uint32_t>(c, c->b_eng[E_T2], m);
                launch(c, "pair_list", dim3(grid_stride_blocks(c, nA, 256, 8)), dim3(256), 0,
                       k_pair_list, nA, (const uint64_t *)keys, (const int32_t *)fp,
                       (const int32_t *)sidA, klo, khi, ks);
                iota_u32(c, ord, m);
                NGS_CHECK_CUDA(cudaMemcpyAsync(t1, klo, 4 * m, cudaMemcpyDeviceToDevice, c->st));
                radix_sort_u32(c, t1, ord, t2, pk2, m, 32);  // by lo id
                gather_u32(c, khi, ord, m, t1);
                radix_sort_u32(c, t1, ord, t2, pk2, m, 32);  // then by cost bits
                gather_u32(c, ks, ord, m, t2);
                uint32_t *t3 = ws<uint32_t>(c, c->b_eng[E_T3], m);
                gather_u32(c, khi, ord, m, t3);             // cost bits in (cost, lo) order
                // stable by scene, carrying the cost bits alongside through a second payload pass
                uint32_t *ord2 = ws<uint32_t>(c, c->b_eng[E_ORD2], m);
                iota_u32(c, ord2, m);
                radix_sort_u32(c, t2, ord2, t1, pk2, m, bits_for(S));
                gather_u32(c, t3, ord2, m, t1);             // cost bits in (scene, cost, lo) order
                gather_u32(c, ord, ord2, m, t3);            // list index in that order
                const int64_t *dseg = upload(c, c->b_eng[E_SEG], seg.data(), S + 1);
                const int64_t *dP = upload(c, c->b_eng[E_P], P.data(), S);
                launch(c, "scene_caps", dim3(blocks_for(S, 128)), dim3(128), 0, k_scene_caps,
                       (const uint32_t *)t1, (const uint32_t *)klo, (const uint32_t *)t3, dseg, dP,
                       S, thr);
                sync_stream(c);
            }
            apply_cap(c, g, sidA, thr, capped ? 1 : 0, partner);
        }
        fp64_total += (int64_t)c->h_pin[1];
        tie_total += (int64_t)c->h_pin[5];
        if (st && pass < NGS_STATS_MAX_PASSES) {
            st->pass_n[pass] = nA;
            st->pass_edges[pass] = g.n_edges;
            st->pass_pairs[pass] = np;
            st->matching_rounds += c->rounds;
        }
        pass++;
        for (int s = 0; s < S; s++)
            if (!out_done[s] && pairs_s[s] == 0) running[s] = 0;  // no pair: this scene stops
        if (np > 0) {
            int32_t *role = ws<int32_t>(c, c->b_role, nA);
            partner_to_role(c, partner, cidA, nA, role);
            B.n = nA;
            const int64_t nn = merge_compact(c, A, role, B, cidA, cidB);
            rows_sorted = false;
            if (R > 1 && pass % R != 0) {
                // the next pass carries these lists: keep them and the row maps
                refresh_map(c, nA, role, ws<int32_t>(c, c->b_rmap, nA), ws<int32_t>(c, c->b_rsrc, nn));
                std::swap(c->b_nbr, c->b_prevnbr);
                have_prev = true;
                n_prev = nA;
                k_prev = g.k_eff;
            }
            std::swap(A, B);
            std::swap(cidA, cidB);
            int64_t cur = 0;
            for (int s = 0; s < S; s++) {
                wstart[s] = cur;
                if (!out_done[s]) {
                    n[s] -= pairs_s[s];
                    cur += n[s];
                    running[s] = running[s] && n[s] > tgt[s] && n[s] > 1;
                }
            }
            wstart[S] = cur;
            if (cur != nn) NGS_FAIL(NGS_ERR_STATE, "merge kept %lld rows, expected %lld",
                                    (long long)nn, (long long)cur);
            A.n = cur;
        }
        bool any = false;
        for (int s = 0; s < S; s++) any = any || (!out_done[s] && running[s]);
        if (!any) break;
    }
    extract(true);
    c->g_valid = false;
    if (st) {
        int64_t tot = 0;
        for (int s = 0; s < S; s++) tot += sc[s].n;
        st->n_output = tot;
        st->passes = pass;
        st->fp64_cost_edges = fp64_total;
        st->near_tie_slots = tie_total;
        st->requeried_rows = requeried_total;
        st->eig_floor_hits = c->floor_hits;
        st->gpu_launches = c->launches - launches0;
        st->host_syncs = c->syncs - syncs0;
    }
}
