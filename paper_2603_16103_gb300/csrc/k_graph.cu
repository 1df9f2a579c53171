// Undirected merge graph from the directed kNN lists (Algorithm 1
// UndirectedUnionEdges), kept in "slot" form: slot s = v*k + t is the t-th
// directed neighbour u = nbr[s] of v.  The undirected edge {v,u} exists when
// u is in v's list or v is in u's list.
//   * A slot is mutual when v is also in u's list; mirror[s] is then the
//     partner slot, otherwise -1.  (The row form, for k dividing 32, stores a
//     slot code instead that also carries which endpoint is lower; see
//     k_slot_classify_rows.)
//   * Each undirected edge has exactly one canonical slot: a non-mutual slot,
//     or the mutual slot whose row has the lower canonical id.  erec[] lists
//     one record (slot, lo row, hi row, mirror) per canonical slot in slot
//     order; |E| = their number.  mirror: the partner slot of a mutual edge,
//     else -2 - r with r the edge's position in rev[].
//   * rev[] lists, per vertex u, the non-mutual slots that point at u (its
//     in-edges not already in its own list); revcost[] holds their costs
//     in the same order, so a vertex reads its in-edge costs contiguously.
// So the incident edges of v are its k slots plus its rev entries, each once,
// and costs live per slot (mirrored for mutual edges).  No sort is needed on
// the simplification path; the C-ABI view additionally sorts the canonical
// slots lexicographically by (lo, hi) canonical id.
#include "ngs_device.cuh"
#include "ngs_internal.h"

namespace {

__device__ __forceinline__ uint32_t cid_of(const int32_t *cid, int32_t v) {
    return cid ? (uint32_t)cid[v] : (uint32_t)v;
}

__global__ void k_slot_classify(const int32_t *__restrict__ nbr, int64_t n, int k,
                                const int32_t *__restrict__ cid, int32_t *mirror, int32_t *canon,
                                int32_t *revcnt) {
    const int64_t m = n * k;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)(s / k);
        const int32_t u = nbr[s];
        const int32_t *row = nbr + (int64_t)u * k;
        int tp = -1;
        if ((k & 3) == 0) {
            // 16-byte loads of u's row, first match kept
            for (int t = k - 4; t >= 0; t -= 4) {
                const int4 r = __ldg((const int4 *)(row + t));
                if (r.w == v) tp = t + 3;
                if (r.z == v) tp = t + 2;
                if (r.y == v) tp = t + 1;
                if (r.x == v) tp = t;
            }
        } else {
            for (int t = k - 1; t >= 0; t--)
                if (row[t] == v) tp = t;
        }
        if (tp >= 0) {
            mirror[s] = u * k + tp;
            canon[s] = cid_of(cid, v) < cid_of(cid, u) ? 1 : 0;
        } else {
            mirror[s] = -1;
            canon[s] = 1;
            atomicAdd(&revcnt[u], 1);
        }
    }
}

// Canonical slots -> edge records (slot, lo row, hi row, mirror slot), where
// lo is the endpoint with the lower canonical id; reverse index entries.
__global__ void k_slot_fill(const int32_t *__restrict__ nbr, int64_t n, int k,
                            const int32_t *__restrict__ cid, const int32_t *__restrict__ mirror,
                            const int32_t *__restrict__ canon, const int32_t *__restrict__ epos,
                            const int32_t *__restrict__ rev_ptr, int32_t *revfill, int4 *erec,
                            int32_t *rev) {
    const int64_t m = n * k;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < m;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = nbr[s];
        const int32_t mr = mirror[s];
        int32_t rp = -1;
        if (mr < 0) {
            rp = rev_ptr[u] + atomicAdd(&revfill[u], 1);
            rev[rp] = (int32_t)s;
        }
        if (canon[s]) {
            const int32_t v = (int32_t)(s / k);
            const bool vlo = cid_of(cid, v) < cid_of(cid, u);
            erec[epos[s]] = make_int4((int32_t)s, vlo ? v : u, vlo ? u : v, mr >= 0 ? mr : -2 - rp);
        }
    }
}

// Row-local form for k dividing 32: a warp holds whole rows, so the edge
// position of a canonical slot is the row's start (a scan over per-row
// counts) plus the canonical slots before it in the row (a ballot), and no
// per-slot flag array or n*k-element scan is needed.
template <int K>
__global__ void k_slot_classify_rows(const int32_t *__restrict__ nbr, int64_t n,
                                     const int32_t *__restrict__ cid, int32_t *mirror,
                                     int32_t *rowcnt, int32_t *revcnt) {
    // The K ids of a target row are read by K/4 lanes (16 bytes each, one
    // contiguous 4K-byte row), 128/K rows per round, K/4 rounds for the 32
    // slots of the warp; each lane then takes the position found for its own
    // slot by a shuffle.
    constexpr int LPR = K / 4;          // lanes per target row
    constexpr int RPI = 32 / LPR;       // target rows per round
    constexpr int ITERS = 32 / RPI;     // rounds (= K / 4)
    const int64_t m = n * K;
    const int lane = threadIdx.x & 31;
    const unsigned rowmask = K == 32 ? FULL_MASK : ((1u << K) - 1u);
    for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < m; b0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = b0 + threadIdx.x;
        const bool valid = s < m;
        const int32_t v = (int32_t)(s / K);
        const int32_t u = valid ? nbr[s] : 0;
        const int64_t wbase = s - lane;  // slot of lane 0
        int tpr[ITERS];
#pragma unroll
        for (int it = 0; it < ITERS; it++) {
            const int j = it * RPI + lane / LPR;   // slot whose target row this lane reads
            const int chunk = lane % LPR;
            const int32_t uj = __shfl_sync(FULL_MASK, u, j);
            const int32_t vj = (int32_t)((wbase + j) / K);
            int found = -1;
            if (wbase + j < m) {
                const int4 r = __ldg((const int4 *)(nbr + (int64_t)uj * K) + chunk);
                const int t0 = 4 * chunk;
                if (r.w == vj) found = t0 + 3;
                if (r.z == vj) found = t0 + 2;
                if (r.y == vj) found = t0 + 1;
                if (r.x == vj) found = t0;
            }
            // a row holds v at most once: the group's maximum is the position
#pragma unroll
            for (int o = 1; o < LPR; o <<= 1) found = max(found, __shfl_xor_sync(FULL_MASK, found, o));
            tpr[it] = found;
        }
        int tp = -1;
#pragma unroll
        for (int it = 0; it < ITERS; it++) {
            const int x = __shfl_sync(FULL_MASK, tpr[it], (lane % RPI) * LPR);
            if (lane / RPI == it) tp = x;
        }
        // slot code for the fill: partner slot (mutual, v the lower id), -3
        // (mutual, not canonical), -1 / -2 (not mutual, v lower / higher)
        bool canon = false;
        if (valid) {
            const bool vlo = cid_of(cid, v) < cid_of(cid, u);
            if (tp >= 0) {
                mirror[s] = vlo ? u * K + tp : -3;
                canon = vlo;
            } else {
                mirror[s] = vlo ? -1 : -2;
                canon = true;
                atomicAdd(&revcnt[u], 1);
            }
        }
        const unsigned cm = __ballot_sync(FULL_MASK, canon);
        const int first = lane - lane % K;  // first lane of this slot's row
        if (valid && lane == first) rowcnt[s / K] = __popc(cm & (rowmask << first));
    }
}

// Fill from the slot codes of k_slot_classify_rows: no canonical-id loads.
__global__ void k_slot_fill_rows(const int32_t *__restrict__ nbr, int64_t n, int k,
                                 const int32_t *__restrict__ code,
                                 const int32_t *__restrict__ rowpos,
                                 const int32_t *__restrict__ rev_ptr, int32_t *revfill, int4 *erec,
                                 int32_t *rev) {
    const int64_t m = n * k;
    const int lane = threadIdx.x & 31;
    for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < m; b0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = b0 + threadIdx.x;
        bool canon = false;
        int32_t u = 0, c = -3, v = 0, rp = 0, rv = 0;
        if (s < m) {
            v = (int32_t)(s / k);
            u = __ldg(nbr + s);
            c = __ldg(code + s);
            rp = __ldg(rowpos + v);      // loaded before they are known to be needed
            rv = __ldg(rev_ptr + u);
            canon = c != -3;
        }
        const bool in_rev = c == -1 || c == -2;
        int32_t at = 0;
        if (in_rev) at = atomicAdd(&revfill[u], 1);
        const unsigned cm = __ballot_sync(FULL_MASK, canon);
        const int first = lane - lane % k;
        if (canon) {
            const int32_t pos = rp + __popc(cm & ((1u << lane) - 1u) & ~((1u << first) - 1u));
            const bool vlo = c >= 0 || c == -1;
            // 4th field: the mirror slot of a mutual edge, else -2 - (in-slot position)
            erec[pos] = make_int4((int32_t)s, vlo ? v : u, vlo ? u : v, c >= 0 ? c : -2 - (rv + at));
        }
        if (in_rev) rev[rv + at] = (int32_t)s;
    }
}

__global__ void k_zero2(int32_t *a, int32_t *b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        a[i] = 0;
        b[i] = 0;
    }
}

// lexicographic view: keys (lo, hi) of each edge record
__global__ void k_lex_keys(const int4 *__restrict__ erec, int64_t ne,
                           const int32_t *__restrict__ cid, uint32_t *klo, uint32_t *khi,
                           uint32_t *val) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int4 r = erec[e];
        klo[e] = cid_of(cid, r.y);
        khi[e] = cid_of(cid, r.z);
        val[e] = (uint32_t)e;
    }
}

__global__ void k_lex_view(const uint32_t *__restrict__ klo, const uint32_t *__restrict__ khi,
                           const uint32_t *__restrict__ perm, const int4 *__restrict__ erec,
                           int64_t ne, int32_t *elo, int32_t *ehi, int4 *erec_lex) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        elo[e] = (int32_t)klo[e];
        ehi[e] = (int32_t)khi[e];
        erec_lex[e] = erec[perm[e]];
    }
}

// ---------------------------------------------------------------- local refresh
// Sec. 3.4, local neighbourhood refresh: the kNN is queried again near the
// splats a pass created, instead of for every row.  The lists
// of a pass are carried through its merge: a kept row keeps the new ids of
// its old neighbours when they are still k_eff distinct splats other than
// itself; new splats and rows whose list collapsed are queried again.

__global__ void k_refresh_keep(int64_t n, const int32_t *__restrict__ role, int32_t *keep) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        keep[v] = role[v] != -2;
}

__global__ void k_refresh_map(int64_t n_old, const int32_t *__restrict__ role,
                              const int32_t *__restrict__ pos, int32_t *map_old, int32_t *src_new) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_old;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = role[o];
        if (r == -2) continue;
        const int32_t p = pos[o];
        map_old[o] = p;
        src_new[p] = r == -1 ? (int32_t)o : -1;
        if (r >= 0) map_old[r] = p;  // the removed partner names the merged splat
    }
}

__device__ __forceinline__ float dist2_rn3(float dx, float dy, float dz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// ascending bitonic network over N register keys
template <int N>
__device__ __forceinline__ void sort_asc_u64(uint64_t (&a)[N]) {
#pragma unroll
    for (int k = 2; k <= N; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < N; i++) {
                const int l = i ^ j;
                if (l > i) {
                    const uint64_t x = a[i], y = a[l];
                    const bool up = (i & k) == 0;
                    const bool sw = up ? (x > y) : (x < y);
                    a[i] = sw ? y : x;
                    a[l] = sw ? x : y;
                }
            }
}

// K = k_eff in {4, 8, 16, 32}; K = 0 for any width up to NGS_MAX_K
// An old list entry outside [0, n_old) sets *err and the row is queried.
template <int K>
__global__ void k_refresh_rows(int64_t n, int keff, int k_old, int64_t n_old,
                               const int32_t *__restrict__ src_new,
                               const int32_t *__restrict__ prev, const int32_t *__restrict__ map_old,
                               const float *__restrict__ xyz, const int32_t *__restrict__ cid,
                               int32_t *nbr, int32_t *qflag, int32_t *err) {
    constexpr int KM = K > 0 ? K : NGS_MAX_K;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = src_new[r];
        bool rq = o < 0 || k_old != keff;
        uint64_t key[KM];
        if (!rq) {
            const float x = xyz[3 * r], y = xyz[3 * r + 1], z = xyz[3 * r + 2];
#pragma unroll
            for (int t = 0; t < KM; t++) {
                if (K == 0 && t >= keff) {
                    key[t] = ~0ull;
                    continue;
                }
                const int32_t po = prev[(int64_t)o * k_old + t];
                if (po < 0 || po >= n_old) {
                    atomicOr(err, 1);
                    rq = true;
                    key[t] = ~0ull;
                    continue;
                }
                const int32_t m = map_old[po];
                rq = rq || m == (int32_t)r;
                const float d2 = dist2_rn3(__fsub_rn(x, xyz[3 * (int64_t)m]),
                                           __fsub_rn(y, xyz[3 * (int64_t)m + 1]),
                                           __fsub_rn(z, xyz[3 * (int64_t)m + 2]));
                const uint32_t id = cid ? (uint32_t)cid[m] : (uint32_t)m;
                key[t] = ((uint64_t)__float_as_uint(d2) << 32) | id;
            }
            sort_asc_u64<KM>(key);
            // a repeated id gives equal keys, now side by side
#pragma unroll
            for (int t = 0; t + 1 < KM; t++)
                if (K > 0 || t + 1 < keff) rq = rq || key[t] == key[t + 1];
        }
        qflag[r] = rq ? 1 : 0;
        if (!rq) {
#pragma unroll
            for (int t = 0; t < KM; t++)
                if (K > 0 || t < keff) nbr[r * keff + t] = (int32_t)(uint32_t)key[t];
        }
    }
}

__global__ void k_check_ids(const int32_t *__restrict__ a, int64_t m, int64_t n, int32_t *err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        if (a[i] < 0 || a[i] >= n) atomicOr(err, 1);
}

__global__ void k_qpos_flags(int64_t n, const uint32_t *__restrict__ order,
                             const int32_t *__restrict__ qflag, int32_t *f) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        f[p] = qflag[order[p]];
}

__global__ void k_qpos_write(int64_t n, const int32_t *__restrict__ f,
                             const int32_t *__restrict__ fpos, int32_t *qlist) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        if (f[p]) qlist[fpos[p]] = (int32_t)p;
}

}  // namespace

void build_edges(ngs_ctx *c, const int32_t *nbr, GraphDev &g) {
    const int64_t n = g.n;
    const int k = g.k_eff;
    g.n_edges = 0;
    g.nbr = nbr;
    if (n <= 1 || k <= 0) return;
    const int64_t m = n * k;
    g.mirror = ws<int32_t>(c, c->b_adj, m);
    int32_t *canon = ws<int32_t>(c, c->b_flag, m + 1);
    int32_t *epos = ws<int32_t>(c, c->b_adjeid, m + 1);
    int32_t *revcnt = ws<int32_t>(c, c->b_deg, n + 1);
    int32_t *revfill = ws<int32_t>(c, c->b_fill, n + 1);
    g.rev_ptr = ws<int32_t>(c, c->b_rstart, n + 1);
    launch(c, "zero2", dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0, k_zero2, revcnt,
           revfill, n);
    const bool rows = k % 4 == 0 && 32 % k == 0;  // a warp holds whole rows of int4 chunks
    if (rows) {
        const dim3 gr(grid_stride_blocks(c, m, 256, 16)), bl(256);
        switch (k) {
        case 4: launch(c, "slot_classify", gr, bl, 0, k_slot_classify_rows<4>, nbr, n, g.cid, g.mirror, canon, revcnt); break;
        case 8: launch(c, "slot_classify", gr, bl, 0, k_slot_classify_rows<8>, nbr, n, g.cid, g.mirror, canon, revcnt); break;
        case 16: launch(c, "slot_classify", gr, bl, 0, k_slot_classify_rows<16>, nbr, n, g.cid, g.mirror, canon, revcnt); break;
        default: launch(c, "slot_classify", gr, bl, 0, k_slot_classify_rows<32>, nbr, n, g.cid, g.mirror, canon, revcnt); break;
        }
        scan_i32(c, canon, epos, n);  // per-row canonical counts -> row starts
    } else {
        launch(c, "slot_classify", dim3(grid_stride_blocks(c, m, 256, 16)), dim3(256), 0,
               k_slot_classify, nbr, n, k, g.cid, g.mirror, canon, revcnt);
        scan_i32(c, canon, epos, m);
    }
    scan_i32(c, revcnt, g.rev_ptr, n);
    get_small(c, c->h_pin, epos + (rows ? n : m), 4);
    get_small(c, (int32_t *)c->h_pin + 1, g.rev_ptr + n, 4);
    sync_stream(c);
    g.n_edges = ((int32_t *)c->h_pin)[0];
    const int64_t nrev = ((int32_t *)c->h_pin)[1];
    g.erec = ws<int4>(c, c->b_elo, g.n_edges);
    g.rev = ws<int32_t>(c, c->b_upc, nrev);
    g.revcost = ws<float>(c, c->b_revcost, nrev);
    if (rows)
        launch(c, "slot_fill", dim3(grid_stride_blocks(c, m, 256, 16)), dim3(256), 0,
               k_slot_fill_rows, nbr, n, k, (const int32_t *)g.mirror,
               (const int32_t *)epos, (const int32_t *)g.rev_ptr, revfill, g.erec, g.rev);
    else
        launch(c, "slot_fill", dim3(grid_stride_blocks(c, m, 256, 16)), dim3(256), 0, k_slot_fill,
               nbr, n, k, g.cid, (const int32_t *)g.mirror, (const int32_t *)canon,
               (const int32_t *)epos, (const int32_t *)g.rev_ptr, revfill, g.erec, g.rev);
    g.cost_slot = ws<float>(c, c->b_cost, m);
}

void build_lex_view(ngs_ctx *c, GraphDev &g) {
    const int64_t ne = g.n_edges;
    if (ne <= 0) return;
    uint32_t *klo = ws<uint32_t>(c, c->b_codes, ne), *khi = ws<uint32_t>(c, c->b_codes2, ne);
    uint32_t *val = ws<uint32_t>(c, c->b_vals, ne);
    uint32_t *t1 = ws<uint32_t>(c, c->b_vals2, ne);
    launch(c, "lex_keys", dim3(grid_stride_blocks(c, ne, 256, 8)), dim3(256), 0, k_lex_keys,
           (const int4 *)g.erec, ne, g.cid, klo, khi, val);
    // LSD over (lo, hi): stable sort by hi, then by lo.  Payload = record index.
    uint32_t *idx = ws<uint32_t>(c, c->b_cid, ne), *idx2 = ws<uint32_t>(c, c->b_cid2, ne);
    uint32_t *ktmp = ws<uint32_t>(c, c->b_pos, ne);
    iota_u32(c, idx, ne);
    NGS_CHECK_CUDA(cudaMemcpyAsync(t1, khi, 4 * ne, cudaMemcpyDeviceToDevice, c->st));
    radix_sort_u32(c, t1, idx, ktmp, idx2, ne, 32);
    gather_u32(c, klo, idx, ne, t1);          // lo in hi-sorted order
    radix_sort_u32(c, t1, idx, ktmp, idx2, ne, 32);
    g.elo = ws<int32_t>(c, c->b_ehi, ne);
    g.ehi = ws<int32_t>(c, c->b_nbr2, ne);
    g.erec_lex = ws<int4>(c, c->b_lexrec, ne);
    gather_u32(c, khi, idx, ne, ktmp);
    launch(c, "lex_view", dim3(grid_stride_blocks(c, ne, 256, 8)), dim3(256), 0, k_lex_view,
           (const uint32_t *)t1, (const uint32_t *)ktmp, (const uint32_t *)idx,
           (const int4 *)g.erec, ne, g.elo, g.ehi, g.erec_lex);
}

void refresh_map(ngs_ctx *c, int64_t n_old, const int32_t *role, int32_t *map_old,
                 int32_t *src_new) {
    if (n_old <= 0) return;
    // new rows: the exclusive scan of the surviving old rows
    int32_t *keep = ws<int32_t>(c, c->b_qflag, n_old + 1);
    int32_t *pos = ws<int32_t>(c, c->b_qlist, n_old + 1);
    const unsigned grid = grid_stride_blocks(c, n_old, 256, 8);
    launch(c, "refresh_keep", dim3(grid), dim3(256), 0, k_refresh_keep, n_old, role, keep);
    scan_i32(c, keep, pos, n_old);
    launch(c, "refresh_map", dim3(grid), dim3(256), 0, k_refresh_map, n_old, role,
           (const int32_t *)pos, map_old, src_new);
}

int64_t refresh_rows(ngs_ctx *c, int64_t n, int k_eff, int k_old, int64_t n_old,
                     const int32_t *src_new, const int32_t *prev, const int32_t *map_old,
                     const float *xyz, const int32_t *cid, const uint32_t *order, int32_t *nbr,
                     int32_t *qlist) {
    if (n <= 0) return 0;
    int32_t *qflag = ws<int32_t>(c, c->b_qflag, n + 1);
    int32_t *err = (int32_t *)ws<uint8_t>(c, c->b_status, 64) + 12;
    NGS_CHECK_CUDA(cudaMemsetAsync(err, 0, 4, c->st));
    const dim3 gr(grid_stride_blocks(c, n, 128, 16)), bl(128);
#define REFRESH_LAUNCH(KT)                                                                      \
    launch(c, "refresh_rows", gr, bl, 0, k_refresh_rows<KT>, n, k_eff, k_old, n_old, src_new,   \
           prev, map_old, xyz, cid, nbr, qflag, err)
    switch (k_eff) {
    case 4: REFRESH_LAUNCH(4); break;
    case 8: REFRESH_LAUNCH(8); break;
    case 16: REFRESH_LAUNCH(16); break;
    case 32: REFRESH_LAUNCH(32); break;
    default: REFRESH_LAUNCH(0); break;
    }
#undef REFRESH_LAUNCH
    get_small(c, (int32_t *)(c->h_pin + 6) + 1, err, 4);
    // sorted positions of the rows to query
    int32_t *f = ws<int32_t>(c, c->b_keep, n + 1);
    int32_t *fpos = ws<int32_t>(c, c->b_pos, n + 1);
    const unsigned grid = grid_stride_blocks(c, n, 256, 8);
    launch(c, "qpos_flags", dim3(grid), dim3(256), 0, k_qpos_flags, n, order,
           (const int32_t *)qflag, f);
    scan_i32(c, f, fpos, n);
    launch(c, "qpos_write", dim3(grid), dim3(256), 0, k_qpos_write, n, (const int32_t *)f,
           (const int32_t *)fpos, qlist);
    get_small(c, c->h_pin + 6, fpos + n, 4);
    sync_stream(c);
    if (((int32_t *)(c->h_pin + 6))[1])
        NGS_FAIL(NGS_ERR_INVALID_ARG, "refresh: a previous list entry is outside [0, %lld)",
                 (long long)n_old);
    return *(int32_t *)(c->h_pin + 6);
}

bool ids_in_range(ngs_ctx *c, const int32_t *a, int64_t m, int64_t n) {
    if (m <= 0) return true;
    int32_t *err = (int32_t *)ws<uint8_t>(c, c->b_status, 64) + 13;
    NGS_CHECK_CUDA(cudaMemsetAsync(err, 0, 4, c->st));
    launch(c, "check_ids", dim3(grid_stride_blocks(c, m, 256, 8)), dim3(256), 0, k_check_ids, a, m,
           n, err);
    get_small(c, (int32_t *)(c->h_pin + 7), err, 4);
    sync_stream(c);
    return *(int32_t *)(c->h_pin + 7) == 0;
}
