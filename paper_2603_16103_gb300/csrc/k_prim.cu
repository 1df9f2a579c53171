// Device-wide primitives: exclusive scan, stable LSD radix sort and radix
// select.  The scan is single-pass (decoupled look-back) with bounded waits;
// the sort and select are deterministic multi-kernel designs (no waiting).
#include <cstring>

#include "ngs_device.cuh"
#include "ngs_internal.h"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-wide exclusive scan of one int per thread; returns the prefix and
// the block total in *total.
__device__ int block_excl_scan(int v, int *total) {
    __shared__ int wsum[32];
    __shared__ int wtot;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = warp_incl_scan(v, lane);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int nw = blockDim.x >> 5;
    if (warp == 0) {
        int w = lane < nw ? wsum[lane] : 0;
        int wi = warp_incl_scan(w, lane);
        if (lane < nw) wsum[lane] = wi - w;
        if (lane == nw - 1) wtot = wi;
    }
    __syncthreads();
    int res = incl - v + wsum[warp];
    *total = wtot;
    __syncthreads();
    return res;
}

__global__ void k_scan_reduce(const int32_t *__restrict__ in, int64_t n, int32_t *part) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int s = 0;
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; r++) {
        int64_t i = base + r * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    int tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_scan_partials(int32_t *part, int64_t nb) {
    // single block: exclusive scan of part[0..nb) in chunks
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int v = i < nb ? part[i] : 0;
        int tot;
        int ex = block_excl_scan(v, &tot);
        if (i < nb) part[i] = ex + carry;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) part[nb] = carry;
}

// Same result with 16-byte accesses: the tile is taken in SCAN_ITEMS / 4
// rounds of 4 consecutive items per thread, so every warp load and store
// covers 512 contiguous bytes (in and out 16-byte aligned; in == out allowed).
__global__ void k_scan_apply_v4(const int32_t *in, int32_t *out, int64_t n, const int32_t *part) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int carry = part[blockIdx.x];
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS / 4; r++) {
        const int64_t i0 = base + (int64_t)r * (4 * SCAN_THREADS) + 4 * threadIdx.x;
        int4 v = make_int4(0, 0, 0, 0);
        if (i0 + 3 < n) {
            v = *(const int4 *)(in + i0);
        } else if (i0 < n) {
            v.x = in[i0];
            if (i0 + 1 < n) v.y = in[i0 + 1];
            if (i0 + 2 < n) v.z = in[i0 + 2];
        }
        int tot;
        const int ex = block_excl_scan(v.x + v.y + v.z + v.w, &tot) + carry;
        const int4 o = make_int4(ex, ex + v.x, ex + v.x + v.y, ex + v.x + v.y + v.z);
        if (i0 + 3 < n) {
            *(int4 *)(out + i0) = o;
        } else if (i0 < n) {
            out[i0] = o.x;
            if (i0 + 1 < n) out[i0 + 1] = o.y;
            if (i0 + 2 < n) out[i0 + 2] = o.z;
        }
        carry += tot;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = part[gridDim.x];
}

__global__ void k_scan_apply(const int32_t *in, int32_t *out, int64_t n, const int32_t *part) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; r++) {
        int64_t i = base + r;
        v[r] = i < n ? in[i] : 0;
        s += v[r];
    }
    int tot;
    int ex = block_excl_scan(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; r++) {
        int64_t i = base + r;
        if (i < n) out[i] = ex;
        ex += v[r];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = part[gridDim.x];
}

// ---------------------------------------------------------------- single-pass scan
// Exclusive scan in one kernel by decoupled look-back (Merrill and Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016): tile t
// is block t (blocks start in index order, so a tile's predecessors are
// running or done; a counter handing out tile ids costs a serialised atomic
// per tile, a third of the time of the 134 M-entry cell-table scan); each
// publishes its aggregate,
// then walks back over its predecessors' published words (an aggregate, or
// an inclusive prefix that ends the walk), publishes its own inclusive prefix
// and writes its outputs.  Published word: flag (bits 63..62: 1 aggregate,
// 2 inclusive) | 32-bit value.
//
// Every wait is bounded: a predecessor that has published nothing after
// `budget` clock cycles has its tile summed from the inputs instead (then
// read again: if it published meanwhile its word is used), and *err is set
// (reported as NGS_ERR_TIMEOUT).  Results stay exact, also in place: a tile
// writes outputs only after publishing, so inputs read while it has published
// nothing are still inputs.  delay_tile (tests of the bounded wait) makes that
// tile wait 4 budgets before publishing.
constexpr int LB_THREADS = 256;
constexpr int LB_ITEMS = 32;  // consecutive items per thread: 8192 per tile
constexpr int LB_TILE = LB_THREADS * LB_ITEMS;
constexpr int LB_WORDS = 4;   // predecessors read per lane and round: a window of 128
constexpr uint64_t LB_AGG = 1ull << 62, LB_INC = 2ull << 62;

__device__ __forceinline__ void st_release_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// polling load: the word carries its own value, so no acquire ordering is needed
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Exclusive prefix of tile `tile` by warp 0.  Each round reads the 128
// nearest unread predecessors (lane l the four at distances 4l .. 4l+3); the
// nearest inclusive word ends the walk, and every nearer word must hold an
// aggregate (else the round is read again); without an inclusive word the
// 128 aggregates are added and the window moves back.  The inclusive
// frontier so advances up to 128 tiles (1 M items) per L2 round trip.
__device__ __forceinline__ int lookback_warp(const int32_t *in, int64_t n, int64_t tile,
                                             uint64_t *status, long long budget, bool &late) {
    const int lane = threadIdx.x & 31;
    const long long t0 = clock64();
    int prefix = 0;
    for (int64_t p = tile - 1;;) {
        uint64_t w[LB_WORDS];
#pragma unroll
        for (int k = 0; k < LB_WORDS; k++) {
            const int64_t q = p - LB_WORDS * lane - k;
            w[k] = q >= 0 ? ld_relaxed_u64(status + 1 + q) : LB_INC;  // before tile 0: 0
        }
        // nearest inclusive word of this lane (LB_WORDS: none), then of the warp
        int lfi = LB_WORDS;
#pragma unroll
        for (int k = LB_WORDS - 1; k >= 0; k--)
            if ((w[k] >> 62) == 2) lfi = k;
        unsigned inc = __ballot_sync(FULL_MASK, lfi < LB_WORDS);
        int fl = inc ? __ffs(inc) - 1 : 32;  // first lane holding one
        // words needed: all of lanes before fl, those up to lfi in lane fl
        auto needed = [&](int k) { return lane < fl || (lane == fl && k <= lfi); };
        bool miss = false;
#pragma unroll
        for (int k = 0; k < LB_WORDS; k++) miss = miss || (needed(k) && (w[k] >> 62) == 0);
        if (__any_sync(FULL_MASK, miss)) {
            long long el = lane == 0 ? clock64() - t0 : 0;
            el = __shfl_sync(FULL_MASK, el, 0);
            if (!late && el <= budget) {  // wait: read the window again
                __nanosleep(64);
                continue;
            }
            late = true;
            // out of budget: a needed tile that published nothing is summed
            // from its inputs, unless it publishes meanwhile
#pragma unroll
            for (int k = 0; k < LB_WORDS; k++) {
                if (needed(k) && (w[k] >> 62) == 0) {
                    const int64_t q = p - LB_WORDS * lane - k;
                    int s = 0;
                    const int64_t e = (q + 1) * LB_TILE < n ? (q + 1) * LB_TILE : n;
                    for (int64_t i = q * LB_TILE; i < e; i++) s += in[i];
                    __threadfence();  // the inputs were read before the word is read again
                    const uint64_t w2 = ld_relaxed_u64(status + 1 + q);
                    w[k] = (w2 >> 62) ? w2 : (LB_AGG | (uint32_t)s);
                }
            }
            lfi = LB_WORDS;
#pragma unroll
            for (int k = LB_WORDS - 1; k >= 0; k--)
                if ((w[k] >> 62) == 2) lfi = k;
            inc = __ballot_sync(FULL_MASK, lfi < LB_WORDS);
            fl = inc ? __ffs(inc) - 1 : 32;
        }
        int v = 0;
#pragma unroll
        for (int k = 0; k < LB_WORDS; k++)
            if (needed(k)) v += (int)(uint32_t)w[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
        prefix += v;
        if (inc) return prefix;
        p -= 32 * LB_WORDS;
    }
}

__global__ void __launch_bounds__(LB_THREADS)
    k_scan_lookback(const int32_t *in, int32_t *out, int64_t n, int64_t ntiles,
                    uint64_t *status /* [1 + t] tile t */, long long budget,
                    int64_t delay_tile, volatile int32_t *err) {
    __shared__ int s_prefix;
    const int64_t tile = blockIdx.x;
    const int64_t i0 = tile * LB_TILE + (int64_t)threadIdx.x * LB_ITEMS;
    const bool full = i0 + LB_ITEMS <= n;
    int v[LB_ITEMS];
    if (full && ((((uintptr_t)in) & 15) == 0)) {
#pragma unroll
        for (int r = 0; r < LB_ITEMS / 4; r++) {
            const int4 a = *(const int4 *)(in + i0 + 4 * r);
            v[4 * r] = a.x; v[4 * r + 1] = a.y; v[4 * r + 2] = a.z; v[4 * r + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int r = 0; r < LB_ITEMS; r++) v[r] = i0 + r < n ? in[i0 + r] : 0;
    }
    int sum = 0;
#pragma unroll
    for (int r = 0; r < LB_ITEMS; r++) sum += v[r];
    int tot;
    const int ex = block_excl_scan(sum, &tot);
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0 && tile == delay_tile) {
            const long long t0 = clock64();
            while (clock64() - t0 < 4 * budget) {
            }
        }
        __syncwarp();
        int prefix = 0;
        if (tile == 0) {
            if (threadIdx.x == 0) st_release_u64(status + 1, LB_INC | (uint32_t)tot);
        } else {
            if (threadIdx.x == 0) st_release_u64(status + 1 + tile, LB_AGG | (uint32_t)tot);
            bool late = false;
            prefix = lookback_warp(in, n, tile, status, budget, late);
            if (threadIdx.x == 0) {
                if (late) *err = NGS_ERR_TIMEOUT;
                st_release_u64(status + 1 + tile, LB_INC | (uint32_t)(prefix + tot));
            }
        }
        if (threadIdx.x == 0) s_prefix = prefix;
    }
    __syncthreads();
    int o = s_prefix + ex;
    if (full && ((((uintptr_t)out) & 15) == 0)) {
#pragma unroll
        for (int r = 0; r < LB_ITEMS / 4; r++) {
            int4 q;
            q.x = o; o += v[4 * r];
            q.y = o; o += v[4 * r + 1];
            q.z = o; o += v[4 * r + 2];
            q.w = o; o += v[4 * r + 3];
            *(int4 *)(out + i0 + 4 * r) = q;
        }
    } else {
#pragma unroll
        for (int r = 0; r < LB_ITEMS; r++) {
            if (i0 + r < n) out[i0 + r] = o;
            o += v[r];
        }
    }
    if (tile == ntiles - 1 && threadIdx.x == 0) out[n] = s_prefix + tot;
}

// ---------------------------------------------------------------- small uploads
// A few bytes from the host travel as a kernel parameter instead of through a
// copy engine, so they never share one with a large transfer in flight (the
// SH upload of ngs_simplify_host runs on a second stream meanwhile).
constexpr size_t PUT_MAX = 3072;
struct PutPayload {
    unsigned char b[PUT_MAX];
};

__global__ void k_put(unsigned char *dst, const PutPayload p, int bytes) {
    for (int i = threadIdx.x; i < bytes; i += blockDim.x) dst[i] = p.b[i];
}

// The reverse for small results: a kernel stores them into pinned host
// memory (device-accessible), again without a copy engine.
__global__ void k_get(unsigned char *hdst, const unsigned char *__restrict__ src, int bytes) {
    for (int i = threadIdx.x; i < bytes; i += blockDim.x) hdst[i] = src[i];
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void k_rs_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                          int32_t *hist, int64_t ntiles) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan, in place, of each digit's row of tile counts (one block per
// digit, rows of the digit-major histogram); the row total goes to tot[d].
__global__ void __launch_bounds__(1024) k_rs_rowscan(int32_t *hist, int64_t ntiles, int32_t *tot) {
    int32_t *row = hist + (int64_t)blockIdx.x * ntiles;
    int carry = 0;
    for (int64_t b = 0; b < ntiles; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const int v = i < ntiles ? row[i] : 0;
        int t;
        const int ex = block_excl_scan(v, &t);  // ends with a barrier
        if (i < ntiles) row[i] = carry + ex;
        carry += t;
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

// Stable scatter of one tile.  Warp w ranks the tile's items
// [256 w, 256 w + 256) in index order, 32 at a time, against its own digit
// counts (warp match, no block barrier); one prefix per digit over the warps
// then places every item in shared memory in digit order, and the tile is
// written out from there, consecutive threads at consecutive positions of a
// digit's run.  offs[d * ntiles + t] counts the keys of digit d in tiles
// before t, tot[d] all keys of digit d; a tile's count of digit d is the
// difference of two adjacent entries of its row.
__global__ void __launch_bounds__(RS_THREADS)
    k_rs_scatter(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                 uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
                 const int32_t *__restrict__ offs, const int32_t *__restrict__ tot,
                 int64_t ntiles) {
    constexpr int NW = RS_THREADS / 32;
    static_assert(RS_ITEMS * 32 * NW == RS_TILE, "a warp ranks RS_ITEMS rows of 32 items");
    __shared__ uint32_t sk[RS_TILE], sv[RS_TILE];
    __shared__ int wh[NW][256];  // per-warp digit counts, then per-warp start positions
    __shared__ int gb[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const int tcount = (int)(n - base < RS_TILE ? n - base : RS_TILE);
#pragma unroll
    for (int w = 0; w < NW; w++) wh[w][tid] = 0;
    int lo;
    {
        const int64_t at = (int64_t)tid * ntiles + blockIdx.x;
        const int o = offs[at];
        const int td = tot[tid];
        const int cnt = (blockIdx.x + 1 < ntiles ? offs[at + 1] : td) - o;
        int all, tcnt;
        const int base = block_excl_scan(td, &all);  // keys of smaller digits
        lo = block_excl_scan(cnt, &tcnt);            // ends with a barrier: wh is zero
        gb[tid] = base + o - lo;                     // global position = gb[d] + local position
    }
    const unsigned lt_mask = (1u << lane) - 1u;
    uint32_t key[RS_ITEMS], val[RS_ITEMS];
    int dg[RS_ITEMS], rk[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        const int j = warp * (32 * RS_ITEMS) + r * 32 + lane;
        const bool valid = j < tcount;
        key[r] = valid ? kin[base + j] : 0u;
        val[r] = valid ? vin[base + j] : 0u;
        const int d = valid ? (int)((key[r] >> shift) & 255u) : 256 + lane;  // invalid: own group
        const unsigned peers = __match_any_sync(FULL_MASK, d);
        const int before = valid ? wh[warp][d] : 0;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wh[warp][d] = before + __popc(peers);
        __syncwarp();
        dg[r] = d;
        rk[r] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    {
        int p = lo;  // digit tid: its local start, then each warp's share in order
#pragma unroll
        for (int w = 0; w < NW; w++) {
            const int t = wh[w][tid];
            wh[w][tid] = p;
            p += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        if (dg[r] < 256) {
            const int lp = wh[warp][dg[r]] + rk[r];
            if ((unsigned)lp < (unsigned)RS_TILE) {
                sk[lp] = key[r];
                sv[lp] = val[r];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        const int j = r * RS_THREADS + tid;
        if (j < tcount) {
            const uint32_t k = sk[j];
            const int64_t p = (int64_t)gb[(k >> shift) & 255u] + j;
            if ((uint64_t)p < (uint64_t)n) {
                kout[p] = k;
                vout[p] = sv[j];
            }
        }
    }
}

// ---------------------------------------------------------------- radix select
// state: [0] prefix lo32, [1] prefix hi32, [2] mask lo, [3] mask hi, [4..5] rank (int64)
struct SelState {
    uint64_t prefix;
    uint64_t mask;
    int64_t rank;
};

__global__ void k_sel_init(SelState *s, int64_t k, int32_t *hist) {
    if (threadIdx.x == 0) {
        s->prefix = 0;
        s->mask = 0;
        s->rank = k;
    }
    hist[threadIdx.x] = 0;
}

template <class K>
__global__ void k_sel_hist(const K *__restrict__ keys, int64_t n, const SelState *s, int shift,
                           int32_t *hist, bool skip_max) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    uint64_t prefix = s->prefix, mask = s->mask;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = (uint64_t)keys[i];
        if (skip_max && k == (uint64_t)(K)(~(K)0)) continue;
        if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 255u], 1);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_sel_decide(SelState *s, int32_t *hist, int shift) {
    __shared__ int h[256];
    h[threadIdx.x] = hist[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t r = s->rank, cum = 0;
        int d = 255;
        for (int b = 0; b < 256; b++) {
            if (r < cum + h[b]) {
                d = b;
                break;
            }
            cum += h[b];
        }
        s->rank = r - cum;
        s->prefix |= (uint64_t)d << shift;
        s->mask |= (uint64_t)255u << shift;
    }
    __syncthreads();
    hist[threadIdx.x] = 0;
}

__global__ void k_iota(uint32_t *a, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (uint32_t)i;
}

__global__ void k_gather_u32(const uint32_t *__restrict__ src, const uint32_t *__restrict__ idx,
                             int64_t n, uint32_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = src[idx[i]];
}

template <class K>
__global__ void k_sel_out(const SelState *s, K *out) {
    *out = (K)s->prefix;
}

}  // namespace

void scan_i32(ngs_ctx *c, const int32_t *in, int32_t *out, int64_t n) {
    if (c->tune.scan_method == 1 && c->err_word) {
        // single pass; the tile words start at zero
        int64_t nt = (n + LB_TILE - 1) / LB_TILE;
        if (nt < 1) nt = 1;
        uint64_t *st = ws<uint64_t>(c, c->b_scan_part, nt + 1);
        NGS_CHECK_CUDA(cudaMemsetAsync(st, 0, sizeof(uint64_t) * (nt + 1), c->st));
        launch(c, "scan", dim3((unsigned)nt), dim3(LB_THREADS), 0, k_scan_lookback, in, out, n, nt,
               st, (long long)c->tune.wait_budget_cycles, (int64_t)c->tune.wait_test_tile, c->err_word);
        return;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb < 1) nb = 1;
    int32_t *part = ws<int32_t>(c, c->b_scan_part, nb + 1);
    launch(c, "scan_reduce", dim3((unsigned)nb), dim3(SCAN_THREADS), 0, k_scan_reduce, in, n, part);
    launch(c, "scan_partials", dim3(1), dim3(1024), 0, k_scan_partials, part, nb);
    if ((((uintptr_t)in | (uintptr_t)out) & 15) == 0)
        launch(c, "scan_apply", dim3((unsigned)nb), dim3(SCAN_THREADS), 0, k_scan_apply_v4, in, out,
               n, (const int32_t *)part);
    else
        launch(c, "scan_apply", dim3((unsigned)nb), dim3(SCAN_THREADS), 0, k_scan_apply, in, out, n,
               (const int32_t *)part);
}

void radix_sort_u32(ngs_ctx *c, uint32_t *keys, uint32_t *vals, uint32_t *keys_tmp,
                    uint32_t *vals_tmp, int64_t n, int bits) {
    if (n <= 1) return;
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    // digit-major tile counts, then the 256 digit totals
    int32_t *hist = ws<int32_t>(c, c->b_hist, 256 * ntiles + 256 + 1);
    int32_t *tot = hist + 256 * ntiles;
    uint32_t *ka = keys, *va = vals, *kb = keys_tmp, *vb = vals_tmp;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        launch(c, "rs_hist", dim3((unsigned)ntiles), dim3(RS_THREADS), 0, k_rs_hist,
               (const uint32_t *)ka, n, shift, hist, ntiles);
        launch(c, "rs_rowscan", dim3(256), dim3(1024), 0, k_rs_rowscan, hist, ntiles, tot);
        launch(c, "rs_scatter", dim3((unsigned)ntiles), dim3(RS_THREADS), 0, k_rs_scatter,
               (const uint32_t *)ka, (const uint32_t *)va, kb, vb, n, shift,
               (const int32_t *)hist, (const int32_t *)tot, ntiles);
        uint32_t *t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    if (ka != keys) {
        NGS_CHECK_CUDA(cudaMemcpyAsync(keys, ka, n * 4, cudaMemcpyDeviceToDevice, c->st));
        NGS_CHECK_CUDA(cudaMemcpyAsync(vals, va, n * 4, cudaMemcpyDeviceToDevice, c->st));
    }
}

template <class K>
static void radix_select_impl(ngs_ctx *c, const K *keys, int64_t n, int64_t k, K *d_out,
                              bool skip_max) {
    uint8_t *misc = ws<uint8_t>(c, c->b_misc, 4096);
    SelState *st = (SelState *)misc;
    int32_t *hist = (int32_t *)(misc + 256);
    launch(c, "sel_init", dim3(1), dim3(256), 0, k_sel_init, st, k, hist);
    unsigned grid = grid_stride_blocks(c, n, 256, 4);
    for (int shift = (int)(8 * sizeof(K)) - 8; shift >= 0; shift -= 8) {
        launch(c, "sel_hist", dim3(grid), dim3(256), 0, k_sel_hist<K>, keys, n,
               (const SelState *)st, shift, hist, skip_max);
        launch(c, "sel_decide", dim3(1), dim3(256), 0, k_sel_decide, st, hist, shift);
    }
    launch(c, "sel_out", dim3(1), dim3(1), 0, k_sel_out<K>, (const SelState *)st, d_out);
}

void radix_select_u32(ngs_ctx *c, const uint32_t *keys, int64_t n, int64_t k, uint32_t *d_out) {
    radix_select_impl<uint32_t>(c, keys, n, k, d_out, false);
}

void radix_select_u64(ngs_ctx *c, const uint64_t *keys, int64_t n, int64_t k, uint64_t *d_out) {
    radix_select_impl<uint64_t>(c, keys, n, k, d_out, true);
}

void iota_u32(ngs_ctx *c, uint32_t *a, int64_t n) {
    launch(c, "iota", dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0, k_iota, a, n);
}

void gather_u32(ngs_ctx *c, const uint32_t *src, const uint32_t *idx, int64_t n, uint32_t *out) {
    launch(c, "gather_u32", dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0, k_gather_u32,
           src, idx, n, out);
}

void put_small(ngs_ctx *c, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return;
    if (bytes > PUT_MAX) {
        NGS_CHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->st));
        return;
    }
    PutPayload p;
    memcpy(p.b, src, bytes);
    launch(c, "put", dim3(1), dim3(256), 0, k_put, (unsigned char *)dst, p, (int)bytes);
}

void get_small(ngs_ctx *c, void *hdst, const void *dsrc, size_t bytes) {
    if (bytes == 0) return;
    launch(c, "get", dim3(1), dim3(256), 0, k_get, (unsigned char *)hdst,
           (const unsigned char *)dsrc, (int)bytes);
}
