// Disjoint pair selection (Sec. 3.4, Algorithm 1 GreedyDisjointPairs).
//
// The greedy rule -- sort edges by cost, scan, take an edge when both
// endpoints are free, stop after P picks -- is computed as a locally-dominant
// matching under the same strict order (cost, lo canonical id, hi canonical
// id), NaN ranked as +inf and -0 as +0:
//   * every free vertex points at its best edge to a free neighbour;
//   * mutual pointers are matched (such an edge is the minimum of all edges
//     touching either endpoint, so greedy would take it too);
//   * a vertex re-scans only when its target was matched elsewhere.
// Under a strict total order this reaches exactly the greedy matching.  A
// second form reaches the same matching by proposals (Manne and
// Halappanavar's Suitor scheme) in one kernel; see k_suitor.  The cap keeps
// the P smallest matched edges, which are the greedy's first P picks, found
// by a radix select on (cost bits, lo canonical id).
#include "ngs_device.cuh"
#include "ngs_internal.h"

namespace {

__device__ __forceinline__ uint32_t cid_of(const int32_t *cid, int32_t v) {
    return cid ? (uint32_t)cid[v] : (uint32_t)v;
}

__global__ void k_match_init(int64_t n, int32_t *mate, int32_t *cand) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        mate[v] = -1;
        cand[v] = -2;  // unknown
    }
}

// Re-scan the incident edges of free vertices whose pointer is unknown or
// stale: the k slots of the vertex, then its non-mutual in-slots.  All edges
// considered here contain v, and for a fixed v the order of (lo, hi) is the
// order of the other endpoint's canonical id (a lower neighbour gives a
// lower lo; two higher neighbours share lo = v).  Ties on cost are therefore
// broken by that id alone, loaded only when a tie occurs.
__device__ __forceinline__ void consider(int32_t u, float cst, const int32_t *__restrict__ cid,
                                         const int32_t *__restrict__ mate, bool all_free,
                                         int32_t &best, uint32_t &bk) {
    if (!all_free && mate[u] != -1) return;
    const uint32_t k = cost_order_bits(cst);
    if (best < 0 || k < bk) {
        best = u;
        bk = k;
    } else if (k == bk && cid_of(cid, u) < cid_of(cid, best)) {
        best = u;
    }
}

// K > 0: the list width k_eff = K, a multiple of 4; the slots are read as
// 16-byte vectors and the loop is unrolled, so the ids, costs and partner
// states of a vertex's slots are all in flight at once.  K = 0: any width.
template <int K>
__global__ void k_match_scan(const int32_t *__restrict__ wl, const int32_t *__restrict__ wl_count,
                             int64_t n_all, int kk, const int32_t *__restrict__ nbr,
                             const float *__restrict__ cost_slot,
                             const int32_t *__restrict__ rev_ptr, const int32_t *__restrict__ rev,
                             const int32_t *__restrict__ cid, const int32_t *__restrict__ mate,
                             int32_t *cand, uint32_t *candkey) {
    const int64_t cnt = wl ? (int64_t)*wl_count : n_all;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < cnt;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = wl ? (int64_t)wl[idx] : idx;
        if (mate[v] != -1) continue;
        int32_t c = cand[v];
        if (c == -1) continue;                  // no free neighbour: stays single
        if (c >= 0 && mate[c] == -1) continue;  // target still free: still the best
        const bool all_free = wl == nullptr;  // round 0: no vertex is matched yet
        int32_t best = -1;
        uint32_t bk = 0xffffffffu;
        const int64_t base = v * kk;
        if (K > 0) {
            // ids and costs, then every partner state, then the choice
            constexpr int KK = K > 0 ? K : 4;
            int32_t us[KK], ms[KK];
            float cs[KK];
            const int4 *nb4 = (const int4 *)(nbr + base);
            const float4 *cs4 = (const float4 *)(cost_slot + base);
#pragma unroll
            for (int t4 = 0; t4 < K / 4; t4++) {
                const int4 u4 = __ldg(nb4 + t4);
                const float4 c4 = __ldg(cs4 + t4);
                us[4 * t4] = u4.x; us[4 * t4 + 1] = u4.y; us[4 * t4 + 2] = u4.z; us[4 * t4 + 3] = u4.w;
                cs[4 * t4] = c4.x; cs[4 * t4 + 1] = c4.y; cs[4 * t4 + 2] = c4.z; cs[4 * t4 + 3] = c4.w;
            }
#pragma unroll
            for (int t = 0; t < KK; t++) ms[t] = all_free ? -1 : __ldg(mate + us[t]);
#pragma unroll
            for (int t = 0; t < KK; t++)
                if (ms[t] == -1) consider(us[t], cs[t], cid, mate, true, best, bk);
        } else {
            for (int t = 0; t < kk; t++)
                consider(nbr[base + t], cost_slot[base + t], cid, mate, all_free, best, bk);
        }
        // in-slots four at a time: slots, then costs and partner states
        const int32_t r1 = rev_ptr[v + 1];
        for (int32_t r = rev_ptr[v]; r < r1; r += 4) {
            int32_t ss[4], uu[4], mm[4];
            float cc[4];
#pragma unroll
            for (int q = 0; q < 4; q++) ss[q] = r + q < r1 ? __ldg(rev + r + q) : -1;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                uu[q] = ss[q] >= 0 ? ss[q] / kk : 0;
                cc[q] = ss[q] >= 0 ? __ldg(cost_slot + ss[q]) : 0.f;
                mm[q] = (ss[q] < 0) ? 0 : (all_free ? -1 : __ldg(mate + uu[q]));
            }
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (mm[q] == -1) consider(uu[q], cc[q], cid, mate, true, best, bk);
        }
        cand[v] = best;
        candkey[v] = bk;
    }
}

using ScanKernel = void (*)(const int32_t *, const int32_t *, int64_t, int, const int32_t *,
                           const float *, const int32_t *, const int32_t *, const int32_t *,
                           const int32_t *, int32_t *, uint32_t *);

ScanKernel scan_kernel(int k) {
    switch (k) {
    case 4: return k_match_scan<4>;
    case 8: return k_match_scan<8>;
    case 16: return k_match_scan<16>;
    case 32: return k_match_scan<32>;
    default: return k_match_scan<0>;
    }
}

// Match mutual pointers; count new pairs of this round; vertices that stay
// free with a candidate go to the next round's worklist.
__global__ void k_match_pair(const int32_t *__restrict__ wl, const int32_t *__restrict__ wl_count,
                             int64_t n_all, const int32_t *__restrict__ cand, int32_t *mate,
                             int32_t *round_count, int32_t *wl_next, int32_t *wl_next_count) {
    const int64_t cnt = wl ? (int64_t)*wl_count : n_all;
    const int lane = threadIdx.x & 31;
    int found = 0;
    // warp-uniform loop: one worklist atomic per warp and iteration
    for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < cnt;
         b0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t idx = b0 + threadIdx.x;
        bool push = false;
        int32_t v = -1;
        if (idx < cnt) {
            v = wl ? wl[idx] : (int32_t)idx;
            const int32_t u = mate[v] == -1 ? cand[v] : -1;
            if (u >= 0) {
                if (cand[u] == v) {
                    mate[v] = u;
                    if (v < u) found++;
                } else {
                    push = true;
                }
            }
        }
        const unsigned pm = __ballot_sync(FULL_MASK, push);
        if (pm) {
            int32_t at = 0;
            if (lane == __ffs(pm) - 1) at = atomicAdd(wl_next_count, __popc(pm));
            at = __shfl_sync(FULL_MASK, at, __ffs(pm) - 1);
            if (push) wl_next[at + __popc(pm & ((1u << lane) - 1u))] = v;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) found += __shfl_xor_sync(FULL_MASK, found, o);
    if ((threadIdx.x & 31) == 0 && found) atomicAdd(round_count, found);
}

// 64-bit selection key of each matched pair at its lower-cid endpoint:
// (cost bits << 32) | lo cid; other vertices get UINT64_MAX.
__global__ void k_pair_keys(int64_t n, const int32_t *__restrict__ mate,
                            const uint32_t *__restrict__ candkey, const int32_t *__restrict__ cid,
                            uint64_t *keys) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = mate[v];
        uint64_t k = ~0ull;
        if (u >= 0) {
            uint32_t cv = cid_of(cid, (int32_t)v), cu = cid_of(cid, u);
            if (cv < cu) k = ((uint64_t)candkey[v] << 32) | cv;
        }
        keys[v] = k;
    }
}

// partner[v] = mate[v] if the pair's key <= its scene's threshold (or no
// cap), else -1.  sid == nullptr: one scene, threshold thr[0].
__global__ void k_apply_cap(int64_t n, const int32_t *__restrict__ mate,
                            const uint32_t *__restrict__ candkey, const int32_t *__restrict__ cid,
                            const int32_t *__restrict__ sid, const uint64_t *__restrict__ thr,
                            int capped, int32_t *partner) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = mate[v];
        int32_t p = -1;
        if (u >= 0) {
            const uint64_t T = capped ? thr[sid ? sid[v] : 0] : ~0ull;
            uint32_t cv = cid_of(cid, (int32_t)v), cu = cid_of(cid, u);
            uint64_t k = ((uint64_t)candkey[v] << 32) | (cv < cu ? cv : cu);
            if (k <= T) p = u;
        }
        partner[v] = p;
    }
}

__global__ void k_lo_flags(int64_t n, const int32_t *__restrict__ partner,
                           const int32_t *__restrict__ cid, int32_t *flag) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = partner[v];
        flag[v] = (u >= 0 && cid_of(cid, (int32_t)v) < cid_of(cid, u)) ? 1 : 0;
    }
}

__global__ void k_write_pairs(int64_t n, const int32_t *__restrict__ partner,
                              const int32_t *__restrict__ flag, const int32_t *__restrict__ pos,
                              int32_t *pairs) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (flag[v]) {
            int32_t p = pos[v];
            pairs[2 * p] = (int32_t)v;
            pairs[2 * p + 1] = partner[v];
        }
    }
}

// ---------------------------------------------------------------- proposals
// offer[v] = the best offer v holds: (cost order bits << 32) | the proposer's
// canonical id.  For a fixed v this orders its edges exactly as (cost, lo,
// hi), since lo and hi differ only in the other endpoint.  pos_of_cid maps a
// canonical id back to its row.
__global__ void k_suitor_init(int64_t n, const int32_t *__restrict__ cid, unsigned long long *offer,
                              int32_t *pos_of_cid) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        offer[v] = ~0ull;
        if (cid) pos_of_cid[cid[v]] = (int32_t)v;
    }
}

// Each thread starts at one vertex u and proposes along u's best edge among
// those that would improve the other endpoint's offer (ordered by cost, then
// the other endpoint's canonical id, i.e. by (cost, lo, hi) for a fixed u).
// The proposal is an atomicMin on that endpoint's offer; if it wins, the
// previous holder (if any) has lost its partner and this thread continues
// with it; if another offer got there first, u looks again.  Offers only
// decrease, so the process ends; with a strict total order on the edges the
// mutual offers at the end are the greedy matching, whatever the order in
// which the threads run.  Offers are read through L2 (coherent with the
// atomics).  A thread that takes more than max_steps proposals sets status
// and stops; the caller then uses the round form instead.  Launched in
// 64-thread blocks at 32 registers (full occupancy): more warps hide the
// latency of the offer loads.
template <int K>
__global__ void __launch_bounds__(64, 32)
    k_suitor(int64_t n, int kk, const int32_t *__restrict__ nbr, const float *__restrict__ cost_slot,
             const int32_t *__restrict__ rev_ptr, const int32_t *__restrict__ rev,
             const int32_t *__restrict__ cid, const int32_t *__restrict__ pos_of_cid,
             unsigned long long *offer, int32_t *status, int max_steps) {
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v0 < n;
         v0 += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = (int32_t)v0;
        for (int step = 0; u >= 0; step++) {
            if (step >= max_steps) {
                atomicOr(status, 1);
                break;
            }
            const unsigned long long cu = cid_of(cid, u);
            int32_t best = -1;
            uint32_t bk = 0xffffffffu;
            // an edge to v at cost c is a candidate if u's offer would beat v's
            auto consider = [&](int32_t v, float c, unsigned long long held) {
                const uint32_t k = cost_order_bits(c);
                if ((((unsigned long long)k << 32) | cu) >= held) return;
                if (best < 0 || k < bk || (k == bk && cid_of(cid, v) < cid_of(cid, best))) {
                    best = v;
                    bk = k;
                }
            };
            const int64_t base = (int64_t)u * kk;
            if (K > 0) {
                // four slots at a time: ids and costs as 16-byte vectors, then
                // their offers; few live registers, so many warps hide the
                // latency of the offer loads
                const int4 *nb4 = (const int4 *)(nbr + base);
                const float4 *cs4 = (const float4 *)(cost_slot + base);
#pragma unroll 1
                for (int t4 = 0; t4 < K / 4; t4++) {
                    const int4 v4 = __ldg(nb4 + t4);
                    const float4 c4 = __ldg(cs4 + t4);
                    const int32_t vs[4] = {v4.x, v4.y, v4.z, v4.w};
                    const float cs[4] = {c4.x, c4.y, c4.z, c4.w};
                    unsigned long long hs[4];
#pragma unroll
                    for (int t = 0; t < 4; t++) hs[t] = __ldcg(offer + vs[t]);
#pragma unroll
                    for (int t = 0; t < 4; t++) consider(vs[t], cs[t], hs[t]);
                }
            } else {
                for (int t = 0; t < kk; t++) {
                    const int32_t v = nbr[base + t];
                    consider(v, cost_slot[base + t], __ldcg(offer + v));
                }
            }
            const int32_t r1 = rev_ptr[u + 1];
            for (int32_t r = rev_ptr[u]; r < r1; r += 4) {
                int32_t ss[4], vv[4];
                float cc[4];
                unsigned long long hh[4];
#pragma unroll
                for (int q = 0; q < 4; q++) ss[q] = r + q < r1 ? __ldg(rev + r + q) : -1;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    vv[q] = ss[q] >= 0 ? ss[q] / kk : 0;
                    cc[q] = ss[q] >= 0 ? __ldg(cost_slot + ss[q]) : 0.f;
                    hh[q] = ss[q] >= 0 ? __ldcg(offer + vv[q]) : 0ull;
                }
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (ss[q] >= 0) consider(vv[q], cc[q], hh[q]);
            }
            if (best < 0) break;  // no edge left that u could win: u stays single
            const unsigned long long mine = ((unsigned long long)bk << 32) | cu;
            const unsigned long long prev = atomicMin(offer + best, mine);
            if (prev > mine) {
                // u holds best's offer now; the previous holder proposes again
                u = prev == ~0ull ? -1
                                  : (cid ? pos_of_cid[(uint32_t)prev] : (int32_t)(uint32_t)prev);
            }
            // else a better offer arrived first: u looks again
        }
    }
}

// Mutual offers are the pairs: mate[], the pair's cost bits in candkey[]
// (as the round form leaves them), and the number of pairs.
__global__ void k_suitor_mates(int64_t n, const unsigned long long *__restrict__ offer,
                               const int32_t *__restrict__ cid, const int32_t *__restrict__ pos_of_cid,
                               int32_t *mate, uint32_t *candkey, int32_t *pairs) {
    int found = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long w = offer[v];
        int32_t m = -1;
        if (w != ~0ull) {
            const int32_t u = cid ? pos_of_cid[(uint32_t)w] : (int32_t)(uint32_t)w;
            const uint32_t cv = cid_of(cid, (int32_t)v);
            if ((uint32_t)offer[u] == cv) {
                m = u;
                if (cv < (uint32_t)w) found++;
            }
        }
        mate[v] = m;
        candkey[v] = m >= 0 ? (uint32_t)(w >> 32) : 0xffffffffu;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) found += __shfl_xor_sync(FULL_MASK, found, o);
    if ((threadIdx.x & 31) == 0 && found) atomicAdd(pairs, found);
}

using SuitorKernel = void (*)(int64_t, int, const int32_t *, const float *, const int32_t *,
                              const int32_t *, const int32_t *, const int32_t *,
                              unsigned long long *, int32_t *, int);

SuitorKernel suitor_kernel(int k) {
    switch (k) {
    case 4: return k_suitor<4>;
    case 8: return k_suitor<8>;
    case 16: return k_suitor<16>;
    case 32: return k_suitor<32>;
    default: return k_suitor<0>;
    }
}

// Device-side control of the captured rounds.  State (int32): [0] worklist A
// size, [1] worklist B size, [2] pairs of round A, [3] pairs of round B,
// [4] rounds done, [5] pairs in all, [6] round limit reached, [7] pairs of
// round 0.
constexpr int MS_CNT_A = 0, MS_CNT_B = 1, MS_M_A = 2, MS_M_B = 3, MS_ROUNDS = 4, MS_TOTAL = 5,
              MS_LIMIT = 6, MS_M0 = 7;

// the loop state into pinned host memory (see get_small)
__global__ void k_get_state(int32_t *hstate, const int32_t *st) {
    if (threadIdx.x < 8) hstate[threadIdx.x] = st[threadIdx.x];
}

__global__ void k_match_ctl0(cudaGraphConditionalHandle h, int32_t *st) {
    st[MS_ROUNDS] = 1;
    st[MS_TOTAL] = st[MS_M0];
    st[MS_LIMIT] = 0;
    cudaGraphSetConditional(h, st[MS_M0] > 0 ? 1u : 0u);
}

// after a body of two rounds: the first round that matched nothing ends the loop
__global__ void k_match_ctl(cudaGraphConditionalHandle h, int32_t *st, int max_rounds) {
    const int32_t ma = st[MS_M_A], mb = st[MS_M_B];
    st[MS_TOTAL] += ma + mb;
    unsigned more = 0;
    if (ma == 0) {
        st[MS_ROUNDS] += 1;
    } else if (mb == 0) {
        st[MS_ROUNDS] += 2;
    } else {
        st[MS_ROUNDS] += 2;
        more = st[MS_ROUNDS] < max_rounds ? 1u : 0u;
        if (!more) st[MS_LIMIT] = 1;
    }
    cudaGraphSetConditional(h, more);
}

}  // namespace

// The rounds after the first as one CUDA graph: a WHILE conditional node
// whose body runs two rounds (worklist A -> B -> A) and a control kernel that
// ends the loop on the first round without a new pair.  No host round trip
// until the loop ends.  Returns false (nothing launched) when the graph
// cannot be built, in which case the caller runs the rounds from the host.
static bool match_rounds_graph(ngs_ctx *c, const GraphDev &g, int32_t *mate, int32_t *cand,
                               uint32_t *candkey, int32_t *const wl[2], int32_t *stt,
                               unsigned grid, int max_rounds, int32_t *hstate) {
    const int64_t n = g.n;
    if (!c->cap_st && cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->cap_st = nullptr;
        return false;
    }
    cudaStream_t cs = c->cap_st;  // capture only records; the graph runs on c->st
    const ScanKernel scan = scan_kernel(g.k_eff);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = false;
    do {
        if (cudaGraphCreate(&graph, 0) != cudaSuccess) break;
        cudaGraphConditionalHandle h;
        if (cudaGraphConditionalHandleCreate(&h, graph, 0, 0) != cudaSuccess) break;
        if (cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            break;
        k_match_ctl0<<<1, 1, 0, cs>>>(h, stt);
        if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) break;
        size_t nn = 0;
        if (cudaGraphGetNodes(graph, nullptr, &nn) != cudaSuccess || nn != 1) break;
        cudaGraphNode_t ctl0;
        if (cudaGraphGetNodes(graph, &ctl0, &nn) != cudaSuccess) break;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        if (cudaGraphAddNode(&cnode, graph, &ctl0, nullptr, 1, &cp) != cudaSuccess) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            break;
        cudaMemsetAsync(stt + MS_CNT_B, 0, 3 * sizeof(int32_t), cs);  // B size, both round counts
        scan<<<grid, 256, 0, cs>>>(wl[0], stt + MS_CNT_A, n, g.k_eff, g.nbr,
                                             (const float *)g.cost_slot, (const int32_t *)g.rev_ptr,
                                             (const int32_t *)g.rev, g.cid, (const int32_t *)mate,
                                             cand, candkey);
        k_match_pair<<<grid, 256, 0, cs>>>(wl[0], stt + MS_CNT_A, n, (const int32_t *)cand, mate,
                                             stt + MS_M_A, wl[1], stt + MS_CNT_B);
        cudaMemsetAsync(stt + MS_CNT_A, 0, sizeof(int32_t), cs);
        scan<<<grid, 256, 0, cs>>>(wl[1], stt + MS_CNT_B, n, g.k_eff, g.nbr,
                                             (const float *)g.cost_slot, (const int32_t *)g.rev_ptr,
                                             (const int32_t *)g.rev, g.cid, (const int32_t *)mate,
                                             cand, candkey);
        k_match_pair<<<grid, 256, 0, cs>>>(wl[1], stt + MS_CNT_B, n, (const int32_t *)cand, mate,
                                             stt + MS_M_B, wl[0], stt + MS_CNT_A);
        k_match_ctl<<<1, 1, 0, cs>>>(h, stt, max_rounds);
        if (cudaStreamEndCapture(cs, &body) != cudaSuccess) break;
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) break;
        ok = true;
    } while (false);
    if (!ok) {
        cudaStreamCaptureStatus cst;
        if (cudaStreamIsCapturing(cs, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
            cudaGraph_t dummy = nullptr;
            cudaStreamEndCapture(cs, &dummy);
            if (dummy) cudaGraphDestroy(dummy);
        }
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        return false;
    }
    int slot = -1;
    cudaEvent_t a = nullptr;
    if (c->prof) {
        slot = prof_slot(c, "match_graph");
        prof_begin(c, slot, &a);
    }
    const cudaError_t le = cudaGraphLaunch(exec, c->st);
    if (c->prof) prof_end(c, slot, a);
    cudaError_t se = cudaSuccess;
    if (le == cudaSuccess) {
        k_get_state<<<1, 32, 0, c->st>>>(hstate, stt);
        se = cudaGetLastError();
        if (se == cudaSuccess) {
            c->syncs++;
            se = cudaStreamSynchronize(c->st);
        }
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (le != cudaSuccess) NGS_FAIL(NGS_ERR_CUDA, "match graph launch: %s", cudaGetErrorString(le));
    if (se != cudaSuccess) NGS_FAIL(NGS_ERR_CUDA, "match graph: %s", cudaGetErrorString(se));
    return true;
}

// The proposal form: returns false (and no result) if a thread exceeded its
// step limit.  pos_of_cid: n ints of scratch.
static bool match_suitor(ngs_ctx *c, const GraphDev &g, int32_t *mate, int32_t *pos_of_cid,
                         uint32_t *candkey, int64_t *matched) {
    const int64_t n = g.n;
    unsigned long long *offer = ws<unsigned long long>(c, c->b_offer, n);
    int32_t *stt = ws<int32_t>(c, c->b_mstate, 16);
    NGS_CHECK_CUDA(cudaMemsetAsync(stt, 0, 2 * sizeof(int32_t), c->st));
    const unsigned grid = grid_stride_blocks(c, n, 256, 8);
    launch(c, "suitor_init", dim3(grid), dim3(256), 0, k_suitor_init, n, g.cid, offer, pos_of_cid);
    // one thread per starting vertex, in small blocks: the proposal chains
    // differ in length (about 1.7 proposals and 0.35 lost bids per vertex,
    // chains of at most 8 on the 6M-splat scene)
    launch(c, "suitor", dim3(blocks_for(n, 64)), dim3(64), 0, suitor_kernel(g.k_eff), n, g.k_eff, g.nbr,
           (const float *)g.cost_slot, (const int32_t *)g.rev_ptr, (const int32_t *)g.rev, g.cid,
           (const int32_t *)pos_of_cid, offer, stt, c->tune.match_max_steps);
    launch(c, "suitor_mates", dim3(grid), dim3(256), 0, k_suitor_mates, n,
           (const unsigned long long *)offer, g.cid, (const int32_t *)pos_of_cid, mate, candkey,
           stt + 1);
    int32_t *hs = (int32_t *)(c->h_pin + 32);
    get_small(c, hs, stt, 2 * sizeof(int32_t));
    sync_stream(c);
    if (hs[0]) return false;
    *matched = hs[1];
    return true;
}

int64_t match_rounds(ngs_ctx *c, const GraphDev &g) {
    const int64_t n = g.n;
    c->rounds = 0;
    if (n <= 0) return 0;
    int32_t *mate = ws<int32_t>(c, c->b_mate, n);
    int32_t *cand = ws<int32_t>(c, c->b_cand, n);
    uint32_t *candkey = ws<uint32_t>(c, c->b_candkey, n);
    if (g.n_edges > 0 && c->tune.match_method == 2) {
        // cand serves as the proposal form's id map
        int64_t matched = 0;
        if (match_suitor(c, g, mate, cand, candkey, &matched)) {
            c->rounds = 1;
            return matched;
        }
        // a thread hit its step limit: the round form from the start
    }
    const int max_rounds = 4096;
    int32_t *counts = ws<int32_t>(c, c->b_counts, 2 * max_rounds);
    int32_t *wl_counts = counts + max_rounds;  // worklist size feeding round r+1
    NGS_CHECK_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * 2 * max_rounds, c->st));
    int32_t *wl[2] = {ws<int32_t>(c, c->b_sel2, n), ws<int32_t>(c, c->b_cflag2, n)};
    const unsigned grid = grid_stride_blocks(c, n, 256, 8);
    launch(c, "match_init", dim3(grid), dim3(256), 0, k_match_init, n, mate, cand);
    int64_t matched = 0;
    int r = 0;
    if (g.n_edges > 0 && c->tune.match_method >= 1) {  // rounds in a CUDA graph
        int32_t *stt = ws<int32_t>(c, c->b_mstate, 16);
        NGS_CHECK_CUDA(cudaMemsetAsync(stt, 0, 16 * sizeof(int32_t), c->st));
        // round 0 over every vertex, then the captured loop
        launch(c, "match_scan", dim3(grid), dim3(256), 0, scan_kernel(g.k_eff), (const int32_t *)nullptr,
               (const int32_t *)nullptr, n, g.k_eff, g.nbr, (const float *)g.cost_slot,
               (const int32_t *)g.rev_ptr, (const int32_t *)g.rev, g.cid, (const int32_t *)mate,
               cand, candkey);
        launch(c, "match_pair", dim3(grid), dim3(256), 0, k_match_pair, (const int32_t *)nullptr,
               (const int32_t *)nullptr, n, (const int32_t *)cand, mate, stt + MS_M0, wl[0],
               stt + MS_CNT_A);
        int32_t *hs = (int32_t *)(c->h_pin + 32);
        // the later rounds' worklists are smaller: one wave of 4 blocks per SM
        const unsigned grid_later = std::min<unsigned>(grid, (unsigned)c->num_sms * 4);
        if (match_rounds_graph(c, g, mate, cand, candkey, wl, stt, grid_later, max_rounds, hs)) {
            if (hs[MS_LIMIT]) NGS_FAIL(NGS_ERR_TIMEOUT, "matching did not converge in %d rounds", max_rounds);
            c->rounds = hs[MS_ROUNDS];
            c->launches += 1 + 5 * (int64_t)((hs[MS_ROUNDS]) / 2);  // control + body kernels
            return hs[MS_TOTAL];
        }
        // no graph: continue from round 1 on the host (round 0 is done)
        NGS_CHECK_CUDA(cudaMemcpyAsync(counts, stt + MS_M0, sizeof(int32_t), cudaMemcpyDeviceToDevice, c->st));
        NGS_CHECK_CUDA(cudaMemcpyAsync(wl_counts, stt + MS_CNT_A, sizeof(int32_t), cudaMemcpyDeviceToDevice, c->st));
        int32_t *h0 = (int32_t *)(c->h_pin + 32);
        get_small(c, h0, counts, sizeof(int32_t));
        sync_stream(c);
        matched = h0[0];
        r = 1;
        if (h0[0] == 0) {
            c->rounds = 1;
            return 0;
        }
    }
    if (g.n_edges > 0) {
        // rounds are launched in batches; a batch is checked once on the host.
        // Round 0 visits every vertex, later rounds only the worklist.
        int batch = 4;
        bool done = false;
        while (!done) {
            if (r + batch > max_rounds)
                NGS_FAIL(NGS_ERR_TIMEOUT, "matching did not converge in %d rounds", max_rounds);
            for (int b = 0; b < batch; b++, r++) {
                const int32_t *in_wl = r == 0 ? nullptr : wl[(r - 1) & 1];
                const int32_t *in_cnt = r == 0 ? nullptr : wl_counts + (r - 1);
                launch(c, "match_scan", dim3(grid), dim3(256), 0, scan_kernel(g.k_eff), in_wl, in_cnt, n,
                       g.k_eff, g.nbr, (const float *)g.cost_slot, (const int32_t *)g.rev_ptr,
                       (const int32_t *)g.rev, g.cid, (const int32_t *)mate, cand, candkey);
                launch(c, "match_pair", dim3(grid), dim3(256), 0, k_match_pair, in_wl, in_cnt, n,
                       (const int32_t *)cand, mate, counts + r, wl[r & 1], wl_counts + r);
            }
            int32_t *hc = (int32_t *)(c->h_pin + 32);
            get_small(c, hc, counts + r - batch, sizeof(int32_t) * batch);
            sync_stream(c);
            for (int b = 0; b < batch; b++) {
                matched += hc[b];
                if (hc[b] == 0) {
                    done = true;
                    c->rounds = r - batch + b + 1;
                    break;
                }
            }
            batch = batch < 16 ? batch * 2 : 16;
        }
    }
    return matched;
}

void pair_keys(ngs_ctx *c, const GraphDev &g, uint64_t *keys) {
    const int64_t n = g.n;
    launch(c, "pair_keys", dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0, k_pair_keys, n,
           (const int32_t *)c->b_mate.p, (const uint32_t *)c->b_candkey.p, g.cid, keys);
}

void apply_cap(ngs_ctx *c, const GraphDev &g, const int32_t *sid, const uint64_t *thr,
               int capped, int32_t *partner) {
    const int64_t n = g.n;
    launch(c, "apply_cap", dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0, k_apply_cap, n,
           (const int32_t *)c->b_mate.p, (const uint32_t *)c->b_candkey.p, g.cid, sid, thr, capped,
           partner);
}

int64_t select_pairs(ngs_ctx *c, const GraphDev &g, int64_t max_pairs, int32_t *partner) {
    const int64_t n = g.n;
    if (n <= 0) return 0;
    int64_t matched = 0;
    c->rounds = 0;
    if (max_pairs > 0) {
        matched = match_rounds(c, g);
    } else {
        ws<int32_t>(c, c->b_mate, n);
        ws<uint32_t>(c, c->b_candkey, n);
        launch(c, "match_init", dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0, k_match_init, n,
               (int32_t *)c->b_mate.p, ws<int32_t>(c, c->b_cand, n));
    }
    const bool capped = matched > max_pairs;
    uint64_t *thr = (uint64_t *)ws<uint8_t>(c, c->b_sel, 64);
    if (capped) {
        uint64_t *keys = (uint64_t *)ws<uint8_t>(c, c->b_flag, sizeof(uint64_t) * n);
        pair_keys(c, g, keys);
        radix_select_u64(c, keys, n, max_pairs - 1, thr);
    }
    apply_cap(c, g, nullptr, thr, capped ? 1 : 0, partner);
    return capped ? max_pairs : matched;
}

int64_t partner_to_pairs(ngs_ctx *c, const int32_t *partner, const int32_t *cid, int64_t n,
                         int32_t *pairs_out) {
    if (n <= 0) return 0;
    int32_t *flag = ws<int32_t>(c, c->b_keep, n + 1);
    int32_t *pos = ws<int32_t>(c, c->b_pos, n + 1);
    const unsigned grid = grid_stride_blocks(c, n, 256, 8);
    launch(c, "lo_flags", dim3(grid), dim3(256), 0, k_lo_flags, n, partner, cid, flag);
    scan_i32(c, flag, pos, n);
    get_small(c, c->h_pin, pos + n, sizeof(int32_t));
    launch(c, "write_pairs", dim3(grid), dim3(256), 0, k_write_pairs, n, partner,
           (const int32_t *)flag, (const int32_t *)pos, pairs_out);
    sync_stream(c);
    return *(int32_t *)c->h_pin;
}
