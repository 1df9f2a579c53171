// Undirected merge graph from the directed kNN lists (Algorithm 1
// UndirectedUnionEdges): the symmetric adjacency (each vertex lists every
// neighbour it shares an undirected edge with, sorted by canonical id) and
// the unique edge list {lo, hi} with cid[lo] < cid[hi].  Edges are numbered
// row by row (rows in internal order, each row's upper neighbours by
// canonical id), which is lexicographic order when rows are canonical.
#include "ngs_device.cuh"
#include "ngs_internal.h"

namespace {

constexpr int ROW_SORT_MAX = 128;  // rows up to this length are sorted in registers

__device__ __forceinline__ uint32_t cid_of(const int32_t *cid, int32_t v) {
    return cid ? (uint32_t)cid[v] : (uint32_t)v;
}

__global__ void k_indeg(const int32_t *__restrict__ nbr, int64_t m, int32_t *indeg) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&indeg[nbr[t]], 1);
}

__global__ void k_capacity(const int32_t *__restrict__ indeg, int64_t n, int ke, int32_t *cap,
                           int32_t *fill) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        cap[v] = ke + indeg[v];
        fill[v] = 0;
    }
}

__global__ void k_fill(const int32_t *__restrict__ nbr, int64_t n, int ke,
                       const int32_t *__restrict__ rstart, int32_t *fill, int32_t *adj) {
    int64_t m = n * ke;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = t / ke;
        int a = (int)(t - v * ke);
        int32_t u = nbr[t];
        adj[rstart[v] + a] = u;                       // out-edge of v
        int s = atomicAdd(&fill[u], 1);
        adj[rstart[u] + ke + s] = (int32_t)v;         // in-edge of u
    }
}

// One warp per row: bitonic sort of up to 128 (cid, index) keys held four per
// lane (element i = r*32 + lane), then drop duplicates and write the unique
// neighbours back to the row start.  deg[v] = unique count, upc[v] = number
// with a larger canonical id than v.  Longer rows are left for k_row_long.
__global__ void k_row_sort(const int32_t *__restrict__ rstart, int64_t n,
                           const int32_t *__restrict__ cid, int32_t *adj, int32_t *deg,
                           int32_t *upc) {
    int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (v >= n) return;
    int32_t rs = rstart[v];
    int L = rstart[v + 1] - rs;
    if (L > ROW_SORT_MAX) {
        if (lane == 0) deg[v] = -1;
        return;
    }
    uint64_t x[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        int i = r * 32 + lane;
        if (i < L) {
            int32_t u = adj[rs + i];
            x[r] = ((uint64_t)cid_of(cid, u) << 32) | (uint32_t)u;
        } else {
            x[r] = ~0ull;
        }
    }
#pragma unroll
    for (int k = 2; k <= 128; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int rj = j >> 5;
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int p = r ^ rj;
                    if (p > r) {
                        int i = r * 32 + lane;
                        bool asc = (i & k) == 0;
                        uint64_t a = x[r], b = x[p];
                        bool sw = asc ? (a > b) : (a < b);
                        x[r] = sw ? b : a;
                        x[p] = sw ? a : b;
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    int i = r * 32 + lane;
                    uint64_t o = __shfl_xor_sync(FULL_MASK, x[r], j);
                    bool asc = (i & k) == 0;
                    bool lower = (lane & j) == 0;
                    uint64_t mn = x[r] < o ? x[r] : o, mx = x[r] < o ? o : x[r];
                    x[r] = (lower == asc) ? mn : mx;
                }
            }
        }
    }
    uint32_t cv = cid_of(cid, (int32_t)v);
    const unsigned lt = (1u << lane) - 1u;
    int base = 0, up = 0;
    uint64_t last_prev = 0;
#pragma unroll
    for (int r = 0; r < 4; r++) {
        int i = r * 32 + lane;
        uint64_t prev = __shfl_up_sync(FULL_MASK, x[r], 1);
        if (lane == 0) prev = last_prev;
        bool uniq = i < L && (i == 0 || x[r] != prev);
        unsigned m = __ballot_sync(FULL_MASK, uniq);
        if (uniq) adj[rs + base + __popc(m & lt)] = (int32_t)(uint32_t)(x[r] & 0xffffffffu);
        up += __popc(__ballot_sync(FULL_MASK, uniq && (uint32_t)(x[r] >> 32) > cv));
        base += __popc(m);
        last_prev = __shfl_sync(FULL_MASK, x[r], 31);
    }
    if (lane == 0) {
        deg[v] = base;
        upc[v] = up;
    }
}

// Rows longer than ROW_SORT_MAX (rare): insertion sort by one thread.
__global__ void k_row_long(const int32_t *__restrict__ rstart, int64_t n,
                           const int32_t *__restrict__ cid, int32_t *adj, int32_t *deg,
                           int32_t *upc) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (deg[v] != -1) continue;
        int32_t rs = rstart[v];
        int L = rstart[v + 1] - rs;
        int32_t *a = adj + rs;
        for (int i = 1; i < L; i++) {
            int32_t u = a[i];
            uint32_t cu = cid_of(cid, u);
            int j = i - 1;
            while (j >= 0 && cid_of(cid, a[j]) > cu) {
                a[j + 1] = a[j];
                j--;
            }
            a[j + 1] = u;
        }
        uint32_t cv = cid_of(cid, (int32_t)v);
        int cnt = 0, up = 0;
        for (int i = 0; i < L; i++) {
            if (i > 0 && a[i] == a[cnt - 1]) continue;
            a[cnt++] = a[i];
            if (cid_of(cid, a[i]) > cv) up++;
        }
        deg[v] = cnt;
        upc[v] = up;
    }
}

// Edge list and the edge id of every adjacency entry.
__global__ void k_edges(const int32_t *__restrict__ rstart, const int32_t *__restrict__ deg,
                        const int32_t *__restrict__ upc, const int32_t *__restrict__ eptr,
                        int64_t n, const int32_t *__restrict__ cid, const int32_t *__restrict__ adj,
                        int32_t *adj_eid, int32_t *elo, int32_t *ehi) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t rs = rstart[v];
        int d = deg[v], nlow = d - upc[v];
        uint32_t cv = cid_of(cid, (int32_t)v);
        int32_t e0 = eptr[v];
        for (int t = 0; t < d; t++) {
            int32_t u = adj[rs + t];
            if (t >= nlow) {
                int32_t e = e0 + (t - nlow);
                elo[e] = (int32_t)v;
                ehi[e] = u;
                adj_eid[rs + t] = e;
            } else {
                // edge (u, v) is an upper entry of row u: binary search for cv
                int32_t urs = rstart[u];
                int ud = deg[u], ulow = ud - upc[u];
                int lo = ulow, hi = ud - 1;
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (cid_of(cid, adj[urs + mid]) < cv) lo = mid + 1;
                    else hi = mid;
                }
                adj_eid[rs + t] = eptr[u] + (lo - ulow);
            }
        }
    }
}

}  // namespace

void build_edges(ngs_ctx *c, const int32_t *nbr, GraphDev &g) {
    const int64_t n = g.n;
    const int ke = g.k_eff;
    g.n_edges = 0;
    if (n <= 1 || ke <= 0) return;
    int32_t *indeg = ws<int32_t>(c->b_deg, n + 1);
    int32_t *fill = ws<int32_t>(c->b_fill, n + 1);
    g.rstart = ws<int32_t>(c->b_rstart, n + 1);
    NGS_CHECK_CUDA(cudaMemsetAsync(indeg, 0, sizeof(int32_t) * n, c->st));
    launch(c, "graph_indeg", dim3(grid_stride_blocks(c, n * ke, 256, 8)), dim3(256), 0, k_indeg,
           nbr, n * ke, indeg);
    launch(c, "graph_capacity", dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0, k_capacity,
           (const int32_t *)indeg, n, ke, g.rstart, fill);
    scan_i32(c, g.rstart, g.rstart, n);
    const int64_t cap_total = 2 * n * (int64_t)ke;  // sum of capacities
    g.adj = ws<int32_t>(c->b_adj, cap_total);
    g.adj_eid = ws<int32_t>(c->b_adjeid, cap_total);
    launch(c, "graph_fill", dim3(grid_stride_blocks(c, n * ke, 256, 8)), dim3(256), 0, k_fill, nbr,
           n, ke, (const int32_t *)g.rstart, fill, g.adj);
    g.deg = indeg;  // reuse: indeg is no longer needed
    int32_t *upc = ws<int32_t>(c->b_upc, n + 1);
    launch(c, "graph_row_sort", dim3(blocks_for(n * 32, 256)), dim3(256), 0, k_row_sort,
           (const int32_t *)g.rstart, n, g.cid, g.adj, g.deg, upc);
    launch(c, "graph_row_long", dim3(grid_stride_blocks(c, n, 256, 2)), dim3(256), 0, k_row_long,
           (const int32_t *)g.rstart, n, g.cid, g.adj, g.deg, upc);
    g.eptr = ws<int32_t>(c->b_eptr, n + 1);
    scan_i32(c, upc, g.eptr, n);
    NGS_CHECK_CUDA(cudaMemcpyAsync(c->h_pin, g.eptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                   c->st));
    sync_stream(c);
    g.n_edges = *(int32_t *)c->h_pin;
    g.elo = ws<int32_t>(c->b_elo, g.n_edges);
    g.ehi = ws<int32_t>(c->b_ehi, g.n_edges);
    launch(c, "graph_edges", dim3(grid_stride_blocks(c, n, 128, 16)), dim3(128), 0, k_edges,
           (const int32_t *)g.rstart, (const int32_t *)g.deg, (const int32_t *)upc,
           (const int32_t *)g.eptr, n, g.cid, (const int32_t *)g.adj, g.adj_eid, g.elo, g.ehi);
}
