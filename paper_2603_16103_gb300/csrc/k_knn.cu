// k-nearest-neighbour search over splat centres (Sec. 3.1, Algorithm 1 KNN).
//
// Points are ordered along a 30-bit Morton curve and cut into leaves of 32
// (one warp).  An implicit complete binary tree of axis-aligned boxes sits on
// top of the leaves.  One warp answers the 32 queries of one leaf: it scans
// its own leaf first, then walks the tree depth first, visiting a node only
// if some lane's box distance is within that lane's current k-th distance.
// Each lane keeps a register-resident sorted list of (d^2, canonical id)
// keys, so the result is exactly the k_eff nearest with ties by canonical id.
// Box distances and point distances use the same FP32 expression without
// contraction, so pruning never drops a point the list would accept.
#include "ngs_device.cuh"
#include "ngs_internal.h"

namespace {

__device__ __forceinline__ float dist2_rn(float dx, float dy, float dz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ float box_dist2(const float4 &q, const float4 &lo, const float4 &hi) {
    float dx = fmaxf(fmaxf(__fsub_rn(lo.x, q.x), __fsub_rn(q.x, hi.x)), 0.0f);
    float dy = fmaxf(fmaxf(__fsub_rn(lo.y, q.y), __fsub_rn(q.y, hi.y)), 0.0f);
    float dz = fmaxf(fmaxf(__fsub_rn(lo.z, q.z), __fsub_rn(q.z, hi.z)), 0.0f);
    return dist2_rn(dx, dy, dz);
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// frame_acc: [0..2] min order bits, [3..5] max order bits, [6] non-finite count
__global__ void k_frame_init(uint32_t *acc) {
    int t = threadIdx.x;
    if (t < 3) acc[t] = 0xffffffffu;
    else if (t < 6) acc[t] = 0u;
    else if (t == 6) acc[t] = 0u;
}

__global__ void k_frame_reduce(const float *__restrict__ xyz, int64_t n, uint32_t *acc) {
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            float v = xyz[3 * i + a];
            if (!isfinite(v)) {
                bad++;
                continue;
            }
            mn[a] = fminf(mn[a], v);
            mx[a] = fmaxf(mx[a], v);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        mn[a] = warp_min(mn[a]);
        mx[a] = warp_max(mx[a]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(FULL_MASK, bad, o);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (mn[a] <= mx[a]) {
                atomicMin(&acc[a], float_order_bits(mn[a]));
                atomicMax(&acc[3 + a], float_order_bits(mx[a]));
            }
        }
        if (bad) atomicAdd(&acc[6], (uint32_t)bad);
    }
}

// frame: lo.x lo.y lo.z scale (cells per unit); frame[4] = non-finite count
__global__ void k_frame_final(const uint32_t *acc, float *frame) {
    float lo[3], side = 0.0f;
    for (int a = 0; a < 3; a++) {
        if (acc[a] == 0xffffffffu) {  // no finite point
            lo[a] = 0.0f;
            continue;
        }
        lo[a] = order_bits_float(acc[a]);
        float hi = order_bits_float(acc[3 + a]);
        side = fmaxf(side, hi - lo[a]);
    }
    if (!(side > 0.0f)) side = 1.0f;
    frame[0] = lo[0];
    frame[1] = lo[1];
    frame[2] = lo[2];
    frame[3] = 1024.0f / (side * 1.0001f);
    frame[4] = __uint_as_float(acc[6]);
}

__global__ void k_morton(const float *__restrict__ xyz, int64_t n, const float *__restrict__ frame,
                         uint32_t *keys, uint32_t *vals) {
    float lx = frame[0], ly = frame[1], lz = frame[2], sc = frame[3];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float q[3] = {(xyz[3 * i] - lx) * sc, (xyz[3 * i + 1] - ly) * sc, (xyz[3 * i + 2] - lz) * sc};
        uint32_t c[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            float v = q[a];
            c[a] = (v >= 1023.0f) ? 1023u : (v > 0.0f ? (uint32_t)v : 0u);  // NaN -> 0
        }
        keys[i] = spread10(c[0]) | (spread10(c[1]) << 1) | (spread10(c[2]) << 2);
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_gather_pts(const float *__restrict__ xyz, const int32_t *__restrict__ cid,
                             const uint32_t *__restrict__ order, int64_t n, float4 *pts) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = order ? (int64_t)order[p] : p;
        uint32_t id = cid ? (uint32_t)cid[i] : (uint32_t)i;
        pts[p] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], __uint_as_float(id));
    }
}

// ---------------------------------------------------------------- tree
__global__ void k_tree_leaves(const float4 *__restrict__ pts, int64_t n, int64_t nb, int64_t P,
                              float4 *nodes) {
    int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (b >= P) return;
    float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
    float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
    if (b < nb) {
        int64_t p = b * NGS_LEAF + lane;
        float x = INFINITY, y = INFINITY, z = INFINITY, X = -INFINITY, Y = -INFINITY, Z = -INFINITY;
        if (p < n) {
            float4 v = pts[p];
            x = X = v.x;
            y = Y = v.y;
            z = Z = v.z;
        }
        lo = make_float4(warp_min(x), warp_min(y), warp_min(z), 0.f);
        hi = make_float4(warp_max(X), warp_max(Y), warp_max(Z), 0.f);
    }
    if (lane == 0) {
        nodes[2 * (P + b)] = lo;
        nodes[2 * (P + b) + 1] = hi;
    }
}

__global__ void k_tree_level(float4 *nodes, int64_t first, int64_t count) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    int64_t i = first + t;
    float4 a0 = nodes[4 * i], a1 = nodes[4 * i + 1], b0 = nodes[4 * i + 2], b1 = nodes[4 * i + 3];
    nodes[2 * i] = make_float4(fminf(a0.x, b0.x), fminf(a0.y, b0.y), fminf(a0.z, b0.z), 0.f);
    nodes[2 * i + 1] = make_float4(fmaxf(a1.x, b1.x), fmaxf(a1.y, b1.y), fmaxf(a1.z, b1.z), 0.f);
}

// ---------------------------------------------------------------- query
constexpr int KNN_WARPS = 4;
constexpr int KNN_STACK = 64;

// Register-resident k-best list of 64-bit keys (d^2 bits << 32 | canonical
// id) kept in DESCENDING order: slot 0 holds the current k-th key, slots
// [keff, KMAX) hold 0 (below every key) so every register index is static.
template <int KMAX>
struct TopK {
    uint64_t key[KMAX];

    __device__ __forceinline__ void init(int keff) {
#pragma unroll
        for (int i = 0; i < KMAX; i++) key[i] = i < keff ? ~0ull : 0ull;
    }
    __device__ __forceinline__ uint64_t kth() const { return key[0]; }
    // insert x < key[0]: drop key[0], keep the list sorted descending
    __device__ __forceinline__ void insert(uint64_t x) {
#pragma unroll
        for (int i = 0; i < KMAX; i++) {
            uint64_t nxt = i + 1 < KMAX ? key[i + 1] : 0ull;
            key[i] = nxt > x ? nxt : (x < key[i] ? x : key[i]);
        }
    }
    __device__ __forceinline__ float kth_d2() const {
        return key[0] == ~0ull ? INFINITY : __uint_as_float((uint32_t)(key[0] >> 32));
    }
};

// Candidates that pass a lane's threshold are queued per lane in shared
// memory and inserted in warp-wide rounds afterwards, so the warp pays for
// max-over-lanes insertions instead of one insertion per candidate any lane
// accepts.
template <int KMAX>
__device__ __forceinline__ void scan_leaf(const float4 *__restrict__ pts, int64_t n, int64_t leaf,
                                          const float4 &q, int64_t qp, bool qvalid, int lane,
                                          uint64_t (*queue)[32], TopK<KMAX> &tk) {
    int64_t cp = leaf * NGS_LEAF + lane;
    bool cvalid = cp < n;
    float4 c = cvalid ? pts[cp] : make_float4(0.f, 0.f, 0.f, 0.f);
    int cnt = __popc(__ballot_sync(FULL_MASK, cvalid));  // valid candidates are a prefix
    const uint64_t thr = tk.kth();
    int qlen = 0;
    for (int j = 0; j < cnt; j++) {
        float cx = __shfl_sync(FULL_MASK, c.x, j);
        float cy = __shfl_sync(FULL_MASK, c.y, j);
        float cz = __shfl_sync(FULL_MASK, c.z, j);
        uint32_t cw = __float_as_uint(__shfl_sync(FULL_MASK, c.w, j));
        float d2 = dist2_rn(__fsub_rn(q.x, cx), __fsub_rn(q.y, cy), __fsub_rn(q.z, cz));
        uint64_t kk = ((uint64_t)__float_as_uint(d2) << 32) | cw;
        if (qvalid && leaf * NGS_LEAF + j != qp && kk < thr) queue[qlen++][lane] = kk;
    }
    int rounds = __reduce_max_sync(FULL_MASK, qlen);
    for (int r = 0; r < rounds; r++) {
        if (r < qlen) {
            uint64_t x = queue[r][lane];
            if (x < tk.kth()) tk.insert(x);
        }
    }
    __syncwarp();
}

template <int KMAX>
__global__ void __launch_bounds__(KNN_WARPS * 32)
    k_knn(const float4 *__restrict__ pts, int64_t n, int64_t nb, int64_t P,
          const float4 *__restrict__ nodes, int keff, int out_by_cid, int32_t *__restrict__ nbr) {
    __shared__ int stack_all[KNN_WARPS][KNN_STACK];
    __shared__ uint64_t queue_all[KNN_WARPS][NGS_LEAF][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * KNN_WARPS + warp;
    if (b >= nb) return;  // uniform per warp
    int *stack = stack_all[warp];
    uint64_t(*queue)[32] = queue_all[warp];
    const int64_t qp = b * NGS_LEAF + lane;
    const bool qvalid = qp < n;
    const float4 q = qvalid ? pts[qp] : make_float4(0.f, 0.f, 0.f, 0.f);
    TopK<KMAX> tk;
    tk.init(keff);
    scan_leaf<KMAX>(pts, n, b, q, qp, qvalid, lane, queue, tk);
    const int64_t own = P + b;
    int sp = 0;
    if (lane == 0) stack[0] = 1;
    sp = 1;
    __syncwarp();
    while (sp > 0) {
        int64_t node = stack[--sp];
        __syncwarp();
        if (node == own) continue;
        float4 lo = nodes[2 * node], hi = nodes[2 * node + 1];
        bool nonempty = lo.x <= hi.x;
        float md = box_dist2(q, lo, hi);
        bool need = qvalid && nonempty && md <= tk.kth_d2();
        if (!__any_sync(FULL_MASK, need)) continue;
        if (node >= P) {
            scan_leaf<KMAX>(pts, n, node - P, q, qp, qvalid, lane, queue, tk);
        } else {
            int64_t c0 = 2 * node, c1 = 2 * node + 1;
            float d0 = box_dist2(q, nodes[2 * c0], nodes[2 * c0 + 1]);
            float d1 = box_dist2(q, nodes[2 * c1], nodes[2 * c1 + 1]);
            int v0 = __popc(__ballot_sync(FULL_MASK, qvalid && d0 <= d1));
            int v1 = __popc(__ballot_sync(FULL_MASK, qvalid && d0 > d1));
            int64_t first = v0 >= v1 ? c0 : c1, second = v0 >= v1 ? c1 : c0;
            if (lane == 0) {
                stack[sp] = (int)second;      // popped last
                stack[sp + 1] = (int)first;   // popped next
            }
            sp += 2;
            __syncwarp();
        }
    }
    if (qvalid) {
        // neighbours are written as canonical ids; rows by canonical id
        // (out_by_cid) or by search position
        int64_t row = out_by_cid ? (int64_t)__float_as_uint(q.w) : qp;
#pragma unroll
        for (int i = 0; i < KMAX; i++) {  // slot i holds rank keff-1-i
            if (i < keff) nbr[row * keff + (keff - 1 - i)] = (int32_t)(uint32_t)(tk.key[i] & 0xffffffffu);
        }
    }
}

__global__ void k_cid_to_pos(const int32_t *__restrict__ cid, int64_t n, int32_t *pos_of_cid) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        pos_of_cid[cid[p]] = (int32_t)p;
}

__global__ void k_map_ids(int32_t *a, int64_t m, const int32_t *__restrict__ pos_of_cid) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = pos_of_cid[a[i]];
}

}  // namespace

void morton_frame(ngs_ctx *c, const float *xyz, int64_t n, float *frame) {
    uint32_t *acc = ws<uint32_t>(c->b_bbox, 8);
    launch(c, "frame_init", dim3(1), dim3(32), 0, k_frame_init, acc);
    launch(c, "frame_reduce", dim3(grid_stride_blocks(c, n, 256, 4)), dim3(256), 0,
           k_frame_reduce, xyz, n, acc);
    launch(c, "frame_final", dim3(1), dim3(1), 0, k_frame_final, (const uint32_t *)acc, frame);
}

void morton_keys(ngs_ctx *c, const float *xyz, int64_t n, const float *frame, uint32_t *keys,
                 uint32_t *vals) {
    launch(c, "morton", dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0, k_morton, xyz, n,
           frame, keys, vals);
}

void gather_points(ngs_ctx *c, const float *xyz, const int32_t *cid, const uint32_t *order,
                   int64_t n, float4 *pts) {
    launch(c, "gather_pts", dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0, k_gather_pts,
           xyz, cid, order, n, pts);
}

void knn_search(ngs_ctx *c, const KnnInput &in, int k_eff, int32_t *nbr) {
    int64_t n = in.n;
    if (n <= 1 || k_eff <= 0) return;
    int64_t nb = (n + NGS_LEAF - 1) / NGS_LEAF;
    int64_t P = 1;
    while (P < nb) P <<= 1;
    float4 *nodes = ws<float4>(c->b_nodes, 4 * P);
    launch(c, "tree_leaves", dim3(blocks_for(P * 32, 256)), dim3(256), 0, k_tree_leaves, in.pts,
           n, nb, P, nodes);
    for (int64_t first = P / 2; first >= 1; first /= 2)
        launch(c, "tree_level", dim3(blocks_for(first, 256)), dim3(256), 0, k_tree_level, nodes,
               first, first);
    dim3 grid(blocks_for(nb, KNN_WARPS)), block(KNN_WARPS * 32);
    int by_cid = in.out_by_cid;
    const float4 *cn = nodes;
    if (k_eff <= 4)
        launch(c, "knn_k4", grid, block, 0, k_knn<4>, in.pts, n, nb, P, cn, k_eff, by_cid, nbr);
    else if (k_eff <= 8)
        launch(c, "knn_k8", grid, block, 0, k_knn<8>, in.pts, n, nb, P, cn, k_eff, by_cid, nbr);
    else if (k_eff <= 16)
        launch(c, "knn_k16", grid, block, 0, k_knn<16>, in.pts, n, nb, P, cn, k_eff, by_cid, nbr);
    else
        launch(c, "knn_k32", grid, block, 0, k_knn<32>, in.pts, n, nb, P, cn, k_eff, by_cid, nbr);
    if (!by_cid) {
        // search order = rows: translate the canonical ids to rows
        int32_t *pos_of_cid = ws<int32_t>(c->b_nbr2, n);
        launch(c, "knn_cid_to_pos", dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0,
               k_cid_to_pos, in.cid, n, pos_of_cid);
        launch(c, "knn_map_ids", dim3(grid_stride_blocks(c, n * k_eff, 256, 8)), dim3(256), 0,
               k_map_ids, nbr, n * k_eff, (const int32_t *)pos_of_cid);
    }
}
