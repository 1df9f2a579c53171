// k-nearest-neighbour search over splat centres (Sec. 3.1, Algorithm 1 KNN).
//
// Centres are quantised on a 1024^3 grid over the scene's bounding cube and
// sorted by Morton code, so every cell of every coarser level 2^l (l <= 10)
// is a contiguous range of the sorted array.  A dense table of range starts
// at one level l_t (8^l_t >= 4 n cells, at most 8^9) gives O(1) ranges for l <= l_t and a
// short binary search inside a table cell for finer levels.
// Each query (one thread, threads in Morton order) picks the finest level
// whose 3x3x3 block of cells around it holds at least 64 points.  It scans
// its own cell, then the 26 around it (faces, edges, corners; a cell is
// skipped when its box is already farther than the query's current k-th
// distance), then whole shells of cells until its k-th distance is strictly
// inside the scanned block (with margins for FP32 rounding of
// distances and of the quantisation), so the list is exactly the k_eff
// nearest by (d^2, canonical id).  Distances are (dx^2 + dy^2) + dz^2 in
// FP32 without contraction.
#include "ngs_device.cuh"
#include "ngs_internal.h"

namespace {

__device__ __forceinline__ float dist2_rn(float dx, float dy, float dz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
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

// ---------------------------------------------------------------- cell table
// T[c] = first sorted position whose global cell id is >= c, for every c in
// [0, tlen] (T[tlen] = n): the start of cell c and the end of cell c - 1.
// The global cell id of position p is toff[scene] + (Morton code >> the
// scene's level shift); it does not decrease along the sorted positions.
// Position p (0 < p < n) therefore owns the cells (id(p-1), id(p)]: all of
// them start at p; position 0 owns [0, id(0)] and a virtual position n owns
// (id(n-1), tlen].  Each position writes its run; a run longer than 64 cells
// (the empty space between surfaces) is cut into chunks of at most 16384
// cells that whole blocks write, so one huge gap does not serialise on one
// block.  Every cell is written once: no zeroing, no atomics per point and no
// scan over the (mostly empty) table.
constexpr int CELL_RUN_DIRECT = 64;
constexpr int CELL_CHUNK = 16384;

__device__ __forceinline__ int64_t gcell_at(const uint32_t *__restrict__ scode,
                                            const int32_t *__restrict__ ssid,
                                            const int32_t *__restrict__ lts,
                                            const int64_t *__restrict__ toff, int64_t p) {
    const int sc = ssid ? ssid[p] : 0;
    return toff[sc] + (int64_t)(scode[p] >> (3 * (10 - lts[sc])));
}

// chunk record: x = first cell, y = (cell count << 32) | position
__global__ void k_cell_runs(const uint32_t *__restrict__ scode, const int32_t *__restrict__ ssid,
                            int64_t n, const int32_t *__restrict__ lts,
                            const int64_t *__restrict__ toff, int64_t tlen, int32_t *T,
                            longlong2 *chunks, unsigned long long *nchunk) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t hi = p < n ? gcell_at(scode, ssid, lts, toff, p) : tlen;
        const int64_t lo = p > 0 ? gcell_at(scode, ssid, lts, toff, p - 1) + 1 : 0;
        const int64_t len = hi - lo + 1;
        if (len <= CELL_RUN_DIRECT) {
            for (int64_t c = lo; c <= hi; c++) T[c] = (int32_t)p;
        } else {
            const int64_t m = (len + CELL_CHUNK - 1) / CELL_CHUNK;
            const unsigned long long at = atomicAdd(nchunk, (unsigned long long)m);
            for (int64_t j = 0; j < m; j++) {
                const int64_t c0 = lo + j * CELL_CHUNK;
                const int64_t cl = len - j * CELL_CHUNK < CELL_CHUNK ? len - j * CELL_CHUNK : CELL_CHUNK;
                chunks[at + j] = make_longlong2(c0, (long long)(((uint64_t)cl << 32) | (uint32_t)p));
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_cell_chunks(const longlong2 *__restrict__ chunks,
                                                     const unsigned long long *__restrict__ nchunk,
                                                     int32_t *T) {
    const int64_t cnt = (int64_t)*nchunk;
    for (int64_t r = blockIdx.x; r < cnt; r += gridDim.x) {
        const longlong2 ch = chunks[r];
        const int cl = (int)((uint64_t)ch.y >> 32);
        const int32_t v = (int32_t)(uint32_t)ch.y;
        for (int i = threadIdx.x; i < cl; i += blockDim.x) T[ch.x + i] = v;
    }
}

// ---------------------------------------------------------------- query
__device__ __forceinline__ uint32_t compact10(uint32_t v) {
    v &= 0x09249249u;
    v = (v ^ (v >> 2)) & 0x030c30c3u;
    v = (v ^ (v >> 4)) & 0x0300f00fu;
    v = (v ^ (v >> 8)) & 0x030000ffu;
    v = (v ^ (v >> 16)) & 0x000003ffu;
    return v;
}

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
};

struct GridCtx {
    const uint32_t *scode;
    const int32_t *T;
    int lt;  // table level
};

// Sorted-position range of the level-l cell with Morton prefix `pre`.
__device__ __forceinline__ void cell_range(const GridCtx &g, int l, uint32_t pre, int32_t &a,
                                           int32_t &b) {
    if (l <= g.lt) {
        int sh = 3 * (g.lt - l);
        a = g.T[(int64_t)pre << sh];
        b = g.T[((int64_t)pre + 1) << sh];
    } else {
        int sh = 3 * (l - g.lt);
        uint32_t par = pre >> sh;
        int32_t A = g.T[par], B = g.T[par + 1];
        const uint32_t lo_code = pre << (3 * (10 - l));
        const uint32_t hi_code = (pre + 1) << (3 * (10 - l));
        int32_t x = A, y = B;  // lower_bound(lo_code)
        while (x < y) {
            int32_t m = (x + y) >> 1;
            if (g.scode[m] < lo_code) x = m + 1; else y = m;
        }
        a = x;
        y = B;  // lower_bound(hi_code) in [a, B)
        while (x < y) {
            int32_t m = (x + y) >> 1;
            if (g.scode[m] < hi_code) x = m + 1; else y = m;
        }
        b = x;
    }
}

__device__ __forceinline__ uint32_t interleave(uint32_t x, uint32_t y, uint32_t z) {
    return spread10(x) | (spread10(y) << 1) | (spread10(z) << 2);
}

constexpr int KNN_QCAP = 16;   // per-lane candidate queue (shared memory)
constexpr int KNN_BLOCK = 256;

// Points in the 3x3x3 block of level-l cells around cell (cx, cy, cz).
__device__ __forceinline__ int block_count(const GridCtx &g, int l, int32_t cx, int32_t cy,
                                           int32_t cz) {
    const int32_t gmax = (1 << l) - 1;
    uint32_t sx[3], sy[3], sz[3];
    bool okx[3], oky[3], okz[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const int32_t x = cx + d - 1, y = cy + d - 1, z = cz + d - 1;
        okx[d] = x >= 0 && x <= gmax;
        oky[d] = y >= 0 && y <= gmax;
        okz[d] = z >= 0 && z <= gmax;
        sx[d] = spread10((uint32_t)x);
        sy[d] = spread10((uint32_t)y) << 1;
        sz[d] = spread10((uint32_t)z) << 2;
    }
    int tot = 0;
#pragma unroll
    for (int dx = 0; dx < 3; dx++)
#pragma unroll
        for (int dy = 0; dy < 3; dy++)
#pragma unroll
            for (int dz = 0; dz < 3; dz++) {
                if (!(okx[dx] && oky[dy] && okz[dz])) continue;
                int32_t lo, hi;
                cell_range(g, l, sx[dx] | sy[dy] | sz[dz], lo, hi);
                tot += hi - lo;
            }
    return tot;
}

// Descending bitonic sort of N register keys (static indices only).
template <int N>
__device__ __forceinline__ void sort_desc(uint64_t (&a)[N]) {
#pragma unroll
    for (int k = 2; k <= N; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < N; i++) {
                const int l = i ^ j;
                if (l > i) {
                    const uint64_t x = a[i], y = a[l];
                    const bool sw = ((i & k) == 0) ? (x < y) : (x > y);
                    a[i] = sw ? y : x;
                    a[l] = sw ? x : y;
                }
            }
}

// Merge up to 8 queued keys (queue rows b0 .. b0+7 of this lane) into a full
// list of KMAX keys by a network: the chunk sorted ascending against the list
// (descending) keeps the elementwise smaller keys, which are the KMAX
// smallest of both as a bitonic sequence; a bitonic merge puts them back in
// descending order.  Same list as inserting the keys one by one.
template <int KMAX>
__device__ __forceinline__ void merge_chunk8(uint64_t (*queue)[32], int lane, int b0, int qlen,
                                             TopK<KMAX> &tk) {
    uint64_t a[8];
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = b0 + i < qlen ? queue[b0 + i][lane] : ~0ull;
    sort_desc<8>(a);
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const uint64_t y = a[7 - i];
        if (y < tk.key[i]) tk.key[i] = y;
    }
#pragma unroll
    for (int j = KMAX / 2; j > 0; j >>= 1)
#pragma unroll
        for (int i = 0; i < KMAX; i++)
            if ((i & j) == 0) {
                const uint64_t x = tk.key[i], y = tk.key[i + j];
                const bool gt = x > y;
                tk.key[i] = gt ? x : y;
                tk.key[i + j] = gt ? y : x;
            }
}

// Insert each lane's queued keys into its list.  A lane whose list is still
// empty (all k_eff = KMAX slots unused) takes its queue by one sorting network
// instead of one insertion per key: the result is the same list (the queued
// keys, largest first, padded with the empty marker).  Otherwise the queue is
// taken in warp-wide chunks of 8 rows: a chunk in which some lane holds 4 or
// more keys goes through the merge network (full-width lists only), a smaller
// one by single insertions.
template <int KMAX>
__device__ __forceinline__ void flush_queue(uint64_t (*queue)[32], int lane, int &qlen,
                                            TopK<KMAX> &tk, int keff) {
    const bool fresh = keff == KMAX && qlen > 0 && qlen <= KMAX && tk.key[KMAX - 1] == ~0ull;
    if (fresh) {
        uint64_t a[KMAX];
#pragma unroll
        for (int i = 0; i < KMAX; i++) a[i] = i < qlen ? queue[i][lane] : ~0ull;
        sort_desc<KMAX>(a);
#pragma unroll
        for (int i = 0; i < KMAX; i++) tk.key[i] = a[i];
        qlen = 0;
    }
    const int rounds = __reduce_max_sync(FULL_MASK, qlen);
    if (KMAX == 16 && keff == KMAX) {  // keff is the same for every lane
        for (int b0 = 0; b0 < rounds; b0 += 8) {
            const int cnt = min(8, rounds - b0);
            if (cnt >= 4) {
                merge_chunk8<KMAX>(queue, lane, b0, qlen, tk);
            } else {
                for (int r = b0; r < b0 + cnt; r++) {
                    if (r < qlen) {
                        uint64_t x = queue[r][lane];
                        if (x < tk.kth()) tk.insert(x);
                    }
                }
            }
        }
    } else {
        for (int r = 0; r < rounds; r++) {
            if (r < qlen) {
                uint64_t x = queue[r][lane];
                if (x < tk.kth()) tk.insert(x);
            }
        }
    }
    qlen = 0;
    __syncwarp();
}

// The 26 neighbours of a cell ordered by distance class: faces, edges, corners.
__device__ const char3 kShell1[26] = {
    {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}, {-1, -1, 0},
    {-1, 1, 0}, {1, -1, 0}, {1, 1, 0}, {-1, 0, -1}, {-1, 0, 1}, {1, 0, -1}, {1, 0, 1},
    {0, -1, -1}, {0, -1, 1}, {0, 1, -1}, {0, 1, 1}, {-1, -1, -1}, {-1, -1, 1}, {-1, 1, -1},
    {-1, 1, 1}, {1, -1, -1}, {1, -1, 1}, {1, 1, -1}, {1, 1, 1}};

// Cells of the shell at Chebyshev distance r around the query cell, in a
// fixed order (for r = 1: the 6 face neighbours, 12 edge and 8 corner cells).
__device__ __forceinline__ bool shell_cell(int r, int t, int &dx, int &dy, int &dz) {
    if (r == 0) {
        dx = dy = dz = 0;
        return t == 0;
    }
    if (r == 1) {
        if (t >= 26) return false;
        const char3 o = kShell1[t];
        dx = o.x;
        dy = o.y;
        dz = o.z;
        return true;
    }
    const int side = 2 * r + 1;
    if (t >= side * side * side) return false;
    dx = t / (side * side) - r;
    dy = (t / side) % side - r;
    dz = t % side - r;
    return true;
}

// One thread per query, threads in Morton order.  Each lane walks its own
// stream of cells (shell r = 0, 1, 2, ... around its cell), scanning a cell
// at a time; candidates under the lane's threshold are queued and inserted
// in warp-wide rounds, so list updates are not serialised by divergence.
template <int KMAX>
__global__ void __launch_bounds__(KNN_BLOCK, 3)
    k_knn_grid(const float4 *__restrict__ pts, const uint32_t *__restrict__ scode,
               const uint32_t *__restrict__ sidx, const int32_t *__restrict__ ssid, int64_t n,
               const int32_t *__restrict__ Tall, const int32_t *__restrict__ lts,
               const int64_t *__restrict__ toff, const float *__restrict__ frames, int keff,
               int out_by_cid, int block_min, const int32_t *__restrict__ qlist, int64_t nq,
               int32_t *__restrict__ nbr) {
    __shared__ uint64_t queue_all[KNN_BLOCK / 32][KNN_QCAP][32];
    const int lane = threadIdx.x & 31;
    uint64_t(*queue)[32] = queue_all[threadIdx.x >> 5];
    // query t: sorted position t, or qlist[t] (ascending positions) when given
    const int64_t qt = (int64_t)blockIdx.x * KNN_BLOCK + threadIdx.x;
    const bool valid = qt < nq;
    const int64_t qp = valid ? (qlist ? (int64_t)qlist[qt] : qt) : n;
    // this query's scene: its Morton frame and its cell table
    const int sc = (ssid && valid) ? ssid[qp] : 0;
    const int lt = lts[sc];
    const GridCtx g{scode, Tall + toff[sc], lt};
    const float *frame = frames + 8 * sc;
    const float lx = frame[0], ly = frame[1], lz = frame[2], scale = frame[3];
    const float inv_scale = 1.0f / scale;
    const float4 q = valid ? pts[qp] : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t code = valid ? scode[qp] : 0u;
    // level: the finest (up to the table level) whose 3x3x3 block around the
    // query holds at least 64 points, one level finer when that still holds
    // 64 and the block is crowded
    const uint32_t qx = compact10(code), qy = compact10(code >> 1), qz = compact10(code >> 2);
    int l = lt;
    if (valid) {
        int bc = block_count(g, l, qx >> (10 - l), qy >> (10 - l), qz >> (10 - l));
        while (l > 1 && bc < block_min) {
            l--;
            bc = block_count(g, l, qx >> (10 - l), qy >> (10 - l), qz >> (10 - l));
        }
        if (bc > 6 * block_min && l < 10) {
            int b2 = block_count(g, l + 1, qx >> (9 - l), qy >> (9 - l), qz >> (9 - l));
            if (b2 >= block_min) l++;
        }
    }
    const int sh = 10 - l;
    const int32_t cx = (int32_t)(qx >> sh), cy = (int32_t)(qy >> sh), cz = (int32_t)(qz >> sh);
    const int32_t gmax = (1 << l) - 1;
    const float h = inv_scale * (float)(1 << sh);  // cell side at level l
    const float margin = 1e-3f * inv_scale;
    TopK<KMAX> tk;
    tk.init(keff);
    int qlen = 0;
    bool active = valid;
    for (int r = 0;; r++) {
        int t = 0;
        int32_t p = 0, b = 0;
        bool more = active;
        while (__any_sync(FULL_MASK, more)) {
            if (more) {
                // next non-empty cell of the shell
                while (p >= b) {
                    int dx, dy, dz;
                    if (!shell_cell(r, t, dx, dy, dz)) {
                        more = false;
                        break;
                    }
                    t++;
                    const int ch = max(max(abs(dx), abs(dy)), abs(dz));
                    const int32_t x = cx + dx, y = cy + dy, z = cz + dz;
                    if (ch != r || x < 0 || y < 0 || z < 0 || x > gmax || y > gmax || z > gmax)
                        continue;
                    // skip a cell that no point of it could enter the list from: its
                    // box (widened by the quantisation margin) is farther than the
                    // current k-th distance with the FP32 slack of d^2
                    if (r > 0 && tk.kth() != ~0ull) {
                        const float ex = fmaxf(fmaxf((lx + (float)x * h - margin) - q.x,
                                                     q.x - (lx + (float)(x + 1) * h + margin)), 0.f);
                        const float ey = fmaxf(fmaxf((ly + (float)y * h - margin) - q.y,
                                                     q.y - (ly + (float)(y + 1) * h + margin)), 0.f);
                        const float ez = fmaxf(fmaxf((lz + (float)z * h - margin) - q.z,
                                                     q.z - (lz + (float)(z + 1) * h + margin)), 0.f);
                        const float kd = __uint_as_float((uint32_t)(tk.kth() >> 32));
                        if ((ex * ex + ey * ey + ez * ez) * (1.0f - 4e-6f) > kd) continue;
                    }
                    cell_range(g, l, interleave((uint32_t)x, (uint32_t)y, (uint32_t)z), p, b);
                }
                // scan the cell while the queue has room
                for (; more && p < b && qlen < KNN_QCAP; p++) {
                    if (p == qp) continue;
                    const float4 c = pts[p];
                    const float d2 =
                        dist2_rn(__fsub_rn(q.x, c.x), __fsub_rn(q.y, c.y), __fsub_rn(q.z, c.z));
                    const uint64_t kk = ((uint64_t)__float_as_uint(d2) << 32) | __float_as_uint(c.w);
                    if (kk < tk.kth()) queue[qlen++][lane] = kk;
                }
            }
            if (__any_sync(FULL_MASK, qlen == KNN_QCAP)) flush_queue<KMAX>(queue, lane, qlen, tk, keff);
        }
        flush_queue<KMAX>(queue, lane, qlen, tk, keff);
        if (active) {
            // distance from q to the outside of the scanned block; a face on
            // the grid boundary has no point beyond it
            float G = INFINITY;
            bool covers_all = true;
            if (cx - r > 0) { G = fminf(G, q.x - (lx + (float)(cx - r) * h)); covers_all = false; }
            if (cx + r < gmax) { G = fminf(G, (lx + (float)(cx + r + 1) * h) - q.x); covers_all = false; }
            if (cy - r > 0) { G = fminf(G, q.y - (ly + (float)(cy - r) * h)); covers_all = false; }
            if (cy + r < gmax) { G = fminf(G, (ly + (float)(cy + r + 1) * h) - q.y); covers_all = false; }
            if (cz - r > 0) { G = fminf(G, q.z - (lz + (float)(cz - r) * h)); covers_all = false; }
            if (cz + r < gmax) { G = fminf(G, (lz + (float)(cz + r + 1) * h) - q.z); covers_all = false; }
            if (covers_all) {
                active = false;
            } else {
                G -= margin;
                if (tk.kth() != ~0ull && G > 0.f) {
                    const float kd = __uint_as_float((uint32_t)(tk.kth() >> 32));
                    if (kd <= G * G * (1.0f - 4e-6f)) active = false;
                }
            }
        }
        if (!__any_sync(FULL_MASK, active)) break;
    }
    if (valid) {
        const int64_t row = out_by_cid ? (int64_t)__float_as_uint(q.w) : (int64_t)sidx[qp];
#pragma unroll
        for (int i = 0; i < KMAX; i++)  // slot i holds rank keff-1-i
            if (i < keff) nbr[row * keff + (keff - 1 - i)] = (int32_t)(uint32_t)(tk.key[i] & 0xffffffffu);
    }
}

__global__ void k_cid_to_pos(const int32_t *__restrict__ cid, int64_t n, int32_t *pos_of_cid) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        pos_of_cid[cid[p]] = (int32_t)p;
}

// a: a 16-byte aligned workspace array
__global__ void k_map_ids(int32_t *a, int64_t m, const int32_t *__restrict__ pos_of_cid) {
    // four ids per thread (16-byte accesses, four gathers in flight), then the tail
    const int64_t m4 = m >> 2;
    int4 *a4 = (int4 *)a;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m4;
         i += (int64_t)gridDim.x * blockDim.x) {
        int4 x = a4[i];
        x.x = __ldg(pos_of_cid + x.x);
        x.y = __ldg(pos_of_cid + x.y);
        x.z = __ldg(pos_of_cid + x.z);
        x.w = __ldg(pos_of_cid + x.w);
        a4[i] = x;
    }
    for (int64_t i = 4 * m4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = pos_of_cid[a[i]];
}

}  // namespace

void morton_frame(ngs_ctx *c, const float *xyz, int64_t n, float *frame) {
    uint32_t *acc = ws<uint32_t>(c, c->b_bbox, 8);
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

int knn_table_level(int64_t n, int cells_per_point) {
    int lt = 1;
    while (lt < 9 && ((int64_t)1 << (3 * lt)) < (int64_t)cells_per_point * n) lt++;
    return lt;
}

void knn_search(ngs_ctx *c, const KnnInput &in, int k_eff, int32_t *nbr) {
    const int64_t n = in.n;
    if (n <= 1 || k_eff <= 0) return;
    const int S = in.nscenes;
    // per-scene table levels (about 4 or more cells per point, at most 8^9
    // cells) and offsets of the concatenated tables; a scene's table ends
    // with one extra zero count so that the global exclusive scan gives every
    // cell its sorted start position and the scene its end
    // (small scene counts stay on the stack: the allocation-free entry point
    // calls this with one scene)
    int32_t lt_stack[4];
    int64_t off_stack[5];
    std::vector<int32_t> lt_heap;
    std::vector<int64_t> off_heap;
    int32_t *hlt = lt_stack;
    int64_t *hoff = off_stack;
    if (S > 4) {
        lt_heap.resize(S);
        off_heap.resize(S + 1);
        hlt = lt_heap.data();
        hoff = off_heap.data();
    }
    hoff[0] = 0;
    for (int s = 0; s < S; s++) {
        hlt[s] = knn_table_level(in.scene_n[s], c->tune.cells_per_point);
        hoff[s + 1] = hoff[s] + ((int64_t)1 << (3 * hlt[s])) + 1;
    }
    const int64_t tlen = hoff[S];
    uint8_t *small = ws<uint8_t>(c, c->b_knnsc, 16 * (S + 1) + 256);
    int32_t *dlt = (int32_t *)small;
    int64_t *doff = (int64_t *)(small + ((4 * (size_t)S + 15) & ~(size_t)15));
    put_small(c, dlt, hlt, 4 * (size_t)S);
    put_small(c, doff, hoff, 8 * (size_t)(S + 1));
    int32_t *T = ws<int32_t>(c, c->b_nodes, tlen + 1);
    // chunks: at most one per position plus one per CELL_CHUNK cells
    const int64_t max_chunks = n + 2 + tlen / CELL_CHUNK;
    uint8_t *lr = ws<uint8_t>(c, c->b_knnlong, 16 * (max_chunks + 1));
    unsigned long long *nchunk = (unsigned long long *)lr;
    longlong2 *chunks = (longlong2 *)(lr + 16);
    NGS_CHECK_CUDA(cudaMemsetAsync(nchunk, 0, 8, c->st));
    launch(c, "cell_runs", dim3(grid_stride_blocks(c, n + 1, 256, 8)), dim3(256), 0, k_cell_runs,
           in.scode, in.ssid, n, (const int32_t *)dlt, (const int64_t *)doff, tlen, T, chunks,
           nchunk);
    launch(c, "cell_chunks", dim3((unsigned)c->num_sms * 8), dim3(256), 0, k_cell_chunks,
           (const longlong2 *)chunks, (const unsigned long long *)nchunk, T);
    const int64_t nq = in.qlist ? in.nq : n;
    const unsigned grid = blocks_for(nq, KNN_BLOCK);
    const int32_t *cT = T;
#define KNN_LAUNCH(KM, NAME)                                                                   \
    launch(c, NAME, dim3(grid), dim3(KNN_BLOCK), 0, k_knn_grid<KM>, in.pts, in.scode, in.sidx,   \
           in.ssid, n, cT, (const int32_t *)dlt, (const int64_t *)doff, in.frames, k_eff,      \
           in.out_by_cid, c->tune.knn_block_min, in.qlist, nq, nbr)
    if (nq > 0) {
        if (k_eff <= 4) KNN_LAUNCH(4, "knn_k4");
        else if (k_eff <= 8) KNN_LAUNCH(8, "knn_k8");
        else if (k_eff <= 16) KNN_LAUNCH(16, "knn_k16");
        else KNN_LAUNCH(32, "knn_k32");
    }
#undef KNN_LAUNCH
    if (!in.out_by_cid) {
        // rows are internal indices; translate the neighbours' canonical ids
        int32_t *pos_of_cid = ws<int32_t>(c, c->b_nbr2, n);
        launch(c, "knn_cid_to_pos", dim3(grid_stride_blocks(c, n, 256, 8)), dim3(256), 0,
               k_cid_to_pos, in.cid, n, pos_of_cid);
        launch(c, "knn_map_ids", dim3(grid_stride_blocks(c, n * k_eff, 256, 8)), dim3(256), 0,
               k_map_ids, nbr, n * k_eff, (const int32_t *)pos_of_cid);
    }
}
