// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ngs.h"

// NGS_MAX_N (ngs.h) bounds the rows of one call; n * k_eff must also stay at
// or below NGS_MAX_SLOTS, so that slot indices v * k_eff + j fit int32
#define NGS_MAX_SLOTS ((int64_t)1 << 30)
#define NGS_LEAF 32                     // kNN tree leaf = one warp of points

// ---------------------------------------------------------------- errors
void ngs_set_error(const char *fmt, ...);

struct NgsError {
    int code;
};

#define NGS_CHECK_CUDA(call)                                                         \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            ngs_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                 \
                          cudaGetErrorString(e_));                                   \
            throw NgsError{e_ == cudaErrorMemoryAllocation ? NGS_ERR_OOM : NGS_ERR_CUDA}; \
        }                                                                            \
    } while (0)

#define NGS_FAIL(code, ...)            \
    do {                               \
        ngs_set_error(__VA_ARGS__);    \
        throw NgsError{code};          \
    } while (0)

// ---------------------------------------------------------------- workspace
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};
// Grow-only device buffer (contents are not preserved on growth).  Memory
// comes from the library's stream-ordered pool on the ctx's stream: growing
// a buffer frees the old block after the work already queued on that stream
// and never synchronises the device, so contexts on other streams keep
// running.
struct ngs_ctx;
void *ws_get(ngs_ctx *c, DevBuf &b, size_t bytes);
template <class T>
T *ws(ngs_ctx *c, DevBuf &b, int64_t count) {
    return (T *)ws_get(c, b, (size_t)(count > 0 ? count : 1) * sizeof(T));
}

// ---------------------------------------------------------------- ctx
struct KStat {
    const char *name;
    int64_t launches;
    double ms;
};

struct PendingEv {
    int stat;
    cudaEvent_t a, b;
};

// Splat arrays in device memory (SoA).
struct SplatView {
    float *xyz, *ls, *rot, *logit, *sh;
    int64_t n;
    int F;
};

struct GraphDev {
    int64_t n;
    int k_eff;
    const int32_t *cid;     // canonical ids (nullptr = identity)
    const int32_t *nbr;     // n*k directed neighbours (slot s = v*k + t)
    int32_t *mirror;        // n*k partner slot of a mutual edge, else -1 (row form: slot code)
    int4 *erec;             // |E| edge records (slot, lo row, hi row, mirror slot or -2 - rev position)
    int32_t *rev_ptr;       // n+1 offsets into rev
    int32_t *rev;           // non-mutual slots pointing at each vertex
    float *revcost;         // cost of each rev entry (the same order)
    float *cost_slot;       // n*k cost of the edge of each slot
    int64_t n_edges;        // |E| (host copy)
    int32_t *elo, *ehi;     // C-ABI view: lexicographic edges (canonical ids)
    int4 *erec_lex;         // edge records in lexicographic order
};

// Performance parameters (results do not depend on them), set by
// ngs_set_tuning or ngs_autotune.
struct Tuning {
    int knn_block_min = 64;      // points the kNN 3x3x3 block must hold
    int cells_per_point = 4;     // cell-table density (cells >= this x points)
    int cost_blocks_per_sm = 8;  // edge-cost grid, 256-thread blocks per SM
    int match_method = 2;        // 2 proposals, 1 rounds in a CUDA graph, 0 host-driven rounds
    int match_max_steps = 1 << 16;  // proposal steps per thread before the round form takes over
    int scan_method = 0;         // 0: reduce, partials, apply; 1: single pass (decoupled look-back)
    int wait_budget_cycles = 2000000000;  // a device-wide wait gives up after this many cycles
    int wait_test_tile = -1;     // tests of the bounded waits: this scan tile publishes late
};

struct ngs_ctx {
    ngs_params prm;
    Tuning tune;
    cudaStream_t st;
    int device;
    int num_sms;

    // graph of the last ngs_build_graph (canonical mode)
    bool g_valid = false;
    int64_t g_n = 0;
    int32_t g_k = 0;
    int64_t g_edges = 0;
    const float *g_xyz = nullptr;
    GraphDev g{};

    // workspaces
    DevBuf b_pts, b_codes, b_codes2, b_vals, b_vals2, b_hist, b_bbox, b_frame;
    DevBuf b_nodes, b_nbr, b_deg, b_cap, b_rstart, b_adj, b_adjeid, b_fill, b_upc, b_eptr;
    DevBuf b_elo, b_ehi, b_rec, b_cost, b_rng;
    DevBuf b_mate, b_cand, b_candkey, b_counts, b_sel, b_role, b_keep, b_pos, b_flag;
    DevBuf b_scan_part, b_status, b_misc, b_cid, b_cid2, b_cflag, b_cscan;
    DevBuf b_sA[5], b_sB[5];     // ping-pong splat arrays
    DevBuf b_pairs, b_partner, b_nbr2, b_lexrec, b_sel2, b_cflag2, b_knnsc;
    DevBuf b_host_dev[5];        // device staging for ngs_simplify_host
    DevBuf b_sC[5];              // third splat array set (several scenes at once)
    DevBuf b_fp64list;           // edges whose cost is evaluated in FP64
    DevBuf b_tiebits, b_tielist; // near-tie slot marks and the slots to recompute in FP64
    DevBuf b_revcost;            // in-edge costs in rev order
    DevBuf b_knnlong;            // long runs of empty cells of the kNN cell table
    DevBuf b_prevnbr, b_rmap, b_rsrc, b_qflag, b_qlist;  // local refresh: old lists, id maps, queries
    DevBuf b_mstate;             // device-side state of the captured matching rounds
    DevBuf b_offer;              // best offer per vertex (proposal form of the matching)
    DevBuf b_eng[32];            // per-scene tables and scratch of the multi-scene engine

    // pinned host scratch
    int64_t *h_pin = nullptr;
    // where a kernel records that a bounded device-wide wait ran out (pinned
    // host memory, h_pin + 8, checked by sync_stream; a device word in the
    // allocation-free entry point); nullptr: the scan uses no waits
    volatile int32_t *err_word = nullptr;

    // instrumentation
    bool prof = false;
    std::vector<KStat> kstats;
    std::vector<PendingEv> pending;
    std::vector<cudaEvent_t> ev_free;
    int64_t launches = 0;
    int64_t syncs = 0;            // host waits on the ctx stream
    int64_t ws_bytes = 0;         // device workspace currently held
    bool ws_fixed = false;        // workspaces are bound to fixed memory: growing one fails
    cudaStream_t cap_st = nullptr;  // private stream the graph is captured on
    cudaStream_t up_st = nullptr;   // second upload stream of ngs_simplify_host
    cudaEvent_t up_ev = nullptr;    // SH upload finished
    cudaEvent_t up_first = nullptr; // opacity and centres uploaded (on st)
    cudaEvent_t up_rest = nullptr;  // log-scales and rotations uploaded
    cudaEvent_t rest_wait = nullptr;  // set for one engine call: scales/rotations not yet on the device
    cudaEvent_t sh_wait = nullptr;  // set for one engine call: SH input not yet on the device
    DevBuf b_order0;                 // initial Morton permutation kept for the deferred SH gather

    // per-call counters
    int64_t fp64_edges = 0;
    int64_t tie_slots = 0;
    int64_t requeried = 0;        // rows queried by the last graph build (refresh or full)
    int64_t floor_hits = 0;
    int32_t rounds = 0;
};

// Launch bookkeeping: records events when profiling, counts launches, and
// converts launch errors into exceptions.
int prof_slot(ngs_ctx *c, const char *name);
void prof_begin(ngs_ctx *c, int slot, cudaEvent_t *a);
void prof_end(ngs_ctx *c, int slot, cudaEvent_t a);

template <class Kernel, class... Args>
void launch(ngs_ctx *c, const char *name, dim3 grid, dim3 block, size_t smem, Kernel k,
            Args... args) {
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return;
    int slot = -1;
    cudaEvent_t a = nullptr;
    if (c->prof) {
        slot = prof_slot(c, name);
        prof_begin(c, slot, &a);
    }
    k<<<grid, block, smem, c->st>>>(args...);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) NGS_FAIL(NGS_ERR_CUDA, "launch %s: %s", name, cudaGetErrorString(e));
    c->launches++;
    if (c->prof) prof_end(c, slot, a);
}

inline unsigned blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : b);
}
// Grid of a grid-stride kernel: a multiple of the SM count, at most `need`.
inline unsigned grid_stride_blocks(ngs_ctx *c, int64_t work, int threads, int per_sm) {
    int64_t need = (work + threads - 1) / threads;
    int64_t cap = (int64_t)c->num_sms * per_sm;
    if (need < 1) need = 1;
    return (unsigned)(need < cap ? need : cap);
}

void sync_stream(ngs_ctx *c);

// ---------------------------------------------------------------- primitives (k_prim.cu)
// Exclusive scan of n int32 counts into out[0..n] (out[n] = total).  in may
// alias out.  Totals must fit in int32.
void scan_i32(ngs_ctx *c, const int32_t *in, int32_t *out, int64_t n);
// Stable LSD radix sort of (key, val) pairs by the low `bits` bits of key.
// Result in (keys, vals); tmp buffers of n entries are provided.
void radix_sort_u32(ngs_ctx *c, uint32_t *keys, uint32_t *vals, uint32_t *keys_tmp,
                    uint32_t *vals_tmp, int64_t n, int bits);
void iota_u32(ngs_ctx *c, uint32_t *a, int64_t n);
// Host bytes to device memory on the ctx stream; small sizes go as a kernel
// parameter (no copy engine).  The source may be reused on return.
void put_small(ngs_ctx *c, void *dst, const void *src, size_t bytes);
// Device bytes into pinned host memory (c->h_pin) by a kernel on the ctx
// stream; valid on the host after the stream is synchronised.
void get_small(ngs_ctx *c, void *hdst, const void *dsrc, size_t bytes);
// out[i] = src[idx[i]]
void gather_u32(ngs_ctx *c, const uint32_t *src, const uint32_t *idx, int64_t n, uint32_t *out);
// k-th smallest (0-based) of n 32-bit orderable keys -> *d_out (device).
void radix_select_u32(ngs_ctx *c, const uint32_t *keys, int64_t n, int64_t k, uint32_t *d_out);
// k-th smallest (0-based) among the 64-bit keys; entries equal to
// UINT64_MAX are padding and never selected.  Result -> *d_out (device).
void radix_select_u64(ngs_ctx *c, const uint64_t *keys, int64_t n, int64_t k, uint64_t *d_out);

// ---------------------------------------------------------------- graph (k_knn.cu, k_graph.cu)
// Input of the kNN search: points grouped by scene and sorted by 30-bit
// Morton code in their scene's frame.
//   pts[p]  = (x, y, z, canonical id bits) at sorted position p
//   scode[p] = Morton code (ascending within a scene), sidx[p] = internal row
//   ssid[p] = scene of position p (nullptr: one scene)
//   frames  = nscenes x 8 floats (lo.xyz, cells per unit, ...), device
//   scene_n = points per scene (host, nscenes entries)
//   out_by_cid = 1: canonical id == internal row; 0: rows are internal
//   indices and neighbours are translated from canonical ids via cid[]
//   (cid of each internal row).
struct KnnInput {
    const float4 *pts;
    const uint32_t *scode;
    const uint32_t *sidx;
    const int32_t *ssid;
    const float *frames;
    const int64_t *scene_n;
    int nscenes;
    int64_t n;
    int out_by_cid;
    const int32_t *cid;
    const int32_t *qlist = nullptr;  // sorted positions to query (nullptr: all n)
    int64_t nq = 0;                  // their count (with qlist)
};
int knn_table_level(int64_t n, int cells_per_point = 4);
// neighbours per splat in a pass over n splats: min(max(1, k), n - 1)
inline int k_eff_of(int64_t n, int k) {
    int ke = k < 1 ? 1 : k;
    if ((int64_t)ke > n - 1) ke = (int)(n - 1);
    return ke;
}
inline void check_slots(int64_t n, int k, const char *fn) {
    if (n >= 2 && n * (int64_t)k_eff_of(n, k) > NGS_MAX_SLOTS)
        NGS_FAIL(NGS_ERR_INVALID_ARG, "%s: n=%lld times k_eff=%d is above %lld", fn, (long long)n,
                 k_eff_of(n, k), (long long)NGS_MAX_SLOTS);
}
// Algorithm 1 over S scenes at once (scenes[s] in place, targets[s] >= 1);
// S == 1 is ngs_simplify.  For S > 1 every target must exceed
// min(max(1, k), NGS_MAX_K) so that all scenes share one k_eff.
void engine_simplify(ngs_ctx *c, ngs_splats *scenes, const int64_t *targets, int S, ngs_stats *st);
// Compute the Morton frame (lo.xyz, 1/side) of n centres into frame[4].
void morton_frame(ngs_ctx *c, const float *xyz, int64_t n, float *frame);
// Morton keys of n centres in `frame`, with vals = 0..n-1 (or given).
void morton_keys(ngs_ctx *c, const float *xyz, int64_t n, const float *frame, uint32_t *keys,
                 uint32_t *vals);
// Gather float4 points (x,y,z,cid) in the order of `order` (nullptr = identity).
void gather_points(ngs_ctx *c, const float *xyz, const int32_t *cid, const uint32_t *order,
                   int64_t n, float4 *pts);
// Directed kNN: nbr[row*k_eff + t] = internal index of the t-th neighbour.
void knn_search(ngs_ctx *c, const KnnInput &in, int k_eff, int32_t *nbr);

// Build the slot-form undirected graph from nbr (see k_graph.cu).
void build_edges(ngs_ctx *c, const int32_t *nbr, GraphDev &g);
// Lexicographic edge list (elo, ehi, lex_slot) of the graph, for the C ABI.
void build_lex_view(ngs_ctx *c, GraphDev &g);

// Local neighbourhood refresh (Sec. 3.4).  After a merge of n_old rows
// (role: >= 0 partner for the lower member, -2 removed, -1 kept; surviving
// rows keep their order), map_old[o] = new row of old row o (a removed row
// takes its partner's) and src_new[r] = old row of a kept new row r, -1 for a
// merged splat.  Uses b_qflag and b_qlist as scratch.
void refresh_map(ngs_ctx *c, int64_t n_old, const int32_t *role, int32_t *map_old,
                 int32_t *src_new);
// Lists of the n new rows carried from prev (n_old x k_old, rows of the old
// set): a kept row whose mapped list has k_eff distinct ids other than itself
// gets them sorted by (FP32 d^2, canonical id), written as canonical ids
// (cid[m], or m when cid is null); the others are flagged in qflag[r] for a
// query.  Then qlist receives the sorted positions (order: sorted position
// -> row) of the flagged rows; returns their count (host).  An old list entry
// outside [0, n_old) fails with NGS_ERR_INVALID_ARG.
// true when every a[i], i < m, lies in [0, n) (synchronises)
bool ids_in_range(ngs_ctx *c, const int32_t *a, int64_t m, int64_t n);
int64_t refresh_rows(ngs_ctx *c, int64_t n, int k_eff, int k_old, int64_t n_old,
                     const int32_t *src_new, const int32_t *prev, const int32_t *map_old,
                     const float *xyz, const int32_t *cid, const uint32_t *order, int32_t *nbr,
                     int32_t *qlist);

// ---------------------------------------------------------------- cost (k_cost.cu)
// Cost of every edge into g.cost_slot (both slots of a mutual edge).  With
// lex = true the edges are visited in lexicographic order and also written
// to cost_out[e]; otherwise cost_out may be nullptr.
void edge_costs(ngs_ctx *c, const SplatView &s, GraphDev &g, uint32_t pass, bool lex,
                float *cost_out);
// cost_slot from caller costs given in lexicographic edge order.
void costs_to_slots(ngs_ctx *c, GraphDev &g, const float *cost_lex);
// float-float arithmetic on host doubles (ngs_selftest_ff)
void ff_selftest(ngs_ctx *c, int op, const double *x, const double *y, int64_t n, double *out);

// ---------------------------------------------------------------- matching (k_match.cu)
// Greedy matching under (cost, canonical pair) capped to max_pairs.  Writes
// partner[v] (selected partner or -1) and returns the pair count (host).
int64_t select_pairs(ngs_ctx *c, const GraphDev &g, int64_t max_pairs, int32_t *partner);
// Locally-dominant rounds only: mate[] in c->b_mate, edge cost keys in
// c->b_candkey; returns the number of matched pairs.
int64_t match_rounds(ngs_ctx *c, const GraphDev &g);
// keys[v] = (cost bits << 32 | lo cid) at the lower-cid endpoint of each
// matched pair, UINT64_MAX elsewhere.
void pair_keys(ngs_ctx *c, const GraphDev &g, uint64_t *keys);
// partner[v] from mate[] with per-scene thresholds thr[sid[v]] (capped = 0: none).
void apply_cap(ngs_ctx *c, const GraphDev &g, const int32_t *sid, const uint64_t *thr,
               int capped, int32_t *partner);
// pairs_out (2*count) sorted by lo from partner[]; returns count.
int64_t partner_to_pairs(ngs_ctx *c, const int32_t *partner, const int32_t *cid, int64_t n,
                         int32_t *pairs_out);

// ---------------------------------------------------------------- merge (k_merge.cu)
// role[v]: >=0 partner (v is the lower-cid member, merged into row v),
// -2 removed, -1 kept.  Returns the new count; out receives the compacted
// rows.  If cid != nullptr, cid_out receives the updated canonical ids.
int64_t merge_compact(ngs_ctx *c, const SplatView &in, const int32_t *role, SplatView &out,
                      const int32_t *cid, int32_t *cid_out);
// pairs (lo,hi) -> role[] with validation; returns false on invalid pairs.
bool pairs_to_role(ngs_ctx *c, const int32_t *pairs, int64_t npairs, int64_t n, int32_t *role);
// partner[] (from select_pairs) -> role[] using canonical ids.
void partner_to_role(ngs_ctx *c, const int32_t *partner, const int32_t *cid, int64_t n,
                     int32_t *role);
// Opacity pre-filter keep flags (1/0) and the kept count (host).
int64_t prefilter_flags(ngs_ctx *c, const float *logit, int64_t n, double tau, int32_t *keep);
// Stable compaction of splat rows by keep flags (exclusive scan in pos).
void compact_rows(ngs_ctx *c, const SplatView &in, const int32_t *keep, const int32_t *pos,
                  SplatView &out);
// Scatter rows: out[dst[v]] = in[v].
void scatter_rows(ngs_ctx *c, const SplatView &in, const int32_t *dst, SplatView &out);
// Gather rows: out[v] = in[src[v]].
// Only the SH rows (sh) or only the other fields (!sh); F a multiple of 4, F <= 64.
void gather_rows_part(ngs_ctx *c, const SplatView &in, const uint32_t *src, SplatView &out, bool sh);
void gather_rows(ngs_ctx *c, const SplatView &in, const uint32_t *src, SplatView &out);

// Host-side common random numbers for pass `pass` (SplitMix64 + Box-Muller):
// z[3*S] normals and u[S] uniforms, rounded to float.
void host_mc_draws(uint64_t seed, uint32_t pass, int S, float *z, float *u);
