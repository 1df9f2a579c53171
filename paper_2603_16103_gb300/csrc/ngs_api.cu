// C ABI of the library (include/ngs.h): context, workspaces, instrumentation
// and the host orchestration of the simplification pass (Algorithm 1).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include <algorithm>
#include <utility>

#include "ngs_internal.h"

// ---------------------------------------------------------------- errors
static thread_local char g_err[512] = "";

void ngs_set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

extern "C" const char *ngs_last_error(void) { return g_err; }

#define API_BEGIN try {
#define API_END                                         \
    }                                                   \
    catch (const NgsError &e) {                         \
        return e.code;                                  \
    }                                                   \
    catch (...) {                                       \
        ngs_set_error("unexpected host exception");     \
        return NGS_ERR_CUDA;                            \
    }                                                   \
    return NGS_OK;

// ---------------------------------------------------------------- workspace
// One memory pool per device, private to the library.  Its release threshold
// is unlimited, so blocks freed when a buffer grows stay cached for the next
// request instead of going back to the driver at every synchronisation.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static cudaMemPool_t pool_of(int dev) {
    if (dev < 0 || dev >= 64) NGS_FAIL(NGS_ERR_CUDA, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        NGS_CHECK_CUDA(cudaMemPoolCreate(&p, &props));
        uint64_t thr = UINT64_MAX;
        NGS_CHECK_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr));
        g_pool[dev] = p;
    }
    return g_pool[dev];
}

void *ws_get(ngs_ctx *c, DevBuf &b, size_t bytes) {
    if (bytes <= b.bytes) return b.p;
    if (c->ws_fixed)
        NGS_FAIL(NGS_ERR_STATE, "fixed workspace: %zu bytes needed, %zu bound", bytes, b.bytes);
    if (b.p) {
        NGS_CHECK_CUDA(cudaFreeAsync(b.p, c->st));  // after the queued work that used it
        c->ws_bytes -= (int64_t)b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t want = bytes + bytes / 8 + 256;
    void *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, want, pool_of(c->device), c->st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        NGS_FAIL(NGS_ERR_OOM, "device allocation of %zu bytes failed: %s", want,
                 cudaGetErrorString(e));
    }
    b.p = p;
    b.bytes = want;
    c->ws_bytes += (int64_t)want;
    return p;
}

extern "C" int ngs_pool_usage(int device, int64_t *used_bytes, int64_t *reserved_bytes) {
    if (device < 0 || device >= 64 || !used_bytes || !reserved_bytes) {
        ngs_set_error("ngs_pool_usage: bad device index or NULL output");
        return NGS_ERR_INVALID_ARG;
    }
    cudaMemPool_t p;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        p = g_pool[device];
    }
    *used_bytes = *reserved_bytes = 0;
    if (!p) return NGS_OK;
    uint64_t u = 0, r = 0;
    cudaError_t e = cudaMemPoolGetAttribute(p, cudaMemPoolAttrUsedMemCurrent, &u);
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(p, cudaMemPoolAttrReservedMemCurrent, &r);
    if (e != cudaSuccess) {
        ngs_set_error("ngs_pool_usage: %s", cudaGetErrorString(e));
        return NGS_ERR_CUDA;
    }
    *used_bytes = (int64_t)u;
    *reserved_bytes = (int64_t)r;
    return NGS_OK;
}

static void ws_free(ngs_ctx *c, DevBuf &b) {
    if (b.p) cudaFreeAsync(b.p, c->st);
    c->ws_bytes -= (int64_t)b.bytes;
    b.p = nullptr;
    b.bytes = 0;
}

void sync_stream(ngs_ctx *c) {
    c->syncs++;
    NGS_CHECK_CUDA(cudaStreamSynchronize(c->st));
    if (c->h_pin && c->err_word == (volatile int32_t *)(c->h_pin + 8) && *c->err_word) {
        const int e = *c->err_word;
        *c->err_word = 0;
        NGS_FAIL(e, "a device-wide wait ran past ngs_tuning.wait_budget_cycles (the waiting blocks "
                    "completed the work without it)");
    }
}

// ---------------------------------------------------------------- profiling
int prof_slot(ngs_ctx *c, const char *name) {
    for (size_t i = 0; i < c->kstats.size(); i++)
        if (strcmp(c->kstats[i].name, name) == 0) return (int)i;
    c->kstats.push_back(KStat{name, 0, 0.0});
    return (int)c->kstats.size() - 1;
}

static cudaEvent_t ev_get(ngs_ctx *c) {
    if (!c->ev_free.empty()) {
        cudaEvent_t e = c->ev_free.back();
        c->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e;
    NGS_CHECK_CUDA(cudaEventCreate(&e));
    return e;
}

void prof_begin(ngs_ctx *c, int slot, cudaEvent_t *a) {
    (void)slot;
    *a = ev_get(c);
    NGS_CHECK_CUDA(cudaEventRecord(*a, c->st));
}

static void prof_resolve(ngs_ctx *c) {
    if (c->pending.empty()) return;
    NGS_CHECK_CUDA(cudaStreamSynchronize(c->st));
    for (auto &p : c->pending) {
        float ms = 0.f;
        NGS_CHECK_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
        c->kstats[p.stat].launches++;
        c->kstats[p.stat].ms += ms;
        c->ev_free.push_back(p.a);
        c->ev_free.push_back(p.b);
    }
    c->pending.clear();
}

void prof_end(ngs_ctx *c, int slot, cudaEvent_t a) {
    cudaEvent_t b = ev_get(c);
    NGS_CHECK_CUDA(cudaEventRecord(b, c->st));
    c->pending.push_back(PendingEv{slot, a, b});
    if (c->pending.size() > 4096) prof_resolve(c);
}

// ---------------------------------------------------------------- random numbers
// SplitMix64 (Steele, Lea & Flood, 2014): a Weyl sequence with increment
// 0x9E3779B97F4A7C15 passed through a 64-bit finaliser.  Pass p starts from
// seed XOR (p * 0xD1B54A32D192ED03).  Uniforms take the top 53 bits, (0, 1].
// Normals use the Box-Muller transform (Box & Muller, 1958) in FP64.
namespace {
struct SplitMix {
    uint64_t x;
    uint64_t next() {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t r = x;
        r ^= r >> 30;
        r *= 0xBF58476D1CE4E5B9ull;
        r ^= r >> 27;
        r *= 0x94D049BB133111EBull;
        r ^= r >> 31;
        return r;
    }
    double unit() { return (double)((next() >> 11) + 1) / 9007199254740992.0; }
};
}  // namespace

void host_mc_draws(uint64_t seed, uint32_t pass, int S, float *z, float *u) {
    SplitMix g{seed ^ ((uint64_t)pass * 0xD1B54A32D192ED03ull)};
    const double two_pi = 6.283185307179586476925286766559;
    for (int s = 0; s < S; s++) {
        double a = g.unit(), b = g.unit(), cc = g.unit(), dd = g.unit();
        double ra = sqrt(-2.0 * log(a)), rc = sqrt(-2.0 * log(cc));
        z[3 * s] = (float)(ra * cos(two_pi * b));
        z[3 * s + 1] = (float)(ra * sin(two_pi * b));
        z[3 * s + 2] = (float)(rc * cos(two_pi * dd));
        u[s] = (float)g.unit();
    }
}

// ---------------------------------------------------------------- params
extern "C" void ngs_default_params(ngs_params *p) {
    memset(p, 0, sizeof(*p));
    p->k = 16;
    p->mc_samples = 1;
    p->cost_mode = 0;
    p->tau = 0.005;
    p->lambda_geo = 1.0f;
    p->lambda_app = 1.0f;
    p->seed = 0;
    p->max_passes = 64;
    p->fp64_policy = 0;
    p->prefilter = 1;
    p->eig_floor = 1e-30;
    p->cost_tol = 3e-5;
    p->refresh_period = 1;
}

static int check_params(const ngs_params *p) {
    if (p->k < 1 || p->k > NGS_MAX_K) return 0;
    if (p->mc_samples < 1 || p->mc_samples > NGS_MAX_S) return 0;
    if (p->cost_mode < 0 || p->cost_mode > 3) return 0;
    if (!(p->tau >= 0.0 && p->tau < 1.0)) return 0;
    if (p->max_passes < 0 || p->max_passes > NGS_STATS_MAX_PASSES) return 0;
    if (p->fp64_policy < 0 || p->fp64_policy > 3) return 0;
    if (!(p->eig_floor > 0.0)) return 0;
    if (!(p->cost_tol >= 0.0 && p->cost_tol <= 1e-4)) return 0;
    if (p->refresh_period < 1 || p->refresh_period > NGS_STATS_MAX_PASSES) return 0;
    return 1;
}

extern "C" int ngs_create(ngs_ctx **out, const ngs_params *p, void *stream) {
    if (!out) {
        ngs_set_error("ngs_create: ctx pointer is NULL");
        return NGS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    ngs_params prm;
    if (p) prm = *p;
    else ngs_default_params(&prm);
    if (!check_params(&prm)) {
        ngs_set_error("ngs_create: parameter out of range");
        return NGS_ERR_INVALID_ARG;
    }
    ngs_ctx *c = new (std::nothrow) ngs_ctx();
    if (!c) return NGS_ERR_OOM;
    API_BEGIN
    c->prm = prm;
    c->st = (cudaStream_t)stream;
    NGS_CHECK_CUDA(cudaGetDevice(&c->device));
    NGS_CHECK_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    NGS_CHECK_CUDA(cudaMallocHost(&c->h_pin, 1 << 16));
    memset(c->h_pin, 0, 1 << 16);
    c->err_word = (volatile int32_t *)(c->h_pin + 8);
    *out = c;
    }
    catch (const NgsError &e) {
        delete c;
        return e.code;
    }
    return NGS_OK;
}

static void release_all(ngs_ctx *c) {
    DevBuf *bufs[] = {&c->b_pts, &c->b_codes, &c->b_codes2, &c->b_vals, &c->b_vals2, &c->b_hist,
                      &c->b_bbox, &c->b_frame, &c->b_nodes, &c->b_nbr, &c->b_deg, &c->b_cap,
                      &c->b_rstart, &c->b_adj, &c->b_adjeid, &c->b_fill, &c->b_upc, &c->b_eptr,
                      &c->b_elo, &c->b_ehi, &c->b_rec, &c->b_cost, &c->b_rng, &c->b_mate,
                      &c->b_cand, &c->b_candkey, &c->b_counts, &c->b_sel, &c->b_role, &c->b_keep,
                      &c->b_pos, &c->b_flag, &c->b_scan_part, &c->b_status, &c->b_misc, &c->b_cid,
                      &c->b_cid2, &c->b_cflag, &c->b_cscan, &c->b_pairs, &c->b_partner, &c->b_nbr2,
                      &c->b_lexrec, &c->b_sel2, &c->b_cflag2, &c->b_knnsc, &c->b_fp64list, &c->b_mstate, &c->b_offer, &c->b_order0,
                      &c->b_tiebits, &c->b_tielist, &c->b_revcost, &c->b_knnlong, &c->b_prevnbr, &c->b_rmap, &c->b_rsrc, &c->b_qflag,
                      &c->b_qlist};
    for (DevBuf *b : bufs) ws_free(c, *b);
    for (int k = 0; k < 5; k++) {
        ws_free(c, c->b_sA[k]);
        ws_free(c, c->b_sB[k]);
        ws_free(c, c->b_host_dev[k]);
        ws_free(c, c->b_sC[k]);
    }
    for (DevBuf &b : c->b_eng) ws_free(c, b);
    c->g_valid = false;
    cudaStreamSynchronize(c->st);
    // hand the now unused blocks back to the driver (blocks other contexts
    // still hold stay in the pool)
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (c->device >= 0 && c->device < 64) pool = g_pool[c->device];
    }
    if (pool) cudaMemPoolTrimTo(pool, 0);
}

extern "C" int ngs_release_workspace(ngs_ctx *c) {
    if (!c) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    NGS_CHECK_CUDA(cudaStreamSynchronize(c->st));
    release_all(c);
    API_END
}

extern "C" int ngs_destroy(ngs_ctx *c) {
    if (!c) return NGS_OK;
    cudaStreamSynchronize(c->st);
    release_all(c);
    for (auto &p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->ev_free) cudaEventDestroy(e);
    if (c->h_pin) cudaFreeHost(c->h_pin);
    if (c->cap_st) cudaStreamDestroy(c->cap_st);
    if (c->up_st) {
        cudaStreamSynchronize(c->up_st);
        cudaStreamDestroy(c->up_st);
        cudaEventDestroy(c->up_ev);
        cudaEventDestroy(c->up_first);
        cudaEventDestroy(c->up_rest);
    }
    delete c;
    return NGS_OK;
}

extern "C" int ngs_set_params(ngs_ctx *c, const ngs_params *p) {
    if (!c || !p || !check_params(p)) {
        ngs_set_error("ngs_set_params: invalid argument");
        return NGS_ERR_INVALID_ARG;
    }
    c->prm = *p;
    c->g_valid = false;
    return NGS_OK;
}

// ---------------------------------------------------------------- helpers
static void check_splats(const ngs_splats *s, const char *fn) {
    if (!s) NGS_FAIL(NGS_ERR_INVALID_ARG, "%s: splats is NULL", fn);
    if (s->n < 0 || s->n > s->cap || s->n > NGS_MAX_N)
        NGS_FAIL(NGS_ERR_INVALID_ARG, "%s: bad n=%lld cap=%lld (max %lld)", fn, (long long)s->n,
                 (long long)s->cap, (long long)NGS_MAX_N);
    if (s->sh_dim < 1 || s->sh_dim > 64) NGS_FAIL(NGS_ERR_INVALID_ARG, "%s: sh_dim out of range", fn);
    if (s->n > 0 && (!s->xyz || !s->log_scale || !s->rot || !s->opacity_logit || !s->sh))
        NGS_FAIL(NGS_ERR_INVALID_ARG, "%s: NULL array", fn);
    if (((s->sh_dim & 3) == 0 && ((uintptr_t)s->sh & 15)) || ((uintptr_t)s->rot & 15))
        NGS_FAIL(NGS_ERR_INVALID_ARG, "%s: rot (and sh when sh_dim %% 4 == 0) must be 16-byte aligned",
                 fn);
}

static SplatView view_of(const ngs_splats *s) {
    return SplatView{s->xyz, s->log_scale, s->rot, s->opacity_logit, s->sh, s->n, s->sh_dim};
}

static SplatView scratch_view(ngs_ctx *c, DevBuf *b, int64_t n, int F) {
    SplatView v;
    v.xyz = ws<float>(c, b[0], 3 * n);
    v.ls = ws<float>(c, b[1], 3 * n);
    v.rot = ws<float>(c, b[2], 4 * n);
    v.logit = ws<float>(c, b[3], n);
    v.sh = ws<float>(c, b[4], (int64_t)F * n);
    v.n = n;
    v.F = F;
    (void)c;
    return v;
}

static void copy_rows_d2d(ngs_ctx *c, const SplatView &src, SplatView &dst, int64_t n) {
    if (n <= 0) return;
    const int F = src.F;
    NGS_CHECK_CUDA(cudaMemcpyAsync(dst.xyz, src.xyz, 12 * n, cudaMemcpyDeviceToDevice, c->st));
    NGS_CHECK_CUDA(cudaMemcpyAsync(dst.ls, src.ls, 12 * n, cudaMemcpyDeviceToDevice, c->st));
    NGS_CHECK_CUDA(cudaMemcpyAsync(dst.rot, src.rot, 16 * n, cudaMemcpyDeviceToDevice, c->st));
    NGS_CHECK_CUDA(cudaMemcpyAsync(dst.logit, src.logit, 4 * n, cudaMemcpyDeviceToDevice, c->st));
    NGS_CHECK_CUDA(cudaMemcpyAsync(dst.sh, src.sh, 4 * (size_t)F * n, cudaMemcpyDeviceToDevice, c->st));
}


static void check_finite_frame(ngs_ctx *c, const float *frame) {
    get_small(c, c->h_pin + 4, frame + 4, 4);
    sync_stream(c);
    uint32_t bad = *(uint32_t *)(c->h_pin + 4);
    if (bad) NGS_FAIL(NGS_ERR_INVALID_ARG, "%u non-finite centre coordinates", bad);
}

// ---------------------------------------------------------------- step by step
extern "C" int ngs_prefilter(ngs_ctx *c, ngs_splats *s) {
    if (!c) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    check_splats(s, "ngs_prefilter");
    const int64_t n = s->n;
    if (n <= 0) return NGS_OK;
    int32_t *keep = ws<int32_t>(c, c->b_role, n + 1);
    int64_t kept = prefilter_flags(c, s->opacity_logit, n, c->prm.tau, keep);
    if (kept < n) {
        SplatView in = view_of(s);
        SplatView tmp = scratch_view(c, c->b_sB, n, s->sh_dim);
        compact_rows(c, in, keep, (const int32_t *)c->b_pos.p, tmp);
        copy_rows_d2d(c, tmp, in, kept);
        sync_stream(c);
    }
    s->n = kept;
    c->g_valid = false;
    API_END
}

// canonical-mode graph of `s` into c->g
static void graph_canonical(ngs_ctx *c, const ngs_splats *s) {
    const int64_t n = s->n;
    GraphDev &g = c->g;
    g = GraphDev{};
    check_slots(n, c->prm.k, "ngs_build_graph");
    g.n = n;
    g.k_eff = n >= 2 ? k_eff_of(n, c->prm.k) : 0;
    g.cid = nullptr;
    if (n >= 2) {
        float *frame = ws<float>(c, c->b_frame, 8);
        morton_frame(c, s->xyz, n, frame);
        check_finite_frame(c, frame);
        uint32_t *keys = ws<uint32_t>(c, c->b_codes, n), *vals = ws<uint32_t>(c, c->b_vals, n);
        uint32_t *k2 = ws<uint32_t>(c, c->b_codes2, n), *v2 = ws<uint32_t>(c, c->b_vals2, n);
        morton_keys(c, s->xyz, n, frame, keys, vals);
        radix_sort_u32(c, keys, vals, k2, v2, n, 30);
        float4 *pts = ws<float4>(c, c->b_pts, n);
        gather_points(c, s->xyz, nullptr, vals, n, pts);
        int32_t *nbr = ws<int32_t>(c, c->b_nbr, n * g.k_eff);
        const int64_t sn = n;
        knn_search(c, KnnInput{pts, keys, vals, nullptr, frame, &sn, 1, n, 1, nullptr}, g.k_eff, nbr);
        build_edges(c, nbr, g);
        build_lex_view(c, g);
    }
    c->g_valid = true;
    c->g_n = n;
    c->g_k = g.k_eff;
    c->g_edges = g.n_edges;
    c->g_xyz = s->xyz;
}

// canonical-mode graph of `s`, the result of merging `pairs` into a set of
// n_old splats whose lists were prev_nbr (Sec. 3.4 local refresh)
static int64_t graph_canonical_refresh(ngs_ctx *c, const ngs_splats *s, const int32_t *prev_nbr,
                                       int64_t n_old, int k_old, const int32_t *pairs,
                                       int64_t np) {
    const int64_t n = s->n;
    if (n_old < 0 || n_old > NGS_MAX_N || np < 0 || n != n_old - np)
        NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_build_graph_refresh: n=%lld is not n_old=%lld - n_pairs=%lld",
                 (long long)n, (long long)n_old, (long long)np);
    if (n_old >= 2 && (k_old < 1 || k_old > NGS_MAX_K || !prev_nbr))
        NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_build_graph_refresh: bad previous lists (k_old=%d)", k_old);
    if (np > 0 && !pairs) NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_build_graph_refresh: pairs is NULL");
    GraphDev &g = c->g;
    g = GraphDev{};
    c->g_valid = false;
    check_slots(n, c->prm.k, "ngs_build_graph_refresh");
    g.n = n;
    g.k_eff = n >= 2 ? k_eff_of(n, c->prm.k) : 0;
    g.cid = nullptr;
    int64_t nq = 0;
    if (n >= 2) {
        int32_t *prev = ws<int32_t>(c, c->b_prevnbr, n_old * k_old);
        NGS_CHECK_CUDA(cudaMemcpyAsync(prev, prev_nbr, sizeof(int32_t) * n_old * k_old,
                                       cudaMemcpyDeviceToDevice, c->st));
        if (!ids_in_range(c, prev, n_old * k_old, n_old))
            NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_build_graph_refresh: a list entry is outside [0, %lld)",
                     (long long)n_old);
        int32_t *role = ws<int32_t>(c, c->b_role, n_old);
        if (!pairs_to_role(c, pairs, np, n_old, role))
            NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_build_graph_refresh: pairs out of range, unordered or not disjoint");
        int32_t *map_old = ws<int32_t>(c, c->b_rmap, n_old), *src = ws<int32_t>(c, c->b_rsrc, n);
        refresh_map(c, n_old, role, map_old, src);
        float *frame = ws<float>(c, c->b_frame, 8);
        morton_frame(c, s->xyz, n, frame);
        check_finite_frame(c, frame);
        uint32_t *keys = ws<uint32_t>(c, c->b_codes, n), *vals = ws<uint32_t>(c, c->b_vals, n);
        uint32_t *k2 = ws<uint32_t>(c, c->b_codes2, n), *v2 = ws<uint32_t>(c, c->b_vals2, n);
        morton_keys(c, s->xyz, n, frame, keys, vals);
        radix_sort_u32(c, keys, vals, k2, v2, n, 30);
        float4 *pts = ws<float4>(c, c->b_pts, n);
        gather_points(c, s->xyz, nullptr, vals, n, pts);
        int32_t *nbr = ws<int32_t>(c, c->b_nbr, n * g.k_eff);
        int32_t *qlist = ws<int32_t>(c, c->b_qlist, n + 1);
        nq = refresh_rows(c, n, g.k_eff, k_old, n_old, src, prev, map_old, s->xyz, nullptr, vals,
                          nbr, qlist);
        const int64_t sn = n;
        knn_search(c, KnnInput{pts, keys, vals, nullptr, frame, &sn, 1, n, 1, nullptr, qlist, nq},
                   g.k_eff, nbr);
        build_edges(c, nbr, g);
        build_lex_view(c, g);
    }
    c->g_valid = true;
    c->g_n = n;
    c->g_k = g.k_eff;
    c->g_edges = g.n_edges;
    c->g_xyz = s->xyz;
    return nq;
}

extern "C" int ngs_build_graph_refresh(ngs_ctx *c, const ngs_splats *s, const int32_t *prev_nbr,
                                       int64_t n_old, int32_t k_old, const int32_t *pairs,
                                       int64_t n_pairs, ngs_graph *out, int64_t *n_requeried) {
    if (!c || !out) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    check_splats(s, "ngs_build_graph_refresh");
    const int64_t nq = graph_canonical_refresh(c, s, prev_nbr, n_old, k_old, pairs, n_pairs);
    if (n_requeried) *n_requeried = nq;
    out->n = s->n;
    out->k_eff = c->g.k_eff;
    out->n_edges = c->g.n_edges;
    out->nbr = (const int32_t *)c->b_nbr.p;
    out->edge_lo = c->g.n_edges ? c->g.elo : nullptr;
    out->edge_hi = c->g.n_edges ? c->g.ehi : nullptr;
    API_END
}

extern "C" int ngs_build_graph(ngs_ctx *c, const ngs_splats *s, ngs_graph *out) {
    if (!c || !out) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    check_splats(s, "ngs_build_graph");
    graph_canonical(c, s);
    out->n = s->n;
    out->k_eff = c->g.k_eff;
    out->n_edges = c->g.n_edges;
    out->nbr = (const int32_t *)c->b_nbr.p;
    out->edge_lo = c->g.n_edges ? c->g.elo : nullptr;
    out->edge_hi = c->g.n_edges ? c->g.ehi : nullptr;
    API_END
}

static void check_graph(ngs_ctx *c, const ngs_graph *g, const char *fn) {
    if (!g) NGS_FAIL(NGS_ERR_INVALID_ARG, "%s: graph is NULL", fn);
    if (!c->g_valid || g->n != c->g_n || g->n_edges != c->g_edges)
        NGS_FAIL(NGS_ERR_STATE, "%s: graph is not the ctx's current graph", fn);
}

extern "C" int ngs_edge_costs(ngs_ctx *c, const ngs_splats *s, const ngs_graph *g, uint32_t pass,
                              float *cost) {
    if (!c) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    check_splats(s, "ngs_edge_costs");
    check_graph(c, g, "ngs_edge_costs");
    if (s->n != c->g_n || s->xyz != c->g_xyz)
        NGS_FAIL(NGS_ERR_STATE, "ngs_edge_costs: splats differ from the graph's");
    if (g->n_edges > 0 && !cost) NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_edge_costs: cost is NULL");
    c->fp64_edges = 0;
    edge_costs(c, view_of(s), c->g, pass, true, cost);
    API_END
}

extern "C" int ngs_select_pairs(ngs_ctx *c, const ngs_graph *g, const float *cost,
                                int64_t max_pairs, int32_t *pairs_out, int64_t *n_pairs) {
    if (!c || !n_pairs) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    check_graph(c, g, "ngs_select_pairs");
    *n_pairs = 0;
    if (max_pairs < 0) NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_select_pairs: max_pairs < 0");
    if (g->n_edges > 0 && (!cost || (max_pairs > 0 && !pairs_out)))
        NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_select_pairs: NULL array");
    const int64_t n = c->g.n;
    if (n <= 1 || g->n_edges == 0 || max_pairs == 0) return NGS_OK;
    int32_t *partner = ws<int32_t>(c, c->b_partner, n);
    costs_to_slots(c, c->g, cost);
    select_pairs(c, c->g, max_pairs, partner);
    *n_pairs = partner_to_pairs(c, partner, nullptr, n, pairs_out);
    API_END
}

extern "C" int ngs_merge_compact(ngs_ctx *c, ngs_splats *s, const int32_t *pairs, int64_t n_pairs) {
    if (!c) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    check_splats(s, "ngs_merge_compact");
    const int64_t n = s->n;
    if (n_pairs < 0 || n_pairs > n / 2 || (n_pairs > 0 && !pairs))
        NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_merge_compact: bad pair list");
    if (n_pairs == 0) return NGS_OK;
    int32_t *role = ws<int32_t>(c, c->b_role, n);
    if (!pairs_to_role(c, pairs, n_pairs, n, role))
        NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_merge_compact: pairs out of range, unordered or not disjoint");
    SplatView in = view_of(s);
    SplatView tmp = scratch_view(c, c->b_sB, n, s->sh_dim);
    int64_t nout = merge_compact(c, in, role, tmp, nullptr, nullptr);
    copy_rows_d2d(c, tmp, in, nout);
    sync_stream(c);
    s->n = nout;
    c->g_valid = false;
    API_END
}

// ---------------------------------------------------------------- end to end
extern "C" int ngs_simplify(ngs_ctx *c, ngs_splats *s, int64_t target, ngs_stats *st) {
    if (!c) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    check_splats(s, "ngs_simplify");
    if (target < 1) NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_simplify: target_count < 1");
    engine_simplify(c, s, &target, 1, st);
    API_END
}

extern "C" int ngs_batch_simplify(ngs_ctx *c, ngs_splats *scenes, const int64_t *targets,
                                  int32_t nscenes, ngs_stats *st) {
    if (!c) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    if (nscenes < 0 || nscenes > NGS_MAX_SCENES)
        NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_batch_simplify: nscenes=%d outside [0, %d]",
                 (int)nscenes, NGS_MAX_SCENES);
    if (nscenes > 0 && (!scenes || !targets))
        NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_batch_simplify: NULL scenes or targets");
    int64_t total = 0;
    for (int s = 0; s < nscenes; s++) {
        check_splats(&scenes[s], "ngs_batch_simplify");
        if (scenes[s].sh_dim != scenes[0].sh_dim)
            NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_batch_simplify: scene %d sh_dim %d != %d", s,
                     scenes[s].sh_dim, scenes[0].sh_dim);
        if (targets[s] < 1)
            NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_batch_simplify: scene %d target_count < 1", s);
        total += scenes[s].n;
    }
    if (total > NGS_MAX_N)
        NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_batch_simplify: %lld splats in total, above %lld",
                 (long long)total, (long long)NGS_MAX_N);
    // scenes whose target leaves room for a full neighbour list share one
    // engine run; the others (target <= k) run alone, one after another
    std::vector<ngs_splats> big;
    std::vector<int64_t> big_t;
    std::vector<int> big_idx;
    ngs_stats acc, one;
    memset(&acc, 0, sizeof(acc));
    const int ke = k_eff_of(INT64_MAX, c->prm.k);
    const int64_t l0 = c->launches, s0 = c->syncs;
    auto add = [&](const ngs_stats &x) {
        acc.n_input += x.n_input;
        acc.n_filtered += x.n_filtered;
        acc.n_output += x.n_output;
        for (int p = 0; p < NGS_STATS_MAX_PASSES; p++) {
            acc.pass_n[p] += x.pass_n[p];
            acc.pass_edges[p] += x.pass_edges[p];
            acc.pass_pairs[p] += x.pass_pairs[p];
        }
        acc.passes = acc.passes > x.passes ? acc.passes : x.passes;
        acc.matching_rounds += x.matching_rounds;
        acc.fp64_cost_edges += x.fp64_cost_edges;
        acc.near_tie_slots += x.near_tie_slots;
        acc.requeried_rows += x.requeried_rows;
        acc.eig_floor_hits += x.eig_floor_hits;
    };
    for (int s = 0; s < nscenes; s++) {
        if (targets[s] > ke) {
            big.push_back(scenes[s]);
            big_t.push_back(targets[s]);
            big_idx.push_back(s);
        } else {
            engine_simplify(c, &scenes[s], &targets[s], 1, &one);
            add(one);
        }
    }
    if (!big.empty()) {
        engine_simplify(c, big.data(), big_t.data(), (int)big.size(), &one);
        add(one);
        for (size_t i = 0; i < big.size(); i++) scenes[big_idx[i]].n = big[i].n;
    }
    acc.gpu_launches = c->launches - l0;
    acc.host_syncs = c->syncs - s0;
    if (st) *st = acc;
    API_END
}

extern "C" int ngs_simplify_host(ngs_ctx *c, ngs_splats *h, int64_t target, ngs_stats *st) {
    if (!c) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    check_splats(h, "ngs_simplify_host");
    if (target < 1) NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_simplify_host: target_count < 1");
    const int64_t n = h->n;
    const int F = h->sh_dim;
    ngs_splats d = *h;
    d.xyz = ws<float>(c, c->b_host_dev[0], 3 * n);
    d.log_scale = ws<float>(c, c->b_host_dev[1], 3 * n);
    d.rot = ws<float>(c, c->b_host_dev[2], 4 * n);
    d.opacity_logit = ws<float>(c, c->b_host_dev[3], n);
    d.sh = ws<float>(c, c->b_host_dev[4], (int64_t)F * n);
    d.cap = n;
    const size_t sz[5] = {12, 12, 16, 4, 4 * (size_t)F};
    float *hp[5] = {h->xyz, h->log_scale, h->rot, h->opacity_logit, h->sh};
    float *dp[5] = {d.xyz, d.log_scale, d.rot, d.opacity_logit, d.sh};
    // Uploads in the order the engine needs them, so that the link is not
    // shared while the first kernels wait: opacities and centres on the ctx
    // stream (pre-filter, Morton frame and keys), then on a second stream the
    // log-scales and rotations (first needed by the row gather after the sort)
    // and the SH array, most of the bytes (first needed by the edge costs).
    // The engine waits for each only where it first reads it.
    if (!c->up_st) {
        NGS_CHECK_CUDA(cudaStreamCreateWithFlags(&c->up_st, cudaStreamNonBlocking));
        NGS_CHECK_CUDA(cudaEventCreateWithFlags(&c->up_ev, cudaEventDisableTiming));
        NGS_CHECK_CUDA(cudaEventCreateWithFlags(&c->up_first, cudaEventDisableTiming));
        NGS_CHECK_CUDA(cudaEventCreateWithFlags(&c->up_rest, cudaEventDisableTiming));
    }
    NGS_CHECK_CUDA(cudaMemcpyAsync(dp[3], hp[3], sz[3] * n, cudaMemcpyHostToDevice, c->st));
    NGS_CHECK_CUDA(cudaMemcpyAsync(dp[0], hp[0], sz[0] * n, cudaMemcpyHostToDevice, c->st));
    NGS_CHECK_CUDA(cudaEventRecord(c->up_first, c->st));  // also: the staging buffers exist
    NGS_CHECK_CUDA(cudaStreamWaitEvent(c->up_st, c->up_first, 0));
    NGS_CHECK_CUDA(cudaMemcpyAsync(dp[1], hp[1], sz[1] * n, cudaMemcpyHostToDevice, c->up_st));
    NGS_CHECK_CUDA(cudaMemcpyAsync(dp[2], hp[2], sz[2] * n, cudaMemcpyHostToDevice, c->up_st));
    NGS_CHECK_CUDA(cudaEventRecord(c->up_rest, c->up_st));
    NGS_CHECK_CUDA(cudaMemcpyAsync(dp[4], hp[4], sz[4] * n, cudaMemcpyHostToDevice, c->up_st));
    NGS_CHECK_CUDA(cudaEventRecord(c->up_ev, c->up_st));
    c->rest_wait = c->up_rest;
    c->sh_wait = c->up_ev;
    try {
        engine_simplify(c, &d, &target, 1, st);
    } catch (...) {
        c->sh_wait = c->rest_wait = nullptr;
        cudaStreamWaitEvent(c->st, c->up_ev, 0);  // the staging buffers stay busy until then
        throw;
    }
    c->sh_wait = c->rest_wait = nullptr;
    NGS_CHECK_CUDA(cudaStreamWaitEvent(c->st, c->up_ev, 0));
    for (int k = 0; k < 5; k++)
        NGS_CHECK_CUDA(cudaMemcpyAsync(hp[k], dp[k], sz[k] * d.n, cudaMemcpyDeviceToHost, c->st));
    sync_stream(c);
    h->n = d.n;
    API_END
}

extern "C" int ngs_selftest_ff(ngs_ctx *c, int32_t op, const double *x, const double *y,
                               int64_t n, double *out) {
    if (!c) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    if (op < 0 || op > 7) NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_selftest_ff: op %d out of range", op);
    if (n < 0) NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_selftest_ff: n < 0");
    if (n > 0 && (!x || !out || ((op == 4 || op == 6 || op == 7) && !y)))
        NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_selftest_ff: null pointer");
    ff_selftest(c, op, x, (op == 4 || op == 6 || op == 7) ? y : nullptr, n, out);
    API_END
}

// ---------------------------------------------------------------- instrumentation API
extern "C" int ngs_profile_enable(ngs_ctx *c, int enable) {
    if (!c) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    if (!enable) prof_resolve(c);
    c->prof = enable != 0;
    API_END
}

extern "C" int ngs_profile_count(ngs_ctx *c) {
    if (!c) return 0;
    try {
        prof_resolve(c);
    } catch (...) {
    }
    return (int)c->kstats.size();
}

extern "C" int ngs_profile_get(ngs_ctx *c, int i, const char **name, int64_t *launches, double *ms) {
    if (!c) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    prof_resolve(c);
    if (i < 0 || i >= (int)c->kstats.size()) NGS_FAIL(NGS_ERR_INVALID_ARG, "profile index");
    if (name) *name = c->kstats[i].name;
    if (launches) *launches = c->kstats[i].launches;
    if (ms) *ms = c->kstats[i].ms;
    API_END
}

extern "C" int ngs_profile_reset(ngs_ctx *c) {
    if (!c) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    prof_resolve(c);
    c->kstats.clear();
    API_END
}

extern "C" int64_t ngs_launch_count(ngs_ctx *c) { return c ? c->launches : 0; }

extern "C" int64_t ngs_workspace_bytes(ngs_ctx *c) { return c ? c->ws_bytes : 0; }

extern "C" void ngs_default_tuning(ngs_tuning *t) {
    if (!t) return;
    const Tuning d;
    t->knn_block_min = d.knn_block_min;
    t->cells_per_point = d.cells_per_point;
    t->cost_blocks_per_sm = d.cost_blocks_per_sm;
    t->match_method = d.match_method;
    t->match_max_steps = d.match_max_steps;
    t->scan_method = d.scan_method;
    t->wait_budget_cycles = d.wait_budget_cycles;
    t->wait_test_tile = d.wait_test_tile;
}

extern "C" int ngs_get_tuning(ngs_ctx *c, ngs_tuning *t) {
    if (!c || !t) return NGS_ERR_INVALID_ARG;
    t->knn_block_min = c->tune.knn_block_min;
    t->cells_per_point = c->tune.cells_per_point;
    t->cost_blocks_per_sm = c->tune.cost_blocks_per_sm;
    t->match_method = c->tune.match_method;
    t->match_max_steps = c->tune.match_max_steps;
    t->scan_method = c->tune.scan_method;
    t->wait_budget_cycles = c->tune.wait_budget_cycles;
    t->wait_test_tile = c->tune.wait_test_tile;
    return NGS_OK;
}

extern "C" int ngs_set_tuning(ngs_ctx *c, const ngs_tuning *t) {
    if (!c || !t) return NGS_ERR_INVALID_ARG;
    const int cpp = t->cells_per_point;
    if (t->knn_block_min < 16 || t->knn_block_min > 1024 ||
        !(cpp == 1 || cpp == 2 || cpp == 4 || cpp == 8) || t->cost_blocks_per_sm < 1 ||
        t->cost_blocks_per_sm > 64 || t->match_method < 0 || t->match_method > 2 ||
        t->match_max_steps < 1 || t->match_max_steps > (1 << 30) || t->wait_budget_cycles < 1 ||
        t->wait_test_tile < -1 || t->scan_method < 0 || t->scan_method > 1) {
        ngs_set_error("ngs_set_tuning: field out of range");
        return NGS_ERR_INVALID_ARG;
    }
    c->tune.knn_block_min = t->knn_block_min;
    c->tune.cells_per_point = cpp;
    c->tune.cost_blocks_per_sm = t->cost_blocks_per_sm;
    c->tune.match_method = t->match_method;
    c->tune.match_max_steps = t->match_max_steps;
    c->tune.scan_method = t->scan_method;
    c->tune.wait_budget_cycles = t->wait_budget_cycles;
    c->tune.wait_test_tile = t->wait_test_tile;
    return NGS_OK;
}

extern "C" int ngs_autotune(ngs_ctx *c, const ngs_splats *s, ngs_tuning *best, double *ms_best) {
    if (!c) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    check_splats(s, "ngs_autotune");
    if (s->n < 2) NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_autotune: the sample needs at least 2 splats");
    cudaEvent_t e0, e1;
    NGS_CHECK_CUDA(cudaEventCreate(&e0));
    NGS_CHECK_CUDA(cudaEventCreate(&e1));
    auto timed = [&](auto &&fn) {
        float best_ms = 1e30f;
        for (int rep = 0; rep < 2; rep++) {
            NGS_CHECK_CUDA(cudaEventRecord(e0, c->st));
            fn();
            NGS_CHECK_CUDA(cudaEventRecord(e1, c->st));
            NGS_CHECK_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            NGS_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            best_ms = ms < best_ms ? ms : best_ms;
        }
        return best_ms;
    };
    try {
        // stage 1: the kNN graph (Morton sort, cell table, search, edges)
        const int bms[3] = {48, 64, 96}, cpps[3] = {2, 4, 8};
        float t_graph = 1e30f;
        Tuning tb = c->tune;
        for (int bm : bms)
            for (int cpp : cpps) {
                c->tune.knn_block_min = bm;
                c->tune.cells_per_point = cpp;
                // the sample and its first half and quarter: later passes run on
                // fewer splats, where the cell-table level (and so the best
                // density) differs
                float t = timed([&] { graph_canonical(c, s); });
                for (int64_t part = s->n / 2; part >= 4096 && part >= s->n / 4; part /= 2) {
                    ngs_splats sub = *s;
                    sub.n = part;
                    t += timed([&] { graph_canonical(c, &sub); });
                }
                if (t < t_graph) {
                    t_graph = t;
                    tb.knn_block_min = bm;
                    tb.cells_per_point = cpp;
                }
            }
        c->tune.knn_block_min = tb.knn_block_min;
        c->tune.cells_per_point = tb.cells_per_point;
        graph_canonical(c, s);
        // stage 2: the edge costs on that graph
        const int cbs[3] = {4, 8, 12};
        float t_cost = 1e30f;
        for (int cb : cbs) {
            c->tune.cost_blocks_per_sm = cb;
            const float t = timed([&] { edge_costs(c, view_of(s), c->g, 0, false, nullptr); });
            if (t < t_cost) {
                t_cost = t;
                tb.cost_blocks_per_sm = cb;
            }
        }
        c->tune = tb;
        c->g_valid = false;
        if (best) ngs_get_tuning(c, best);
        if (ms_best) *ms_best = (double)t_graph + (double)t_cost;
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    API_END
}

extern "C" int ngs_set_stream(ngs_ctx *c, void *stream) {
    if (!c) return NGS_ERR_INVALID_ARG;
    API_BEGIN
    if ((cudaStream_t)stream != c->st) {
        NGS_CHECK_CUDA(cudaStreamSynchronize(c->st));
        c->st = (cudaStream_t)stream;
    }
    API_END
}
