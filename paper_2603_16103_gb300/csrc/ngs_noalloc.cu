// kNN search for callers that cannot allocate device memory.
//
// Some hosts own all device memory themselves (a renderer or engine that
// reserves its memory budget up front, a plugin that may only use buffers
// handed to it) or run where cudaMalloc is not acceptable (it may
// synchronise the device, which a real-time frame loop cannot afford).
// ngs_knn_noalloc serves them: the caller passes the centres and the output
// table, and every temporary of the search lives in one file-scope device
// array of fixed size, so the call performs no device allocation at all.
//
// The array is shared by every call in the process on a given device and
// keeps the previous call's contents; the search rewrites or clears all of
// it that it reads (the cell counts are cleared with a memset on the
// caller's stream).  Calls that overlap on the GPU (different streams, or
// different host threads on one device) race on it and must be serialised
// by the caller.  The array's device address is looked up with
// cudaGetSymbolAddress on the first call on each device (with that device
// current); that first call should therefore come before any stream capture.
// The address is looked up again when the device's context has changed since
// (after cudaDeviceReset the array is loaded anew, at another address).
#include <cuda.h>

#include <mutex>

#include "ngs_internal.h"

namespace {

constexpr int64_t kMaxN = NGS_NOALLOC_MAX_N;
constexpr int64_t kTiles = (kMaxN + 2047) / 2048;        // radix-sort tiles
constexpr int kTableLevel = 6;                            // 8^6 >= 4 * kMaxN
constexpr int64_t kCells = (int64_t)1 << (3 * kTableLevel);
static_assert(kCells >= 4 * kMaxN, "cell table too small for the maximum n");

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// slices of the scratch array (bytes)
constexpr size_t kAcc = align256(8 * 4);
constexpr size_t kFrame = align256(8 * 4);
constexpr size_t kKeys = align256(4 * kMaxN);
constexpr size_t kHist = align256(4 * (256 * kTiles + 256 + 1));  // tile counts, digit totals
constexpr size_t kPart = align256(4 * (kCells / 2048 + 2));
constexpr size_t kPts = align256(16 * kMaxN);
constexpr size_t kTable = align256(4 * (kCells + 2));
constexpr size_t kLong = align256(16 * (kMaxN + 3 + kCells / 16384));  // chunks of empty cells
constexpr size_t kKnnSc = align256(16 * 2 + 256);
constexpr size_t kScratchBytes = kAcc + kFrame + 4 * kKeys + kHist + kPart + kPts + kTable + kKnnSc + kLong;

__device__ __align__(256) unsigned char g_knn_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_dev[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

// The current driver context, fetched through the runtime's driver entry
// point (no link-time dependency on libcuda); nullptr if unavailable.
CUcontext current_context() {
    using CtxGetCurrent = CUresult (*)(CUcontext *);
    static CtxGetCurrent fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return (CtxGetCurrent)f;
    }();
    CUcontext cx = nullptr;
    if (fn && fn(&cx) != CUDA_SUCCESS) cx = nullptr;
    return cx;
}

void bind(DevBuf &b, unsigned char *&cur, size_t bytes) {
    b.p = cur;
    b.bytes = bytes;
    cur += bytes;
}

}  // namespace

extern "C" int ngs_knn_noalloc(const float *xyz, int64_t n, int32_t k, int32_t *nbr,
                               void *stream) {
    if (n < 0 || n > kMaxN) {
        ngs_set_error("ngs_knn_noalloc: n=%lld outside [0, %lld]", (long long)n,
                      (long long)kMaxN);
        return NGS_ERR_INVALID_ARG;
    }
    if (k < 1 || k > NGS_MAX_K) {
        ngs_set_error("ngs_knn_noalloc: k=%d outside [1, %d]", (int)k, NGS_MAX_K);
        return NGS_ERR_INVALID_ARG;
    }
    if (n <= 1) return NGS_OK;  // k_eff = 0: nothing to write
    if (!xyz || !nbr) {
        ngs_set_error("ngs_knn_noalloc: NULL array");
        return NGS_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        ngs_set_error("ngs_knn_noalloc: no usable current device (%s)", cudaGetErrorString(e));
        return NGS_ERR_CUDA;
    }
    // the table level must fit the fixed cell-table slice
    if (knn_table_level(n, Tuning{}.cells_per_point) > kTableLevel) {
        ngs_set_error("ngs_knn_noalloc: cell table for n=%lld exceeds the fixed slice",
                      (long long)n);
        return NGS_ERR_INVALID_ARG;
    }
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        // set-up once per device (and again if the device's context changed)
        const CUcontext cx = current_context();
        if (!g_scratch_dev[dev] || cx != g_scratch_ctx[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_knn_scratch);
            if (e != cudaSuccess || !p) {
                ngs_set_error("ngs_knn_noalloc: cudaGetSymbolAddress failed: %s",
                              cudaGetErrorString(e));
                return NGS_ERR_CUDA;
            }
            g_scratch_dev[dev] = p;
            g_scratch_ctx[dev] = current_context();
        }
        base = g_scratch_dev[dev];
    }
    ngs_ctx c;  // stack context: no workspace ever grows beyond the bound slices
    c.ws_fixed = true;  // a slice too small fails the call instead of allocating
    ngs_default_params(&c.prm);
    c.prm.k = k;
    c.st = (cudaStream_t)stream;
    c.device = dev;
    e = cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        ngs_set_error("ngs_knn_noalloc: %s", cudaGetErrorString(e));
        return NGS_ERR_CUDA;
    }
    unsigned char *cur = (unsigned char *)base;
    bind(c.b_bbox, cur, kAcc);
    bind(c.b_frame, cur, kFrame);
    bind(c.b_codes, cur, kKeys);
    bind(c.b_vals, cur, kKeys);
    bind(c.b_codes2, cur, kKeys);
    bind(c.b_vals2, cur, kKeys);
    bind(c.b_hist, cur, kHist);
    bind(c.b_scan_part, cur, kPart);
    bind(c.b_pts, cur, kPts);
    bind(c.b_nodes, cur, kTable);
    bind(c.b_knnsc, cur, kKnnSc);
    bind(c.b_knnlong, cur, kLong);
    int rc = NGS_OK;
    try {
        const int ke = (int)(k < n - 1 ? k : n - 1);
        float *frame = (float *)c.b_frame.p;
        morton_frame(&c, xyz, n, frame);
        uint32_t bad = 0;
        NGS_CHECK_CUDA(cudaMemcpyAsync(&bad, frame + 4, 4, cudaMemcpyDeviceToHost, c.st));
        NGS_CHECK_CUDA(cudaStreamSynchronize(c.st));
        if (bad) NGS_FAIL(NGS_ERR_INVALID_ARG, "ngs_knn_noalloc: %u non-finite coordinates", bad);
        uint32_t *keys = (uint32_t *)c.b_codes.p, *vals = (uint32_t *)c.b_vals.p;
        morton_keys(&c, xyz, n, frame, keys, vals);
        radix_sort_u32(&c, keys, vals, (uint32_t *)c.b_codes2.p, (uint32_t *)c.b_vals2.p, n, 30);
        float4 *pts = (float4 *)c.b_pts.p;
        gather_points(&c, xyz, nullptr, vals, n, pts);
        const int64_t sn = n;
        knn_search(&c, KnnInput{pts, keys, vals, nullptr, frame, &sn, 1, n, 1, nullptr}, ke, nbr);
    } catch (const NgsError &err) {
        rc = err.code;
    } catch (...) {
        ngs_set_error("ngs_knn_noalloc: unexpected host exception");
        rc = NGS_ERR_CUDA;
    }
    // the slices belong to the static array: detach them before the stack ctx goes away
    DevBuf *bound[] = {&c.b_bbox, &c.b_frame, &c.b_codes, &c.b_vals, &c.b_codes2,
                       &c.b_vals2, &c.b_hist, &c.b_scan_part, &c.b_pts, &c.b_nodes, &c.b_knnsc, &c.b_knnlong};
    for (DevBuf *b : bound) *b = DevBuf{};
    return rc;
}
