// Serving form: a request loop with HBM-budget admission, concurrent worker
// slots (one ctx + stream + host thread each) and continuous batching of
// small jobs through the multi-scene engine.
//
// Scheduling (all under one mutex):
//   * jobs queue in submission order;
//   * a free worker looks at the oldest queued job; it starts it once
//     max(workspace the worker holds, estimate of what it would run) plus
//     what every other worker holds or has reserved fits the budget.  Idle
//     workers release their workspace when that is what stands in the way;
//   * with grouping, the worker also takes later queued small jobs (in queue
//     order, same SH width, target above k) while the rows and the budget
//     allow, and runs the group as one ngs_batch_simplify;
//   * a job finishes when its run returns; waiters are woken.
// The GPU work of a run is exactly ngs_simplify / ngs_batch_simplify on the
// worker's ctx, so every job's output equals ngs_simplify on it alone.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ngs_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    ngs_splats s;
    ngs_job_info info;
    int64_t est = 0;
};

}  // namespace

struct ngs_server {
    ngs_params prm;
    ngs_server_config cfg;
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Job> jobs;
    uint64_t next_id = 1;
    int64_t next_group = 1;
    bool stopping = false;
    // per worker: workspace held (bytes), estimate of the running group (0 if idle),
    // release request, launches so far
    std::vector<int64_t> held, running_est, launches;
    std::vector<uint8_t> release;
    std::vector<std::thread> threads;
    ngs_server_stats st = {};
    int start_error = 0;
    int started = 0;

    double now() const {
        return std::chrono::duration<double>(Clock::now() - t0).count();
    }
    int64_t reserved_except(int w) const {
        int64_t r = 0;
        for (size_t v = 0; v < held.size(); v++)
            if ((int)v != w) r += std::max(held[v], running_est[v]);
        return r;
    }
    void refresh_totals() {
        int64_t res = 0, ws = 0;
        for (size_t v = 0; v < held.size(); v++) {
            res += running_est[v];
            ws += held[v];
        }
        st.reserved_bytes = res;
        st.peak_reserved_bytes = std::max(st.peak_reserved_bytes, res);
        st.workspace_bytes = ws;
        st.peak_workspace_bytes = std::max(st.peak_workspace_bytes, ws);
    }
};

extern "C" void ngs_server_default_config(ngs_server_config *c) {
    if (!c) return;
    c->slots = 4;
    c->group_small = 1;
    c->hbm_budget_bytes = (int64_t)150e9;
    c->bytes_per_splat = 1536;
    c->small_rows = 1000000;
    c->group_rows = 4000000;
    c->dry_run_ns_per_splat = 0.0;
    c->priority_rows = 1000000;
}

namespace {

// Pick the next run for worker w (lock held).  Returns the job ids, empty if
// nothing can start now.
std::vector<uint64_t> pick(ngs_server *S, int w, int64_t *est_out) {
    std::vector<uint64_t> group;
    if (S->queue.empty()) return group;
    Job &h = S->jobs[S->queue.front()];
    const int64_t others = S->reserved_except(w);
    const int64_t budget = S->cfg.hbm_budget_bytes;
    if (others + std::max(S->held[w], h.est) > budget) {
        // idle workers holding workspace give it back; running ones finish first
        for (size_t v = 0; v < S->held.size(); v++)
            if ((int)v != w && S->running_est[v] == 0 && S->held[v] > 0 && !S->release[v]) {
                S->release[v] = 1;
                S->cv.notify_all();
            }
        return group;
    }
    group.push_back(S->queue.front());
    int64_t est = h.est, rows = h.info.n_in;
    const int ke = k_eff_of(INT64_MAX, S->prm.k);
    if (S->cfg.group_small && h.info.n_in <= S->cfg.small_rows && h.info.target > ke) {
        for (size_t q = 1; q < S->queue.size(); q++) {
            Job &j = S->jobs[S->queue[q]];
            if (j.info.n_in > S->cfg.small_rows || j.info.target <= ke ||
                j.s.sh_dim != h.s.sh_dim)
                continue;
            if (rows + j.info.n_in > S->cfg.group_rows) break;
            if (others + std::max(S->held[w], est + j.est) > budget) break;
            group.push_back(S->queue[q]);
            est += j.est;
            rows += j.info.n_in;
        }
    }
    // remove the picked ids from the queue, keeping the others' order
    std::deque<uint64_t> rest;
    size_t gi = 0;
    for (uint64_t id : S->queue) {
        if (gi < group.size() && id == group[gi]) gi++;
        else rest.push_back(id);
    }
    S->queue.swap(rest);
    *est_out = est;
    return group;
}

void worker(ngs_server *S, int w) {
    const bool dry = S->cfg.dry_run_ns_per_splat > 0;
    ngs_ctx *ctx = nullptr;
    cudaStream_t st_hi = nullptr, st_lo = nullptr;
    int err = NGS_OK;
    if (!dry) {
        int lo = 0, hi = 0;
        if (cudaSetDevice(S->device) != cudaSuccess ||
            cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&st_hi, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&st_lo, cudaStreamNonBlocking, lo) != cudaSuccess)
            err = NGS_ERR_CUDA;
        if (err == NGS_OK) err = ngs_create(&ctx, &S->prm, st_lo);
    }
    std::unique_lock<std::mutex> lock(S->mu);
    if (err != NGS_OK && !S->start_error) S->start_error = err;
    S->started++;
    S->cv.notify_all();
    while (true) {
        if (S->release[w]) {
            S->release[w] = 0;
            if (ctx) {
                lock.unlock();
                ngs_release_workspace(ctx);
                const int64_t h = ngs_workspace_bytes(ctx);
                lock.lock();
                S->held[w] = h;
            }
            S->refresh_totals();
            S->cv.notify_all();
            continue;
        }
        int64_t est = 0;
        std::vector<uint64_t> group;
        if (err == NGS_OK) group = pick(S, w, &est);
        if (group.empty()) {
            if (S->stopping && (S->queue.empty() || err != NGS_OK)) break;
            S->cv.wait(lock);
            continue;
        }
        const int64_t gid = S->next_group++;
        std::vector<ngs_splats> sc;
        std::vector<int64_t> tg;
        int64_t rows = 0;
        const double t_start = S->now();
        for (uint64_t id : group) {
            Job &j = S->jobs[id];
            j.info.status = NGS_JOB_RUNNING;
            j.info.slot = w;
            j.info.group = gid;
            j.info.group_size = (int32_t)group.size();
            j.info.start_s = t_start;
            sc.push_back(j.s);
            tg.push_back(j.info.target);
            rows += j.info.n_in;
        }
        S->running_est[w] = est;
        S->st.queued = (int64_t)S->queue.size();
        S->st.running += (int64_t)group.size();
        S->st.groups++;
        S->refresh_totals();
        lock.unlock();

        std::vector<int> rc(group.size(), NGS_OK);
        if (ctx) {
            // short runs first (shortest-job-first on the SMs): a run below
            // priority_rows rows takes the high-priority stream
            const bool high = S->cfg.priority_rows > 0 && rows < S->cfg.priority_rows;
            const int r = ngs_set_stream(ctx, high ? st_hi : st_lo);
            if (r != NGS_OK)
                for (int &x : rc) x = r;
        }
        if (rc[0] != NGS_OK) {
        } else if (dry) {
            std::this_thread::sleep_for(
                std::chrono::nanoseconds((int64_t)(S->cfg.dry_run_ns_per_splat * (double)rows)));
            for (size_t i = 0; i < sc.size(); i++) sc[i].n = std::min(sc[i].n, tg[i]);
        } else if (group.size() == 1) {
            rc[0] = ngs_simplify(ctx, &sc[0], tg[0], nullptr);
        } else {
            int r = ngs_batch_simplify(ctx, sc.data(), tg.data(), (int32_t)sc.size(), nullptr);
            if (r == NGS_ERR_INVALID_ARG) {
                // input validation fails before any output is written: run the
                // jobs one by one so that only the offending job fails
                for (size_t i = 0; i < sc.size(); i++) rc[i] = ngs_simplify(ctx, &sc[i], tg[i], nullptr);
            } else {
                for (size_t i = 0; i < sc.size(); i++) rc[i] = r;
            }
        }
        const double t_end = S->now();
        const int64_t h = ctx ? ngs_workspace_bytes(ctx) : 0;
        const int64_t nl = ctx ? ngs_launch_count(ctx) : 0;

        lock.lock();
        for (size_t i = 0; i < group.size(); i++) {
            Job &j = S->jobs[group[i]];
            j.info.finish_s = t_end;
            j.info.status = rc[i] == NGS_OK ? NGS_JOB_DONE : rc[i];
            j.info.n_out = rc[i] == NGS_OK ? sc[i].n : -1;
            if (rc[i] == NGS_OK) S->st.finished++;
            else S->st.failed++;
        }
        S->st.running -= (int64_t)group.size();
        S->running_est[w] = 0;
        S->held[w] = h;
        S->launches[w] = nl;
        int64_t tot = 0;
        for (int64_t x : S->launches) tot += x;
        S->st.gpu_launches = tot;
        S->refresh_totals();
        S->cv.notify_all();
    }
    lock.unlock();
    if (ctx) ngs_destroy(ctx);
    if (st_hi) cudaStreamDestroy(st_hi);
    if (st_lo) cudaStreamDestroy(st_lo);
}

}  // namespace

extern "C" int ngs_server_create(ngs_server **out, const ngs_params *p, const ngs_server_config *cfg) {
    if (!out) {
        ngs_set_error("ngs_server_create: server pointer is NULL");
        return NGS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    ngs_server_config c;
    if (cfg) c = *cfg;
    else ngs_server_default_config(&c);
    if (c.slots < 1 || c.slots > 64 || c.hbm_budget_bytes <= 0 || c.bytes_per_splat <= 0 ||
        c.small_rows < 0 || c.group_rows < 1 || !(c.dry_run_ns_per_splat >= 0.0) ||
        c.priority_rows < 0) {
        ngs_set_error("ngs_server_create: configuration out of range");
        return NGS_ERR_INVALID_ARG;
    }
    ngs_server *S = new (std::nothrow) ngs_server();
    if (!S) return NGS_ERR_OOM;
    if (p) S->prm = *p;
    else ngs_default_params(&S->prm);
    S->cfg = c;
    S->t0 = Clock::now();
    if (c.dry_run_ns_per_splat <= 0 && cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        ngs_set_error("ngs_server_create: no current CUDA device");
        return NGS_ERR_CUDA;
    }
    S->held.assign(c.slots, 0);
    S->running_est.assign(c.slots, 0);
    S->launches.assign(c.slots, 0);
    S->release.assign(c.slots, 0);
    for (int w = 0; w < c.slots; w++) S->threads.emplace_back(worker, S, w);
    int err;
    {
        std::unique_lock<std::mutex> lock(S->mu);
        S->cv.wait(lock, [&] { return S->started == c.slots; });
        err = S->start_error;
    }
    if (err != NGS_OK) {  // a worker could not create its stream or ctx
        ngs_server_destroy(S);
        ngs_set_error("ngs_server_create: a worker failed to start (code %d)", err);
        return err;
    }
    *out = S;
    return NGS_OK;
}

extern "C" int ngs_server_destroy(ngs_server *S) {
    if (!S) return NGS_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stopping = true;
    }
    S->cv.notify_all();
    for (auto &t : S->threads) t.join();
    delete S;
    return NGS_OK;
}

extern "C" int ngs_serve_submit(ngs_server *S, const ngs_splats *job, int64_t target, uint64_t *id) {
    if (!S || !job || !id) {
        ngs_set_error("ngs_serve_submit: NULL argument");
        return NGS_ERR_INVALID_ARG;
    }
    if (target < 1 || job->n < 0 || job->n > job->cap || job->sh_dim < 1 || job->sh_dim > 64) {
        ngs_set_error("ngs_serve_submit: bad job (n=%lld cap=%lld sh_dim=%d target=%lld)",
                      (long long)job->n, (long long)job->cap, job->sh_dim, (long long)target);
        return NGS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stopping) {
        ngs_set_error("ngs_serve_submit: server is stopping");
        return NGS_ERR_STATE;
    }
    Job j;
    j.s = *job;
    j.est = S->cfg.bytes_per_splat * job->n;
    memset(&j.info, 0, sizeof(j.info));
    j.info.status = NGS_JOB_QUEUED;
    j.info.slot = -1;
    j.info.n_in = job->n;
    j.info.target = target;
    j.info.n_out = -1;
    j.info.submit_s = S->now();
    const uint64_t jid = S->next_id++;
    S->st.submitted++;
    if (j.est > S->cfg.hbm_budget_bytes) {
        j.info.status = NGS_ERR_BUDGET;
        j.info.finish_s = j.info.submit_s;
        S->jobs.emplace(jid, j);
        S->st.failed++;
        *id = jid;
        ngs_set_error("ngs_serve_submit: job of %lld splats needs about %lld bytes, above the "
                      "budget of %lld", (long long)job->n, (long long)j.est,
                      (long long)S->cfg.hbm_budget_bytes);
        return NGS_ERR_BUDGET;
    }
    S->jobs.emplace(jid, j);
    S->queue.push_back(jid);
    S->st.queued = (int64_t)S->queue.size();
    *id = jid;
    S->cv.notify_all();
    return NGS_OK;
}

static int job_result(const Job &j, int *done, int64_t *n_out) {
    const bool fin = j.info.status <= 0;
    if (done) *done = fin ? 1 : 0;
    if (n_out) *n_out = j.info.n_out;
    if (fin && j.info.status < 0) {
        ngs_set_error("job failed with code %d", j.info.status);
        return j.info.status;
    }
    return NGS_OK;
}

extern "C" int ngs_serve_poll(ngs_server *S, uint64_t id, int *done, int64_t *n_out) {
    if (!S) return NGS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) {
        ngs_set_error("ngs_serve_poll: unknown job %llu", (unsigned long long)id);
        return NGS_ERR_INVALID_ARG;
    }
    return job_result(it->second, done, n_out);
}

extern "C" int ngs_serve_wait(ngs_server *S, uint64_t id, double timeout_s, int64_t *n_out) {
    if (!S) return NGS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) {
        ngs_set_error("ngs_serve_wait: unknown job %llu", (unsigned long long)id);
        return NGS_ERR_INVALID_ARG;
    }
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s));
    while (it->second.info.status > 0) {
        if (S->cv.wait_until(lock, deadline) == std::cv_status::timeout &&
            it->second.info.status > 0) {
            ngs_set_error("ngs_serve_wait: job %llu not finished after %g s",
                          (unsigned long long)id, timeout_s);
            return NGS_ERR_TIMEOUT;
        }
    }
    int done = 0;
    return job_result(it->second, &done, n_out);
}

extern "C" int ngs_serve_info(ngs_server *S, uint64_t id, ngs_job_info *info) {
    if (!S || !info) return NGS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) {
        ngs_set_error("ngs_serve_info: unknown job %llu", (unsigned long long)id);
        return NGS_ERR_INVALID_ARG;
    }
    *info = it->second.info;
    return NGS_OK;
}

extern "C" int ngs_server_get_stats(ngs_server *S, ngs_server_stats *out) {
    if (!S || !out) return NGS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    *out = S->st;
    return S->start_error;
}

extern "C" double ngs_server_clock(ngs_server *S) { return S ? S->now() : 0.0; }

extern "C" int ngs_serve_replay(ngs_server *S, const ngs_splats *jobs, const int64_t *targets,
                                const double *arrival_s, int32_t n_jobs, uint64_t *job_ids) {
    if (!S || n_jobs < 0 || (n_jobs > 0 && (!jobs || !targets || !arrival_s))) {
        ngs_set_error("ngs_serve_replay: bad arguments");
        return NGS_ERR_INVALID_ARG;
    }
    std::vector<uint64_t> ids(n_jobs, 0);
    int first_err = NGS_OK;
    const Clock::time_point start = Clock::now();
    for (int i = 0; i < n_jobs; i++) {
        std::this_thread::sleep_until(start + std::chrono::duration_cast<Clock::duration>(
                                                  std::chrono::duration<double>(arrival_s[i])));
        const int r = ngs_serve_submit(S, &jobs[i], targets[i], &ids[i]);
        if (r != NGS_OK && first_err == NGS_OK) first_err = r;
    }
    for (int i = 0; i < n_jobs; i++)
        if (ids[i]) ngs_serve_wait(S, ids[i], 1e9, nullptr);
    if (job_ids)
        for (int i = 0; i < n_jobs; i++) job_ids[i] = ids[i];
    return first_err;
}
