// Serving loop: solves arrive as requests, are admitted while their device
// memory fits a budget, have their fields and sources copied to the GPU by
// loader threads while the previous batch runs, and are traced by a worker
// thread that forms a new batch from every loaded request at each iteration
// (continuous batching: a request arriving during a batch joins the next one
// as soon as memory allows). The worker enqueues the source stage of all the
// batch's requests back to back with one wait, then traces them in one
// persistent launch. Finisher threads copy each request's Gamma and heating
// to the caller's host buffers and record its latency (submit to done), off
// the worker's path. Solver handles are pooled by grid size: a finished
// request's handle (device arrays, stream, pinned readback block) serves the
// next request of the same n, so steady-state serving allocates nothing; idle
// handles count against the budget and the least recently used are released
// when a request of another size needs the room.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rt_handle.h"

using namespace nyx;

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }

enum { kPending = 0, kLoading = 1, kReady = 2, kRunning = 3, kDone = 4 };

struct SrvReq {
    int64_t id = 0;
    rt_config cfg{};
    const double* nh = nullptr;
    const double* x = nullptr;
    const int32_t* cells = nullptr;
    const double* ndot = nullptr;
    int64_t nsrc = 0;
    double* gamma_out = nullptr;
    double* heat_out = nullptr;
    int64_t mem = 0;
    rt_handle* h = nullptr;
    rt_stats st{};
    int rc = RT_OK;
    std::string err;
    int state = kPending;
    double t_submit = 0, t_done = 0, t_ready = 0, t_traced = 0;
};

// Device bytes a handle holds: n_H, x, Gamma, heating (FP64), kappa, and a
// source workspace of src_cap entries; the shared batch workspace is reserved
// once for the server.
int64_t handle_bytes(int n, int precision, int64_t src_cap)
{
    const int64_t cells = (int64_t)n * n * n;
    return cells * (32 + (precision == RT_FP32 ? 4 : 8)) + 160 * std::max<int64_t>(src_cap, 1024) + (1 << 16);
}

// Source capacity a handle with capacity cap has after taking nsrc sources
// (the growth rule of the handle's source workspace).
int64_t grown_cap(int64_t cap, int64_t nsrc)
{
    return nsrc <= cap ? cap : std::max<int64_t>(nsrc, std::max<int64_t>(1024, 2 * cap));
}

// Optional event trace (NYXRT_SERVER_TRACE=<file>): one line per event with
// the time since server start, the event, the request id and a value; written
// when the server is destroyed. Off by default (one branch per event).
struct TraceEv {
    double t;
    const char* what;
    int64_t id;
    double v;
};

struct Idle {
    rt_handle* h;
    int64_t mem;
    uint64_t used;      // LRU stamp
};

}  // namespace

struct rt_server {
    rt_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_load, cv_work, cv_done;
    std::deque<SrvReq*> pending, ready;
    std::unordered_map<int64_t, SrvReq*> reqs;
    int64_t next_id = 1;
    int64_t budget = 0, in_use = 0, peak = 0;
    bool stop = false;
    std::vector<std::thread> loaders;
    std::thread worker;
    std::vector<std::thread> finishers;
    std::deque<std::pair<std::vector<SrvReq*>, int>> finished;   // traced batches and their status
    std::condition_variable cv_fin;
    std::vector<cudaStream_t> streams;          // free streams for new request handles
    std::vector<Idle> idle;                     // pooled handles of finished requests
    int64_t pooled = 0;                         // device bytes the pooled handles hold
    uint64_t tick = 0;
    rt_batch* batch = nullptr;
    std::vector<double> lat;
    int64_t submitted = 0, completed = 0, failed = 0, batches = 0, segments = 0;
    double busy_ms = 0.0, load_ms = 0.0, bind_ms = 0.0, run_ms = 0.0, finish_ms = 0.0, src_ms = 0.0;
    double wait_admit_ms = 0.0, wait_batch_ms = 0.0, wait_finish_ms = 0.0;
    Clock::time_point t0;
    std::string err;
    std::string trace_path;
    std::mutex trace_mu;
    std::vector<TraceEv> trace;
};

namespace {

void trace(rt_server* s, const char* what, int64_t id, double v = 0.0)
{
    if (s->trace_path.empty()) return;
    const double t = ms_since(s->t0);
    std::lock_guard<std::mutex> lk(s->trace_mu);
    s->trace.push_back({t, what, id, v});
}

cudaStream_t take_stream(rt_server* s)
{
    if (!s->streams.empty()) {
        cudaStream_t st = s->streams.back();
        s->streams.pop_back();
        return st;
    }
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return st;
}

// Mark a request finished and account for it (lock held); its handle has
// been pooled or destroyed already.
void finish_locked(rt_server* s, SrvReq* r, int rc, const std::string& err)
{
    s->in_use -= r->mem;
    r->rc = rc;
    r->err = err;
    r->state = kDone;
    r->t_done = ms_since(s->t0);
    if (rc == RT_OK) {
        ++s->completed;
        s->lat.push_back(r->t_done - r->t_submit);
    } else {
        ++s->failed;
    }
}

// Return a request's handle to the pool (lock held). A handle in an error
// state is destroyed by the caller instead.
void pool_put_locked(rt_server* s, rt_handle* h)
{
    const int64_t mem = handle_bytes(h->cfg.n, h->cfg.precision, h->sw.cap);
    s->idle.push_back({h, mem, ++s->tick});
    s->pooled += mem;
}

// Destroy a handle and keep its stream for later handles.
void release_handle(rt_server* s, rt_handle* h)
{
    cudaStream_t st = h->stream;
    rt_destroy(h);
    std::lock_guard<std::mutex> lk(s->mu);
    if (st) s->streams.push_back(st);
}

// Admission plan for request r: reuse the most recently pooled handle of its
// grid size when that fits the budget beside the admitted requests (growing
// only its source workspace), else a fresh handle. Returns the device bytes
// the request will hold, or -1 while neither fits; *match is the pooled
// handle to reuse, or -1.
int64_t plan(const rt_server* s, const SrvReq* r, int* match)
{
    *match = -1;
    int m = -1;
    for (size_t i = 0; i < s->idle.size(); ++i)
        if (s->idle[i].h->cfg.n == r->cfg.n && (m < 0 || s->idle[i].used > s->idle[(size_t)m].used)) m = (int)i;
    if (m >= 0) {
        const rt_handle* h = s->idle[(size_t)m].h;
        const int64_t need = handle_bytes(h->cfg.n, h->cfg.precision, grown_cap(h->sw.cap, r->nsrc));
        if (s->in_use + need <= s->budget) {
            *match = m;
            return need;
        }
    }
    const int64_t need = handle_bytes(r->cfg.n, r->cfg.precision, grown_cap(0, r->nsrc));
    return s->in_use + need <= s->budget ? need : -1;
}

void loader_main(rt_server* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        SrvReq* r = nullptr;
        rt_handle* reuse = nullptr;
        std::vector<rt_handle*> evict;
        cudaStream_t stream = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // admissible once the request fits beside the admitted ones: idle
            // handles of other sizes are released to make room
            s->cv_load.wait(lk, [&] {
                if (s->stop) return true;
                if (s->pending.empty()) return false;
                int m = -1;
                return plan(s, s->pending.front(), &m) >= 0;
            });
            if (s->stop) return;
            r = s->pending.front();
            s->pending.pop_front();
            int m = -1;
            r->mem = plan(s, r, &m);
            if (m >= 0) {
                reuse = s->idle[(size_t)m].h;
                s->pooled -= s->idle[(size_t)m].mem;
                s->idle.erase(s->idle.begin() + m);
            }
            while (s->in_use + s->pooled + r->mem > s->budget && !s->idle.empty()) {
                size_t lru = 0;
                for (size_t i = 1; i < s->idle.size(); ++i)
                    if (s->idle[i].used < s->idle[lru].used) lru = i;
                evict.push_back(s->idle[lru].h);
                s->pooled -= s->idle[lru].mem;
                s->idle.erase(s->idle.begin() + (long)lru);
            }
            s->in_use += r->mem;
            s->peak = std::max(s->peak, s->in_use + s->pooled);
            r->state = kLoading;
            s->wait_admit_ms += ms_since(s->t0) - r->t_submit;
            if (!reuse) stream = take_stream(s);
        }
        const Clock::time_point tl = Clock::now();
        trace(s, reuse ? "load_reuse" : "load_new", r->id, (double)r->mem);
        for (rt_handle* h : evict) release_handle(s, h);
        int rc = RT_OK;
        std::string err;
        if (reuse) {
            r->h = reuse;
            rc = handle_reconfigure(reuse, &r->cfg);
        } else if (!stream) {
            rc = RT_ECUDA;
            err = "stream creation failed";
        } else {
            rc = rt_create(&r->cfg, stream, &r->h);
            if (rc) {
                err = rt_last_error(nullptr);
                std::lock_guard<std::mutex> lk(s->mu);
                s->streams.push_back(stream);
            }
        }
        // copies only: the source stage runs for the whole batch in the worker
        trace(s, "handle_ready", r->id);
        if (rc == RT_OK) rc = rt_set_fields(r->h, r->nh, r->x, RT_HOST);
        trace(s, "fields_copied", r->id);
        if (rc == RT_OK && r->nsrc > 0) rc = rt_add_sources(r->h, r->cells, r->ndot, r->nsrc, RT_HOST);
        trace(s, "loaded", r->id, (double)r->nsrc);
        if (rc != RT_OK && r->h && err.empty()) err = r->h->err;
        if (rc != RT_OK && r->h) {
            release_handle(s, r->h);
            r->h = nullptr;
        }
        std::lock_guard<std::mutex> lk(s->mu);
        s->load_ms += ms_since(tl);
        if (rc != RT_OK) {
            finish_locked(s, r, rc, err);
            s->cv_done.notify_all();
            s->cv_load.notify_all();
        } else {
            r->state = kReady;
            r->t_ready = ms_since(s->t0);
            s->ready.push_back(r);
            s->cv_work.notify_one();
        }
    }
}

void worker_main(rt_server* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<SrvReq*> take;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->ready.empty(); });
            if (s->stop) return;
            while (!s->ready.empty() && (int)take.size() < s->cfg.max_batch) {
                take.push_back(s->ready.front());
                s->ready.pop_front();
            }
            const double now = ms_since(s->t0);
            for (SrvReq* r : take) {
                r->state = kRunning;
                s->wait_batch_ms += now - r->t_ready;
            }
        }
        const Clock::time_point tb = Clock::now();
        for (SrvReq* r : take) trace(s, "batch_take", r->id, (double)take.size());
        // ---- every request's source stage, enqueued back to back, one wait
        std::vector<rt_handle*> all;
        for (SrvReq* r : take) all.push_back(r->h);
        std::vector<int> rcs(all.size(), RT_OK);
        sources_enqueue_many(all.data(), (int)all.size(), rcs.data());
        trace(s, "src_enqueued", -1, ms_since(tb));
        sources_wait_many(all.data(), (int)all.size(), rcs.data());
        const double src_ms = ms_since(tb);
        trace(s, "src_done", -1, src_ms);
        std::vector<SrvReq*> run, bad;
        std::vector<rt_handle*> hs;
        for (size_t i = 0; i < take.size(); ++i) {
            take[i]->rc = rcs[i];
            if (rcs[i] != RT_OK) {
                take[i]->err = take[i]->h->err;
                bad.push_back(take[i]);
            } else {
                run.push_back(take[i]);
                hs.push_back(take[i]->h);
            }
        }
        int rc = RT_OK;
        std::string err;
        if (!hs.empty()) {
            if (!s->batch) {
                rc = rt_batch_create(hs.data(), (int32_t)hs.size(), nullptr, &s->batch);
                if (rc == RT_OK) {
                    rt_batch_params p{};
                    rt_batch_get_params(s->batch, &p);
                    if (s->cfg.slice > 0) p.slice = s->cfg.slice;
                    if (s->cfg.group_bytes >= 0) p.group_bytes = s->cfg.group_bytes;
                    rc = rt_batch_set_params(s->batch, &p);
                }
            } else {
                rc = batch_bind(s->batch, hs.data(), (int32_t)hs.size());
            }
        }
        const double bind_ms = ms_since(tb);
        float ms = 0.f;
        const Clock::time_point tr = Clock::now();
        if (rc == RT_OK && !hs.empty()) rc = batch_run_direct(s->batch, &ms);
        const double run_ms = ms_since(tr);
        trace(s, "bind_done", -1, bind_ms);
        trace(s, "run_done", -1, (double)ms);
        if (rc == RT_OK)
            for (size_t i = 0; i < run.size(); ++i) batch_fill_stats(s->batch, i, ms, &run[i]->st);
        if (rc != RT_OK) {
            err = s->batch ? rt_batch_last_error(s->batch) : "batch creation failed";
            for (SrvReq* r : run) {
                r->rc = rc;
                r->err = err;
            }
        }
        run.insert(run.end(), bad.begin(), bad.end());
        std::lock_guard<std::mutex> lk(s->mu);
        if (rc != RT_OK && s->batch) {       // a failed batch is rebuilt from scratch next time
            rt_batch_destroy(s->batch);
            s->batch = nullptr;
        }
        if (!hs.empty()) ++s->batches;
        s->busy_ms += ms;
        s->bind_ms += bind_ms;
        s->src_ms += src_ms;
        s->run_ms += run_ms;
        const double now = ms_since(s->t0);
        for (SrvReq* r : run) r->t_traced = now;
        s->finished.emplace_back(std::move(run), rc);
        s->cv_fin.notify_one();
    }
}

// Copy results out, return each request's handle to the pool, mark it done (finisher threads share
// the queue of traced batches). A batch's result copies are all issued first, each on its request's
// stream, and waited for afterwards, so they overlap one another on the copy engines.
void finisher_main(rt_server* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::pair<std::vector<SrvReq*>, int> job;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_fin.wait(lk, [&] { return s->stop || !s->finished.empty(); });
            if (s->finished.empty()) return;
            job = std::move(s->finished.front());
            s->finished.pop_front();
            const double now = ms_since(s->t0);
            for (SrvReq* r : job.first) s->wait_finish_ms += now - r->t_traced;
        }
        const Clock::time_point tf = Clock::now();
        std::vector<int> rcs(job.first.size());
        std::vector<std::string> errs(job.first.size());
        for (size_t k = 0; k < job.first.size(); ++k) {
            SrvReq* r = job.first[k];
            trace(s, "fin_begin", r->id);
            rcs[k] = r->rc;
            if (rcs[k] != RT_OK) {
                errs[k] = r->err;
                continue;
            }
            rt_handle* h = r->h;
            const size_t fb = sizeof(double) * (size_t)h->ncell;
            if ((r->gamma_out && cudaMemcpyAsync(r->gamma_out, h->d_gamma, fb, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) ||
                (r->heat_out && cudaMemcpyAsync(r->heat_out, h->d_heat, fb, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)) {
                cudaGetLastError();
                rcs[k] = RT_ECUDA;
                errs[k] = "result copy failed";
            }
        }
        for (size_t k = 0; k < job.first.size(); ++k) {
            SrvReq* r = job.first[k];
            rt_handle* h = r->h;
            r->h = nullptr;
            if (rcs[k] == RT_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) {
                cudaGetLastError();
                rcs[k] = RT_ECUDA;
                errs[k] = "result copy failed";
            }
            trace(s, "fin_copied", r->id);
            const bool keep = rcs[k] == RT_OK && !h->sticky;
            if (!keep) release_handle(s, h);
            std::lock_guard<std::mutex> lk(s->mu);
            if (keep) pool_put_locked(s, h);
            if (rcs[k] == RT_OK)
                for (int l = 0; l < RT_MAX_LEVELS; ++l) s->segments += r->st.segments[l];
            finish_locked(s, r, rcs[k], errs[k]);
            s->cv_done.notify_all();
            s->cv_load.notify_all();
            trace(s, "done", r->id);
        }
        std::lock_guard<std::mutex> lk(s->mu);
        s->finish_ms += ms_since(tf);
    }
}

}  // namespace

extern "C" {

void rt_server_config_default(rt_server_config* c)
{
    std::memset(c, 0, sizeof(*c));
    c->precision = RT_FP32;
    c->max_batch = 64;
    c->hbm_budget = 0;
    c->slice = int64_t(1) << 23;
    c->group_bytes = int64_t(48) << 20;
    c->loaders = 4;
    c->max_n = 256;
}

int rt_server_create(const rt_server_config* cfg, rt_server** out)
{
    if (!out || !cfg) return RT_EINVAL;
    *out = nullptr;
    if ((cfg->precision != RT_FP32 && cfg->precision != RT_FP64) || cfg->max_batch < 1 || cfg->hbm_budget < 0 ||
        cfg->loaders < 1 || cfg->loaders > 64)
        return RT_EINVAL;
    rt_server* s = new rt_server();
    s->cfg = *cfg;
    if (const char* tp = std::getenv("NYXRT_SERVER_TRACE")) s->trace_path = tp;
    cudaGetDevice(&s->device);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return RT_ECUDA;
    }
    // reserve the shared batch workspace (one slice per level) and a margin
    const int64_t reserve = (int64_t)24 * std::max<int64_t>(cfg->slice, int64_t(1) << 22) * 14 + (int64_t(4) << 30);
    s->budget = cfg->hbm_budget > 0 ? cfg->hbm_budget : std::max<int64_t>(0, (int64_t)free_b - reserve);
    {   // build the direction table up to the deepest level a grid of max_n cells can need
        rt_config probe;
        rt_config_default(&probe, std::max(1, std::min(1024, cfg->max_n)), 1.0);
        probe.precision = cfg->precision;
        rt_handle* h = nullptr;
        if (rt_create(&probe, nullptr, &h) == RT_OK) rt_destroy(h);
    }
    s->t0 = Clock::now();
    // keep memory freed by finished requests in the stream-ordered pool for the next ones
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
        uint64_t keep = (uint64_t)s->budget;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    for (int i = 0; i < std::max(1, cfg->loaders); ++i) s->loaders.emplace_back(loader_main, s);
    s->worker = std::thread(worker_main, s);
    for (int i = 0; i < 4; ++i) s->finishers.emplace_back(finisher_main, s);
    *out = s;
    return RT_OK;
}

int rt_server_submit(rt_server* s, const rt_config* cfg, const double* n_H, const double* x_ion, const int32_t* cell_ijk,
                     const double* ndot, int64_t nsrc, double* gamma_out, double* heat_out, int64_t* id_out)
{
    if (!s || !cfg || !n_H || !x_ion || !id_out || nsrc < 0 || (nsrc > 0 && (!cell_ijk || !ndot))) return RT_EINVAL;
    if (cfg->precision != s->cfg.precision || cfg->chem_iterate || cfg->n < 1 || cfg->n > 1024)
        return RT_EINVAL;
    SrvReq* r = new SrvReq();
    r->cfg = *cfg;
    r->nh = n_H;
    r->x = x_ion;
    r->cells = cell_ijk;
    r->ndot = ndot;
    r->nsrc = nsrc;
    r->gamma_out = gamma_out;
    r->heat_out = heat_out;
    r->mem = handle_bytes(cfg->n, cfg->precision, grown_cap(0, nsrc));
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->mem > s->budget) {
        delete r;
        s->err = "request larger than the server's device-memory budget";
        return RT_ENOMEM;
    }
    r->id = s->next_id++;
    r->t_submit = ms_since(s->t0);
    trace(s, "submit", r->id, (double)cfg->n);
    s->reqs[r->id] = r;
    s->pending.push_back(r);
    ++s->submitted;
    *id_out = r->id;
    s->cv_load.notify_one();
    return RT_OK;
}

int rt_server_poll(rt_server* s, int64_t id, double wait_s, rt_stats* st, double* latency_ms)
{
    if (!s) return RT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return RT_EINVAL;
    SrvReq* r = it->second;
    if (r->state != kDone && wait_s > 0)
        s->cv_done.wait_for(lk, std::chrono::duration<double>(wait_s), [&] { return r->state == kDone; });
    if (r->state != kDone) return RT_EPENDING;
    if (st) *st = r->st;
    if (latency_ms) *latency_ms = r->t_done - r->t_submit;
    const int rc = r->rc;
    if (rc != RT_OK) s->err = r->err;
    s->reqs.erase(it);
    delete r;
    return rc;
}

int rt_server_stats_get(rt_server* s, rt_server_stats* out)
{
    if (!s || !out) return RT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->batches = s->batches;
    out->queued = (int64_t)(s->pending.size() + s->ready.size());
    out->mem_budget = s->budget;
    out->mem_in_use = s->in_use;
    out->mem_peak = s->peak;
    out->segments = s->segments;
    out->busy_ms = s->busy_ms;
    out->load_ms = s->load_ms;
    out->bind_ms = s->bind_ms;
    out->run_ms = s->run_ms;
    out->finish_ms = s->finish_ms;
    out->src_ms = s->src_ms;
    out->wait_admit_ms = s->wait_admit_ms;
    out->wait_batch_ms = s->wait_batch_ms;
    out->wait_finish_ms = s->wait_finish_ms;
    out->elapsed_ms = ms_since(s->t0);
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto q = [&](double p) { return v[(size_t)std::min<double>(v.size() - 1, std::floor(p * (v.size() - 1) + 0.5))]; };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_ms = sum / v.size();
    }
    return RT_OK;
}

const char* rt_server_last_error(const rt_server* s) { return s ? s->err.c_str() : ""; }

int rt_server_destroy(rt_server* s)
{
    if (!s) return RT_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_load.notify_all();
    s->cv_work.notify_all();
    s->cv_fin.notify_all();
    for (auto& t : s->loaders)
        if (t.joinable()) t.join();
    if (s->worker.joinable()) s->worker.join();
    for (auto& t : s->finishers)
        if (t.joinable()) t.join();
    for (auto& kv : s->reqs) {
        SrvReq* r = kv.second;
        if (r->h) {
            s->streams.push_back(r->h->stream);
            rt_destroy(r->h);
        }
        delete r;
    }
    for (Idle& e : s->idle) {
        s->streams.push_back(e.h->stream);
        rt_destroy(e.h);
    }
    if (s->batch) rt_batch_destroy(s->batch);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    if (!s->trace_path.empty()) {
        if (FILE* f = std::fopen(s->trace_path.c_str(), "a")) {
            for (const TraceEv& e : s->trace) std::fprintf(f, "%.4f %s %lld %.6g\n", e.t, e.what, (long long)e.id, e.v);
            std::fprintf(f, "---\n");
            std::fclose(f);
        }
    }
    delete s;
    return RT_OK;
}

}  // extern "C"
