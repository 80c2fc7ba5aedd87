// Serving loop: solves arrive as requests, are admitted while their device
// memory fits a budget, are loaded onto the GPU (handle, fields, sources,
// source stage) by loader threads while the previous batch runs, and are
// traced by a worker thread that forms a new batch from every loaded request
// at each iteration (continuous batching: a request arriving during a batch
// joins the next one as soon as memory allows). A finisher thread copies each
// request's Gamma and heating to the caller's host buffers, releases its
// device memory and records its latency (submit to done), off the worker's
// path, so the next batch starts as soon as the previous one ends.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
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
    cudaStream_t stream = nullptr;
    rt_stats st{};
    int rc = RT_OK;
    std::string err;
    int state = kPending;
    double t_submit = 0, t_done = 0;
};

// Device bytes a request holds while admitted: n_H, x, Gamma, heating (FP64),
// kappa, and the source workspace; the shared batch workspace is reserved once.
int64_t request_bytes(const rt_config& c, int64_t nsrc)
{
    const int64_t cells = (int64_t)c.n * c.n * c.n;
    return cells * (32 + (c.precision == RT_FP32 ? 4 : 8)) + 160 * std::max<int64_t>(nsrc, 1024) + (1 << 16);
}

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
    std::vector<cudaStream_t> streams;          // free streams for request handles
    rt_batch* batch = nullptr;
    std::vector<double> lat;
    int64_t submitted = 0, completed = 0, failed = 0, batches = 0, segments = 0;
    double busy_ms = 0.0, load_ms = 0.0, bind_ms = 0.0, run_ms = 0.0, finish_ms = 0.0;
    Clock::time_point t0;
    std::string err;
};

namespace {

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

// Mark a request finished and account for it (lock held; its handle is
// already destroyed).
void finish_locked(rt_server* s, SrvReq* r, int rc, const std::string& err)
{
    if (r->stream) s->streams.push_back(r->stream);
    r->stream = nullptr;
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

void loader_main(rt_server* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        SrvReq* r = nullptr;
        cudaStream_t stream = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_load.wait(lk, [&] {
                return s->stop || (!s->pending.empty() && s->in_use + s->pending.front()->mem <= s->budget);
            });
            if (s->stop) return;
            r = s->pending.front();
            s->pending.pop_front();
            s->in_use += r->mem;
            s->peak = std::max(s->peak, s->in_use);
            r->state = kLoading;
            stream = take_stream(s);
            r->stream = stream;
        }
        const Clock::time_point tl = Clock::now();
        int rc = stream ? RT_OK : RT_ECUDA;
        std::string err = stream ? "" : "stream creation failed";
        if (rc == RT_OK) {
            rc = rt_create(&r->cfg, stream, &r->h);
            if (rc) err = rt_last_error(nullptr);
        }
        if (rc == RT_OK) rc = rt_set_fields(r->h, r->nh, r->x, RT_HOST);
        if (rc == RT_OK && r->nsrc > 0) rc = rt_add_sources(r->h, r->cells, r->ndot, r->nsrc, RT_HOST);
        if (rc == RT_OK) rc = handle_prepare_sources(r->h);
        if (rc != RT_OK && r->h && err.empty()) err = r->h->err;
        if (rc != RT_OK && r->h) {
            rt_destroy(r->h);
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
            for (SrvReq* r : take) r->state = kRunning;
        }
        std::vector<rt_handle*> hs;
        for (SrvReq* r : take) hs.push_back(r->h);
        int rc = RT_OK;
        std::string err;
        const Clock::time_point tb = Clock::now();
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
        const double bind_ms = ms_since(tb);
        float ms = 0.f;
        const Clock::time_point tr = Clock::now();
        if (rc == RT_OK) rc = batch_run_direct(s->batch, &ms);
        const double run_ms = ms_since(tr);
        if (rc == RT_OK)
            for (size_t i = 0; i < take.size(); ++i) batch_fill_stats(s->batch, i, ms, &take[i]->st);
        if (rc != RT_OK) {
            err = s->batch ? rt_batch_last_error(s->batch) : "batch creation failed";
            for (SrvReq* r : take) r->err = err;
        }
        std::lock_guard<std::mutex> lk(s->mu);
        if (rc != RT_OK && s->batch) {       // a failed batch is rebuilt from scratch next time
            rt_batch_destroy(s->batch);
            s->batch = nullptr;
        }
        ++s->batches;
        s->busy_ms += ms;
        s->bind_ms += bind_ms;
        s->run_ms += run_ms;
        s->finished.emplace_back(std::move(take), rc);
        s->cv_fin.notify_one();
    }
}

// Copy results out, release each request's device memory, mark it done
// (two finisher threads share the queue of traced batches).
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
        }
        int rc = job.second;
        for (SrvReq* r : job.first) {
            const Clock::time_point tf = Clock::now();
            int rrc = rc;
            std::string err = rrc != RT_OK ? r->err : std::string();
            if (rrc == RT_OK) {
                const size_t fb = sizeof(double) * (size_t)r->h->ncell;
                if ((r->gamma_out && cudaMemcpyAsync(r->gamma_out, r->h->d_gamma, fb, cudaMemcpyDeviceToHost, r->stream) != cudaSuccess) ||
                    (r->heat_out && cudaMemcpyAsync(r->heat_out, r->h->d_heat, fb, cudaMemcpyDeviceToHost, r->stream) != cudaSuccess) ||
                    cudaStreamSynchronize(r->stream) != cudaSuccess) {
                    cudaGetLastError();
                    rrc = RT_ECUDA;
                    err = "result copy failed";
                }
            }
            rt_destroy(r->h);
            r->h = nullptr;
            std::lock_guard<std::mutex> lk(s->mu);
            s->finish_ms += ms_since(tf);
            if (rrc == RT_OK)
                for (int l = 0; l < RT_MAX_LEVELS; ++l) s->segments += r->st.segments[l];
            finish_locked(s, r, rrc, err);
            s->cv_done.notify_all();
            s->cv_load.notify_all();
        }
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
    for (int i = 0; i < 2; ++i) s->finishers.emplace_back(finisher_main, s);
    *out = s;
    return RT_OK;
}

int rt_server_submit(rt_server* s, const rt_config* cfg, const double* n_H, const double* x_ion, const int32_t* cell_ijk,
                     const double* ndot, int64_t nsrc, double* gamma_out, double* heat_out, int64_t* id_out)
{
    if (!s || !cfg || !n_H || !x_ion || !id_out || nsrc < 0 || (nsrc > 0 && (!cell_ijk || !ndot))) return RT_EINVAL;
    if (cfg->precision != s->cfg.precision || cfg->chem_iterate || cfg->n < 1 || cfg->n > 1024) return RT_EINVAL;
    SrvReq* r = new SrvReq();
    r->cfg = *cfg;
    r->nh = n_H;
    r->x = x_ion;
    r->cells = cell_ijk;
    r->ndot = ndot;
    r->nsrc = nsrc;
    r->gamma_out = gamma_out;
    r->heat_out = heat_out;
    r->mem = request_bytes(*cfg, nsrc);
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->mem > s->budget) {
        delete r;
        s->err = "request larger than the server's device-memory budget";
        return RT_ENOMEM;
    }
    r->id = s->next_id++;
    r->t_submit = ms_since(s->t0);
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
        if (r->h) rt_destroy(r->h);
        if (r->stream) s->streams.push_back(r->stream);
        delete r;
    }
    if (s->batch) rt_batch_destroy(s->batch);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
    return RT_OK;
}

}  // extern "C"
