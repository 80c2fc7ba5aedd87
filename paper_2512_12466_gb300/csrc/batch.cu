// Batched form of the step: many independent solves (their own grids, fields,
// sources and parameters, one common precision) traced by one cooperative,
// persistent launch of batch_kernel fed by a device work queue, optionally
// captured in a CUDA graph and replayed, with launch shapes chosen by an
// autotuner that times candidate shapes on the batch itself.
//
// Per run, on the batch's private stream: for every solve Gamma is cleared and
// kappa rebuilt from the handle's current n_H and x; the batch kernel traces
// all rays of all solves; finalize writes every solve's heating and deposited
// photons; the per-solve statistics come back in one copy. Sources (after
// dedup, sort and merging) and the n_th default are fixed when the batch is
// created.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "rt_handle.h"

using namespace nyx;

namespace {

__global__ void tag_sources_kernel(const SrcEntry* __restrict__ in, int64_t m, int32_t solve,
                                   SrcEntry* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        SrcEntry e = in[i];
        e.pad = solve;
        out[i] = e;
    }
}

constexpr int kMaxSlices = 1 << 16;
// A solve that traced at least this many segments in its last run gets a launch of its own (the
// single-solve kernel); lighter solves share launches, where batching pays.
constexpr unsigned long long kHeavySegments = 1ULL << 26;

}  // namespace

struct rt_batch {
    std::vector<rt_handle*> hs;
    int precision = RT_FP32;
    int device = 0;
    int sm_count = 152;
    cudaStream_t stream = nullptr;         // private, non-blocking (capturable)
    std::vector<double> n_th, emitted;
    std::vector<int64_t> n_src_in, n_dedup, n_emit;
    std::vector<int> merged;
    std::vector<BatchSolve> hsolve;
    std::vector<unsigned long long> work;   // segments each solve traced in the last run (0: not run yet)
    int64_t cap_src = 0, cap_solves = 0;
    int table_level = 0;
    const int4* dirs = nullptr;
    bool use_geo = false;                  // FP32 solves sharing one split radius: geometry tables
    GeomLevel geo[RT_MAX_LEVELS + 1];
    BatchSolve* d_solves = nullptr;
    DevStats* d_stats = nullptr;
    DevStats* h_stats = nullptr;           // pinned
    SrcEntry* d_src = nullptr;
    int64_t nsrc = 0;
    RayStore rays[RT_MAX_LEVELS + 1];
    unsigned long long* d_counts = nullptr;
    unsigned long long* d_tiles = nullptr;
    unsigned* d_err = nullptr;
    unsigned* h_err = nullptr;             // pinned
    rt_batch_params params{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool captured = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::string err;
    bool sticky = false;
    int launches = 0;
};

namespace {

int bfail(rt_batch* b, int code, const std::string& msg)
{
    b->err = msg;
    if (code == RT_ECUDA || code == RT_EDEVICE || code == RT_ETIMEOUT) b->sticky = true;
    return code;
}

#define B_CUDA(b, call, what)                                                                      \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            cudaGetLastError();                                                                    \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA,                \
                         std::string(what) + ": " + cudaGetErrorString(e_));                       \
        }                                                                                          \
    } while (0)

int alloc_rays(rt_batch* b, int64_t cap)
{
    for (auto& r : b->rays) {
        cudaFree(r.base);
        r.base = nullptr;
        r.cap = 0;
    }
    const int real = b->precision == RT_FP32 ? 4 : 8;
    for (int l = 1; l <= b->table_level + 1 && l <= RT_MAX_LEVELS; ++l) {
        void* p = nullptr;
        B_CUDA(b, cudaMalloc(&p, ray_bytes(cap, real)), "batch ray buffers");
        b->rays[l].base = p;
        b->rays[l].cap = cap;
    }
    return RT_OK;
}

int max_blocks_per_sm(rt_batch* b, int block, bool table, bool single)
{
    return batch_blocks_per_sm(b->precision, block, table, single);
}

// Blocks per SM of a launch: the requested number, or (0) all that fit, within the occupancy of
// the kernel variant that runs (walking or table-driven, one solve or many).
int launch_blocks_per_sm(rt_batch* b, bool single)
{
    const int occ = max_blocks_per_sm(b, b->params.block, b->use_geo, single);
    return b->params.blocks_per_sm > 0 ? std::min(b->params.blocks_per_sm, occ) : occ;
}

// One cooperative launch over the solves whose sources are [src_first, src_first + src_count) of
// the batch catalog; single >= 0: that is exactly solve `single`.
template <class R>
int launch_trace(rt_batch* b, int64_t src_first, int64_t src_count, int single)
{
    BatchArgs<R> a;
    a.single = single >= 0 ? 1 : 0;
    a.one = single >= 0 ? b->hsolve[(size_t)single] : BatchSolve{};
    a.solves = b->d_solves;
    a.src = b->d_src + src_first;
    a.nsrc = src_count;
    a.src_base = (unsigned)src_first;
    a.dirs = b->dirs;
    a.table_level = b->table_level;
    for (int l = 0; l <= RT_MAX_LEVELS; ++l) a.buf[l] = ray_view<R>(b->rays[l]);
    a.slice = b->params.slice;
    a.tile = b->params.tile;
    a.counts = b->d_counts;
    a.tiles = b->d_tiles;
    a.max_slices = kMaxSlices;
    a.any_hash = 0;
    for (const BatchSolve& bs : b->hsolve) a.any_hash |= bs.hash;
    a.use_geo = b->use_geo ? 1 : 0;
    for (int l = 0; l <= RT_MAX_LEVELS; ++l) a.geo[l] = b->geo[l];
    a.err = b->d_err;
    const int grid = b->sm_count * launch_blocks_per_sm(b, single >= 0);
    cudaError_t e;
    if constexpr (sizeof(R) == 4) e = launch_batch_f32(a, grid, b->params.block, b->stream);
    else e = launch_batch_f64(a, grid, b->params.block, b->stream);
    B_CUDA(b, e, "batch kernel launch");
    return RT_OK;
}

// The device work of one run, enqueued on b->stream (also what a graph captures).
int enqueue(rt_batch* b)
{
    cudaStream_t s = b->stream;
    b->launches = 0;
    for (size_t i = 0; i < b->hs.size(); ++i) {
        rt_handle* h = b->hs[i];
        B_CUDA(b, cudaMemsetAsync(h->d_gamma, 0, sizeof(double) * (size_t)h->ncell, s), "gamma clear");
        if (b->precision == RT_FP32)
            b->launches += launch_prepare_kappa_f32(h->d_nh, h->d_x, h->ncell, h->sdx, b->n_th[i],
                                                    static_cast<float*>(h->d_kap), s);
        else
            b->launches += launch_prepare_kappa_f64(h->d_nh, h->d_x, h->ncell, h->sdx, b->n_th[i],
                                                    static_cast<double*>(h->d_kap), s);
    }
    B_CUDA(b, cudaGetLastError(), "kappa launch");
    B_CUDA(b, cudaMemsetAsync(b->d_stats, 0, sizeof(DevStats) * b->hs.size(), s), "stats clear");
    B_CUDA(b, cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), s), "error clear");
    // consecutive groups of solves whose kappa + Gamma fit the budget, one launch each; a solve
    // that fills half the budget or more, or traced many segments in the last run, runs alone (the
    // single-solve kernel, whose solve parameters are kernel parameters rather than per-lane loads)
    const int rbytes = b->precision == RT_FP32 ? 12 : 16;
    const int64_t gb = b->params.group_bytes;
    auto big = [&](size_t i) {
        return (gb > 0 && 2 * rbytes * b->hs[i]->ncell >= gb) || (i < b->work.size() && b->work[i] >= kHeavySegments);
    };
    size_t i0 = 0;
    int64_t src0 = 0;
    while (i0 < b->hs.size()) {
        size_t i1 = i0;
        int64_t bytes = 0, srcs = 0;
        while (i1 < b->hs.size()) {
            const int64_t add = rbytes * b->hs[i1]->ncell;
            if (i1 > i0 && (big(i0) || big(i1) || (gb > 0 && bytes + add > gb))) break;
            bytes += add;
            srcs += b->n_emit[i1];
            ++i1;
        }
        if (srcs > 0) {
            B_CUDA(b, cudaMemsetAsync(b->d_counts, 0, sizeof(unsigned long long) * kMaxSlices, s), "counter clear");
            B_CUDA(b, cudaMemsetAsync(b->d_tiles, 0, sizeof(unsigned long long) * kMaxSlices, s), "counter clear");
            const int single = i1 == i0 + 1 ? (int)i0 : -1;
            const int rc = b->precision == RT_FP32 ? launch_trace<float>(b, src0, srcs, single)
                                                   : launch_trace<double>(b, src0, srcs, single);
            if (rc) return rc;
            b->launches += 1;
        }
        src0 += srcs;
        i0 = i1;
    }
    for (size_t i = 0; i < b->hs.size(); ++i) {
        rt_handle* h = b->hs[i];
        b->launches += launch_finalize(h->d_gamma, h->d_nh, h->d_x, h->ncell, h->cfg.e_heat_erg, h->vol, h->d_heat,
                                       b->d_stats + i, s);
    }
    B_CUDA(b, cudaGetLastError(), "finalize launch");
    B_CUDA(b, cudaMemcpyAsync(b->h_stats, b->d_stats, sizeof(DevStats) * b->hs.size(), cudaMemcpyDeviceToHost, s),
           "stats read");
    B_CUDA(b, cudaMemcpyAsync(b->h_err, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "error read");
    return RT_OK;
}

void drop_graph(rt_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->captured = false;
}

int capture(rt_batch* b)
{
    drop_graph(b);
    B_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    const int rc = enqueue(b);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc || e != cudaSuccess) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        b->sticky = false;
        if (!rc) b->err = std::string("stream capture failed: ") + cudaGetErrorString(e);
        return RT_ECUDA;
    }
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        b->err = "graph instantiation failed";
        return RT_ECUDA;
    }
    b->graph = g;
    b->captured = true;
    return RT_OK;
}

// One run: wait for the handles' streams, replay the graph (or enqueue), wait.
int run_once(rt_batch* b, float* ms)
{
    for (rt_handle* h : b->hs) B_CUDA(b, cudaStreamSynchronize(h->stream), "handle stream");
    B_CUDA(b, cudaEventRecord(b->ev0, b->stream), "event");
    if (b->captured) {
        B_CUDA(b, cudaGraphLaunch(b->exec, b->stream), "graph launch");
    } else {
        const int rc = enqueue(b);
        if (rc) return rc;
    }
    B_CUDA(b, cudaEventRecord(b->ev1, b->stream), "event");
    B_CUDA(b, cudaStreamSynchronize(b->stream), "batch run");
    if (*b->h_err) return bfail(b, RT_EDEVICE, "batch kernel reported an internal error (buffer, slice or level limit)");
    if (ms) B_CUDA(b, cudaEventElapsedTime(ms, b->ev0, b->ev1), "event");
    b->work.assign(b->hs.size(), 0ULL);           // the next launches' grouping (a graph keeps its own)
    for (size_t i = 0; i < b->hs.size(); ++i)
        for (int l = 0; l < RT_MAX_LEVELS; ++l) b->work[i] += b->h_stats[i].segments[l];
    return RT_OK;
}

int apply_params(rt_batch* b, const rt_batch_params& p)
{
    if ((p.block != 128 && p.block != 256) || p.tile < 32 || p.tile % 32 || p.slice < 1024 ||
        p.slice > (int64_t(1) << 28) || p.blocks_per_sm < 0 || p.group_bytes < 0)
        return bfail(b, RT_EINVAL,
                     "batch params: block 128|256, tile a multiple of 32, slice in [1024, 2^28], group_bytes >= 0");
    int occ = 0;
    for (int v = 0; v < 4; ++v) occ = std::max(occ, max_blocks_per_sm(b, p.block, v & 1, v & 2));
    if (p.blocks_per_sm > occ) return bfail(b, RT_EINVAL, "batch params: blocks_per_sm above the occupancy limit");
    const bool realloc = p.slice != b->params.slice || !b->rays[1].base;
    b->params = p;
    if (realloc) {
        B_CUDA(b, cudaStreamSynchronize(b->stream), "batch stream");
        const int rc = alloc_rays(b, p.slice);
        if (rc) return rc;
    }
    if (b->captured) return capture(b);
    return RT_OK;
}

}  // namespace

void nyx::batch_fill_stats(const rt_batch* b, size_t i, float ms, rt_stats* st)
{
    std::memset(st, 0, sizeof(*st));
    const DevStats& d = b->h_stats[i];
    st->n_src_in = b->n_src_in[i];
    st->n_src_dedup = b->n_dedup[i];
    st->n_src_emit = b->n_emit[i];
    st->merged = b->merged[i];
    st->chem_iters = 1;
    st->level_max = b->hs[i]->level_max;
    st->launches = b->launches;
    for (int l = 0; l < RT_MAX_LEVELS; ++l) {
        st->rays[l] = (int64_t)d.rays[l];
        st->splits[l] = (int64_t)d.splits[l];
        st->escaped[l] = (int64_t)d.escaped[l];
        st->dropped_tau[l] = (int64_t)d.dropped_tau[l];
        st->dropped_level[l] = (int64_t)d.dropped_level[l];
        st->segments[l] = (int64_t)d.segments[l];
        st->secondary[l] = (int64_t)d.secondary[l];
    }
    st->visit_hash = d.visit_hash;
    st->emitted_ph = b->emitted[i];
    st->absorbed_ph = d.absorbed;
    st->escaped_ph = d.escaped_ph;
    st->dropped_ph = d.dropped_ph;
    st->deposited_ph = d.deposited;
    st->ms_trace = ms;
    st->ms_step = ms;
    st->ms_march = ms;
    st->march_launches = 1;
}

cudaStream_t nyx::batch_stream(const rt_batch* b) { return b->stream; }

int nyx::batch_run_direct(rt_batch* b, float* ms) { return run_once(b, ms); }

// (Re)bind a batch to a set of handles: run each handle's source stage, build
// the tagged catalog and the solve table. Allocations are kept and grown only
// when too small, so a long-lived batch (the server's) can be re-targeted every
// iteration without touching the allocator in steady state.
int nyx::batch_bind(rt_batch* b, rt_handle* const* handles, int32_t count)
{
    drop_graph(b);
    b->hs.assign(handles, handles + count);
    b->work.clear();                               // grouping history belongs to the previous solves
    b->n_th.clear();
    b->emitted.clear();
    b->n_src_in.clear();
    b->n_dedup.clear();
    b->n_emit.clear();
    b->merged.clear();
    b->nsrc = 0;
    int table_level = 0;
    for (rt_handle* h : b->hs) {
        if (h->device != b->device) return bfail(b, RT_EINVAL, "all handles of a batch must be on one device");
        if (h->cfg.precision != b->precision) return bfail(b, RT_EINVAL, "all handles of a batch must share the precision");
        if (!h->fields_set) return bfail(b, RT_ESTATE, "rt_set_fields has not been called on a handle");
        if (h->cfg.chem_iterate) return bfail(b, RT_EINVAL, "the batched form traces at fixed x (chem_iterate must be 0)");
        if (h->cfg.spectrum != RT_SPECTRUM_GRAY)
            return bfail(b, RT_EINVAL, "the batched form integrates the gray rate (spectrum must be RT_SPECTRUM_GRAY)");
        if (h->sticky) return bfail(b, RT_ESTATE, "a handle is in an error state");
    }
    DeviceGuard g(b->device);
    // ---- each solve's source stage (Sec. 2.8), unless a loader ran it ahead
    for (rt_handle* h : b->hs) {
        if (!h->src_ready) {
            const int rc = handle_prepare_sources(h);
            if (rc) return bfail(b, rc, std::string("source stage: ") + h->err);
        }
        h->src_ready = false;
        b->n_th.push_back(h->src_nth);
        b->emitted.push_back(h->src_emitted);
        b->n_src_in.push_back(h->nsrc);
        b->n_dedup.push_back(h->src_dedup);
        b->n_emit.push_back(h->n_emit);
        b->merged.push_back(h->src_merged ? 1 : 0);
        table_level = std::max(table_level, h->table_level);
        b->nsrc += h->n_emit;
    }
    {   // the device's direction table, grown to the deepest level any solve reaches
        std::string why;
        const int rc = ensure_directions(b->device, table_level, &b->dirs, why);
        if (rc) return bfail(b, rc, why);
    }
    if (!b->stream) {
        B_CUDA(b, cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "stream");
        B_CUDA(b, cudaEventCreate(&b->ev0), "event");
        B_CUDA(b, cudaEventCreate(&b->ev1), "event");
        B_CUDA(b, cudaMalloc(&b->d_counts, sizeof(unsigned long long) * kMaxSlices), "counters");
        B_CUDA(b, cudaMalloc(&b->d_tiles, sizeof(unsigned long long) * kMaxSlices), "counters");
        B_CUDA(b, cudaMalloc(&b->d_err, sizeof(unsigned)), "error word");
        B_CUDA(b, cudaMallocHost(&b->h_err, sizeof(unsigned)), "error word");
        *b->h_err = 0;
    }
    {   // FP32 solves that share a split radius read every level's geometry from the tables
        // (built here, outside any capture, for the largest grid of the batch)
        b->use_geo = b->precision == RT_FP32 && !b->hs.empty();
        int nmax = 0;
        for (rt_handle* h : b->hs) {
            if (h->rq != b->hs[0]->rq || h->rs != b->hs[0]->rs || (h->cfg.flags & RT_FLAG_NO_GEOMETRY_TABLE))
                b->use_geo = false;
            nmax = std::max(nmax, h->cfg.n);
        }
        for (int l = 0; l <= RT_MAX_LEVELS; ++l) b->geo[l] = GeomLevel();
        for (int l = 0; b->use_geo && l <= table_level; ++l)
            if (!geometry_level(b->device, b->hs[0]->rq, l, nmax, b->hs[0]->rs, b->dirs + healpix_level_offset(l),
                                b->stream, false, &b->geo[l]))
                b->use_geo = false;
    }
    // ---- all solves' emitted sources in one catalog, tagged with their solve index
    if (b->nsrc > b->cap_src || !b->d_src) {
        B_CUDA(b, cudaStreamSynchronize(b->stream), "batch stream");
        cudaFree(b->d_src);
        b->d_src = nullptr;
        b->cap_src = std::max<int64_t>(b->nsrc, 1024);
        B_CUDA(b, cudaMalloc(&b->d_src, sizeof(SrcEntry) * (size_t)b->cap_src), "catalog");
    }
    int64_t off = 0;
    for (size_t i = 0; i < b->hs.size(); ++i) {
        const int64_t m = b->n_emit[i];
        if (m > 0) {
            const int grid = (int)std::min<int64_t>((m + 255) / 256, 1024);
            tag_sources_kernel<<<grid, 256, 0, b->stream>>>(b->hs[i]->d_emit, m, (int32_t)i, b->d_src + off);
            B_CUDA(b, cudaGetLastError(), "catalog launch");
        }
        off += m;
    }
    // ---- solve table and per-solve statistics
    const int64_t ns = (int64_t)b->hs.size();
    if (ns > b->cap_solves) {
        B_CUDA(b, cudaStreamSynchronize(b->stream), "batch stream");
        cudaFree(b->d_stats);
        cudaFreeHost(b->h_stats);
        cudaFree(b->d_solves);
        b->d_stats = nullptr;
        b->h_stats = nullptr;
        b->d_solves = nullptr;
        b->cap_solves = std::max<int64_t>(ns, 64);
        B_CUDA(b, cudaMalloc(&b->d_stats, sizeof(DevStats) * (size_t)b->cap_solves), "stats");
        B_CUDA(b, cudaMallocHost(&b->h_stats, sizeof(DevStats) * (size_t)b->cap_solves), "stats");
        B_CUDA(b, cudaMalloc(&b->d_solves, sizeof(BatchSolve) * (size_t)b->cap_solves), "solve table");
    }
    b->hsolve.assign(b->hs.size(), BatchSolve{});
    int64_t first = 0;
    for (size_t i = 0; i < b->hs.size(); ++i) {
        rt_handle* h = b->hs[i];
        BatchSolve& s = b->hsolve[i];
        s.kap = h->d_kap;
        s.gamma = h->d_gamma;
        s.st = b->d_stats + i;
        s.n = h->cfg.n;
        s.level_max = h->level_max;
        s.overlap_mode = h->cfg.overlap_mode;
        s.hash = (h->cfg.flags & RT_FLAG_VISIT_HASH) ? 1 : 0;
        s.rq = h->rq;
        s.rs = h->rs;
        s.tau_max = h->cfg.tau_max;
        s.src_off = (uint32_t)first;
        s.pad_ = 0;
        first += b->n_emit[i];
    }
    B_CUDA(b, cudaMemcpyAsync(b->d_solves, b->hsolve.data(), sizeof(BatchSolve) * b->hsolve.size(),
                              cudaMemcpyHostToDevice, b->stream), "solve table");
    B_CUDA(b, cudaStreamSynchronize(b->stream), "batch setup");
    if (table_level > b->table_level || !b->rays[1].base) {
        b->table_level = std::max(b->table_level, table_level);
        if (b->params.slice > 0) {
            const int rc = alloc_rays(b, b->params.slice);
            if (rc) return rc;
        }
    }
    return RT_OK;
}

extern "C" {

const char* rt_batch_last_error(const rt_batch* b) { return b ? b->err.c_str() : ""; }

int rt_batch_destroy(rt_batch* b)
{
    if (!b) return RT_OK;
    DeviceGuard g(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (auto& r : b->rays) cudaFree(r.base);
    cudaFree(b->d_solves);
    cudaFree(b->d_stats);
    cudaFree(b->d_src);
    cudaFree(b->d_counts);
    cudaFree(b->d_tiles);
    cudaFree(b->d_err);
    cudaFreeHost(b->h_stats);
    cudaFreeHost(b->h_err);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
    return RT_OK;
}

int rt_batch_create(rt_handle* const* handles, int32_t count, void* cuda_stream, rt_batch** out)
{
    (void)cuda_stream;
    if (!out || !handles || count < 1) return RT_EINVAL;
    *out = nullptr;
    for (int32_t i = 0; i < count; ++i)
        if (!handles[i]) return RT_EINVAL;
    rt_batch* b = new rt_batch();
    b->precision = handles[0]->cfg.precision;
    b->device = handles[0]->device;
    b->sm_count = handles[0]->sm_count;
    *out = b;
    int rc = batch_bind(b, handles, count);
    if (rc) return rc;
    rt_batch_params p{};
    p.block = 256;
    p.blocks_per_sm = 0;   // every block the kernel that runs was built to fit
    p.tile = 256;
    p.slice = int64_t(1) << 22;
    p.group_bytes = int64_t(48) << 20;
    b->params.slice = 0;
    return apply_params(b, p);
}

int rt_batch_set_params(rt_batch* b, const rt_batch_params* p)
{
    if (!b || !p) return RT_EINVAL;
    if (b->sticky) return RT_ESTATE;
    DeviceGuard g(b->device);
    return apply_params(b, *p);
}

int rt_batch_get_params(const rt_batch* b, rt_batch_params* p)
{
    if (!b || !p) return RT_EINVAL;
    *p = b->params;
    return RT_OK;
}

int rt_batch_capture(rt_batch* b)
{
    if (!b) return RT_EINVAL;
    if (b->sticky) return RT_ESTATE;
    DeviceGuard g(b->device);
    return capture(b);
}

int rt_batch_tune(rt_batch* b, int32_t repeats, rt_batch_params* best_out, double* best_ms)
{
    if (!b) return RT_EINVAL;
    if (b->sticky) return RT_ESTATE;
    DeviceGuard g(b->device);
    const bool was_captured = b->captured;
    drop_graph(b);
    const rt_batch_params start = b->params;
    rt_batch_params best = start;
    double best_t = 1e300;
    const int reps = std::max(1, (int)repeats);
    const int blocks[2] = {128, 256};
    const int tiles[3] = {64, 256, 1024};
    const int64_t slices[3] = {int64_t(1) << 21, int64_t(1) << 23, int64_t(1) << 25};
    const int64_t groups[2] = {int64_t(48) << 20, 0};
    for (int64_t gb : groups)
    for (int bl : blocks) {
        const int occ = max_blocks_per_sm(b, bl, b->use_geo, false);
        std::vector<int> bpss{0};                    // all that fit, then 1 and 2 if fewer
        for (int v : {1, 2})
            if (v < occ) bpss.push_back(v);
        for (int bps : bpss) {
            for (int64_t sl : slices) {
                for (int ti : tiles) {
                    rt_batch_params p{};
                    p.block = bl;
                    p.blocks_per_sm = bps;
                    p.tile = ti;
                    p.slice = sl;
                    p.group_bytes = gb;
                    int rc = apply_params(b, p);
                    if (rc) return rc;
                    float t = 0.f, tmin = 1e30f;
                    for (int r = 0; r < reps; ++r) {
                        rc = run_once(b, &t);
                        if (rc) return rc;
                        tmin = std::min(tmin, t);
                    }
                    if (tmin < best_t) {
                        best_t = tmin;
                        best = p;
                    }
                }
            }
        }
    }
    int rc = apply_params(b, best);
    if (rc) return rc;
    if (was_captured) {
        rc = capture(b);
        if (rc) return rc;
    }
    if (best_out) *best_out = best;
    if (best_ms) *best_ms = best_t;
    return RT_OK;
}

int rt_batch_run(rt_batch* b, double* const* gamma_out, double* const* heat_out, int where, rt_stats* stats)
{
    NvtxRange nvtx("rt_batch_run");
    if (!b) return RT_EINVAL;
    if (b->sticky) return RT_ESTATE;
    if (where != RT_HOST && where != RT_DEVICE) return bfail(b, RT_EINVAL, "bad where");
    DeviceGuard g(b->device);
    float ms = 0.f;
    int rc = run_once(b, &ms);
    if (rc) return rc;
    const cudaMemcpyKind k = where == RT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    for (size_t i = 0; i < b->hs.size(); ++i) {
        rt_handle* h = b->hs[i];
        const size_t fb = sizeof(double) * (size_t)h->ncell;
        if (gamma_out && gamma_out[i]) B_CUDA(b, cudaMemcpyAsync(gamma_out[i], h->d_gamma, fb, k, b->stream), "gamma copy");
        if (heat_out && heat_out[i]) B_CUDA(b, cudaMemcpyAsync(heat_out[i], h->d_heat, fb, k, b->stream), "heat copy");
    }
    B_CUDA(b, cudaStreamSynchronize(b->stream), "output copy");
    if (stats)
        for (size_t i = 0; i < b->hs.size(); ++i) batch_fill_stats(b, i, ms, stats + i);
    return RT_OK;
}

}  // extern "C"
