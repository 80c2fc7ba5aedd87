// Batched form of the step: many independent solves (their own grids, fields,
// sources and parameters, one common precision) traced together, optionally
// captured in a CUDA graph and replayed, with launch shapes chosen by an
// autotuner that times candidate shapes on the batch itself.
//
// Light solves (where launches and host round trips would dominate) share
// cooperative, persistent launches of batch_kernel fed by a device work queue.
// Heavy solves (many segments in the last run, a large grid, or the
// frequency-integrated rate) are cut into chunks of sources; each chunk is
// traced by one launch of the per-level march kernel per HEALPix level, every
// launch sized on the device from the parents the previous level counted, so
// no host round trip separates the levels. The chunks are spread over parallel
// lanes (streams forked from the batch stream and joined back), whose launches
// overlap on the device and fill each other's tails.
//
// Per run, on the batch's private stream: for every solve Gamma is cleared and
// kappa rebuilt from the handle's current n_H and x; the light and heavy solves
// are traced; finalize writes every solve's heating and deposited photons; the
// per-solve statistics come back in one copy. Sources (after dedup, sort and
// merging) and the n_th default are fixed when the batch is created.
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
// Heavy solves: lanes, and the ray-record bytes one lane's chunk may need at most (a chunk holds as
// many sources as keep every level's parent records within it).
constexpr int kLanes = 4;
constexpr int64_t kLaneRecordBytes = int64_t(768) << 20;
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
    bool use_geo = false;                  // every level tabled: the persistent kernel reads tables
    bool geo_shared = false;               // every solve shares one split radius and boundary: tables apply
    bool geo_ok[RT_MAX_LEVELS + 1] = {};   // level l has a table in the batch's precision
    GeomLevel geo[RT_MAX_LEVELS + 1];
    // heavy solves: per-level launches over chunks of sources on parallel lanes
    cudaStream_t lane[kLanes] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kLanes] = {};
    RayStore lane_rays[kLanes][RT_MAX_LEVELS + 1];  // parents of level l of the lane's current chunk
    int64_t lane_cap[RT_MAX_LEVELS + 1] = {};       // records per level and lane
    unsigned long long* d_lane_count = nullptr;     // kLanes x (RT_MAX_LEVELS + 1) parent counters
    std::vector<int64_t> chunk;                     // sources per chunk of each solve
    std::vector<int64_t> tlev;                      // per solve: levels that read tables in the last run
    BatchSolve* d_solves = nullptr;
    DevStats* d_stats = nullptr;
    DevStats* h_stats = nullptr;           // pinned
    DevStats* m_stats = nullptr;           // its device address (mapped)
    SrcEntry* d_src = nullptr;
    int64_t nsrc = 0;
    RayStore rays[RT_MAX_LEVELS + 1];
    unsigned long long* d_counts = nullptr;
    unsigned long long* d_tiles = nullptr;
    unsigned* d_err = nullptr;
    unsigned* h_err = nullptr;             // pinned
    unsigned* m_err = nullptr;             // its device address (mapped)
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

int max_blocks_per_sm(rt_batch* b, int block, bool table, bool single, bool freq = false)
{
    return batch_blocks_per_sm(b->precision, block, table, single, freq);
}

// Blocks per SM of a launch: the requested number, or (0) all that fit, within the occupancy of
// the kernel variant that runs (walking or table-driven, one solve or many, gray or blackbody).
int launch_blocks_per_sm(rt_batch* b, bool single, bool freq)
{
    const int occ = max_blocks_per_sm(b, b->params.block, b->use_geo, single, freq);
    return b->params.blocks_per_sm > 0 ? std::min(b->params.blocks_per_sm, occ) : occ;
}

// One cooperative launch over the solves whose sources are [src_first, src_first + src_count) of
// the batch catalog; single >= 0: that is exactly solve `single`. Solve `first` stands for the
// launch's rate: every solve of a launch has the same (gray, or blackbody at one temperature).
template <class R>
int launch_trace(rt_batch* b, int64_t src_first, int64_t src_count, int single, size_t first)
{
    BatchArgs<R> a;
    const rt_handle* hf = b->hs[first];
    a.freq = hf->cfg.spectrum != RT_SPECTRUM_GRAY ? 1 : 0;
    if constexpr (sizeof(R) == 4) a.spec = hf->spec_f;
    else a.spec = hf->spec_d;
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
    const int grid = b->sm_count * launch_blocks_per_sm(b, single >= 0, a.freq != 0);
    cudaError_t e;
    if constexpr (sizeof(R) == 4) e = launch_batch_f32(a, grid, b->params.block, b->stream);
    else e = launch_batch_f64(a, grid, b->params.block, b->stream);
    B_CUDA(b, e, "batch kernel launch");
    return RT_OK;
}

// Parent records a chunk of `count` sources can need at level l >= 1: its level l-1 rays, at most
// 12 4^(l-1) per source.
int64_t chunk_records(int64_t count, int l) { return count * 12 * (int64_t(1) << (2 * (l - 1))); }

// Solve i takes the heavy path: enough work in its last run to fill the device by itself. Before
// any run a solve is light: a chunk's buffers are sized for every ray of every level, so a heavy
// path taken blindly by an opaque many-source solve would be thousands of nearly empty launches.
bool heavy_solve(const rt_batch* b, size_t i)
{
    const int hs = b->params.heavy_shift;
    if (hs < 0) return true;
    return i < b->work.size() && b->work[i] >= (hs > 0 ? (1ULL << hs) : kHeavySegments);
}

// Chunk sizes of the heavy solves of the next run (as many sources as keep every level's parent
// records within the lane budget) and the lanes' ray buffers, grown to the largest chunk of any
// level. Outside any capture: run before a direct run and before capturing one.
int ensure_lanes(rt_batch* b)
{
    b->chunk.assign(b->hs.size(), 1);
    int64_t need[RT_MAX_LEVELS + 1] = {};
    for (size_t i = 0; i < b->hs.size(); ++i) {
        if (!heavy_solve(b, i)) continue;
        const int L = b->hs[i]->table_level;
        int64_t per_src = 0;
        for (int l = 1; l <= L; ++l) per_src += chunk_records(1, l);
        const int64_t c =
            std::max<int64_t>(1, std::min<int64_t>(b->n_emit[i], kLaneRecordBytes / (24 * std::max<int64_t>(1, per_src))));
        b->chunk[i] = c;
        for (int l = 1; l <= L; ++l) need[l] = std::max(need[l], chunk_records(c, l));
    }
    const int real = b->precision == RT_FP32 ? 4 : 8;
    for (int l = 1; l <= RT_MAX_LEVELS; ++l) {
        if (need[l] <= b->lane_cap[l]) continue;
        B_CUDA(b, cudaStreamSynchronize(b->stream), "batch stream");
        for (int k = 0; k < kLanes; ++k) {
            B_CUDA(b, cudaStreamSynchronize(b->lane[k]), "lane stream");
            cudaFree(b->lane_rays[k][l].base);
            b->lane_rays[k][l] = RayStore();
        }
        b->lane_cap[l] = 0;
        for (int k = 0; k < kLanes; ++k) {
            void* p = nullptr;
            B_CUDA(b, cudaMalloc(&p, ray_bytes(need[l], real)), "lane ray buffers");
            b->lane_rays[k][l].base = p;
            b->lane_rays[k][l].cap = need[l];
        }
        b->lane_cap[l] = need[l];
    }
    return RT_OK;
}

// One chunk of a heavy solve: sources [first, first + count) of its catalog, every level traced by one
// launch on lane k, sized on the device from the parents the previous level counted. Returns the
// levels that read geometry tables.
template <class R>
int enqueue_chunk(rt_batch* b, size_t i, int64_t first, int64_t count, int k, int64_t* tabled)
{
    rt_handle* h = b->hs[i];
    cudaStream_t s = b->lane[k];
    unsigned long long* cnt = b->d_lane_count + (size_t)k * (RT_MAX_LEVELS + 1);
    B_CUDA(b, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (RT_MAX_LEVELS + 1), s), "lane counters");
    const int L = h->table_level;
    const bool tables = b->geo_shared && !(h->cfg.flags & RT_FLAG_NO_GEOMETRY_TABLE);
    for (int l = 0; l <= L; ++l) {
        MarchArgs<R> a;
        a.level = l;
        a.n = h->cfg.n;
        a.c0 = l == 0 ? 12 * first : 0;
        a.c1 = l == 0 ? 12 * (first + count) : 4 * chunk_records(count, l);
        a.in_count = l == 0 ? nullptr : cnt + l;
        a.dirs = b->dirs + healpix_level_offset(l);
        a.src = h->d_emit;
        a.in = l == 0 ? RayBuf<R>() : ray_view<R>(b->lane_rays[k][l]);
        // rays of the deepest level a solve reaches end before their split sphere or at level_max
        a.out = (l < L && l + 1 <= h->level_max) ? ray_view<R>(b->lane_rays[k][l + 1]) : RayBuf<R>();
        a.out_count = cnt + l + 1;
        a.kap = static_cast<const R*>(h->d_kap);
        a.gamma = h->d_gamma;
        a.rq = h->rq;
        a.level_max = h->level_max;
        a.tau_max = (R)h->cfg.tau_max;
        a.overlap_mode = h->cfg.overlap_mode;
        a.hash = (h->cfg.flags & RT_FLAG_VISIT_HASH) ? 1 : 0;
        a.rs = h->rs;
        if constexpr (sizeof(R) == 8) a.spec = h->spec_d;
        else a.spec = h->spec_f;
        a.st = b->d_stats + i;
        const int64_t want = (a.c1 - a.c0 + 255) / 256;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)b->sm_count * 8));
        const bool table = tables && b->geo_ok[l];
        if constexpr (sizeof(R) == 8) {
            if (table) launch_march_table_f64(a, b->geo[l], grid, 256, s);
            else launch_march_f64(a, grid, 256, s);
        } else {
            if (table) launch_march_table_f32(a, b->geo[l], grid, 256, s);
            else launch_march_f32(a, grid, 256, s);
        }
        B_CUDA(b, cudaGetLastError(), "march launch");
        b->launches += 1;
        if (table) *tabled |= int64_t(1) << l;
    }
    return RT_OK;
}

// The heavy solves: fork the lanes from the batch stream, give each chunk to the lane with the least
// estimated work so far (segments of the last run, or cells times sources before any), join back.
int enqueue_heavy(rt_batch* b, const std::vector<char>& hv)
{
    cudaStream_t s = b->stream;
    B_CUDA(b, cudaEventRecord(b->ev_fork, s), "fork");
    for (int k = 0; k < kLanes; ++k) B_CUDA(b, cudaStreamWaitEvent(b->lane[k], b->ev_fork, 0), "fork");
    double load[kLanes] = {};
    for (size_t i = 0; i < b->hs.size(); ++i) {
        if (!hv[i] || b->n_emit[i] == 0) continue;
        const int64_t m = b->n_emit[i], c = std::max<int64_t>(1, b->chunk[i]);
        const double est = (i < b->work.size() && b->work[i] > 0) ? (double)b->work[i]
                                                                 : (double)b->hs[i]->ncell * (double)m;
        int64_t tabled = 0;
        for (int64_t f = 0; f < m; f += c) {
            const int64_t cc = std::min(c, m - f);
            int k = 0;
            for (int q = 1; q < kLanes; ++q)
                if (load[q] < load[k]) k = q;
            load[k] += est * (double)cc / (double)m;
            const int rc = b->precision == RT_FP32 ? enqueue_chunk<float>(b, i, f, cc, k, &tabled)
                                                   : enqueue_chunk<double>(b, i, f, cc, k, &tabled);
            if (rc) return rc;
        }
        b->tlev[i] = tabled;
    }
    for (int k = 0; k < kLanes; ++k) {
        B_CUDA(b, cudaEventRecord(b->ev_join[k], b->lane[k]), "join");
        B_CUDA(b, cudaStreamWaitEvent(s, b->ev_join[k], 0), "join");
    }
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
    auto big = [&](size_t i) { return gb > 0 && 2 * rbytes * b->hs[i]->ncell >= gb; };
    std::vector<char> hv(b->hs.size());
    bool any_heavy = false;
    for (size_t i = 0; i < b->hs.size(); ++i) {
        hv[i] = heavy_solve(b, i) ? 1 : 0;
        any_heavy = any_heavy || hv[i];
        b->tlev[i] = 0;
    }
    size_t i0 = 0;
    int64_t src0 = 0;
    while (i0 < b->hs.size()) {
        if (hv[i0]) {                               // traced on the lanes below
            src0 += b->n_emit[i0];
            ++i0;
            continue;
        }
        size_t i1 = i0;
        int64_t bytes = 0, srcs = 0;
        // one rate per launch: gray, or the blackbody at one temperature
        auto same_rate = [&](size_t i) {
            const rt_config& a = b->hs[i0]->cfg;
            const rt_config& c = b->hs[i]->cfg;
            return a.spectrum == c.spectrum && (a.spectrum == RT_SPECTRUM_GRAY || a.t_bb_K == c.t_bb_K);
        };
        while (i1 < b->hs.size() && !hv[i1]) {
            const int64_t add = rbytes * b->hs[i1]->ncell;
            if (i1 > i0 && (big(i0) || big(i1) || (gb > 0 && bytes + add > gb) || !same_rate(i1))) break;
            bytes += add;
            srcs += b->n_emit[i1];
            ++i1;
        }
        if (srcs > 0) {
            B_CUDA(b, cudaMemsetAsync(b->d_counts, 0, sizeof(unsigned long long) * kMaxSlices, s), "counter clear");
            B_CUDA(b, cudaMemsetAsync(b->d_tiles, 0, sizeof(unsigned long long) * kMaxSlices, s), "counter clear");
            const int single = i1 == i0 + 1 ? (int)i0 : -1;
            const int rc = b->precision == RT_FP32 ? launch_trace<float>(b, src0, srcs, single, i0)
                                                   : launch_trace<double>(b, src0, srcs, single, i0);
            if (rc) return rc;
            b->launches += 1;
            if (b->use_geo)
                for (size_t i = i0; i < i1; ++i) b->tlev[i] = (int64_t(2) << b->table_level) - 1;
        }
        src0 += srcs;
        i0 = i1;
    }
    if (any_heavy) {
        const int rc = enqueue_heavy(b, hv);
        if (rc) return rc;
    }
    for (size_t i = 0; i < b->hs.size(); ++i) {
        rt_handle* h = b->hs[i];
        b->launches += launch_finalize(h->d_gamma, h->d_nh, h->d_x, h->ncell, h->cfg.e_heat_erg, h->vol, h->d_heat,
                                       b->d_stats + i, s);
    }
    B_CUDA(b, cudaGetLastError(), "finalize launch");
    // statistics and error word written into pinned memory by a kernel, not copied: a server's
    // result copies of the previous batch may occupy the copy engines
    ReadbackList rb;
    rb.add(b->d_stats, b->m_stats, sizeof(DevStats) * b->hs.size());
    rb.add(b->d_err, b->m_err, sizeof(unsigned));
    b->launches += launch_readback(rb, s);
    B_CUDA(b, cudaGetLastError(), "readback launch");
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
    const int lrc = ensure_lanes(b);
    if (lrc) return lrc;
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

// One run, in two halves: launch (wait for the handles' streams, replay the graph or enqueue)
// and finish (wait for the batch stream, check the error words, read the time and each solve's
// work for the next grouping). A caller may do other host work between the two.
int run_launch(rt_batch* b)
{
    for (rt_handle* h : b->hs) B_CUDA(b, cudaStreamSynchronize(h->stream), "handle stream");
    if (!b->captured) {                   // the heavy solves' lanes, before the timed region
        const int rc = ensure_lanes(b);
        if (rc) return rc;
    }
    B_CUDA(b, cudaEventRecord(b->ev0, b->stream), "event");
    if (b->captured) {
        B_CUDA(b, cudaGraphLaunch(b->exec, b->stream), "graph launch");
    } else {
        const int rc = enqueue(b);
        if (rc) return rc;
    }
    B_CUDA(b, cudaEventRecord(b->ev1, b->stream), "event");
    return RT_OK;
}

int run_finish(rt_batch* b, float* ms)
{
    B_CUDA(b, cudaStreamSynchronize(b->stream), "batch run");
    if (*b->h_err) return bfail(b, RT_EDEVICE, "batch kernel reported an internal error (buffer, slice or level limit)");
    for (size_t i = 0; i < b->hs.size(); ++i)
        if (b->h_stats[i].err) return bfail(b, RT_EDEVICE, "a march launch of a heavy solve reported an internal error");
    if (ms) B_CUDA(b, cudaEventElapsedTime(ms, b->ev0, b->ev1), "event");
    b->work.assign(b->hs.size(), 0ULL);           // the next launches' grouping (a graph keeps its own)
    for (size_t i = 0; i < b->hs.size(); ++i)
        for (int l = 0; l < RT_MAX_LEVELS; ++l) b->work[i] += b->h_stats[i].segments[l];
    return RT_OK;
}

int run_once(rt_batch* b, float* ms)
{
    const int rc = run_launch(b);
    return rc ? rc : run_finish(b, ms);
}

int apply_params(rt_batch* b, const rt_batch_params& p)
{
    if ((p.block != 128 && p.block != 256) || p.tile < 32 || p.tile % 32 || p.slice < 1024 ||
        p.slice > (int64_t(1) << 28) || p.blocks_per_sm < 0 || p.group_bytes < 0 || p.heavy_shift < -1 ||
        p.heavy_shift > 62)
        return bfail(b, RT_EINVAL,
                     "batch params: block 128|256, tile a multiple of 32, slice in [1024, 2^28], group_bytes >= 0, "
                     "heavy_shift in [-1, 62]");
    int occ = 0;
    for (int v = 0; v < 8; ++v) occ = std::max(occ, max_blocks_per_sm(b, p.block, v & 1, v & 2, v & 4));
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
    st->table_levels = i < b->tlev.size() ? b->tlev[i] : 0;
}

cudaStream_t nyx::batch_stream(const rt_batch* b) { return b->stream; }

int nyx::batch_run_direct(rt_batch* b, float* ms) { return run_once(b, ms); }

int nyx::batch_launch(rt_batch* b) { return run_launch(b); }

int nyx::batch_finish(rt_batch* b, float* ms) { return run_finish(b, ms); }

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
        B_CUDA(b, cudaHostGetDevicePointer(reinterpret_cast<void**>(&b->m_err), b->h_err, 0), "error word");
        *b->h_err = 0;
        B_CUDA(b, cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming), "event");
        for (int k = 0; k < kLanes; ++k) {
            B_CUDA(b, cudaStreamCreateWithFlags(&b->lane[k], cudaStreamNonBlocking), "lane stream");
            B_CUDA(b, cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming), "event");
        }
        B_CUDA(b, cudaMalloc(&b->d_lane_count, sizeof(unsigned long long) * kLanes * (RT_MAX_LEVELS + 1)),
               "lane counters");
    }
    {   // solves that share a split radius and boundary read the geometry tables of the batch's
        // precision, built here (outside any capture) for the largest grid of the batch: the
        // persistent kernel (FP32) when every level has one, the heavy path level by level
        b->geo_shared = !b->hs.empty();
        bool any_table = false, every_table = true;
        int nmax = 0;
        for (rt_handle* h : b->hs) {
            if (h->rq != b->hs[0]->rq || h->rs != b->hs[0]->rs) b->geo_shared = false;
            if (h->cfg.flags & RT_FLAG_NO_GEOMETRY_TABLE) every_table = false;
            else any_table = true;
            nmax = std::max(nmax, h->cfg.n);
        }
        bool all = b->geo_shared && any_table;
        for (int l = 0; l <= RT_MAX_LEVELS; ++l) {
            b->geo[l] = GeomLevel();
            b->geo_ok[l] = false;
        }
        for (int l = 0; b->geo_shared && any_table && l <= table_level; ++l) {
            b->geo_ok[l] = geometry_level(b->device, b->hs[0]->rq, l, nmax, b->hs[0]->rs,
                                          b->dirs + healpix_level_offset(l), b->stream, b->precision == RT_FP64,
                                          &b->geo[l]);
            all = all && b->geo_ok[l];
        }
        b->use_geo = all && every_table;
    }
    b->chunk.assign(b->hs.size(), 1);
    b->tlev.assign(b->hs.size(), 0);
    // ---- all solves' emitted sources in one catalog, tagged with their solve index. Buffers grow
    // geometrically and stream-ordered on the batch stream: a plain cudaFree would wait for every
    // stream of the device (a server's loaders copying the next requests included).
    if (b->nsrc > b->cap_src || !b->d_src) {
        if (b->d_src) B_CUDA(b, cudaFreeAsync(b->d_src, b->stream), "catalog");
        b->d_src = nullptr;
        b->cap_src = std::max<int64_t>(std::max<int64_t>(b->nsrc, 2 * b->cap_src), 1024);
        B_CUDA(b, cudaMallocAsync(&b->d_src, sizeof(SrcEntry) * (size_t)b->cap_src, b->stream), "catalog");
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
        B_CUDA(b, cudaStreamSynchronize(b->stream), "batch stream");   // the pinned block is read on the host
        if (b->d_stats) B_CUDA(b, cudaFreeAsync(b->d_stats, b->stream), "stats");
        if (b->d_solves) B_CUDA(b, cudaFreeAsync(b->d_solves, b->stream), "solve table");
        cudaFreeHost(b->h_stats);
        b->d_stats = nullptr;
        b->h_stats = nullptr;
        b->m_stats = nullptr;
        b->d_solves = nullptr;
        b->cap_solves = std::max<int64_t>(std::max<int64_t>(ns, 2 * b->cap_solves), 256);
        B_CUDA(b, cudaMallocAsync(&b->d_stats, sizeof(DevStats) * (size_t)b->cap_solves, b->stream), "stats");
        B_CUDA(b, cudaMallocHost(&b->h_stats, sizeof(DevStats) * (size_t)b->cap_solves), "stats");
        B_CUDA(b, cudaHostGetDevicePointer(reinterpret_cast<void**>(&b->m_stats), b->h_stats, 0), "stats");
        B_CUDA(b, cudaMallocAsync(&b->d_solves, sizeof(BatchSolve) * (size_t)b->cap_solves, b->stream), "solve table");
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
    for (int k = 0; k < kLanes; ++k) {
        if (b->lane[k]) cudaStreamSynchronize(b->lane[k]);
        for (auto& r : b->lane_rays[k]) cudaFree(r.base);
        if (b->lane[k]) cudaStreamDestroy(b->lane[k]);
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    cudaFree(b->d_lane_count);
    if (b->stream) {
        if (b->d_solves) cudaFreeAsync(b->d_solves, b->stream);
        if (b->d_stats) cudaFreeAsync(b->d_stats, b->stream);
        if (b->d_src) cudaFreeAsync(b->d_src, b->stream);
        cudaStreamSynchronize(b->stream);
    }
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
                    p.heavy_shift = start.heavy_shift;
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
