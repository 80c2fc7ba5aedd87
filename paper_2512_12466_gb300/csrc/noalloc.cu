// rt_step_noalloc: a variant of rt_step that allocates no memory, for small
// grids (n <= 32). It is meant for callers that are not allowed to allocate
// device memory at the point where they need a step: code running inside a
// memory-capped or externally managed pool, real-time loops that must not
// enter the CUDA allocator, or hosts embedding the library where every
// allocation has to be budgeted up front. Instead of cudaMalloc'd buffers,
// every piece of scratch memory the step needs (the HEALPix direction table,
// the optical-depth field, the source-dedup workspace, one ray buffer per
// level, counters and statistics) lives in one fixed-size array in this
// file, which every GPU that loads the library holds until the process exits.
//
// The caller still owns and passes the inputs (n_H, x, sources) and the
// outputs (Gamma, heating), all device memory.
//
// Set-up: the first call on each device takes that device's address of the
// array (cudaGetSymbolAddress; in host code the array's name is only a
// host-side stand-in, not a device address) and copies the direction table
// into it with a synchronous copy, so make that first call before any stream
// capture. Every later call shares the same array and overwrites what the
// previous call left there (the counters and statistics are cleared at the
// start of each call); calls that overlap on the GPU (different streams, or
// different host threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "rt_internal.h"

using namespace nyx;

namespace {

constexpr int kNaMaxN = 32;                       // grid cells per side
constexpr int64_t kNaMaxSources = 4096;           // sources per call (before dedup)
constexpr int kNaMaxTableLevel = 7;               // highest HEALPix level the table holds
constexpr int64_t kNaRayCap = 16384;              // ray records per level buffer = children per launch
constexpr int kNaMaxLevels = kNaMaxTableLevel + 1;

constexpr size_t pad256(size_t b) { return (b + 255) / 256 * 256; }

// Layout of the array (bytes, each part 256-byte aligned).
constexpr size_t kDirEntries = 4 * ((size_t(1) << (2 * (kNaMaxTableLevel + 1))) - 1);
constexpr size_t kOffDirs = 0;
constexpr size_t kOffKap = kOffDirs + pad256(sizeof(int4) * kDirEntries);
constexpr size_t kOffStats = kOffKap + pad256(sizeof(double) * kNaMaxN * kNaMaxN * kNaMaxN);
constexpr size_t kOffCount = kOffStats + pad256(sizeof(DevStats));
constexpr size_t kOffScalar = kOffCount + pad256(sizeof(unsigned long long) * (RT_MAX_LEVELS + 1));
constexpr size_t kOffSrc = kOffScalar + 256;
constexpr size_t kSrcBytes = 12 * 3 + 8 * 3 + 8 + 4 * 4;   // per-source workspace (generous)
constexpr size_t kOffEmit = kOffSrc + pad256(kSrcBytes * kNaMaxSources) + 256 * 16;
constexpr size_t kOffRays = kOffEmit + pad256(sizeof(SrcEntry) * kNaMaxSources);
constexpr size_t kRayBytes = 6 * pad256(4 * kNaRayCap);     // 24 bytes per record, either layout
constexpr size_t kScratchBytes = kOffRays + kRayBytes * (kNaMaxLevels + 1);

// The scratch memory of rt_step_noalloc (about 8.5 MB per device).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceState {
    unsigned char* base = nullptr;   // device address of g_scratch on this device
    bool ready = false;
};
constexpr int kMaxDevices = 64;
std::mutex g_mu;
DeviceState g_dev[kMaxDevices];
int4 g_host_dirs[kDirEntries];       // host copy used once per device at set-up

// Error text goes to the caller's buffer (no allocation here either).
thread_local char* g_err = nullptr;
thread_local int g_err_len = 0;

int set_error(int code, const char* msg)
{
    if (g_err && g_err_len > 0) {
        int i = 0;
        for (; i < g_err_len - 1 && msg[i]; ++i) g_err[i] = msg[i];
        g_err[i] = 0;
    }
    return code;
}

int setup_device(int dev, unsigned char** base)
{
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState& s = g_dev[dev];
    if (!s.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) {
            cudaGetLastError();
            return set_error(RT_ECUDA, "rt_step_noalloc: cudaGetSymbolAddress of the scratch array failed");
        }
        static bool table_built = false;
        if (!table_built) {
            healpix_direction_table(kNaMaxTableLevel, g_host_dirs);
            table_built = true;
        }
        if (cudaMemcpy(static_cast<unsigned char*>(p) + kOffDirs, g_host_dirs, sizeof(g_host_dirs),
                       cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return set_error(RT_ECUDA, "rt_step_noalloc: copy of the direction table failed");
        }
        s.base = static_cast<unsigned char*>(p);
        s.ready = true;
    }
    *base = s.base;
    return RT_OK;
}

template <class R>
RayBuf<R> ray_slot(unsigned char* base, int level)
{
    unsigned char* p = base + kOffRays + kRayBytes * (size_t)level;
    RayBuf<R> b;
    b.src = reinterpret_cast<uint32_t*>(p);
    b.pix = reinterpret_cast<uint32_t*>(p + pad256(4 * kNaRayCap));
    b.P = reinterpret_cast<R*>(p + 2 * pad256(4 * kNaRayCap));
    b.tau = reinterpret_cast<R*>(p + 2 * pad256(4 * kNaRayCap) + pad256(sizeof(R) * kNaRayCap));
    if (sizeof(R) == 4) {
        b.cP = reinterpret_cast<float*>(p + 4 * pad256(4 * kNaRayCap));
        b.ctau = reinterpret_cast<float*>(p + 5 * pad256(4 * kNaRayCap));
    }
    b.cap = kNaRayCap;
    return b;
}

struct Ctx {
    cudaStream_t s;
    unsigned char* base;
    DevStats* st;
    unsigned long long* count;
    int n;
    int64_t rq;
    int64_t rs;          // periodic boundaries: travel-distance cutoff (2^-24 cells); 0: none
    int level_max;
    int table_level;
    int64_t n_emit;
    const void* kap;
    double* gamma;
    double tau_max;
    int overlap_mode;
    int hash;
    int launches;
};

// Level recursion with children processed in slices of at most kNaRayCap,
// so each level's buffer never holds more than kNaRayCap parents.
template <class R>
int na_level(Ctx& c, int level, int64_t nparents)
{
    const int64_t total = level == 0 ? 12 * c.n_emit : 4 * nparents;
    if (total <= 0) return RT_OK;
    if (level > c.table_level) return set_error(RT_EDEVICE, "rt_step_noalloc: ray level beyond the table");
    const bool can_split = level + 1 <= c.level_max;
    for (int64_t c0 = 0; c0 < total; c0 += kNaRayCap) {
        const int64_t c1 = std::min(total, c0 + kNaRayCap);
        if (cudaMemsetAsync(c.count + level + 1, 0, sizeof(unsigned long long), c.s) != cudaSuccess)
            return set_error(RT_ECUDA, "rt_step_noalloc: counter clear failed");
        MarchArgs<R> a;
        a.level = level;
        a.n = c.n;
        a.c0 = c0;
        a.c1 = c1;
        a.dirs = reinterpret_cast<const int4*>(c.base + kOffDirs) + healpix_level_offset(level);
        a.src = reinterpret_cast<const SrcEntry*>(c.base + kOffEmit);
        a.in = ray_slot<R>(c.base, level);
        a.out = can_split ? ray_slot<R>(c.base, level + 1) : RayBuf<R>();
        a.out_count = c.count + level + 1;
        a.kap = static_cast<const R*>(c.kap);
        a.gamma = c.gamma;
        a.rq = c.rq;
        a.rs = c.rs;
        a.level_max = c.level_max;
        a.tau_max = (R)c.tau_max;
        a.overlap_mode = c.overlap_mode;
        a.hash = c.hash;
        a.st = c.st;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((c1 - c0 + 255) / 256, 152 * 8));
        if constexpr (sizeof(R) == 8) c.launches += launch_march_f64(a, grid, 256, c.s);
        else c.launches += launch_march_f32(a, grid, 256, c.s);
        if (cudaGetLastError() != cudaSuccess) return set_error(RT_ECUDA, "rt_step_noalloc: march launch failed");
        unsigned long long next = 0;
        unsigned err = 0;
        if (cudaMemcpyAsync(&next, c.count + level + 1, sizeof(next), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
            cudaMemcpyAsync(&err, &c.st->err, sizeof(err), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
            cudaStreamSynchronize(c.s) != cudaSuccess) {
            cudaGetLastError();
            return set_error(RT_ECUDA, "rt_step_noalloc: march failed");
        }
        if (err) return set_error(RT_EDEVICE, "rt_step_noalloc: march kernel reported an internal error");
        if (next > 0) {
            int rc = na_level<R>(c, level + 1, (int64_t)next);
            if (rc) return rc;
        }
    }
    return RT_OK;
}

}  // namespace

extern "C" int rt_step_noalloc(const rt_config* cfg, void* cuda_stream, const double* n_H, const double* x_ion,
                               const int32_t* cell_ijk, const double* ndot, int64_t nsrc, double* gamma_out,
                               double* heat_out, rt_stats* st, char* err, int32_t err_len)
{
    g_err = err;
    g_err_len = err_len;
    set_error(RT_OK, "");
    if (!cfg || !n_H || !x_ion || !gamma_out || nsrc < 0 || (nsrc > 0 && (!cell_ijk || !ndot)))
        return set_error(RT_EINVAL, "rt_step_noalloc: missing argument");
    const int n = cfg->n;
    if (n < 1 || n > kNaMaxN) return set_error(RT_EINVAL, "rt_step_noalloc: n must be in 1..32");
    if (nsrc > kNaMaxSources) return set_error(RT_EINVAL, "rt_step_noalloc: at most 4096 sources per call");
    if (cfg->merge_mode != RT_MERGE_OFF || cfg->chem_iterate || cfg->spectrum != RT_SPECTRUM_GRAY)
        return set_error(RT_EINVAL,
                         "rt_step_noalloc: source merging, chemistry and the spectrum table are not available here");
    if ((cfg->precision != RT_FP64 && cfg->precision != RT_FP32) || !(cfg->box_cm > 0) || !(cfg->sigma_cm2 > 0) ||
        !(cfg->n_min_ray >= 1.0) || !(cfg->tau_max > 0) || cfg->overlap_mode < 0 || cfg->overlap_mode > 5 ||
        (cfg->periodic != 0 && cfg->periodic != 1) || cfg->level_max > kMaxLevel)
        return set_error(RT_EINVAL, "rt_step_noalloc: invalid configuration");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return set_error(RT_ECUDA, "rt_step_noalloc: no current CUDA device");
    }
    // split radius and level cap, as in rt_create
    const double dx = cfg->box_cm / (double)n;
    const int64_t rq =
        (int64_t)std::floor(std::sqrt(3.0 / (3.141592653589793 * cfg->n_min_ray)) * (double)(1 << kRadBits) + 0.5);
    int reach = 0;
    while (std::ldexp((double)rq, reach - kRadBits) < std::sqrt(3.0) * (double)n) ++reach;
    const int level_max = cfg->level_max >= 0 ? cfg->level_max : std::min(reach + 1, kMaxLevel);
    const int table_level = std::min(level_max, reach);
    if (table_level > kNaMaxTableLevel)
        return set_error(RT_EINVAL, "rt_step_noalloc: rays would need HEALPix levels above 7 (lower n_min_ray or level_max)");

    unsigned char* base = nullptr;
    int rc = setup_device(dev, &base);
    if (rc) return rc;

    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int64_t ncell = (int64_t)n * n * n;
    Ctx c;
    c.s = s;
    c.base = base;
    c.st = reinterpret_cast<DevStats*>(base + kOffStats);
    c.count = reinterpret_cast<unsigned long long*>(base + kOffCount);
    c.n = n;
    c.rq = rq;
    c.rs = cfg->periodic ? (int64_t)std::floor(std::sqrt(3.0) * (double)n * (double)(1 << kRadBits) + 0.5) : 0;
    c.level_max = level_max;
    c.table_level = table_level;
    c.kap = base + kOffKap;
    c.gamma = gamma_out;
    c.tau_max = cfg->tau_max;
    c.overlap_mode = cfg->overlap_mode;
    c.hash = (cfg->flags & RT_FLAG_VISIT_HASH) ? 1 : 0;
    c.launches = 0;
    double* scalar = reinterpret_cast<double*>(base + kOffScalar);

    // the source workspace, carved from the array
    SourceWork w;
    unsigned char* p = base + kOffSrc;
    auto take = [&](size_t bytes) { unsigned char* r = p; p += pad256(bytes); return r; };
    w.cells_raw = reinterpret_cast<int32_t*>(const_cast<int32_t*>(cell_ijk));
    w.ndot_raw = const_cast<double*>(ndot);
    w.keys = reinterpret_cast<uint64_t*>(take(8 * kNaMaxSources));
    w.keys_b = reinterpret_cast<uint64_t*>(take(8 * kNaMaxSources));
    w.keys_c = reinterpret_cast<uint64_t*>(take(8 * kNaMaxSources));
    w.order = reinterpret_cast<int32_t*>(take(4 * kNaMaxSources));
    w.order_b = reinterpret_cast<int32_t*>(take(4 * kNaMaxSources));
    w.flag = reinterpret_cast<int32_t*>(take(4 * kNaMaxSources));
    w.head_pos = reinterpret_cast<int32_t*>(take(4 * kNaMaxSources));
    w.cells_a = reinterpret_cast<int32_t*>(take(12 * kNaMaxSources));
    w.ndot_a = reinterpret_cast<double*>(take(8 * kNaMaxSources));
    w.count = reinterpret_cast<int32_t*>(take(16));
    w.cap = kNaMaxSources;
    if (p > base + kOffEmit) return set_error(RT_EINVAL, "rt_step_noalloc: source workspace layout overflow");
    SrcEntry* emit = reinterpret_cast<SrcEntry*>(base + kOffEmit);

    auto cu = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error(RT_ECUDA, what);
            return RT_ECUDA;
        }
        return RT_OK;
    };
    if ((rc = cu(cudaMemsetAsync(c.st, 0, sizeof(DevStats), s), "rt_step_noalloc: statistics clear failed"))) return rc;
    c.launches += launch_validate_fields(n_H, x_ion, ncell, c.st, s);
    c.launches += launch_validate_sources(cell_ijk, ndot, nsrc, n, c.st, s);
    c.launches += launch_dedup_sort(w, nsrc, n, s);
    const bool want_mean = cfg->n_th_cm3 < 0;
    if (want_mean) {
        if ((rc = cu(cudaMemsetAsync(scalar, 0, sizeof(double), s), "rt_step_noalloc: clear failed"))) return rc;
        c.launches += launch_mean_nh(n_H, ncell, scalar, s);
    }
    if ((rc = cu(cudaGetLastError(), "rt_step_noalloc: launch failed"))) return rc;
    unsigned bad = 0;
    int32_t m32 = 0;
    double sum_nh = 0.0;
    if ((rc = cu(cudaMemcpyAsync(&bad, &c.st->bad_input, sizeof(bad), cudaMemcpyDeviceToHost, s), "rt_step_noalloc: read failed"))) return rc;
    if (nsrc > 0 && (rc = cu(cudaMemcpyAsync(&m32, w.count, sizeof(m32), cudaMemcpyDeviceToHost, s), "rt_step_noalloc: read failed"))) return rc;
    if (want_mean && (rc = cu(cudaMemcpyAsync(&sum_nh, scalar, sizeof(double), cudaMemcpyDeviceToHost, s), "rt_step_noalloc: read failed")))
        return rc;
    if ((rc = cu(cudaStreamSynchronize(s), "rt_step_noalloc: source stage failed"))) return rc;
    if (bad) return set_error(RT_EINVAL, "rt_step_noalloc: invalid field or source values");
    const int64_t m = nsrc > 0 ? m32 : 0;
    c.n_emit = m;
    c.launches += launch_build_emit(w, m, cfg->sigma_cm2 / (dx * dx), emit, c.st, s);
    const double n_th = want_mean ? 0.01 * (sum_nh / (double)ncell) : cfg->n_th_cm3;
    const double sdx = cfg->sigma_cm2 * dx;
    if (cfg->precision == RT_FP32)
        c.launches += launch_prepare_kappa_f32(n_H, x_ion, ncell, sdx, n_th, reinterpret_cast<float*>(base + kOffKap), s);
    else
        c.launches += launch_prepare_kappa_f64(n_H, x_ion, ncell, sdx, n_th, reinterpret_cast<double*>(base + kOffKap), s);
    if ((rc = cu(cudaMemsetAsync(gamma_out, 0, sizeof(double) * (size_t)ncell, s), "rt_step_noalloc: gamma clear failed"))) return rc;
    if ((rc = cu(cudaGetLastError(), "rt_step_noalloc: launch failed"))) return rc;
    rc = cfg->precision == RT_FP32 ? na_level<float>(c, 0, 0) : na_level<double>(c, 0, 0);
    if (rc) return rc;
    c.launches += launch_finalize(gamma_out, n_H, x_ion, ncell, cfg->e_heat_erg, dx * dx * dx, heat_out, c.st, s);
    if ((rc = cu(cudaGetLastError(), "rt_step_noalloc: finalize launch failed"))) return rc;
    DevStats d;
    if ((rc = cu(cudaMemcpyAsync(&d, c.st, sizeof(d), cudaMemcpyDeviceToHost, s), "rt_step_noalloc: stats read failed"))) return rc;
    if ((rc = cu(cudaStreamSynchronize(s), "rt_step_noalloc: step failed"))) return rc;
    if (d.err) return set_error(RT_EDEVICE, "rt_step_noalloc: a kernel reported an internal error");
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->n_src_in = nsrc;
        st->n_src_dedup = m;
        st->n_src_emit = m;
        st->chem_iters = 1;
        st->level_max = level_max;
        st->launches = c.launches;
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
        st->emitted_ph = d.emitted;
        st->absorbed_ph = d.absorbed;
        st->escaped_ph = d.escaped_ph;
        st->dropped_ph = d.dropped_ph;
        st->deposited_ph = d.deposited;
    }
    return RT_OK;
}
