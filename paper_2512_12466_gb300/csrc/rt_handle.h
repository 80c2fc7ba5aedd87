// The rt_handle struct and host-runtime helpers shared by the translation
// units behind the C ABI (rt_api.cu, batch.cu). Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "rt_internal.h"

namespace nyx {

struct DeviceGuard {
    int old = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&old);
        if (old != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (old >= 0 && cur != old) cudaSetDevice(old);
    }
};

// One level's ray records, allocated as one block.
struct RayStore {
    void* base = nullptr;
    int64_t cap = 0;
};

template <class T>
inline T* carve(char*& p, int64_t count)
{
    T* r = reinterpret_cast<T*>(p);
    p += ((sizeof(T) * (size_t)count + 255) / 256) * 256;
    return r;
}

inline size_t ray_bytes(int64_t cap, int real_size)
{
    auto pad = [](size_t b) { return ((b + 255) / 256) * 256; };
    size_t b = 2 * pad(4 * (size_t)cap) + 2 * pad((size_t)real_size * (size_t)cap);
    if (real_size == 4) b += 2 * pad(4 * (size_t)cap);
    return b;
}

template <class R>
inline RayBuf<R> ray_view(const RayStore& s)
{
    RayBuf<R> b;
    if (!s.base) return b;
    char* p = static_cast<char*>(s.base);
    b.src = carve<uint32_t>(p, s.cap);
    b.pix = carve<uint32_t>(p, s.cap);
    b.P = carve<R>(p, s.cap);
    b.tau = carve<R>(p, s.cap);
    if (sizeof(R) == 4) {
        b.cP = carve<float>(p, s.cap);
        b.ctau = carve<float>(p, s.cap);
    }
    b.cap = s.cap;
    return b;
}

}  // namespace nyx

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
// A named range on the profiler's timeline for the lifetime of the object (NVTX; free when no tool
// is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#else
struct NvtxRange {
    explicit NvtxRange(const char*) {}
};
#endif

struct rt_handle {
    rt_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 152;
    int64_t ncell = 0;
    double dx = 0, vol = 0, sdx = 0, s_over_dx2 = 0;
    int64_t rq = 0;
    int64_t rs = 0;                          // periodic: travel-distance cutoff sqrt(3) n (2^-24 cells)
    nyx::SpecTable<double> spec_d;           // RT_SPECTRUM_BLACKBODY tables (device)
    nyx::SpecTable<float> spec_f;
    int level_max = 0;
    int table_level = 0;
    const int4* dirs = nullptr;

    double* d_nh = nullptr;
    double* d_x = nullptr;
    double* d_xavg = nullptr;
    double* d_xend = nullptr;
    double* d_gamma = nullptr;
    double* d_heat = nullptr;
    void* d_kap = nullptr;
    double* d_scalar = nullptr;           // reduction scratch

    nyx::SourceWork sw;
    int64_t nsrc = 0;
    nyx::SrcEntry* d_emit = nullptr;
    int64_t n_emit = 0;
    bool catalog_valid = false;              // cells_a/ndot_a[0..n_emit) hold the catalog last traced

    nyx::RayStore rays[RT_MAX_LEVELS + 1];
    unsigned long long* d_count = nullptr;   // one per level
    nyx::DevStats* d_st = nullptr;
    void* h_pin = nullptr;                   // one pinned block holding the four below
    char* d_pin = nullptr;                   // the same block's device address (mapped)
    nyx::DevStats* h_st = nullptr;
    unsigned long long* h_count = nullptr;
    int32_t* h_i32 = nullptr;                // scratch
    double* h_f64 = nullptr;                 // scratch

    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double ms_march = 0.0;
    bool fields_set = false;
    bool sticky = false;
    int launches = 0;
    int march_launches = 0;
    int64_t table_levels = 0;        // bit l: level l read the geometry tables in the last trace
    std::string err;
    // source stage run ahead of a batch (handle_prepare_sources)
    bool src_ready = false;
    bool src_merged = false;
    int64_t src_dedup = 0;
    double src_nth = 0.0;
    double src_emitted = 0.0;
};

namespace nyx {

int fail(rt_handle* h, int code, const std::string& msg);
int cuda_fail(rt_handle* h, cudaError_t e, const char* what);
// The device address of a pointer into the handle's pinned block.
template <class T>
inline T* pinned_dev(const rt_handle* h, T* host)
{
    return reinterpret_cast<T*>(h->d_pin + (reinterpret_cast<char*>(host) - static_cast<char*>(h->h_pin)));
}
int prepare_sources(rt_handle* h, bool* merged_out, int64_t* n_dedup_out);
int ensure_directions(int device, int level, const int4** out, std::string& err);
// The geometry table of a level for grids of n cells, with the entries of the FP32 march (fp64
// false) or the FP64 one, built on stream s if needed; false if the level has none for that
// precision (over the device's table budget), so its rays are walked.
bool geometry_level(int device, long long rq, int level, int n, long long rs, const int4* dirs_level,
                    cudaStream_t s, bool fp64, GeomLevel* out);
// The RT_SPECTRUM_BLACKBODY tables at t_bb for `device` (device < 0: host table only).
int spectrum_table(int device, double t_bb, SpecTable<double>* d, SpecTable<float>* f, std::string& why);
int handle_prepare_sources(rt_handle* h);
int handle_reconfigure(rt_handle* h, const rt_config* cfg);
int sources_enqueue_many(rt_handle* const* hs, int count, int* rcs);
int sources_wait_many(rt_handle* const* hs, int count, int* rcs);
int batch_bind(rt_batch* b, rt_handle* const* handles, int32_t count);
int batch_run_direct(rt_batch* b, float* ms);
// The two halves of batch_run_direct: enqueue the run (returns once it is on the device), then
// wait for it and check it.
int batch_launch(rt_batch* b);
int batch_finish(rt_batch* b, float* ms);
void batch_fill_stats(const rt_batch* b, size_t i, float ms, rt_stats* st);
cudaStream_t batch_stream(const rt_batch* b);

}  // namespace nyx

#define RT_CUDA(h, call, what)                                      \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return nyx::cuda_fail(h, e_, what);  \
    } while (0)

#define RT_LAUNCHED(h, what)                                        \
    do {                                                            \
        cudaError_t e_ = cudaGetLastError();                        \
        if (e_ != cudaSuccess) return nyx::cuda_fail(h, e_, what);  \
    } while (0)
