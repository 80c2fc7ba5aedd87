// Per-cell kernels around the march: input validation, the absorber and
// optical-depth field (Sec. 2.6: a_abs = (1 - x) n_H; Eq. 2), the heating
// and deposited-photon reduction after the trace, and the C2-Ray
// time-averaged ionization update of Eq. 3 (Sec. 2.3). All are HBM-streaming
// grid-stride loops over the flat n^3 arrays.
#include <cstdint>

#include "rt_internal.h"

namespace nyx {
namespace {

constexpr int kBlock = 256;

int grid_for(int64_t count)
{
    int64_t g = (count + kBlock - 1) / kBlock;
    if (g > 152 * 16) g = 152 * 16;
    return g < 1 ? 1 : (int)g;
}

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double part[kBlock / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) part[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        v = lane < kBlock / 32 ? part[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

__global__ void __launch_bounds__(kBlock) validate_fields_kernel(const double* __restrict__ nh,
                                                                 const double* __restrict__ x, int64_t ncell,
                                                                 DevStats* st)
{
    unsigned bad = 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const double a = nh[c], b = x[c];
        if (!(a >= 0.0) || !isfinite(a) || !(b >= 0.0 && b <= 1.0)) ++bad;
    }
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_down_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&st->bad_input, bad);
}

// kappa = (sigma dx) ((1 - x) n_H), the optical depth per cell length.
// Stored negated (sign bit set) when the cell may not receive a secondary
// deposit under Eqs. 7-8 (n_H < n_th, or n_HI = 0). The decision chain uses
// round-to-nearest intrinsics only.
template <class R>
__global__ void __launch_bounds__(kBlock) prepare_kappa_kernel(const double* __restrict__ nh,
                                                               const double* __restrict__ x, int64_t ncell,
                                                               double sdx, double n_th, R* __restrict__ kap)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const double a = nh[c];
        const double nhi = __dmul_rn(__dsub_rn(1.0, x[c]), a);
        const double k = __dmul_rn(sdx, nhi);
        const bool elig = (a >= n_th) && (nhi > 0.0);
        const double v = elig ? k : -k;
        if constexpr (sizeof(R) == 4) kap[c] = __double2float_rn(v);
        else kap[c] = v;
    }
}

// heat = e_heat Gamma n_HI; deposited photons = sum Gamma n_HI dx^3.
__global__ void __launch_bounds__(kBlock) finalize_kernel(const double* __restrict__ gamma,
                                                          const double* __restrict__ nh,
                                                          const double* __restrict__ x, int64_t ncell,
                                                          double e_heat, double vol, double* __restrict__ heat,
                                                          DevStats* st)
{
    double dep = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const double g = gamma[c];
        const double nhi = (1.0 - x[c]) * nh[c];
        if (heat) heat[c] = e_heat * g * nhi;
        dep += g * nhi * vol;
    }
    dep = block_sum(dep);
    if (threadIdx.x == 0) atomicAdd(&st->deposited, dep);
}

// One C2-Ray update at fixed Gamma (Eq. 3): with ionization rate
// I = Gamma + n_e C_H and recombination rate R = n_e C alpha_B constant over
// dt, x(dt) = x_eq + (x0 - x_eq) e^{-dt (I+R)} and the time average
// <x> = x_eq + (x0 - x_eq) (1 - e^{-dt (I+R)}) / (dt (I+R)); n_e = <x>_prev n_H.
__global__ void __launch_bounds__(kBlock) chem_kernel(const double* __restrict__ nh, const double* __restrict__ x0,
                                                      double* __restrict__ xavg, double* __restrict__ xend,
                                                      const double* __restrict__ gamma, int64_t ncell, double dt,
                                                      double alpha_B, double C_H, double clump, DevStats* st)
{
    double md = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const double xp = xavg[c];
        const double ne = xp * nh[c];
        const double ion = gamma[c] + ne * C_H;
        const double tot = ion + ne * clump * alpha_B;
        double xe, xa;
        const double xs = x0[c];
        if (tot > 0.0) {
            const double xeq = ion / tot;
            const double u = dt * tot;
            xe = xeq + (xs - xeq) * exp(-u);
            xa = xeq + (xs - xeq) * (-expm1(-u) / u);
        } else {
            xe = xs;
            xa = xs;
        }
        md = fmax(md, fabs(xa - xp));
        xavg[c] = xa;
        xend[c] = xe;
    }
    for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_down_sync(0xffffffffu, md, o));
    // non-negative doubles order like their bit patterns: an integer max is exact
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<unsigned long long*>(&st->maxdiff), (unsigned long long)__double_as_longlong(md));
}

__global__ void __launch_bounds__(kBlock) sum_kernel(const double* __restrict__ v, int64_t ncell, double* out)
{
    double s = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x)
        s += v[c];
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

}  // namespace

int launch_validate_fields(const double* nh, const double* x, int64_t ncell, DevStats* st, cudaStream_t s)
{
    validate_fields_kernel<<<grid_for(ncell), kBlock, 0, s>>>(nh, x, ncell, st);
    return 1;
}

int launch_prepare_kappa_f64(const double* nh, const double* x, int64_t ncell, double sdx, double n_th,
                              double* kap, cudaStream_t s)
{
    prepare_kappa_kernel<double><<<grid_for(ncell), kBlock, 0, s>>>(nh, x, ncell, sdx, n_th, kap);
    return 1;
}

int launch_prepare_kappa_f32(const double* nh, const double* x, int64_t ncell, double sdx, double n_th,
                              float* kap, cudaStream_t s)
{
    prepare_kappa_kernel<float><<<grid_for(ncell), kBlock, 0, s>>>(nh, x, ncell, sdx, n_th, kap);
    return 1;
}

int launch_finalize(const double* gamma, const double* nh, const double* x, int64_t ncell, double e_heat,
                     double vol, double* heat, DevStats* st, cudaStream_t s)
{
    finalize_kernel<<<grid_for(ncell), kBlock, 0, s>>>(gamma, nh, x, ncell, e_heat, vol, heat, st);
    return 1;
}

int launch_chem_update(const double* nh, const double* x0, double* xavg, double* xend, const double* gamma,
                        int64_t ncell, double dt, double alpha_B, double C_H, double clump, DevStats* st,
                        cudaStream_t s)
{
    chem_kernel<<<grid_for(ncell), kBlock, 0, s>>>(nh, x0, xavg, xend, gamma, ncell, dt, alpha_B, C_H, clump, st);
    return 1;
}

int launch_sum_x(const double* x, int64_t ncell, DevStats* st, cudaStream_t s)
{
    sum_kernel<<<grid_for(ncell), kBlock, 0, s>>>(x, ncell, &st->xsum);
    return 1;
}

int launch_mean_nh(const double* nh, int64_t ncell, double* out, cudaStream_t s)
{
    sum_kernel<<<grid_for(ncell), kBlock, 0, s>>>(nh, ncell, out);
    return 1;
}

__global__ void __launch_bounds__(256) readback_kernel(const ReadbackList r)
{
    for (int k = 0; k < r.n; ++k)
        for (int i = threadIdx.x; i < r.words[k]; i += blockDim.x) r.dst[k][i] = r.src[k][i];
    __threadfence_system();
}

int launch_readback(const ReadbackList& r, cudaStream_t s)
{
    if (r.n == 0) return 0;
    readback_kernel<<<1, 256, 0, s>>>(r);
    return 1;
}

}  // namespace nyx
