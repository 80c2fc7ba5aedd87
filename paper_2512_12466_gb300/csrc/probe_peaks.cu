// Throughput probe (a measurement tool beside the library, not part of its ABI): fused
// multiply-add throughput of the FP32 and FP64 pipes on the current device, the denominators of
// the march kernels' ALU rooflines, and FP64 atomic-add throughput, the denominator of their
// deposit roofline. Every thread runs eight independent FMA chains (enough to
// cover the pipe latency at full occupancy); the grid fills every SM; the kernel is timed with
// CUDA events after a warm-up launch. One FMA counts two floating-point operations.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

template <class T>
__global__ void __launch_bounds__(256) fma_chains(const T a, const T b, const int64_t iters, T* out)
{
    T x0 = (T)threadIdx.x, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int64_t i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b);
        x1 = fma(x1, a, b);
        x2 = fma(x2, a, b);
        x3 = fma(x3, a, b);
        x4 = fma(x4, a, b);
        x5 = fma(x5, a, b);
        x6 = fma(x6, a, b);
        x7 = fma(x7, a, b);
    }
    // one store per thread keeps every chain live
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

template <class T>
int run(const int64_t iters, double* tflops, double* ms_out)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -3;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chains<T>, 256, 0) != cudaSuccess || per_sm < 1)
        return -3;
    const int grid = sms * per_sm;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * (size_t)grid * 256) != cudaSuccess) return -2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = (T)0.999999, b = (T)1e-7;
    fma_chains<T><<<grid, 256>>>(a, b, iters / 8 + 1, out);                      // warm-up
    cudaEventRecord(e0);
    fma_chains<T><<<grid, 256>>>(a, b, iters, out);
    cudaEventRecord(e1);
    const cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return -3;
    const double flops = 2.0 * 8.0 * (double)iters * (double)grid * 256.0;
    *tflops = flops / ((double)ms * 1e-3) / 1e12;
    *ms_out = ms;
    return 0;
}

// FP64 atomic adds whose result is unused (reductions performed in L2), as the march's deposits
// are: each thread adds `iters` times into an array of n doubles, at addresses spread by a hash
// (pattern 0: every lane of a warp a different, random cell), consecutive within a warp (pattern
// 1: the lanes of a warp cover 32 neighbouring cells), or shared by groups of lanes (pattern 2:
// groups of 4 lanes add to one random cell; pattern 3: groups of 16), as rays of one source that
// cross the same cell in the same step do.
__global__ void __launch_bounds__(256) red_f64(double* __restrict__ a, const int64_t n, const int64_t iters,
                                                const int pattern)
{
    const uint64_t gid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (int64_t i = 0; i < iters; ++i) {
        uint64_t k;
        if (pattern == 0 || pattern >= 2) {
            const uint64_t g = pattern == 2 ? gid >> 2 : (pattern == 3 ? gid >> 4 : gid);
            uint64_t z = g * 0x9e3779b97f4a7c15ULL + (uint64_t)i * 0xbf58476d1ce4e5b9ULL;
            z ^= z >> 31;
            z *= 0x94d049bb133111ebULL;
            z ^= z >> 29;
            k = z % (uint64_t)n;
        } else {
            k = ((gid >> 5) * 0x9e3779b97f4a7c15ULL + (uint64_t)i * 40503ULL) % (uint64_t)(n / 32) * 32 + (gid & 31);
        }
        atomicAdd(a + k, 1.0);
    }
}

int run_red(const int64_t n, const int64_t iters, const int pattern, double* per_s, double* ms_out)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -3;
    double* a = nullptr;
    if (cudaMalloc(&a, sizeof(double) * (size_t)n) != cudaSuccess) return -2;
    cudaMemset(a, 0, sizeof(double) * (size_t)n);
    const int grid = sms * 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    red_f64<<<grid, 256>>>(a, n, iters / 8 + 1, pattern);                    // warm-up
    cudaEventRecord(e0);
    red_f64<<<grid, 256>>>(a, n, iters, pattern);
    cudaEventRecord(e1);
    const cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(a);
    if (err != cudaSuccess) return -3;
    *per_s = (double)iters * grid * 256.0 / ((double)ms * 1e-3);
    *ms_out = ms;
    return 0;
}

}  // namespace

extern "C" {

// FP64 atomic adds per second into an array of n doubles (n >= 32, a multiple of 32), pattern 0
// random cells, 1 neighbouring cells per warp, 2 and 3 one random cell per group of 4 and 16 lanes;
// `iters` adds per thread. 0 on success.
int nyxrt_probe_red_f64(int64_t n, int64_t iters, int pattern, double* per_s, double* ms)
{
    if (!per_s || !ms || iters < 1 || n < 32 || n % 32 || pattern < 0 || pattern > 3) return -1;
    return run_red(n, iters, pattern, per_s, ms);
}


// FMA throughput of one precision (32: FP32, 64: FP64) over `iters` iterations of eight chains per
// thread: *tflops = 2 x FMAs / kernel time, *ms the kernel time. 0 on success, a negative code if
// a CUDA call failed or the precision is not 32 or 64.
int nyxrt_probe_fma(int bits, int64_t iters, double* tflops, double* ms)
{
    if (!tflops || !ms || iters < 1) return -1;
    if (bits == 32) return run<float>(iters, tflops, ms);
    if (bits == 64) return run<double>(iters, tflops, ms);
    return -1;
}

}  // extern "C"
