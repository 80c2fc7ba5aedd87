// Source handling before the march (Sec. 2.8): sources that share a cell
// are merged by summing their rates, the catalog is sorted lexicographically
// by (ix, iy, iz), and optionally sources whose ionized bubbles overlap are
// merged (Alg. 3: MAX_RADIUS by shell sampling, union-find over overlapping
// pairs, one source per group at the member nearest the flux-weighted
// centroid). Catalogs are tens of thousands of entries: the sorts are stable
// LSD radix sorts in one block over only the key bits in use, and the pair
// test sweeps the pairs of the sources whose bubble radius is positive (the
// only ones that can merge); every per-group sum runs sequentially in member
// order, so the emitted catalog is deterministic.
#include <algorithm>
#include <cstdint>

#include "rt_internal.h"

namespace nyx {
namespace {

constexpr int kBlock = 256;

int blocks_for(int64_t count)
{
    const int64_t g = (count + kBlock - 1) / kBlock;
    return g < 1 ? 1 : (int)g;
}

// Bits per axis of a cell coordinate in [0, n).
int axis_bits(int n)
{
    int b = 0;
    while ((1LL << b) < (long long)n) ++b;
    return b;
}

// Lexicographic (x, y, z) key of a cell, b bits per axis.
__device__ __forceinline__ uint64_t cell_key(int x, int y, int z, int b)
{
    return ((uint64_t)x << (2 * b)) | ((uint64_t)y << b) | (uint64_t)z;
}

__global__ void validate_sources_kernel(const int32_t* __restrict__ cells, const double* __restrict__ ndot,
                                        int64_t nsrc, int n, DevStats* st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nsrc; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = cells[3 * i], y = cells[3 * i + 1], z = cells[3 * i + 2];
        const double v = ndot[i];
        if ((unsigned)x >= (unsigned)n || (unsigned)y >= (unsigned)n || (unsigned)z >= (unsigned)n || !(v > 0.0) ||
            !isfinite(v))
            atomicAdd(&st->bad_input, 1u);
    }
}

__global__ void cell_keys_kernel(const int32_t* __restrict__ cells, int64_t m, int b, uint64_t* __restrict__ keys)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = cell_key(cells[3 * i], cells[3 * i + 1], cells[3 * i + 2], b);
}

// Stable sort of keys[0..m) by their low `bits` bits: order[p] = the index of the p-th smallest,
// equal keys in index order (keys itself is left as it is; keys_b and keys_c, order_b: scratch).
// One block of 1024 threads (32 warps), least significant digit first, 8 bits a pass: warp w owns
// a contiguous chunk of the sequence; a pass counts each warp's digits, scans the counts in
// (digit, warp) order and scatters every warp's chunk in sequence order, 32 keys an iteration, a lane
// placed after the lower lanes of its iteration that share its digit (found with 8 ballots) - so
// every pass is stable and the result is the stable sort.
constexpr int kSortThreads = 1024;

__global__ void __launch_bounds__(kSortThreads) radix_sort_kernel(const uint64_t* __restrict__ keys, int64_t m,
                                                                  int bits, uint64_t* keys_b, uint64_t* keys_c,
                                                                  int32_t* order_b, int32_t* __restrict__ order)
{
    __shared__ int32_t cnt[256 * 33];      // [digit][warp], rows padded to 33 so a warp's lanes spread over banks
    __shared__ int32_t wsum[32];
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    const int64_t chunk = (m + 31) / 32;
    const int64_t c0 = min(m, (int64_t)wp * chunk), c1 = min(m, c0 + chunk);
    const int passes = (bits + 7) / 8;
    const uint64_t* kin = keys;
    const int32_t* iin = nullptr;                   // pass 0 reads the identity
    uint64_t* kout = keys_b;
    int32_t* iout = (passes & 1) ? order : order_b; // the last pass writes `order`
    for (int pass = 0; pass < passes; ++pass) {
        const int sh = 8 * pass;
        for (int q = t; q < 256 * 33; q += kSortThreads) cnt[q] = 0;
        __syncthreads();
        for (int64_t i = c0 + lane; i < c1; i += 128) {   // four independent loads in flight a lane
            uint64_t kk[4];
            for (int u = 0; u < 4; ++u) kk[u] = i + 32 * u < c1 ? kin[i + 32 * u] : 0ULL;
            for (int u = 0; u < 4; ++u)
                if (i + 32 * u < c1) atomicAdd(&cnt[((int)(kk[u] >> sh) & 255) * 33 + wp], 1);
        }
        __syncthreads();
        // exclusive scan of the 8192 counters in (digit, warp) order: thread t owns counters
        // [8t, 8t + 8), i.e. digit t / 4, warps 8 (t % 4) .. 8 (t % 4) + 7
        const int sd = t >> 2, sw = 8 * (t & 3);
        int32_t loc[8], run = 0;
        for (int q = 0; q < 8; ++q) {
            loc[q] = run;
            run += cnt[sd * 33 + sw + q];
        }
        int32_t incl = run;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[wp] = incl;
        __syncthreads();
        if (wp == 0) {
            int32_t v = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            wsum[lane] = v;                          // inclusive over warps
        }
        __syncthreads();
        const int32_t base = (incl - run) + (wp > 0 ? wsum[wp - 1] : 0);
        for (int q = 0; q < 8; ++q) cnt[sd * 33 + sw + q] = base + loc[q];
        __syncthreads();
        // scatter, each warp its chunk in order; the next iteration's key and index are requested
        // before this iteration's are placed
        uint64_t kn = c0 + lane < c1 ? kin[c0 + lane] : 0ULL;
        int32_t xn = c0 + lane < c1 ? (iin ? iin[c0 + lane] : (int32_t)(c0 + lane)) : 0;
        for (int64_t r0 = c0; r0 < c1; r0 += 32) {
            const int64_t i = r0 + lane;
            const bool v = i < c1;
            const uint64_t k = kn;
            const int32_t x = xn;
            const int64_t inext = i + 32;
            kn = inext < c1 ? kin[inext] : 0ULL;
            xn = inext < c1 ? (iin ? iin[inext] : (int32_t)inext) : 0;
            const int d = (int)(k >> sh) & 255;
            unsigned peers = __ballot_sync(0xffffffffu, v);
            for (int b = 0; b < 8; ++b) {
                const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1);
                peers &= ((d >> b) & 1) ? bb : ~bb;
            }
            int32_t* slot = &cnt[d * 33 + wp];
            if (v) {
                const int32_t dst = *slot + __popc(peers & ((1u << lane) - 1u));
                kout[dst] = k;
                iout[dst] = x;
            }
            __syncwarp();
            if (v && (peers >> lane) == 1u) *slot += __popc(peers);   // the highest lane of its digit
            __syncwarp();
        }
        __syncthreads();
        kin = kout;
        kout = (kout == keys_b) ? keys_c : keys_b;
        iin = iout;
        iout = (iout == order) ? order_b : order;
    }
    if (passes == 0)
        for (int64_t i = t; i < m; i += kSortThreads) order[i] = (int32_t)i;
}

// flag[p] = 1 where sorted entry p starts a run of equal keys.
__global__ void run_heads_kernel(const uint64_t* __restrict__ keys, const int32_t* __restrict__ order, int64_t m,
                                 uint64_t mask, int32_t* __restrict__ flag)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x)
        flag[p] = (p == 0) || ((keys[order[p]] & mask) != (keys[order[p - 1]] & mask));
}

// Exclusive prefix sum of flag[0..m) into pos, total into *total (one block).
__global__ void __launch_bounds__(1024) scan_kernel(const int32_t* __restrict__ flag, int64_t m,
                                                    int32_t* __restrict__ pos, int32_t* __restrict__ total)
{
    __shared__ int32_t sh[1024];
    const int t = threadIdx.x;
    const int64_t per = (m + 1023) / 1024;
    const int64_t b = t * per, e = (b + per < m) ? b + per : m;
    int32_t local = 0;
    for (int64_t p = b; p < e; ++p) local += flag[p];
    sh[t] = local;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int32_t v = t >= o ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += v;
        __syncthreads();
    }
    int32_t off = sh[t] - local;
    for (int64_t p = b; p < e; ++p) {
        pos[p] = off;
        off += flag[p];
    }
    if (t == 1023) *total = sh[1023];
}

// For each run head: sum the rates of the run in sorted (= input) order.
__global__ void dedup_sum_kernel(const uint64_t* __restrict__ keys, const int32_t* __restrict__ order,
                                 const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, int64_t m,
                                 const int32_t* __restrict__ cells, const double* __restrict__ ndot,
                                 int32_t* __restrict__ out_cells, double* __restrict__ out_ndot)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[p]) continue;
        const int32_t i = order[p];
        double s = ndot[i];
        for (int64_t q = p + 1; q < m && !flag[q]; ++q) s = __dadd_rn(s, ndot[order[q]]);
        const int32_t u = pos[p];
        out_cells[3 * u] = cells[3 * i];
        out_cells[3 * u + 1] = cells[3 * i + 1];
        out_cells[3 * u + 2] = cells[3 * i + 2];
        out_ndot[u] = s;
    }
}

// ---------------------------------------------------------------- Alg. 3

// Minimum-image component of a cell offset on a periodic grid of n cells
// (Sec. 2.8 computes Alg. 3 under minimum-image geometry when periodic).
__device__ __forceinline__ long long minimg(long long d, long long n)
{
    long long r = d % n;
    if (r < 0) r += n;
    return 2 * r > n ? r - n : r;
}

// MAX_RADIUS: one block per source. Shells r = dr, 2 dr, ... <= R_max are
// sampled at the HEALPix directions of the sample level; a sample is the
// cell floor(c + 1/2 + r d), wrapped into the grid when periodic; the shell's
// point set is the distinct in-grid sample cells (bitonic sort in shared
// memory, then run heads).
template <int NP2>
__global__ void __launch_bounds__(kBlock) radius_kernel(const int32_t* __restrict__ cells, int64_t m, int n,
                                                        const double* __restrict__ x, const int4* __restrict__ dirs,
                                                        int ns, double x_th, double f_req, int n_min, double dr,
                                                        double rmax, int periodic, double* __restrict__ radius)
{
    __shared__ long long key[NP2];
    __shared__ int red[2];
    const int64_t si = blockIdx.x;
    if (si >= m) return;
    const int c[3] = {cells[3 * si], cells[3 * si + 1], cells[3 * si + 2]};
    const int64_t nn = n;
    if (x[((int64_t)c[2] * nn + c[1]) * nn + c[0]] < x_th) {
        if (threadIdx.x == 0) radius[si] = 0.0;
        return;
    }
    const double inv = 1.0 / (double)(1 << kDirBits);
    double result = rmax;
    for (double r = dr; r <= rmax; r = __dadd_rn(r, dr)) {
        for (int p = threadIdx.x; p < NP2; p += blockDim.x) {
            long long k = 0x7fffffffffffffffLL;
            if (p < ns) {
                const int4 d = dirs[p];
                const int dd[3] = {d.x, d.y, d.z};
                long long q[3];
                bool inside = true;
                for (int a = 0; a < 3; ++a) {
                    const double pos = __dadd_rn(__dadd_rn((double)c[a], 0.5), __dmul_rn(r, __dmul_rn((double)dd[a], inv)));
                    q[a] = (long long)floor(pos);
                    if (periodic) q[a] = ((q[a] % nn) + nn) % nn;
                    if (q[a] < 0 || q[a] >= nn) inside = false;
                }
                if (inside) k = (q[2] * nn + q[1]) * nn + q[0];
            }
            key[p] = k;
        }
        __syncthreads();
        for (int size = 2; size <= NP2; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = threadIdx.x; t < NP2 / 2; t += blockDim.x) {
                    const int lo = 2 * t - (t & (stride - 1));
                    const int hi = lo + stride;
                    const bool up = ((lo & size) == 0);
                    const long long a = key[lo], b = key[hi];
                    if ((a > b) == up) { key[lo] = b; key[hi] = a; }
                }
                __syncthreads();
            }
        }
        if (threadIdx.x < 2) red[threadIdx.x] = 0;
        __syncthreads();
        int ntot = 0, nion = 0;
        for (int p = threadIdx.x; p < NP2; p += blockDim.x) {
            const long long k = key[p];
            if (k != 0x7fffffffffffffffLL && (p == 0 || key[p - 1] != k)) {
                ++ntot;
                if (x[k] >= x_th) ++nion;
            }
        }
        atomicAdd(&red[0], ntot);
        atomicAdd(&red[1], nion);
        __syncthreads();
        ntot = red[0];
        nion = red[1];
        bool fail;
        if (ntot < n_min) fail = nion < ntot;
        else fail = __ddiv_rn((double)nion, (double)ntot) < f_req;
        __syncthreads();
        if (fail) {
            result = __dsub_rn(r, dr);
            break;
        }
    }
    if (threadIdx.x == 0) radius[si] = result;
}

// Root of a in the union-find forest; parents are read past L1 (they change under concurrent hooks,
// which are atomicCAS on roots, so a stale read only lengthens the walk or fails a CAS that retries).
__device__ __forceinline__ int uf_find(int* parent, int a)
{
    int p = __ldcg(&parent[a]);
    while (p != a) {
        a = p;
        p = __ldcg(&parent[a]);
    }
    return a;
}

// flag[i] = 1 where source i has a positive bubble radius (only such sources can pair).
__global__ void positive_radius_kernel(const double* __restrict__ radius, int64_t m, int32_t* __restrict__ flag)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = radius[i] > 0.0 ? 1 : 0;
}

// list[pos[i]] = i for the flagged sources (in index order).
__global__ void compact_kernel(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, int64_t m,
                               int32_t* __restrict__ list)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) list[pos[i]] = (int32_t)i;
}

// Pairs of the *np_dev sources of `list` (positive radii, increasing index) whose bubbles
// overlap (d^2 <= (f_ov (r_a + r_b))^2 + eps, d minimum-image when periodic) are united; the
// larger root is hooked under the smaller, so each component's root is its smallest index. The
// np (np - 1) / 2 pairs (ia < ib) are numbered row by row, row ia holding np - 1 - ia of them,
// and the grid strides over that numbering.
__device__ __forceinline__ long long pair_row_start(long long ia, long long np)
{
    return ia * np - ia * (ia + 1) / 2;
}

__global__ void pair_union_kernel(const int32_t* __restrict__ cells, const double* __restrict__ radius,
                                  const int32_t* __restrict__ list, const int32_t* __restrict__ np_dev, int n,
                                  int periodic, double f_ov, double eps, int* parent, DevStats* st)
{
    const long long np = *np_dev;
    const long long total = np * (np - 1) / 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= total) return;
    // the row of pair k: the root of ia^2 - (2 np - 1) ia + 2 k = 0, then corrected to be exact
    const double b2 = (double)(2 * np - 1);
    long long ia = (long long)floor(0.5 * (b2 - sqrt(fmax(b2 * b2 - 8.0 * (double)k, 0.0))));
    ia = ia < 0 ? 0 : (ia > np - 2 ? np - 2 : ia);
    while (ia > 0 && pair_row_start(ia, np) > k) --ia;
    while (ia < np - 2 && pair_row_start(ia + 1, np) <= k) ++ia;
    long long ib = k - pair_row_start(ia, np) + ia + 1;
    for (; k < total; k += stride) {
        const int a = list[ia], b = list[ib];
        const double ra = radius[a], rb = radius[b];
        long long dx = cells[3 * a] - cells[3 * b], dy = cells[3 * a + 1] - cells[3 * b + 1],
                  dz = cells[3 * a + 2] - cells[3 * b + 2];
        if (periodic) {
            dx = minimg(dx, n);
            dy = minimg(dy, n);
            dz = minimg(dz, n);
        }
        const long long d2 = dx * dx + dy * dy + dz * dz;
        const double rs = __dmul_rn(f_ov, __dadd_rn(ra, rb));
        if ((double)d2 <= __dadd_rn(__dmul_rn(rs, rs), eps)) {
            int u = a, v = b;
            for (int tries = 0;; ++tries) {
                u = uf_find(parent, u);
                v = uf_find(parent, v);
                if (u == v) break;
                if (u > v) { const int t = u; u = v; v = t; }
                if (atomicCAS(&parent[v], v, u) == v) break;
                if (tries > (1 << 20)) { atomicOr(&st->err, kErrUnionFind); break; }
            }
        }
        ib += stride;                    // the pair `stride` further on: rows shrink by one each
        while (ib >= np && ia < np - 2) {
            ib -= np - ia - 2;
            ++ia;
        }
    }
}

// Key of source i: its component's root (a stable sort by it keeps members in index order).
__global__ void label_keys_kernel(int* parent, int64_t m, int32_t* __restrict__ label, uint64_t* __restrict__ keys)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = uf_find(parent, (int)i);
        label[i] = r;
        keys[i] = (uint64_t)(uint32_t)r;
    }
}

// One merged source per group (members contiguous in `order`, by index):
// summed rate, flux-weighted centroid rounded and clamped into the grid,
// snapped to the nearest member (first in order on ties). Periodic: members
// unwrapped next to the group's first member, centroid wrapped back into the
// grid, snap by minimum-image distance.
__global__ void group_kernel(const int32_t* __restrict__ order, const int32_t* __restrict__ flag,
                             const int32_t* __restrict__ pos, int64_t m, int n, int periodic,
                             const int32_t* __restrict__ cells, const double* __restrict__ ndot,
                             int32_t* __restrict__ out_cells, double* __restrict__ out_ndot)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[p]) continue;
        int64_t e = p + 1;
        while (e < m && !flag[e]) ++e;
        const int32_t g = order[p];
        double ftot = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for (int64_t q = p; q < e; ++q) {
            const int32_t j = order[q];
            const double v = ndot[j];
            long long u[3] = {cells[3 * j], cells[3 * j + 1], cells[3 * j + 2]};
            if (periodic)
                for (int a = 0; a < 3; ++a) u[a] = cells[3 * g + a] + minimg(u[a] - cells[3 * g + a], n);
            ftot = __dadd_rn(ftot, v);
            sx = __dadd_rn(sx, __dmul_rn(v, (double)u[0]));
            sy = __dadd_rn(sy, __dmul_rn(v, (double)u[1]));
            sz = __dadd_rn(sz, __dmul_rn(v, (double)u[2]));
        }
        const int32_t u = pos[p];
        if (e - p == 1) {
            out_cells[3 * u] = cells[3 * g];
            out_cells[3 * u + 1] = cells[3 * g + 1];
            out_cells[3 * u + 2] = cells[3 * g + 2];
            out_ndot[u] = ndot[g];
            continue;
        }
        long long rc[3];
        const double cs[3] = {sx, sy, sz};
        for (int a = 0; a < 3; ++a) {
            long long v = (long long)floor(__dadd_rn(__ddiv_rn(cs[a], ftot), 0.5));
            if (periodic) v = ((v % n) + n) % n;
            else v = v < 0 ? 0 : (v > n - 1 ? n - 1 : v);
            rc[a] = v;
        }
        int32_t best = -1;
        long long bestd = 0;
        for (int64_t q = p; q < e; ++q) {
            const int32_t j = order[q];
            long long d2 = 0;
            for (int a = 0; a < 3; ++a) {
                long long d = (long long)cells[3 * j + a] - rc[a];
                if (periodic) d = minimg(d, n);
                d2 += d * d;
            }
            if (best < 0 || d2 < bestd) { best = j; bestd = d2; }
        }
        out_cells[3 * u] = cells[3 * best];
        out_cells[3 * u + 1] = cells[3 * best + 1];
        out_cells[3 * u + 2] = cells[3 * best + 2];
        out_ndot[u] = ftot;
    }
}

__global__ void gather_kernel(const int32_t* __restrict__ order, int64_t m, const int32_t* __restrict__ cells,
                              const double* __restrict__ ndot, int32_t* __restrict__ out_cells,
                              double* __restrict__ out_ndot)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = order[p];
        out_cells[3 * p] = cells[3 * i];
        out_cells[3 * p + 1] = cells[3 * i + 1];
        out_cells[3 * p + 2] = cells[3 * i + 2];
        out_ndot[p] = ndot[i];
    }
}

// Entries at or beyond *count sort last.
__global__ void mask_tail_kernel(uint64_t* __restrict__ keys, int64_t m, const int32_t* __restrict__ count)
{
    const int64_t c = *count;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        if (i >= c) keys[i] = ~0ULL;
}

__global__ void iota_kernel(int* parent, int64_t m)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        parent[i] = (int)i;
}

__global__ void build_emit_kernel(const int32_t* __restrict__ cells, const double* __restrict__ ndot, int64_t m,
                                  double s_over_dx2, SrcEntry* __restrict__ out, DevStats* st)
{
    double emitted = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        SrcEntry e;
        e.cx = cells[3 * i];
        e.cy = cells[3 * i + 1];
        e.cz = cells[3 * i + 2];
        e.pad = 0;
        e.ph = __ddiv_rn(ndot[i], 12.0);
        e.gd = __dmul_rn(e.ph, s_over_dx2);
        e.gf = __double2float_rn(e.gd);
        e.pad2 = 0.f;
        out[i] = e;
        emitted += ndot[i];
    }
    for (int o = 16; o > 0; o >>= 1) emitted += __shfl_down_sync(0xffffffffu, emitted, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&st->emitted, emitted);
}

// As build_emit_kernel, with the catalog size read from the device (after
// dedup) so no host round trip is needed between dedup and emission.
__global__ void build_emit_dev_kernel(const int32_t* __restrict__ cells, const double* __restrict__ ndot,
                                      const int32_t* __restrict__ count, double s_over_dx2, SrcEntry* __restrict__ out,
                                      DevStats* st)
{
    const int64_t m = *count;
    double emitted = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        SrcEntry e;
        e.cx = cells[3 * i];
        e.cy = cells[3 * i + 1];
        e.cz = cells[3 * i + 2];
        e.pad = 0;
        e.ph = __ddiv_rn(ndot[i], 12.0);
        e.gd = __dmul_rn(e.ph, s_over_dx2);
        e.gf = __double2float_rn(e.gd);
        e.pad2 = 0.f;
        out[i] = e;
        emitted += ndot[i];
    }
    for (int o = 16; o > 0; o >>= 1) emitted += __shfl_down_sync(0xffffffffu, emitted, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&st->emitted, emitted);
}

}  // namespace

int launch_validate_sources(const int32_t* cells, const double* ndot, int64_t nsrc, int n, DevStats* st,
                             cudaStream_t s)
{
    if (nsrc <= 0) return 0;
    validate_sources_kernel<<<blocks_for(nsrc), kBlock, 0, s>>>(cells, ndot, nsrc, n, st);
    return 1;
}

int launch_dedup_sort(SourceWork& w, int64_t nsrc, int n, cudaStream_t s)
{
    if (nsrc <= 0) return 0;
    const int b = blocks_for(nsrc);
    const int ab = axis_bits(n);
    cell_keys_kernel<<<b, kBlock, 0, s>>>(w.cells_raw, nsrc, ab, w.keys);
    radix_sort_kernel<<<1, kSortThreads, 0, s>>>(w.keys, nsrc, 3 * ab, w.keys_b, w.keys_c, w.order_b, w.order);
    run_heads_kernel<<<b, kBlock, 0, s>>>(w.keys, w.order, nsrc, ~0ULL, w.flag);
    scan_kernel<<<1, 1024, 0, s>>>(w.flag, nsrc, w.head_pos, w.count);
    dedup_sum_kernel<<<b, kBlock, 0, s>>>(w.keys, w.order, w.flag, w.head_pos, nsrc, w.cells_raw, w.ndot_raw,
                                          w.cells_a, w.ndot_a);
    return 5;
}

int launch_merge(SourceWork& w, int64_t m, int n, int periodic, const double* x, const int4* samp_dirs,
                 int samp_count, double x_th, double f_req, int n_min, double dr, double rmax, double f_ov,
                 double eps, DevStats* st, cudaStream_t s)
{
    if (m <= 0) return 0;
    const int b = blocks_for(m);
    const int grid_r = (int)m;
    if (samp_count <= 1024)
        radius_kernel<1024><<<grid_r, kBlock, 0, s>>>(w.cells_a, m, n, x, samp_dirs, samp_count, x_th, f_req, n_min,
                                                      dr, rmax, periodic, w.radius);
    else
        radius_kernel<4096><<<grid_r, kBlock, 0, s>>>(w.cells_a, m, n, x, samp_dirs, samp_count, x_th, f_req, n_min,
                                                      dr, rmax, periodic, w.radius);
    iota_kernel<<<b, kBlock, 0, s>>>(w.parent, m);
    // the sources with a positive radius, compacted (label holds the list, count[1] its length)
    positive_radius_kernel<<<b, kBlock, 0, s>>>(w.radius, m, w.flag);
    scan_kernel<<<1, 1024, 0, s>>>(w.flag, m, w.head_pos, w.count + 1);
    compact_kernel<<<b, kBlock, 0, s>>>(w.flag, w.head_pos, m, w.label);
    pair_union_kernel<<<std::min(b * 64, 152 * 16), kBlock, 0, s>>>(w.cells_a, w.radius, w.label, w.count + 1, n,
                                                                     periodic, f_ov, eps, w.parent, st);
    label_keys_kernel<<<b, kBlock, 0, s>>>(w.parent, m, w.label, w.keys);
    radix_sort_kernel<<<1, kSortThreads, 0, s>>>(w.keys, m, axis_bits((int)std::min<int64_t>(m, 1LL << 30)), w.keys_b,
                                                 w.keys_c, w.order_b, w.order);
    run_heads_kernel<<<b, kBlock, 0, s>>>(w.keys, w.order, m, ~0ULL, w.flag);
    scan_kernel<<<1, 1024, 0, s>>>(w.flag, m, w.head_pos, w.count);
    group_kernel<<<b, kBlock, 0, s>>>(w.order, w.flag, w.head_pos, m, n, periodic, w.cells_a, w.ndot_a, w.cells_b,
                                      w.ndot_b);
    // final lexicographic order of the merged catalog (its size is count[0] <= m; unused tail keys sort last)
    const int ab = axis_bits(n);
    cell_keys_kernel<<<b, kBlock, 0, s>>>(w.cells_b, m, ab, w.keys);
    mask_tail_kernel<<<b, kBlock, 0, s>>>(w.keys, m, w.count);
    radix_sort_kernel<<<1, kSortThreads, 0, s>>>(w.keys, m, 3 * ab, w.keys_b, w.keys_c, w.order_b, w.order);
    gather_kernel<<<b, kBlock, 0, s>>>(w.order, m, w.cells_b, w.ndot_b, w.cells_a, w.ndot_a);
    return 15;
}

int launch_build_emit_dev(const SourceWork& w, int64_t max_m, double s_over_dx2, SrcEntry* out, DevStats* st,
                          cudaStream_t s)
{
    if (max_m <= 0) return 0;
    const int64_t g = std::min<int64_t>((max_m + kBlock - 1) / kBlock, 1024);
    build_emit_dev_kernel<<<(int)g, kBlock, 0, s>>>(w.cells_a, w.ndot_a, w.count, s_over_dx2, out, st);
    return 1;
}

int launch_build_emit(const SourceWork& w, int64_t m, double s_over_dx2, SrcEntry* out, DevStats* st,
                      cudaStream_t s)
{
    if (m <= 0) return 0;
    build_emit_kernel<<<blocks_for(m), kBlock, 0, s>>>(w.cells_a, w.ndot_a, m, s_over_dx2, out, st);
    return 1;
}

}  // namespace nyx
