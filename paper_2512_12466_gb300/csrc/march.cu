// The hot loop of the adaptive ray tracer (Sec. 2.5, Alg. 1 RAYMARCH +
// RAY_FLTR + FILTERCOPYTRANSFORM<3>, fused): one thread marches one ray of
// level l from its start sphere R_{l-1} to its split sphere R_l, cell by cell
// (Amanatides-Woo), depositing the photon-conserving photoionization rate
// (Eq. 1, gray, V_box) with the overlap correction (Eqs. 5-8) into an FP64
// grid with atomic adds, and appends the rays that reach R_l to the next
// level's buffer through a warp-aggregated counter. Children are implicit:
// a parent record (source, pixel p, budget P, tau) stands for the four
// HEALPix children 4p..4p+3 with budget P/4 (S_COPY), so splitting writes one
// record instead of four.
//
// Traversal is exact integer arithmetic on quantised directions: the k-th
// face crossing along axis a is at ray parameter T_a(k) = (2k+1) 2^20 / D_a
// and the split radius is R_l = Rq 2^l / 2^24, so which face comes next,
// where a ray starts and whether it reaches R_l are integer comparisons.
// Segment lengths are exact integers times one per-ray constant. Every
// floating-point operation that feeds a decision (tau against tau_max, the
// D_edge < L_pix/2 test) is an explicit round-to-nearest intrinsic, so the
// bookkeeping is reproducible operation by operation.
#include <cstdint>

#include "rt_internal.h"

namespace nyx {
namespace {

constexpr int S = kDirBits;
constexpr int F = kRadBits;
constexpr long long kB = 1LL << (S - 1 + F);

template <class R>
struct Ieee;

template <>
struct Ieee<double> {
    __device__ __forceinline__ static double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ __forceinline__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ __forceinline__ static double sub(double a, double b) { return __dsub_rn(a, b); }
    __device__ __forceinline__ static double div(double a, double b) { return __ddiv_rn(a, b); }
    __device__ __forceinline__ static double of(long long v) { return __ll2double_rn(v); }
    __device__ __forceinline__ static double small(unsigned v) { return __uint2double_rn(v); }
    __device__ __forceinline__ static double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }
    __device__ __forceinline__ static double em1(double x) { return expm1(x); }
    __device__ __forceinline__ static double qdiv(double a, double b) { return a / b; }
    __device__ __forceinline__ static bool neg(double x) { return __double_as_longlong(x) < 0; }
    __device__ __forceinline__ static double mag(double x) { return fabs(x); }
};

template <>
struct Ieee<float> {
    __device__ __forceinline__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ __forceinline__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ __forceinline__ static float sub(float a, float b) { return __fsub_rn(a, b); }
    __device__ __forceinline__ static float div(float a, float b) { return __fdiv_rn(a, b); }
    __device__ __forceinline__ static float of(long long v) { return __ll2float_rn(v); }
    // exact for 0 <= v < 2^23: 2^23 + v is representable, so (2^23 | v) - 2^23 = v
    __device__ __forceinline__ static float small(unsigned v)
    {
        return __fsub_rn(__uint_as_float(0x4b000000u | v), 8388608.0f);
    }
    __device__ __forceinline__ static float pow2(int e) { return __int_as_float((127 + e) << 23); }
    __device__ __forceinline__ static float em1(float x) { return expm1f(x); }
    __device__ __forceinline__ static float qdiv(float a, float b) { return __fdividef(a, b); }
    __device__ __forceinline__ static bool neg(float x) { return __float_as_int(x) < 0; }
    __device__ __forceinline__ static float mag(float x) { return fabsf(x); }
};

// splitmix64 output function (Steele, Lea & Flood 2014), for the visit hash.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z ^= z >> 30;
    z *= 0xbf58476d1ce4e5b9ULL;
    z ^= z >> 27;
    z *= 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return z;
}

template <class T>
__device__ __forceinline__ T pick3(int i, T a, T b, T c)
{
    return i == 0 ? a : (i == 1 ? b : c);
}

// s += v with Kahan compensation c (FP32 march) or plain (FP64 march).
template <class R>
__device__ __forceinline__ void budget_add(R& s, R& c, R v)
{
    using I = Ieee<R>;
    if constexpr (sizeof(R) == 4) {
        const R y = I::sub(v, c);
        const R t = I::add(s, y);
        c = I::sub(I::sub(t, s), y);
        s = t;
    } else {
        s = I::add(s, v);
    }
}

// Exact float -> double widening with integer operations only: GB300's FP64
// pipe is small, and a conversion per deposit would make it the bottleneck.
__device__ __forceinline__ double widen(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned sign = u >> 31;
    int e = (int)((u >> 23) & 0xffu);
    unsigned m = u & 0x7fffffu;
    if (e == 0) {
        if (m == 0) return __longlong_as_double((long long)((unsigned long long)sign << 63));
        const int sh = __clz(m) - 8;          // normalise a subnormal
        m = (m << sh) & 0x7fffffu;
        e = 1 - sh;
    }
    const unsigned long long bits = ((unsigned long long)sign << 63) |
                                    ((unsigned long long)(unsigned)(e + 896) << 52) |
                                    ((unsigned long long)m << 29);
    return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double widen(double x) { return x; }

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <class R>
__global__ void __launch_bounds__(256, 2) march_kernel(const MarchArgs<R> A)
{
    using I = Ieee<R>;
    const int l = A.level;
    const int n = A.n;
    const int lane = threadIdx.x & 31;
    const long long gwarp = (long long)(blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarp = (long long)(gridDim.x * blockDim.x) >> 5;

    unsigned c_rays = 0, c_split = 0, c_esc = 0, c_dtau = 0, c_dlev = 0, c_seg = 0, c_sec = 0;
    unsigned long long c_hash = 0;
    double c_abs = 0.0, c_escph = 0.0, c_dropph = 0.0;

    const long long rq_end = A.rq << l;
    const long long rq_start = l > 0 ? (A.rq << (l - 1)) : 0;
    const R pV = I::pow2(-(S - 1 + F)), pI = I::pow2(-S), pU = I::pow2(-(S + 1));

    for (long long base = A.c0 + gwarp * 32; base < A.c1; base += nwarp * 32) {
        const long long j = base + lane;
        bool split = false;
        uint32_t o_src = 0, o_pix = 0;
        R o_P = 0, o_tau = 0;
        float o_cP = 0.f, o_ctau = 0.f;
        if (j < A.c1) {
            // ---- the ray: level-0 emission (12 per source) or a child of a parent record
            uint32_t si, pix;
            R P, tau, cP = 0, ctau = 0;
            if (l == 0) {
                si = (uint32_t)(j / 12);
                pix = (uint32_t)(j - 12LL * si);
                P = (R)1;
                tau = (R)0;
            } else {
                const long long q = j >> 2;
                si = A.in.src[q];
                pix = 4u * A.in.pix[q] + (uint32_t)(j & 3);
                P = I::mul(A.in.P[q], (R)0.25);
                tau = A.in.tau[q];
                if constexpr (sizeof(R) == 4) {
                    cP = I::mul(A.in.cP[q], 0.25f);
                    ctau = A.in.ctau[q];
                }
            }
            const SrcEntry se = A.src[si];
            const int4 dv = A.dirs[pix];
            const unsigned D0 = (unsigned)abs(dv.x), D1 = (unsigned)abs(dv.y), D2 = (unsigned)abs(dv.z);
            const int s0 = dv.x < 0 ? -1 : 1, s1 = dv.y < 0 ? -1 : 1, s2 = dv.z < 0 ? -1 : 1;

            // ---- integer event bookkeeping: crossings done at the start sphere, and before the split sphere
            int k0 = 0, k1 = 0, k2 = 0;
            if (l > 0) {
                k0 = (int)((rq_start * D0 + kB) >> (S + F));
                k1 = (int)((rq_start * D1 + kB) >> (S + F));
                k2 = (int)((rq_start * D2 + kB) >> (S + F));
            }
            const int ke0 = (int)(((rq_end * D0 + kB - 1) >> (S - 1 + F)) >> 1);
            const int ke1 = (int)(((rq_end * D1 + kB - 1) >> (S - 1 + F)) >> 1);
            const int ke2 = (int)(((rq_end * D2 + kB - 1) >> (S - 1 + F)) >> 1);
            int i0 = se.cx + s0 * k0, i1 = se.cy + s1 * k1, i2 = se.cz + s2 * k2;
            // A_ab = (2 k_a + 1) D_b: the next crossing on a comes before the one on b iff A_ab < A_ba.
            // With k_a <= t D_a / 2^21 + 1/2 and D_a D_b <= 2^41, A_ab <= t 2^21 + 2^22, which stays
            // below 2^32 while the ray parameter t is below 2040 (any point of a grid up to 1024^3).
            unsigned A01 = (2u * k0 + 1u) * D1, A10 = (2u * k1 + 1u) * D0;
            unsigned A02 = (2u * k0 + 1u) * D2, A20 = (2u * k2 + 1u) * D0;
            unsigned A12 = (2u * k1 + 1u) * D2, A21 = (2u * k2 + 1u) * D1;

            // ---- per-ray constants
            R nrm;
            if constexpr (sizeof(R) == 4) {
                nrm = __int_as_float(dv.w);
            } else {
                const long long nn = (long long)D0 * D0 + (long long)D1 * D1 + (long long)D2 * D2;
                nrm = __dmul_rn(__dsqrt_rn(__ll2double_rn(nn)), I::pow2(-S));
            }
            const R two20 = (R)(1 << (S - 1));
            const R h0 = D0 ? I::div(two20, (R)D0) : (R)0;
            const R h1 = D1 ? I::div(two20, (R)D1) : (R)0;
            const R h2 = D2 ? I::div(two20, (R)D2) : (R)0;
            const R W01 = (D0 && D1) ? I::div(h0, (R)D1) : (R)0;
            const R W02 = (D0 && D2) ? I::div(h0, (R)D2) : (R)0;
            const R W12 = (D1 && D2) ? I::div(h1, (R)D2) : (R)0;
            const R u0 = I::mul((R)D0, pU), u1 = I::mul((R)D1, pU), u2 = I::mul((R)D2, pU);
            const R Lc = I::mul(I::mul(nrm, (R)kSqrtPiOver3), I::pow2(-l));
            R G;
            if constexpr (sizeof(R) == 4) G = se.gf; else G = se.gd;
            const double ph = se.ph;
            const R taumax = A.tau_max;
            const unsigned long long rbase =
                A.hash ? mix64(((unsigned long long)si << 36) | ((unsigned long long)l << 31) | pix) : 0ULL;

            R Ab = 0, cA = 0;           // photons absorbed by this ray (units of ph)
            ++c_rays;
            const bool inside0 = (unsigned)i0 < (unsigned)n && (unsigned)i1 < (unsigned)n && (unsigned)i2 < (unsigned)n;
            if (!inside0) {
                ++c_esc;
                c_escph += ph * (widen(P) - widen(cP));
            }
            unsigned seq = 0;

            // One segment of length ds_p (ray parameter) in the current cell, ending at parameter
            // tnext, where the distance to the exit face along axis b is dn_b: deposit Gamma (Eq. 1,
            // gray, V_box) with the overlap correction (Eqs. 5-8), then update the budgets.
            auto segment = [&](R ds_p, R dn0, R dn1, R dn2, R tnext) {
                const R ds = I::mul(ds_p, nrm);
                const int cell = (i2 * n + i1) * n + i0;
                const R kraw = A.kap[cell];
                const R kap = I::mag(kraw);
                const R dtau = I::mul(kap, ds);
                R a, gseg;
                if (kap > (R)0) {
                    a = P * (-I::em1(-dtau));
                    gseg = I::qdiv(a * G, kap);
                } else {
                    a = (R)0;
                    gseg = (P * G) * ds;
                }
                R f = (R)1, g2 = (R)0;
                int nbcell = -1;
                if (A.overlap_mode != RT_OVERLAP_NONE) {
                    // distances from the segment midpoint to the six faces, order x-, x+, y-, y+, z-, z+
                    const R d0 = I::add(dn0, I::mul(ds_p, u0));
                    const R d1 = I::add(dn1, I::mul(ds_p, u1));
                    const R d2 = I::add(dn2, I::mul(ds_p, u2));
                    const R o0 = I::sub((R)1, d0), o1 = I::sub((R)1, d1), o2 = I::sub((R)1, d2);
                    R dl[6];
                    dl[0] = s0 > 0 ? o0 : d0;
                    dl[1] = s0 > 0 ? d0 : o0;
                    dl[2] = s1 > 0 ? o1 : d1;
                    dl[3] = s1 > 0 ? d1 : o1;
                    dl[4] = s2 > 0 ? o2 : d2;
                    dl[5] = s2 > 0 ? d2 : o2;
                    int face = 0;
                    R De = dl[0];
                    #pragma unroll
                    for (int q = 1; q < 6; ++q) {
                        if (dl[q] < De) { De = dl[q]; face = q; }
                    }
                    const R tm = I::sub(tnext, I::mul(ds_p, (R)0.5));
                    const R Lpix = I::mul(tm, Lc);
                    if (I::add(De, De) < Lpix) {
                        if (A.overlap_mode == RT_OVERLAP_LINEAR) {
                            f = (R)0.5 + I::qdiv(De, Lpix);
                        } else if (A.overlap_mode == RT_OVERLAP_SQUARED) {
                            f = (R)0.5 + I::qdiv(De, Lpix);
                            f = f * f;
                        } else {
                            int j0 = i0, j1 = i1, j2 = i2;
                            const int step = (face & 1) ? 1 : -1;
                            if ((face >> 1) == 0) j0 += step; else if ((face >> 1) == 1) j1 += step; else j2 += step;
                            if ((unsigned)j0 < (unsigned)n && (unsigned)j1 < (unsigned)n && (unsigned)j2 < (unsigned)n) {
                                const int c2 = (j2 * n + j1) * n + j0;
                                const R kn_raw = A.kap[c2];
                                const R kn = I::mag(kn_raw);
                                const bool elig = (A.overlap_mode == RT_OVERLAP_CONSERVATIVE) ? (!I::neg(kn_raw) && kn > (R)0)
                                                                                               : (kn > (R)0);
                                if (elig) {
                                    f = (R)0.5 + I::qdiv(De, Lpix);
                                    g2 = (((R)1 - f) * gseg) * I::qdiv(kap, kn);
                                    nbcell = c2;
                                }
                            }
                        }
                    }
                }
                atomicAdd(&A.gamma[cell], widen(f * gseg));
                if (nbcell >= 0) {
                    atomicAdd(&A.gamma[nbcell], widen(g2));
                    ++c_sec;
                }
                budget_add(tau, ctau, dtau);
                budget_add(P, cP, -a);
                budget_add(Ab, cA, a);
                ++c_seg;
                if (A.hash) c_hash += mix64(rbase ^ ((unsigned long long)seq << 40) ^ (unsigned long long)cell);
                ++seq;
            };

            if (inside0) {
                // first event: the smallest next crossing (ties x, y, z), or the split sphere
                int w = 0;
                if (A10 < A01) w = 1;
                if (w == 0 ? (A20 < A02) : (A21 < A12)) w = 2;
                int kw = pick3(w, k0, k1, k2);
                bool is_end = !(kw < pick3(w, ke0, ke1, ke2));
                int prev = -1, kprev = 0;
                R ds_p = (R)0;
                if (!is_end) {               // from the start sphere to the first crossing
                    const unsigned Dw = pick3(w, D0, D1, D2);
                    const long long num = (long long)(2 * kw + 1) * kB - rq_start * (long long)Dw;
                    ds_p = I::mul(I::of(num), I::mul(pick3(w, h0, h1, h2), pV));
                }
                bool alive = true;
                // ---- segments that end on a face crossing
                while (!is_end) {
                    const R hw = pick3(w, h0, h1, h2);
                    const R invw = I::mul(hw, pI);
                    // exit-point distance to the exit face along b: (A_bw - A_wb) / (2 D_w), 0 on b = w
                    R dn0 = (R)0, dn1 = (R)0, dn2 = (R)0;
                    if (w == 0) {
                        dn1 = I::mul(I::small(A10 - A01), invw);
                        dn2 = I::mul(I::small(A20 - A02), invw);
                    } else if (w == 1) {
                        dn0 = I::mul(I::small(A01 - A10), invw);
                        dn2 = I::mul(I::small(A21 - A12), invw);
                    } else {
                        dn0 = I::mul(I::small(A02 - A20), invw);
                        dn1 = I::mul(I::small(A12 - A21), invw);
                    }
                    segment(ds_p, dn0, dn1, dn2, I::mul(I::small(2u * kw + 1u), hw));
                    if (tau >= taumax) {             // photons spent
                        ++c_dtau;
                        c_dropph += ph * (widen(P) - widen(cP));
                        c_abs += ph * (widen(Ab) - widen(cA));
                        alive = false;
                        break;
                    }
                    // step every axis whose crossing coincides with the winner's
                    const bool t0 = (w == 0) || (w == 1 ? A01 == A10 : A02 == A20);
                    const bool t1 = (w == 1) || (w == 0 ? A10 == A01 : A12 == A21);
                    const bool t2 = (w == 2) || (w == 0 ? A20 == A02 : A21 == A12);
                    if (t0) { ++k0; i0 += s0; A01 += 2u * D1; A02 += 2u * D2; }
                    if (t1) { ++k1; i1 += s1; A10 += 2u * D0; A12 += 2u * D2; }
                    if (t2) { ++k2; i2 += s2; A20 += 2u * D0; A21 += 2u * D1; }
                    prev = w;
                    kprev = kw;
                    if (!((unsigned)i0 < (unsigned)n && (unsigned)i1 < (unsigned)n && (unsigned)i2 < (unsigned)n)) {
                        ++c_esc;
                        c_escph += ph * (widen(P) - widen(cP));
                        c_abs += ph * (widen(Ab) - widen(cA));
                        alive = false;
                        break;
                    }
                    // next event
                    w = 0;
                    if (A10 < A01) w = 1;
                    if (w == 0 ? (A20 < A02) : (A21 < A12)) w = 2;
                    kw = pick3(w, k0, k1, k2);
                    is_end = !(kw < pick3(w, ke0, ke1, ke2));
                    if (!is_end) {
                        if (prev == w) {
                            const R h = pick3(w, h0, h1, h2);
                            ds_p = I::add(h, h);
                        } else {
                            // (2 k_w + 1) D_p - (2 k_prev + 1) D_w, with k_p = k_prev + 1 now; in [1, 2^22]
                            const int pair = prev + w;
                            const unsigned Dw = pick3(w, D0, D1, D2);
                            const unsigned Awp = pair == 1 ? (w == 0 ? A01 : A10) : (pair == 2 ? (w == 0 ? A02 : A20) : (w == 1 ? A12 : A21));
                            const unsigned Apw = pair == 1 ? (w == 0 ? A10 : A01) : (pair == 2 ? (w == 0 ? A20 : A02) : (w == 1 ? A21 : A12));
                            ds_p = I::mul(I::small(Awp - (Apw - 2u * Dw)), pair == 1 ? W01 : (pair == 2 ? W02 : W12));
                        }
                    }
                }
                if (alive) {
                    // ---- the last segment ends on the split sphere R_l, where k_b = kend_b on every axis
                    if (prev < 0) {
                        ds_p = I::mul((R)A.rq, I::pow2(l > 0 ? l - 1 - F : -F));
                    } else {
                        const long long num = rq_end * (long long)pick3(prev, D0, D1, D2) - (long long)(2 * kprev + 1) * kB;
                        ds_p = I::mul(I::of(num), I::mul(pick3(prev, h0, h1, h2), pV));
                    }
                    const R pE = I::pow2(-(S + F));
                    const R e0 = I::mul(I::of((long long)(2 * ke0 + 1) * kB - rq_end * (long long)D0), pE);
                    const R e1 = I::mul(I::of((long long)(2 * ke1 + 1) * kB - rq_end * (long long)D1), pE);
                    const R e2 = I::mul(I::of((long long)(2 * ke2 + 1) * kB - rq_end * (long long)D2), pE);
                    segment(ds_p, e0, e1, e2, I::mul((R)A.rq, I::pow2(l - F)));
                    if (tau >= taumax) {
                        ++c_dtau;
                        c_dropph += ph * (widen(P) - widen(cP));
                        c_abs += ph * (widen(Ab) - widen(cA));
                    } else {
                        c_abs += ph * (widen(Ab) - widen(cA));
                        if (l + 1 > A.level_max) {
                            ++c_dlev;
                            c_dropph += ph * (widen(P) - widen(cP));
                        } else {
                            ++c_split;
                            split = true;
                            o_src = si;
                            o_pix = pix;
                            o_P = P;
                            o_tau = tau;
                            if constexpr (sizeof(R) == 4) {
                                o_cP = cP;
                                o_ctau = ctau;
                            }
                        }
                    }
                }
            }
        }
        // ---- warp-aggregated append of the rays that split (Alg. 1 FILTERCOPYTRANSFORM<3>)
        const unsigned m = __ballot_sync(0xffffffffu, split);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned long long pos0 = 0;
            if (lane == leader) pos0 = atomicAdd(A.out_count, (unsigned long long)__popc(m));
            pos0 = __shfl_sync(0xffffffffu, pos0, leader);
            if (split) {
                const unsigned long long pos = pos0 + __popc(m & ((1u << lane) - 1u));
                if (pos < (unsigned long long)A.out.cap) {
                    A.out.src[pos] = o_src;
                    A.out.pix[pos] = o_pix;
                    A.out.P[pos] = o_P;
                    A.out.tau[pos] = o_tau;
                    if constexpr (sizeof(R) == 4) {
                        A.out.cP[pos] = o_cP;
                        A.out.ctau[pos] = o_ctau;
                    }
                } else {
                    atomicOr(&A.st->err, kErrRayOverflow);
                }
            }
        }
    }

    // ---- statistics and photon ledger: one atomic per warp and counter
    const unsigned long long r_rays = warp_sum((unsigned long long)c_rays);
    const unsigned long long r_split = warp_sum((unsigned long long)c_split);
    const unsigned long long r_esc = warp_sum((unsigned long long)c_esc);
    const unsigned long long r_dtau = warp_sum((unsigned long long)c_dtau);
    const unsigned long long r_dlev = warp_sum((unsigned long long)c_dlev);
    const unsigned long long r_seg = warp_sum((unsigned long long)c_seg);
    const unsigned long long r_sec = warp_sum((unsigned long long)c_sec);
    c_hash = warp_sum(c_hash);
    c_abs = warp_sum(c_abs);
    c_escph = warp_sum(c_escph);
    c_dropph = warp_sum(c_dropph);
    if (lane == 0 && r_rays) {
        DevStats* st = A.st;
        atomicAdd(&st->rays[l], r_rays);
        if (r_split) atomicAdd(&st->splits[l], r_split);
        if (r_esc) atomicAdd(&st->escaped[l], r_esc);
        if (r_dtau) atomicAdd(&st->dropped_tau[l], r_dtau);
        if (r_dlev) atomicAdd(&st->dropped_level[l], r_dlev);
        atomicAdd(&st->segments[l], r_seg);
        if (r_sec) atomicAdd(&st->secondary[l], r_sec);
        if (c_hash) atomicAdd(&st->visit_hash, c_hash);
        atomicAdd(&st->absorbed, c_abs);
        atomicAdd(&st->escaped_ph, c_escph);
        atomicAdd(&st->dropped_ph, c_dropph);
    }
}

}  // namespace

int launch_march_f64(const MarchArgs<double>& a, int grid, int block, cudaStream_t s)
{
    march_kernel<double><<<grid, block, 0, s>>>(a);
    return 1;
}

int launch_march_f32(const MarchArgs<float>& a, int grid, int block, cudaStream_t s)
{
    march_kernel<float><<<grid, block, 0, s>>>(a);
    return 1;
}

}  // namespace nyx
