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
#include <cooperative_groups.h>

#include <algorithm>

#include <cstdint>

#include "rt_internal.h"
#include "dfloat.h"
#include "rate_table.h"

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
    __device__ __forceinline__ static double mn(double a, double b) { return fmin(a, b); }
    // photons absorbed per unit budget over optical depth x >= 0: 1 - e^{-x}
    __device__ __forceinline__ static double absorb(double x) { return -expm1(-x); }
    __device__ __forceinline__ static double qdiv(double a, double b) { return a / b; }
    // Eq. 1 for a segment of optical depth dtau = kap ds, kap > 0: photons absorbed a = P (1 - e^{-dtau})
    // and rate gseg = a G / kap. Below dtau = 2 both come from g(y) = (1 - e^{-y}) / y: a = P dtau g
    // and gseg = P G ds g, with no exponential and no division on GB300's small FP64 unit. g is the
    // degree-13 Chebyshev interpolant of g(1 + t) on t in [-1, 1] (coefficients from
    // gen_rate_poly.py, highest degree first), evaluated by Horner's rule in t = dtau - 1: within
    // 2.4e-16 of g relative over [0, 2). The bound is wide enough that a warp's lanes seldom split
    // between the two forms. Above it, expm1 and the quotient.
    __device__ __forceinline__ static void rate(double P, double G, double kap, double ds, double dtau, double& a,
                                                double& gseg)
    {
        if (lt(dtau, 2.0)) {
            const double t = dtau - 1.0;
            double g = -4.585677284736203e-12;
            g = fma(g, t, 6.465596029808311e-11);
            g = fma(g, t, -8.315200300486033e-10);
            g = fma(g, t, 1.0046307689376594e-08);
            g = fma(g, t, -1.1142554025478742e-07);
            g = fma(g, t, 1.1252035937302869e-06);
            g = fma(g, t, -1.0249196652958194e-05);
            g = fma(g, t, 8.324114893927396e-05);
            g = fma(g, t, -0.0005941848175853081);
            g = fma(g, t, 0.0036598468274018593);
            g = fma(g, t, -0.018988156876153583);
            g = fma(g, t, 0.08030139707139056);
            g = fma(g, t, -0.26424111765711533);
            g = fma(g, t, 0.6321205588285577);
            a = P * (dtau * g);
            gseg = ((P * G) * ds) * g;
        } else {
            a = P * absorb(dtau);
            gseg = qdiv(a * G, kap);
        }
    }
    // a < b and a > 0 for a, b >= 0 (not NaN): the order of their bit patterns as integers, which
    // keeps the comparison off the FP64 pipe
    __device__ __forceinline__ static bool lt(double a, double b) { return __double_as_longlong(a) < __double_as_longlong(b); }
    __device__ __forceinline__ static bool pos(double a) { return __double_as_longlong(a) > 0; }
    __device__ __forceinline__ static bool neg(double x) { return __double_as_longlong(x) < 0; }
    __device__ __forceinline__ static double mag(double x)
    {
        return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffll);
    }
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
    __device__ __forceinline__ static float mn(float a, float b) { return fminf(a, b); }
    // 1 - e^{-x} for x >= 0. Below x = 1/4 the Taylor series of 1 - e^{-x} to x^7 (the
    // alternating tail is below x^8/8! < 4e-10, i.e. < 2e-9 relative); above it
    // 1 - __expf(-x), whose error (a few ulp of e^{-x} < 0.78) is below 1e-6 of the
    // result. Both are evaluated and one selected, so lanes do not diverge.
    __device__ __forceinline__ static float absorb(float x)
    {
        float p = 1.0f / 5040.0f;
        p = fmaf(p, x, -1.0f / 720.0f);
        p = fmaf(p, x, 1.0f / 120.0f);
        p = fmaf(p, x, -1.0f / 24.0f);
        p = fmaf(p, x, 1.0f / 6.0f);
        p = fmaf(p, x, -0.5f);
        p = fmaf(p, x, 1.0f);
        const float series = p * x;
        const float direct = 1.0f - __expf(-x);
        return x < 0.25f ? series : direct;
    }
    __device__ __forceinline__ static float qdiv(float a, float b) { return __fdividef(a, b); }
    // Eq. 1 for a segment of optical depth dtau = kap ds, kap > 0 (see the FP64 form)
    __device__ __forceinline__ static void rate(float P, float G, float kap, float, float dtau, float& a, float& gseg)
    {
        a = P * absorb(dtau);
        gseg = qdiv(a * G, kap);
    }
    __device__ __forceinline__ static bool neg(float x) { return __float_as_int(x) < 0; }
    __device__ __forceinline__ static bool lt(float a, float b) { return a < b; }
    __device__ __forceinline__ static bool pos(float a) { return a > 0.f; }
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

// Exact float -> double widening with integer operations for normal numbers
// (the deposits' case): GB300's FP64 pipe is small, and a conversion per
// deposit there costs more than re-biasing the exponent and shifting the
// mantissa. Zero, subnormals, infinities and NaN take the conversion.
__device__ __forceinline__ double widen(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned mag = u & 0x7fffffffu;
    if (mag - 0x00800000u < 0x7f000000u) {            // normal and finite
        const unsigned hi = ((mag >> 3) + (896u << 20)) | (u & 0x80000000u);
        return __hiloint2double((int)hi, (int)(u << 29));
    }
    return (double)x;
}
__device__ __forceinline__ double widen(double x) { return x; }

// Per-thread tallies for one (solve, level).
struct Tally {
    unsigned rays, split, esc, dtau, dlev, seg, sec;
    unsigned long long hash;
    double abs, escph, dropph;
    __device__ __forceinline__ void clear()
    {
        rays = split = esc = dtau = dlev = seg = sec = 0u;
        hash = 0ULL;
        abs = escph = dropph = 0.0;
    }
};

// What a ray needs from the solve it belongs to.
template <class R>
struct SolveView {
    const R* kap;
    double* gamma;
    int n;
    int level_max;
    int overlap_mode;
    int hash;
    long long rq;
    R tau_max;
    uint32_t src_off;        // first catalog index of this solve (ray ids are solve-local)
    long long rs;            // periodic boundaries: travel-distance cutoff sqrt(3) n (2^-24 cells); 0: none
    SpecTable<R> spec;       // RT_SPECTRUM_BLACKBODY (march_ray<..., true> only)
};

// Periodic boundaries (Sec. 2.5.1): a coordinate moved by one cell wraps around the box.
__device__ __forceinline__ int wrap1(const int v, const int n)
{
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

// A coordinate any number of boxes away, wrapped into [0, n).
__device__ __forceinline__ int wrapn(const int v, const int n)
{
    const int r = v % n;
    return r < 0 ? r + n : r;
}

// Eq. 1 for one segment of optical depth dtau = kap ds (kap = 0: the thin limit): the photons a it
// absorbs per unit photon rate and its rate gseg. Gray: a = P (1 - e^{-dtau}). kFreq, integrated over
// the blackbody spectrum (V.spec), the ray's budget P is its geometric share and the photons it still
// carries are P Phi(tau): the segment absorbs P (Phi(tau) - Phi(tau + dtau)), taken from the cubic
// pieces in tau as a mean slope (no cancellation), and deposits at the thin rate P Psi(tau) where
// kap = 0.
template <class R, bool kFreq>
__device__ __forceinline__ void segment_eq1(const SolveView<R>& V, R P, R tau, R ctau, R G, R kap, R ds, R dtau, R& a,
                                            R& gseg)
{
    using I = Ieee<R>;
    if constexpr (kFreq && sizeof(R) == 8) {
        if (I::pos(kap)) {
            double frac, per_kap;
            lin_absorb(V.spec, tau, dtau, kap, ds, frac, per_kap);
            a = P * frac;
            gseg = (P * G) * per_kap;
        } else {
            a = (R)0;
            gseg = ((P * lin_psi(V.spec, tau)) * G) * ds;
        }
    } else if constexpr (kFreq) {
        const R t0 = I::sub(tau, ctau);
        if (I::pos(kap)) {
            a = P * lin_absorb_f(V.spec, t0, dtau);
            gseg = I::qdiv(a * G, kap);
        } else {
            a = (R)0;
            gseg = ((P * lin_psi_f(V.spec, t0)) * G) * ds;
        }
    } else if (I::pos(kap)) {
        I::rate(P, G, kap, ds, dtau, a, gseg);
    } else {
        a = (R)0;
        gseg = (P * G) * ds;
    }
}

// The photons a ray still carries, in units of its source's photon rate per ray: its compensated
// budget P - cP (gray), or P Phi(tau - ctau) (kFreq).
template <class R, bool kFreq>
__device__ __forceinline__ double ray_remaining(const SolveView<R>& V, R P, R tau, R cP, R ctau)
{
    if constexpr (kFreq && sizeof(R) == 8) {
        return P * lin_phi(V.spec, tau);
    } else if constexpr (kFreq) {
        return widen(P) * widen(lin_phi_f(V.spec, Ieee<R>::sub(tau, ctau)));
    } else {
        return widen(P) - widen(cP);
    }
}

// March one ray of level l (source entry se, quantised direction dv, budget
// P with compensation cP, optical depth tau with compensation ctau) from its
// start sphere to its split sphere, depositing into V.gamma and counting into
// T. Returns true if the ray reached R_l and splits; its final P, tau (and
// compensations) are then in oP, otau, ocP, octau.
// kFreq: Eq. 1 integrated over the blackbody spectrum (V.spec): the budget P stays the ray's
// geometric share and the photons it still carries are P Phi(tau); otherwise the gray rate, with
// P decremented by every absorption.
template <class R, bool kHash, bool kFreq>
__device__ __forceinline__ bool march_ray(const SolveView<R>& V, const int l, const uint32_t si, const uint32_t pix,
                                          R P, R tau, R cP, R ctau, const SrcEntry& se, const int4 dv, Tally& T,
                                          R& oP, R& otau, float& ocP, float& octau)
{
    using I = Ieee<R>;
    // photons the ray still carries, in units of ph
    auto remaining = [&]() -> double { return ray_remaining<R, kFreq>(V, P, tau, cP, ctau); };
    const int n = V.n;
    // the ray ends on its split sphere R_l or, with periodic boundaries, at the travel distance
    // sqrt(3) L_box if that comes first or at the same point, where it stops without splitting
    const bool periodic = V.rs != 0;
    const long long rq_split = V.rq << l;
    const bool split_end = !periodic || rq_split < V.rs;
    const long long rq_end = split_end ? rq_split : V.rs;
    const long long rq_start = l > 0 ? (V.rq << (l - 1)) : 0;
    const R pV = I::pow2(-(S - 1 + F)), pI = I::pow2(-S), pU = I::pow2(-(S + 1));
    bool split = false;
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
    if (periodic) {
        i0 = wrapn(i0, n);
        i1 = wrapn(i1, n);
        i2 = wrapn(i2, n);
    }
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
    const R taumax = V.tau_max;
    const unsigned long long rbase =
        (kHash && V.hash) ? mix64(((unsigned long long)(si - V.src_off) << 36) | ((unsigned long long)l << 31) | pix) : 0ULL;

    // photons this ray absorbs (units of ph) are its budget at the start less its budget at the end:
    // the compensated budget P - cP, differenced in FP64
    const double B0 = remaining();
    ++T.rays;
    const bool inside0 = (unsigned)i0 < (unsigned)n && (unsigned)i1 < (unsigned)n && (unsigned)i2 < (unsigned)n;
    if (!inside0) {
        ++T.esc;
        T.escph += ph * (remaining());
    }
    unsigned seq = 0;

    // One segment of length ds_p (ray parameter) in the current cell, ending at parameter
    // tnext, where the distance to the exit face along axis b is dn_b: deposit Gamma (Eq. 1,
    // gray, V_box) with the overlap correction (Eqs. 5-8), then update the budgets.
    auto segment = [&](const R kraw, R ds_p, R dn0, R dn1, R dn2, R tnext) {
        const R ds = I::mul(ds_p, nrm);
        const int cell = (i2 * n + i1) * n + i0;
        // ---- geometry of the overlap correction first (it needs no kappa), so that the
        // neighbour's kappa is requested while this cell's is still in flight
        R De = (R)0, Lpix = (R)1;
        bool near = false;
        int c2 = -1;            // the cell across the nearest face (Arc / conservative modes), if in the domain
        if (V.overlap_mode != RT_OVERLAP_NONE) {
            // distances from the segment midpoint to the six faces, order x-, x+, y-, y+, z-, z+
            const R d0 = I::add(dn0, I::mul(ds_p, u0));
            const R d1 = I::add(dn1, I::mul(ds_p, u1));
            const R d2 = I::add(dn2, I::mul(ds_p, u2));
            const R o0 = I::sub((R)1, d0), o1 = I::sub((R)1, d1), o2 = I::sub((R)1, d2);
            // D_edge: the smallest of the six distances (a minimum is exact, so its value does
            // not depend on the order); which face attains it is resolved below, only when needed
            const R m0 = I::mn(d0, o0), m1 = I::mn(d1, o1), m2 = I::mn(d2, o2);
            De = I::mn(I::mn(m0, m1), m2);
            const R tm = I::sub(tnext, I::mul(ds_p, (R)0.5));
            Lpix = I::mul(tm, Lc);
            near = I::add(De, De) < Lpix;
            if (near && V.overlap_mode != RT_OVERLAP_LINEAR && V.overlap_mode != RT_OVERLAP_SQUARED) {
                // the first face, in the order x-, x+, y-, y+, z-, z+, at distance D_edge: the first
                // axis whose minimum is D_edge, and on it the upper face only if strictly nearer
                const int ax = m0 == De ? 0 : (m1 == De ? 1 : 2);
                const R dax = pick3(ax, d0, d1, d2), oax = pick3(ax, o0, o1, o2);
                const bool up = pick3(ax, s0, s1, s2) > 0;
                const int step = (up ? dax : oax) < (up ? oax : dax) ? 1 : -1;
                int j0 = i0, j1 = i1, j2 = i2;
                if (ax == 0) j0 += step; else if (ax == 1) j1 += step; else j2 += step;
                if (periodic) {
                    j0 = wrap1(j0, n);
                    j1 = wrap1(j1, n);
                    j2 = wrap1(j2, n);
                }
                if ((unsigned)j0 < (unsigned)n && (unsigned)j1 < (unsigned)n && (unsigned)j2 < (unsigned)n)
                    c2 = (j2 * n + j1) * n + j0;
            }
        }
        const R kn_raw = c2 >= 0 ? V.kap[c2] : (R)0;
        // ---- Eq. 1 for this segment
        const R kap = I::mag(kraw);
        const R dtau = I::mul(kap, ds);
        R a, gseg;
        segment_eq1<R, kFreq>(V, P, tau, ctau, G, kap, ds, dtau, a, gseg);
        // ---- Eqs. 5-8: the share f kept in this cell and the neighbour's deposit
        R f = (R)1, g2 = (R)0;
        int nbcell = -1;
        if (near) {
            if (V.overlap_mode == RT_OVERLAP_LINEAR) {
                f = I::add((R)0.5, I::qdiv(De, Lpix));
            } else if (V.overlap_mode == RT_OVERLAP_SQUARED) {
                f = I::add((R)0.5, I::qdiv(De, Lpix));
                f = f * f;
            } else {
                // naive threshold: the Eq. 5 share applies whatever the neighbour
                if (V.overlap_mode == RT_OVERLAP_NAIVE) f = I::add((R)0.5, I::qdiv(De, Lpix));
                const R kn = I::mag(kn_raw);
                const bool elig = c2 >= 0 && ((V.overlap_mode == RT_OVERLAP_ARC) ? (I::pos(kn))
                                                                                  : (!I::neg(kn_raw) && I::pos(kn)));
                if (elig) {
                    f = I::add((R)0.5, I::qdiv(De, Lpix));
                    g2 = (((R)1 - f) * gseg) * I::qdiv(kap, kn);
                    nbcell = c2;
                }
            }
        }
        atomicAdd(&V.gamma[cell], widen(f * gseg));
        if (nbcell >= 0) {
            atomicAdd(&V.gamma[nbcell], widen(g2));
            ++T.sec;
        }
        budget_add(tau, ctau, dtau);
        if constexpr (!kFreq) budget_add(P, cP, -a);
        if (kHash && V.hash) T.hash += mix64(rbase ^ ((unsigned long long)seq << 40) ^ (unsigned long long)cell);
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
        // kappa of the current cell; the loop requests the next cell's one iteration ahead
        R kcur = V.kap[(i2 * n + i1) * n + i0];
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
            // the step after this segment: every axis whose crossing coincides with the winner's;
            // the cell it leads to is known now, so its kappa is requested before the segment's work
            const bool t0 = (w == 0) || (w == 1 ? A01 == A10 : A02 == A20);
            const bool t1 = (w == 1) || (w == 0 ? A10 == A01 : A12 == A21);
            const bool t2 = (w == 2) || (w == 0 ? A20 == A02 : A21 == A12);
            int ni0 = t0 ? i0 + s0 : i0, ni1 = t1 ? i1 + s1 : i1, ni2 = t2 ? i2 + s2 : i2;
            if (periodic) {
                ni0 = wrap1(ni0, n);
                ni1 = wrap1(ni1, n);
                ni2 = wrap1(ni2, n);
            }
            const bool next_in =
                periodic || ((unsigned)ni0 < (unsigned)n && (unsigned)ni1 < (unsigned)n && (unsigned)ni2 < (unsigned)n);
            const R knext = next_in ? V.kap[(ni2 * n + ni1) * n + ni0] : (R)0;
            segment(kcur, ds_p, dn0, dn1, dn2, I::mul(I::small(2u * kw + 1u), hw));
            if (!I::lt(tau, taumax)) {             // photons spent
                ++T.dtau;
                T.dropph += ph * (remaining());
                T.abs += ph * (B0 - (remaining()));
                alive = false;
                break;
            }
            if (t0) { ++k0; A01 += 2u * D1; A02 += 2u * D2; }
            if (t1) { ++k1; A10 += 2u * D0; A12 += 2u * D2; }
            if (t2) { ++k2; A20 += 2u * D0; A21 += 2u * D1; }
            i0 = ni0;
            i1 = ni1;
            i2 = ni2;
            kcur = knext;
            prev = w;
            kprev = kw;
            if (!next_in) {
                ++T.esc;
                T.escph += ph * (remaining());
                T.abs += ph * (B0 - (remaining()));
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
            // ---- the last segment ends on the end sphere, where k_b = kend_b on every axis
            if (prev < 0) {
                ds_p = split_end ? I::mul((R)V.rq, I::pow2(l > 0 ? l - 1 - F : -F))
                                 : I::mul(I::of(rq_end - rq_start), I::pow2(-F));
            } else {
                const long long num = rq_end * (long long)pick3(prev, D0, D1, D2) - (long long)(2 * kprev + 1) * kB;
                ds_p = I::mul(I::of(num), I::mul(pick3(prev, h0, h1, h2), pV));
            }
            const R pE = I::pow2(-(S + F));
            const R e0 = I::mul(I::of((long long)(2 * ke0 + 1) * kB - rq_end * (long long)D0), pE);
            const R e1 = I::mul(I::of((long long)(2 * ke1 + 1) * kB - rq_end * (long long)D1), pE);
            const R e2 = I::mul(I::of((long long)(2 * ke2 + 1) * kB - rq_end * (long long)D2), pE);
            segment(kcur, ds_p, e0, e1, e2,
                    split_end ? I::mul((R)V.rq, I::pow2(l - F)) : I::mul(I::of(rq_end), I::pow2(-F)));
            if (!I::lt(tau, taumax)) {
                ++T.dtau;
                T.dropph += ph * (remaining());
                T.abs += ph * (B0 - (remaining()));
            } else {
                T.abs += ph * (B0 - (remaining()));
                if (!split_end) {                // travelled sqrt(3) L_box (Sec. 2.5.1)
                    ++T.esc;
                    T.escph += ph * (remaining());
                } else if (l + 1 > V.level_max) {
                    ++T.dlev;
                    T.dropph += ph * (remaining());
                } else {
                    ++T.split;
                    split = true;
                    oP = P;
                    otau = tau;
                    if constexpr (sizeof(R) == 4) {
                        ocP = cP;
                        octau = ctau;
                    }
                }
            }
        }
    }
    T.seg += seq;
    return split;
}

// ---------------------------------------------------------------------------
// Geometry tables. A ray's cells, segment lengths and overlap-correction
// geometry relative to its source depend only on its level and pixel (every
// source sits at a cell centre), so they are walked once per (level, pixel)
// and stored; the table-driven march then does only what depends on the
// data. The walker below takes the same integer steps and the same rounded
// operations as march_ray, so both produce the same segments bit for bit.

// One segment of a walk: its length ds_p (ray parameter), the exit point's distances dn_b to
// the exit faces, the ray parameter where it ends, and the step that follows it (bit a: axis
// a steps; none after the last segment) with the cell it leads to.
template <class R>
struct SegGeo {
    R ds_p, dn0, dn1, dn2, tnext;
    unsigned steps;
    int ni0, ni1, ni2;
    bool next_in;
};

enum { kWalkEnd = 0, kWalkEscaped = 1, kWalkStopped = 2 };

// Exact integer traversal of one ray of level l (Amanatides-Woo on quantised
// directions) from its start sphere R_{l-1} to its split sphere R_l, or out of
// the grid [0, n)^3. The k-th face crossing along axis a is at ray parameter
// T_a(k) = (2k+1) 2^20 / D_a, the split radius is R_l = Rq 2^l / 2^24, and the
// next crossing on a comes before the one on b iff A_ab = (2 k_a + 1) D_b is
// below A_ba, so every decision is an integer comparison and every segment
// length an exact integer times a per-ray constant.
template <class R>
struct Walk {
    unsigned D0, D1, D2;
    int s0, s1, s2;
    int k0, k1, k2, ke0, ke1, ke2;
    unsigned A01, A10, A02, A20, A12, A21;
    R nrm, h0, h1, h2, W01, W02, W12, u0, u1, u2, Lc;
    int i0, i1, i2;          // the current cell

    // Start cell of the ray from cell (c0, c1, c2): the cell holding its point on R_{l-1}.
    // rs: travel-distance cutoff of periodic boundaries (0: none), as in march_ray.
    __device__ __forceinline__ void init(const long long rq, const int l, const int4 dv, const int c0, const int c1,
                                         const int c2, const long long rs)
    {
        using I = Ieee<R>;
        const bool split_end = rs == 0 || (rq << l) < rs;
        const long long rq_end = split_end ? (rq << l) : rs;
        const long long rq_start = l > 0 ? (rq << (l - 1)) : 0;
        D0 = (unsigned)abs(dv.x);
        D1 = (unsigned)abs(dv.y);
        D2 = (unsigned)abs(dv.z);
        s0 = dv.x < 0 ? -1 : 1;
        s1 = dv.y < 0 ? -1 : 1;
        s2 = dv.z < 0 ? -1 : 1;
        // crossings done at the start sphere, and before the split sphere
        k0 = k1 = k2 = 0;
        if (l > 0) {
            k0 = (int)((rq_start * D0 + kB) >> (S + F));
            k1 = (int)((rq_start * D1 + kB) >> (S + F));
            k2 = (int)((rq_start * D2 + kB) >> (S + F));
        }
        ke0 = (int)(((rq_end * D0 + kB - 1) >> (S - 1 + F)) >> 1);
        ke1 = (int)(((rq_end * D1 + kB - 1) >> (S - 1 + F)) >> 1);
        ke2 = (int)(((rq_end * D2 + kB - 1) >> (S - 1 + F)) >> 1);
        i0 = c0 + s0 * k0;
        i1 = c1 + s1 * k1;
        i2 = c2 + s2 * k2;
        // With k_a <= t D_a / 2^21 + 1/2 and D_a D_b <= 2^41, A_ab <= t 2^21 + 2^22, which stays
        // below 2^32 while the ray parameter t is below 2040 (any point of a grid up to 1024^3).
        A01 = (2u * k0 + 1u) * D1;
        A10 = (2u * k1 + 1u) * D0;
        A02 = (2u * k0 + 1u) * D2;
        A20 = (2u * k2 + 1u) * D0;
        A12 = (2u * k1 + 1u) * D2;
        A21 = (2u * k2 + 1u) * D1;
        // per-ray constants
        if constexpr (sizeof(R) == 4) {
            nrm = __int_as_float(dv.w);
        } else {
            const long long nn = (long long)D0 * D0 + (long long)D1 * D1 + (long long)D2 * D2;
            nrm = __dmul_rn(__dsqrt_rn(__ll2double_rn(nn)), I::pow2(-S));
        }
        const R two20 = (R)(1 << (S - 1));
        h0 = D0 ? I::div(two20, (R)D0) : (R)0;
        h1 = D1 ? I::div(two20, (R)D1) : (R)0;
        h2 = D2 ? I::div(two20, (R)D2) : (R)0;
        W01 = (D0 && D1) ? I::div(h0, (R)D1) : (R)0;
        W02 = (D0 && D2) ? I::div(h0, (R)D2) : (R)0;
        W12 = (D1 && D2) ? I::div(h1, (R)D2) : (R)0;
        const R pU = I::pow2(-(S + 1));
        u0 = I::mul((R)D0, pU);
        u1 = I::mul((R)D1, pU);
        u2 = I::mul((R)D2, pU);
        Lc = I::mul(I::mul(nrm, (R)kSqrtPiOver3), I::pow2(-l));
    }

    __device__ __forceinline__ bool inside(const int n) const
    {
        return (unsigned)i0 < (unsigned)n && (unsigned)i1 < (unsigned)n && (unsigned)i2 < (unsigned)n;
    }

    // Walk from the (in-grid) start cell (rq and l as given to init). seg(g) is called for every
    // segment of positive length, in order, with the walker's current cell being the segment's
    // cell; it returns false to stop the ray. Returns kWalkEnd (R_l reached), kWalkEscaped (left
    // the grid) or kWalkStopped.
    template <class Seg>
    __device__ __forceinline__ int run(const int n, const long long rq, const int l, const long long rs, Seg&& seg)
    {
        using I = Ieee<R>;
        const bool split_end = rs == 0 || (rq << l) < rs;
        const long long rq_end = split_end ? (rq << l) : rs;
        const long long rq_start = l > 0 ? (rq << (l - 1)) : 0;
        const R pV = I::pow2(-(S - 1 + F)), pI = I::pow2(-S);
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
        // ---- segments that end on a face crossing
        while (!is_end) {
            const R hw = pick3(w, h0, h1, h2);
            const R invw = I::mul(hw, pI);
            SegGeo<R> g;
            g.ds_p = ds_p;
            // exit-point distance to the exit face along b: (A_bw - A_wb) / (2 D_w), 0 on b = w
            g.dn0 = g.dn1 = g.dn2 = (R)0;
            if (w == 0) {
                g.dn1 = I::mul(I::small(A10 - A01), invw);
                g.dn2 = I::mul(I::small(A20 - A02), invw);
            } else if (w == 1) {
                g.dn0 = I::mul(I::small(A01 - A10), invw);
                g.dn2 = I::mul(I::small(A21 - A12), invw);
            } else {
                g.dn0 = I::mul(I::small(A02 - A20), invw);
                g.dn1 = I::mul(I::small(A12 - A21), invw);
            }
            g.tnext = I::mul(I::small(2u * kw + 1u), hw);
            // the step after this segment: every axis whose crossing coincides with the winner's
            const bool t0 = (w == 0) || (w == 1 ? A01 == A10 : A02 == A20);
            const bool t1 = (w == 1) || (w == 0 ? A10 == A01 : A12 == A21);
            const bool t2 = (w == 2) || (w == 0 ? A20 == A02 : A21 == A12);
            g.steps = (t0 ? 1u : 0u) | (t1 ? 2u : 0u) | (t2 ? 4u : 0u);
            g.ni0 = t0 ? i0 + s0 : i0;
            g.ni1 = t1 ? i1 + s1 : i1;
            g.ni2 = t2 ? i2 + s2 : i2;
            g.next_in = (unsigned)g.ni0 < (unsigned)n && (unsigned)g.ni1 < (unsigned)n && (unsigned)g.ni2 < (unsigned)n;
            if (!seg(g)) return kWalkStopped;
            if (t0) { ++k0; A01 += 2u * D1; A02 += 2u * D2; }
            if (t1) { ++k1; A10 += 2u * D0; A12 += 2u * D2; }
            if (t2) { ++k2; A20 += 2u * D0; A21 += 2u * D1; }
            i0 = g.ni0;
            i1 = g.ni1;
            i2 = g.ni2;
            prev = w;
            kprev = kw;
            if (!g.next_in) return kWalkEscaped;
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
        // ---- the last segment ends on the end sphere, where k_b = kend_b on every axis
        SegGeo<R> g;
        if (prev < 0) {
            g.ds_p = split_end ? I::mul((R)rq, I::pow2(l > 0 ? l - 1 - F : -F)) : I::mul(I::of(rq_end - rq_start), I::pow2(-F));
        } else {
            const long long num = rq_end * (long long)pick3(prev, D0, D1, D2) - (long long)(2 * kprev + 1) * kB;
            g.ds_p = I::mul(I::of(num), I::mul(pick3(prev, h0, h1, h2), pV));
        }
        const R pE = I::pow2(-(S + F));
        g.dn0 = I::mul(I::of((long long)(2 * ke0 + 1) * kB - rq_end * (long long)D0), pE);
        g.dn1 = I::mul(I::of((long long)(2 * ke1 + 1) * kB - rq_end * (long long)D1), pE);
        g.dn2 = I::mul(I::of((long long)(2 * ke2 + 1) * kB - rq_end * (long long)D2), pE);
        g.tnext = split_end ? I::mul((R)rq, I::pow2(l - F)) : I::mul(I::of(rq_end), I::pow2(-F));
        g.steps = 0u;
        g.ni0 = i0;
        g.ni1 = i1;
        g.ni2 = i2;
        g.next_in = false;
        if (!seg(g)) return kWalkStopped;
        return kWalkEnd;
    }
};

// The nearest face to a segment's midpoint (Eqs. 5-6 geometry): D_edge, L_pix, whether
// 2 D_edge < L_pix, and (if face) the axis and side of the first face, in the order x-, x+,
// y-, y+, z-, z+, at distance D_edge.
template <class R>
struct Edge {
    R De, Lpix;
    bool near;
    int ax, step;
};

template <class R>
__device__ __forceinline__ Edge<R> edge(const Walk<R>& W, const SegGeo<R>& g, const bool face)
{
    using I = Ieee<R>;
    Edge<R> e;
    // distances from the segment midpoint to the six faces, order x-, x+, y-, y+, z-, z+
    const R d0 = I::add(g.dn0, I::mul(g.ds_p, W.u0));
    const R d1 = I::add(g.dn1, I::mul(g.ds_p, W.u1));
    const R d2 = I::add(g.dn2, I::mul(g.ds_p, W.u2));
    const R o0 = I::sub((R)1, d0), o1 = I::sub((R)1, d1), o2 = I::sub((R)1, d2);
    // D_edge: the smallest of the six distances (a minimum is exact, so its value does
    // not depend on the order); which face attains it is resolved only when needed
    const R m0 = I::mn(d0, o0), m1 = I::mn(d1, o1), m2 = I::mn(d2, o2);
    e.De = I::mn(I::mn(m0, m1), m2);
    const R tm = I::sub(g.tnext, I::mul(g.ds_p, (R)0.5));
    e.Lpix = I::mul(tm, W.Lc);
    e.near = I::add(e.De, e.De) < e.Lpix;
    e.ax = 0;
    e.step = 0;
    if (face && e.near) {
        // the first axis whose minimum is D_edge, and on it the upper face only if strictly nearer
        e.ax = m0 == e.De ? 0 : (m1 == e.De ? 1 : 2);
        const R dax = pick3(e.ax, d0, d1, d2), oax = pick3(e.ax, o0, o1, o2);
        const bool up = pick3(e.ax, W.s0, W.s1, W.s2) > 0;
        e.step = (up ? dax : oax) < (up ? oax : dax) ? 1 : -1;
    }
    return e;
}

// Warp-aggregated append of the rays that split (Alg. 1 FILTERCOPYTRANSFORM<3>): one
// atomic per warp reserves the records; each splitting lane writes its parent record.
template <class R>
__device__ __forceinline__ void append_split(bool split, uint32_t si, uint32_t pix, R P, R tau, float cP, float ctau,
                                             const RayBuf<R>& out, unsigned long long* count, unsigned* err)
{
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, split);
    if (!m) return;
    const int leader = __ffs(m) - 1;
    unsigned long long pos0 = 0;
    if (lane == leader) pos0 = atomicAdd(count, (unsigned long long)__popc(m));
    pos0 = __shfl_sync(0xffffffffu, pos0, leader);
    if (split) {
        const unsigned long long pos = pos0 + __popc(m & ((1u << lane) - 1u));
        if (pos < (unsigned long long)out.cap) {
            out.src[pos] = si;
            out.pix[pos] = pix;
            out.P[pos] = P;
            out.tau[pos] = tau;
            if constexpr (sizeof(R) == 4) {
                out.cP[pos] = cP;
                out.ctau[pos] = ctau;
            }
        } else {
            atomicOr(err, kErrRayOverflow);
        }
    }
}

// ---------------------------------------------------------------------------
// Geometry-table generation and the table-driven FP32 march.
//
// Entry of segment s of pixel p (8 bytes): x = the FP32 segment length ds (ds_p times the
// direction norm, rounded as in march_ray); y = bits 0-23: the share f kept in the cell when the
// segment is near an edge (Eq. 6), as its float bit pattern less that of 0.5 - 2^-21 (f is
// 0.5 + D_edge / L_pix, in [0.5 - 2^-21, 1] including rounding); bits 24-26: the axes that step
// after the segment (none after the one ending on R_l); bit 27: 2 D_edge < L_pix; bits 28-29:
// axis of the nearest face; bit 30: the nearest face is the upper one; bit 31: the pixel's last
// entry. Entries are stored by blocks of 32 consecutive pixels, segment-major within a block, so
// the four children of a parent (adjacent lanes) read one 32-byte sector per segment.

constexpr unsigned kFBase = 0x3efffff0u;     // float bits of 0.5 - 2^-21

// FP64 entries (16 bytes, same row offsets): x = the bits of the FP64 ds (rounded as in the FP64
// march_ray); y = bits 0-52: the FP64 share f of a near segment as its bit pattern less that of
// 0.5, plus 1 (f in [0.5, 1]: 1 .. 2^52 + 1), 0 otherwise; bits 56-63: the flags of bits 24-31 of
// the FP32 entry (steps, near, face axis and side, last), decided in FP64.
constexpr unsigned long long kDBase = 0x3fdfffffffffffffull;    // double bits of 0.5, less 1

// Walk pixel p of level l from a source at the centre of a virtual grid. Without periodic
// boundaries it has 2 n_cover - 1 cells: a cell offset of n_cover or more along any axis lies
// outside every n_cover^3 grid for every source cell, so that is where the table of the pixel may
// stop. With them (rs > 0) the ray continues to the travel-distance cutoff, so the virtual grid is
// wide enough never to be left first (relative cells are what the table stores; the march wraps).
__device__ __forceinline__ int geom_virtual_grid(const int n_cover, const long long rs)
{
    return rs ? 2 * ((int)(rs >> F) + 3) + 1 : 2 * n_cover - 1;
}

template <class R>
__device__ __forceinline__ void geom_walk_init(Walk<R>& W, const long long rq, const int l, const int4 dv,
                                               const int nv, const long long rs)
{
    const int c = (nv - 1) / 2;
    W.init(rq, l, dv, c, c, c, rs);
}

__global__ void __launch_bounds__(256) geom_count_kernel(const long long rq, const int l, const int4* __restrict__ dirs,
                                                         const long long npix, const int n_cover, const long long rs,
                                                         unsigned* __restrict__ rows)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    unsigned cnt = 0;
    if (p < npix) {
        Walk<float> W;
        const int nv = geom_virtual_grid(n_cover, rs);
        geom_walk_init(W, rq, l, dirs[p], nv, rs);
        if (W.inside(nv)) W.run(nv, rq, l, rs, [&](const SegGeo<float>&) -> bool { ++cnt; return true; });
    }
    // rows of a 32-pixel block: the longest column in it
    for (int o = 16; o > 0; o >>= 1) cnt = max(cnt, __shfl_xor_sync(0xffffffffu, cnt, o));
    if ((threadIdx.x & 31) == 0 && p < npix) rows[p >> 5] = cnt;
}

__global__ void __launch_bounds__(256) geom_fill_kernel(const long long rq, const int l, const int4* __restrict__ dirs,
                                                        const long long npix, const int n_cover, const long long rs,
                                                        const unsigned long long* __restrict__ row0,
                                                        uint2* __restrict__ ent, unsigned* err)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= npix) return;
    Walk<float> W;
    const int nv = geom_virtual_grid(n_cover, rs);
    geom_walk_init(W, rq, l, dirs[p], nv, rs);
    if (!W.inside(nv)) return;
    uint2* col = ent + row0[p >> 5] * 32 + (p & 31);
    unsigned long long s = 0;
    W.run(nv, rq, l, rs, [&](const SegGeo<float>& g) -> bool {
        const Edge<float> e = edge<float>(W, g, true);
        unsigned y = g.steps << 24;
        if (e.near) {
            const float f = __fadd_rn(0.5f, __fdividef(e.De, e.Lpix));
            const unsigned code = __float_as_uint(f) - kFBase;
            if (code > 0xffffffu) atomicOr(err, kErrGeometry);
            y |= (code & 0xffffffu) | (1u << 27) | ((unsigned)e.ax << 28) | (e.step > 0 ? (1u << 30) : 0u);
        }
        if (g.steps == 0u || !g.next_in) y |= 1u << 31;
        col[s * 32] = make_uint2(__float_as_uint(__fmul_rn(g.ds_p, W.nrm)), y);
        ++s;
        return true;
    });
}

__global__ void __launch_bounds__(256) geom_fill64_kernel(const long long rq, const int l, const int4* __restrict__ dirs,
                                                          const long long npix, const int n_cover, const long long rs,
                                                          const unsigned long long* __restrict__ row0,
                                                          const unsigned long long rows_total,
                                                          ulonglong2* __restrict__ ent, unsigned* err)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= npix) return;
    Walk<double> W;
    const int nv = geom_virtual_grid(n_cover, rs);
    geom_walk_init(W, rq, l, dirs[p], nv, rs);
    if (!W.inside(nv)) return;
    const long long b = p >> 5, nb = (npix + 31) >> 5;
    const unsigned long long rows = (b + 1 < nb ? row0[b + 1] : rows_total) - row0[b];
    ulonglong2* col = ent + row0[b] * 32 + (p & 31);
    unsigned long long s = 0;
    W.run(nv, rq, l, rs, [&](const SegGeo<double>& g) -> bool {
        if (s >= rows) {                 // the rows were counted by the same integer traversal
            atomicOr(err, kErrGeometry);
            return false;
        }
        const Edge<double> e = edge<double>(W, g, true);
        unsigned long long y = (unsigned long long)g.steps << 56;
        if (e.near) {
            const double f = __dadd_rn(0.5, e.De / e.Lpix);
            const unsigned long long code = (unsigned long long)__double_as_longlong(f) - kDBase;
            if (code == 0ull || code > (1ull << 52) + 1ull) atomicOr(err, kErrGeometry);
            y |= (code & ((1ull << 53) - 1ull)) | (1ull << 59) | ((unsigned long long)e.ax << 60) |
                 (e.step > 0 ? (1ull << 62) : 0ull);
        }
        if (g.steps == 0u || !g.next_in) y |= 1ull << 63;
        col[s * 32] = make_ulonglong2((unsigned long long)__double_as_longlong(__dmul_rn(g.ds_p, W.nrm)), y);
        ++s;
        return true;
    });
}

// Table entry access by precision: the entry type, its FP32/FP64 segment length, the flag word
// (steps in bits 24-26, near 27, face axis 28-29, upper face 30, last 31) and the share f.
template <class R>
struct TableEntry;

template <>
struct TableEntry<float> {
    using E = uint2;
    __device__ __forceinline__ static const E* ent(const GeomLevel& G) { return G.ent; }
    __device__ __forceinline__ static E none() { return make_uint2(0u, 0u); }
    __device__ __forceinline__ static float ds(const E& e) { return __uint_as_float(e.x); }
    __device__ __forceinline__ static unsigned flags(const E& e) { return e.y; }
    __device__ __forceinline__ static float f(const E& e) { return __uint_as_float((e.y & 0xffffffu) + kFBase); }
};

template <>
struct TableEntry<double> {
    using E = ulonglong2;
    __device__ __forceinline__ static const E* ent(const GeomLevel& G) { return G.ent64; }
    __device__ __forceinline__ static E none() { return make_ulonglong2(0ull, 0ull); }
    __device__ __forceinline__ static double ds(const E& e) { return __longlong_as_double((long long)e.x); }
    __device__ __forceinline__ static unsigned flags(const E& e) { return (unsigned)(e.y >> 32); }
    __device__ __forceinline__ static double f(const E& e)
    {
        return __longlong_as_double((long long)((e.y & ((1ull << 53) - 1ull)) + kDBase));
    }
    // the same f as a double-float, straight from the code: f = (1 + m 2^-52) / 2 with m = code - 1
    // (m = 2^52 is f = 1); head its leading 24 bits, tail the other 29 rounded to 24, as df_of(f)
    __device__ __forceinline__ static dflt f_df(const E& e)
    {
        const unsigned long long m = (e.y & ((1ull << 53) - 1ull)) - 1ull;
        return {__uint_as_float(0x3f000000u + (unsigned)(m >> 29)),
                __fmul_rn(__uint2float_rn((unsigned)m & 0x1fffffffu), __uint_as_float(74u << 23))};   // 2^-53
    }
};

// march_ray with the geometry read from the level's table (FP32 or FP64 physics).
template <class R, bool kHash, bool kFreq>
__device__ __forceinline__ bool march_ray_table(const SolveView<R>& V, const GeomLevel& GL, unsigned* err, const int l,
                                                const uint32_t si, const uint32_t pix, R P, R tau, R cP, R ctau,
                                                const SrcEntry& se, const int4 dv, Tally& T, R& oP, R& otau,
                                                float& ocP, float& octau)
{
    using I = Ieee<R>;
    using TE = TableEntry<R>;
    using E = typename TE::E;
    const int n = V.n;
    const int s0 = dv.x < 0 ? -1 : 1, s1 = dv.y < 0 ? -1 : 1, s2 = dv.z < 0 ? -1 : 1;
    int i0 = se.cx, i1 = se.cy, i2 = se.cz;
    if (l > 0) {                    // the start cell: crossings done at the start sphere
        const long long rq_start = V.rq << (l - 1);
        i0 += s0 * (int)((rq_start * (unsigned)abs(dv.x) + kB) >> (S + F));
        i1 += s1 * (int)((rq_start * (unsigned)abs(dv.y) + kB) >> (S + F));
        i2 += s2 * (int)((rq_start * (unsigned)abs(dv.z) + kB) >> (S + F));
    }
    // periodic boundaries: cells wrap, and the ray's last entry ends at the travel-distance cutoff
    // instead of R_l when that comes first
    const bool periodic = V.rs != 0;
    const bool split_end = !periodic || (V.rq << l) < V.rs;
    if (periodic) {
        i0 = wrapn(i0, n);
        i1 = wrapn(i1, n);
        i2 = wrapn(i2, n);
    }
    R G;
    if constexpr (sizeof(R) == 4) G = se.gf; else G = se.gd;
    const double ph = se.ph;
    const R taumax = V.tau_max;
    const unsigned long long rbase =
        (kHash && V.hash) ? mix64(((unsigned long long)(si - V.src_off) << 36) | ((unsigned long long)l << 31) | pix) : 0ULL;
    const bool face = V.overlap_mode == RT_OVERLAP_ARC || V.overlap_mode == RT_OVERLAP_CONSERVATIVE ||
                      V.overlap_mode == RT_OVERLAP_NAIVE;
    const bool corr = V.overlap_mode != RT_OVERLAP_NONE;
    const long long nn = (long long)n * n;
    const double B0 = ray_remaining<R, kFreq>(V, P, tau, cP, ctau);
    ++T.rays;
    if (!((unsigned)i0 < (unsigned)n && (unsigned)i1 < (unsigned)n && (unsigned)i2 < (unsigned)n)) {
        ++T.esc;
        T.escph += ph * ray_remaining<R, kFreq>(V, P, tau, cP, ctau);
        return false;
    }
    const E* col = TE::ent(GL) + GL.row0[pix >> 5] * 32 + (pix & 31);
    E e = col[0];
    int cell = (i2 * n + i1) * n + i0;
    R kcur = V.kap[cell];
    unsigned seq = 0;
    bool split = false;
    for (;;) {
        // the next entry and the next cell's kappa are requested before this segment's work
        const unsigned fl = TE::flags(e);
        const bool last = (fl >> 31) != 0u;
        const E en = last ? TE::none() : col[(unsigned long long)(seq + 1) * 32];
        const unsigned steps = (fl >> 24) & 7u;
        int ni0 = (steps & 1u) ? i0 + s0 : i0;
        int ni1 = (steps & 2u) ? i1 + s1 : i1;
        int ni2 = (steps & 4u) ? i2 + s2 : i2;
        if (periodic) {
            ni0 = wrap1(ni0, n);
            ni1 = wrap1(ni1, n);
            ni2 = wrap1(ni2, n);
        }
        const bool next_in =
            periodic || ((unsigned)ni0 < (unsigned)n && (unsigned)ni1 < (unsigned)n && (unsigned)ni2 < (unsigned)n);
        const int ncell = (ni2 * n + ni1) * n + ni0;
        const R knext = (steps && next_in) ? V.kap[ncell] : (R)0;
        const bool near = corr && ((fl >> 27) & 1u);
        int c2 = -1;
        if (face && near) {
            const int ax = (int)((fl >> 28) & 3u);
            const int step = ((fl >> 30) & 1u) ? 1 : -1;
            const int jc = pick3(ax, i0, i1, i2) + step;
            if (periodic) {
                const int jw = wrap1(jc, n);
                c2 = cell + (jw - (jc - step)) * (ax == 0 ? 1 : (ax == 1 ? n : (int)nn));
            } else if ((unsigned)jc < (unsigned)n) {
                c2 = cell + step * (ax == 0 ? 1 : (ax == 1 ? n : (int)nn));
            }
        }
        const R kn_raw = c2 >= 0 ? V.kap[c2] : (R)0;
        // ---- Eq. 1 for this segment
        const R ds = TE::ds(e);
        const R kap = I::mag(kcur);
        const R dtau = I::mul(kap, ds);
        R a, gseg;
        segment_eq1<R, kFreq>(V, P, tau, ctau, G, kap, ds, dtau, a, gseg);
        // ---- Eqs. 5-8
        R f = (R)1, g2 = (R)0;
        int nbcell = -1;
        if (near) {
            const R fn = TE::f(e);
            if (V.overlap_mode == RT_OVERLAP_LINEAR) {
                f = fn;
            } else if (V.overlap_mode == RT_OVERLAP_SQUARED) {
                f = fn * fn;
            } else {
                if (V.overlap_mode == RT_OVERLAP_NAIVE) f = fn;   // the Eq. 5 share whatever the neighbour
                const R kn = I::mag(kn_raw);
                const bool elig =
                    c2 >= 0 && ((V.overlap_mode == RT_OVERLAP_ARC) ? (I::pos(kn)) : (!I::neg(kn_raw) && I::pos(kn)));
                if (elig) {
                    f = fn;
                    g2 = (((R)1 - f) * gseg) * I::qdiv(kap, kn);
                    nbcell = c2;
                }
            }
        }
        atomicAdd(&V.gamma[cell], widen(f * gseg));
        if (nbcell >= 0) {
            atomicAdd(&V.gamma[nbcell], widen(g2));
            ++T.sec;
        }
        budget_add(tau, ctau, dtau);
        if constexpr (!kFreq) budget_add(P, cP, -a);
        if (kHash && V.hash) T.hash += mix64(rbase ^ ((unsigned long long)seq << 40) ^ (unsigned long long)cell);
        ++seq;
        if (!I::lt(tau, taumax)) {             // photons spent
            ++T.dtau;
            T.dropph += ph * ray_remaining<R, kFreq>(V, P, tau, cP, ctau);
            break;
        }
        if (!steps) {                    // the segment ended on the end sphere
            if (!split_end) {            // travelled sqrt(3) L_box (Sec. 2.5.1)
                ++T.esc;
                T.escph += ph * ray_remaining<R, kFreq>(V, P, tau, cP, ctau);
            } else if (l + 1 > V.level_max) {
                ++T.dlev;
                T.dropph += ph * ray_remaining<R, kFreq>(V, P, tau, cP, ctau);
            } else {
                ++T.split;
                split = true;
                oP = P;
                otau = tau;
                ocP = (float)cP;         // compensations: FP32 march only (0 in FP64)
                octau = (float)ctau;
            }
            break;
        }
        if (!next_in) {
            ++T.esc;
            T.escph += ph * ray_remaining<R, kFreq>(V, P, tau, cP, ctau);
            break;
        }
        if (last) {                      // cannot happen: a table ends where every grid is left
            atomicOr(err, kErrGeometry);
            break;
        }
        i0 = ni0;
        i1 = ni1;
        i2 = ni2;
        cell = ncell;
        kcur = knext;
        e = en;
    }
    T.seg += seq;
    T.abs += ph * (B0 - ray_remaining<R, kFreq>(V, P, tau, cP, ctau));
    return split;
}

// ---------------------------------------------------------------------------
// FP64 table march in double-float arithmetic. GB300's FP64 unit runs at 1/64 of its FP32
// rate, and only two FP64 operations per segment decide anything: dtau = kap ds and
// tau += dtau, whose result is compared with tau_max. Both stay IEEE FP64, so the bookkeeping
// (rays, splits, segments, terminations, visits) is that of the plain FP64 march bit for bit.
// What only feeds the fields and the photon ledger runs on the FP32 pipe in double-float
// pairs (dfloat.h, about 48 significant bits):
//   - the Eq. 1 factor g(dtau) = (1 - e^{-dtau}) / dtau below dtau = 2, from the Taylor table of
//     rate_table.h (512 intervals, degree 4, in shared memory);
//   - the ray's photon budget, carried as Q = P m_G 2^64, where G = m_G 2^e_G is the source's
//     rate per unit budget and cell of path (the factor 2^64 keeps Q far inside the float
//     range): a segment absorbs Q dtau g of it and deposits the rate Q g ds 2^(e_G - 64), which
//     is Eq. 1 with V_box, P G ds g;
//   - the Eqs. 5-8 shares and the Eq. 8 ratio kap / kap' (a reciprocal and one correction).
// Each deposit is rounded to double by integer operations (df_to_double_pos) for its atomic add.
// From dtau = 2 on (an opaque cell, where most of the budget goes at once) the segment is
// evaluated in FP64 with expm1 and a division, as in the FP64 form of march_ray_table.

// The rate table in shared memory: two float4 arrays, row j's {c0, c0', c1, c1'} at 4 j and its
// {c2, c2', c3, c4} at 4 (kRateIntervals + j), so each is one 16-byte load.
constexpr int kRateSmem = 8 * kRateIntervals;

// g(x) for 0 <= x < 2 from interval j = floor(256 x) of the Taylor table, expanded about y0 = 0
// (j = 0) or the interval's midpoint (j + 1/2) / 256: c0 + r (c1 + r (c2 + r (c3 + r c4))) with
// r = x - y0; the two inner terms in float (below 3e-9 of g together), the three outer ones in
// double-float.
__device__ __forceinline__ dflt rate_factor(const float* __restrict__ tab, const dflt x)
{
    const int j = min(__float2int_rz(__fmul_rn(x.h, 256.f)), kRateIntervals - 1);
    const float4 A = *reinterpret_cast<const float4*>(tab + 4 * j);                          // c0 c0' c1 c1'
    const float4 B = *reinterpret_cast<const float4*>(tab + 4 * (kRateIntervals + j));       // c2 c2' c3 c4
    // r = x - y0: the head difference is exact (Sterbenz, x / y0 in [2/3, 4/3] for j >= 1; y0 = 0
    // for j = 0); with x's tail it is renormalised, so that the cross terms below stay small
    const float y0 = j ? __fmaf_rn(__int2float_rn(j), 0.00390625f, 0.001953125f) : 0.f;   // exact: (j + 1/2) 2^-8
    const dflt r = df_two_sum(__fsub_rn(x.h, y0), x.l);
    const float rh = r.h, rl = r.l;
    const float t = __fmaf_rn(B.w, rh, B.z);
    // u = c2 + r t
    const dflt u = df_fast_two_sum(B.x, __fmaf_rn(rh, t, __fmaf_rn(rl, t, B.y)));
    // v = c1 + r u
    float p = __fmul_rn(rh, u.h);
    float pe = __fmaf_rn(rh, u.h, -p);
    pe = __fmaf_rn(rh, u.l, pe);
    pe = __fmaf_rn(rl, u.h, pe);
    dflt v = df_fast_two_sum(A.z, p);
    v.l = __fadd_rn(v.l, __fadd_rn(pe, A.w));
    // g = c0 + r v
    p = __fmul_rn(rh, v.h);
    pe = __fmaf_rn(rh, v.h, -p);
    pe = __fmaf_rn(rh, v.l, pe);
    pe = __fmaf_rn(rl, v.h, pe);
    dflt g = df_fast_two_sum(A.x, p);
    g.l = __fadd_rn(g.l, __fadd_rn(pe, A.y));
    return g;
}

// d 2^e for a double d >= 0, by its exponent bits (d = 0 stays 0)
__device__ __forceinline__ double scale2(const double d, const int e)
{
    const long long b = __double_as_longlong(d);
    return b == 0 ? d : __longlong_as_double(b + (long long)e * (1LL << 52));
}

// ---- the blackbody rate on the FP32 pipe (FP64 march): the cubic pieces of spectrum.h as
// double-float pairs, evaluated by one code path for every segment between 2^-20 and 2^14.

// Piece and exact position of tau in [2^-20, 2^14) as a double-float (the 47 or 45 fraction bits
// split over head and tail), and the piece's width exponent.
__device__ __forceinline__ int lin_locate_df(const double tau, dflt& t, int& wexp)
{
    const long long b = __double_as_longlong(tau);
    const int e = (int)(b >> 52) - 1023;
    const int hb = e < 0 ? 5 : 7;
    const int fb = 52 - hb;
    const unsigned long long m = (unsigned long long)b & ((1ULL << fb) - 1);
    t.h = __fmul_rn(__uint2float_rn((unsigned)(m >> (fb - 24))), 5.9604644775390625e-08f);           // 2^-24
    t.l = __fmul_rn(__uint2float_rn((unsigned)(m & ((1ULL << (fb - 24)) - 1))), __uint_as_float((unsigned)(127 - fb) << 23));
    wexp = e - hb;
    return e < 0 ? (e - kLinExpLo) * 32 + (int)((b >> 47) & 31) : kLinOmega + (e << 7) + (int)((b >> 45) & 127);
}

__device__ __forceinline__ dflt df_neg(const dflt a)
{
    return {-a.h, -a.l};
}

// (Phi(t0) - Phi(t0 + T)) / T on the piece {a, b}: -(c1 + c2 s1 + c3 s2), s1 = t0 + t1,
// s2 = t0 s1 + t1^2 (the mean slope of the cubic, free of cancellation); t0 = 0 in lin_slope0_df.
__device__ __forceinline__ dflt lin_slope_df(const float4 a, const float4 b, const dflt t0, const dflt T)
{
    const dflt t1 = df_add(t0, T);
    const dflt s1 = df_add(t0, t1);
    const dflt s2 = df_add(df_mul(t0, s1), df_mul(t1, t1));
    const dflt D = df_add(dflt{a.z, a.w}, df_add(df_mul(dflt{b.x, b.y}, s1), df_mul(dflt{b.z, b.w}, s2)));
    return df_neg(D);
}

__device__ __forceinline__ dflt lin_slope0_df(const float4 a, const float4 b, const dflt T)
{
    const dflt D = df_add(dflt{a.z, a.w}, df_mul(T, df_add(dflt{b.x, b.y}, df_mul(T, dflt{b.z, b.w}))));
    return df_neg(D);
}

// Phi(tau0) - Phi(tau0 + dtau) for 2^-20 <= tau0 and tau1 = tau0 + dtau (rounded) < 2^14: the part in
// tau0's piece, the whole pieces after it (node values: Omega below tau = 1, Phi above), and the part
// in tau1's piece. When tau1 lies in the next piece, the depth past the node is dtau less the first
// part, so a segment that just crosses a node keeps its precision; further on, tau1's own position.
__device__ __forceinline__ dflt lin_frac_df(const float4* __restrict__ P, const double tau0, const double tau1,
                                            const double dtau)
{
    dflt t0, t1;
    int w0, w1;
    const int k0 = lin_locate_df(tau0, t0, w0);
    const int k1 = lin_locate_df(tau1, t1, w1);
    const bool same = k1 == k0;
    const dflt T = df_of(scale2(dtau, -w0));                   // dtau in units of piece k0's width
    const dflt T0 = same ? T : df_add(dflt{1.f, 0.f}, df_neg(t0));
    const dflt f0 = df_mul(T0, lin_slope_df(P[2 * k0], P[2 * k0 + 1], t0, T0));
    const dflt R = df_add(df_of(dtau), df_neg(df_scale(T0, w0)));
    const dflt T1 = same ? dflt{0.f, 0.f} : (k1 == k0 + 1 ? df_scale(R, -w1) : t1);
    const dflt f1 = df_mul(T1, lin_slope0_df(P[2 * k1], P[2 * k1 + 1], T1));
    // Phi_a - Phi_b over the whole pieces a = k0 + 1 .. b - 1, b = k1 (none unless k1 >= k0 + 2)
    const int ka = min(k0 + 1, kLinIntervals - 1);
    const float4 pa = P[2 * ka], pb = P[2 * k1];
    const dflt va = {pa.x, pa.y}, vb = {pb.x, pb.y};
    dflt mid;
    if (k1 < kLinOmega) mid = df_add(vb, df_neg(va));                       // Omega_b - Omega_a
    else if (ka >= kLinOmega) mid = df_add(va, df_neg(vb));                 // Phi_a - Phi_b
    else mid = df_add(dflt{1.f, 0.f}, df_neg(df_add(va, vb)));             // 1 - Omega_a - Phi_b
    if (k1 < k0 + 2) mid = dflt{0.f, 0.f};
    return df_add(f0, df_add(mid, f1));
}

// Psi(tau) as a double-float (the optically thin rate), by Horner on tau's piece.
__device__ __forceinline__ dflt lin_psi_df(const SpecTable<double>& S, const double tau)
{
    if (tau < kLinTauLo || tau >= kLinTauHi) return df_of(lin_psi(S, tau));
    dflt t;
    int w;
    const int k = lin_locate_df(tau, t, w);
    const float4 a = S.lin_bf[2 * k], b = S.lin_bf[2 * k + 1];
    const dflt c = df_add(dflt{a.z, a.w}, df_mul(t, df_add(dflt{b.x, b.y}, df_mul(t, dflt{b.z, b.w}))));
    return df_add(dflt{a.x, a.y}, df_mul(t, c));
}

// march_ray_table for FP64 physics, in double-float arithmetic as described above. kFreq: Eq. 1 over
// the blackbody spectrum; Q = P m_G 2^64 then stays the ray's geometric share (its photons are
// P Phi(tau)), and a segment deposits Q 2^64 r 2^(e_G - 128), r its rate per unit budget and G from
// the FP64 pieces in tau (lin_absorb: Phi(tau) - Phi(tau + dtau) over kap; kap = 0: Psi(tau) ds).
template <bool kHash, bool kFreq>
__device__ __forceinline__ bool march_ray_table_df(const SolveView<double>& V, const float* __restrict__ rtab,
                                                   const GeomLevel& GL, unsigned* err, const int l,
                                                   const uint32_t si, const uint32_t pix, const double P0,
                                                   double tau, const SrcEntry& se, const int4 dv, Tally& T,
                                                   double& oP, double& otau)
{
    using I = Ieee<double>;
    using TE = TableEntry<double>;
    using E = typename TE::E;
    const int n = V.n;
    const int s0 = dv.x < 0 ? -1 : 1, s1 = dv.y < 0 ? -1 : 1, s2 = dv.z < 0 ? -1 : 1;
    int i0 = se.cx, i1 = se.cy, i2 = se.cz;
    if (l > 0) {                    // the start cell: crossings done at the start sphere
        const long long rq_start = V.rq << (l - 1);
        i0 += s0 * (int)((rq_start * (unsigned)abs(dv.x) + kB) >> (S + F));
        i1 += s1 * (int)((rq_start * (unsigned)abs(dv.y) + kB) >> (S + F));
        i2 += s2 * (int)((rq_start * (unsigned)abs(dv.z) + kB) >> (S + F));
    }
    const bool periodic = V.rs != 0;
    const bool split_end = !periodic || (V.rq << l) < V.rs;
    if (periodic) {
        i0 = wrapn(i0, n);
        i1 = wrapn(i1, n);
        i2 = wrapn(i2, n);
    }
    const double ph = se.ph;
    const double taumax = V.tau_max;
    const unsigned long long rbase =
        (kHash && V.hash) ? mix64(((unsigned long long)(si - V.src_off) << 36) | ((unsigned long long)l << 31) | pix) : 0ULL;
    const bool face = V.overlap_mode == RT_OVERLAP_ARC || V.overlap_mode == RT_OVERLAP_CONSERVATIVE ||
                      V.overlap_mode == RT_OVERLAP_NAIVE;
    const bool corr = V.overlap_mode != RT_OVERLAP_NONE;
    const long long nn = (long long)n * n;
    ++T.rays;
    const double B0 = kFreq ? P0 * lin_phi(V.spec, tau) : P0;   // the photons the ray starts with
    if (!((unsigned)i0 < (unsigned)n && (unsigned)i1 < (unsigned)n && (unsigned)i2 < (unsigned)n)) {
        ++T.esc;
        T.escph += ph * B0;
        return false;
    }
    // G = m_G 2^e_G; the budget Q = P m_G 2^64, and 1 / m_G to read P back
    int eG;
    const dflt mG = df_mant(se.gd, eG);
    const int e_dep = kFreq ? eG - 128 : eG - 64;
    dflt Q = df_mul(df_of(scale2(P0, 64)), mG);
    dflt mGi;
    mGi.h = __frcp_rn(mG.h);
    mGi.l = __fmul_rn(__fmaf_rn(-mG.l, mGi.h, __fmaf_rn(-mG.h, mGi.h, 1.0f)), mGi.h);
    auto remaining = [&]() -> double {
        if constexpr (kFreq) return P0 * lin_phi(V.spec, tau);
        else return df_to_double(df_mul(Q, mGi), -64);
    };

    const E* col = TE::ent(GL) + GL.row0[pix >> 5] * 32 + (pix & 31);
    E e = col[0];
    int cell = (i2 * n + i1) * n + i0;
    double kcur = V.kap[cell];
    unsigned seq = 0;
    bool split = false;
    for (;;) {
        // the next entry and the next cell's kappa are requested before this segment's work
        const unsigned fl = TE::flags(e);
        const bool last = (fl >> 31) != 0u;
        const E en = last ? TE::none() : col[(unsigned long long)(seq + 1) * 32];
        const unsigned steps = (fl >> 24) & 7u;
        int ni0 = (steps & 1u) ? i0 + s0 : i0;
        int ni1 = (steps & 2u) ? i1 + s1 : i1;
        int ni2 = (steps & 4u) ? i2 + s2 : i2;
        if (periodic) {
            ni0 = wrap1(ni0, n);
            ni1 = wrap1(ni1, n);
            ni2 = wrap1(ni2, n);
        }
        const bool next_in =
            periodic || ((unsigned)ni0 < (unsigned)n && (unsigned)ni1 < (unsigned)n && (unsigned)ni2 < (unsigned)n);
        const int ncell = (ni2 * n + ni1) * n + ni0;
        const double knext = (steps && next_in) ? V.kap[ncell] : 0.0;
        const bool near = corr && ((fl >> 27) & 1u);
        int c2 = -1;
        if (face) {                      // the cell across the nearest face, as selects on every lane
            const int ax = (int)((fl >> 28) & 3u);
            const int step = ((fl >> 30) & 1u) ? 1 : -1;
            const int ia = pick3(ax, i0, i1, i2);
            const int jc = ia + step;
            const int stride = ax == 0 ? 1 : (ax == 1 ? n : (int)nn);
            if (periodic) c2 = cell + (wrap1(jc, n) - ia) * stride;
            else c2 = (unsigned)jc < (unsigned)n ? cell + step * stride : -1;
            if (!near) c2 = -1;
        }
        const double kn_raw = c2 >= 0 ? V.kap[c2] : 0.0;
        // ---- the two deciding FP64 operations: dtau = kap ds here, tau += dtau below
        const double ds = TE::ds(e);
        const double kap = I::mag(kcur);
        const double dtau = I::mul(kap, ds);
        // ---- Eq. 1: w = Q g ds, the segment's rate before the Eq. 5-8 share (double-float),
        // or its FP64 value wd for an opaque segment
        dflt w = {0.f, 0.f};
        dflt ux = {0.f, 0.f};             // gray: the photons the segment absorbs, Q g dtau = kap w
        double wd = 0.0;
        const bool opaque = !kFreq && I::pos(kap) && !I::lt(dtau, 2.0);
        const double tau1 = I::add(tau, dtau);
        int e_seg = e_dep;
        if constexpr (kFreq) {
            // w = Q r with r the segment's rate per unit budget and G: (Phi(tau) - Phi(tau1)) / kap,
            // its 2^-e_kap applied when rounding the deposit; Psi(tau) ds where kap = 0
            if (I::pos(kap)) {
                if (tau >= kLinTauLo && I::lt(tau1, kLinTauHi)) {
                    const dflt frac = lin_frac_df(V.spec.lin_af, tau, tau1, dtau);
                    int ek;
                    const dflt mk = df_mant(kap, ek);
                    dflt inv;
                    inv.h = __frcp_rn(mk.h);
                    inv.l = __fmul_rn(__fmaf_rn(-mk.l, inv.h, __fmaf_rn(-mk.h, inv.h, 1.0f)), inv.h);
                    w = df_mul(Q, df_mul(frac, inv));
                    e_seg = e_dep + 64 - ek;
                } else {                                   // below 2^-20 or past 2^14: FP64
                    double frac, r;
                    lin_absorb(V.spec, tau, dtau, kap, ds, frac, r);
                    w = df_mul(Q, df_of(scale2(r, 64)));
                }
            } else {
                w = df_mul(Q, df_mul(lin_psi_df(V.spec, tau), df_of(ds)));   // optically thin limit
                e_seg = e_dep + 64;
            }
        } else if (!opaque) {
            const dflt dsf = df_of_len(ds);
            if (I::pos(kap)) {
                const dflt x = df_of(dtau);
                const dflt u = df_mul(Q, rate_factor(rtab, x));
                ux = df_mul(u, x);
                Q = df_sub_part(Q, ux);           // ux = Q (1 - e^-dtau) < 7/8 Q below dtau = 2
                w = df_mul(u, dsf);
            } else {
                w = df_mul(Q, dsf);                       // optically thin limit
            }
        } else {
            const double Qd = df_to_double(Q, 0);
            const double aQ = Qd * (-expm1(-dtau));
            wd = aQ / kap;
            Q = df_of(Qd - aQ);
        }
        // ---- Eqs. 5-8: the cell's deposit and the neighbour's
        double dep = 0.0, dep2 = 0.0;
        int nbcell = -1;
        const int mode = V.overlap_mode;
        bool keep_all = !near;                           // f = 1
        bool squared = false, second = false;
        if (near) {
            if (mode == RT_OVERLAP_LINEAR) {
            } else if (mode == RT_OVERLAP_SQUARED) {
                squared = true;
            } else {
                const double kn = I::mag(kn_raw);
                const bool elig = c2 >= 0 && ((mode == RT_OVERLAP_ARC) ? I::pos(kn) : (!I::neg(kn_raw) && I::pos(kn)));
                second = elig;
                keep_all = !elig && mode != RT_OVERLAP_NAIVE;   // naive threshold: the Eq. 5 share regardless
            }
        }
        if (opaque) {
            if (keep_all) {
                dep = scale2(wd, e_dep);
            } else {
                const double fd = TE::f(e);
                dep = scale2(fd * (squared ? fd * wd : wd), e_dep);
                if (second) dep2 = scale2(((1.0 - fd) * wd) * (kap / I::mag(kn_raw)), e_dep);
            }
        } else {
            // one path for every lane: f = 1 where the whole rate stays (1 w is w exactly)
            const dflt f = keep_all ? dflt{1.f, 0.f} : TE::f_df(e);
            const dflt fw = df_mul(f, w);
            dep = df_to_double_pos(squared ? df_mul(f, fw) : fw, e_seg);
            if (second && I::pos(kap)) {           // kap = 0 (an ionized cell) sends 0 to c'
                // 1 - f, renormalised: the head difference is exact and at least f's tail, so a
                // share near f = 1 keeps its relative precision through the products below
                const dflt om = df_fast_two_sum(__fsub_rn(1.0f, f.h), -f.l);
                int en;
                const dflt mn = df_mant(I::mag(kn_raw), en);
                // ux carries dtau's full double-float only from 2^-74 on (df_of keeps the head alone
                // below), so thinner segments and the blackbody rate take the ratio kap / kap'
                if (kFreq || I::lt(dtau, 0x1p-74)) {
                    // Eq. 8: (1 - f) w kap / kap', the ratio of the mantissas by a float reciprocal
                    // and one correction, the exponents applied when rounding to double
                    int ek;
                    const dflt mk = df_mant(kap, ek);
                    const float r0 = __frcp_rn(mn.h);
                    const float q0 = __fmul_rn(mk.h, r0);
                    const float p = __fmul_rn(mn.h, q0);
                    const float pe = __fmaf_rn(mn.h, q0, -p);
                    const float rho = __fmaf_rn(-q0, mn.l, __fadd_rn(__fsub_rn(__fsub_rn(mk.h, p), pe), mk.l));
                    const dflt ratio = {q0, __fmul_rn(rho, r0)};
                    dep2 = df_to_double_pos(df_mul(df_mul(om, w), ratio), e_seg + ek - en);
                } else {
                    // Eq. 8 from the absorbed photons: w kap = Q g dtau = ux, so the share is
                    // (1 - f) ux / kap', by the double-float reciprocal of kap''s mantissa, its
                    // exponent applied when rounding to double
                    dep2 = df_to_double_pos(df_mul(df_mul(om, ux), df_rcp12(mn)), e_seg - en);
                }
            }
        }
        if (second) nbcell = c2;
        atomicAdd(&V.gamma[cell], dep);
        if (nbcell >= 0) {
            atomicAdd(&V.gamma[nbcell], dep2);
            ++T.sec;
        }
        tau = tau1;
        if (kHash && V.hash) T.hash += mix64(rbase ^ ((unsigned long long)seq << 40) ^ (unsigned long long)cell);
        ++seq;
        if (!I::lt(tau, taumax)) {             // photons spent
            ++T.dtau;
            T.dropph += ph * remaining();
            break;
        }
        if (!steps) {                    // the segment ended on the end sphere
            if (!split_end) {            // travelled sqrt(3) L_box (Sec. 2.5.1)
                ++T.esc;
                T.escph += ph * remaining();
            } else if (l + 1 > V.level_max) {
                ++T.dlev;
                T.dropph += ph * remaining();
            } else {
                ++T.split;
                split = true;
                oP = kFreq ? P0 : remaining();
                otau = tau;
            }
            break;
        }
        if (!next_in) {
            ++T.esc;
            T.escph += ph * remaining();
            break;
        }
        if (last) {                      // cannot happen: a table ends where every grid is left
            atomicOr(err, kErrGeometry);
            break;
        }
        i0 = ni0;
        i1 = ni1;
        i2 = ni2;
        cell = ncell;
        kcur = knext;
        e = en;
    }
    T.seg += seq;
    T.abs += ph * (B0 - remaining());
    return split;
}

// Load child j of the level-l parents (level 0: ray j of the emission, 12 per source).
template <class R>
__device__ __forceinline__ void load_ray(int l, long long j, const RayBuf<R>& in, uint32_t& si, uint32_t& pix, R& P,
                                         R& tau, R& cP, R& ctau)
{
    using I = Ieee<R>;
    if (l == 0) {
        si = (uint32_t)(j / 12);
        pix = (uint32_t)(j - 12LL * si);
        P = (R)1;
        tau = (R)0;
        cP = (R)0;
        ctau = (R)0;
    } else {
        const long long q = j >> 2;
        si = in.src[q];
        pix = 4u * in.pix[q] + (uint32_t)(j & 3);
        P = I::mul(in.P[q], (R)0.25);
        tau = in.tau[q];
        cP = (R)0;
        ctau = (R)0;
        if constexpr (sizeof(R) == 4) {
            cP = I::mul(in.cP[q], 0.25f);
            ctau = in.ctau[q];
        }
    }
}

// Sum a tally over the warp lanes in `mask` that carry the same solve, and add
// it into that solve's statistics (one atomic per group and counter).
__device__ __forceinline__ void flush_tally(Tally& T, unsigned mask, DevStats* const* st_of_lane, int l)
{
    const int lane = threadIdx.x & 31;
    DevStats* mine = *st_of_lane;
    while (mask) {
        const int leader = __ffs(mask) - 1;
        const unsigned long long key = __shfl_sync(mask, (unsigned long long)mine, leader);
        const unsigned grp = __ballot_sync(mask, (unsigned long long)mine == key);
        if ((grp >> lane) & 1u) {
            const unsigned rays = __reduce_add_sync(grp, T.rays), split = __reduce_add_sync(grp, T.split);
            const unsigned esc = __reduce_add_sync(grp, T.esc), dtau = __reduce_add_sync(grp, T.dtau);
            const unsigned dlev = __reduce_add_sync(grp, T.dlev), seg = __reduce_add_sync(grp, T.seg);
            const unsigned sec = __reduce_add_sync(grp, T.sec);
            unsigned long long hash = 0ULL;
            double ab = 0.0, ep = 0.0, dp = 0.0;
            for (unsigned g = grp; g; g &= g - 1) {
                const int b = __ffs(g) - 1;
                hash += __shfl_sync(grp, T.hash, b);
                ab += __shfl_sync(grp, T.abs, b);
                ep += __shfl_sync(grp, T.escph, b);
                dp += __shfl_sync(grp, T.dropph, b);
            }
            if (lane == leader && rays) {
                DevStats* st = mine;
                atomicAdd(&st->rays[l], (unsigned long long)rays);
                if (split) atomicAdd(&st->splits[l], (unsigned long long)split);
                if (esc) atomicAdd(&st->escaped[l], (unsigned long long)esc);
                if (dtau) atomicAdd(&st->dropped_tau[l], (unsigned long long)dtau);
                if (dlev) atomicAdd(&st->dropped_level[l], (unsigned long long)dlev);
                atomicAdd(&st->segments[l], (unsigned long long)seg);
                if (sec) atomicAdd(&st->secondary[l], (unsigned long long)sec);
                if (hash) atomicAdd(&st->visit_hash, hash);
                atomicAdd(&st->absorbed, ab);
                atomicAdd(&st->escaped_ph, ep);
                atomicAdd(&st->dropped_ph, dp);
            }
            T.clear();
        }
        mask &= ~grp;
    }
}

// Resident blocks of 256 threads per SM the march kernels are compiled for:
// the FP32 march fits 80 registers without spilling, so three blocks (24
// warps) hide more of its dependency latency than two; the FP64 march is held
// by the FP64 pipe and would spill at that size.
template <class R>
struct MarchOccupancy {
    static constexpr int blocks = sizeof(R) == 4 ? 3 : 2;
};

// One level (or one slice of it) of one solve: thread j marches child j.
// kHash: compiled with the visit hash (only launched when it is asked for).
template <class R, bool kHash, bool kFreq>
__global__ void __launch_bounds__(256, MarchOccupancy<R>::blocks) march_kernel(const MarchArgs<R> A)
{
    const int l = A.level;
    const int lane = threadIdx.x & 31;
    const long long gwarp = (long long)(blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarp = (long long)(gridDim.x * blockDim.x) >> 5;
    SolveView<R> V;
    V.kap = A.kap;
    V.gamma = A.gamma;
    V.n = A.n;
    V.level_max = A.level_max;
    V.overlap_mode = A.overlap_mode;
    V.hash = A.hash;
    V.rq = A.rq;
    V.tau_max = A.tau_max;
    V.src_off = 0;
    V.rs = A.rs;
    V.spec = A.spec;
    // children of this launch: as given, or bounded by the parents the previous level counted
    const long long c1 = A.in_count ? min((long long)A.c1, (long long)A.c0 + 4LL * (long long)*A.in_count) : (long long)A.c1;
    Tally T;
    T.clear();
    for (long long base = A.c0 + gwarp * 32; base < c1; base += nwarp * 32) {
        const long long j = base + lane;
        bool split = false;
        uint32_t si = 0, pix = 0;
        R oP = 0, otau = 0;
        float ocP = 0.f, octau = 0.f;
        if (j < c1) {
            R P, tau, cP, ctau;
            load_ray<R>(l, j, A.in, si, pix, P, tau, cP, ctau);
            split = march_ray<R, kHash, kFreq>(V, l, si, pix, P, tau, cP, ctau, A.src[si], A.dirs[pix], T, oP, otau,
                                               ocP, octau);
        }
        append_split<R>(split, si, pix, oP, otau, ocP, octau, A.out, A.out_count, &A.st->err);
    }
    DevStats* st = A.st;
    flush_tally(T, 0xffffffffu, &st, l);
}

// One level (or one slice of it) of one solve, geometry from the level's table (kFreq: Eq. 1 over
// the blackbody spectrum). Without the walk the FP32 march fits 64 registers, so four blocks (32
// warps) per SM. The FP64 march, latency-bound in its double-float arithmetic, runs three (80
// registers, a spill of a few dozen bytes): 57 against 50 G segments/s with two.
template <class R>
struct TableOccupancy {
    static constexpr int blocks = sizeof(R) == 4 ? 4 : 3;
};

template <class R, bool kHash, bool kFreq>
__global__ void __launch_bounds__(256, TableOccupancy<R>::blocks) march_table_kernel(const MarchArgs<R> A, const GeomLevel GL)
{
    const int l = A.level;
    const int lane = threadIdx.x & 31;
    const long long gwarp = (long long)(blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarp = (long long)(gridDim.x * blockDim.x) >> 5;
    SolveView<R> V;
    V.kap = A.kap;
    V.gamma = A.gamma;
    V.n = A.n;
    V.level_max = A.level_max;
    V.overlap_mode = A.overlap_mode;
    V.hash = A.hash;
    V.rq = A.rq;
    V.tau_max = A.tau_max;
    V.src_off = 0;
    V.rs = A.rs;
    V.spec = A.spec;
    // children of this launch: as given, or bounded by the parents the previous level counted
    const long long c1 = A.in_count ? min((long long)A.c1, (long long)A.c0 + 4LL * (long long)*A.in_count) : (long long)A.c1;
    Tally T;
    T.clear();
    // FP64 march in double-float arithmetic; gray: the Eq. 1 rate table in shared memory (two float4
    // arrays, see rate_factor)
    constexpr bool kDf = sizeof(R) == 8;
    __shared__ __align__(16) float rtab[(kDf && !kFreq) ? kRateSmem : 4];
    if constexpr (kDf && !kFreq) {
        for (int i = threadIdx.x; i < kRateSmem; i += blockDim.x) {
            const int row = (i >> 2) % kRateIntervals, half = (i >> 2) / kRateIntervals;
            rtab[i] = kRateTable[row * kRateCoefs + 4 * half + (i & 3)];
        }
        __syncthreads();
    }
    for (long long base = A.c0 + gwarp * 32; base < c1; base += nwarp * 32) {
        const long long j = base + lane;
        bool split = false;
        uint32_t si = 0, pix = 0;
        R oP = 0, otau = 0;
        float ocP = 0.f, octau = 0.f;
        if (j < c1) {
            R P, tau, cP, ctau;
            load_ray<R>(l, j, A.in, si, pix, P, tau, cP, ctau);
            if constexpr (kDf) {
                split = march_ray_table_df<kHash, kFreq>(V, rtab, GL, &A.st->err, l, si, pix, P, tau, A.src[si],
                                                         A.dirs[pix], T, oP, otau);
            } else {
                split = march_ray_table<R, kHash, kFreq>(V, GL, &A.st->err, l, si, pix, P, tau, cP, ctau, A.src[si],
                                                         A.dirs[pix], T, oP, otau, ocP, octau);
            }
        }
        append_split<R>(split, si, pix, oP, otau, ocP, octau, A.out, A.out_count, &A.st->err);
    }
    DevStats* st = A.st;
    flush_tally(T, 0xffffffffu, &st, l);
}

// All solves of a batch in one cooperative launch. Every block runs the same
// depth-first schedule over (level, slice of children): a slice's children are
// claimed in tiles by warps through a device counter (the work queue), the
// parents that split go to the next level's buffer, and grid.sync() separates
// slices; the next level's slices run before the current level's remaining ones,
// so no buffer ever holds more than one slice's output. Only CUDA's grid barrier
// is waited on: no block spins on another's flag.
// kSingle: the launch holds one solve, passed by value in A.one, so its parameters are the same
// for every lane (kernel parameters, not per-lane loads) and no tally changes hands. Only then does
// the table-driven kernel fit four blocks per SM; with per-lane solve parameters it takes three.
template <class R, bool kHash, bool kTable, bool kSingle, bool kFreq>
__global__ void __launch_bounds__(256, (kTable && kSingle) ? TableOccupancy<R>::blocks : MarchOccupancy<R>::blocks)
    batch_kernel(const BatchArgs<R> A)
{
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    const int lane = threadIdx.x & 31;
    // FP64 solves on the geometry tables: the Eq. 1 rate table of the double-float march in shared
    // memory (gray rate only)
    constexpr bool kDf = kTable && sizeof(R) == 8;
    __shared__ __align__(16) float rtab[(kDf && !kFreq) ? kRateSmem : 4];
    if constexpr (kDf && !kFreq) {
        for (int i = threadIdx.x; i < kRateSmem; i += blockDim.x) {
            const int row = (i >> 2) % kRateIntervals, half = (i >> 2) / kRateIntervals;
            rtab[i] = kRateTable[row * kRateCoefs + 4 * half + (i & 3)];
        }
        __syncthreads();
    }
    int lev[RT_MAX_LEVELS + 1];
    long long tot[RT_MAX_LEVELS + 1], nxt[RT_MAX_LEVELS + 1];
    int depth = 0;
    lev[0] = 0;
    tot[0] = 12LL * A.nsrc;
    nxt[0] = 0;
    int sid = 0;
    while (depth >= 0) {
        if (nxt[depth] >= tot[depth]) {
            --depth;
            continue;
        }
        const int l = lev[depth];
        const long long c0 = nxt[depth];
        const long long c1 = min(tot[depth], c0 + A.slice);
        nxt[depth] = c1;
        if (sid >= A.max_slices || l > A.table_level || depth >= RT_MAX_LEVELS) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(A.err, kErrLevel);
            break;
        }
        const int4* dirs = A.dirs + 4LL * ((1LL << (2 * l)) - 1);
        Tally T;
        T.clear();
        DevStats* cur = nullptr;
        for (;;) {
            long long t = 0;
            if (lane == 0) t = (long long)atomicAdd(&A.tiles[sid], 1ULL);
            t = __shfl_sync(0xffffffffu, t, 0);
            const long long s0 = c0 + t * A.tile;
            if (s0 >= c1) break;
            const long long s1 = min(c1, s0 + (long long)A.tile);
            for (long long base = s0; base < s1; base += 32) {
                const long long j = base + lane;
                bool split = false;
                uint32_t si = 0, pix = 0;
                R oP = 0, otau = 0;
                float ocP = 0.f, octau = 0.f;
                DevStats* st = cur;
                SrcEntry se;
                R P = 0, tau = 0, cP = 0, ctau = 0;
                if (j < s1) {
                    load_ray<R>(l, j, A.buf[l], si, pix, P, tau, cP, ctau);
                    se = A.src[si];
                    st = kSingle ? A.one.st : A.solves[se.pad].st;
                }
                if constexpr (!kSingle) {
                    // a lane whose solve changes hands its tally over first
                    const unsigned chg = __ballot_sync(0xffffffffu, cur != nullptr && st != cur);
                    if (chg) flush_tally(T, chg, &cur, l);
                }
                if (j < s1) {
                    cur = st;
                    const BatchSolve& bs = kSingle ? A.one : A.solves[se.pad];
                    SolveView<R> V;
                    V.kap = static_cast<const R*>(bs.kap);
                    V.gamma = bs.gamma;
                    V.n = bs.n;
                    V.level_max = bs.level_max;
                    V.overlap_mode = bs.overlap_mode;
                    V.hash = bs.hash;
                    V.rq = bs.rq;
                    V.rs = bs.rs;
                    V.tau_max = (R)bs.tau_max;
                    V.src_off = bs.src_off - A.src_base;
                    if constexpr (kFreq) V.spec = A.spec;
                    if constexpr (kDf) {
                        split = march_ray_table_df<kHash, kFreq>(V, rtab, A.geo[l], A.err, l, si, pix, P, tau, se,
                                                                 dirs[pix], T, oP, otau);
                    } else if constexpr (kTable) {
                        split = march_ray_table<float, kHash, kFreq>(V, A.geo[l], A.err, l, si, pix, P, tau, cP, ctau, se,
                                                                     dirs[pix], T, oP, otau, ocP, octau);
                    } else {
                        split = march_ray<R, kHash, kFreq>(V, l, si, pix, P, tau, cP, ctau, se, dirs[pix], T, oP, otau,
                                                           ocP, octau);
                    }
                }
                append_split<R>(split, si, pix, oP, otau, ocP, octau, A.buf[l + 1], &A.counts[sid], A.err);
            }
        }
        const unsigned have = __ballot_sync(0xffffffffu, cur != nullptr);
        if (have) flush_tally(T, have, &cur, l);
        grid.sync();
        const unsigned long long nn = *((volatile unsigned long long*)&A.counts[sid]);
        ++sid;
        if (nn > 0) {
            ++depth;
            lev[depth] = l + 1;
            tot[depth] = 4LL * (long long)nn;
            nxt[depth] = 0;
        }
    }
}

}  // namespace

template <class R>
static int launch_march_impl(const MarchArgs<R>& a, int grid, int block, cudaStream_t s)
{
    const bool freq = a.spec.lin_a != nullptr;
    if (a.hash) {
        if (freq) march_kernel<R, true, true><<<grid, block, 0, s>>>(a);
        else march_kernel<R, true, false><<<grid, block, 0, s>>>(a);
    } else {
        if (freq) march_kernel<R, false, true><<<grid, block, 0, s>>>(a);
        else march_kernel<R, false, false><<<grid, block, 0, s>>>(a);
    }
    return 1;
}

int launch_march_f64(const MarchArgs<double>& a, int grid, int block, cudaStream_t s)
{
    return launch_march_impl<double>(a, grid, block, s);
}

int launch_march_f32(const MarchArgs<float>& a, int grid, int block, cudaStream_t s)
{
    return launch_march_impl<float>(a, grid, block, s);
}

int launch_march_table_f32(const MarchArgs<float>& a, const GeomLevel& g, int grid, int block, cudaStream_t s)
{
    if (a.spec.lin_a) {
        if (a.hash) march_table_kernel<float, true, true><<<grid, block, 0, s>>>(a, g);
        else march_table_kernel<float, false, true><<<grid, block, 0, s>>>(a, g);
    } else {
        if (a.hash) march_table_kernel<float, true, false><<<grid, block, 0, s>>>(a, g);
        else march_table_kernel<float, false, false><<<grid, block, 0, s>>>(a, g);
    }
    return 1;
}

int launch_march_table_f64(const MarchArgs<double>& a, const GeomLevel& g, int grid, int block, cudaStream_t s)
{
    if (a.spec.lin_a) {
        if (a.hash) march_table_kernel<double, true, true><<<grid, block, 0, s>>>(a, g);
        else march_table_kernel<double, false, true><<<grid, block, 0, s>>>(a, g);
    } else {
        if (a.hash) march_table_kernel<double, true, false><<<grid, block, 0, s>>>(a, g);
        else march_table_kernel<double, false, false><<<grid, block, 0, s>>>(a, g);
    }
    return 1;
}

void launch_geom_count(long long rq, int l, const int4* dirs, long long npix, int n_cover, long long rs,
                       unsigned* rows, cudaStream_t s)
{
    const long long grid = (npix + 255) / 256;
    geom_count_kernel<<<(unsigned)grid, 256, 0, s>>>(rq, l, dirs, npix, n_cover, rs, rows);
}

void launch_geom_fill(long long rq, int l, const int4* dirs, long long npix, int n_cover, long long rs,
                      const unsigned long long* row0, uint2* ent, unsigned* err, cudaStream_t s)
{
    const long long grid = (npix + 255) / 256;
    geom_fill_kernel<<<(unsigned)grid, 256, 0, s>>>(rq, l, dirs, npix, n_cover, rs, row0, ent, err);
}

void launch_geom_fill64(long long rq, int l, const int4* dirs, long long npix, int n_cover, long long rs,
                        const unsigned long long* row0, unsigned long long rows_total, ulonglong2* ent,
                        unsigned* err, cudaStream_t s)
{
    const long long grid = (npix + 255) / 256;
    geom_fill64_kernel<<<(unsigned)grid, 256, 0, s>>>(rq, l, dirs, npix, n_cover, rs, row0, rows_total, ent, err);
}

template <class R, bool kSingle, bool kFreq>
static const void* batch_kernel_pick(bool hash, bool table)
{
    if (table)
        return hash ? (const void*)batch_kernel<R, true, true, kSingle, kFreq>
                    : (const void*)batch_kernel<R, false, true, kSingle, kFreq>;
    return hash ? (const void*)batch_kernel<R, true, false, kSingle, kFreq>
                : (const void*)batch_kernel<R, false, false, kSingle, kFreq>;
}

template <class R>
static const void* batch_kernel_for(bool hash, bool table, bool single, bool freq)
{
    if (freq) return single ? batch_kernel_pick<R, true, true>(hash, table) : batch_kernel_pick<R, false, true>(hash, table);
    return single ? batch_kernel_pick<R, true, false>(hash, table) : batch_kernel_pick<R, false, false>(hash, table);
}

template <class R>
static cudaError_t launch_batch_impl(const BatchArgs<R>& a, int grid, int block, cudaStream_t s)
{
    void* args[] = {const_cast<BatchArgs<R>*>(&a)};
    return cudaLaunchCooperativeKernel(batch_kernel_for<R>(a.any_hash != 0, a.use_geo != 0, a.single != 0, a.freq != 0),
                                       dim3(grid), dim3(block), args, 0, s);
}

cudaError_t launch_batch_f64(const BatchArgs<double>& a, int grid, int block, cudaStream_t s)
{
    return launch_batch_impl<double>(a, grid, block, s);
}

cudaError_t launch_batch_f32(const BatchArgs<float>& a, int grid, int block, cudaStream_t s)
{
    return launch_batch_impl<float>(a, grid, block, s);
}

// Co-resident blocks per SM of the batch kernel variant (walking or table-driven, one solve or
// many, gray or blackbody rate): the smaller of its two visit-hash instantiations, so that a
// cooperative launch sized by it fits either.
int batch_blocks_per_sm(int precision, int block, bool table, bool single, bool freq)
{
    int best = 1 << 30;
    for (int hash = 0; hash < 2; ++hash) {
        const void* k = precision == RT_FP32 ? batch_kernel_for<float>(hash, table, single, freq)
                                             : batch_kernel_for<double>(hash, table, single, freq);
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, 0);
        best = std::min(best, nb);
    }
    return best;
}

}  // namespace nyx
