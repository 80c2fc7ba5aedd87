// Frequency-integrated photoionization (Eq. 1 integrated over the source
// spectrum; Sec. 2.5, after C2-Ray): a blackbody source at T_bb and a
// hydrogen cross-section sigma_nu = sigma_0 (nu_0 / nu)^3 above the
// threshold. With s = sigma_nu / sigma_0, a ray that has crossed threshold
// optical depth tau keeps the fraction Phi(tau) = <exp(-tau s)> of its
// photons (average over the photon-number spectrum), absorbs
// Phi(tau) - Phi(tau + dtau) over a segment of optical depth dtau, and in an
// optically thin cell deposits at the rate Psi(tau) = <s exp(-tau s)> per unit
// dtau.
//
// Phi and Psi are read from cubic pieces in tau itself, built once per
// temperature. Below tau = 1, piece k covers [2^e (1 + i/32), 2^e (1 + (i+1)/32))
// with e = kLinExpLo + k / 32 and i = k % 32; from tau = 1 on the pieces are four
// times finer, 128 per octave, where a cubic in tau follows Phi less closely. So
// k and the position t in [0, 1) come exactly from the bits of tau (no
// logarithm), and a piece's width is a power of two. Below 2^-20 Phi follows its
// series in tau; above 2^14 it keeps its value there.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

namespace nyx {

constexpr double kSpecTauHi = 1e4;                          // largest tau_max with the blackbody rate
constexpr int kLinExpLo = -20;
constexpr int kLinOmega = -kLinExpLo * 32;                  // the pieces below tau = 1
constexpr int kLinIntervals = kLinOmega + 14 * 128;         // up to 2^14
constexpr double kLinTauLo = 9.5367431640625e-07;           // 2^-20
constexpr double kLinTauHi = 16384.0;                       // 2^14

// One cubic piece: on piece k, Phi(t) - Phi_k = c1 t + c2 t^2 + c3 t^3 (lin_a) and Psi(t) = v + c1 t
// + c2 t^2 + c3 t^3 (lin_b). In lin_a, v is Phi_k from tau = 1 on and Omega_k = 1 - Phi_k below it,
// so that small absorbed fractions keep their relative precision.
struct __align__(32) LinPiece {
    double v, c1, c2, c3;
};

// The pieces of one temperature on one device (or the host). lin_a / lin_b: the FP64 pieces, read by
// the FP64 walk and, on the host, by rt_spectrum_eval; lin_af / lin_bf: the same as double-float
// pairs for the FP64 table march, two float4 per piece, {v.h, v.l, c1.h, c1.l}, {c2.h, c2.l, c3.h,
// c3.l}; lin_f: the FP32 march's pieces rounded to float, one float4 {v, c1, c2, c3} per piece, the
// Phi pieces then the Psi pieces. psi0 = <s>, xi0 = <s^2>, zeta0 = <s^3> (the series below 2^-20);
// phi_end and psi_end at 2^14. lin_a null: the gray rate.
template <class R>
struct SpecTable {
    const LinPiece* lin_a = nullptr;
    const LinPiece* lin_b = nullptr;
    const float4* lin_af = nullptr;
    const float4* lin_bf = nullptr;
    const float4* lin_f = nullptr;
    double psi0 = 0, xi0 = 0, zeta0 = 0, phi_end = 0, psi_end = 0;
};

__host__ __device__ __forceinline__ long long lin_bits(const double x)
{
#ifdef __CUDA_ARCH__
    return __double_as_longlong(x);
#else
    long long b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}

__host__ __device__ __forceinline__ double lin_double(const long long b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double x;
    std::memcpy(&x, &b, sizeof x);
    return x;
#endif
}

// 2^n as a double, for a normal result
__host__ __device__ __forceinline__ double lin_pow2(const int n)
{
    return lin_double((long long)(1023 + n) << 52);
}

// Piece, exact position t and width 2^wexp of a double tau in [2^-20, 2^14): k from the exponent and
// the top five (below 1) or seven mantissa bits, t from the others (exactly representable).
__host__ __device__ __forceinline__ int lin_locate(const double tau, double& t, int& wexp)
{
    const long long b = lin_bits(tau);
    const int e = (int)(b >> 52) - 1023;
    const int hb = e < 0 ? 5 : 7;
    t = lin_double(0x3FF0000000000000LL | ((b & ((1LL << (52 - hb)) - 1)) << hb)) - 1.0;
    wexp = e - hb;
    return e < 0 ? (e - kLinExpLo) * 32 + (int)((b >> 47) & 31) : kLinOmega + (e << 7) + (int)((b >> 45) & 127);
}

__host__ __device__ __forceinline__ int lin_index(const double tau)
{
    double t;
    int w;
    return lin_locate(tau, t, w);
}

// The width exponent of piece k.
__host__ __device__ __forceinline__ int lin_wexp(const int k)
{
    return k < kLinOmega ? kLinExpLo + k / 32 - 5 : ((k - kLinOmega) >> 7) - 7;
}

// Omega(tau) = 1 - Phi(tau) below 2^-20: tau <s> - tau^2 <s^2> / 2 + tau^3 <s^3> / 6 (the next
// term, below 2^-80 / 24, is dropped).
__host__ __device__ __forceinline__ double lin_series(const SpecTable<double>& S, const double tau)
{
    return tau * fma(-tau, fma(-tau, S.zeta0 * (1.0 / 6.0), 0.5 * S.xi0), S.psi0);
}

// Omega(tau) below tau = 1, Phi(tau) from 1 on.
__host__ __device__ __forceinline__ double lin_rep(const SpecTable<double>& S, const double tau)
{
    if (tau < kLinTauLo) return lin_series(S, tau);
    if (tau >= kLinTauHi) return S.phi_end;
    double t;
    int we;
    const int k = lin_locate(tau, t, we);
    const LinPiece p = S.lin_a[k];
    const double c = t * fma(t, fma(t, p.c3, p.c2), p.c1);
    return k < kLinOmega ? p.v - c : p.v + c;
}

// Phi(tau): the fraction of a ray's photons left after threshold optical depth tau.
__host__ __device__ __forceinline__ double lin_phi(const SpecTable<double>& S, const double tau)
{
    const double r = lin_rep(S, tau);
    return tau < 1.0 ? 1.0 - r : r;
}

// Psi(tau): the optically thin deposition rate per unit threshold optical depth.
__host__ __device__ __forceinline__ double lin_psi(const SpecTable<double>& S, const double tau)
{
    if (tau < kLinTauLo) return fma(-tau, fma(-tau, 0.5 * S.zeta0, S.xi0), S.psi0);
    if (tau >= kLinTauHi) return S.psi_end;
    double t;
    int we;
    const int k = lin_locate(tau, t, we);
    const LinPiece p = S.lin_b[k];
    return fma(t, fma(t, fma(t, p.c3, p.c2), p.c1), p.v);
}

// (Phi(t0) - Phi(t0 + T)) / T on piece p: minus the mean slope of its cubic, (c1 + c2 s1 + c3 s2)
// with s1 = t0 + t1, s2 = t0^2 + t0 t1 + t1^2, so a thin segment loses nothing to cancellation.
__host__ __device__ __forceinline__ double lin_slope(const LinPiece& p, const double t0, const double T)
{
    const double t1 = t0 + T;
    const double s1 = t0 + t1;
    const double s2 = fma(t0, s1, t1 * t1);
    return -fma(p.c3, s2, fma(p.c2, s1, p.c1));
}

// A segment of optical depth dtau = kap ds after tau0 (kap > 0): frac = Phi(tau0) - Phi(tau0 + dtau),
// the fraction of the ray's photons it absorbs, and per_kap = frac / kap. Within one piece the
// difference is T = dtau / width times the piece's mean slope in t (and per_kap = ds / width times
// it, with no division); a segment that ends in the next piece is split at the node; longer ones
// subtract the two values, in Omega below tau = 1 and Phi above, where neither loses its relative
// precision.
__host__ __device__ __forceinline__ void lin_absorb(const SpecTable<double>& S, const double tau0, const double dtau,
                                                    const double kap, const double ds, double& frac, double& per_kap)
{
    const double tau1 = tau0 + dtau;
    if (tau1 < kLinTauLo) {
        const double s1 = tau0 + tau1, s2 = fma(tau0, s1, tau1 * tau1);
        const double D = fma(s2, S.zeta0 * (1.0 / 6.0), fma(-0.5 * S.xi0, s1, S.psi0));
        frac = dtau * D;
        per_kap = ds * D;
        return;
    }
    if (tau0 >= kLinTauLo && tau1 < kLinTauHi) {
        double t0;
        int w0;
        const int k0 = lin_locate(tau0, t0, w0);
        const int k1 = lin_index(tau1);
        const double sc0 = lin_pow2(-w0);                        // 1 / width of piece k0
        if (k1 == k0) {
            const double T = dtau * sc0;
            const double D = lin_slope(S.lin_a[k0], t0, T);
            frac = T * D;
            per_kap = (ds * D) * sc0;
            return;
        }
        if (k1 == k0 + 1) {
            const double T0 = 1.0 - t0;
            const double f0 = T0 * lin_slope(S.lin_a[k0], t0, T0);
            const double R = fma(-T0, lin_pow2(w0), dtau);       // optical depth past the node
            const double T1 = R * lin_pow2(-lin_wexp(k1));
            const double f1 = T1 * lin_slope(S.lin_a[k1], 0.0, T1);
            frac = f0 + f1;
            per_kap = frac / kap;
            return;
        }
    }
    const double r0 = lin_rep(S, tau0), r1 = lin_rep(S, tau1);
    frac = tau1 < 1.0 ? r1 - r0 : (tau0 < 1.0 ? (1.0 - r1) - r0 : r0 - r1);
    per_kap = frac / kap;
}

#ifdef __CUDACC__
// ---- the FP32 march: the same pieces rounded to float (lin_f), located from the bits of a float tau.

__device__ __forceinline__ float lin_pow2f(const int n)
{
    return __uint_as_float((unsigned)(127 + n) << 23);
}

__device__ __forceinline__ int lin_locate_f(const float tau, float& t, int& wexp)
{
    const unsigned b = __float_as_uint(tau);
    const int e = (int)(b >> 23) - 127;
    const int hb = e < 0 ? 5 : 7;
    t = __uint_as_float(0x3F800000u | ((b & ((1u << (23 - hb)) - 1u)) << hb)) - 1.0f;
    wexp = e - hb;
    return e < 0 ? (e - kLinExpLo) * 32 + (int)((b >> 18) & 31) : kLinOmega + (e << 7) + (int)((b >> 16) & 127);
}

__device__ __forceinline__ float lin_slope_f(const float4 p, const float t0, const float T)
{
    const float t1 = t0 + T;
    const float s1 = t0 + t1;
    const float s2 = fmaf(t0, s1, t1 * t1);
    return -fmaf(p.w, s2, fmaf(p.z, s1, p.y));
}

// Omega(tau) below tau = 1, Phi(tau) from 1 on (FP32).
__device__ __forceinline__ float lin_rep_f(const SpecTable<float>& S, const float tau)
{
    if (tau < (float)kLinTauLo) return tau * fmaf(-tau, (float)(0.5 * S.xi0), (float)S.psi0);
    if (tau >= (float)kLinTauHi) return (float)S.phi_end;
    float t;
    int we;
    const int k = lin_locate_f(tau, t, we);
    const float4 p = S.lin_f[k];
    const float c = t * fmaf(t, fmaf(t, p.w, p.z), p.y);
    return k < kLinOmega ? p.x - c : p.x + c;
}

__device__ __forceinline__ float lin_phi_f(const SpecTable<float>& S, const float tau)
{
    const float r = lin_rep_f(S, tau);
    return tau < 1.0f ? 1.0f - r : r;
}

__device__ __forceinline__ float lin_psi_f(const SpecTable<float>& S, const float tau)
{
    if (tau < (float)kLinTauLo) return fmaf(-tau, (float)S.xi0, (float)S.psi0);
    if (tau >= (float)kLinTauHi) return (float)S.psi_end;
    float t;
    int we;
    const int k = lin_locate_f(tau, t, we);
    const float4 p = S.lin_f[kLinIntervals + k];
    return fmaf(t, fmaf(t, fmaf(t, p.w, p.z), p.y), p.x);
}

__device__ __forceinline__ float lin_slope0_f(const float4 p, const float T)
{
    return -fmaf(T, fmaf(T, p.w, p.z), p.y);
}

// Phi(tau0) - Phi(tau0 + dtau) (FP32, kap > 0): as lin_absorb, by one code path for every segment
// between 2^-20 and 2^14 (the part in tau0's piece, the whole pieces between from node values, the
// part in tau1's piece), so the lanes of a warp do not diverge on where their segments end.
__device__ __forceinline__ float lin_absorb_f(const SpecTable<float>& S, const float tau0, const float dtau)
{
    const float tau1 = tau0 + dtau;
    if (tau0 >= (float)kLinTauLo && tau1 < (float)kLinTauHi) {
        float t0, t1;
        int w0, w1;
        const int k0 = lin_locate_f(tau0, t0, w0);
        const int k1 = lin_locate_f(tau1, t1, w1);
        const float4* P = S.lin_f;
        const float4 p0 = P[k0];
        const bool same = k1 == k0;
        const float T0 = same ? dtau * lin_pow2f(-w0) : 1.0f - t0;
        const float f0 = T0 * lin_slope_f(p0, t0, T0);
        const float4 p1 = P[k1];
        const float T1 = same ? 0.0f : (k1 == k0 + 1 ? fmaf(-T0, lin_pow2f(w0), dtau) * lin_pow2f(-w1) : t1);
        const float f1 = T1 * lin_slope0_f(p1, T1);
        const int ka = min(k0 + 1, kLinIntervals - 1);     // Phi_a - Phi_b, a = k0 + 1, b = k1
        const float va = P[ka].x, vb = p1.x;
        float mid = k1 < kLinOmega ? vb - va : (ka >= kLinOmega ? va - vb : (1.0f - vb) - va);
        mid = k1 >= k0 + 2 ? mid : 0.0f;
        return f0 + (mid + f1);
    }
    if (tau1 < (float)kLinTauLo) return dtau * fmaf(-0.5f * (float)S.xi0, tau0 + tau1, (float)S.psi0);
    const float r0 = lin_rep_f(S, tau0), r1 = lin_rep_f(S, tau1);
    return tau1 < 1.0f ? r1 - r0 : (tau0 < 1.0f ? (1.0f - r1) - r0 : r0 - r1);
}
#endif

}  // namespace nyx
