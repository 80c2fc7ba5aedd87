// Frequency-integrated photoionization (Eq. 1 integrated over the source
// spectrum; Sec. 2.5, after C2-Ray): a blackbody source at T_bb and a
// hydrogen cross-section sigma_nu = sigma_0 (nu_0 / nu)^3 above the
// threshold. With s = sigma_nu / sigma_0, a ray that has crossed threshold
// optical depth tau keeps the fraction Phi(tau) = <exp(-tau s)> of its
// photons (average over the photon-number spectrum), absorbs
// Phi(tau) - Phi(tau + dtau) over a segment of optical depth dtau, and in an
// optically thin cell deposits at the rate Psi(tau) = <s exp(-tau s)> per unit
// dtau. Phi and Psi are tabulated once per temperature on a logarithmic grid
// in tau with their derivatives in ln tau, and read back by cubic Hermite
// interpolation.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace nyx {

constexpr double kSpecTauLo = 1e-8;       // first grid point; below it the expansions in tau
constexpr int kSpecPerDecade = 64;
constexpr int kSpecDecades = 12;          // up to tau = 1e4
constexpr int kSpecPoints = kSpecPerDecade * kSpecDecades + 1;
constexpr double kSpecTauHi = 1e4;

// The FP64 march reads Phi and Psi from cubic pieces in tau itself. Below tau = 1, piece k covers
// [2^e (1 + i/32), 2^e (1 + (i+1)/32)) with e = kLinExpLo + k / 32 and i = k % 32; from tau = 1 on the
// pieces are four times finer, 128 per octave, where a cubic in tau follows Phi less closely. So k
// and the position t in [0, 1) come exactly from the bits of a double tau (no logarithm), and a
// piece's width is a power of two. Below 2^-20 Phi follows its series in tau; above 2^14 it keeps its
// value there.
constexpr int kLinExpLo = -20;
constexpr int kLinOmega = -kLinExpLo * 32;                  // the pieces below tau = 1
constexpr int kLinIntervals = kLinOmega + 14 * 128;         // up to 2^14
constexpr double kLinTauLo = 9.5367431640625e-07;           // 2^-20
constexpr double kLinTauHi = 16384.0;                       // 2^14

// One cubic piece: on interval k, Phi(t) - Phi_k = c1 t + c2 t^2 + c3 t^3 (lin_a) and Psi(t) = v + c1 t
// + c2 t^2 + c3 t^3 (lin_b). In lin_a, v is Phi_k from tau = 1 on and Omega_k = 1 - Phi_k below it,
// so that small absorbed fractions keep their relative precision.
struct __align__(32) LinPiece {
    double v, c1, c2, c3;
};

// Table of one temperature: v[4 j .. 4 j + 3] = Phi, dPhi/dln tau, Psi, dPsi/dln tau at
// tau_j = kSpecTauLo 10^(j / kSpecPerDecade); psi0 = Psi(0), xi0 = <s^2>. lin_a, lin_b and the
// values after them: the FP64 march's pieces (double tables only); zeta0 = <s^3>.
template <class R>
struct SpecTable {
    const R* v = nullptr;
    R psi0 = 0, xi0 = 0;
    const LinPiece* lin_a = nullptr;
    const LinPiece* lin_b = nullptr;
    double zeta0 = 0, phi_end = 0, psi_end = 0;
    // the same pieces as double-float pairs for the FP32 pipe, two float4 per piece:
    // {v.h, v.l, c1.h, c1.l}, {c2.h, c2.l, c3.h, c3.l}
    const float4* lin_af = nullptr;
    const float4* lin_bf = nullptr;
};

template <class R>
__host__ __device__ inline R spec_log(R x)
{
    return log(x);
}

// Phi(tau) and Psi(tau) from a table; tau >= 0.
template <class R>
__host__ __device__ inline void spec_eval(const SpecTable<R>& T, R tau, R& phi, R& psi)
{
    if (tau < (R)kSpecTauLo) {
        phi = (R)1 - tau * T.psi0;
        psi = T.psi0 - tau * T.xi0;
        return;
    }
    const R inv_h = (R)(kSpecPerDecade / 2.302585092994046);     // 1 / ln-spacing
    const R h = (R)(2.302585092994046 / kSpecPerDecade);
    R u = (spec_log<R>(tau) - (R)(-18.420680743952367)) * inv_h;  // ln(1e-8)
    int j = (int)u;
    if (j >= kSpecPoints - 1) {
        phi = T.v[4 * (kSpecPoints - 1)];
        psi = T.v[4 * (kSpecPoints - 1) + 2];
        return;
    }
    const R t = u - (R)j;
    const R t2 = t * t, t3 = t2 * t;
    const R h00 = (R)2 * t3 - (R)3 * t2 + (R)1, h10 = t3 - (R)2 * t2 + t;
    const R h01 = (R)3 * t2 - (R)2 * t3, h11 = t3 - t2;
    const R* a = T.v + 4 * j;
    phi = h00 * a[0] + h10 * h * a[1] + h01 * a[4] + h11 * h * a[5];
    psi = h00 * a[2] + h10 * h * a[3] + h01 * a[6] + h11 * h * a[7];
}

// Phi(tau) alone (the same operations as spec_eval's Phi): what a segment that absorbs
// P (Phi(tau) - Phi(tau + dtau)) needs at its far end.
template <class R>
__host__ __device__ inline R spec_phi(const SpecTable<R>& T, R tau)
{
    if (tau < (R)kSpecTauLo) return (R)1 - tau * T.psi0;
    const R inv_h = (R)(kSpecPerDecade / 2.302585092994046);
    const R h = (R)(2.302585092994046 / kSpecPerDecade);
    R u = (spec_log<R>(tau) - (R)(-18.420680743952367)) * inv_h;
    int j = (int)u;
    if (j >= kSpecPoints - 1) return T.v[4 * (kSpecPoints - 1)];
    const R t = u - (R)j;
    const R t2 = t * t, t3 = t2 * t;
    const R h00 = (R)2 * t3 - (R)3 * t2 + (R)1, h10 = t3 - (R)2 * t2 + t;
    const R h01 = (R)3 * t2 - (R)2 * t3, h11 = t3 - t2;
    const R* a = T.v + 4 * j;
    return h00 * a[0] + h10 * h * a[1] + h01 * a[4] + h11 * h * a[5];
}

#ifdef __CUDACC__
// Piece, exact position t and width 2^wexp of a double tau in [2^-20, 2^14): k from the exponent
// and the top five (below 1) or seven mantissa bits, t from the others (exactly representable).
__device__ __forceinline__ int lin_locate(const double tau, double& t, int& wexp)
{
    const long long b = __double_as_longlong(tau);
    const int e = (int)(b >> 52) - 1023;
    const int hb = e < 0 ? 5 : 7;
    t = __longlong_as_double(0x3FF0000000000000LL | ((b & ((1LL << (52 - hb)) - 1)) << hb)) - 1.0;
    wexp = e - hb;
    return e < 0 ? (e - kLinExpLo) * 32 + (int)((b >> 47) & 31) : kLinOmega + (e << 7) + (int)((b >> 45) & 127);
}

__device__ __forceinline__ int lin_index(const double tau)
{
    const long long b = __double_as_longlong(tau);
    const int e = (int)(b >> 52) - 1023;
    return e < 0 ? (e - kLinExpLo) * 32 + (int)((b >> 47) & 31) : kLinOmega + (e << 7) + (int)((b >> 45) & 127);
}

// The width exponent of piece k.
__device__ __forceinline__ int lin_wexp(const int k)
{
    return k < kLinOmega ? kLinExpLo + k / 32 - 5 : ((k - kLinOmega) >> 7) - 7;
}

// 2^n for a normal result
__device__ __forceinline__ double lin_pow2(const int n)
{
    return __longlong_as_double((long long)(1023 + n) << 52);
}

// Omega(tau) = 1 - Phi(tau) below 2^-20: tau <s> - tau^2 <s^2> / 2 + tau^3 <s^3> / 6 (the next
// term, below 2^-80 / 24, is dropped).
__device__ __forceinline__ double lin_series(const SpecTable<double>& S, const double tau)
{
    return tau * fma(-tau, fma(-tau, S.zeta0 * (1.0 / 6.0), 0.5 * S.xi0), S.psi0);
}

// Omega(tau) below tau = 1, Phi(tau) from 1 on.
__device__ __forceinline__ double lin_rep(const SpecTable<double>& S, const double tau)
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
__device__ __forceinline__ double lin_phi(const SpecTable<double>& S, const double tau)
{
    const double r = lin_rep(S, tau);
    return tau < 1.0 ? 1.0 - r : r;
}

// Psi(tau): the optically thin deposition rate per unit threshold optical depth.
__device__ __forceinline__ double lin_psi(const SpecTable<double>& S, const double tau)
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
__device__ __forceinline__ double lin_slope(const LinPiece& p, const double t0, const double T)
{
    const double t1 = t0 + T;
    const double s1 = t0 + t1;
    const double s2 = fma(t0, s1, t1 * t1);
    return -fma(p.c3, s2, fma(p.c2, s1, p.c1));
}

// A segment of optical depth dtau = kap ds after tau0 (kap > 0): frac = Phi(tau0) - Phi(tau0 + dtau),
// the fraction of the ray's photons it absorbs, and per_kap = frac / kap. Within one piece the
// difference is T = dtau / width times the piece's mean slope in t (and per_kap = ds / width times
// it, with no division); a segment that ends
// in the next piece is split at the node; longer ones subtract the two values, in Omega below tau = 1
// and Phi above, where neither loses its relative precision.
__device__ __forceinline__ void lin_absorb(const SpecTable<double>& S, const double tau0, const double dtau,
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
#endif

}  // namespace nyx
