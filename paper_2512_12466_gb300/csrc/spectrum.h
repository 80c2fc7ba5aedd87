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

#include <cmath>

namespace nyx {

constexpr double kSpecTauLo = 1e-8;       // first grid point; below it the expansions in tau
constexpr int kSpecPerDecade = 64;
constexpr int kSpecDecades = 12;          // up to tau = 1e4
constexpr int kSpecPoints = kSpecPerDecade * kSpecDecades + 1;
constexpr double kSpecTauHi = 1e4;

// Table of one temperature: v[4 j .. 4 j + 3] = Phi, dPhi/dln tau, Psi, dPsi/dln tau at
// tau_j = kSpecTauLo 10^(j / kSpecPerDecade); psi0 = Psi(0), xi0 = <s^2>.
template <class R>
struct SpecTable {
    const R* v = nullptr;
    R psi0 = 0, xi0 = 0;
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

}  // namespace nyx
