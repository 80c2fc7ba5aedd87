// Host runtime of libnyxrt and its C ABI (include/nyxrt.h).
//
// One rt_handle owns one grid's device state: n_H and x, the optical-depth
// field, the Gamma accumulator, the source catalog and one ray buffer per
// HEALPix level. rt_step runs the Sec. 2.8 source pipeline, then the ray
// tracing loop of Alg. 2 as one fused march+split launch per level (and per
// slice when a level's rays exceed the per-launch bound), then the heating
// and ledger reduction; with chemistry it iterates trace and the C2-Ray
// update (Sec. 2.4). The host reads back one counter per launch to size the
// next level; everything else stays on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "rt_handle.h"
#include "spectrum.h"

using namespace nyx;

namespace {

thread_local std::string g_create_error;

// Children marched per launch; a level with more is processed in slices, each
// followed by its whole sub-tree, which bounds every ray buffer to this many
// records.
constexpr int64_t kMaxChildrenPerLaunch = int64_t(1) << 27;
constexpr int kMarchBlock = 256;
constexpr int kMarchBlocksPerSm = 12;

struct DirTable {
    int level = -1;
    int4* dev = nullptr;
};
std::mutex g_dir_mu;
std::map<int, DirTable> g_dirs;          // per device; superseded tables stay allocated (handles may use them)




}  // namespace

int nyx::ensure_directions(int device, int level, const int4** out, std::string& err)
{
    std::lock_guard<std::mutex> lk(g_dir_mu);
    DirTable& t = g_dirs[device];
    if (t.level < level) {
        const int64_t count = healpix_level_offset(level + 1);
        std::vector<int4> host;
        try {
            host.resize((size_t)count);
        } catch (const std::bad_alloc&) {
            err = "host allocation of the direction table failed";
            return RT_ENOMEM;
        }
        healpix_direction_table(level, host.data());
        int4* d = nullptr;
        if (cudaMalloc(&d, sizeof(int4) * (size_t)count) != cudaSuccess) {
            cudaGetLastError();
            err = "device allocation of the direction table failed";
            return RT_ENOMEM;
        }
        if (cudaMemcpy(d, host.data(), sizeof(int4) * (size_t)count, cudaMemcpyHostToDevice) != cudaSuccess) {
            err = "copy of the direction table failed";
            cudaFree(d);
            return RT_ECUDA;
        }
        t.dev = d;
        t.level = level;
    }
    *out = t.dev;
    return RT_OK;
}


namespace {

// Geometry tables (FP32 march): one per (device, split radius, level, grid size covered). A
// table is never freed while the process runs (handles on other streams may be reading it);
// a larger grid, or one more than a quarter smaller, gets a new one. Their total per device stays within a budget, by default a
// quarter of the device's memory (NYXRT_GEOMETRY_BUDGET_MB overrides it): on a GB300 that holds
// every level of a 256^3 box in both precisions (46 GB) beside those of a 128^3 box. A level that
// does not fit is marched by walking its rays instead.
struct GeomTable {
    long long rq;
    long long rs;             // periodic travel-distance cutoff; 0: none
    int level;
    int n_cover;
    bool complete;            // no pixel cut short: serves every grid size
    unsigned long long total; // rows (of 32 entries)
    unsigned long long* row0; // row offset of each 32-pixel block (device)
    uint2* ent;               // FP32 entries, built on first use
    ulonglong2* ent64;        // FP64 entries, built on first use
    size_t failed_rows, failed32, failed64;  // budget when that build was tried and did not fit or
                                             // failed (0: never); tried again once the budget is larger
};
std::mutex g_geom_mu;
std::map<int, std::vector<GeomTable>> g_geom;   // never shrinks; entries are updated in place
std::map<int, size_t> g_geom_bytes;

// With NYXRT_GEOMETRY_TRACE set, every table build writes one line to stderr: what was built, its
// size, the budget and the outcome.
void geometry_trace(const char* what, int level, int n_cover, size_t bytes, size_t used, size_t budget, const char* outcome)
{
    static const bool on = std::getenv("NYXRT_GEOMETRY_TRACE") != nullptr;
    if (!on) return;
    std::fprintf(stderr, "nyxrt-geometry %s level %d n_cover %d bytes %zu used %zu budget %zu: %s\n", what, level, n_cover,
                 bytes, used, budget, outcome);
    std::fflush(stderr);
}

size_t geometry_budget(int device)
{
    if (const char* e = std::getenv("NYXRT_GEOMETRY_BUDGET_MB")) return (size_t)std::strtoull(e, nullptr, 10) << 20;
    size_t free_b = 0, total_b = 0;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != device) cudaSetDevice(device);
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        total_b = 0;
    }
    if (cur != device) cudaSetDevice(cur);
    return total_b / 4;
}

}  // namespace

bool nyx::geometry_level(int device, long long rq, int level, int n, long long rs, const int4* dirs_level,
                         cudaStream_t s, bool fp64, GeomLevel* out)
{
    std::lock_guard<std::mutex> lk(g_geom_mu);
    std::vector<GeomTable>& list = g_geom[device];
    // the smallest table that covers grids of n cells and was built for at most n + n/4: one built for
    // a much larger grid, complete or not, holds rows this grid never reads (level 10 at 1024^3 is
    // 38 GB in FP32, against 10 GB at 256^3), so a grid that small gets its own
    GeomTable* t = nullptr;
    for (GeomTable& c : list)
        if (c.rq == rq && c.rs == rs && c.level == level && (c.complete || c.n_cover >= n) &&
            c.n_cover <= n + n / 4 && (!t || c.n_cover < t->n_cover))
            t = &c;
    const long long npix = 12LL << (2 * level);
    const long long nb = (npix + 31) / 32;
    const size_t budget = geometry_budget(device);
    if (!t) {
        GeomTable c{rq, rs, level, n, false, 0ull, nullptr, nullptr, nullptr, 0, 0, 0};
        // every ray reaches R_l inside the virtual grid of 2n - 1 cells when R_l + 1 < n; with periodic
        // boundaries the table runs to the travel-distance cutoff, fixed by rs alone
        c.complete = rs != 0 || std::ldexp((double)rq, level - kRadBits) + 2.0 < (double)n;
        list.push_back(c);
        t = &list.back();
    }
    if (!t->row0 && (t->failed_rows == 0 || budget > t->failed_rows)) {
        // the rows of every 32-pixel block: counted once, shared by both precisions' entries
        unsigned* d_rows = nullptr;
        std::vector<unsigned> rows((size_t)nb);
        std::vector<unsigned long long> off((size_t)nb);
        const size_t row0_bytes = sizeof(unsigned long long) * (size_t)nb;
        unsigned long long total = 0;
        bool ok = g_geom_bytes[device] + row0_bytes <= budget &&
                  cudaMalloc(&d_rows, sizeof(unsigned) * (size_t)nb) == cudaSuccess;
        if (ok) {
            launch_geom_count(rq, level, dirs_level, npix, t->n_cover, rs, d_rows, s);
            ok = cudaMemcpyAsync(rows.data(), d_rows, sizeof(unsigned) * (size_t)nb, cudaMemcpyDeviceToHost, s) ==
                     cudaSuccess &&
                 cudaStreamSynchronize(s) == cudaSuccess;
        }
        for (long long b = 0; ok && b < nb; ++b) {
            off[(size_t)b] = total;
            total += rows[(size_t)b];
        }
        unsigned long long* row0 = nullptr;
        ok = ok && cudaMalloc(&row0, row0_bytes) == cudaSuccess &&
             cudaMemcpyAsync(row0, off.data(), row0_bytes, cudaMemcpyHostToDevice, s) == cudaSuccess &&
             cudaStreamSynchronize(s) == cudaSuccess;
        cudaGetLastError();
        cudaFree(d_rows);
        geometry_trace("rows", level, t->n_cover, row0_bytes, g_geom_bytes[device], budget, ok ? "built" : "failed");
        if (ok) {
            t->row0 = row0;
            t->total = total;
            g_geom_bytes[device] += row0_bytes;
        } else {
            cudaFree(row0);
            t->failed_rows = std::max<size_t>(budget, 1);
        }
    }
    if (!t->row0) return false;
    size_t& failed = fp64 ? t->failed64 : t->failed32;
    const bool have = fp64 ? t->ent64 != nullptr : t->ent != nullptr;
    if (!have && (failed == 0 || budget > failed)) {
        const size_t esz = fp64 ? sizeof(ulonglong2) : sizeof(uint2);
        const size_t bytes = (size_t)t->total * 32 * esz;
        void* ent = nullptr;
        unsigned* d_err = nullptr;
        unsigned herr = 0;
        const bool fits = g_geom_bytes[device] + bytes <= budget;
        bool ok = fits && cudaMalloc(&ent, std::max<size_t>(16, bytes)) == cudaSuccess &&
                  cudaMalloc(&d_err, sizeof(unsigned)) == cudaSuccess &&
                  cudaMemsetAsync(d_err, 0, sizeof(unsigned), s) == cudaSuccess;
        const bool allocated = ok;
        if (ok) {
            if (fp64)
                launch_geom_fill64(rq, level, dirs_level, npix, t->n_cover, rs, t->row0, t->total,
                                   static_cast<ulonglong2*>(ent), d_err, s);
            else
                launch_geom_fill(rq, level, dirs_level, npix, t->n_cover, rs, t->row0, static_cast<uint2*>(ent), d_err, s);
            ok = cudaMemcpyAsync(&herr, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                 cudaStreamSynchronize(s) == cudaSuccess && herr == 0;
        }
        cudaGetLastError();
        cudaFree(d_err);
        geometry_trace(fp64 ? "fp64 entries" : "fp32 entries", level, t->n_cover, bytes, g_geom_bytes[device], budget,
                       ok ? "built" : (!fits ? "over budget" : (!allocated ? "allocation failed" : "fill error")));
        if (ok) {
            if (fp64) t->ent64 = static_cast<ulonglong2*>(ent);
            else t->ent = static_cast<uint2*>(ent);
            g_geom_bytes[device] += bytes;
        } else {
            cudaFree(ent);
            failed = std::max<size_t>(budget, 1);
        }
    }
    if (fp64 ? t->ent64 == nullptr : t->ent == nullptr) return false;
    out->ent = t->ent;
    out->ent64 = t->ent64;
    out->row0 = t->row0;
    return true;
}

namespace {

// Blackbody spectrum tables (RT_SPECTRUM_BLACKBODY), one per (device, temperature), kept until the
// process exits. Built on the host: with u = nu_0 / nu in (0, 1], s = sigma_nu / sigma_0 = u^3 and
// the photon-number spectrum y^2 / (exp(theta y) - 1) dy becomes u^-4 / (exp(theta / u) - 1) du
// (theta = h nu_0 / (k T_bb)); the moments <s^p exp(-tau s)> are integrated by composite Simpson's
// rule over u (the integrand and its derivatives vanish at u = 0).
struct SpecEntry {
    double t_bb;
    std::vector<LinPiece> lin_a, lin_b;   // the cubic pieces in tau (host copy, for rt_spectrum_eval)
    double psi0, xi0, zeta0, phi_end, psi_end;
    const LinPiece* dev_lin;              // lin_a then lin_b
    const float4* dev_linf;               // the same as double-float pairs, two float4 per piece
    const float4* dev_linF;               // rounded to float, one float4 per piece
};
std::mutex g_spec_mu;
std::map<int, std::deque<SpecEntry>> g_spec;   // a deque: entries never move once added

constexpr double kHNu0Erg = 13.598 * 1.602176634e-12;   // hydrogen ionization threshold, erg
constexpr double kKbErgK = 1.380649e-16;

// The cubic pieces in tau (kLinIntervals of them, laid out as spectrum.h describes), by composite
// Simpson's rule over u with 4096 intervals. At node tau_j (and width w_j = tau_{j+1} - tau_j) it
// integrates Phi,
// Psi = <s e^{-tau s}>, Xi = <s^2 e^{-tau s}>, Omega = <1 - e^{-tau s}> and the increments
// dPhi_j = Phi_j - Phi_{j+1} = <e^{-tau_j s} (1 - e^{-w_j s})> and dPsi_j likewise, each written with
// expm1 so that no difference of nearly equal values is taken. The cubic of piece j is the Hermite
// interpolant of the node values and of their tau-derivatives (-Psi for Phi, -Xi for Psi), in
// t = (tau - tau_j) / w_j; its coefficients follow from the two values and two slopes.
void spectrum_lin_build(double theta, SpecEntry& e)
{
    const int N = 4096;
    const double du = 1.0 / N;
    std::vector<double> W(N + 1), sv(N + 1);
    double M0 = 0.0, M1 = 0.0, M2 = 0.0, M3 = 0.0;
    for (int i = 1; i <= N; ++i) {
        const double u = i * du;
        const double base = std::exp(-theta / u) / (-std::expm1(-theta / u)) / (u * u * u * u);
        const double wgt = (i == N) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        W[i] = wgt * base * du / 3.0;
        sv[i] = u * u * u;
        M0 += W[i];
        M1 += W[i] * sv[i];
        M2 += W[i] * sv[i] * sv[i];
        M3 += W[i] * sv[i] * sv[i] * sv[i];
    }
    const int J = kLinIntervals;
    std::vector<double> phi(J + 1), psi(J + 1), xi(J + 1), om(J + 1), dphi(J), dpsi(J), wid(J);
    auto node = [&](int j) {
        double tau, w;                                        // node tau_j and piece width
        if (j < kLinOmega) {
            tau = std::ldexp(1.0 + (double)(j % 32) / 32.0, kLinExpLo + j / 32);
            w = std::ldexp(1.0, kLinExpLo + j / 32 - 5);
        } else {
            const int q = j - kLinOmega;
            tau = std::ldexp(1.0 + (double)(q % 128) / 128.0, q / 128);
            w = std::ldexp(1.0, q / 128 - 7);
        }
        double a[6] = {0, 0, 0, 0, 0, 0};
        for (int i = 1; i <= N; ++i) {
            const double sx = sv[i];
            const double E = W[i] * std::exp(-tau * sx);
            a[0] += E;
            a[1] += E * sx;
            a[2] += E * sx * sx;
            a[3] += W[i] * -std::expm1(-tau * sx);
            if (j < J) {
                const double X = E * -std::expm1(-w * sx);
                a[4] += X;
                a[5] += X * sx;
            }
        }
        phi[j] = a[0] / M0;
        psi[j] = a[1] / M0;
        xi[j] = a[2] / M0;
        om[j] = a[3] / M0;
        if (j < J) {
            dphi[j] = a[4] / M0;
            dpsi[j] = a[5] / M0;
            wid[j] = w;
        }
    };
    const int nth = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    // node q, q + nth, ... on thread q; a thread that cannot be started leaves its nodes to this one
    std::vector<std::thread> pool;
    int started = 0;
    try {
        for (; started < nth; ++started)
            pool.emplace_back([&, started] {
                for (int j = started; j <= J; j += nth) node(j);
            });
    } catch (const std::system_error&) {
    }
    for (auto& t : pool) t.join();
    for (int q = started; q < nth; ++q)
        for (int j = q; j <= J; j += nth) node(j);
    e.lin_a.resize(J);
    e.lin_b.resize(J);
    for (int j = 0; j < J; ++j) {
        const double w = wid[j];
        const double m0 = -w * psi[j], m1 = -w * psi[j + 1];          // t-slopes of Phi at the ends
        e.lin_a[j] = {j < kLinOmega ? om[j] : phi[j], m0, -3.0 * dphi[j] - 2.0 * m0 - m1, 2.0 * dphi[j] + m0 + m1};
        const double n0 = -w * xi[j], n1 = -w * xi[j + 1];            // t-slopes of Psi
        e.lin_b[j] = {psi[j], n0, -3.0 * dpsi[j] - 2.0 * n0 - n1, 2.0 * dpsi[j] + n0 + n1};
    }
    e.psi0 = M1 / M0;
    e.xi0 = M2 / M0;
    e.zeta0 = M3 / M0;
    e.phi_end = phi[J];
    e.psi_end = psi[J];
}

const SpecEntry* spectrum_entry_locked(int device, double t_bb, std::string& why);

// The entry of (device, t_bb), built on first use; null (with `why`) if host or device memory ran
// out. No exception leaves it.
const SpecEntry* spectrum_entry(int device, double t_bb, std::string& why)
{
    std::lock_guard<std::mutex> lk(g_spec_mu);
    try {
        return spectrum_entry_locked(device, t_bb, why);
    } catch (const std::bad_alloc&) {
        why = "host allocation of the spectrum table failed";
        return nullptr;
    }
}

const SpecEntry* spectrum_entry_locked(int device, double t_bb, std::string& why)
{
    std::deque<SpecEntry>& list = g_spec[device];
    for (const SpecEntry& e : list)
        if (e.t_bb == t_bb) return &e;
    SpecEntry e{t_bb, {}, {}, 0.0, 0.0, 0.0, 0.0, 0.0, nullptr, nullptr, nullptr};
    spectrum_lin_build(kHNu0Erg / (kKbErgK * t_bb), e);
    if (device >= 0) {
        LinPiece* dl = nullptr;
        float4* dlf = nullptr;
        float4* dlF = nullptr;
        const size_t nl = e.lin_a.size();
        // double-float pairs: head = the value rounded to float, tail = the rest rounded to float
        std::vector<float4> lf(4 * nl), lF(2 * nl);
        auto pair = [](double x, float& h, float& l) {
            h = (float)x;
            l = (float)(x - (double)h);
        };
        for (size_t q = 0; q < 2 * nl; ++q) {
            const LinPiece& p = q < nl ? e.lin_a[q] : e.lin_b[q - nl];
            float4& u = lf[2 * q];
            float4& v = lf[2 * q + 1];
            pair(p.v, u.x, u.y);
            pair(p.c1, u.z, u.w);
            pair(p.c2, v.x, v.y);
            pair(p.c3, v.z, v.w);
            lF[q] = make_float4((float)p.v, (float)p.c1, (float)p.c2, (float)p.c3);
        }
        if (cudaMalloc(&dl, sizeof(LinPiece) * 2 * nl) != cudaSuccess ||
            cudaMalloc(&dlf, sizeof(float4) * lf.size()) != cudaSuccess ||
            cudaMalloc(&dlF, sizeof(float4) * lF.size()) != cudaSuccess ||
            cudaMemcpy(dl, e.lin_a.data(), sizeof(LinPiece) * nl, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(dl + nl, e.lin_b.data(), sizeof(LinPiece) * nl, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(dlf, lf.data(), sizeof(float4) * lf.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(dlF, lF.data(), sizeof(float4) * lF.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(dl);
            cudaFree(dlf);
            cudaFree(dlF);
            why = "device allocation of the spectrum table failed";
            return nullptr;
        }
        e.dev_lin = dl;
        e.dev_linf = dlf;
        e.dev_linF = dlF;
    }
    list.push_back(std::move(e));
    return &list.back();
}

}  // namespace

// Host evaluation of the pieces at t_bb (the host copy; entries are immutable once added): the same
// functions the FP64 march runs.
static bool spec_eval_host(double t_bb, double tau, double* phi, double* psi)
{
    std::string why;
    const SpecEntry* e = spectrum_entry(-1, t_bb, why);
    if (!e) return false;
    SpecTable<double> T;
    T.lin_a = e->lin_a.data();
    T.lin_b = e->lin_b.data();
    T.psi0 = e->psi0;
    T.xi0 = e->xi0;
    T.zeta0 = e->zeta0;
    T.phi_end = e->phi_end;
    T.psi_end = e->psi_end;
    *phi = nyx::lin_phi(T, tau);
    *psi = nyx::lin_psi(T, tau);
    return true;
}

// One segment's absorbed fraction, as the FP64 march computes it (kap = 1, so ds = dtau).
static bool spec_absorb_host(double t_bb, double tau, double dtau, double* frac)
{
    std::string why;
    const SpecEntry* e = spectrum_entry(-1, t_bb, why);
    if (!e) return false;
    SpecTable<double> T;
    T.lin_a = e->lin_a.data();
    T.lin_b = e->lin_b.data();
    T.psi0 = e->psi0;
    T.xi0 = e->xi0;
    T.zeta0 = e->zeta0;
    T.phi_end = e->phi_end;
    T.psi_end = e->psi_end;
    double per_kap;
    nyx::lin_absorb(T, tau, dtau, 1.0, dtau, *frac, per_kap);
    return true;
}

int nyx::spectrum_table(int device, double t_bb, SpecTable<double>* d, SpecTable<float>* f, std::string& why)
{
    const SpecEntry* e = spectrum_entry(device, t_bb, why);
    if (!e) return RT_ENOMEM;
    SpecTable<double> t;
    t.lin_a = e->dev_lin;
    t.lin_b = e->dev_lin ? e->dev_lin + e->lin_a.size() : nullptr;
    t.lin_af = e->dev_linf;
    t.lin_bf = e->dev_linf ? e->dev_linf + 2 * e->lin_a.size() : nullptr;
    t.lin_f = e->dev_linF;
    t.psi0 = e->psi0;
    t.xi0 = e->xi0;
    t.zeta0 = e->zeta0;
    t.phi_end = e->phi_end;
    t.psi_end = e->psi_end;
    *d = t;
    SpecTable<float> u;
    u.lin_a = t.lin_a;
    u.lin_b = t.lin_b;
    u.lin_af = t.lin_af;
    u.lin_bf = t.lin_bf;
    u.lin_f = t.lin_f;
    u.psi0 = t.psi0;
    u.xi0 = t.xi0;
    u.zeta0 = t.zeta0;
    u.phi_end = t.phi_end;
    u.psi_end = t.psi_end;
    *f = u;
    return RT_OK;
}

namespace nyx {

int configure(rt_handle* h, const rt_config* cfg, std::string& why);
bool valid_config(const rt_config* c, std::string& why);

// Host-side fault injection for tests: with NYXRT_FAULT_ALLOC=k (k >= 1) in the environment, the k-th
// handle allocation the library makes through dalloc in this process fails as if the device were out
// of memory (no device work is involved; every caller must return RT_ENOMEM and stay usable). With
// NYXRT_FAULT_ALLOC_TRACE set, every dalloc call writes its ordinal to stderr ("nyxrt-dalloc k"), so
// a test can find which ordinals a stage makes before it injects one.
long long fault_alloc_at()
{
    static const long long k = [] {
        const char* e = std::getenv("NYXRT_FAULT_ALLOC");
        return e ? std::atoll(e) : 0LL;
    }();
    return k;
}
bool fault_alloc_trace()
{
    static const bool t = std::getenv("NYXRT_FAULT_ALLOC_TRACE") != nullptr;
    return t;
}
std::atomic<long long> g_alloc_count{0};

// Handle memory is stream-ordered: allocating or freeing it never waits for
// work on other streams (a server creates and frees handles while batches run).
cudaError_t dalloc(rt_handle* h, void** p, size_t bytes)
{
    const long long k = fault_alloc_at();
    if (k > 0 || fault_alloc_trace()) {
        const long long ord = ++g_alloc_count;
        if (fault_alloc_trace()) {
            std::fprintf(stderr, "nyxrt-dalloc %lld\n", ord);
            std::fflush(stderr);
        }
        if (ord == k) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMallocAsync(p, bytes, h->stream);
}
void dfree(rt_handle* h, void* p)
{
    if (p) cudaFreeAsync(p, h->stream);
}

int fail(rt_handle* h, int code, const std::string& msg)
{
    h->err = msg;
    if (code == RT_ECUDA || code == RT_EDEVICE || code == RT_ETIMEOUT) h->sticky = true;
    return code;
}

int cuda_fail(rt_handle* h, cudaError_t e, const char* what)
{
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return fail(h, RT_ENOMEM, std::string(what) + ": out of device memory");
    return fail(h, RT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int grow_sources(rt_handle* h, int64_t need)
{
    if (need <= h->sw.cap) return RT_OK;
    int64_t cap = std::max<int64_t>(need, std::max<int64_t>(1024, 2 * h->sw.cap));
    SourceWork nw;
    nw.cap = cap;
    auto alloc = [&](void** p, size_t bytes) { return dalloc(h, p, bytes); };
    cudaError_t e = cudaSuccess;
    e = e ? e : alloc((void**)&nw.cells_raw, 12 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.ndot_raw, 8 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.keys, 8 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.keys_b, 8 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.keys_c, 8 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.order, 4 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.order_b, 4 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.flag, 4 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.head_pos, 4 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.cells_a, 12 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.ndot_a, 8 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.cells_b, 12 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.ndot_b, 8 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.label, 4 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.parent, 4 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.radius, 8 * (size_t)cap);
    e = e ? e : alloc((void**)&nw.count, 16);
    SrcEntry* emit = nullptr;
    e = e ? e : alloc((void**)&emit, sizeof(SrcEntry) * (size_t)cap);
    auto release = [h](SourceWork& w) {
        void* ps[] = {w.cells_raw, w.ndot_raw, w.keys, w.keys_b, w.keys_c, w.order, w.order_b, w.flag, w.head_pos,
                      w.cells_a, w.ndot_a, w.cells_b, w.ndot_b, w.label, w.parent, w.radius, w.count};
        for (void* q : ps) dfree(h, q);
    };
    if (e != cudaSuccess) {
        release(nw);
        dfree(h, emit);
        return cuda_fail(h, e, "source buffers");
    }
    if (h->nsrc > 0) {
        RT_CUDA(h, cudaMemcpyAsync(nw.cells_raw, h->sw.cells_raw, 12 * (size_t)h->nsrc, cudaMemcpyDeviceToDevice, h->stream),
                "source copy");
        RT_CUDA(h, cudaMemcpyAsync(nw.ndot_raw, h->sw.ndot_raw, 8 * (size_t)h->nsrc, cudaMemcpyDeviceToDevice, h->stream),
                "source copy");
    }
    release(h->sw);
    dfree(h, h->d_emit);
    h->sw = nw;
    h->d_emit = emit;
    return RT_OK;
}

template <class R>
int ensure_rays(rt_handle* h, int level, int64_t need)
{
    RayStore& s = h->rays[level];
    if (s.cap >= need) return RT_OK;
    int64_t cap = std::max<int64_t>(need, std::min<int64_t>(kMaxChildrenPerLaunch, std::max<int64_t>(4096, 2 * s.cap)));
    dfree(h, s.base);
    s.base = nullptr;
    s.cap = 0;
    void* p = nullptr;
    RT_CUDA(h, dalloc(h, &p, ray_bytes(cap, (int)sizeof(R))), "ray buffer");
    s.base = p;
    s.cap = cap;
    return RT_OK;
}

// March all rays of `level` whose parents are the first n records of the
// level's buffer (level 0: the emitted sources), then recurse into the
// next level, one slice of children at a time.
template <class R>
int run_level(rt_handle* h, int level, int64_t nparents)
{
    char range[32];
    std::snprintf(range, sizeof(range), "march level %d", level);
    NvtxRange nvtx(range);
    const int64_t total = level == 0 ? 12 * h->n_emit : 4 * nparents;
    if (total <= 0) return RT_OK;
    if (level > h->table_level || level > kMaxLevel)
        return fail(h, RT_EDEVICE, "ray level beyond the direction table");
    const bool can_split = level + 1 <= h->level_max;
    for (int64_t c0 = 0; c0 < total; c0 += kMaxChildrenPerLaunch) {
        const int64_t c1 = std::min(total, c0 + kMaxChildrenPerLaunch);
        if (can_split) {
            int rc = ensure_rays<R>(h, level + 1, c1 - c0);
            if (rc) return rc;
        }
        RT_CUDA(h, cudaMemsetAsync(h->d_count + level + 1, 0, sizeof(unsigned long long), h->stream), "counter");
        MarchArgs<R> a;
        a.level = level;
        a.n = h->cfg.n;
        a.c0 = c0;
        a.c1 = c1;
        a.dirs = h->dirs + healpix_level_offset(level);
        a.src = h->d_emit;
        a.in = ray_view<R>(h->rays[level]);
        a.out = can_split ? ray_view<R>(h->rays[level + 1]) : RayBuf<R>();
        a.out_count = h->d_count + level + 1;
        a.kap = static_cast<const R*>(h->d_kap);
        a.gamma = h->d_gamma;
        a.rq = h->rq;
        a.level_max = h->level_max;
        a.tau_max = (R)h->cfg.tau_max;
        a.overlap_mode = h->cfg.overlap_mode;
        a.hash = (h->cfg.flags & RT_FLAG_VISIT_HASH) ? 1 : 0;
        a.rs = h->rs;
        if constexpr (sizeof(R) == 8) a.spec = h->spec_d;
        else a.spec = h->spec_f;
        a.st = h->d_st;
        const int64_t warps = (c1 - c0 + 31) / 32;
        const int64_t want = (warps + kMarchBlock / 32 - 1) / (kMarchBlock / 32);
        // grid-stride blocks of equal share: 12 per SM is a whole number of waves for the march
        // kernels' 2, 3 and 4 resident blocks per SM, so no last wave runs an SM part-empty
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)h->sm_count * kMarchBlocksPerSm));
        // the level's geometry table for this precision (built once per device, outside the timed launch)
        GeomLevel gl;
        const bool table = !(h->cfg.flags & RT_FLAG_NO_GEOMETRY_TABLE) &&
                           geometry_level(h->device, h->rq, level, h->cfg.n, h->rs, a.dirs, h->stream, sizeof(R) == 8,
                                          &gl);
        RT_CUDA(h, cudaEventRecord(h->ev[4], h->stream), "event");
        if constexpr (sizeof(R) == 8) {
            if (table) launch_march_table_f64(a, gl, grid, kMarchBlock, h->stream);
            else launch_march_f64(a, grid, kMarchBlock, h->stream);
        } else {
            if (table) launch_march_table_f32(a, gl, grid, kMarchBlock, h->stream);
            else launch_march_f32(a, grid, kMarchBlock, h->stream);
        }
        RT_LAUNCHED(h, "march launch");
        RT_CUDA(h, cudaEventRecord(h->ev[5], h->stream), "event");
        h->launches++;
        h->march_launches++;
        if (table) h->table_levels |= int64_t(1) << level;
        RT_CUDA(h, cudaMemcpyAsync(h->h_count + level + 1, h->d_count + level + 1, sizeof(unsigned long long),
                                   cudaMemcpyDeviceToHost, h->stream), "counter read");
        RT_CUDA(h, cudaMemcpyAsync(h->h_i32, &h->d_st->err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream),
                "error read");
        RT_CUDA(h, cudaStreamSynchronize(h->stream), "march");
        if (h->h_i32[0]) return fail(h, RT_EDEVICE, "march kernel reported an internal error");
        float ms = 0.f;
        RT_CUDA(h, cudaEventElapsedTime(&ms, h->ev[4], h->ev[5]), "event");
        h->ms_march += ms;
        const int64_t next = (int64_t)h->h_count[level + 1];
        if (next > 0) {
            int rc = run_level<R>(h, level + 1, next);
            if (rc) return rc;
        }
    }
    return RT_OK;
}

int trace(rt_handle* h, const double* xuse)
{
    RT_CUDA(h, cudaMemsetAsync(h->d_gamma, 0, sizeof(double) * (size_t)h->ncell, h->stream), "gamma clear");
    // per-trace part of the statistics: per-level counters, hash and ledger
    RT_CUDA(h, cudaMemsetAsync(h->d_st, 0, offsetof(DevStats, deposited), h->stream), "stats clear");
    double n_th = h->cfg.n_th_cm3;
    if (n_th < 0) n_th = 0.01 * h->h_f64[1];
    if (h->cfg.precision == RT_FP32)
        launch_prepare_kappa_f32(h->d_nh, xuse, h->ncell, h->sdx, n_th, static_cast<float*>(h->d_kap), h->stream);
    else
        launch_prepare_kappa_f64(h->d_nh, xuse, h->ncell, h->sdx, n_th, static_cast<double*>(h->d_kap), h->stream);
    RT_LAUNCHED(h, "kappa launch");
    h->launches++;
    h->march_launches = 0;
    h->table_levels = 0;
    h->ms_march = 0.0;
    RT_CUDA(h, cudaEventRecord(h->ev[1], h->stream), "event");
    int rc = h->cfg.precision == RT_FP32 ? run_level<float>(h, 0, 0) : run_level<double>(h, 0, 0);
    if (rc) return rc;
    RT_CUDA(h, cudaEventRecord(h->ev[2], h->stream), "event");
    return RT_OK;
}

// Sec. 2.8 source stage of a step: validation of device-resident inputs,
// dedup + sort, the n_th default, Alg. 3 merging when on, and the emitted
// catalog (h->d_emit, h->n_emit). Leaves h->h_f64[1] = mean n_H (default n_th).
int prepare_sources(rt_handle* h, bool* merged_out, int64_t* n_dedup_out)
{
    NvtxRange nvtx("source stage (dedup, sort, Alg. 3)");
    cudaStream_t s = h->stream;
    *merged_out = false;
    h->catalog_valid = false;            // the buffers below are rewritten; valid again once emitted
    // ---- validation of device-resident inputs
    h->launches += launch_validate_fields(h->d_nh, h->d_x, h->ncell, h->d_st, s);
    h->launches += launch_validate_sources(h->sw.cells_raw, h->sw.ndot_raw, h->nsrc, h->cfg.n, h->d_st, s);
    RT_LAUNCHED(h, "validation launch");

    // ---- sources: dedup + sort (Sec. 2.8)
    h->launches += launch_dedup_sort(h->sw, h->nsrc, h->cfg.n, s);
    RT_LAUNCHED(h, "source launch");
    bool want_mean_nh = h->cfg.n_th_cm3 < 0;
    if (want_mean_nh) {
        RT_CUDA(h, cudaMemsetAsync(h->d_scalar, 0, sizeof(double), s), "scalar clear");
        h->launches += launch_mean_nh(h->d_nh, h->ncell, h->d_scalar, s);
    }
    if (h->cfg.merge_mode == RT_MERGE_AUTO) h->launches += launch_sum_x(h->d_x, h->ncell, h->d_st, s);
    RT_LAUNCHED(h, "reduction launch");
    RT_CUDA(h, cudaMemcpyAsync(h->h_st, h->d_st, sizeof(DevStats), cudaMemcpyDeviceToHost, s), "stats read");
    if (h->nsrc > 0)
        RT_CUDA(h, cudaMemcpyAsync(h->h_i32, h->sw.count, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "count read");
    if (want_mean_nh)
        RT_CUDA(h, cudaMemcpyAsync(h->h_f64, h->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, s), "mean read");
    RT_CUDA(h, cudaStreamSynchronize(s), "source stage");
    if (h->h_st->bad_input) return fail(h, RT_EINVAL, "invalid field or source values (n_H < 0, x outside [0,1], non-finite, bad source)");
    h->h_f64[1] = want_mean_nh ? h->h_f64[0] / (double)h->ncell : 0.0;
    int64_t m = h->nsrc > 0 ? h->h_i32[0] : 0;
    *n_dedup_out = m;
    const double xbar = h->h_st->xsum / (double)h->ncell;

    // ---- Alg. 3 source merging
    if (m > 0 && (h->cfg.merge_mode == RT_MERGE_FORCED ||
                  (h->cfg.merge_mode == RT_MERGE_AUTO && xbar > h->cfg.automerge_xbar))) {
        const int Ls = h->cfg.merge_samp_level;
        h->launches += launch_merge(h->sw, m, h->cfg.n, h->cfg.periodic, h->d_x, h->dirs + healpix_level_offset(Ls),
                                    (int)(12 * (int64_t(1) << (2 * Ls))), h->cfg.merge_x_th, h->cfg.merge_f_req,
                                    h->cfg.merge_n_min, h->cfg.merge_dr_cells, h->cfg.merge_rmax_cells,
                                    h->cfg.merge_f_ov, h->cfg.merge_eps, h->d_st, s);
        RT_LAUNCHED(h, "merge launch");
        RT_CUDA(h, cudaMemcpyAsync(h->h_i32, h->sw.count, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "count read");
        RT_CUDA(h, cudaMemcpyAsync(h->h_i32 + 1, &h->d_st->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "err read");
        RT_CUDA(h, cudaStreamSynchronize(s), "merge");
        if (h->h_i32[1]) return fail(h, RT_EDEVICE, "source merge reported an internal error");
        m = h->h_i32[0];
        *merged_out = true;
    }
    h->launches += launch_build_emit(h->sw, m, h->s_over_dx2, h->d_emit, h->d_st, s);
    RT_LAUNCHED(h, "emit launch");
    h->n_emit = m;
    h->catalog_valid = true;

    return RT_OK;
}

// Re-target an idle handle to a new configuration with the same grid size,
// precision and chemistry setting (its allocations fit as they are).
int handle_reconfigure(rt_handle* h, const rt_config* cfg)
{
    std::string why;
    if (h->sticky) return RT_ESTATE;
    if (cfg->n != h->cfg.n || cfg->precision != h->cfg.precision || (cfg->chem_iterate != 0) != (h->cfg.chem_iterate != 0))
        return fail(h, RT_EINVAL, "reconfiguration needs the same n, precision and chemistry setting");
    if (!valid_config(cfg, why)) return fail(h, RT_EINVAL, why);
    const int rc = configure(h, cfg, why);
    if (rc) return fail(h, rc, why);
    h->nsrc = 0;
    h->fields_set = false;
    h->src_ready = false;
    h->catalog_valid = false;
    h->err.clear();
    return RT_OK;
}

// The source stage of many handles at once, in two halves. sources_enqueue_many enqueues, for handles
// without merging, every kernel (validation, dedup + sort, mean n_H, emission with the count read on
// the device) and the statistics readback on all handles' streams; handles with merging take the
// synchronous path there. sources_wait_many then waits once per stream and records the results.
// rcs[i] receives handle i's outcome (one bad request fails alone); each returns the number of
// handles that failed so far.
int sources_enqueue_many(rt_handle* const* hs, int count, int* rcs)
{
    auto enqueue = [](rt_handle* h) -> int {
        cudaStream_t s = h->stream;
        h->launches = 0;
        h->catalog_valid = false;
        RT_CUDA(h, cudaMemsetAsync(h->d_st, 0, sizeof(DevStats), s), "stats clear");
        h->launches += launch_validate_fields(h->d_nh, h->d_x, h->ncell, h->d_st, s);
        h->launches += launch_validate_sources(h->sw.cells_raw, h->sw.ndot_raw, h->nsrc, h->cfg.n, h->d_st, s);
        h->launches += launch_dedup_sort(h->sw, h->nsrc, h->cfg.n, s);
        if (h->cfg.n_th_cm3 < 0) {
            RT_CUDA(h, cudaMemsetAsync(h->d_scalar, 0, sizeof(double), s), "scalar clear");
            h->launches += launch_mean_nh(h->d_nh, h->ncell, h->d_scalar, s);
        }
        if (h->nsrc > 0) h->launches += launch_build_emit_dev(h->sw, h->nsrc, h->s_over_dx2, h->d_emit, h->d_st, s);
        // statistics, count and mean written into the pinned block by a kernel (a server's result
        // copies of other requests may occupy the copy engines)
        ReadbackList rb;
        rb.add(h->d_st, pinned_dev(h, h->h_st), sizeof(DevStats));
        if (h->nsrc > 0) rb.add(h->sw.count, pinned_dev(h, h->h_i32), sizeof(int32_t));
        if (h->cfg.n_th_cm3 < 0) rb.add(h->d_scalar, pinned_dev(h, h->h_f64), sizeof(double));
        h->launches += launch_readback(rb, s);
        RT_LAUNCHED(h, "source stage launch");
        return RT_OK;
    };
    int failed = 0;
    for (int i = 0; i < count; ++i) {
        rt_handle* h = hs[i];
        rcs[i] = RT_OK;
        if (h->src_ready) continue;
        rcs[i] = h->cfg.merge_mode != RT_MERGE_OFF ? handle_prepare_sources(h) : enqueue(h);
        failed += rcs[i] != RT_OK;
    }
    return failed;
}

int sources_wait_many(rt_handle* const* hs, int count, int* rcs)
{
    int failed = 0;
    for (int i = 0; i < count; ++i) {
        rt_handle* h = hs[i];
        if (rcs[i] == RT_OK && !h->src_ready) {
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) rcs[i] = cuda_fail(h, cudaGetLastError(), "source stage");
            else if (h->h_st->bad_input)
                rcs[i] = fail(h, RT_EINVAL, "invalid field or source values (n_H < 0, x outside [0,1], non-finite, bad source)");
        }
        if (rcs[i] != RT_OK) { ++failed; continue; }
        if (h->src_ready) continue;
        const int64_t m = h->nsrc > 0 ? h->h_i32[0] : 0;
        h->n_emit = m;
        h->catalog_valid = true;
        h->src_ready = true;
        h->src_merged = false;
        h->src_dedup = m;
        h->src_nth = h->cfg.n_th_cm3 >= 0 ? h->cfg.n_th_cm3 : 0.01 * (h->h_f64[0] / (double)h->ncell);
        h->src_emitted = h->h_st->emitted;
    }
    return failed;
}

// Run the source stage ahead of a batch (a server's loader does this while the
// GPU traces the previous batch); batch_bind then uses the recorded results.
int handle_prepare_sources(rt_handle* h)
{
    h->launches = 0;
    RT_CUDA(h, cudaMemsetAsync(h->d_st, 0, sizeof(DevStats), h->stream), "stats clear");
    bool merged = false;
    int64_t nd = 0;
    const int rc = prepare_sources(h, &merged, &nd);
    if (rc) return rc;
    RT_CUDA(h, cudaMemcpyAsync(h->h_st, h->d_st, sizeof(DevStats), cudaMemcpyDeviceToHost, h->stream), "stats");
    RT_CUDA(h, cudaStreamSynchronize(h->stream), "source stage");
    h->src_ready = true;
    h->src_merged = merged;
    h->src_dedup = nd;
    h->src_nth = h->cfg.n_th_cm3 >= 0 ? h->cfg.n_th_cm3 : 0.01 * h->h_f64[1];
    h->src_emitted = h->h_st->emitted;
    return RT_OK;
}

// Derived quantities of a configuration (cell size, split radius, level cap,
// direction table); allocation-independent, so a pooled handle of the same n
// and precision can be re-targeted to a new request.
int configure(rt_handle* h, const rt_config* cfg, std::string& why)
{
    h->cfg = *cfg;
    const int64_t n = cfg->n;
    h->ncell = n * n * n;
    // the same IEEE operations as the problem statement: dx = L / n
    h->dx = cfg->box_cm / (double)n;
    h->vol = h->dx * h->dx * h->dx;
    h->sdx = cfg->sigma_cm2 * h->dx;
    h->s_over_dx2 = cfg->sigma_cm2 / (h->dx * h->dx);
    // R_0 = sqrt(3 / (pi N_min)) in units of 2^-24 cells (Eq. 4 with Omega_c = dx^2 / R^2)
    h->rq = (int64_t)std::floor(std::sqrt(3.0 / (3.141592653589793 * cfg->n_min_ray)) * (double)(1 << kRadBits) + 0.5);
    // periodic boundaries (Sec. 2.5.1): rays stop at travel distance sqrt(3) L_box = sqrt(3) n cells,
    // in the same fixed point as the split radius
    h->rs = cfg->periodic ? (int64_t)std::floor(std::sqrt(3.0) * (double)n * (double)(1 << kRadBits) + 0.5) : 0;
    // smallest level whose split sphere encloses the grid from any cell centre
    int reach = 0;
    while (std::ldexp((double)h->rq, reach - kRadBits) < std::sqrt(3.0) * (double)n) ++reach;
    h->level_max = cfg->level_max >= 0 ? cfg->level_max : std::min(reach + 1, kMaxLevel);
    h->table_level = std::min(h->level_max, reach);
    const int need_level = std::max(h->table_level, cfg->merge_samp_level);
    h->spec_d = SpecTable<double>();
    h->spec_f = SpecTable<float>();
    if (cfg->spectrum == RT_SPECTRUM_BLACKBODY) {
        const int rc = spectrum_table(h->device, cfg->t_bb_K, &h->spec_d, &h->spec_f, why);
        if (rc) return rc;
    }
    return ensure_directions(h->device, need_level, &h->dirs, why);
}

bool valid_config(const rt_config* c, std::string& why)
{
    if (c->n < 1 || c->n > 1024) { why = "n must be in 1..1024"; return false; }
    if (!(c->box_cm > 0) || !std::isfinite(c->box_cm)) { why = "box_cm must be positive"; return false; }
    if (c->precision != RT_FP64 && c->precision != RT_FP32) { why = "precision must be RT_FP64 or RT_FP32"; return false; }
    if (!(c->sigma_cm2 > 0)) { why = "sigma_cm2 must be positive"; return false; }
    if (!(c->n_min_ray >= 1.0)) { why = "n_min_ray must be >= 1"; return false; }
    if (!(c->tau_max > 0)) { why = "tau_max must be positive"; return false; }
    if (c->overlap_mode < 0 || c->overlap_mode > 5) { why = "overlap_mode must be 0..5"; return false; }
    if (c->merge_mode < 0 || c->merge_mode > 2) { why = "merge_mode must be 0..2"; return false; }
    if (c->merge_samp_level < 0 || c->merge_samp_level > 4) { why = "merge_samp_level must be 0..4"; return false; }
    if (!(c->merge_dr_cells > 0)) { why = "merge_dr_cells must be positive"; return false; }
    if (c->level_max > kMaxLevel) { why = "level_max must be <= 13"; return false; }
    if (c->periodic != 0 && c->periodic != 1) { why = "periodic must be 0 or 1"; return false; }
    if (c->spectrum != RT_SPECTRUM_GRAY && c->spectrum != RT_SPECTRUM_BLACKBODY) {
        why = "spectrum must be RT_SPECTRUM_GRAY or RT_SPECTRUM_BLACKBODY";
        return false;
    }
    if (c->spectrum == RT_SPECTRUM_BLACKBODY && (!(c->t_bb_K > 0) || !std::isfinite(c->t_bb_K) || !(c->tau_max <= kSpecTauHi))) {
        why = "RT_SPECTRUM_BLACKBODY needs t_bb_K > 0 and tau_max <= 1e4";
        return false;
    }
    return true;
}

}  // namespace

extern "C" {

void rt_config_default(rt_config* c, int32_t n, double box_cm)
{
    std::memset(c, 0, sizeof(*c));
    c->n = n;
    c->box_cm = box_cm;
    c->precision = RT_FP64;
    c->sigma_cm2 = 6.3e-18;
    c->n_min_ray = 4.0;
    c->level_max = -1;
    c->overlap_mode = RT_OVERLAP_CONSERVATIVE;
    c->tau_max = 30.0;
    c->n_th_cm3 = -1.0;
    c->e_heat_erg = 1.602176634e-12;
    c->merge_mode = RT_MERGE_OFF;
    c->merge_samp_level = 3;
    c->automerge_xbar = 0.018;
    c->merge_x_th = 0.9;
    c->merge_f_req = 0.9;
    c->merge_dr_cells = 2.0;
    c->merge_rmax_cells = 16.0;
    c->merge_f_ov = 1.0;
    c->merge_eps = 1e-6;
    c->merge_n_min = 8;
    c->chem_iterate = 0;
    c->alpha_B = 2.59e-13;
    c->C_H = 0.0;
    c->clumping = 1.0;
    c->chem_tol = 1e-6;
    c->chem_max_iter = 100;
    c->flags = 0;
    c->periodic = 0;
    c->spectrum = RT_SPECTRUM_GRAY;
    c->t_bb_K = 1e5;
}

const char* rt_version(void) { return "nyxrt 0.1 (sm_103a)"; }

const char* rt_last_error(const rt_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int rt_destroy(rt_handle* h)
{
    if (!h) return RT_OK;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    {
        void* ps[] = {h->d_nh, h->d_x, h->d_xavg, h->d_xend, h->d_gamma, h->d_heat, h->d_kap, h->d_scalar,
                      h->d_emit, h->d_count, h->d_st};
        for (void* q : ps) dfree(h, q);
        SourceWork& w = h->sw;
        void* ws[] = {w.cells_raw, w.ndot_raw, w.keys, w.keys_b, w.keys_c, w.order, w.order_b, w.flag, w.head_pos,
                      w.cells_a, w.ndot_a, w.cells_b, w.ndot_b, w.label, w.parent, w.radius, w.count};
        for (void* q : ws) dfree(h, q);
        for (auto& r : h->rays) dfree(h, r.base);
    }
    if (h->h_pin) cudaFreeHost(h->h_pin);
    for (auto& e : h->ev) if (e) cudaEventDestroy(e);
    cudaGetLastError();
    delete h;
    return RT_OK;
}

int rt_create(const rt_config* cfg, void* cuda_stream, rt_handle** out)
{
    if (!out) return RT_EINVAL;
    *out = nullptr;
    g_create_error.clear();
    if (!cfg) { g_create_error = "cfg is NULL"; return RT_EINVAL; }
    std::string why;
    if (!valid_config(cfg, why)) { g_create_error = why; return RT_EINVAL; }
    rt_handle* h = new (std::nothrow) rt_handle();
    if (!h) { g_create_error = "host allocation failed"; return RT_ENOMEM; }
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    int rc = configure(h, cfg, why);
    if (rc) { g_create_error = why; rt_destroy(h); return rc; }
    cudaError_t e = cudaSuccess;
    const size_t fb = sizeof(double) * (size_t)h->ncell;
    e = e ? e : dalloc(h, (void**)&h->d_nh, fb);
    e = e ? e : dalloc(h, (void**)&h->d_x, fb);
    e = e ? e : dalloc(h, (void**)&h->d_gamma, fb);
    e = e ? e : dalloc(h, (void**)&h->d_heat, fb);
    e = e ? e : dalloc(h, &h->d_kap, cfg->precision == RT_FP32 ? fb / 2 : fb);
    if (cfg->chem_iterate) {
        e = e ? e : dalloc(h, (void**)&h->d_xavg, fb);
        e = e ? e : dalloc(h, (void**)&h->d_xend, fb);
    }
    e = e ? e : dalloc(h, (void**)&h->d_scalar, 64);
    e = e ? e : dalloc(h, (void**)&h->d_count, sizeof(unsigned long long) * (RT_MAX_LEVELS + 1));
    e = e ? e : dalloc(h, (void**)&h->d_st, sizeof(DevStats));
    {   // one pinned block for every host-side readback
        const size_t a = (sizeof(DevStats) + 63) & ~size_t(63);
        const size_t b = (sizeof(unsigned long long) * (RT_MAX_LEVELS + 1) + 63) & ~size_t(63);
        e = e ? e : cudaMallocHost(&h->h_pin, a + b + 128);
        e = e ? e : cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->d_pin), h->h_pin, 0);
        if (e == cudaSuccess) {
            char* q = static_cast<char*>(h->h_pin);
            h->h_st = reinterpret_cast<DevStats*>(q);
            h->h_count = reinterpret_cast<unsigned long long*>(q + a);
            h->h_i32 = reinterpret_cast<int32_t*>(q + a + b);
            h->h_f64 = reinterpret_cast<double*>(q + a + b + 64);
        }
    }
    for (auto& ev : h->ev) e = e ? e : cudaEventCreate(&ev);
    e = e ? e : cudaStreamSynchronize(h->stream);   // the allocations are usable from any stream after this
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_create_error = std::string("allocation failed: ") + cudaGetErrorString(e);
        rt_destroy(h);
        return e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA;
    }
    *out = h;
    return RT_OK;
}

int rt_set_fields(rt_handle* h, const double* n_H, const double* x_ion, int where)
{
    if (!h || !n_H || !x_ion || (where != RT_HOST && where != RT_DEVICE)) return h ? fail(h, RT_EINVAL, "bad arguments") : RT_EINVAL;
    if (h->sticky) return RT_ESTATE;
    DeviceGuard g(h->device);
    const size_t fb = sizeof(double) * (size_t)h->ncell;
    const cudaMemcpyKind k = where == RT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    RT_CUDA(h, cudaMemcpyAsync(h->d_nh, n_H, fb, k, h->stream), "field copy");
    RT_CUDA(h, cudaMemcpyAsync(h->d_x, x_ion, fb, k, h->stream), "field copy");
    if (where == RT_HOST) RT_CUDA(h, cudaStreamSynchronize(h->stream), "field copy");
    h->fields_set = true;
    return RT_OK;
}

int rt_add_sources(rt_handle* h, const int32_t* cell_ijk, const double* ndot, int64_t n, int where)
{
    if (!h) return RT_EINVAL;
    if (n < 0 || (n > 0 && (!cell_ijk || !ndot)) || (where != RT_HOST && where != RT_DEVICE))
        return fail(h, RT_EINVAL, "bad arguments");
    if (h->sticky) return RT_ESTATE;
    if (n == 0) return RT_OK;
    if (h->nsrc + n > (int64_t(1) << 30)) return fail(h, RT_EINVAL, "too many sources");
    if (where == RT_HOST) {
        for (int64_t i = 0; i < n; ++i) {
            for (int a = 0; a < 3; ++a)
                if (cell_ijk[3 * i + a] < 0 || cell_ijk[3 * i + a] >= h->cfg.n) return fail(h, RT_EINVAL, "source cell outside the grid");
            if (!(ndot[i] > 0) || !std::isfinite(ndot[i])) return fail(h, RT_EINVAL, "source rate must be positive and finite");
        }
    }
    DeviceGuard g(h->device);
    h->catalog_valid = false;
    int rc = grow_sources(h, h->nsrc + n);
    if (rc) return rc;
    const cudaMemcpyKind k = where == RT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    RT_CUDA(h, cudaMemcpyAsync(h->sw.cells_raw + 3 * h->nsrc, cell_ijk, 12 * (size_t)n, k, h->stream), "source copy");
    RT_CUDA(h, cudaMemcpyAsync(h->sw.ndot_raw + h->nsrc, ndot, 8 * (size_t)n, k, h->stream), "source copy");
    if (where == RT_HOST) RT_CUDA(h, cudaStreamSynchronize(h->stream), "source copy");
    h->nsrc += n;
    return RT_OK;
}

int rt_spectrum_eval(double t_bb_K, double tau, double* phi, double* psi)
{
    if (!phi || !psi || !(t_bb_K > 0) || !std::isfinite(t_bb_K) || !(tau >= 0) || !(tau <= kSpecTauHi)) return RT_EINVAL;
    return spec_eval_host(t_bb_K, tau, phi, psi) ? RT_OK : RT_ENOMEM;
}

int rt_spectrum_absorb(double t_bb_K, double tau, double dtau, double* frac)
{
    if (!frac || !(t_bb_K > 0) || !std::isfinite(t_bb_K) || !(tau >= 0) || !(tau <= kSpecTauHi) || !(dtau > 0) ||
        !(dtau <= kSpecTauHi))
        return RT_EINVAL;
    return spec_absorb_host(t_bb_K, tau, dtau, frac) ? RT_OK : RT_ENOMEM;
}

int64_t rt_geometry_table_bytes(int32_t device)
{
    std::lock_guard<std::mutex> lk(g_geom_mu);
    auto it = g_geom_bytes.find(device);
    return it == g_geom_bytes.end() ? 0 : (int64_t)it->second;
}

int rt_reconfigure(rt_handle* h, const rt_config* cfg)
{
    if (!h || !cfg) return h ? fail(h, RT_EINVAL, "cfg is NULL") : RT_EINVAL;
    DeviceGuard g(h->device);
    return handle_reconfigure(h, cfg);
}

int rt_clear_sources(rt_handle* h)
{
    if (!h) return RT_EINVAL;
    if (h->sticky) return RT_ESTATE;
    h->nsrc = 0;
    h->catalog_valid = false;
    return RT_OK;
}

int rt_get_sources(rt_handle* h, int32_t* cells_out, double* ndot_out, int64_t capacity, int64_t* count, int where)
{
    if (!h) return RT_EINVAL;
    if (!count || capacity < 0 || (capacity > 0 && (!cells_out || !ndot_out)) || (where != RT_HOST && where != RT_DEVICE))
        return fail(h, RT_EINVAL, "bad arguments");
    if (h->sticky) return RT_ESTATE;
    if (!h->catalog_valid) return fail(h, RT_ESTATE, "no step has traced the current sources");
    *count = h->n_emit;
    const int64_t m = std::min(capacity, h->n_emit);
    if (m > 0) {
        DeviceGuard g(h->device);
        const cudaMemcpyKind k = where == RT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        RT_CUDA(h, cudaMemcpyAsync(cells_out, h->sw.cells_a, 12 * (size_t)m, k, h->stream), "catalog copy");
        RT_CUDA(h, cudaMemcpyAsync(ndot_out, h->sw.ndot_a, 8 * (size_t)m, k, h->stream), "catalog copy");
        RT_CUDA(h, cudaStreamSynchronize(h->stream), "catalog copy");
    }
    return RT_OK;
}

// Checkpoint file: the 8-byte magic, then uint32 version, uint32 sizeof(rt_config), the rt_config,
// int64 cell count, n_H and x (float64 each), int64 source count, the sources' cells (int32 x 3)
// and rates (float64), all little-endian as the host writes them.
static const char kCkptMagic[8] = {'N', 'Y', 'X', 'R', 'T', 'C', 'K', '1'};
static const uint32_t kCkptVersion = 1;

int rt_save(rt_handle* h, const char* path)
{
    if (!h) return RT_EINVAL;
    if (!path) return fail(h, RT_EINVAL, "path is NULL");
    if (h->sticky) return RT_ESTATE;
    if (!h->fields_set) return fail(h, RT_ESTATE, "rt_set_fields has not been called");
    DeviceGuard g(h->device);
    const int64_t nc = h->ncell, ns = h->nsrc;
    std::vector<double> nh, x, nd;
    std::vector<int32_t> cells;
    try {
        nh.resize((size_t)nc);
        x.resize((size_t)nc);
        nd.resize((size_t)ns);
        cells.resize((size_t)(3 * ns));
    } catch (const std::bad_alloc&) {
        return fail(h, RT_ENOMEM, "out of host memory for the checkpoint buffers");
    }
    RT_CUDA(h, cudaMemcpyAsync(nh.data(), h->d_nh, 8 * (size_t)nc, cudaMemcpyDeviceToHost, h->stream), "checkpoint copy");
    RT_CUDA(h, cudaMemcpyAsync(x.data(), h->d_x, 8 * (size_t)nc, cudaMemcpyDeviceToHost, h->stream), "checkpoint copy");
    if (ns > 0) {
        RT_CUDA(h, cudaMemcpyAsync(cells.data(), h->sw.cells_raw, 12 * (size_t)ns, cudaMemcpyDeviceToHost, h->stream),
                "checkpoint copy");
        RT_CUDA(h, cudaMemcpyAsync(nd.data(), h->sw.ndot_raw, 8 * (size_t)ns, cudaMemcpyDeviceToHost, h->stream),
                "checkpoint copy");
    }
    RT_CUDA(h, cudaStreamSynchronize(h->stream), "checkpoint copy");
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(h, RT_EINVAL, std::string("cannot open ") + path + " for writing");
    const uint32_t hdr[2] = {kCkptVersion, (uint32_t)sizeof(rt_config)};
    bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8 && std::fwrite(hdr, 4, 2, f) == 2 &&
              std::fwrite(&h->cfg, sizeof(rt_config), 1, f) == 1 && std::fwrite(&nc, 8, 1, f) == 1 &&
              std::fwrite(nh.data(), 8, (size_t)nc, f) == (size_t)nc && std::fwrite(x.data(), 8, (size_t)nc, f) == (size_t)nc &&
              std::fwrite(&ns, 8, 1, f) == 1;
    if (ok && ns > 0)
        ok = std::fwrite(cells.data(), 4, (size_t)(3 * ns), f) == (size_t)(3 * ns) &&
             std::fwrite(nd.data(), 8, (size_t)ns, f) == (size_t)ns;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(h, RT_EINVAL, std::string("writing ") + path + " failed");
    return RT_OK;
}

int rt_load(const char* path, void* cuda_stream, rt_handle** out)
{
    if (!out) return RT_EINVAL;
    *out = nullptr;
    g_create_error.clear();
    if (!path) { g_create_error = "path is NULL"; return RT_EINVAL; }
    FILE* f = std::fopen(path, "rb");
    if (!f) { g_create_error = std::string("cannot open ") + path; return RT_EINVAL; }
    // the file's size first: every count the header claims is checked against it before any
    // buffer is sized from that count
    long long fsize = -1;
    if (std::fseek(f, 0, SEEK_END) == 0) fsize = (long long)std::ftell(f);
    std::rewind(f);
    char magic[8];
    uint32_t hdr[2] = {0, 0};
    rt_config cfg{};
    int64_t nc = -1, ns = -1;
    const long long head = 8 + 8 + (long long)sizeof(rt_config) + 8;    // magic, version, config, cell count
    bool ok = fsize >= head && std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkptMagic, 8) == 0 &&
              std::fread(hdr, 4, 2, f) == 2 && hdr[0] == kCkptVersion && hdr[1] == sizeof(rt_config) &&
              std::fread(&cfg, sizeof(rt_config), 1, f) == 1 && std::fread(&nc, 8, 1, f) == 1 &&
              cfg.n >= 1 && cfg.n <= 1024 && nc == (int64_t)cfg.n * cfg.n * cfg.n;
    const long long at_ns = head + 16 * (long long)nc;                  // n_H and x, then the source count
    ok = ok && fsize >= at_ns + 8 && std::fseek(f, (long)at_ns, SEEK_SET) == 0 && std::fread(&ns, 8, 1, f) == 1 &&
         ns >= 0 && ns <= (int64_t(1) << 30) && fsize == at_ns + 8 + 20 * (long long)ns;
    std::vector<double> nh, x, nd;
    std::vector<int32_t> cells;
    if (ok) {
        try {
            nh.resize((size_t)nc);
            x.resize((size_t)nc);
            cells.resize((size_t)(3 * ns));
            nd.resize((size_t)ns);
        } catch (const std::bad_alloc&) {
            std::fclose(f);
            g_create_error = "out of host memory reading " + std::string(path);
            return RT_ENOMEM;
        }
        ok = std::fseek(f, (long)head, SEEK_SET) == 0 && std::fread(nh.data(), 8, (size_t)nc, f) == (size_t)nc &&
             std::fread(x.data(), 8, (size_t)nc, f) == (size_t)nc && std::fseek(f, (long)(at_ns + 8), SEEK_SET) == 0;
    }
    if (ok && ns > 0)
        ok = std::fread(cells.data(), 4, (size_t)(3 * ns), f) == (size_t)(3 * ns) &&
             std::fread(nd.data(), 8, (size_t)ns, f) == (size_t)ns;
    std::fclose(f);
    if (!ok) { g_create_error = std::string(path) + " is not a complete checkpoint of this library"; return RT_EINVAL; }
    rt_handle* h = nullptr;
    int rc = rt_create(&cfg, cuda_stream, &h);
    if (rc) return rc;
    rc = rt_set_fields(h, nh.data(), x.data(), RT_HOST);
    if (!rc && ns > 0) rc = rt_add_sources(h, cells.data(), nd.data(), ns, RT_HOST);
    if (rc) {
        g_create_error = h->err;
        rt_destroy(h);
        return rc;
    }
    *out = h;
    return RT_OK;
}

int rt_get_x(rt_handle* h, double* x_out, int where)
{
    if (!h || !x_out || (where != RT_HOST && where != RT_DEVICE)) return h ? fail(h, RT_EINVAL, "bad arguments") : RT_EINVAL;
    if (h->sticky) return RT_ESTATE;
    DeviceGuard g(h->device);
    RT_CUDA(h, cudaMemcpyAsync(x_out, h->d_x, sizeof(double) * (size_t)h->ncell,
                               where == RT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream), "x copy");
    RT_CUDA(h, cudaStreamSynchronize(h->stream), "x copy");
    return RT_OK;
}

int rt_step(rt_handle* h, double dt_s, double* gamma_out, double* heat_out, int where, rt_stats* st)
{
    NvtxRange nvtx("rt_step");
    if (!h) return RT_EINVAL;
    if (h->sticky) return RT_ESTATE;
    if (where != RT_HOST && where != RT_DEVICE) return fail(h, RT_EINVAL, "bad where");
    if (!h->fields_set) return fail(h, RT_ESTATE, "rt_set_fields has not been called");
    if (h->cfg.chem_iterate && !(dt_s > 0)) return fail(h, RT_EINVAL, "dt_s must be positive with chem_iterate");
    DeviceGuard g(h->device);
    cudaStream_t s = h->stream;
    h->launches = 0;
    h->err.clear();
    RT_CUDA(h, cudaMemsetAsync(h->d_st, 0, sizeof(DevStats), s), "stats clear");
    RT_CUDA(h, cudaEventRecord(h->ev[0], s), "event");

    bool merged = false;
    int64_t n_dedup = 0;
    {
        const int rc = prepare_sources(h, &merged, &n_dedup);
        if (rc) return rc;
    }
    const int64_t m = h->n_emit;

    // ---- trace, optionally iterated with the C2-Ray update (Sec. 2.4)
    int iters = 0;
    double resid = 0.0;
    const double* xuse = h->d_x;
    if (h->cfg.chem_iterate) {
        RT_CUDA(h, cudaMemcpyAsync(h->d_xavg, h->d_x, sizeof(double) * (size_t)h->ncell, cudaMemcpyDeviceToDevice, s), "x copy");
        xuse = h->d_xavg;
        const int maxit = h->cfg.chem_max_iter > 0 ? h->cfg.chem_max_iter : 100;
        for (;;) {
            int rc = trace(h, h->d_xavg);
            if (rc) return rc;
            ++iters;
            // the update overwrites <x>; keep the traced one for heating until convergence is known
            RT_CUDA(h, cudaMemcpyAsync(h->d_heat, h->d_xavg, sizeof(double) * (size_t)h->ncell, cudaMemcpyDeviceToDevice, s),
                    "x copy");
            RT_CUDA(h, cudaMemsetAsync(&h->d_st->maxdiff, 0, sizeof(double), s), "clear");
            h->launches += launch_chem_update(h->d_nh, h->d_x, h->d_xavg, h->d_xend, h->d_gamma, h->ncell, dt_s,
                                              h->cfg.alpha_B, h->cfg.C_H, h->cfg.clumping, h->d_st, s);
            RT_LAUNCHED(h, "chemistry launch");
            RT_CUDA(h, cudaMemcpyAsync(h->h_f64 + 2, &h->d_st->maxdiff, sizeof(double), cudaMemcpyDeviceToHost, s),
                    "residual read");
            RT_CUDA(h, cudaStreamSynchronize(s), "chemistry");
            resid = h->h_f64[2];
            if (resid < h->cfg.chem_tol || iters >= maxit) break;
        }
        // heating uses the <x> the last trace used (saved in d_heat); new x = x(t + dt)
        std::swap(h->d_xavg, h->d_heat);
        xuse = h->d_xavg;
    } else {
        int rc = trace(h, h->d_x);
        if (rc) return rc;
        iters = 1;
    }

    // ---- heating, deposited photons
    RT_CUDA(h, cudaMemsetAsync(&h->d_st->deposited, 0, sizeof(double), s), "clear");
    h->launches += launch_finalize(h->d_gamma, h->d_nh, xuse, h->ncell, h->cfg.e_heat_erg, h->vol, h->d_heat, h->d_st, s);
    RT_LAUNCHED(h, "finalize launch");
    if (h->cfg.chem_iterate)
        RT_CUDA(h, cudaMemcpyAsync(h->d_x, h->d_xend, sizeof(double) * (size_t)h->ncell, cudaMemcpyDeviceToDevice, s),
                "x update");
    const size_t fb = sizeof(double) * (size_t)h->ncell;
    const cudaMemcpyKind k = where == RT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (gamma_out) RT_CUDA(h, cudaMemcpyAsync(gamma_out, h->d_gamma, fb, k, s), "gamma copy");
    if (heat_out) RT_CUDA(h, cudaMemcpyAsync(heat_out, h->d_heat, fb, k, s), "heat copy");
    RT_CUDA(h, cudaEventRecord(h->ev[3], s), "event");
    RT_CUDA(h, cudaMemcpyAsync(h->h_st, h->d_st, sizeof(DevStats), cudaMemcpyDeviceToHost, s), "stats read");
    RT_CUDA(h, cudaStreamSynchronize(s), "step");
    if (h->h_st->err) return fail(h, RT_EDEVICE, "a kernel reported an internal error");

    if (st) {
        std::memset(st, 0, sizeof(*st));
        const DevStats& d = *h->h_st;
        st->n_src_in = h->nsrc;
        st->n_src_dedup = n_dedup;
        st->n_src_emit = m;
        st->merged = merged ? 1 : 0;
        st->chem_iters = iters;
        st->level_max = h->level_max;
        st->launches = h->launches;
        for (int l = 0; l < RT_MAX_LEVELS; ++l) {
            st->rays[l] = (int64_t)d.rays[l];
            st->splits[l] = (int64_t)d.splits[l];
            st->escaped[l] = (int64_t)d.escaped[l];
            st->dropped_tau[l] = (int64_t)d.dropped_tau[l];
            st->dropped_level[l] = (int64_t)d.dropped_level[l];
            st->segments[l] = (int64_t)d.segments[l];
            st->secondary[l] = (int64_t)d.secondary[l];
        }
        st->emitted_ph = d.emitted;
        st->visit_hash = d.visit_hash;
        st->absorbed_ph = d.absorbed;
        st->escaped_ph = d.escaped_ph;
        st->dropped_ph = d.dropped_ph;
        st->deposited_ph = d.deposited;
        st->chem_residual = resid;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev[1], h->ev[2]);
        st->ms_trace = ms;
        cudaEventElapsedTime(&ms, h->ev[0], h->ev[3]);
        st->ms_step = ms;
        st->ms_march = h->ms_march;
        st->march_launches = h->march_launches;
        st->table_levels = h->table_levels;
    }
    return RT_OK;
}

}  // extern "C"
