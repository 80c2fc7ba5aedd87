/*
 * rt_oracle.c -- plain, slow CPU oracle for the adaptive ray march of
 * "Nyx-RT: Adaptive Ray Tracing in the Nyx Hydrodynamical Code"
 * (arXiv 2512.12466).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; it is compiled
 * with gcc -O2 -ffp-contract=off so every floating-point operation is the
 * IEEE operation written here.
 *
 * What it computes, in the paper's order:
 *   - absorber density n_HI = (1 - x) n_H (Sec. 2.6) and the optical depth per
 *     cell length kappa = sigma n_HI dx (Eq. 2, gray cross-section);
 *   - source deduplication and lexicographic sort (Sec. 2.8), optional
 *     bubble-radius source merging (Alg. 3);
 *   - the ray-tracing loop (Alg. 2): 12 HEALPix level-0 rays per source,
 *     march (Alg. 1 RAYMARCH, Amanatides-Woo), filter (RAY_FLTR) and 4-way
 *     split (S_COPY/S_TSFM) at the radius where the split criterion Eq. 4
 *     first holds;
 *   - the photon-conserving photoionization rate per segment (Eq. 1 with
 *     V_box = h^3, gray) and the overlap correction (Eq. 5-6, conservative
 *     thresholding Eq. 7-8);
 *   - the C2-Ray time-averaged chemistry update of Eq. 3 and the iterative
 *     Gamma <-> x solve (Sec. 2.3-2.4);
 *   - a photon ledger: emitted = absorbed + escaped + dropped.
 *
 * Readings of the paper fixed here (each also listed in the design notes):
 *   R-dir   Ray directions are HEALPix nested pixel centres (Gorski et al.
 *           2005) quantised to 2^-21 per component: D_a = round(|d_a| 2^21).
 *           Rays run along o + t (sD / 2^21) with t the ray parameter; path
 *           length is t |sD| / 2^21.  All traversal decisions are exact
 *           integer comparisons.
 *   R-split Eq. 4 with Omega_c = dx^2/R^2 and Omega(l) = 4pi/(12 4^l) holds
 *           from R_l = 2^l sqrt(3/(pi N_min)) on; a level-l ray runs from
 *           R_{l-1} (0 for l = 0) to R_l, where its 4 children start.  R_0 is
 *           quantised to Rq / 2^24.
 *   R-start A child whose start point lies exactly on a face is in the cell it
 *           is entering.  Ties between face crossings step all tied axes.
 *   R-tau   tau_max is tested after every deposit; the rest of the budget is
 *           "dropped".
 *   R-edge  D_edge is the distance from the segment midpoint to the nearest of
 *           the six faces (order x-, x+, y-, y+, z-, z+, first wins ties);
 *           c' is the cell across it; L_pix = r_mid sqrt(pi/3) / 2^l.
 *   R-elig  Eq. 7-8 eligibility also needs n'_HI > 0 and c' inside the grid.
 *   R-chem  n_e = <x> n_H, C2-Ray closed form for constant rates.
 *   R-merge Alg. 3 samples are HEALPix level-Ls directions (quantised as above),
 *           a sample cell is floor(c + 1/2 + r d); P(r) is the set of distinct
 *           in-grid sample cells; both radii must be positive for a merge edge.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_S 21                 /* direction fractional bits */
#define ORC_F 24                 /* split-radius fractional bits */
#define ORC_MAXLEV 16
#define ORC_STACK 128
#define ORC_SQRT_PI_3 1.0233267079464885   /* sqrt(pi/3): pixel width = r sqrt(Omega(l)) */

/* Beam-overlap treatments of Sec. 2.6: none; Eq. 5 alone; Eqs. 5-6; Eqs. 7-8
 * (conservative threshold); the squared f_c; and the naive threshold, which
 * keeps Eq. 5 but drops the Eq. 6 deposit when n'_H < n_th (the first
 * remedy the paper tried, which loses photons). */
enum { ORC_OVERLAP_NONE = 0, ORC_OVERLAP_LINEAR = 1, ORC_OVERLAP_ARC = 2,
       ORC_OVERLAP_CONSERVATIVE = 3, ORC_OVERLAP_SQUARED = 4, ORC_OVERLAP_NAIVE = 5 };

typedef struct {
    int32_t n;
    int32_t precision;           /* 0: FP64 physics, 1: FP32 physics with Kahan budgets */
    double box_cm;
    double sigma_cm2;
    double n_min_ray;
    int32_t level_max;           /* < 0: smallest l with R_l >= sqrt(3) n, plus one */
    int32_t overlap_mode;
    double tau_max;
    double n_th_cm3;             /* Eq. 7-8 threshold on n'_H */
    double e_heat_erg;
    int32_t merge_mode;          /* 0 off, 1 forced, 2 automerge */
    int32_t merge_samp_level;
    double automerge_xbar;
    double merge_x_th, merge_f_req;
    double merge_dr_cells, merge_rmax_cells, merge_f_ov, merge_eps;
    int32_t merge_n_min;
    int32_t chem_iterate;
    double dt_s, alpha_B, C_H, clumping, chem_tol;
    int32_t chem_max_iter;
    int32_t periodic;            /* 1: periodic boundaries (Sec. 2.5.1) */
    int32_t spectrum;            /* 0: gray sigma; 1: frequency-integrated Eq. 1 (Sec. 2.5) */
    int32_t nq;                  /* quadrature nodes over frequency (spectrum 1) */
    const double* q_s;           /* sigma_nu / sigma_0 at each node */
    const double* q_w;           /* normalised photon-number weight of each node (they sum to 1) */
} orc_config;

typedef struct {
    int64_t n_src_in, n_src_dedup, n_src_emit;
    int32_t merged, chem_iters;
    int32_t level_max, pad_;
    int64_t rays[ORC_MAXLEV], splits[ORC_MAXLEV], escaped[ORC_MAXLEV];
    int64_t dropped_tau[ORC_MAXLEV], dropped_level[ORC_MAXLEV];
    int64_t segments[ORC_MAXLEV], secondary[ORC_MAXLEV];
    uint64_t visit_hash;
    double emitted_ph, absorbed_ph, escaped_ph, dropped_ph, deposited_ph;
    double chem_residual;
} orc_stats;

/* Compensated (Kahan) FP64 accumulator for the global photon totals. */
typedef struct { double s, c; } orc_sum;

static void orc_sum_add(orc_sum* acc, double v)
{
    const double y = v - acc->c;
    const double t = acc->s + y;
    acc->c = (t - acc->s) - y;
    acc->s = t;
}

typedef struct {
    int64_t n;
    const double* kap_d;         /* signed kappa; sign bit set = not eligible as c' (Eq. 7-8) */
    const float* kap_f;
    double* gamma;
    double sigma_over_dx2;
    int64_t rq;
    int level_max;
    double tau_max;
    int overlap_mode;
    int spectrum;                /* Eq. 1 over frequency: quadrature nodes below */
    int nq;
    const double* q_s;
    const double* q_w;
    int periodic;                /* Sec. 2.5.1: rays wrap around the box ... */
    int64_t rs;                  /* ... and stop at travel distance sqrt(3) L_box (2^-F cells) */
    orc_stats* st;
    orc_sum emitted, absorbed, escaped, dropped;
    int64_t* rec_ray;
    int32_t* rec_seq;
    int64_t* rec_cell;
    double* rec_ds;
    int64_t rec_cap, rec_n;
} orc_ctx;

/* ------------------------------------------------------------------ */
/* Hashing of the visit list (bookkeeping only).                      */

/* splitmix64 output function (Steele, Lea & Flood 2014). */
static uint64_t orc_mix64(uint64_t z)
{
    z ^= z >> 30;
    z *= 0xbf58476d1ce4e5b9ULL;
    z ^= z >> 27;
    z *= 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return z;
}

uint64_t orc_mix64_export(uint64_t z) { return orc_mix64(z); }

/* ------------------------------------------------------------------ */
/* HEALPix nested pixel centres (Sec. 2.5: rays are HEALPix pixels;   */
/* children of pixel p at level l are 4p..4p+3 at level l+1).         */

static const int orc_jrll[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
static const int orc_jpll[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

/* Unit vector of nested pixel `pix` at level `level` (N_side = 2^level),
 * following Gorski et al. (2005): face and in-face (x, y) from the bit
 * interleave, ring index, then z and phi of the ring. */
void orc_pix2vec(int32_t level, int64_t pix, double v[3])
{
    const int64_t nside = (int64_t)1 << level;
    const int64_t npface = nside * nside;
    const int face = (int)(pix / npface);
    int64_t ipf = pix % npface;
    int64_t ix = 0, iy = 0;
    for (int b = 0; b < level; b++) {           /* de-interleave: even bits -> x, odd bits -> y */
        ix |= ((ipf >> (2 * b)) & 1) << b;
        iy |= ((ipf >> (2 * b + 1)) & 1) << b;
    }
    const int64_t jr = orc_jrll[face] * nside - ix - iy - 1;   /* ring number, 1 .. 4 nside - 1 */
    int64_t nr;
    int kshift;
    double z, sth;
    if (jr < nside) {                            /* north polar cap */
        nr = jr;
        const double q = (double)(nr * nr) / (double)(3 * nside * nside);
        z = 1.0 - q;
        sth = sqrt(q * (2.0 - q));
        kshift = 0;
    } else if (jr > 3 * nside) {                 /* south polar cap */
        nr = 4 * nside - jr;
        const double q = (double)(nr * nr) / (double)(3 * nside * nside);
        z = q - 1.0;
        sth = sqrt(q * (2.0 - q));
        kshift = 0;
    } else {                                     /* equatorial belt */
        nr = nside;
        z = ((double)(2 * nside - jr) * 2.0) / (double)(3 * nside);
        sth = sqrt((1.0 - z) * (1.0 + z));
        kshift = (int)((jr - nside) & 1);
    }
    int64_t jp = (orc_jpll[face] * nr + ix - iy + 1 + kshift) / 2;
    if (jp > 4 * nside) jp -= 4 * nside;
    if (jp < 1) jp += 4 * nside;
    const double phi = (((double)jp - 0.5 * (double)(kshift + 1)) * 1.5707963267948966) / (double)nr;
    v[0] = sth * cos(phi);
    v[1] = sth * sin(phi);
    v[2] = z;
}

/* Quantised ray direction (reading R-dir): sd_a = sign(d_a) round(|d_a| 2^S),
 * and |sd| / 2^S in FP64. */
void orc_direction(int32_t level, int64_t pix, int32_t sd[3], double* nrm)
{
    double v[3];
    orc_pix2vec(level, pix, v);
    int64_t ss = 0;
    for (int a = 0; a < 3; a++) {
        const double m = fabs(v[a]) * (double)(1 << ORC_S);
        const int32_t q = (int32_t)floor(m + 0.5);
        sd[a] = v[a] < 0 ? -q : q;
        ss += (int64_t)q * q;
    }
    *nrm = sqrt((double)ss) / (double)(1 << ORC_S);
}

/* T_a(ka) < T_b(kb), with T(k) = (2k+1)/D (infinite when D = 0). */
static int orc_t_less(int64_t ka, int64_t Da, int64_t kb, int64_t Db)
{
    return (2 * ka + 1) * Db < (2 * kb + 1) * Da;
}

/* Split radius numerator (reading R-split): R_0 = sqrt(3/(pi N_min)) in
 * units of 2^-F cells.  Eq. 4: Omega_c / Omega(l) < N_min with
 * Omega_c = 1/R^2 and Omega(l) = 4 pi / (12 4^l)  <=>  R > 2^l sqrt(3/(pi N_min)). */
int64_t orc_split_rq(double n_min_ray)
{
    const double r0 = sqrt(3.0 / (3.141592653589793 * n_min_ray));
    return (int64_t)floor(r0 * (double)(1 << ORC_F) + 0.5);
}

/* Periodic boundaries (Sec. 2.5.1): a ray stops once its travel distance
 * reaches sqrt(3) L_box, i.e. sqrt(3) n cells; in the split radius's fixed
 * point (2^-F cells), rounded to nearest. */
int64_t orc_periodic_rs(int32_t n)
{
    return (int64_t)floor(sqrt(3.0) * (double)n * (double)(1 << ORC_F) + 0.5);
}

/* Default l_max: smallest l with R_l >= sqrt(3) n, plus one, so it never
 * binds on a non-periodic grid. */
int32_t orc_default_level_max(int32_t n, double n_min_ray)
{
    const int64_t rq = orc_split_rq(n_min_ray);
    const double reach = sqrt(3.0) * (double)n;
    int l = 0;
    while (ldexp((double)rq, l - ORC_F) < reach) l++;
    return l + 1;
}

/* ------------------------------------------------------------------ */
/* The march, in FP64 and FP32 physics.                               */

/* Frequency-integrated photoionization (Eq. 1; Sec. 2.5, after C2-Ray): a
 * ray's photons are spread over frequency with normalised weights w_k at
 * cross-section ratios s_k = sigma_nu/sigma_0, so optical depth tau at the
 * threshold is tau s_k at node k.  Fraction of the ray's photons that
 * survive tau: Phi(tau) = sum_k w_k exp(-tau s_k).  Fraction absorbed over a
 * segment of optical depth dtau after tau: sum_k w_k exp(-tau s_k) (1 - exp(-dtau s_k)),
 * with expm1 so that thin segments keep their precision.  Optically thin
 * rate per unit dtau: sum_k w_k s_k exp(-tau s_k). */
static double orc_phi(const orc_ctx* C, double tau)
{
    double s = 0.0;
    for (int k = 0; k < C->nq; k++) s += C->q_w[k] * exp(-tau * C->q_s[k]);
    return s;
}

static double orc_absorbed(const orc_ctx* C, double tau, double dtau)
{
    double s = 0.0;
    for (int k = 0; k < C->nq; k++) s += C->q_w[k] * exp(-tau * C->q_s[k]) * (-expm1(-dtau * C->q_s[k]));
    return s;
}

static double orc_thin_rate(const orc_ctx* C, double tau)
{
    double s = 0.0;
    for (int k = 0; k < C->nq; k++) s += C->q_w[k] * C->q_s[k] * exp(-tau * C->q_s[k]);
    return s;
}

#define REAL double
#define SFX(x) x##_d
#define R_EXPM1 expm1
#define R_FABS fabs
#define R_LDEXP ldexp
#define R_SIGNBIT signbit
#define KAPPA_FIELD kap_d
#define R_KAHAN 0
#include "march_body.h"
#undef REAL
#undef SFX
#undef R_EXPM1
#undef R_FABS
#undef R_LDEXP
#undef R_SIGNBIT
#undef KAPPA_FIELD
#undef R_KAHAN

#define REAL float
#define SFX(x) x##_f
#define R_EXPM1 expm1f
#define R_FABS fabsf
#define R_LDEXP ldexpf
#define R_SIGNBIT signbit
#define KAPPA_FIELD kap_f
#define R_KAHAN 1
#include "march_body.h"
#undef REAL
#undef SFX
#undef R_EXPM1
#undef R_FABS
#undef R_LDEXP
#undef R_SIGNBIT
#undef KAPPA_FIELD
#undef R_KAHAN

/* ------------------------------------------------------------------ */
/* Field preparation (Sec. 2.6: a_abs = (1 - x) n_H; Eq. 2).          */

/* kappa = (sigma dx) ((1 - x) n_H); stored negated (sign bit set) when the
 * cell cannot receive a secondary deposit under Eq. 7-8: n_H < n_th or
 * n_HI = 0. */
void orc_prepare_kappa(int64_t ncell, const double* n_h, const double* x, double sigma_dx,
                       double n_th, double* kap)
{
    for (int64_t c = 0; c < ncell; c++) {
        const double nhi = (1.0 - x[c]) * n_h[c];
        const double k = sigma_dx * nhi;
        const int elig = (n_h[c] >= n_th) && (nhi > 0.0);
        kap[c] = elig ? k : -k;
    }
}

/* ------------------------------------------------------------------ */
/* Sources (Sec. 2.8): deduplicate by cell summing fluxes, sort.      */

typedef struct { int32_t c[3]; int64_t idx; } orc_key;

static int orc_key_cmp(const void* pa, const void* pb)
{
    const orc_key* a = (const orc_key*)pa;
    const orc_key* b = (const orc_key*)pb;
    for (int q = 0; q < 3; q++) {
        if (a->c[q] != b->c[q]) return a->c[q] < b->c[q] ? -1 : 1;
    }
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

/* Sort by (ix, iy, iz) lexicographically (input order among equal cells),
 * sum the rates of sources sharing a cell in that order.  Returns the count. */
int64_t orc_sources_dedup(const int32_t* cells, const double* ndot, int64_t nsrc,
                          int32_t* out_cells, double* out_ndot)
{
    orc_key* keys = (orc_key*)malloc(sizeof(orc_key) * (size_t)(nsrc > 0 ? nsrc : 1));
    for (int64_t j = 0; j < nsrc; j++) {
        for (int q = 0; q < 3; q++) keys[j].c[q] = cells[3 * j + q];
        keys[j].idx = j;
    }
    qsort(keys, (size_t)nsrc, sizeof(orc_key), orc_key_cmp);
    int64_t m = 0;
    for (int64_t j = 0; j < nsrc; j++) {
        const orc_key* k = &keys[j];
        if (m > 0 && out_cells[3 * (m - 1)] == k->c[0] && out_cells[3 * (m - 1) + 1] == k->c[1] &&
            out_cells[3 * (m - 1) + 2] == k->c[2]) {
            out_ndot[m - 1] += ndot[k->idx];
        } else {
            for (int q = 0; q < 3; q++) out_cells[3 * m + q] = k->c[q];
            out_ndot[m] = ndot[k->idx];
            m++;
        }
    }
    free(keys);
    return m;
}

static int orc_i64_cmp(const void* a, const void* b)
{
    const int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Minimum-image component of a cell offset on a periodic grid of n cells:
 * d mod n in [0, n), less n when above n/2. */
static int64_t orc_minimg(int64_t d, int64_t n)
{
    int64_t r = ((d % n) + n) % n;
    return 2 * r > n ? r - n : r;
}

/* Alg. 3 MAX_RADIUS: grow shells by dr while the sampled shell is ionized.
 * With periodic boundaries a sample outside the grid wraps into it (the
 * paper computes Alg. 3 under minimum-image geometry); otherwise it is not
 * evaluated. */
double orc_max_radius(int32_t n, const double* x, const int32_t c[3], int32_t samp_level,
                      double x_th, double f_req, int32_t n_min, double dr, double rmax, int32_t periodic)
{
    const int64_t nn = n;
    if (x[((int64_t)c[2] * nn + c[1]) * nn + c[0]] < x_th) return 0.0;
    const int64_t ns = 12 * ((int64_t)1 << (2 * samp_level));
    int32_t* dirs = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)ns);
    for (int64_t p = 0; p < ns; p++) {
        double nrm;
        orc_direction(samp_level, p, &dirs[3 * p], &nrm);
    }
    int64_t* cellv = (int64_t*)malloc(sizeof(int64_t) * (size_t)ns);
    double r = dr;
    double result = rmax;
    while (r <= rmax) {
        int64_t m = 0;
        for (int64_t p = 0; p < ns; p++) {
            int64_t q[3];
            int inside = 1;
            for (int a = 0; a < 3; a++) {
                const double pos = ((double)c[a] + 0.5) + r * ((double)dirs[3 * p + a] / (double)(1 << ORC_S));
                q[a] = (int64_t)floor(pos);
                if (periodic) q[a] = ((q[a] % nn) + nn) % nn;
                if (q[a] < 0 || q[a] >= nn) inside = 0;
            }
            if (inside) cellv[m++] = (q[2] * nn + q[1]) * nn + q[0];
        }
        qsort(cellv, (size_t)m, sizeof(int64_t), orc_i64_cmp);
        int64_t ntot = 0, nion = 0;
        for (int64_t j = 0; j < m; j++) {
            if (j > 0 && cellv[j] == cellv[j - 1]) continue;
            ntot++;
            if (x[cellv[j]] >= x_th) nion++;
        }
        int fail;
        if (ntot < n_min) fail = (nion < ntot);                       /* all samples must be ionized */
        else fail = ((double)nion / (double)ntot < f_req);
        if (fail) { result = r - dr; break; }
        r += dr;
    }
    free(cellv);
    free(dirs);
    return result;
}

static int64_t orc_find(int64_t* parent, int64_t a)
{
    while (parent[a] != a) {
        parent[a] = parent[parent[a]];
        a = parent[a];
    }
    return a;
}

typedef struct { int32_t c[3]; double ndot; } orc_msrc;

static int orc_msrc_cmp(const void* pa, const void* pb)
{
    const orc_msrc* a = (const orc_msrc*)pa;
    const orc_msrc* b = (const orc_msrc*)pb;
    for (int q = 0; q < 3; q++) {
        if (a->c[q] != b->c[q]) return a->c[q] < b->c[q] ? -1 : 1;
    }
    return 0;
}

/* Alg. 3 MERGE_SOURCES on a deduplicated, sorted catalog.  Sources whose
 * bubbles overlap (d^2 <= (f_ov (r_a + r_b))^2 + eps, both radii positive)
 * are joined by union-find; each group becomes one source with the summed
 * rate at the member cell nearest to the rounded flux-weighted centroid.
 * Writes the merged catalog sorted lexicographically; returns its size.
 * `radius` receives the per-source bubble radii; `label` the group root. */
int64_t orc_merge_sources(int32_t n, const double* x, const int32_t* cells, const double* ndot,
                          int64_t nsrc, int32_t samp_level, double x_th, double f_req, int32_t n_min,
                          double dr, double rmax, double f_ov, double eps, int32_t periodic,
                          double* radius, int64_t* label, int32_t* out_cells, double* out_ndot)
{
    for (int64_t j = 0; j < nsrc; j++)
        radius[j] = orc_max_radius(n, x, &cells[3 * j], samp_level, x_th, f_req, n_min, dr, rmax, periodic);
    int64_t* parent = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nsrc > 0 ? nsrc : 1));
    for (int64_t j = 0; j < nsrc; j++) parent[j] = j;
    for (int64_t a = 0; a < nsrc; a++) {
        if (!(radius[a] > 0)) continue;
        for (int64_t b = a + 1; b < nsrc; b++) {
            if (!(radius[b] > 0)) continue;
            int64_t d2 = 0;
            for (int q = 0; q < 3; q++) {
                int64_t d = (int64_t)cells[3 * a + q] - cells[3 * b + q];
                if (periodic) d = orc_minimg(d, n);                  /* minimum-image distance */
                d2 += d * d;
            }
            const double rs = f_ov * (radius[a] + radius[b]);
            if ((double)d2 <= rs * rs + eps) {
                int64_t ra = orc_find(parent, a), rb = orc_find(parent, b);
                if (ra != rb) {
                    if (ra < rb) parent[rb] = ra; else parent[ra] = rb;
                }
            }
        }
    }
    for (int64_t j = 0; j < nsrc; j++) label[j] = orc_find(parent, j);

    orc_msrc* out = (orc_msrc*)malloc(sizeof(orc_msrc) * (size_t)(nsrc > 0 ? nsrc : 1));
    int64_t m = 0;
    for (int64_t g = 0; g < nsrc; g++) {
        if (label[g] != g) continue;                 /* g is the first (smallest) member of its group */
        double ftot = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        int64_t count = 0;
        for (int64_t j = g; j < nsrc; j++) {
            if (label[j] != g) continue;
            /* periodic: each member unwrapped next to the group's first member */
            double u[3];
            for (int q = 0; q < 3; q++)
                u[q] = periodic ? (double)(cells[3 * g + q] + orc_minimg((int64_t)cells[3 * j + q] - cells[3 * g + q], n))
                                : (double)cells[3 * j + q];
            ftot += ndot[j];
            sx += ndot[j] * u[0];
            sy += ndot[j] * u[1];
            sz += ndot[j] * u[2];
            count++;
        }
        if (count == 1) {
            for (int q = 0; q < 3; q++) out[m].c[q] = cells[3 * g + q];
            out[m].ndot = ndot[g];
            m++;
            continue;
        }
        const double cen[3] = {sx / ftot, sy / ftot, sz / ftot};
        int64_t rc[3];
        for (int q = 0; q < 3; q++) {
            rc[q] = (int64_t)floor(cen[q] + 0.5);
            if (periodic) {
                rc[q] = ((rc[q] % n) + n) % n;         /* wrap back into the grid */
            } else {
                if (rc[q] < 0) rc[q] = 0;              /* non-periodic: clamp into the grid */
                if (rc[q] > n - 1) rc[q] = n - 1;
            }
        }
        int64_t best = -1, bestd = 0;
        for (int64_t j = g; j < nsrc; j++) {
            if (label[j] != g) continue;
            int64_t d2 = 0;
            for (int q = 0; q < 3; q++) {
                int64_t d = (int64_t)cells[3 * j + q] - rc[q];
                if (periodic) d = orc_minimg(d, n);
                d2 += d * d;
            }
            if (best < 0 || d2 < bestd) { best = j; bestd = d2; }
        }
        for (int q = 0; q < 3; q++) out[m].c[q] = cells[3 * best + q];
        out[m].ndot = ftot;
        m++;
    }
    qsort(out, (size_t)m, sizeof(orc_msrc), orc_msrc_cmp);
    for (int64_t j = 0; j < m; j++) {
        for (int q = 0; q < 3; q++) out_cells[3 * j + q] = out[j].c[q];
        out_ndot[j] = out[j].ndot;
    }
    free(out);
    free(parent);
    return m;
}

/* ------------------------------------------------------------------ */
/* Chemistry (Eq. 3) with the C2-Ray time average (Sec. 2.3).         */

/* For constant rates over dt: ionization I = Gamma + n_e C_H, recombination
 * R = n_e C alpha_B; x_eq = I/(I+R), t_i = 1/(I+R);
 * x(dt) = x_eq + (x0 - x_eq) exp(-dt/t_i),
 * <x>  = x_eq + (x0 - x_eq) (1 - exp(-dt/t_i)) t_i/dt.
 * n_e = <x>_prev n_H (hydrogen only).  Returns max |<x>_new - <x>_prev|. */
double orc_chem_update(int64_t ncell, const double* n_h, const double* x0, double* xavg,
                       const double* gamma, double dt, double alpha_B, double C_H, double clump,
                       double* xend)
{
    double maxd = 0.0;
    for (int64_t c = 0; c < ncell; c++) {
        const double ne = xavg[c] * n_h[c];
        const double ion = gamma[c] + ne * C_H;
        const double rec = ne * clump * alpha_B;
        const double tot = ion + rec;
        double xe, xa;
        if (tot > 0.0) {
            const double xeq = ion / tot;
            const double u = dt * tot;
            xe = xeq + (x0[c] - xeq) * exp(-u);
            xa = xeq + (x0[c] - xeq) * (-expm1(-u) / u);
        } else {
            xe = x0[c];
            xa = x0[c];
        }
        const double d = fabs(xa - xavg[c]);
        if (d > maxd) maxd = d;
        xavg[c] = xa;
        xend[c] = xe;
    }
    return maxd;
}

/* ------------------------------------------------------------------ */
/* One trace of all sources at fixed x.                               */

static void orc_trace(const orc_config* cfg, int64_t rq, int level_max, const double* n_h,
                      const double* xuse, const int32_t* cells, const double* ndot, int64_t nsrc,
                      double* gamma, orc_stats* st, int64_t* rec_ray, int32_t* rec_seq,
                      int64_t* rec_cell, double* rec_ds, int64_t rec_cap, int64_t* rec_n)
{
    const int64_t n = cfg->n;
    const int64_t ncell = n * n * n;
    const double dx = cfg->box_cm / (double)n;
    double* kap = (double*)malloc(sizeof(double) * (size_t)ncell);
    orc_prepare_kappa(ncell, n_h, xuse, cfg->sigma_cm2 * dx, cfg->n_th_cm3, kap);
    float* kapf = NULL;
    if (cfg->precision == 1) {
        kapf = (float*)malloc(sizeof(float) * (size_t)ncell);
        for (int64_t c = 0; c < ncell; c++) kapf[c] = (float)kap[c];
    }
    memset(gamma, 0, sizeof(double) * (size_t)ncell);
    orc_ctx C;
    memset(&C, 0, sizeof(C));
    C.n = n;
    C.kap_d = kap;
    C.kap_f = kapf;
    C.gamma = gamma;
    C.sigma_over_dx2 = cfg->sigma_cm2 / (dx * dx);
    C.rq = rq;
    C.level_max = level_max;
    C.tau_max = cfg->tau_max;
    C.overlap_mode = cfg->overlap_mode;
    C.periodic = cfg->periodic != 0;
    C.spectrum = cfg->spectrum;
    C.nq = cfg->nq;
    C.q_s = cfg->q_s;
    C.q_w = cfg->q_w;
    C.rs = C.periodic ? orc_periodic_rs((int32_t)n) : 0;
    C.st = st;
    C.rec_ray = rec_ray;
    C.rec_seq = rec_seq;
    C.rec_cell = rec_cell;
    C.rec_ds = rec_ds;
    C.rec_cap = rec_cap;
    if (cfg->precision == 1) trace_all_f(&C, cells, ndot, nsrc);
    else trace_all_d(&C, cells, ndot, nsrc);
    st->emitted_ph = C.emitted.s;
    st->absorbed_ph = C.absorbed.s;
    st->escaped_ph = C.escaped.s;
    st->dropped_ph = C.dropped.s;
    if (rec_n) *rec_n = C.rec_n;
    free(kapf);
    free(kap);
}

/* Full solve: sources, optional merge, trace (and chemistry iterations),
 * heating = e_heat Gamma n_HI, ledger.  Returns 0 on success, negative on
 * invalid input.  x_out receives x at the end of the step (the input x when
 * chemistry is off).  Record arrays may be NULL (rec_cap = 0). */
int orc_run(const orc_config* cfg, const double* n_h, const double* x_in, const int32_t* cells_in,
            const double* ndot_in, int64_t nsrc, double* gamma, double* heat, double* x_out,
            orc_stats* st, int64_t* rec_ray, int32_t* rec_seq, int64_t* rec_cell, double* rec_ds,
            int64_t rec_cap, int64_t* rec_n, int32_t* emit_cells, double* emit_ndot)
{
    if (cfg->n <= 0 || cfg->n > 1024 || !(cfg->n_min_ray >= 1.0) || !(cfg->box_cm > 0) ||
        !(cfg->sigma_cm2 > 0) || !(cfg->tau_max > 0) || cfg->overlap_mode < ORC_OVERLAP_NONE ||
        cfg->overlap_mode > ORC_OVERLAP_NAIVE || (cfg->periodic != 0 && cfg->periodic != 1) ||
        (cfg->spectrum != 0 && cfg->spectrum != 1) || (cfg->spectrum == 1 && (cfg->nq < 1 || !cfg->q_s || !cfg->q_w)))
        return -1;
    const int64_t n = cfg->n;
    const int64_t ncell = n * n * n;
    for (int64_t j = 0; j < nsrc; j++) {
        for (int q = 0; q < 3; q++)
            if (cells_in[3 * j + q] < 0 || cells_in[3 * j + q] >= n) return -1;
        if (!(ndot_in[j] > 0) || !isfinite(ndot_in[j])) return -1;
    }
    for (int64_t c = 0; c < ncell; c++) {
        if (!(n_h[c] >= 0) || !isfinite(n_h[c]) || !(x_in[c] >= 0 && x_in[c] <= 1)) return -1;
    }
    memset(st, 0, sizeof(*st));
    const int64_t rq = orc_split_rq(cfg->n_min_ray);
    int level_max = cfg->level_max >= 0 ? cfg->level_max : orc_default_level_max(cfg->n, cfg->n_min_ray);
    if (level_max > 13) level_max = 13;
    st->level_max = level_max;
    st->n_src_in = nsrc;

    int32_t* dc = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(nsrc > 0 ? nsrc : 1));
    double* dn = (double*)malloc(sizeof(double) * (size_t)(nsrc > 0 ? nsrc : 1));
    int64_t m = orc_sources_dedup(cells_in, ndot_in, nsrc, dc, dn);
    st->n_src_dedup = m;
    int do_merge = 0;
    if (cfg->merge_mode == 1) do_merge = 1;
    if (cfg->merge_mode == 2) {
        double sx = 0.0;
        for (int64_t c = 0; c < ncell; c++) sx += x_in[c];
        do_merge = (sx / (double)ncell) > cfg->automerge_xbar;
    }
    if (do_merge && m > 0) {
        double* rad = (double*)malloc(sizeof(double) * (size_t)m);
        int64_t* lab = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
        int32_t* mc = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)m);
        double* mn = (double*)malloc(sizeof(double) * (size_t)m);
        int64_t mm = orc_merge_sources(cfg->n, x_in, dc, dn, m, cfg->merge_samp_level, cfg->merge_x_th,
                                       cfg->merge_f_req, cfg->merge_n_min, cfg->merge_dr_cells,
                                       cfg->merge_rmax_cells, cfg->merge_f_ov, cfg->merge_eps, cfg->periodic,
                                       rad, lab, mc, mn);
        memcpy(dc, mc, sizeof(int32_t) * 3 * (size_t)mm);
        memcpy(dn, mn, sizeof(double) * (size_t)mm);
        m = mm;
        free(rad);
        free(lab);
        free(mc);
        free(mn);
        st->merged = 1;
    }
    st->n_src_emit = m;
    if (emit_cells) memcpy(emit_cells, dc, sizeof(int32_t) * 3 * (size_t)m);
    if (emit_ndot) memcpy(emit_ndot, dn, sizeof(double) * (size_t)m);

    double* xavg = (double*)malloc(sizeof(double) * (size_t)ncell);
    memcpy(xavg, x_in, sizeof(double) * (size_t)ncell);
    memcpy(x_out, x_in, sizeof(double) * (size_t)ncell);
    int iters = 0;
    if (cfg->chem_iterate) {
        double* xnew = (double*)malloc(sizeof(double) * (size_t)ncell);
        double* xend = (double*)malloc(sizeof(double) * (size_t)ncell);
        const int maxit = cfg->chem_max_iter > 0 ? cfg->chem_max_iter : 100;
        double resid = 0.0;
        for (;;) {
            memset(st->rays, 0, sizeof(int64_t) * ORC_MAXLEV * 7);
            st->visit_hash = 0;
            st->emitted_ph = st->absorbed_ph = st->escaped_ph = st->dropped_ph = 0.0;
            orc_trace(cfg, rq, level_max, n_h, xavg, dc, dn, m, gamma, st, rec_ray, rec_seq, rec_cell,
                      rec_ds, rec_cap, rec_n);
            iters++;
            memcpy(xnew, xavg, sizeof(double) * (size_t)ncell);
            resid = orc_chem_update(ncell, n_h, x_in, xnew, gamma, cfg->dt_s, cfg->alpha_B, cfg->C_H,
                                    cfg->clumping, xend);
            memcpy(x_out, xend, sizeof(double) * (size_t)ncell);
            if (resid < cfg->chem_tol || iters >= maxit) break;
            memcpy(xavg, xnew, sizeof(double) * (size_t)ncell);
        }
        st->chem_residual = resid;
        free(xnew);
        free(xend);
    } else {
        orc_trace(cfg, rq, level_max, n_h, xavg, dc, dn, m, gamma, st, rec_ray, rec_seq, rec_cell, rec_ds,
                  rec_cap, rec_n);
        iters = 1;
    }
    st->chem_iters = iters;

    /* Heating and the deposited-photon check use the x the last trace used. */
    const double dx = cfg->box_cm / (double)n;
    const double vol = dx * dx * dx;
    orc_sum dep = {0.0, 0.0};
    for (int64_t c = 0; c < ncell; c++) {
        const double nhi = (1.0 - xavg[c]) * n_h[c];
        heat[c] = cfg->e_heat_erg * gamma[c] * nhi;
        orc_sum_add(&dep, gamma[c] * nhi * vol);
    }
    st->deposited_ph = dep.s;
    free(xavg);
    free(dc);
    free(dn);
    return 0;
}

/* Size of the structs, for the Python binding's layout check. */
int64_t orc_sizeof_config(void) { return (int64_t)sizeof(orc_config); }
int64_t orc_sizeof_stats(void) { return (int64_t)sizeof(orc_stats); }
