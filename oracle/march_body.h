/*
 * Oracle ray march, written once and included twice by rt_oracle.c:
 * once with REAL = double (FP64 physics) and once with REAL = float
 * (FP32 physics with Kahan-compensated photon and optical-depth budgets).
 * Geometry is exact integer arithmetic in both; deposits and the photon
 * ledger are FP64 in both.
 *
 * TEST INFRASTRUCTURE ONLY: see the header of rt_oracle.c.
 *
 * Expects the includer to define: REAL, SFX(name), R_EXPM1, R_FABS,
 * R_LDEXP, R_SIGNBIT, KAPPA_FIELD (member of orc_ctx holding REAL kappa),
 * R_KAHAN (1 for compensated sums, 0 for plain sums).
 */

typedef struct {
    int32_t level;
    int64_t pix;
    REAL P, cP;        /* photon budget in units of Ndot/12, and its compensation */
    REAL tau, ctau;    /* optical depth accumulated from the source, and its compensation */
} SFX(ray);

/* Photons a ray still carries (units of its budget): the compensated budget
 * P - cP (gray: P is decremented by every absorption), or, with the
 * frequency-integrated rate, P Phi(tau): P then stays the geometric budget and
 * the attenuation lives in Phi. */
static double SFX(remaining)(const orc_ctx* C, REAL P, REAL cP, REAL tau, REAL ctau)
{
    if (C->spectrum) return (double)P * orc_phi(C, (double)tau - (double)ctau);
    return (double)P - (double)cP;
}

/* Compensated (Kahan) accumulation s += v, used in FP32 mode. */
static void SFX(kahan_add)(REAL* s, REAL* c, REAL v)
{
#if R_KAHAN
    REAL y = v - *c;
    REAL t = *s + y;
    *c = (t - *s) - y;
    *s = t;
#else
    (void)c;
    *s = *s + v;
#endif
}

/*
 * March one ray of level l from the start sphere R_{l-1} (the source cell
 * centre for l = 0) to its split sphere R_l, cell by cell (Alg. 1 RAYMARCH,
 * Amanatides-Woo traversal), depositing photoionization rate into the grid
 * (Eq. 1 with V_box, gray cross-section; Eqs. 5-8 overlap correction).
 * Returns 1 and fills kids[4] when the ray reaches R_l and may split
 * (Alg. 1 RAY_FLTR + S_COPY), else 0 (escaped or dropped).
 */
static int SFX(march)(orc_ctx* C, int64_t srcidx, const int32_t cell0[3], double ndot,
                      const SFX(ray)* ray, SFX(ray) kids[4])
{
    const int S = ORC_S, F = ORC_F;
    const int64_t B = (int64_t)1 << (S - 1 + F);       /* crossing times are odd multiples of B/(2^F D) */
    const int l = ray->level;
    const int64_t n = C->n;
    orc_stats* st = C->st;

    int32_t sd[3];
    double nrm_d;
    orc_direction(l, ray->pix, sd, &nrm_d);
    int64_t D[3];
    int s[3];
    for (int a = 0; a < 3; a++) {
        D[a] = sd[a] < 0 ? -(int64_t)sd[a] : (int64_t)sd[a];
        s[a] = sd[a] < 0 ? -1 : 1;
    }

    /* Integer event bookkeeping.  Along axis a the k-th face crossing
     * (k = 0, 1, ...) happens at parametric time T_a(k) = (2k+1) 2^(S-1) / D_a;
     * the split radius is R_l = Rq 2^l / 2^F.  The ray ends at R_l, or, with
     * periodic boundaries (Sec. 2.5.1), at the travel distance sqrt(3) L_box
     * if that comes first or at the same point (RAY_FLTR keeps only rays with
     * s < sqrt(3) L_box), in which case it stops there without splitting.
     * Gend/Gstart are the end and start radii scaled by 2^F D_a. */
    const int64_t Rsplit = C->rq << l;
    const int split_end = !C->periodic || Rsplit < C->rs;
    const int64_t Rend = split_end ? Rsplit : C->rs;
    const int64_t Rstart = l > 0 ? (C->rq << (l - 1)) : 0;
    int64_t Gend[3], Gstart[3], k[3], kend[3];
    for (int a = 0; a < 3; a++) {
        Gend[a] = Rend * D[a];
        Gstart[a] = Rstart * D[a];
        k[a] = l > 0 ? (Gstart[a] + B) >> (S + F) : 0;          /* crossings with T <= R_{l-1} */
        kend[a] = ((Gend[a] + B - 1) >> (S - 1 + F)) >> 1;       /* crossings with T <  the end */
    }
    int64_t i[3];
    for (int a = 0; a < 3; a++) {
        i[a] = cell0[a] + s[a] * k[a];
        if (C->periodic) i[a] = ((i[a] % n) + n) % n;           /* wrap into the box */
    }

    /* Per-ray REAL constants (IEEE operations in a fixed order). */
    const REAL nrm = (REAL)nrm_d;
    REAL h[3], V[3], inv2D[3], u[3];
    for (int a = 0; a < 3; a++) {
        h[a] = D[a] ? (REAL)(1 << (S - 1)) / (REAL)D[a] : (REAL)0;   /* 2^(S-1)/D_a   */
        V[a] = R_LDEXP(h[a], -(S - 1 + F));                          /* 2^-F/D_a      */
        inv2D[a] = R_LDEXP(h[a], -S);                                /* 1/(2 D_a)     */
        u[a] = R_LDEXP((REAL)D[a], -(S + 1));                        /* D_a/2^(S+1)   */
    }
    REAL W[3][3] = {{0}};                                            /* 2^(S-1)/(D_a D_b) */
    for (int a = 0; a < 3; a++)
        for (int b = a + 1; b < 3; b++)
            if (D[a] && D[b]) W[a][b] = W[b][a] = h[a] / (REAL)D[b];
    const REAL Lc = R_LDEXP(nrm * (REAL)ORC_SQRT_PI_3, -l);          /* L_pix per unit distance */
    const REAL G = (REAL)((ndot / 12.0) * C->sigma_over_dx2);       /* rate per unit budget per cell length */
    const double ph = ndot / 12.0;                                   /* photons/s per unit budget */

    const uint64_t rid = ((uint64_t)srcidx << 36) | ((uint64_t)l << 31) | (uint64_t)ray->pix;
    const uint64_t rbase = orc_mix64(rid);

    REAL P = ray->P, cP = ray->cP, tau = ray->tau, ctau = ray->ctau;
    REAL A = 0, cA = 0;                                              /* photons absorbed by this ray */

    st->rays[l]++;
    if (i[0] < 0 || i[0] >= n || i[1] < 0 || i[1] >= n || i[2] < 0 || i[2] >= n) {
        st->escaped[l]++;
        orc_sum_add(&C->escaped, ph * SFX(remaining)(C, P, cP, tau, ctau));
        return 0;
    }

    int prev = -1;            /* -1: previous event is the start sphere; else the axis last crossed */
    int64_t kprev = 0;        /* crossing index of that previous crossing */
    int64_t seq = 0;
    for (;;) {
        /* Next face crossing: smallest T_a, ties resolved x, y, z (Amanatides-Woo). */
        int w = 0;
        if (orc_t_less(k[1], D[1], k[w], D[w])) w = 1;
        if (orc_t_less(k[2], D[2], k[w], D[w])) w = 2;
        const int is_end = !(k[w] < kend[w]);                        /* split sphere comes first */

        /* Parametric length of this segment, from exact integer numerators. */
        REAL ds_p;
        if (!is_end) {
            if (prev < 0)
                ds_p = (REAL)((2 * k[w] + 1) * B - Gstart[w]) * V[w];
            else if (prev == w)
                ds_p = h[w] + h[w];
            else
                ds_p = (REAL)((2 * k[w] + 1) * D[prev] - (2 * kprev + 1) * D[w]) * W[prev][w];
        } else {
            if (prev < 0)
                ds_p = split_end ? R_LDEXP((REAL)C->rq, l > 0 ? l - 1 - F : -F)
                                 : R_LDEXP((REAL)(Rend - Rstart), -F);
            else
                ds_p = (REAL)(Gend[prev] - (2 * kprev + 1) * B) * V[prev];
        }
        const REAL ds = ds_p * nrm;                                  /* path length in cells */

        const int64_t cell = (i[2] * n + i[1]) * n + i[0];
        const REAL kraw = C->KAPPA_FIELD[cell];
        const REAL kap = R_FABS(kraw);
        const REAL dtau = kap * ds;                                  /* Eq. 2 over the segment */
        REAL a, gseg;
        if (C->spectrum) {                                           /* Eq. 1 integrated over frequency */
            const double t0 = (double)tau - (double)ctau;
            if (kap > 0) {
                a = (REAL)((double)P * orc_absorbed(C, t0, (double)dtau));
                gseg = (a * G) / kap;
            } else {
                a = 0;
                gseg = (REAL)((double)P * orc_thin_rate(C, t0)) * G * ds;
            }
        } else if (kap > 0) {
            a = P * (-R_EXPM1(-dtau));                               /* photons absorbed */
            gseg = (a * G) / kap;                                    /* Eq. 1, gray, V_box: a/(n_HI V) */
        } else {
            a = 0;
            gseg = (P * G) * ds;                                     /* optically thin limit */
        }

        /* Geometric overlap correction (Eqs. 5-8). */
        REAL f = 1, g2 = 0;
        int64_t nbcell = -1;
        if (C->overlap_mode != ORC_OVERLAP_NONE) {
            REAL dl[6];
            for (int b = 0; b < 3; b++) {
                REAL dn;
                if (!is_end) {
                    dn = (b == w) ? (REAL)0
                                  : (REAL)((2 * k[b] + 1) * D[w] - (2 * k[w] + 1) * D[b]) * inv2D[w];
                } else {
                    dn = R_LDEXP((REAL)((2 * k[b] + 1) * B - Gend[b]), -(S + F));
                }
                const REAL delta = dn + ds_p * u[b];                /* midpoint to exit face along b */
                const REAL other = (REAL)1 - delta;
                dl[2 * b] = s[b] > 0 ? other : delta;                /* lower face b- */
                dl[2 * b + 1] = s[b] > 0 ? delta : other;            /* upper face b+ */
            }
            int face = 0;
            REAL De = dl[0];
            for (int q = 1; q < 6; q++)
                if (dl[q] < De) { De = dl[q]; face = q; }
            const REAL tnext = is_end ? (split_end ? R_LDEXP((REAL)C->rq, l - F) : R_LDEXP((REAL)Rend, -F))
                                      : (REAL)(2 * k[w] + 1) * h[w];
            const REAL tm = tnext - ds_p * (REAL)0.5;
            const REAL Lpix = tm * Lc;                               /* pixel width at the midpoint */
            const int near_edge = (De + De) < Lpix;
            if (near_edge) {
                if (C->overlap_mode == ORC_OVERLAP_LINEAR) {
                    f = (REAL)0.5 + De / Lpix;
                } else if (C->overlap_mode == ORC_OVERLAP_SQUARED) {
                    f = (REAL)0.5 + De / Lpix;
                    f = f * f;
                } else {
                    /* naive threshold: the primary share applies whatever the neighbour */
                    if (C->overlap_mode == ORC_OVERLAP_NAIVE) f = (REAL)0.5 + De / Lpix;
                    int64_t j[3] = {i[0], i[1], i[2]};
                    j[face >> 1] += (face & 1) ? 1 : -1;
                    if (C->periodic) j[face >> 1] = ((j[face >> 1] % n) + n) % n;
                    if (j[0] >= 0 && j[0] < n && j[1] >= 0 && j[1] < n && j[2] >= 0 && j[2] < n) {
                        const int64_t c2 = (j[2] * n + j[1]) * n + j[0];
                        const REAL kn_raw = C->KAPPA_FIELD[c2];
                        const REAL kn = R_FABS(kn_raw);
                        const int elig = (C->overlap_mode == ORC_OVERLAP_CONSERVATIVE ||
                                          C->overlap_mode == ORC_OVERLAP_NAIVE)
                                             ? (!R_SIGNBIT(kn_raw) && kn > 0)   /* n'_H >= n_th (Eq. 7-8) */
                                             : (kn > 0);                          /* Eq. 5-6 */
                        if (elig) {
                            f = (REAL)0.5 + De / Lpix;
                            g2 = (((REAL)1 - f) * gseg) * (kap / kn);    /* Eq. 6 / Eq. 8 */
                            nbcell = c2;
                        }
                    }
                }
            }
        }
        C->gamma[cell] += (double)(f * gseg);
        if (nbcell >= 0) {
            C->gamma[nbcell] += (double)g2;
            st->secondary[l]++;
        }

        SFX(kahan_add)(&tau, &ctau, dtau);
        if (!C->spectrum) SFX(kahan_add)(&P, &cP, -a);
        SFX(kahan_add)(&A, &cA, a);

        st->segments[l]++;
        st->visit_hash += orc_mix64(rbase ^ ((uint64_t)seq << 40) ^ (uint64_t)cell);
        if (C->rec_n < C->rec_cap) {
            C->rec_ray[C->rec_n] = (int64_t)rid;
            C->rec_seq[C->rec_n] = (int32_t)seq;
            C->rec_cell[C->rec_n] = cell;
            C->rec_ds[C->rec_n] = (double)ds;
        }
        C->rec_n++;
        seq++;

        if (tau >= (REAL)C->tau_max) {                               /* photons spent (RAY_FLTR tau test) */
            st->dropped_tau[l]++;
            orc_sum_add(&C->dropped, ph * SFX(remaining)(C, P, cP, tau, ctau));
            orc_sum_add(&C->absorbed, ph * ((double)A - (double)cA));
            return 0;
        }
        if (is_end && !split_end) {                                  /* travelled sqrt(3) L_box (Sec. 2.5.1) */
            st->escaped[l]++;
            orc_sum_add(&C->escaped, ph * SFX(remaining)(C, P, cP, tau, ctau));
            orc_sum_add(&C->absorbed, ph * ((double)A - (double)cA));
            return 0;
        }
        if (is_end) {                                                /* reached the split sphere (Eq. 4) */
            orc_sum_add(&C->absorbed, ph * ((double)A - (double)cA));
            if (l + 1 > C->level_max) {
                st->dropped_level[l]++;
                orc_sum_add(&C->dropped, ph * SFX(remaining)(C, P, cP, tau, ctau));
                return 0;
            }
            st->splits[l]++;
            for (int q = 0; q < 4; q++) {                            /* S_COPY: HEALPix children 4p+q */
                kids[q].level = l + 1;
                kids[q].pix = 4 * ray->pix + q;
                kids[q].P = P * (REAL)0.25;
                kids[q].cP = cP * (REAL)0.25;
                kids[q].tau = tau;
                kids[q].ctau = ctau;
            }
            return 1;
        }

        /* Step every axis whose crossing coincides with the winner's. */
        const int64_t kw = k[w];
        int tie[3];
        for (int b = 0; b < 3; b++)
            tie[b] = (b == w) || ((2 * k[b] + 1) * D[w] == (2 * kw + 1) * D[b]);
        for (int b = 0; b < 3; b++)
            if (tie[b]) {
                k[b]++;
                i[b] += s[b];
                if (C->periodic) i[b] = ((i[b] % n) + n) % n;
            }
        prev = w;
        kprev = kw;
        if (i[0] < 0 || i[0] >= n || i[1] < 0 || i[1] >= n || i[2] < 0 || i[2] >= n) {
            st->escaped[l]++;
            orc_sum_add(&C->escaped, ph * SFX(remaining)(C, P, cP, tau, ctau));
            orc_sum_add(&C->absorbed, ph * ((double)A - (double)cA));
            return 0;
        }
    }
}

/* Alg. 2: spawn 12 level-0 rays per source, then march/filter/split until no
 * rays remain.  Depth-first per source (the order only changes the FP64
 * summation order of deposits). */
static void SFX(trace_all)(orc_ctx* C, const int32_t* cells, const double* ndot, int64_t nsrc)
{
    SFX(ray) stack[ORC_STACK];
    for (int64_t j = 0; j < nsrc; j++) {
        int top = 0;
        for (int p = 11; p >= 0; p--) {
            stack[top].level = 0;
            stack[top].pix = p;
            stack[top].P = (REAL)1;
            stack[top].cP = 0;
            stack[top].tau = 0;
            stack[top].ctau = 0;
            top++;
        }
        orc_sum_add(&C->emitted, ndot[j]);
        while (top > 0) {
            SFX(ray) r = stack[--top];
            SFX(ray) kids[4];
            if (SFX(march)(C, j, &cells[3 * j], ndot[j], &r, kids)) {
                for (int q = 3; q >= 0; q--) stack[top++] = kids[q];
            }
        }
    }
}
