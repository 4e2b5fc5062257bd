/*
 * gDPM CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 implementation of the coupled
 * photon/electron Monte Carlo dose calculation of Jia et al. (gDPM v2.0,
 * arXiv:1107.3355), written to be checked by eye against the method's
 * definitions.  It shares no code with the CUDA path.  Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline and reference legs
 * may load it.
 *
 * What the paper fixes, and where:
 *   - Sec. 2.1: Woodcock tracking for photons; condensed history for
 *     electrons with discrete ("hard") inelastic and bremsstrahlung events
 *     above cutoffs, continuous slowing down (CSDA) below them, long
 *     multiple-scattering steps that may cross voxel boundaries; positrons
 *     transported as electrons with two annihilation photons at track end.
 *   - Sec. 2.2.1: N_b equal batches; per-voxel mean dose and uncertainty
 *     from the batch spread.
 *   - Sec. 2.2.2: cross sections read from tables by linear interpolation.
 *   - Sec. 2.3.1: beamlet sampling from the cumulative fluence P(I), and
 *     the Metropolis chain of Algorithm A1; Walker's alias method is a
 *     third sampler of the same distribution f_I.
 *   - Sec. 2.3.2: the spectrum split into equal energy intervals, histories
 *     of a batch allotted to intervals by spectrum weight, energy uniform
 *     inside an interval.
 *   - Sec. 4 (physics variants): with ORC_SAUTER the photoelectron leaves at an
 *     angle from Sauter's K-shell distribution instead of along the photon.
 *   - Sec. 3.1: absorption energies (electron 200 keV, photon 50 keV);
 *     sigma/Dmax over D > 0.5 Dmax.
 * The paper defers every physics formula to DPM and states none.  The
 * formulas below are readings of the named closed forms (Klein-Nishina,
 * Z^4/E^3 photoelectric, Bethe-Heitler-shaped pair, Bethe stopping power,
 * Moller, Kramers-type 1/k bremsstrahlung, screened Rutherford angular
 * distribution with Rossi-Greisen scattering power), each marked READING.
 *
 * Pins (tests/test_oracle_pins.py, test_oracle_beamlets.py,
 * test_oracle_variants.py, test_oracle_paper_values.py): each function is
 * checked against closed forms, invariants, exact probabilities or
 * brute-force histograms, and the batch precision against the values the
 * paper prints (Table 1).  Parity unpinned: agreement of the dose itself with
 * DPM's physics data, which is not available; the formulas here are readings.
 * The test entries at the end of the file (orc_sample, orc_first_interaction,
 * orc_rotate, ...) call the transport's own functions, so a pin on a sampler
 * or on the Woodcock flight tests the code that makes the dose.
 *
 * Units: MeV, cm, g/cm3; per-unit-density quantities in cm2/g or MeV cm2/g.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- constants */
#define MC2 0.51099895             /* electron rest energy, MeV (CODATA 2018) */
#define RE 2.8179403262e-13        /* classical electron radius, cm */
#define ALPHA (1.0 / 137.035999084)
#define NAVO 6.02214076e23
#define ES_MS 21.2                 /* Rossi-Greisen scattering energy, MeV */
/* READING: photoelectric constant, cm2 MeV3, set so that water's mu_pe
 * equals its Compton mu at 30 keV (the paper gives no value). */
#define C_PE 3.9365358876e-32
#define MAJ_INFLATE (1.0 + 1e-6)   /* READING: Woodcock majorant margin */
#define PI 3.14159265358979323846

#define ORC_MAX_MAT 8
#define ORC_MAX_EL 16
#define ORC_MAX_BINS 256

enum { ORC_SAMPLE_CDF = 0, ORC_SAMPLE_ALIAS = 1, ORC_SAMPLE_METROPOLIS = 2 };

#define ORC_SAUTER 8               /* photoelectron direction from Sauter's distribution */
#define ORC_NO_ANNIHILATION 1
#define ORC_COMPTON_ONLY 2
#define ORC_NO_HARD 4

enum { PT_PHOTON = 0, PT_ELECTRON = 1, PT_POSITRON = 2 };
enum { GEO_PENCIL = 0, GEO_POINT_FIELD = 1, GEO_BEAMLETS = 2 };

typedef struct {
    int n_el;
    int Z[ORC_MAX_EL];
    double A[ORC_MAX_EL];
    double w[ORC_MAX_EL];
    double I;                      /* mean excitation energy, MeV */
} orc_material;

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    const uint8_t *mat;
    const float *rho;
    int n_mat;
    orc_material mats[ORC_MAX_MAT];
    double e_min, e_max;
    int n_energy;
    double eabs_ph, eabs_el;       /* absorption energies; also W_cb, W_cc */
    double ms_loss;                /* fraction of T lost by CSDA in one MS step */
    int particle, geometry;
    double origin[3], direction[3], center[3], axis_u[3], axis_v[3];
    double half_u, half_v;
    int n_bins;
    double edges[ORC_MAX_BINS + 1];
    double weights[ORC_MAX_BINS];
    int n_beamlets;
    const double *beamlets;        /* rows of 17: src3 centre3 au3 av3 u0 u1 v0 v1 w */
    unsigned long long n_hist;
    int n_batches;
    unsigned long long seed;
    unsigned int request_id;
    int flags;
    int beamlet_sampler;           /* ORC_SAMPLE_* */
    int metro_chains;              /* Metropolis chains C (Algorithm A1) */
    unsigned long long first_hist; /* id of the problem's first history (the
                                      histories are first_hist .. first_hist+n_hist-1) */
} orc_problem;

typedef struct {
    double source_energy, deposited, escaped, discarded;
    long long n_primary;
    long long ph_created, ph_terminated, ph_flights, ph_real, compton, photoelectric, pair;
    long long el_created, el_terminated, el_steps, moller, brems, annihilations;
    long long local_deposits;
    double dmax, sigma_over_dmax;
} orc_result;

/* per-history record (optional output) */
enum { HR_PH_REAL = 0, HR_EL_STEPS = 1, HR_HARD = 2, HR_BANKED = 3, HR_NI = 4 };
enum { HD_ESCAPED = 0, HD_EL_MASSPATH = 1, HD_ND = 2 };

/* ------------------------------------------------------------- Philox RNG
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
 * 32x32->64 multiplies; key bumped by the Weyl constants between rounds.
 * READING (keying): key = (seed_lo, seed_hi ^ request_id); counter =
 * (history id, particle id lo, particle id hi, draw index). */
static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* SplitMix64 output function (Steele, Lea, Flood 2014). READING: the id of
 * the k-th banked secondary of particle p is splitmix64(p ^ (k+1)*golden). */
#define GOLDEN64 0x9E3779B97F4A7C15ull
static uint64_t splitmix64(uint64_t state)
{
    uint64_t z = state + GOLDEN64;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static uint64_t child_id(uint64_t parent, uint32_t k)
{
    return splitmix64(parent ^ ((uint64_t)(k + 1) * GOLDEN64));
}

/* ---------------------------------------------------------------- particles */
typedef struct {
    double x[3], u[3], E;
    int iv[3];                     /* voxel indices (tracked exactly for electrons) */
    int type;
    uint32_t hist;
    uint64_t pid;
    uint32_t ctr;                  /* next Philox draw index */
    uint32_t nchild;               /* secondaries banked so far */
} orc_particle;

/* ------------------------------------------------------------------- tables */
typedef struct {
    int n_mat, n;
    double lemin, dle;             /* ln E grid: ln E_i = lemin + i*dle */
    double *E;
    double *mu_c, *mu_pe, *mu_pair;     /* [m*n+i], cm2/g */
    double *scol, *srest, *sig_m, *sig_b, *range;
    double *mumax;                 /* [i], cm^-1, majorant for this phantom */
    double x0[ORC_MAX_MAT], sigmax[ORC_MAX_MAT], bconst[ORC_MAX_MAT], r_eabs[ORC_MAX_MAT];
    double ne[ORC_MAX_MAT];
} orc_tables;

typedef struct {
    const orc_problem *P;
    orc_tables T;
    uint32_t key[2];
    double *edep;                  /* batch energy grid, MeV */
    orc_result *res;
    int *hrec; double *hrecd;      /* per-history records or NULL */
    uint64_t cur_hist;
    uint64_t hrec_base;            /* history id of record row 0 */
    orc_particle *stack; size_t sp, scap;
    int flags;
    /* beamlet sampling (Sec. 2.3.1) over the nf beamlets of positive weight */
    int nf;
    int *bl_index;                 /* [nf] row of the k-th positive-weight beamlet */
    double *bl_f;                  /* [nf] its weight f */
    double *al_prob; int *al_alias;/* [nf] Walker alias table */
    int *ch_state;                 /* [C] current beamlet of each Metropolis chain */
    uint64_t *ch_next;             /* [C] next step index of each chain */
} orc_sim;

/* per-unit-mass number densities */
static double mat_ne(const orc_material *m)
{
    double s = 0;
    for (int i = 0; i < m->n_el; i++) s += m->w[i] * m->Z[i] / m->A[i];
    return NAVO * s;
}
static double mat_ni(const orc_material *m, int i) { return NAVO * m->w[i] / m->A[i]; }

/* Klein-Nishina total cross section per electron, cm2 (closed form). */
static double sigma_kn(double E)
{
    double k = E / MC2;
    double l = log(1.0 + 2.0 * k);
    return 2.0 * PI * RE * RE *
           ((1.0 + k) / (k * k) * (2.0 * (1.0 + k) / (1.0 + 2.0 * k) - l / k) +
            l / (2.0 * k) - (1.0 + 3.0 * k) / ((1.0 + 2.0 * k) * (1.0 + 2.0 * k)));
}
static double mu_compton(const orc_material *m, double E) { return mat_ne(m) * sigma_kn(E); }

/* READING: photoelectric mu/rho = C_PE * sum_i n_i Z_i^4 / E^3. */
static double mu_photo(const orc_material *m, double E)
{
    double s = 0;
    for (int i = 0; i < m->n_el; i++) {
        double z = m->Z[i];
        s += mat_ni(m, i) * z * z * z * z;
    }
    return C_PE * s / (E * E * E);
}

/* READING: pair mu/rho = sum_i n_i alpha re^2 Z(Z+1) [28/9 ln(183 Z^-1/3) - 2/27]
 * ((k-2)/k)^3 for k = E/mc2 > 2 (complete-screening asymptote, cubic threshold). */
static double mu_pair(const orc_material *m, double E)
{
    double k = E / MC2;
    if (k <= 2.0) return 0.0;
    double th = (k - 2.0) / k;
    double s = 0;
    for (int i = 0; i < m->n_el; i++) {
        double z = m->Z[i];
        s += mat_ni(m, i) * z * (z + 1.0) * (28.0 / 9.0 * log(183.0 * pow(z, -1.0 / 3.0)) - 2.0 / 27.0);
    }
    return ALPHA * RE * RE * s * th * th * th;
}

/* READING: bremsstrahlung constant B (cm2/g) with dSigma_b/dk = B/k on
 * (0, T]; the same B is 1/X0 (Rossi's radiation-length approximation). */
static double brems_const(const orc_material *m)
{
    double s = 0;
    for (int i = 0; i < m->n_el; i++) {
        double z = m->Z[i];
        s += mat_ni(m, i) * z * (z + 1.0) * log(183.0 * pow(z, -1.0 / 3.0));
    }
    return 4.0 * ALPHA * RE * RE * s;
}

/* Bethe collision stopping power (ICRU-37 form for electrons), no density
 * effect (READING), MeV cm2/g. */
static double s_col(const orc_material *m, double T)
{
    double tau = T / MC2;
    double b2 = tau * (tau + 2.0) / ((tau + 1.0) * (tau + 1.0));
    double ir = m->I / MC2;
    double F = 1.0 - b2 + (tau * tau / 8.0 - (2.0 * tau + 1.0) * log(2.0)) / ((tau + 1.0) * (tau + 1.0));
    double L = log(tau * tau * (tau + 2.0) / (2.0 * ir * ir)) + F;
    return 2.0 * PI * RE * RE * MC2 * mat_ne(m) / b2 * L;
}

/* Moller differential cross section per unit mass, dSigma/dW (cm2/g/MeV). */
static double moller_dsdw(const orc_material *m, double T, double W)
{
    double tau = T / MC2;
    double b2 = tau * (tau + 2.0) / ((tau + 1.0) * (tau + 1.0));
    double g = tau / (tau + 1.0);
    double c2 = (2.0 * tau + 1.0) / ((tau + 1.0) * (tau + 1.0));
    double V = T - W;
    return 2.0 * PI * RE * RE * MC2 * mat_ne(m) / b2 *
           (1.0 / (W * W) + 1.0 / (V * V) + g * g / (T * T) - c2 / (W * V));
}

/* adaptive Simpson quadrature */
typedef double (*orc_fn)(const void *ctx, double x);
static double simpson_rec(orc_fn f, const void *c, double a, double b, double fa, double fm,
                          double fb, double whole, double tol, int depth)
{
    double m = 0.5 * (a + b), lm = 0.5 * (a + m), rm = 0.5 * (m + b);
    double flm = f(c, lm), frm = f(c, rm);
    double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
    double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
    double d = left + right - whole;
    if (depth <= 0 || fabs(d) <= 15.0 * tol) return left + right + d / 15.0;
    return simpson_rec(f, c, a, m, fa, flm, fm, left, 0.5 * tol, depth - 1) +
           simpson_rec(f, c, m, b, fm, frm, fb, right, 0.5 * tol, depth - 1);
}
static double integrate_n(orc_fn f, const void *c, double a, double b, double rtol, int np)
{
    if (a == b) return 0.0;
    /* split into np panels so the initial estimate is meaningful */
    double s = 0.0, h = (b - a) / np;
    double est = 0.0;
    for (int i = 0; i < np; i++) {
        double x0 = a + i * h, x1 = x0 + h;
        double f0 = f(c, x0), f1 = f(c, x1), fm = f(c, 0.5 * (x0 + x1));
        est += fabs(h / 6.0 * (f0 + 4.0 * fm + f1));
    }
    for (int i = 0; i < np; i++) {
        double x0 = a + i * h, x1 = (i == np - 1) ? b : x0 + h;
        double f0 = f(c, x0), f1 = f(c, x1), fm = f(c, 0.5 * (x0 + x1));
        double whole = (x1 - x0) / 6.0 * (f0 + 4.0 * fm + f1);
        s += simpson_rec(f, c, x0, x1, f0, fm, f1, whole, rtol * est / np, 40);
    }
    return s;
}
static double integrate(orc_fn f, const void *c, double a, double b, double rtol)
{
    return integrate_n(f, c, a, b, rtol, 16);
}

typedef struct { const orc_material *m; double T; double wcc, wcb; } mctx;
static double f_moller_sig(const void *c, double W)
{
    const mctx *q = (const mctx *)c;
    return moller_dsdw(q->m, q->T, W);
}
static double f_moller_loss(const void *c, double W)
{
    const mctx *q = (const mctx *)c;
    return W * moller_dsdw(q->m, q->T, W);
}
/* hard Moller macroscopic cross section (cm2/g): W in [W_cc, T/2] */
static double sig_moller(const orc_material *m, double T, double wcc)
{
    if (T <= 2.0 * wcc) return 0.0;
    mctx q = {m, T, wcc, 0};
    return integrate(f_moller_sig, &q, wcc, 0.5 * T, 1e-11);
}
/* energy lost to hard Moller events per unit mass path (MeV cm2/g) */
static double loss_moller(const orc_material *m, double T, double wcc)
{
    if (T <= 2.0 * wcc) return 0.0;
    mctx q = {m, T, wcc, 0};
    return integrate(f_moller_loss, &q, wcc, 0.5 * T, 1e-11);
}
/* restricted total stopping power: soft collisions + soft radiation (k < W_cb) */
static double s_restricted(const orc_material *m, double T, double wcc, double wcb)
{
    double srad = brems_const(m) * (T < wcb ? T : wcb);
    return s_col(m, T) - loss_moller(m, T, wcc) + srad;
}
static double sig_brems(const orc_material *m, double T, double wcb)
{
    return T > wcb ? brems_const(m) * log(T / wcb) : 0.0;
}
static double f_inv_srest(const void *c, double T)
{
    const mctx *q = (const mctx *)c;
    return 1.0 / s_restricted(q->m, T, q->wcc, q->wcb);
}
/* CSDA range from the electron absorption energy, g/cm2 (negative below it) */
static double range_exact(const orc_material *m, double T, double eabs, double wcc, double wcb)
{
    mctx q = {m, 0, wcc, wcb};
    return integrate(f_inv_srest, &q, eabs, T, 1e-11);
}

/* Screened Rutherford: <1-mu> = 2A[(1+A) ln(1+1/A) - 1]; solve for A by
 * bisection in ln A.  G1 >= 1 means isotropic and is handled by the caller. */
static double g1_of_A(double A) { return 2.0 * A * ((1.0 + A) * log1p(1.0 / A) - 1.0); }
static double solve_A(double G1)
{
    double lo = log(1e-30), hi = log(1e12);
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (g1_of_A(exp(mid)) < G1) lo = mid; else hi = mid;
    }
    return exp(0.5 * (lo + hi));
}

/* Build the per-material tables on the log-uniform grid (Sec. 2.2.2:
 * tabulate, then interpolate linearly). */
static void tables_build(const orc_problem *P, orc_tables *T)
{
    int n = P->n_energy, M = P->n_mat;
    T->n = n; T->n_mat = M;
    T->lemin = log(P->e_min);
    T->dle = (log(P->e_max) - log(P->e_min)) / (n - 1);
    T->E = (double *)malloc(sizeof(double) * n);
    size_t mn = (size_t)M * n;
    T->mu_c = calloc(mn, sizeof(double)); T->mu_pe = calloc(mn, sizeof(double));
    T->mu_pair = calloc(mn, sizeof(double)); T->scol = calloc(mn, sizeof(double));
    T->srest = calloc(mn, sizeof(double)); T->sig_m = calloc(mn, sizeof(double));
    T->sig_b = calloc(mn, sizeof(double)); T->range = calloc(mn, sizeof(double));
    T->mumax = calloc(n, sizeof(double));
    for (int i = 0; i < n; i++) T->E[i] = exp(T->lemin + i * T->dle);
    int compton_only = (P->flags & ORC_COMPTON_ONLY) != 0;
    for (int m = 0; m < M; m++) {
        const orc_material *mt = &P->mats[m];
        T->ne[m] = mat_ne(mt);
        T->bconst[m] = brems_const(mt);
        T->x0[m] = 1.0 / T->bconst[m];
        double smax = 0.0;
        for (int i = 0; i < n; i++) {
            double E = T->E[i];
            size_t k = (size_t)m * n + i;
            T->mu_c[k] = mu_compton(mt, E);
            T->mu_pe[k] = compton_only ? 0.0 : mu_photo(mt, E);
            T->mu_pair[k] = compton_only ? 0.0 : mu_pair(mt, E);
            T->scol[k] = s_col(mt, E);
            T->srest[k] = s_restricted(mt, E, P->eabs_el, P->eabs_ph);
            T->sig_m[k] = sig_moller(mt, E, P->eabs_el);
            T->sig_b[k] = sig_brems(mt, E, P->eabs_ph);
            double sh = T->sig_m[k] + T->sig_b[k];
            if (sh > smax) smax = sh;
        }
        T->sigmax[m] = smax;
        /* CSDA range R(E_i) = int_{E_abs}^{E_i} dT/S_r, accumulated interval
         * by interval over the grid, then shifted so that R(E_abs) = 0 */
        mctx q = {mt, 0, P->eabs_el, P->eabs_ph};
        double *R = T->range + (size_t)m * n;
        R[0] = 0.0;
        for (int i = 1; i < n; i++)
            R[i] = R[i - 1] + integrate_n(f_inv_srest, &q, T->E[i - 1], T->E[i], 1e-12, 2);
        double c_eabs = integrate(f_inv_srest, &q, T->E[0], P->eabs_el, 1e-12);
        for (int i = 0; i < n; i++) R[i] -= c_eabs;
    }
    /* Woodcock majorant over the materials present, at their largest density */
    double rmax[ORC_MAX_MAT];
    for (int m = 0; m < M; m++) rmax[m] = 0.0;
    size_t V = (size_t)P->nx * P->ny * P->nz;
    for (size_t v = 0; v < V; v++) {
        int m = P->mat[v];
        if (P->rho[v] > rmax[m]) rmax[m] = P->rho[v];
    }
    for (int i = 0; i < n; i++) {
        double mx = 0.0;
        for (int m = 0; m < M; m++) {
            size_t k = (size_t)m * n + i;
            double mu = (T->mu_c[k] + T->mu_pe[k] + T->mu_pair[k]) * rmax[m];
            if (mu > mx) mx = mu;
        }
        T->mumax[i] = MAJ_INFLATE * mx;
    }
}

static void tables_free(orc_tables *T)
{
    free(T->E); free(T->mu_c); free(T->mu_pe); free(T->mu_pair); free(T->scol);
    free(T->srest); free(T->sig_m); free(T->sig_b); free(T->range); free(T->mumax);
}

/* position on the grid: linear interpolation in ln E (Sec. 2.2.2) */
static void grid_pos(const orc_tables *T, double E, int *i, double *f)
{
    double u = (log(E) - T->lemin) / T->dle;
    int k = (int)floor(u);
    if (k < 0) k = 0;
    if (k > T->n - 2) k = T->n - 2;
    double ff = u - k;
    if (ff < 0.0) ff = 0.0;
    if (ff > 1.0) ff = 1.0;
    *i = k; *f = ff;
}
static double lerp_tab(const double *t, int i, double f) { return t[i] + f * (t[i + 1] - t[i]); }
static double tab_at(const orc_tables *T, const double *tab, int m, double E)
{
    int i; double f;
    grid_pos(T, E, &i, &f);
    return lerp_tab(tab + (size_t)m * T->n, i, f);
}
/* inverse of the interpolated range: the T with R_interp(T) = r */
static double range_inverse(const orc_tables *T, int m, double r)
{
    const double *R = T->range + (size_t)m * T->n;
    int lo = 0, hi = T->n - 1;
    if (r <= R[0]) return T->E[0];
    if (r >= R[hi]) return T->E[hi];
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (R[mid] <= r) lo = mid; else hi = mid;
    }
    double f = (r - R[lo]) / (R[lo + 1] - R[lo]);
    return exp(T->lemin + (lo + f) * T->dle);
}

/* ---------------------------------------------------------------- geometry */
static void draw4(orc_sim *S, orc_particle *p, double u[4])
{
    uint32_t c[4] = {p->hist, (uint32_t)p->pid, (uint32_t)(p->pid >> 32), p->ctr};
    uint32_t o[4];
    philox4x32_10(c, S->key, o);
    p->ctr++;
    for (int k = 0; k < 4; k++) u[k] = ((double)o[k] + 0.5) * (1.0 / 4294967296.0);
}

static int inside(const orc_problem *P, const double x[3])
{
    return x[0] >= 0.0 && x[0] <= P->nx * P->dx && x[1] >= 0.0 && x[1] <= P->ny * P->dy &&
           x[2] >= 0.0 && x[2] <= P->nz * P->dz;
}
static void voxel_of(const orc_problem *P, const double x[3], int iv[3])
{
    int n[3] = {P->nx, P->ny, P->nz};
    double d[3] = {P->dx, P->dy, P->dz};
    for (int a = 0; a < 3; a++) {
        int k = (int)floor(x[a] / d[a]);
        if (k < 0) k = 0;
        if (k > n[a] - 1) k = n[a] - 1;
        iv[a] = k;
    }
}
static size_t vidx(const orc_problem *P, const int iv[3])
{
    return (size_t)iv[0] + (size_t)P->nx * ((size_t)iv[1] + (size_t)P->ny * iv[2]);
}

/* Rotate direction u by polar cosine cost and azimuth phi.  Convention
 * (READING, shared by every implementation of this model): the azimuth is
 * measured from e1 = (u_x u_z, u_y u_z, -(1-u_z^2))/s with e2 = (-u_y, u_x, 0)/s,
 * s = sqrt(1-u_z^2); for s^2 < 1e-10 take e1 = x-axis, e2 = y-axis. */
static void rotate(double u[3], double cost, double phi)
{
    double sint = sqrt(fmax(0.0, 1.0 - cost * cost));
    double e1[3], e2[3];
    double s2 = 1.0 - u[2] * u[2];
    if (s2 < 1e-10) {
        e1[0] = 1; e1[1] = 0; e1[2] = 0;
        e2[0] = 0; e2[1] = 1; e2[2] = 0;
    } else {
        double s = sqrt(s2);
        e1[0] = u[0] * u[2] / s; e1[1] = u[1] * u[2] / s; e1[2] = -s;
        e2[0] = -u[1] / s; e2[1] = u[0] / s; e2[2] = 0.0;
    }
    double cp = cos(phi), sp = sin(phi);
    double n[3];
    for (int a = 0; a < 3; a++) n[a] = cost * u[a] + sint * (cp * e1[a] + sp * e2[a]);
    double l = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int a = 0; a < 3; a++) u[a] = n[a] / l;
}

/* READING (physics variant): Sauter's K-shell photoelectron distribution in
 * mu = cos(theta) for a photoelectron of kinetic energy T (binding energy
 * neglected, as for the photoelectric product above), gamma = 1 + T/mc2,
 * beta = sqrt(1 - 1/gamma^2):
 *   p(mu) ~ (1 - mu^2) / (1 - beta mu)^4 * [1 + b (1 - beta mu)],
 *   b = gamma (gamma - 1) (gamma - 2) / 2.
 * Sampling: propose mu from q(mu) ~ 1/(1 - beta mu)^2 on [-1, 1] by inverting
 * its distribution, 1/(1 - beta mu) = 1/(1 + beta) + xi 2 beta/(1 - beta^2),
 * and accept with (1 - mu^2)(1 - beta^2)/(1 - beta mu)^2 * g(mu)/g_max, where
 * g = 1 + b (1 - beta mu) and g_max its largest value on [-1, 1] (both
 * factors are at most 1).  Draws per trial: (proposal, accept, phi, -). */
static void sample_sauter(orc_sim *S, orc_particle *p, double T, double *mu, double *phi)
{
    double g = 1.0 + T / MC2;
    double beta = sqrt(fmax(0.0, 1.0 - 1.0 / (g * g)));
    double b = 0.5 * g * (g - 1.0) * (g - 2.0);
    double gmax = b >= 0 ? 1.0 + b * (1.0 + beta) : 1.0 + b * (1.0 - beta);
    double c[4];
    *mu = 0.0;
    *phi = 0.0;
    for (int it = 0; it < 4096; it++) {
        draw4(S, p, c);
        double x = 1.0 / (1.0 + beta) + c[0] * 2.0 * beta / (1.0 - beta * beta);
        double m = (1.0 - 1.0 / x) / beta;
        if (m > 1.0) m = 1.0;
        if (m < -1.0) m = -1.0;
        double d = 1.0 - beta * m;
        double w = (1.0 - m * m) * (1.0 - beta * beta) / (d * d) * (1.0 + b * d) / gmax;
        *mu = m;
        *phi = 2.0 * PI * c[2];
        if (c[1] < w) break;
    }
}

/* Move a primary from outside onto the phantom surface.  Returns 0 if the
 * ray misses.  The entry coordinate is set exactly on the face. */
static int enter_box(const orc_problem *P, double x[3], const double u[3])
{
    if (inside(P, x)) return 1;
    double L[3] = {P->nx * P->dx, P->ny * P->dy, P->nz * P->dz};
    double tmin = -INFINITY, tmax = INFINITY;
    int amin = -1;
    for (int a = 0; a < 3; a++) {
        if (u[a] == 0.0) {
            if (x[a] < 0.0 || x[a] > L[a]) return 0;
            continue;
        }
        double t1 = (0.0 - x[a]) / u[a], t2 = (L[a] - x[a]) / u[a];
        double lo = fmin(t1, t2), hi = fmax(t1, t2);
        if (lo > tmin) { tmin = lo; amin = a; }
        if (hi < tmax) tmax = hi;
    }
    if (amin < 0 || tmax <= tmin || tmax <= 0.0) return 0;
    for (int a = 0; a < 3; a++) x[a] += tmin * u[a];
    x[amin] = (u[amin] > 0.0) ? 0.0 : L[amin];
    for (int a = 0; a < 3; a++) x[a] = fmin(fmax(x[a], 0.0), L[a]);
    return 1;
}

/* ---------------------------------------------------------------- tallies */
static void deposit(orc_sim *S, const int iv[3], double e)
{
    if (e == 0.0) return;
    S->edep[vidx(S->P, iv)] += e;
}

static void push(orc_sim *S, const orc_particle *p)
{
    if (S->sp == S->scap) {
        S->scap = S->scap ? 2 * S->scap : 1024;
        S->stack = (orc_particle *)realloc(S->stack, S->scap * sizeof(orc_particle));
    }
    S->stack[S->sp++] = *p;
}

/* Bank a secondary (Sec. 2.2.1: secondaries go to the stacks).  Electrons
 * below the absorption energy are deposited on the spot; positrons are
 * always banked (their annihilation is handled at track end). */
static void bank(orc_sim *S, orc_particle *parent, int type, double E, const double x[3],
                 const double u[3], const int iv[3])
{
    if (type == PT_ELECTRON && E < S->P->eabs_el) {
        deposit(S, iv, E);
        S->res->local_deposits++;
        return;
    }
    if (type == PT_PHOTON && E < S->P->eabs_ph) {
        deposit(S, iv, E);
        S->res->local_deposits++;
        return;
    }
    orc_particle c;
    memset(&c, 0, sizeof c);
    for (int a = 0; a < 3; a++) { c.x[a] = x[a]; c.u[a] = u[a]; c.iv[a] = iv[a]; }
    c.E = E; c.type = type; c.hist = parent->hist;
    c.pid = child_id(parent->pid, parent->nchild);
    parent->nchild++;
    c.ctr = 0; c.nchild = 0;
    if (type == PT_PHOTON) S->res->ph_created++; else S->res->el_created++;
    if (S->hrec) S->hrec[(S->cur_hist - S->hrec_base) * HR_NI + HR_BANKED]++;
    push(S, &c);
}

/* ---------------------------------------------------------------- samplers
 * One function per interaction sampler, called by the transport and by
 * orc_sample (which the sampler pins test), so that the pins reach the code
 * that makes the dose. */

/* Klein-Nishina in eps = E'/E by the two-branch mixture method (1/eps and
 * eps branches, rejection on 1 - eps sin^2/(1+eps^2)).  Returns eps, the
 * photon's polar cosine 1 - t, and the fourth uniform of the accepted draw
 * (the caller's azimuth). */
static double kn_sample(orc_sim *S, orc_particle *p, double E, double *cost, double *c3)
{
    double k = E / MC2;
    double e0 = 1.0 / (1.0 + 2.0 * k);
    double a1 = log(1.0 + 2.0 * k), a2 = 0.5 * (1.0 - e0 * e0);
    double eps, t, c[4];
    for (;;) {
        draw4(S, p, c);
        if (c[0] * (a1 + a2) < a1) eps = exp(-a1 * c[1]);
        else eps = sqrt(e0 * e0 + (1.0 - e0 * e0) * c[1]);
        t = (1.0 - eps) / (k * eps);
        double sin2 = t * (2.0 - t);
        double g = 1.0 - eps * sin2 / (1.0 + eps * eps);
        if (c[2] <= g) break;
    }
    *cost = 1.0 - t;
    *c3 = c[3];
    return eps;
}

/* Moller energy fraction eps = W/T on [W_cc/T, 1/2]: proposal 1/eps^2,
 * rejection on the rest of the Moller density.  Also returns the third
 * uniform of the accepted draw (the caller's azimuth). */
static double moller_sample(orc_sim *S, orc_particle *p, double Tn, double wcc, double *w2)
{
    double tau = Tn / MC2;
    double c1 = (tau / (tau + 1.0)) * (tau / (tau + 1.0));
    double c2 = (2.0 * tau + 1.0) / ((tau + 1.0) * (tau + 1.0));
    double ec = wcc / Tn, eps, w[4];
    for (;;) {
        draw4(S, p, w);
        eps = ec / (1.0 - w[0] * (1.0 - 2.0 * ec));
        double x = eps / (1.0 - eps);
        double g = 1.0 + x * x + c1 * eps * eps - c2 * x;
        if (w[1] * (2.0 + 0.25 * c1) <= g) break;
    }
    *w2 = w[2];
    return eps;
}

/* Polar cosine of an electron of kinetic energy W leaving a binary
 * collision of an electron of kinetic energy T (energy and momentum
 * conservation, target at rest). */
static double binary_cos(double T, double W)
{
    return sqrt(W * (T + 2.0 * MC2) / (T * (W + 2.0 * MC2)));
}

/* Hard bremsstrahlung photon energy on [W_cb, T] for dSigma/dk = B/k:
 * k = W_cb (T/W_cb)^xi. */
static double brems_k(double Tn, double wcb, double xi)
{
    return wcb * pow(Tn / wcb, xi);
}

/* Screened Rutherford p(mu) ~ (1 - mu + 2A)^-2 by inversion of its
 * cumulative distribution at the uniform u. */
static double sr_mu(double A, double u)
{
    return 1.0 - 2.0 * A * u / (1.0 - u + A);
}

/* ---------------------------------------------------------------- photons */
static void compton(orc_sim *S, orc_particle *p, int *alive)
{
    double E = p->E, cost, c3;
    double eps = kn_sample(S, p, E, &cost, &c3);
    double phi = 2.0 * PI * c3;
    double Ep = eps * E, Te = E - Ep;
    double uold[3] = {p->u[0], p->u[1], p->u[2]};
    rotate(p->u, cost, phi);
    double de[3], l = 0;
    for (int a = 0; a < 3; a++) { de[a] = E * uold[a] - Ep * p->u[a]; l += de[a] * de[a]; }
    l = sqrt(l);
    for (int a = 0; a < 3; a++) de[a] /= l;
    S->res->compton++;
    bank(S, p, PT_ELECTRON, Te, p->x, de, p->iv);
    if (Ep < S->P->eabs_ph) {
        deposit(S, p->iv, Ep);
        S->res->local_deposits++;
        S->res->ph_terminated++;
        *alive = 0;
    } else {
        p->E = Ep;
    }
}

/* One Woodcock flight against the majorant mu_max(E) (Sec. 2.2.1 photon
 * transport): fly -ln(u0)/mu_max; if still inside, the collision is real
 * with probability mu(E, m) rho / mu_max (u1), and then Compton,
 * photoelectric or pair by the partial coefficients (u2).  Returns 0 when
 * the photon left the phantom, 1 for a virtual collision, 2 for a real one
 * with *type 0 Compton, 1 photoelectric, 2 pair. */
static int woodcock_flight(orc_sim *S, orc_particle *p, const double u[4], int *type)
{
    const orc_problem *P = S->P;
    const orc_tables *T = &S->T;
    int n = T->n;
    int i; double f;
    grid_pos(T, p->E, &i, &f);
    double mumax = lerp_tab(T->mumax, i, f);
    double s = -log(u[0]) / mumax;
    for (int a = 0; a < 3; a++) p->x[a] += s * p->u[a];
    if (!inside(P, p->x)) return 0;
    voxel_of(P, p->x, p->iv);
    size_t v = vidx(P, p->iv);
    int m = P->mat[v];
    double rho = P->rho[v];
    double muc = lerp_tab(T->mu_c + (size_t)m * n, i, f);
    double mupe = lerp_tab(T->mu_pe + (size_t)m * n, i, f);
    double mupp = lerp_tab(T->mu_pair + (size_t)m * n, i, f);
    double mut = muc + mupe + mupp;
    if (u[1] * mumax >= mut * rho) return 1;     /* virtual (delta) collision */
    double r = u[2] * mut;
    *type = r < muc ? 0 : (r < muc + mupe ? 1 : 2);
    return 2;
}

/* Photoelectric absorption (READING): the photoelectron takes the photon's
 * whole energy (no binding), along the photon or, with ORC_SAUTER, at an
 * angle from Sauter's K-shell distribution. */
static void photoelectric_event(orc_sim *S, orc_particle *p)
{
    double d[3] = {p->u[0], p->u[1], p->u[2]};
    if (S->P->flags & ORC_SAUTER) {
        double mu, phi;
        sample_sauter(S, p, p->E, &mu, &phi);
        rotate(d, mu, phi);
    }
    bank(S, p, PT_ELECTRON, p->E, p->x, d, p->iv);
}

/* Pair production by a photon of energy E > 2 m c^2 (READING): the electron
 * takes the share xi of E - 2 m c^2, the positron the rest, both along the
 * photon. */
static void pair_event(orc_sim *S, orc_particle *p, double xi)
{
    double tav = p->E - 2.0 * MC2;
    double t1 = xi * tav, t2 = tav - t1;
    bank(S, p, PT_ELECTRON, t1, p->x, p->u, p->iv);
    bank(S, p, PT_POSITRON, t2, p->x, p->u, p->iv);
}

static void photon_track(orc_sim *S, orc_particle *p)
{
    const orc_problem *P = S->P;
    if (p->E < P->eabs_ph) {           /* never transported */
        if (inside(P, p->x)) { voxel_of(P, p->x, p->iv); deposit(S, p->iv, p->E); }
        else S->res->escaped += p->E;
        S->res->ph_terminated++;
        return;
    }
    int alive = 1;
    while (alive) {
        double u[4];
        draw4(S, p, u);
        int type = 0;
        int fl = woodcock_flight(S, p, u, &type);
        if (fl == 0) {
            S->res->escaped += p->E;
            S->res->ph_terminated++;
            return;
        }
        S->res->ph_flights++;
        if (fl == 1) continue;
        S->res->ph_real++;
        if (S->hrec) S->hrec[(S->cur_hist - S->hrec_base) * HR_NI + HR_PH_REAL]++;
        if (type == 0) {
            compton(S, p, &alive);
        } else if (type == 1) {
            S->res->photoelectric++;
            photoelectric_event(S, p);
            S->res->ph_terminated++;
            alive = 0;
        } else {
            S->res->pair++;
            pair_event(S, p, u[3]);     /* rest mass accounted at the positron's end */
            S->res->ph_terminated++;
            alive = 0;
        }
    }
}

/* ---------------------------------------------------------------- electrons */
/* Walk a straight segment of mass thickness `mass` (g/cm2) through the voxel
 * grid (3-D DDA), depositing `dpm` MeV per g/cm2 in each voxel crossed.  If
 * `defer_last`, the final piece is not deposited (the caller puts the step's
 * remainder there).  Returns 1 if the particle left the phantom. */
static int walk(orc_sim *S, orc_particle *p, double mass, double dpm, double *dep_sum,
                int defer_last)
{
    const orc_problem *P = S->P;
    int n[3] = {P->nx, P->ny, P->nz};
    double d[3] = {P->dx, P->dy, P->dz};
    double left = mass;
    while (left > 0.0) {
        double tb = INFINITY;
        int ab = -1;
        for (int a = 0; a < 3; a++) {
            double t;
            if (p->u[a] > 0.0) t = ((p->iv[a] + 1) * d[a] - p->x[a]) / p->u[a];
            else if (p->u[a] < 0.0) t = (p->iv[a] * d[a] - p->x[a]) / p->u[a];
            else continue;
            if (t < tb) { tb = t; ab = a; }
        }
        if (tb < 0.0) tb = 0.0;
        double rho = P->rho[vidx(P, p->iv)];
        if (rho * tb >= left) {
            double t = left / rho;
            for (int a = 0; a < 3; a++) p->x[a] += t * p->u[a];
            if (!defer_last) { deposit(S, p->iv, dpm * left); *dep_sum += dpm * left; }
            left = 0.0;
            break;
        }
        for (int a = 0; a < 3; a++) p->x[a] += tb * p->u[a];
        double piece = rho * tb;
        if (piece > 0.0) { deposit(S, p->iv, dpm * piece); *dep_sum += dpm * piece; }
        left -= piece;
        p->iv[ab] += (p->u[ab] > 0.0) ? 1 : -1;
        if (p->iv[ab] < 0 || p->iv[ab] >= n[ab]) return 1;
    }
    return 0;
}

static void annihilate(orc_sim *S, orc_particle *p)
{
    if (S->P->flags & ORC_NO_ANNIHILATION) {
        S->res->discarded += 2.0 * MC2;
        return;
    }
    double a[4];
    draw4(S, p, a);
    double cost = 2.0 * a[0] - 1.0, phi = 2.0 * PI * a[1];
    double sint = sqrt(fmax(0.0, 1.0 - cost * cost));
    double d1[3] = {sint * cos(phi), sint * sin(phi), cost};
    double d2[3] = {-d1[0], -d1[1], -d1[2]};
    S->res->annihilations++;
    bank(S, p, PT_PHOTON, MC2, p->x, d1, p->iv);
    bank(S, p, PT_PHOTON, MC2, p->x, d2, p->iv);
}

static void electron_absorb(orc_sim *S, orc_particle *p)
{
    deposit(S, p->iv, p->E);
    S->res->el_terminated++;
    if (p->type == PT_POSITRON) annihilate(S, p);
}

static void electron_escape(orc_sim *S, orc_particle *p, double energy)
{
    S->res->escaped += energy;
    if (S->hrec) S->hrecd[(S->cur_hist - S->hrec_base) * HD_ND + HD_ESCAPED] += energy;
    if (p->type == PT_POSITRON) {
        if (S->P->flags & ORC_NO_ANNIHILATION) S->res->discarded += 2.0 * MC2;
        else {
            S->res->escaped += 2.0 * MC2;
            if (S->hrec) S->hrecd[(S->cur_hist - S->hrec_base) * HD_ND + HD_ESCAPED] += 2.0 * MC2;
        }
    }
    S->res->el_terminated++;
}

enum { EV_CUT = 0, EV_HARD = 1, EV_MS = 2 };

/* Hard Moller collision of an electron of kinetic energy Tn (Sec. 2.1 hard
 * inelastic event above W_cc): eps = W/Tn from moller_sample; the delta ray
 * (energy W) is banked at the binary-collision cosine and azimuth ph, and
 * the primary (energy Tn - W) turns by its own binary cosine at ph + pi, so
 * that momentum is conserved. */
static void moller_event(orc_sim *S, orc_particle *p, double Tn, double wcc)
{
    double w2;
    double eps = moller_sample(S, p, Tn, wcc, &w2);
    double ph = 2.0 * PI * w2;
    double W = eps * Tn, Tp = Tn - W;
    double cd = binary_cos(Tn, W);
    double cp = binary_cos(Tn, Tp);
    double ud[3] = {p->u[0], p->u[1], p->u[2]};
    rotate(ud, cd, ph);
    bank(S, p, PT_ELECTRON, W, p->x, ud, p->iv);
    rotate(p->u, cp, ph + PI);
    p->E = Tp;
}

/* Hard bremsstrahlung of an electron of kinetic energy Tn (READING): a
 * photon of energy k = W_cb (Tn/W_cb)^xi along the electron, which goes on
 * with Tn - k. */
static void brems_event(orc_sim *S, orc_particle *p, double Tn, double wcb, double xi)
{
    double kph = brems_k(Tn, wcb, xi);
    bank(S, p, PT_PHOTON, kph, p->x, p->u, p->iv);
    p->E = Tn - kph;
}

static void electron_track(orc_sim *S, orc_particle *p)
{
    const orc_problem *P = S->P;
    const orc_tables *T = &S->T;
    const double eabs = P->eabs_el, wcc = P->eabs_el, wcb = P->eabs_ph;
    const int nohard = (P->flags & ORC_NO_HARD) != 0;
    for (;;) {
        if (p->E < eabs) { electron_absorb(S, p); return; }
        double u[4];
        draw4(S, p, u);
        S->res->el_steps++;
        if (S->hrec) S->hrec[(S->cur_hist - S->hrec_base) * HR_NI + HR_EL_STEPS]++;
        int m = P->mat[vidx(P, p->iv)];
        double Tk = p->E;
        /* step limits, all as mass thickness in the start material */
        double R0 = tab_at(T, T->range, m, Tk);
        double x_cut = R0 - T->r_eabs[m];
        double x_ms = R0 - tab_at(T, T->range, m, (1.0 - P->ms_loss) * Tk);
        double x_hard = nohard ? INFINITY : -log(u[0]) / T->sigmax[m];
        int ev;
        double xs;
        if (x_cut <= x_ms && x_cut <= x_hard) { ev = EV_CUT; xs = x_cut; }
        else if (x_hard <= x_ms) { ev = EV_HARD; xs = x_hard; }
        else { ev = EV_MS; xs = x_ms; }
        if (xs < 0.0) xs = 0.0;
        double Tend = (ev == EV_CUT) ? eabs : range_inverse(T, m, R0 - xs);
        double dT = Tk - Tend;
        if (S->hrec) S->hrecd[(S->cur_hist - S->hrec_base) * HD_ND + HD_EL_MASSPATH] += xs;
        /* multiple scattering: screened Rutherford angle matched to the
         * Rossi-Greisen first moment G1 at the mid-step energy (READING) */
        double Tm = 0.5 * (Tk + Tend);
        double pbc = Tm * (Tm + 2.0 * MC2) / (Tm + MC2);
        double G1 = xs * (ES_MS / pbc) * (ES_MS / pbc) / (2.0 * T->x0[m]);
        double mu;
        if (G1 >= 1.0) mu = 2.0 * u[2] - 1.0;
        else {
            double A = solve_A(G1);
            mu = sr_mu(A, u[2]);
        }
        double phi = 2.0 * PI * u[3];
        double zeta = u[1];
        /* random hinge: straight zeta*xs, deflect, straight (1-zeta)*xs */
        double dpm = xs > 0.0 ? dT / xs : 0.0;
        double dep = 0.0;
        if (walk(S, p, zeta * xs, dpm, &dep, 0)) { electron_escape(S, p, Tk - dep); return; }
        rotate(p->u, mu, phi);
        if (walk(S, p, (1.0 - zeta) * xs, dpm, &dep, 1)) { electron_escape(S, p, Tk - dep); return; }
        deposit(S, p->iv, dT - dep);
        p->E = Tend;
        if (ev == EV_CUT) { electron_absorb(S, p); return; }
        if (ev != EV_HARD) continue;
        /* hard-event candidate: accept with Sigma_h(T)/Sigma_max */
        double v[4];
        draw4(S, p, v);
        double Tn = p->E;
        double sm = (Tn > 2.0 * wcc) ? tab_at(T, T->sig_m, m, Tn) : 0.0;
        double sb = (Tn > wcb) ? tab_at(T, T->sig_b, m, Tn) : 0.0;
        double sh = sm + sb;
        if (!(v[0] * T->sigmax[m] < sh)) continue;
        if (S->hrec) S->hrec[(S->cur_hist - S->hrec_base) * HR_NI + HR_HARD]++;
        if (v[1] * sh < sm) {
            S->res->moller++;
            moller_event(S, p, Tn, wcc);
        } else {
            S->res->brems++;
            brems_event(S, p, Tn, wcb, v[2]);
        }
    }
}

/* ---------------------------------------------------------------- sources */
/* Histories of a batch allotted to spectrum intervals by weight: floor plus
 * largest remainder, ties to the lower interval (Sec. 2.3.2). */
static void allot(const orc_problem *P, uint64_t nb, uint64_t *cnt)
{
    int K = P->n_bins;
    double wsum = 0;
    for (int j = 0; j < K; j++) wsum += P->weights[j];
    uint64_t given = 0;
    double rem[ORC_MAX_BINS];
    for (int j = 0; j < K; j++) {
        double q = (double)nb * (P->weights[j] / wsum);
        cnt[j] = (uint64_t)floor(q);
        rem[j] = q - floor(q);
        given += cnt[j];
    }
    while (given < nb) {
        int best = -1;
        for (int j = 0; j < K; j++)
            if (P->weights[j] > 0 && (best < 0 || rem[j] > rem[best])) best = j;
        cnt[best]++;
        rem[best] = -1.0;
        given++;
    }
}

/* ------------------------------------------------------- beamlet samplers
 * Sec. 2.3.1: the beamlet I of a particle is drawn with probability
 * f_I / sum f, over the beamlets of positive fluence only (the paper drops
 * zero-fluence beamlets first).  Three samplers of that distribution:
 *  - cumulative: the I with P(I) <= r < P(I+1), r the history's uniform;
 *  - Walker alias: a uniform index J and a uniform u; I = J when u is below
 *    J's cut-off, else J's alias.  Table built by Vose's procedure;
 *  - Metropolis (Algorithm A1): a chain of beamlet indices; each particle
 *    proposes a uniform J and moves the chain there with probability
 *    min(1, f_J / f_Iprev), else repeats Iprev.
 * READING (chains that do not depend on scheduling): C chains in place of
 * one per GPU thread.  History h is step floor(h / C) of chain h mod C, so
 * the seed alone fixes every history's beamlet.  Chain c starts at a
 * uniform index from the Philox block at counter (c, 0, 1, 0); the step of
 * history h uses the block at counter (h, 0, 0, 0).  (Particle ids 0 and
 * 2^32 are never given to a particle.)  Alias and Metropolis read two words
 * x0, x1 of the block: J = floor(x0 nf / 2^32), u = (x1 + 1/2) / 2^32.
 * The acceptance u < f_J / f_I is evaluated as u f_I < f_J in FP64. */
static void source_block(const orc_sim *S, uint32_t c0, uint32_t c2, uint32_t out[4])
{
    uint32_t c[4] = {c0, 0u, c2, 0u};
    philox4x32_10(c, S->key, out);
}

static int uniform_index(uint32_t x, int n)
{
    return (int)(((uint64_t)x * (uint64_t)n) >> 32);
}

static double word_uniform(uint32_t x)
{
    return ((double)x + 0.5) * (1.0 / 4294967296.0);
}

static void chain_start(orc_sim *S, int c)
{
    uint32_t w[4];
    source_block(S, (uint32_t)c, 1u, w);
    S->ch_state[c] = uniform_index(w[0], S->nf);
    S->ch_next[c] = 0;
}

static void samplers_init(orc_sim *S)
{
    const orc_problem *P = S->P;
    if (P->geometry != GEO_BEAMLETS || P->n_beamlets < 1) return;
    int n = 0;
    for (int b = 0; b < P->n_beamlets; b++)
        if (P->beamlets[b * 17 + 16] > 0) n++;
    S->nf = n;
    S->bl_index = malloc(sizeof(int) * n);
    S->bl_f = malloc(sizeof(double) * n);
    S->al_prob = malloc(sizeof(double) * n);
    S->al_alias = malloc(sizeof(int) * n);
    n = 0;
    for (int b = 0; b < P->n_beamlets; b++)
        if (P->beamlets[b * 17 + 16] > 0) {
            S->bl_index[n] = b;
            S->bl_f[n] = P->beamlets[b * 17 + 16];
            n++;
        }
    /* Vose: scaled weights q_k = f_k nf / sum f; repeatedly pair the last
     * "small" (q < 1) with the last "large" entry, which gives the small one
     * its cut-off and donates 1 - q_small of its own mass. */
    double sum = 0;
    for (int k = 0; k < n; k++) sum += S->bl_f[k];
    double scale = (double)n / sum;
    double *q = malloc(sizeof(double) * n);
    int *small = malloc(sizeof(int) * n), *large = malloc(sizeof(int) * n);
    int ns = 0, nl = 0;
    for (int k = 0; k < n; k++) {
        q[k] = S->bl_f[k] * scale;
        if (q[k] < 1.0) small[ns++] = k; else large[nl++] = k;
    }
    while (ns > 0 && nl > 0) {
        int l = small[--ns], g = large[--nl];
        S->al_prob[l] = q[l];
        S->al_alias[l] = g;
        q[g] = (q[g] + q[l]) - 1.0;
        if (q[g] < 1.0) small[ns++] = g; else large[nl++] = g;
    }
    while (nl > 0) { int g = large[--nl]; S->al_prob[g] = 1.0; S->al_alias[g] = g; }
    while (ns > 0) { int l = small[--ns]; S->al_prob[l] = 1.0; S->al_alias[l] = l; }
    free(q); free(small); free(large);
    if (P->beamlet_sampler == ORC_SAMPLE_METROPOLIS) {
        int C = P->metro_chains;
        S->ch_state = malloc(sizeof(int) * C);
        S->ch_next = malloc(sizeof(uint64_t) * C);
        for (int c = 0; c < C; c++) chain_start(S, c);
    }
}

static void samplers_free(orc_sim *S)
{
    free(S->bl_index); free(S->bl_f); free(S->al_prob); free(S->al_alias);
    free(S->ch_state); free(S->ch_next);
    S->bl_index = S->al_alias = S->ch_state = NULL;
    S->bl_f = S->al_prob = NULL;
    S->ch_next = NULL;
}

/* Beamlet (position k in the positive-weight list) of history h; r is the
 * history's own uniform, used by the cumulative sampler. */
static int pick_beamlet(orc_sim *S, uint32_t h, double r)
{
    const orc_problem *P = S->P;
    int nf = S->nf;
    uint32_t w[4];
    if (P->beamlet_sampler == ORC_SAMPLE_ALIAS) {
        source_block(S, h, 0u, w);
        int J = uniform_index(w[0], nf);
        return word_uniform(w[1]) < S->al_prob[J] ? J : S->al_alias[J];
    }
    if (P->beamlet_sampler == ORC_SAMPLE_METROPOLIS) {
        uint64_t C = (uint64_t)P->metro_chains;
        int c = (int)(h % C);
        uint64_t step = h / C;
        if (S->ch_next[c] > step) chain_start(S, c);
        while (S->ch_next[c] <= step) {
            uint32_t hs = (uint32_t)((uint64_t)c + S->ch_next[c] * C);
            source_block(S, hs, 0u, w);
            int J = uniform_index(w[0], nf);
            int I = S->ch_state[c];
            if (word_uniform(w[1]) * S->bl_f[I] < S->bl_f[J]) S->ch_state[c] = J;
            S->ch_next[c]++;
        }
        return S->ch_state[c];
    }
    /* cumulative P(I), summed over all beamlets as given */
    double tot = 0;
    for (int b = 0; b < P->n_beamlets; b++) tot += P->beamlets[b * 17 + 16];
    double x = r * tot, acc = 0;
    for (int k = 0; k < nf; k++) {
        acc += S->bl_f[k];
        if (x < acc) return k;
    }
    return nf - 1;
}

static void make_primary(orc_sim *S, uint32_t h, double elo, double ehi, orc_particle *p)
{
    const orc_problem *P = S->P;
    memset(p, 0, sizeof *p);
    p->hist = h; p->pid = 1; p->ctr = 0; p->nchild = 0;
    p->type = P->particle == 0 ? PT_PHOTON : PT_ELECTRON;
    double u[4];
    draw4(S, p, u);
    p->E = elo + (ehi - elo) * u[2];
    if (P->geometry == GEO_PENCIL) {
        double l = 0;
        for (int a = 0; a < 3; a++) { p->x[a] = P->origin[a]; l += P->direction[a] * P->direction[a]; }
        for (int a = 0; a < 3; a++) p->u[a] = P->direction[a] / sqrt(l);
    } else {
        const double *src, *cen, *au, *av;
        double a0, a1, b0, b1;
        if (P->geometry == GEO_POINT_FIELD) {
            src = P->origin; cen = P->center; au = P->axis_u; av = P->axis_v;
            a0 = -P->half_u; a1 = P->half_u; b0 = -P->half_v; b1 = P->half_v;
        } else {
            int I = S->bl_index[pick_beamlet(S, h, u[3])];
            const double *row = P->beamlets + (size_t)I * 17;
            src = row; cen = row + 3; au = row + 6; av = row + 9;
            a0 = row[12]; a1 = row[13]; b0 = row[14]; b1 = row[15];
        }
        double su = a0 + (a1 - a0) * u[0], sv = b0 + (b1 - b0) * u[1];
        double aim[3], l = 0;
        for (int a = 0; a < 3; a++) {
            aim[a] = cen[a] + su * au[a] + sv * av[a];
            p->x[a] = src[a];
            p->u[a] = aim[a] - src[a];
            l += p->u[a] * p->u[a];
        }
        l = sqrt(l);
        for (int a = 0; a < 3; a++) p->u[a] /= l;
    }
}

/* ---------------------------------------------------------------- driver */
static void run_history(orc_sim *S, orc_particle *prim)
{
    const orc_problem *P = S->P;
    S->res->n_primary++;
    S->res->source_energy += prim->E;
    if (prim->type == PT_PHOTON) S->res->ph_created++; else S->res->el_created++;
    if (!enter_box(P, prim->x, prim->u)) {
        S->res->escaped += prim->E;
        if (S->hrec) S->hrecd[(S->cur_hist - S->hrec_base) * HD_ND + HD_ESCAPED] += prim->E;
        if (prim->type == PT_PHOTON) S->res->ph_terminated++; else S->res->el_terminated++;
        return;
    }
    voxel_of(P, prim->x, prim->iv);
    S->sp = 0;
    push(S, prim);
    while (S->sp > 0) {
        orc_particle p = S->stack[--S->sp];
        if (p.type == PT_PHOTON) {
            double esc0 = S->res->escaped;
            photon_track(S, &p);
            if (S->hrec) S->hrecd[(S->cur_hist - S->hrec_base) * HD_ND + HD_ESCAPED] += S->res->escaped - esc0;
        } else {
            electron_track(S, &p);
        }
    }
}

static int sim_init(orc_sim *S, const orc_problem *P, orc_result *res)
{
    memset(S, 0, sizeof *S);
    S->P = P;
    S->res = res;
    memset(res, 0, sizeof *res);
    tables_build(P, &S->T);
    for (int m = 0; m < P->n_mat; m++)
        S->T.r_eabs[m] = tab_at(&S->T, S->T.range, m, P->eabs_el);
    S->key[0] = (uint32_t)P->seed;
    S->key[1] = (uint32_t)(P->seed >> 32) ^ P->request_id;
    samplers_init(S);
    return 0;
}

/* Full dose calculation: N_b batches (Sec. 2.2.1); returns mean dose and its
 * standard error per voxel in MeV/g per source history. */
int orc_run(const orc_problem *P, double *dose, double *sigma, orc_result *res,
            int *hist_rec, double *hist_recd)
{
    if (P->n_batches < 2 || P->n_hist < (unsigned long long)P->n_batches || P->n_mat < 1 ||
        P->n_mat > ORC_MAX_MAT || P->n_bins < 1 || P->n_bins > ORC_MAX_BINS)
        return -1;
    if (P->beamlet_sampler < ORC_SAMPLE_CDF || P->beamlet_sampler > ORC_SAMPLE_METROPOLIS ||
        (P->beamlet_sampler == ORC_SAMPLE_METROPOLIS && P->metro_chains < 1))
        return -1;
    if (P->first_hist + P->n_hist > (1ull << 32)) return -1;   /* history ids are 32-bit */
    orc_sim S;
    sim_init(&S, P, res);
    S.hrec = hist_rec; S.hrecd = hist_recd;
    S.hrec_base = P->first_hist;
    if (hist_rec) memset(hist_rec, 0, sizeof(int) * HR_NI * P->n_hist);
    if (hist_recd) memset(hist_recd, 0, sizeof(double) * HD_ND * P->n_hist);
    size_t V = (size_t)P->nx * P->ny * P->nz;
    double *s1 = calloc(V, sizeof(double)), *s2 = calloc(V, sizeof(double));
    S.edep = calloc(V, sizeof(double));
    uint64_t cnt[ORC_MAX_BINS];
    uint64_t first = P->first_hist;
    int NB = P->n_batches;
    for (int b = 0; b < NB; b++) {
        uint64_t nb = P->n_hist / NB + ((uint64_t)b < P->n_hist % NB ? 1 : 0);
        memset(S.edep, 0, V * sizeof(double));
        allot(P, nb, cnt);
        uint64_t h = first;
        for (int j = 0; j < P->n_bins; j++) {
            for (uint64_t q = 0; q < cnt[j]; q++, h++) {
                orc_particle prim;
                S.cur_hist = h;
                make_primary(&S, (uint32_t)h, P->edges[j], P->edges[j + 1], &prim);
                run_history(&S, &prim);
            }
        }
        for (size_t v = 0; v < V; v++) {
            double x = S.edep[v] / (double)nb;
            s1[v] += x;
            s2[v] += x * x;
            res->deposited += S.edep[v];
        }
        first += nb;
    }
    double dV = P->dx * P->dy * P->dz;
    double dmax = 0;
    for (size_t v = 0; v < V; v++) {
        double mean = s1[v] / NB;
        double var = (s2[v] - NB * mean * mean) / ((double)NB * (NB - 1));
        if (var < 0) var = 0;
        double mass = P->rho[v] * dV;
        dose[v] = mean / mass;
        sigma[v] = sqrt(var) / mass;
        /* READING: the Sec. 3.1 precision metric over tissue-like voxels only
         * (rho >= 0.05 g/cm3); air voxels of tiny mass have meaningless noise */
        if (P->rho[v] >= 0.05f && dose[v] > dmax) dmax = dose[v];
    }
    double acc = 0; long long na = 0;
    for (size_t v = 0; v < V; v++)
        if (P->rho[v] >= 0.05f && dose[v] > 0.5 * dmax) { acc += sigma[v]; na++; }
    res->dmax = dmax;
    res->sigma_over_dmax = (na > 0 && dmax > 0) ? acc / na / dmax : 0.0;
    free(s1); free(s2); free(S.edep); free(S.stack);
    tables_free(&S.T);
    samplers_free(&S);
    return 0;
}

/* ======================================================================
 * Entry points used only by the oracle's own checks (pins).
 * ==================================================================== */

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    philox4x32_10(ctr, key, out);
}
uint64_t orc_child_id(uint64_t parent, uint32_t k) { return child_id(parent, k); }

/* Exact (non-tabulated) model functions for material m of the problem. */
enum {
    OF_SIGMA_KN = 0, OF_MU_C, OF_MU_PE, OF_MU_PAIR, OF_SCOL, OF_LOSS_MOLLER, OF_SIG_MOLLER,
    OF_SREST, OF_SIG_BREMS, OF_RANGE, OF_BCONST, OF_NE, OF_G1_OF_A, OF_SOLVE_A
};
double orc_eval(const orc_problem *P, int m, int fn, double x)
{
    const orc_material *mt = &P->mats[m];
    switch (fn) {
    case OF_SIGMA_KN: return sigma_kn(x);
    case OF_MU_C: return mu_compton(mt, x);
    case OF_MU_PE: return mu_photo(mt, x);
    case OF_MU_PAIR: return mu_pair(mt, x);
    case OF_SCOL: return s_col(mt, x);
    case OF_LOSS_MOLLER: return loss_moller(mt, x, P->eabs_el);
    case OF_SIG_MOLLER: return sig_moller(mt, x, P->eabs_el);
    case OF_SREST: return s_restricted(mt, x, P->eabs_el, P->eabs_ph);
    case OF_SIG_BREMS: return sig_brems(mt, x, P->eabs_ph);
    case OF_RANGE: return range_exact(mt, x, P->eabs_el, P->eabs_el, P->eabs_ph);
    case OF_BCONST: return brems_const(mt);
    case OF_NE: return mat_ne(mt);
    case OF_G1_OF_A: return g1_of_A(x);
    case OF_SOLVE_A: return solve_A(x);
    }
    return NAN;
}

/* Export the interpolation tables (for table checks).  Arrays sized
 * n_energy (E, mumax) or n_mat*n_energy; per-material scalars n_mat. */
int orc_tables_export(const orc_problem *P, double *E, double *mu_c, double *mu_pe,
                      double *mu_pair, double *scol, double *srest, double *sig_m,
                      double *sig_b, double *range, double *mumax, double *x0,
                      double *sigmax)
{
    orc_tables T;
    tables_build(P, &T);
    size_t n = T.n, mn = (size_t)T.n_mat * n;
    memcpy(E, T.E, n * sizeof(double));
    memcpy(mumax, T.mumax, n * sizeof(double));
    memcpy(mu_c, T.mu_c, mn * sizeof(double)); memcpy(mu_pe, T.mu_pe, mn * sizeof(double));
    memcpy(mu_pair, T.mu_pair, mn * sizeof(double)); memcpy(scol, T.scol, mn * sizeof(double));
    memcpy(srest, T.srest, mn * sizeof(double)); memcpy(sig_m, T.sig_m, mn * sizeof(double));
    memcpy(sig_b, T.sig_b, mn * sizeof(double)); memcpy(range, T.range, mn * sizeof(double));
    for (int m = 0; m < T.n_mat; m++) { x0[m] = T.x0[m]; sigmax[m] = T.sigmax[m]; }
    tables_free(&T);
    return 0;
}

/* Interpolated-table lookups as the transport uses them. */
enum { OT_MU_C = 0, OT_MU_PE, OT_MU_PAIR, OT_SIG_M, OT_SIG_B, OT_RANGE, OT_RANGE_INV, OT_MUMAX };
int orc_table_lookup(const orc_problem *P, int m, int which, const double *x, double *y, int n)
{
    orc_tables T;
    tables_build(P, &T);
    for (int i = 0; i < n; i++) {
        switch (which) {
        case OT_MU_C: y[i] = tab_at(&T, T.mu_c, m, x[i]); break;
        case OT_MU_PE: y[i] = tab_at(&T, T.mu_pe, m, x[i]); break;
        case OT_MU_PAIR: y[i] = tab_at(&T, T.mu_pair, m, x[i]); break;
        case OT_SIG_M: y[i] = tab_at(&T, T.sig_m, m, x[i]); break;
        case OT_SIG_B: y[i] = tab_at(&T, T.sig_b, m, x[i]); break;
        case OT_RANGE: y[i] = tab_at(&T, T.range, m, x[i]); break;
        case OT_RANGE_INV: y[i] = range_inverse(&T, m, x[i]); break;
        case OT_MUMAX: { int k; double f; grid_pos(&T, x[i], &k, &f); y[i] = lerp_tab(T.mumax, k, f); } break;
        }
    }
    tables_free(&T);
    return 0;
}

/* Draw n samples from one of the interaction samplers, each sample from its
 * own Philox stream (history = sample index, particle id 1). */
enum { OS_KN = 0, OS_MOLLER, OS_BREMS, OS_SR, OS_ISO, OS_SAUTER };
int orc_sample(int which, double a, double b, long long n, unsigned long long seed,
               double *out1, double *out2)
{
    orc_problem P;
    memset(&P, 0, sizeof P);
    P.eabs_el = b; P.eabs_ph = b;
    orc_sim S;
    memset(&S, 0, sizeof S);
    S.P = &P;
    orc_result res;
    memset(&res, 0, sizeof res);
    S.res = &res;
    S.key[0] = (uint32_t)seed; S.key[1] = (uint32_t)(seed >> 32);
    for (long long s = 0; s < n; s++) {
        orc_particle p;
        memset(&p, 0, sizeof p);
        p.hist = (uint32_t)s; p.pid = 1;
        if (which == OS_KN) {
            double cost, c3;
            out1[s] = kn_sample(&S, &p, a, &cost, &c3);
            out2[s] = cost;
        } else if (which == OS_MOLLER) {
            double w2;
            double eps = moller_sample(&S, &p, a, b, &w2);
            out1[s] = eps;
            if (out2) out2[s] = binary_cos(a, eps * a);
        } else if (which == OS_BREMS) {
            double v[4];
            draw4(&S, &p, v);
            out1[s] = brems_k(a, b, v[2]);
        } else if (which == OS_SAUTER) {
            double mu, phi;
            sample_sauter(&S, &p, a, &mu, &phi);
            out1[s] = mu;
            if (out2) out2[s] = phi;
        } else if (which == OS_SR) {
            double u[4];
            draw4(&S, &p, u);
            out1[s] = sr_mu(a, u[2]);
        } else {
            double u[4];
            draw4(&S, &p, u);
            out1[s] = 2.0 * u[0] - 1.0;
            if (out2) out2[s] = 2.0 * PI * u[1];
        }
    }
    return 0;
}

/* First real photon interaction of each primary (for the attenuation
 * check): out_z = depth of the interaction (-1 if the photon left),
 * out_type = 0 Compton, 1 photoelectric, 2 pair, -1 escaped. */
int orc_first_interaction(const orc_problem *P, long long n, double *out_z, int *out_type)
{
    orc_sim S;
    orc_result res;
    sim_init(&S, P, &res);
    for (long long h = 0; h < n; h++) {
        orc_particle p;
        make_primary(&S, (uint32_t)h, P->edges[0], P->edges[1], &p);
        out_z[h] = -1.0; out_type[h] = -1;
        if (!enter_box(P, p.x, p.u)) continue;
        for (;;) {
            double u[4];
            draw4(&S, &p, u);
            int type = 0;
            int fl = woodcock_flight(&S, &p, u, &type);
            if (fl == 0) break;
            if (fl == 1) continue;
            out_z[h] = p.x[2];
            out_type[h] = type;
            break;
        }
    }
    tables_free(&S.T);
    samplers_free(&S);
    return 0;
}

/* Spectrum allotment for one batch of nb histories (for its check). */
int orc_allot(const orc_problem *P, unsigned long long nb, unsigned long long *cnt)
{
    uint64_t c[ORC_MAX_BINS];
    allot(P, nb, c);
    for (int j = 0; j < P->n_bins; j++) cnt[j] = c[j];
    return 0;
}

/* One interaction event as the transport applies it (for the kinematics
 * checks): kind 0 a Compton collision of a photon of energy E, kind 1 a
 * hard Moller collision of an electron of kinetic energy E with cut `cut`,
 * kind 2 the annihilation of a positron at rest at the end of its track,
 * kind 3 pair production by a photon of energy E (its share from the
 * fourth uniform of one draw, as the flight supplies it), kind 4 the
 * photoelectric absorption of a photon of energy E (Sauter angles when
 * cut != 0), kind 5 a hard bremsstrahlung event of an electron of kinetic
 * energy E with cut W_cb = cut (its uniform the third of one draw, as the
 * hard-event candidate supplies it).
 * The particle moves along the unit vector u; sample s uses history s.
 * out[8 s ..]: the particle after the event (E, u), then the banked
 * secondary (E, u); for kinds 2 and 3 the two banked particles (for kind 3
 * the electron, then the positron).  Absorption energies
 * are set to zero, so every secondary is banked.  Returns 0, or -1 for a
 * bad kind. */
int orc_event(int kind, double E, const double u[3], double cut, unsigned long long seed,
              long long n, double *out)
{
    if (kind < 0 || kind > 5) return -1;
    orc_problem P;
    memset(&P, 0, sizeof P);
    P.nx = P.ny = P.nz = 1;
    if (kind == 4 && cut != 0.0) P.flags |= ORC_SAUTER;
    orc_sim S;
    memset(&S, 0, sizeof S);
    S.P = &P;
    orc_result res;
    memset(&res, 0, sizeof res);
    S.res = &res;
    S.key[0] = (uint32_t)seed; S.key[1] = (uint32_t)(seed >> 32);
    for (long long s = 0; s < n; s++) {
        orc_particle p;
        memset(&p, 0, sizeof p);
        p.hist = (uint32_t)s; p.pid = 1; p.E = E;
        p.type = (kind == 0 || kind == 3 || kind == 4) ? PT_PHOTON
               : (kind == 2 ? PT_POSITRON : PT_ELECTRON);
        for (int a = 0; a < 3; a++) p.u[a] = u[a];
        S.sp = 0;
        double *o = out + 8 * s;
        if (kind == 2 || kind == 3) {
            if (kind == 2) {
                annihilate(&S, &p);
            } else {
                double w[4];
                draw4(&S, &p, w);
                pair_event(&S, &p, w[3]);
            }
            for (int k = 0; k < 2; k++) {
                o[4 * k] = S.sp == 2 ? S.stack[k].E : -1.0;
                for (int a = 0; a < 3; a++) o[4 * k + 1 + a] = S.sp == 2 ? S.stack[k].u[a] : 0.0;
            }
            continue;
        }
        if (kind == 0) {
            int alive = 1;
            compton(&S, &p, &alive);
        } else if (kind == 1) {
            moller_event(&S, &p, E, cut);
        } else if (kind == 4) {
            photoelectric_event(&S, &p);
        } else {
            double v[4];
            draw4(&S, &p, v);
            brems_event(&S, &p, E, cut, v[2]);
        }
        o[0] = p.E;
        for (int a = 0; a < 3; a++) o[1 + a] = p.u[a];
        o[4] = S.sp ? S.stack[S.sp - 1].E : -1.0;
        for (int a = 0; a < 3; a++) o[5 + a] = S.sp ? S.stack[S.sp - 1].u[a] : 0.0;
    }
    free(S.stack);
    return 0;
}

/* Direction rotation as the transport applies it (for its check). */
void orc_rotate(const double u[3], double cost, double phi, double out[3])
{
    double v[3] = {u[0], u[1], u[2]};
    rotate(v, cost, phi);
    out[0] = v[0]; out[1] = v[1]; out[2] = v[2];
}

/* Primaries [first, first+n) of batch 0 of the problem (as the transport
 * makes them), after entering the phantom: out rows x y z u v w E entered. */
int orc_sources(const orc_problem *P, unsigned long long first, unsigned long long n, double *out)
{
    orc_sim S;
    orc_result res;
    sim_init(&S, P, &res);
    uint64_t nb0 = P->n_hist / P->n_batches + (P->n_hist % P->n_batches ? 1 : 0);
    uint64_t cnt[ORC_MAX_BINS];
    allot(P, nb0, cnt);
    for (uint64_t s = 0; s < n; s++) {
        uint64_t local = first + s, acc = 0;
        int j = 0;
        while (j < P->n_bins - 1 && local >= acc + cnt[j]) { acc += cnt[j]; j++; }
        orc_particle p;
        make_primary(&S, (uint32_t)local, P->edges[j], P->edges[j + 1], &p);
        int in = enter_box(P, p.x, p.u);
        double *o = out + 8 * s;
        for (int a = 0; a < 3; a++) { o[a] = p.x[a]; o[3 + a] = p.u[a]; }
        o[6] = p.E; o[7] = in ? 1.0 : 0.0;
    }
    tables_free(&S.T);
    samplers_free(&S);
    return 0;
}

/* The positive-weight beamlet list and its Walker alias table: index[k]
 * is the beamlet row of list entry k; returns nf. */
int orc_beamlet_tables(const orc_problem *P, int *index, double *prob, int *alias)
{
    orc_sim S;
    orc_result res;
    sim_init(&S, P, &res);
    int nf = S.nf;
    for (int k = 0; k < nf; k++) {
        index[k] = S.bl_index[k];
        prob[k] = S.al_prob[k];
        alias[k] = S.al_alias[k];
    }
    tables_free(&S.T);
    samplers_free(&S);
    return nf;
}

/* Beamlet rows picked for histories [first, first+n) by the problem's
 * sampler, histories taken in increasing order as the transport does. */
int orc_beamlet_picks(const orc_problem *P, unsigned long long first, unsigned long long n,
                      int *out)
{
    orc_sim S;
    orc_result res;
    sim_init(&S, P, &res);
    for (uint64_t s = 0; s < n; s++) {
        uint32_t h = (uint32_t)(first + s);
        orc_particle p;
        memset(&p, 0, sizeof p);
        p.hist = h; p.pid = 1; p.ctr = 0;
        double u[4];
        draw4(&S, &p, u);
        out[s] = S.bl_index[pick_beamlet(&S, h, u[3])];
    }
    tables_free(&S.T);
    samplers_free(&S);
    return 0;
}

/* Per-history records of histories [first, first+n) of the full problem
 * (same batch split and spectrum allotment as orc_run); dose discarded.
 * rec: n*HR_NI ints, recd: n*HD_ND doubles, indexed from `first`. */
int orc_history_records(const orc_problem *P, unsigned long long first, unsigned long long n,
                        int *rec, double *recd)
{
    orc_sim S;
    orc_result res;
    sim_init(&S, P, &res);
    size_t V = (size_t)P->nx * P->ny * P->nz;
    S.edep = calloc(V, sizeof(double));
    memset(rec, 0, sizeof(int) * HR_NI * n);
    memset(recd, 0, sizeof(double) * HD_ND * n);
    uint64_t cnt[ORC_MAX_BINS];
    int NB = P->n_batches;
    uint64_t bstart = 0;
    for (int b = 0; b < NB; b++) {
        uint64_t nb = P->n_hist / NB + ((uint64_t)b < P->n_hist % NB ? 1 : 0);
        uint64_t lo = first > bstart ? first : bstart;
        uint64_t hi = (first + n) < (bstart + nb) ? (first + n) : (bstart + nb);
        if (lo < hi) {
            allot(P, nb, cnt);
            for (uint64_t h = lo; h < hi; h++) {
                uint64_t local = h - bstart, acc = 0;
                int j = 0;
                while (j < P->n_bins - 1 && local >= acc + cnt[j]) { acc += cnt[j]; j++; }
                S.hrec = rec;
                S.hrecd = recd;
                S.hrec_base = first;
                S.cur_hist = h;
                orc_particle prim;
                make_primary(&S, (uint32_t)h, P->edges[j], P->edges[j + 1], &prim);
                run_history(&S, &prim);
            }
        }
        bstart += nb;
    }
    free(S.edep); free(S.stack);
    tables_free(&S.T);
    samplers_free(&S);
    return 0;
}
