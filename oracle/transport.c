/*
 * Oracle for the photoexcitation-rate transport: a plain, serial, obviously
 * correct CPU restatement of the method.  TEST INFRASTRUCTURE ONLY: this file
 * may be used by the tests, by the smoke check and by the benchmark's CPU
 * baseline leg, and by nothing on the product path.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * What it follows (van Baal & Jerkstrand, ExTraSS):
 *   - Sobolev optical depth, Eq. (tau_Sobolev), App. A.1; escape probability
 *     beta_S, Eq. (beta_Sobolev), App. A.1; a line is an interaction point only
 *     if tau > 1e-4 in the traversed cell (Sec. 2.3.2).
 *   - Ray path: straight segments to the next cell wall; on every step the
 *     photon frequency is updated to the comoving frame and the lines whose
 *     comoving resonance lies between the segment's start and end frequency
 *     are met in order (Sec. 2.3.2).  Snapshot mode, homologous v = r/t (Sec. 2).
 *   - Attenuation: the line removes N_phot (1 - e^-tau) photons; the
 *     photoexcitation estimator counts them divided by the stimulated-emission
 *     correction f_corr (Sec. 2.3.2); the ray continues while its remaining
 *     photon energy at the line is >= 1e-6 of its starting energy
 *     (Secs. 2.3, 2.3.2).
 *   - Viewing directions: 20 x 20 equal-angle (theta, phi) bins (Sec. 2);
 *     output on a 0.1 % logarithmic wavelength grid (Sec. 2.3).
 *   - Line emissivity A_ul dE_ul beta N_u, Eq. (thin_emissivity), App. A.1.
 *   - Photoionization on every path segment (Sec. 2.3.1): tau_PI,i =
 *     sigma_PI,i d n_i for every level whose threshold lies below the photon
 *     energy, sigma_PI from the hydrogenic form of Eq. (sigma_OTSPI); the
 *     segment absorbs N (1 - e^-tau), tau = sum_i tau_PI,i, shared among the
 *     levels in proportion to tau_PI,i; the excess photon energy over each
 *     threshold is heating; Gamma_PI,i = N_abs,i / (n_i V).
 * Readings where the paper is silent are documented with each function.
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC (no FMA contraction, so the
 * same source gives the same numbers on x86-64 and aarch64).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* cgs constants */
#define XO_C 2.99792458e10
#define XO_H 6.62607015e-27
#define XO_K 1.380649e-16
#define XO_E 4.80320471e-10
#define XO_ME 9.1093837015e-28
#define XO_PI 3.14159265358979323846
#define XO_LN2 0.69314718055994530942

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11, "Parallel random
 * numbers: as easy as 1, 2, 3").  Counter (c0..c3), key (k0,k1); ten rounds
 * of two 64x64->128 multiplications with the key bumped by the Weyl
 * constants between rounds. */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void xo_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x0, &hi0, &lo0);
        mulhilo64(M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform double in [0,1) from the top 53 bits of a 64-bit word. */
static double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* Draw e of packet p: four uniforms from counter (p, e, 0, 0), key (seed, 0). */
static void draw4(uint64_t seed, int64_t p, uint64_t e, double u[4]) {
    uint64_t ctr[4] = {(uint64_t)p, e, 0, 0}, key[2] = {seed, 0}, x[4];
    xo_philox4x64_10(ctr, key, x);
    for (int i = 0; i < 4; i++) u[i] = u01(x[i]);
}

/* ------------------------------------------------------------------ */
/* Eq. (tau_Sobolev): tau = A_ul/(8 pi) (g_u/g_l) lambda^3 n_l (1 - g_l n_u/(g_u n_l)) t.
 * A_ul from f_lu by the standard oscillator-strength relation
 * A_ul = 8 pi^2 e^2 / (m_e c lambda^2) (g_l/g_u) f_lu.  For n_l = 0 the bracket
 * is multiplied out (n_l - g_l n_u / g_u), which gives tau <= 0. */
double xo_einstein_A(double lambda_cm, double g_l, double g_u, double f_lu) {
    return 8.0 * XO_PI * XO_PI * XO_E * XO_E / (XO_ME * XO_C * lambda_cm * lambda_cm) * (g_l / g_u) * f_lu;
}

double xo_tau_sobolev(double A_ul, double g_l, double g_u, double lambda_cm,
                      double n_l, double n_u, double t) {
    double pre = A_ul / (8.0 * XO_PI) * (g_u / g_l) * lambda_cm * lambda_cm * lambda_cm;
    if (n_l > 0.0) return pre * n_l * (1.0 - g_l * n_u / (g_u * n_l)) * t;
    return pre * (-(g_l / g_u) * n_u) * t;
}

/* Eq. (beta_Sobolev): beta = (1 - e^-tau)/tau for tau > 0.  For tau <= 0
 * (empty lower level, population inversion) the escape probability is taken
 * as 1: nothing traps the line (the formula would grow like e^|tau|). */
double xo_beta_sobolev(double tau) {
    if (tau <= 0.0) return 1.0;
    return -expm1(-tau) / tau;
}

/* ------------------------------------------------------------------ */
typedef struct {
    int32_t nx, ny, nz;
    double v_max, t;
    const double *L_cell;      /* [ncell] erg/s, band emission (emission_mode 0) */
    double band_lo_A, band_hi_A;
    int32_t nlev, nline;
    const double *g;           /* [nlev] */
    const double *E_level;     /* [nlev] erg */
    const double *pops;        /* [ncell*nlev] cm^-3 */
    const int32_t *lo, *up;    /* [nline] */
    const double *lambda_A, *f_lu; /* [nline] */
    const double *ne, *Te;     /* [ncell] */
    const double *ups_down;    /* [nlev] sum over j<u of Upsilon_ju (SCATTER only) */
    /* spherical grid: nx, ny, nz cells in r, theta, phi between the edges
     * (velocities in cm/s, angles in radians; first theta 0, last pi; first
     * phi 0, last 2 pi); geometry 0: the Cartesian cube */
    int32_t geometry;
    const double *r_edges, *th_edges, *ph_edges;
    /* photoionizing levels (Sec. 2.3.1); n_pi = 0: none */
    int32_t n_pi;
    const int32_t *pi_level;   /* [n_pi] global level index */
    const double *pi_Eion;     /* [n_pi] erg, ionization energy of the level's ion (from its ground) */
    const int32_t *pi_charge;  /* [n_pi] charge of the level's ion */
} xo_problem;

typedef struct {
    int64_t n_packets, p_begin, p_end;
    uint64_t seed;
    int32_t mode;              /* 0 attenuation (paper), 1 scatter / fluorescence */
    int32_t emission_mode;     /* 0 flat-in-nu band with L_cell, 1 line emissivity */
    double tau_min, e_cut;
    int32_t n_theta, n_phi;
    double spec_lam0_A, spec_dlog;
    int32_t spec_nbins;
    int64_t max_events;
    int32_t sampler;           /* 0 Monte Carlo packets, 1 rays per (cell, bin, viewer) */
} xo_params;

enum { L_EMIT_N, L_ESC_N, L_ABS_N, L_DROP_N, L_EMIT_E, L_ESC_E, L_OOB_E, L_EVENTS,
       L_TESTS, L_GUARD, L_THERMAL_E, L_INTERACT, L_ABS_E_CMF, L_REEMIT_E_CMF,
       L_PI_N, L_PI_E, L_NLEDGER };

typedef struct {
    const xo_problem *pb;
    const xo_params *pr;
    int64_t ncell;
    double R, dx, dy, dz, ct;
    int32_t *order;      /* sorted position -> original line index */
    int32_t *pos;        /* original line index -> sorted position */
    double *nu;          /* [nline] sorted, descending */
    double *A;           /* [nline] original order */
    double *Lc;          /* [ncell] cell luminosity */
    int64_t *qoff;       /* [ncell+1] packet quota prefix */
    double *wline;       /* [ncell*nline] line emission weights (emission_mode 1) */
    int32_t *down_off, *down_line;   /* CSR over upper levels of radiative down-lines */
    double *pi_tau;      /* [n_pi] work space of one photoionization segment */
    /* spherical grid: shell radii (cm), cos theta of the polar edges (flag of an
     * equatorial edge, crossed as the plane z = 0), cos and sin of the
     * azimuthal edges (edge nz is edge 0), cell volumes */
    double *sR, *cth, *cph, *sph, *vol;
    int32_t *eq;
    /* RAYS sampler: emitting cells, emitting bins, viewing directions */
    int64_t n_rcell;
    int64_t *rcell;      /* natural indices of the cells with L_c > 0 */
    int32_t n_rbin;
    double *rbin_nu;     /* comoving start frequency of each emitting bin */
    int32_t *rbin_cursor;/* first line its rays test */
    double *rbin_frac;   /* band emission: the bin's share of the band */
    int32_t *rbin_off, *rbin_line;   /* line emission: lines of each bin (CSR, ascending index) */
    double *view_n;      /* [n_theta n_phi][3] direction of each viewer's centre */
    double *view_w;      /* [n_theta n_phi] dOmega_k / 4 pi */
} prep_t;

static const double *g_sort_nu;
static int cmp_desc(const void *a, const void *b) {
    int32_t i = *(const int32_t *)a, j = *(const int32_t *)b;
    if (g_sort_nu[i] > g_sort_nu[j]) return -1;
    if (g_sort_nu[i] < g_sort_nu[j]) return 1;
    return (i < j) ? -1 : (i > j);
}

/* Largest-remainder integer quota: N L_c / sum(L) rounded down, the remaining
 * packets to the largest fractional parts (ties to the lower cell index). */
typedef struct { double frac; int64_t c; } rem_t;
static int cmp_rem(const void *a, const void *b) {
    const rem_t *x = a, *y = b;
    if (x->frac > y->frac) return -1;
    if (x->frac < y->frac) return 1;
    return (x->c < y->c) ? -1 : (x->c > y->c);
}

void xo_packet_quota(const double *L, int64_t ncell, int64_t N, int64_t *qoff) {
    double tot = 0.0;
    for (int64_t c = 0; c < ncell; c++) tot += L[c];
    rem_t *r = malloc(sizeof(rem_t) * (size_t)(ncell > 0 ? ncell : 1));
    int64_t *n = calloc((size_t)(ncell > 0 ? ncell : 1), sizeof(int64_t));
    int64_t used = 0;
    for (int64_t c = 0; c < ncell; c++) {
        double q = (tot > 0.0) ? ((double)N * L[c]) / tot : 0.0;
        double fl = floor(q);
        n[c] = (int64_t)fl;
        used += n[c];
        r[c].frac = q - fl;
        r[c].c = c;
    }
    qsort(r, (size_t)ncell, sizeof(rem_t), cmp_rem);
    for (int64_t k = 0; k < N - used && k < ncell; k++) n[r[k].c] += 1;
    qoff[0] = 0;
    for (int64_t c = 0; c < ncell; c++) qoff[c + 1] = qoff[c] + n[c];
    free(r); free(n);
}

static int prep(prep_t *P, const xo_problem *pb, const xo_params *pr) {
    memset(P, 0, sizeof(*P));
    P->pb = pb; P->pr = pr;
    P->ncell = (int64_t)pb->nx * pb->ny * pb->nz;
    P->R = pb->v_max * pb->t;
    P->dx = 2.0 * P->R / pb->nx; P->dy = 2.0 * P->R / pb->ny; P->dz = 2.0 * P->R / pb->nz;
    P->ct = XO_C * pb->t;
    int32_t nl = pb->nline;
    double *nu_orig = malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1));
    P->order = malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
    P->pos = malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
    P->nu = malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1));
    P->A = malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1));
    for (int32_t l = 0; l < nl; l++) {
        double lam = pb->lambda_A[l] * 1e-8;
        nu_orig[l] = XO_C / lam;
        P->order[l] = l;
        P->A[l] = xo_einstein_A(lam, pb->g[pb->lo[l]], pb->g[pb->up[l]], pb->f_lu[l]);
    }
    g_sort_nu = nu_orig;
    qsort(P->order, (size_t)nl, sizeof(int32_t), cmp_desc);
    for (int32_t k = 0; k < nl; k++) { P->pos[P->order[k]] = k; P->nu[k] = nu_orig[P->order[k]]; }
    free(nu_orig);
    /* radiative down-lines of every upper level, ascending original index */
    P->down_off = calloc((size_t)pb->nlev + 1, sizeof(int32_t));
    P->down_line = malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
    for (int32_t l = 0; l < nl; l++) P->down_off[pb->up[l] + 1]++;
    for (int32_t u = 0; u < pb->nlev; u++) P->down_off[u + 1] += P->down_off[u];
    int32_t *fill = calloc((size_t)pb->nlev + 1, sizeof(int32_t));
    for (int32_t l = 0; l < nl; l++) { int32_t u = pb->up[l]; P->down_line[P->down_off[u] + fill[u]++] = l; }
    free(fill);
    /* cell luminosities */
    P->Lc = calloc((size_t)P->ncell, sizeof(double));
    if (pr->emission_mode == 0) {
        for (int64_t c = 0; c < P->ncell; c++) P->Lc[c] = pb->L_cell[c];
    } else {
        /* Eq. (thin_emissivity): A_ul dE_ul beta_S N_u, N_u = n_u V_cell */
        P->wline = calloc((size_t)(P->ncell * nl), sizeof(double));
        for (int64_t c = 0; c < P->ncell; c++) {
            double V = P->dx * P->dy * P->dz;
            if (pb->geometry == 1) {    /* (prep's spherical tables come later: the volume here) */
                int32_t ir = (int32_t)(c % pb->nx), it = (int32_t)((c / pb->nx) % pb->ny);
                int32_t ip = (int32_t)(c / ((int64_t)pb->nx * pb->ny));
                double r0 = pb->r_edges[ir] * pb->t, r1 = pb->r_edges[ir + 1] * pb->t;
                V = (r1 * r1 * r1 - r0 * r0 * r0) / 3.0 * (cos(pb->th_edges[it]) - cos(pb->th_edges[it + 1]))
                    * (pb->ph_edges[ip + 1] - pb->ph_edges[ip]);
            }
            const double *n = pb->pops + c * pb->nlev;
            double sum = 0.0;
            for (int32_t l = 0; l < nl; l++) {
                double lam = pb->lambda_A[l] * 1e-8;
                double tau = xo_tau_sobolev(P->A[l], pb->g[pb->lo[l]], pb->g[pb->up[l]], lam,
                                            n[pb->lo[l]], n[pb->up[l]], pb->t);
                double dE = XO_H * XO_C / lam;
                double w = P->A[l] * dE * xo_beta_sobolev(tau) * n[pb->up[l]] * V;
                P->wline[c * nl + l] = w;
                sum += w;
            }
            P->Lc[c] = sum;
        }
    }
    P->qoff = malloc(sizeof(int64_t) * (size_t)(P->ncell + 1));
    xo_packet_quota(P->Lc, P->ncell, pr->n_packets, P->qoff);
    P->pi_tau = calloc((size_t)(pb->n_pi > 0 ? pb->n_pi : 1), sizeof(double));
    if (pb->geometry == 1) {
        P->sR = malloc(sizeof(double) * (size_t)(pb->nx + 1));
        P->cth = malloc(sizeof(double) * (size_t)(pb->ny + 1));
        P->eq = calloc((size_t)(pb->ny + 1), sizeof(int32_t));
        P->cph = malloc(sizeof(double) * (size_t)(pb->nz + 1));
        P->sph = malloc(sizeof(double) * (size_t)(pb->nz + 1));
        P->vol = malloc(sizeof(double) * (size_t)P->ncell);
        for (int32_t i = 0; i <= pb->nx; i++) P->sR[i] = pb->r_edges[i] * pb->t;
        for (int32_t j = 0; j <= pb->ny; j++) {
            P->cth[j] = cos(pb->th_edges[j]);
            P->eq[j] = fabs(P->cth[j]) < 1e-12;
        }
        for (int32_t k = 0; k <= pb->nz; k++) {
            double ph = pb->ph_edges[k == pb->nz ? 0 : k];
            P->cph[k] = cos(ph);
            P->sph[k] = sin(ph);
        }
        for (int64_t c = 0; c < P->ncell; c++) {
            int32_t ir = (int32_t)(c % pb->nx), it = (int32_t)((c / pb->nx) % pb->ny);
            int32_t ip = (int32_t)(c / ((int64_t)pb->nx * pb->ny));
            P->vol[c] = (P->sR[ir + 1] * P->sR[ir + 1] * P->sR[ir + 1] - P->sR[ir] * P->sR[ir] * P->sR[ir]) / 3.0
                        * (P->cth[it] - P->cth[it + 1]) * (pb->ph_edges[ip + 1] - pb->ph_edges[ip]);
        }
    }
    return 0;
}

static void unprep(prep_t *P) {
    free(P->order); free(P->pos); free(P->nu); free(P->A); free(P->Lc); free(P->qoff);
    free(P->wline); free(P->down_off); free(P->down_line); free(P->pi_tau);
    free(P->rcell); free(P->rbin_nu); free(P->rbin_cursor); free(P->rbin_frac);
    free(P->rbin_off); free(P->rbin_line); free(P->view_n); free(P->view_w);
    free(P->sR); free(P->cth); free(P->eq); free(P->cph); free(P->sph); free(P->vol);
}

static int32_t cursor_at(const prep_t *P, double nu);
int64_t xo_lambda_bin(double lam_A, double lam0, double dlog, int32_t nbins);

/* The RAYS sampler (Sec. 2.3): from the middle of every emitting cell, for
 * every wavelength bin j of the output grid that holds emission, one ray
 * towards every viewer k, with N = E_bin,ij (dOmega_k / 4 pi) / (h nu_j).
 * Readings: the paper prints the solid-angle factor as a division by
 * dOmega_k; the rays of a cell and bin must carry its emission isotropically
 * (the stated purpose of the factor), so each carries the share
 * dOmega_k / 4 pi.  A ray leaves along the centre direction of its viewer's
 * (theta, phi) bin.  nu_j is the reddest feature of the bin: for band emission
 * the red edge of the bin's overlap with the band (the ray tests the lines at
 * or below it), for line emission the reddest line in the bin (the ray starts
 * past it, as a line-emitted packet does).  Bins are the output grid's
 * lam0 (1 + dlog)^j.  Returns -1 if an emitting line lies outside the grid. */
static int rays_prep(prep_t *P) {
    const xo_problem *pb = P->pb;
    const xo_params *pr = P->pr;
    int32_t nb = pr->spec_nbins;
    P->rcell = malloc(sizeof(int64_t) * (size_t)(P->ncell > 0 ? P->ncell : 1));
    P->n_rcell = 0;
    for (int64_t c = 0; c < P->ncell; c++)
        if (P->Lc[c] > 0.0) P->rcell[P->n_rcell++] = c;
    P->rbin_nu = malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
    P->rbin_cursor = malloc(sizeof(int32_t) * (size_t)(nb > 0 ? nb : 1));
    P->rbin_frac = calloc((size_t)(nb > 0 ? nb : 1), sizeof(double));
    P->n_rbin = 0;
    if (pr->emission_mode == 0) {
        double nu_lo = XO_C / (pb->band_hi_A * 1e-8), nu_hi = XO_C / (pb->band_lo_A * 1e-8);
        for (int32_t j = 0; j < nb; j++) {
            double l0 = pr->spec_lam0_A * pow(1.0 + pr->spec_dlog, (double)j);
            double l1 = pr->spec_lam0_A * pow(1.0 + pr->spec_dlog, (double)(j + 1));
            double a = l0 > pb->band_lo_A ? l0 : pb->band_lo_A;
            double b = l1 < pb->band_hi_A ? l1 : pb->band_hi_A;
            if (!(b > a)) continue;
            double nu_red = XO_C / (b * 1e-8), nu_blue = XO_C / (a * 1e-8);
            int32_t k = P->n_rbin++;
            P->rbin_nu[k] = nu_red;
            P->rbin_cursor[k] = cursor_at(P, nu_red);
            P->rbin_frac[k] = (nu_blue - nu_red) / (nu_hi - nu_lo);
        }
    } else {
        int32_t nl = pb->nline;
        int32_t *bin_of = malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
        int32_t *cnt = calloc((size_t)nb + 1, sizeof(int32_t));
        for (int32_t l = 0; l < nl; l++) {
            int64_t j = xo_lambda_bin(pb->lambda_A[l], pr->spec_lam0_A, pr->spec_dlog, nb);
            if (j < 0) { free(bin_of); free(cnt); return -1; }
            bin_of[l] = (int32_t)j;
            cnt[j + 1]++;
        }
        int32_t *jmap = malloc(sizeof(int32_t) * (size_t)(nb > 0 ? nb : 1));
        for (int32_t j = 0; j < nb; j++) jmap[j] = cnt[j + 1] > 0 ? P->n_rbin++ : -1;
        P->rbin_off = calloc((size_t)P->n_rbin + 1, sizeof(int32_t));
        P->rbin_line = malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
        for (int32_t l = 0; l < nl; l++) P->rbin_off[jmap[bin_of[l]] + 1]++;
        for (int32_t k = 0; k < P->n_rbin; k++) P->rbin_off[k + 1] += P->rbin_off[k];
        int32_t *fill = calloc((size_t)P->n_rbin + 1, sizeof(int32_t));
        for (int32_t l = 0; l < nl; l++) {
            int32_t k = jmap[bin_of[l]];
            P->rbin_line[P->rbin_off[k] + fill[k]++] = l;
        }
        for (int32_t k = 0; k < P->n_rbin; k++) {
            /* reddest line of the bin; equal frequencies: start past the last of them */
            int32_t best = -1;
            for (int32_t q = P->rbin_off[k]; q < P->rbin_off[k + 1]; q++) {
                int32_t s = P->pos[P->rbin_line[q]];
                if (best < 0 || s > best) best = s;
            }
            P->rbin_nu[k] = P->nu[best];
            P->rbin_cursor[k] = best + 1;
        }
        free(bin_of); free(cnt); free(jmap); free(fill);
    }
    int32_t nv = pr->n_theta * pr->n_phi;
    P->view_n = malloc(sizeof(double) * 3 * (size_t)nv);
    P->view_w = malloc(sizeof(double) * (size_t)nv);
    for (int32_t it = 0; it < pr->n_theta; it++)
        for (int32_t ip = 0; ip < pr->n_phi; ip++) {
            int32_t k = it * pr->n_phi + ip;
            double th = XO_PI * (it + 0.5) / pr->n_theta, ph = 2.0 * XO_PI * (ip + 0.5) / pr->n_phi;
            double th0 = XO_PI * it / pr->n_theta, th1 = XO_PI * (it + 1) / pr->n_theta;
            P->view_n[3 * k] = sin(th) * cos(ph);
            P->view_n[3 * k + 1] = sin(th) * sin(ph);
            P->view_n[3 * k + 2] = cos(th);
            P->view_w[k] = (2.0 * XO_PI / pr->n_phi) * (cos(th0) - cos(th1)) / (4.0 * XO_PI);
        }
    return 0;
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Eq. (sigma_OTSPI): hydrogenic photoionization cross section [cm^2] of a
 * level of energy E_u in an ion of ionization energy E_ion and charge C, for a
 * photon of wavelength lambda below the threshold wavelength
 * lambda_ion = h c / (E_ion - E_u); Gaunt factor 1. */
double xo_sigma_pi(double lambda_cm, double E_u, double E_ion, int32_t C) {
    double lam_ion = XO_H * XO_C / (E_ion - E_u);
    double x = lambda_cm / lam_ion;
    return 7.9e-18 * x * x * x * pow(1.0 - E_u / E_ion, -0.5) / ((C + 1.0) * (C + 1.0));
}

/* Photoionization along the path r + s n, s in [s0, s1], of a packet of N
 * photons with lab frequency nu_lab (Sec. 2.3.1).  Readings: the photon
 * wavelength of the segment is the comoving one at its start, s0 (the
 * paper evaluates sigma_PI "for each distance d that a ray travels"); a level
 * takes part if the photon energy there exceeds its threshold E_ion - E_u, and
 * its path length stops where the comoving frequency, falling along the
 * segment, reaches the threshold ("d is modified").  N_abs = N (1 - e^-tau),
 * level i gets N_abs tau_i / tau; the excess h nu - (E_ion - E_u) of each
 * absorbed photon is heating.  Returns 1 when the packet's photon energy at the
 * segment end has fallen below e_cut of its start (the rest is dropped). */
static int pi_segment(const prep_t *P, int64_t cell, const double *pc, double nu_lab,
                      const double n[3], const double r[3], double s0, double s1, double *N,
                      double E0, double *S_pi, double *heat, double *ledger) {
    const xo_problem *pb = P->pb;
    double d = s1 - s0;
    if (d < 0.0) d = 0.0;
    double q[3] = {r[0] + s0 * n[0], r[1] + s0 * n[1], r[2] + s0 * n[2]};
    double nu_a = nu_lab * (1.0 - dot3(n, q) / P->ct);
    double lam_a = XO_C / nu_a;
    double tot = 0.0;
    for (int32_t k = 0; k < pb->n_pi; k++) {
        double Eu = pb->E_level[pb->pi_level[k]];
        double chi = pb->pi_Eion[k] - Eu;
        P->pi_tau[k] = 0.0;
        if (XO_H * nu_a > chi) {
            double dk = d;
            double s_th = (nu_a - chi / XO_H) * P->ct / nu_lab;   /* where nu_cmf = chi / h */
            if (s_th < dk) dk = s_th;
            double sig = xo_sigma_pi(lam_a, Eu, pb->pi_Eion[k], pb->pi_charge[k]);
            P->pi_tau[k] = sig * dk * pc[pb->pi_level[k]];
            tot += P->pi_tau[k];
        }
    }
    if (tot > 0.0) {
        double ex, ome;
        if (tot > XO_LN2) { ex = exp(-tot); ome = 1.0 - ex; }
        else { ome = -expm1(-tot); ex = 1.0 - ome; }
        double Nabs = *N * ome;
        for (int32_t k = 0; k < pb->n_pi; k++) {
            if (P->pi_tau[k] <= 0.0) continue;
            double share = Nabs * P->pi_tau[k] / tot;
            double chi = pb->pi_Eion[k] - pb->E_level[pb->pi_level[k]];
            if (S_pi) S_pi[cell * pb->n_pi + k] += share;
            if (heat) heat[cell] += share * (XO_H * nu_a - chi);
        }
        ledger[L_PI_N] += Nabs;
        ledger[L_PI_E] += Nabs * XO_H * nu_a;
        *N = *N * ex;
    }
    double nu_b = nu_a - nu_lab * d / P->ct;          /* comoving frequency at the segment end */
    if (*N * XO_H * nu_b < P->pr->e_cut * E0) {
        ledger[L_DROP_N] += *N;
        return 1;
    }
    return 0;
}

static int64_t cell_of_packet(const prep_t *P, int64_t p) {
    /* last c with qoff[c] <= p (cells with zero quota are skipped) */
    int64_t lo = 0, hi = P->ncell;   /* invariant qoff[lo] <= p < qoff[hi] */
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (P->qoff[mid] <= p) lo = mid; else hi = mid;
    }
    return lo;
}

/* first sorted position whose frequency is <= nu (lines sorted descending) */
static int32_t cursor_at(const prep_t *P, double nu) {
    int32_t lo = 0, hi = P->pb->nline;
    while (lo < hi) {
        int32_t mid = (lo + hi) / 2;
        if (P->nu[mid] <= nu) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static void isotropic(double umu, double uphi, double n[3]) {
    double mu = 2.0 * umu - 1.0;
    double phi = 2.0 * XO_PI * uphi;
    double st = sqrt(1.0 - mu * mu);
    n[0] = st * cos(phi); n[1] = st * sin(phi); n[2] = mu;
}


/* Viewing-direction bin: theta in [0,pi] and phi in [0,2pi) cut into equal angles. */
int32_t xo_viewer_bin(const double n[3], int32_t n_theta, int32_t n_phi) {
    double th = acos(n[2]);
    double ph = atan2(n[1], n[0]);
    if (ph < 0.0) ph += 2.0 * XO_PI;
    int32_t it = (int32_t)floor(th / (XO_PI / n_theta));
    int32_t ip = (int32_t)floor(ph / (2.0 * XO_PI / n_phi));
    if (it >= n_theta) it = n_theta - 1;
    if (ip >= n_phi) ip = n_phi - 1;
    if (it < 0) it = 0;
    if (ip < 0) ip = 0;
    return it * n_phi + ip;
}

/* Output wavelength bin on the log grid lambda_k = lam0 (1 + dlog)^k; -1 outside. */
int64_t xo_lambda_bin(double lam_A, double lam0, double dlog, int32_t nbins) {
    if (!(lam_A >= lam0)) return -1;
    double k = floor(log(lam_A / lam0) / log1p(dlog));
    if (k >= (double)nbins) return -1;
    return (int64_t)k;
}

/* Optional sparse estimator sink: one record per estimator increment. */
typedef struct { int64_t cell; int64_t line; double value; } xo_rec;
static xo_rec *g_rec;
static int64_t g_rec_cap, g_rec_n;

static void add_estimator(double *S, int64_t cell, int32_t nline, int32_t l, double v) {
    if (S) S[cell * nline + l] += v;
    if (g_rec) {
        if (g_rec_n < g_rec_cap) { g_rec[g_rec_n].cell = cell; g_rec[g_rec_n].line = l; g_rec[g_rec_n].value = v; }
        g_rec_n++;
    }
}

/* packet_out record per packet: fate, events, N_final, escaped lab energy,
 * viewer, lambda bin, interactions, start cell, N0, nu_cmf at emission,
 * final nu_lab */
#define XO_PKT_FIELDS 11

/* A packet in flight: everything the event loop carries from one cell to the
 * next (resumable, for the spatial decomposition across processes). */
typedef struct {
    int64_t p, c;                       /* packet id, emitting cell */
    int32_t idx[3];                     /* current cell */
    double r[3], n[3];                  /* position (on the entry wall), direction */
    double nu_lab, N, E0, N0, nu_cmf0;
    int32_t cursor;
    int64_t events, interactions, ndraw;
    double s;                           /* spherical grid: path from the emission point r */
} xo_state;
#define XO_STATE_FIELDS 21

/* Where packets that leave a domain go (NULL: the whole grid is the domain). */
typedef struct {
    int32_t z_lo, z_hi;                 /* the domain: cells with z in [z_lo, z_hi) */
    double *out;                        /* XO_STATE_FIELDS doubles per leaving packet */
    int64_t cap, n;
} xo_domain;

static void trace(const prep_t *P, xo_state *st, double *S, double *spec, double *ledger,
                  double *pkt, double *S_pi, double *heat, xo_domain *dom);
static void propagate(const prep_t *P, int64_t p, int64_t c, int32_t idx[3], double r[3], double n[3],
                      double nu_cmf, int32_t cursor, double E0, double *S, double *spec,
                      double *ledger, double *pkt, double *S_pi, double *heat, xo_domain *dom);

static void transport_packet(const prep_t *P, int64_t p, double *S, double *spec,
                             double *ledger, double *pkt, double *S_pi, double *heat, xo_domain *dom) {
    const xo_problem *pb = P->pb;
    const xo_params *pr = P->pr;
    int64_t c = cell_of_packet(P, p);
    int32_t ix = (int32_t)(c % pb->nx), iy = (int32_t)((c / pb->nx) % pb->ny), iz = (int32_t)(c / ((int64_t)pb->nx * pb->ny));
    int64_t nq = P->qoff[c + 1] - P->qoff[c];
    double E0 = P->Lc[c] / (double)nq;      /* packet energy, erg/s */
    double u[4], v[4];
    draw4(pr->seed, p, 0, u);
    draw4(pr->seed, p, 1, v);
    double d[3] = {P->dx, P->dy, P->dz};
    int32_t idx[3] = {ix, iy, iz};
    double r[3];
    if (pb->geometry == 1) {
        /* uniform in the spherical cell: r^3, cos theta and phi uniform */
        double R0 = P->sR[ix], R1 = P->sR[ix + 1];
        double rr = cbrt(R0 * R0 * R0 + u[0] * (R1 * R1 * R1 - R0 * R0 * R0));
        double ct = P->cth[iy] - u[1] * (P->cth[iy] - P->cth[iy + 1]);
        double ph = pb->ph_edges[iz] + u[2] * (pb->ph_edges[iz + 1] - pb->ph_edges[iz]);
        double q = 1.0 - ct * ct, st = q > 0.0 ? sqrt(q) : 0.0;
        r[0] = rr * st * cos(ph); r[1] = rr * st * sin(ph); r[2] = rr * ct;
    } else {
        for (int a = 0; a < 3; a++) r[a] = (-P->R + idx[a] * d[a]) + u[a] * d[a];
    }
    double n[3];
    isotropic(u[3], v[0], n);
    double nu_cmf, nu_lo = XO_C / (pb->band_hi_A * 1e-8), nu_hi = XO_C / (pb->band_lo_A * 1e-8);
    int32_t cursor;
    if (pr->emission_mode == 0) {
        nu_cmf = nu_lo + v[1] * (nu_hi - nu_lo);
        cursor = cursor_at(P, nu_cmf);
    } else {
        /* choose the emitting line by its share of the cell's line emission */
        const double *w = P->wline + c * pb->nline;
        double x = v[1] * P->Lc[c], acc = 0.0;
        int32_t pick = pb->nline - 1;
        for (int32_t l = 0; l < pb->nline; l++) {
            acc += w[l];
            if (x < acc) { pick = l; break; }
        }
        nu_cmf = XO_C / (pb->lambda_A[pick] * 1e-8);
        cursor = P->pos[pick] + 1;           /* start past the emitting line */
    }
    propagate(P, p, c, idx, r, n, nu_cmf, cursor, E0, S, spec, ledger, pkt, S_pi, heat, dom);
}

/* Ray r of the RAYS sampler: r = (cell rank, bin rank, viewer) in row-major
 * order over the emitting cells, the emitting bins and the viewers.  A ray
 * whose cell has no emission in its bin is empty: fate 4, nothing traced. */
static void transport_ray(const prep_t *P, int64_t r, double *S, double *spec, double *ledger,
                          double *pkt, double *S_pi, double *heat, xo_domain *dom) {
    const xo_problem *pb = P->pb;
    const xo_params *pr = P->pr;
    int64_t nv = (int64_t)pr->n_theta * pr->n_phi;
    int64_t ci = r / ((int64_t)P->n_rbin * nv), rem = r - ci * (int64_t)P->n_rbin * nv;
    int32_t jb = (int32_t)(rem / nv), k = (int32_t)(rem - (int64_t)jb * nv);
    int64_t c = P->rcell[ci];
    double E_bin;
    if (pr->emission_mode == 0) {
        E_bin = P->Lc[c] * P->rbin_frac[jb];
    } else {
        E_bin = 0.0;
        for (int32_t q = P->rbin_off[jb]; q < P->rbin_off[jb + 1]; q++)
            E_bin += P->wline[c * pb->nline + P->rbin_line[q]];
    }
    double E0 = E_bin * P->view_w[k];
    if (!(E0 > 0.0)) {
        if (pkt) {
            memset(pkt, 0, sizeof(double) * XO_PKT_FIELDS);
            pkt[0] = 4; pkt[4] = -1; pkt[5] = -1; pkt[7] = (double)c;
        }
        return;
    }
    int32_t idx[3] = {(int32_t)(c % pb->nx), (int32_t)((c / pb->nx) % pb->ny), (int32_t)(c / ((int64_t)pb->nx * pb->ny))};
    double d[3] = {P->dx, P->dy, P->dz};
    double rr[3], n[3];
    for (int a = 0; a < 3; a++) {
        rr[a] = (-P->R + idx[a] * d[a]) + 0.5 * d[a];     /* the middle of the cell */
        n[a] = P->view_n[3 * k + a];
    }
    if (pb->geometry == 1) {
        /* spherical cell: the middle of its radius, polar and azimuthal ranges */
        double rm = 0.5 * (P->sR[idx[0]] + P->sR[idx[0] + 1]);
        double th = 0.5 * (pb->th_edges[idx[1]] + pb->th_edges[idx[1] + 1]);
        double ph = 0.5 * (pb->ph_edges[idx[2]] + pb->ph_edges[idx[2] + 1]);
        rr[0] = rm * sin(th) * cos(ph); rr[1] = rm * sin(th) * sin(ph); rr[2] = rm * cos(th);
    }
    propagate(P, r, c, idx, rr, n, P->rbin_nu[jb], P->rbin_cursor[jb], E0, S, spec, ledger, pkt, S_pi, heat,
              dom);
}

/* The event loop of one packet or ray from its emission (Secs. 2.3, 2.3.2):
 * cell idx (natural index c), position r, direction n, comoving frequency
 * nu_cmf, first line to test `cursor`, energy E0 (erg/s). */
static void propagate(const prep_t *P, int64_t p, int64_t c, int32_t idx[3], double r[3], double n[3],
                      double nu_cmf, int32_t cursor, double E0, double *S, double *spec,
                      double *ledger, double *pkt, double *S_pi, double *heat, xo_domain *dom) {
    xo_state st;
    st.p = p; st.c = c;
    for (int a = 0; a < 3; a++) { st.idx[a] = idx[a]; st.r[a] = r[a]; st.n[a] = n[a]; }
    st.nu_lab = nu_cmf / (1.0 - dot3(n, r) / P->ct);
    st.N = E0 / (XO_H * nu_cmf);
    st.E0 = E0; st.N0 = st.N; st.nu_cmf0 = nu_cmf;
    st.cursor = cursor;
    st.events = st.interactions = st.ndraw = 0;
    st.s = 0.0;
    ledger[L_EMIT_N] += st.N;
    ledger[L_EMIT_E] += E0;
    trace(P, &st, S, spec, ledger, pkt, S_pi, heat, dom);
}

/* The packet's state as XO_STATE_FIELDS doubles (integers exactly). */
static void state_pack(const xo_state *st, double *o) {
    o[0] = (double)st->p; o[1] = (double)st->c;
    for (int a = 0; a < 3; a++) { o[2 + a] = st->idx[a]; o[5 + a] = st->r[a]; o[8 + a] = st->n[a]; }
    o[11] = st->nu_lab; o[12] = st->N; o[13] = st->E0; o[14] = st->N0; o[15] = st->nu_cmf0;
    o[16] = st->cursor; o[17] = (double)st->events; o[18] = (double)st->interactions;
    o[19] = (double)st->ndraw; o[20] = st->s;
}

static void state_unpack(const double *o, xo_state *st) {
    st->p = (int64_t)o[0]; st->c = (int64_t)o[1];
    for (int a = 0; a < 3; a++) { st->idx[a] = (int32_t)o[2 + a]; st->r[a] = o[5 + a]; st->n[a] = o[8 + a]; }
    st->nu_lab = o[11]; st->N = o[12]; st->E0 = o[13]; st->N0 = o[14]; st->nu_cmf0 = o[15];
    st->cursor = (int32_t)o[16]; st->events = (int64_t)o[17]; st->interactions = (int64_t)o[18];
    st->ndraw = (int64_t)o[19];
    st->s = o[20];
}

/* Spherical grid: the path s > s_cur from the emission point p0 along n at
 * which the ray leaves cell idx, and through which face (*kind: 0 outer
 * sphere, 1 inner sphere, 2 lower theta cone, 3 upper theta cone, 4 lower phi
 * half-plane, 5 upper phi half-plane).  Every face's crossing is computed
 * from p0 and n alone, so the face just crossed gives exactly s_cur again and
 * is excluded by s > s_cur.  A cone |z| = cos(theta) |p| counts on its own
 * nappe only (z of the sign of cos theta); an equatorial edge is the plane
 * z = 0; a half-plane counts on its own side of the axis. */
static double cone_cross(const double p0[3], const double n[3], double c, int eq, double b, double pp,
                         double s_cur) {
    if (eq) {
        if (n[2] == 0.0) return INFINITY;
        double s = -p0[2] / n[2];
        return s > s_cur ? s : INFINITY;
    }
    double c2 = c * c;
    double A = n[2] * n[2] - c2, B = p0[2] * n[2] - c2 * b, C = p0[2] * p0[2] - c2 * pp;
    double r[2];
    int nr = 0;
    if (A == 0.0) {
        if (B == 0.0) return INFINITY;
        r[nr++] = -C / (2.0 * B);
    } else {
        double disc = B * B - A * C;
        if (disc < 0.0) return INFINITY;
        double sq = sqrt(disc);
        double s1 = (-B - sq) / A, s2 = (-B + sq) / A;
        r[nr++] = s1 < s2 ? s1 : s2;
        r[nr++] = s1 < s2 ? s2 : s1;
    }
    for (int k = 0; k < nr; k++)
        if (r[k] > s_cur && (p0[2] + r[k] * n[2]) * c > 0.0) return r[k];
    return INFINITY;
}

static double sph_exit(const prep_t *P, const double p0[3], const double n[3], const int32_t idx[3],
                       double s_cur, int *kind) {
    const xo_problem *pb = P->pb;
    double b = dot3(p0, n), pp = dot3(p0, p0);
    double best = INFINITY;
    *kind = -1;
    double R1 = P->sR[idx[0] + 1];
    double disc = b * b - (pp - R1 * R1);
    if (disc > 0.0) {
        double s = -b + sqrt(disc);
        if (s > s_cur && s < best) { best = s; *kind = 0; }
    }
    if (idx[0] > 0) {
        double R0 = P->sR[idx[0]];
        double d0 = b * b - (pp - R0 * R0);
        if (d0 > 0.0) {
            double s = -b - sqrt(d0);
            if (s > s_cur && s < best) { best = s; *kind = 1; }
        }
    }
    for (int e = 0; e < 2; e++) {
        int32_t j = idx[1] + e;
        if (j == 0 || j == pb->ny) continue;            /* the polar axis */
        double s = cone_cross(p0, n, P->cth[j], P->eq[j], b, pp, s_cur);
        if (s < best) { best = s; *kind = 2 + e; }
    }
    if (pb->nz > 1)
        for (int e = 0; e < 2; e++) {
            int32_t k = idx[2] + e;
            double cs = P->cph[k], sn = P->sph[k];
            double den = n[1] * cs - n[0] * sn;           /* n . (-sin, cos, 0) */
            if (den == 0.0) continue;
            double s = -(p0[1] * cs - p0[0] * sn) / den;
            if (!(s > s_cur) || !(s < best)) continue;
            double qx = p0[0] + s * n[0], qy = p0[1] + s * n[1];
            if (qx * cs + qy * sn > 0.0) { best = s; *kind = 4 + e; }
        }
    return best;
}

/* The cell beyond the face of kind `kind` of cell idx (updated in place):
 * returns 1 if that is the outside of the outer sphere (idx[0] = nx), -1 if
 * there was no face (kind < 0), else 0.  Azimuthal indices wrap around. */
static int sph_cross(const xo_problem *pb, int32_t idx[3], int kind) {
    if (kind == 0) return ++idx[0] == pb->nx ? 1 : 0;
    if (kind == 1) idx[0]--;
    else if (kind == 2) idx[1]--;
    else if (kind == 3) idx[1]++;
    else if (kind == 4) idx[2] = idx[2] == 0 ? pb->nz - 1 : idx[2] - 1;
    else if (kind == 5) idx[2] = idx[2] == pb->nz - 1 ? 0 : idx[2] + 1;
    else return -1;
    return 0;
}

/* The event loop on the spherical grid (attenuation mode): as in trace, with
 * the walk through (r, theta, phi) cells; the packet's position is p0 + s n. */
static int pi_segment(const prep_t *P, int64_t cell, const double *pc, double nu_lab,
                      const double n[3], const double r[3], double s0, double s1, double *N,
                      double E0, double *S_pi, double *heat, double *ledger);

static void trace_sph(const prep_t *P, xo_state *st, double *S, double *spec, double *ledger, double *pkt,
                      double *S_pi, double *heat, xo_domain *dom) {
    const xo_problem *pb = P->pb;
    const xo_params *pr = P->pr;
    double ct = P->ct;
    int64_t c = st->c;
    int32_t *idx = st->idx;
    const double *p0 = st->r, *n = st->n;
    double nu_lab = st->nu_lab, N = st->N, E0 = st->E0, s = st->s;
    int32_t cursor = st->cursor;
    int64_t events = st->events;
    int fate = 0;
    double esc_E = 0.0;
    int32_t vbin = -1;
    int64_t lbin = -1;
    for (;;) {
        int64_t cell = ((int64_t)idx[2] * pb->ny + idx[1]) * pb->nx + idx[0];
        const double *pc = pb->pops + cell * pb->nlev;
        int kind;
        double s_exit = sph_exit(P, p0, n, idx, s, &kind);
        double r_end[3];
        for (int a = 0; a < 3; a++) r_end[a] = p0[a] + s_exit * n[a];
        double nu_end = nu_lab * (1.0 - dot3(n, r_end) / ct);
        double s_pi = s;            /* start of the photoionization segment (path from p0) */
        while (cursor < pb->nline && P->nu[cursor] > nu_end) {
            int32_t l = P->order[cursor];
            ledger[L_TESTS] += 1.0;
            double n_l = pc[pb->lo[l]], n_u = pc[pb->up[l]];
            double g_l = pb->g[pb->lo[l]], g_u = pb->g[pb->up[l]];
            double lam = pb->lambda_A[l] * 1e-8;
            double tau = xo_tau_sobolev(P->A[l], g_l, g_u, lam, n_l, n_u, pb->t);
            if (tau > pr->tau_min) {
                double nu_l = P->nu[cursor];
                if (pb->n_pi > 0) {
                    /* the ray moves to the resonance point, photoionizing on the way
                     * (Secs. 2.3.1, 2.3.2); the line sees what photoionization left */
                    double s_l = ct * (1.0 - nu_l / nu_lab) - dot3(n, p0);
                    if (pi_segment(P, cell, pc, nu_lab, n, p0, s_pi, s_l, &N, E0, S_pi, heat, ledger)) {
                        fate = 1;
                        goto done;
                    }
                    if (s_l > s_pi) s_pi = s_l;
                }
                events++;
                ledger[L_EVENTS] += 1.0;
                double f_corr = 1.0 - g_l * n_u / (g_u * n_l);
                double ex, ome;
                if (tau > XO_LN2) { ex = exp(-tau); ome = 1.0 - ex; }
                else { ome = -expm1(-tau); ex = 1.0 - ome; }
                double dN = N * ome;
                add_estimator(S, cell, pb->nline, l, dN / f_corr);
                N = N * ex;
                ledger[L_ABS_N] += dN;
                if (N * XO_H * nu_l < pr->e_cut * E0) {
                    ledger[L_DROP_N] += N;
                    fate = 1;
                    goto done;
                }
                if (events >= pr->max_events) { fate = 3; ledger[L_GUARD] += 1.0; goto done; }
            }
            cursor++;
        }
        if (pb->n_pi > 0 &&
            pi_segment(P, cell, pc, nu_lab, n, p0, s_pi, s_exit, &N, E0, S_pi, heat, ledger)) {
            fate = 1;
            goto done;
        }
        s = s_exit;
        int crossed = sph_cross(pb, idx, kind);
        if (crossed == 1) {                               /* leaves the outer sphere */
            double E = N * XO_H * nu_lab;
            esc_E = E;
            ledger[L_ESC_N] += N;
            ledger[L_ESC_E] += E;
            vbin = xo_viewer_bin(n, pr->n_theta, pr->n_phi);
            lbin = xo_lambda_bin(XO_C / nu_lab * 1e8, pr->spec_lam0_A, pr->spec_dlog, pr->spec_nbins);
            if (lbin >= 0) spec[(int64_t)vbin * pr->spec_nbins + lbin] += E;
            else ledger[L_OOB_E] += E;
            fate = 0;
            goto done;
        } else if (crossed < 0) {
            fate = 3;                                      /* no face ahead (cannot happen inside) */
            ledger[L_GUARD] += 1.0;
            goto done;
        }
        if (dom && (idx[2] < dom->z_lo || idx[2] >= dom->z_hi)) {
            /* the packet enters another domain's phi slices: hand its state on
             * (Sec. 2.4.1), the path s from its emission point included */
            st->nu_lab = nu_lab; st->N = N; st->cursor = cursor; st->events = events; st->s = s;
            if (dom->n < dom->cap) state_pack(st, dom->out + dom->n * XO_STATE_FIELDS);
            dom->n++;
            return;
        }
    }
done:
    if (pkt) {
        pkt[0] = fate; pkt[1] = (double)events; pkt[2] = N; pkt[3] = esc_E;
        pkt[4] = vbin; pkt[5] = (double)lbin; pkt[6] = 0.0; pkt[7] = (double)c;
        pkt[8] = st->N0; pkt[9] = st->nu_cmf0; pkt[10] = nu_lab;
    }
}

/* The event loop from the state st until the packet ends (its record, if
 * asked, written to pkt) or, with a domain, enters a cell outside it (its
 * state then appended to dom->out). */
static void trace(const prep_t *P, xo_state *st, double *S, double *spec, double *ledger,
                  double *pkt, double *S_pi, double *heat, xo_domain *dom) {
    if (P->pb->geometry == 1) {
        trace_sph(P, st, S, spec, ledger, pkt, S_pi, heat, dom);
        return;
    }
    const xo_problem *pb = P->pb;
    const xo_params *pr = P->pr;
    double d[3] = {P->dx, P->dy, P->dz};
    int32_t nn[3] = {pb->nx, pb->ny, pb->nz};
    double ct = P->ct;
    int64_t p = st->p, c = st->c;
    int32_t *idx = st->idx;
    double *r = st->r, *n = st->n;
    double nu_lab = st->nu_lab, N = st->N, E0 = st->E0;
    const double N0 = st->N0, nu_cmf0 = st->nu_cmf0;
    int32_t cursor = st->cursor;
    int64_t events = st->events, interactions = st->interactions, ndraw = st->ndraw;
    int fate = 0;    /* 0 escaped, 1 dropped below the energy cut, 2 thermalised, 3 event guard */
    double esc_E = 0.0;
    int32_t vbin = -1;
    int64_t lbin = -1;
    for (;;) {
        int64_t cell = ((int64_t)idx[2] * pb->ny + idx[1]) * pb->nx + idx[0];
        const double *pc = pb->pops + cell * pb->nlev;
        /* distance to the cell walls, ties to the lowest axis */
        double s_wall = INFINITY;
        int axis = -1;
        for (int a = 0; a < 3; a++) {
            double s;
            if (n[a] > 0.0) s = ((-P->R + (idx[a] + 1) * d[a]) - r[a]) / n[a];
            else if (n[a] < 0.0) s = ((-P->R + idx[a] * d[a]) - r[a]) / n[a];
            else continue;
            if (s < 0.0) s = 0.0;
            if (s < s_wall) { s_wall = s; axis = a; }
        }
        double r_end[3];
        for (int a = 0; a < 3; a++) r_end[a] = r[a] + s_wall * n[a];
        double nu_end = nu_lab * (1.0 - dot3(n, r_end) / ct);
        int restart = 0;
        double s_pi = 0.0;          /* start of the photoionization segment, from r */
        while (cursor < pb->nline && P->nu[cursor] > nu_end) {
            int32_t l = P->order[cursor];
            ledger[L_TESTS] += 1.0;
            double n_l = pc[pb->lo[l]], n_u = pc[pb->up[l]];
            double g_l = pb->g[pb->lo[l]], g_u = pb->g[pb->up[l]];
            double lam = pb->lambda_A[l] * 1e-8;
            double tau = xo_tau_sobolev(P->A[l], g_l, g_u, lam, n_l, n_u, pb->t);
            if (tau > pr->tau_min) {
                double nu_l = P->nu[cursor];
                if (pr->mode == 0 && pb->n_pi > 0) {
                    /* the ray moves to the resonance point, photoionizing on the way
                     * (Sec. 2.3.2); the line sees what photoionization left */
                    double s_l = ct * (1.0 - nu_l / nu_lab) - dot3(n, r);
                    if (pi_segment(P, cell, pc, nu_lab, n, r, s_pi, s_l, &N, E0, S_pi, heat, ledger)) {
                        fate = 1;
                        goto done;
                    }
                    if (s_l > s_pi) s_pi = s_l;
                }
                events++;
                ledger[L_EVENTS] += 1.0;
                double f_corr = 1.0 - g_l * n_u / (g_u * n_l);
                /* 1 - e^-tau and e^-tau, each without cancellation */
                double ex, ome;
                if (tau > XO_LN2) { ex = exp(-tau); ome = 1.0 - ex; }
                else { ome = -expm1(-tau); ex = 1.0 - ome; }
                if (pr->mode == 0) {
                    double dN = N * ome;
                    add_estimator(S, cell, pb->nline, l, dN / f_corr);
                    N = N * ex;                       /* N_phot - N_PE: what goes on */
                    ledger[L_ABS_N] += dN;
                    if (N * XO_H * nu_l < pr->e_cut * E0) {
                        ledger[L_DROP_N] += N;
                        fate = 1;
                        goto done;
                    }
                } else {
                    double w[4];
                    draw4(pr->seed, p, 2 + (uint64_t)ndraw, w);   /* one draw per active resonance */
                    ndraw++;
                    if (w[0] < ome) {
                        interactions++;
                        ledger[L_INTERACT] += 1.0;
                        add_estimator(S, cell, pb->nline, l, N / f_corr);
                        ledger[L_ABS_N] += N;
                        double Ecmf = N * XO_H * nu_l;
                        ledger[L_ABS_E_CMF] += Ecmf;
                        /* re-emission channel: radiative down-lines of the upper
                         * level weighted by A beta, or collisional destruction */
                        int32_t ulev = pb->up[l];
                        double Te = pb->Te[cell], ne = pb->ne[cell];
                        double Ccoll = 8.629e-6 * ne * pb->ups_down[ulev] / (pb->g[ulev] * sqrt(Te));
                        double Wtot = Ccoll;
                        for (int32_t k = P->down_off[ulev]; k < P->down_off[ulev + 1]; k++) {
                            int32_t m = P->down_line[k];
                            double lm = pb->lambda_A[m] * 1e-8;
                            double tm = xo_tau_sobolev(P->A[m], pb->g[pb->lo[m]], g_u, lm,
                                                       pc[pb->lo[m]], pc[ulev], pb->t);
                            Wtot += P->A[m] * xo_beta_sobolev(tm);
                        }
                        double x = w[1] * Wtot, acc = 0.0;
                        int32_t pick = -1;
                        for (int32_t k = P->down_off[ulev]; k < P->down_off[ulev + 1]; k++) {
                            int32_t m = P->down_line[k];
                            double lm = pb->lambda_A[m] * 1e-8;
                            double tm = xo_tau_sobolev(P->A[m], pb->g[pb->lo[m]], g_u, lm,
                                                       pc[pb->lo[m]], pc[ulev], pb->t);
                            acc += P->A[m] * xo_beta_sobolev(tm);
                            if (x < acc) { pick = m; break; }
                        }
                        if (pick < 0) {
                            ledger[L_THERMAL_E] += Ecmf;
                            fate = 2;
                            goto done;
                        }
                        /* move to the resonance point, re-emit isotropically */
                        double s_l = ct * (1.0 - nu_l / nu_lab) - dot3(n, r);
                        for (int a = 0; a < 3; a++) r[a] = r[a] + s_l * n[a];
                        isotropic(w[2], w[3], n);
                        double nu_new = XO_C / (pb->lambda_A[pick] * 1e-8);
                        N = Ecmf / (XO_H * nu_new);
                        ledger[L_REEMIT_E_CMF] += Ecmf;
                        nu_lab = nu_new / (1.0 - dot3(n, r) / ct);
                        cursor = P->pos[pick] + 1;
                        if (events >= pr->max_events) { fate = 3; ledger[L_GUARD] += 1.0; goto done; }
                        restart = 1;
                        break;
                    }
                }
                if (events >= pr->max_events) { fate = 3; ledger[L_GUARD] += 1.0; goto done; }
            }
            cursor++;
        }
        if (restart) continue;
        if (pr->mode == 0 && pb->n_pi > 0 &&
            pi_segment(P, cell, pc, nu_lab, n, r, s_pi, s_wall, &N, E0, S_pi, heat, ledger)) {
            fate = 1;
            goto done;
        }
        /* advance to the wall and step into the next cell */
        for (int a = 0; a < 3; a++) r[a] = r_end[a];
        idx[axis] += (n[axis] > 0.0) ? 1 : -1;
        if (idx[axis] < 0 || idx[axis] >= nn[axis]) {
            double E = N * XO_H * nu_lab;
            esc_E = E;
            ledger[L_ESC_N] += N;
            ledger[L_ESC_E] += E;
            vbin = xo_viewer_bin(n, pr->n_theta, pr->n_phi);
            lbin = xo_lambda_bin(XO_C / nu_lab * 1e8, pr->spec_lam0_A, pr->spec_dlog, pr->spec_nbins);
            if (lbin >= 0) spec[(int64_t)vbin * pr->spec_nbins + lbin] += E;
            else ledger[L_OOB_E] += E;
            fate = 0;
            goto done;
        }
        if (dom && (idx[2] < dom->z_lo || idx[2] >= dom->z_hi)) {
            /* the packet leaves the domain: hand its state on (Sec. 2.4.1) */
            st->nu_lab = nu_lab; st->N = N; st->cursor = cursor;
            st->events = events; st->interactions = interactions; st->ndraw = ndraw;
            if (dom->n < dom->cap) state_pack(st, dom->out + dom->n * XO_STATE_FIELDS);
            dom->n++;
            return;
        }
    }
done:
    if (pkt) {
        pkt[0] = fate; pkt[1] = (double)events; pkt[2] = N; pkt[3] = esc_E;
        pkt[4] = vbin; pkt[5] = (double)lbin; pkt[6] = (double)interactions; pkt[7] = (double)c;
        pkt[8] = N0; pkt[9] = nu_cmf0; pkt[10] = nu_lab;
    }
}

/* Transport packets [p_begin, p_end) of an N-packet emission.  S (natural cell
 * order x caller line order; may be NULL), spec and ledger are accumulated
 * into; pkt (optional) receives XO_PKT_FIELDS doubles per packet; rec
 * (optional) receives one (cell, line, value) record per estimator increment;
 * S_pi [ncell][n_pi] and heat [ncell] (optional) the photons absorbed per
 * photoionizing level and the photoionization heating (erg/s) per cell.
 * Returns 0, or -1 if more than rec_cap records were produced. */
int xo_transport(const xo_problem *pb, const xo_params *pr, double *S, double *spec,
                 double *ledger, double *pkt, xo_rec *rec, int64_t rec_cap, int64_t *rec_n,
                 double *S_pi, double *heat) {
    prep_t P;
    g_rec = rec; g_rec_cap = rec_cap; g_rec_n = 0;
    prep(&P, pb, pr);
    if (pr->sampler == 1 && rays_prep(&P) != 0) { unprep(&P); g_rec = NULL; return -2; }
    for (int64_t p = pr->p_begin; p < pr->p_end; p++) {
        double *pk = pkt ? pkt + (p - pr->p_begin) * XO_PKT_FIELDS : NULL;
        if (pr->sampler == 1) transport_ray(&P, p, S, spec, ledger, pk, S_pi, heat, NULL);
        else transport_packet(&P, p, S, spec, ledger, pk, S_pi, heat, NULL);
    }
    unprep(&P);
    if (rec_n) *rec_n = g_rec_n;
    g_rec = NULL;
    return (rec && g_rec_n > rec_cap) ? -1 : 0;
}

/* Spatial decomposition across processes (Sec. 2.4.1): one domain of the
 * grid, the cells with z in [z_lo, z_hi).  With emit != 0 the packets of
 * [p_begin, p_end) that are emitted in the domain are traced; then the packets
 * of bundle_in (n_in states of XO_STATE_FIELDS doubles, handed on by other
 * domains) resume.  Every packet is traced until it ends or enters a cell of
 * another domain; the states of those are written to bundle_out (at most
 * out_cap, their number in *n_out).  Estimators, spectrum and ledger
 * accumulate as in xo_transport (emission is counted where the packet is
 * emitted).  Attenuation mode, Monte Carlo packets or rays (the rays of the
 * domain's emitting cells).  Returns 0, -1 if bundle_out was too small (its
 * first out_cap states are written), or -2 if an emitting line of the rays
 * lies outside the output grid. */
int xo_transport_domain(const xo_problem *pb, const xo_params *pr, int32_t z_lo, int32_t z_hi,
                        int32_t emit, const double *bundle_in, int64_t n_in, double *bundle_out,
                        int64_t out_cap, int64_t *n_out, double *S, double *spec, double *ledger,
                        double *S_pi, double *heat) {
    prep_t P;
    g_rec = NULL;
    prep(&P, pb, pr);
    xo_domain dom = {z_lo, z_hi, bundle_out, out_cap, 0};
    int64_t nxy = (int64_t)pb->nx * pb->ny;
    if (pr->sampler == 1 && rays_prep(&P) != 0) { unprep(&P); return -2; }
    int64_t per_cell = (int64_t)P.n_rbin * pr->n_theta * pr->n_phi;
    if (emit)
        for (int64_t p = pr->p_begin; p < pr->p_end; p++) {
            int64_t c = pr->sampler == 1 ? P.rcell[p / per_cell] : cell_of_packet(&P, p);
            int32_t z = (int32_t)(c / nxy);
            if (z < z_lo || z >= z_hi) continue;
            if (pr->sampler == 1) transport_ray(&P, p, S, spec, ledger, NULL, S_pi, heat, &dom);
            else transport_packet(&P, p, S, spec, ledger, NULL, S_pi, heat, &dom);
        }
    for (int64_t k = 0; k < n_in; k++) {
        xo_state st;
        state_unpack(bundle_in + k * XO_STATE_FIELDS, &st);
        trace(&P, &st, S, spec, ledger, NULL, S_pi, heat, &dom);
    }
    unprep(&P);
    *n_out = dom.n;
    return dom.n > out_cap ? -1 : 0;
}

/* The walk alone, for a test: the cells a straight path from p0 (cm, inside
 * cell idx0 of the spherical grid) along the unit vector n crosses, in order
 * (natural indices), and the path length at which it leaves each, by the
 * face solver and the cell step of the event loop; at most max cells.
 * Returns the number of cells when the path leaves the outer sphere, or -1
 * (max reached, or no face ahead). */
int64_t xo_sph_walk(const xo_problem *pb, const xo_params *pr, const double *p0, const double *n,
                    const int32_t *idx0, int64_t max, int64_t *cells, double *s_exit) {
    prep_t P;
    prep(&P, pb, pr);
    int32_t idx[3] = {idx0[0], idx0[1], idx0[2]};
    double s = 0.0;
    int64_t ret = -1;
    for (int64_t k = 0; k < max; k++) {
        int kind;
        double se = sph_exit(&P, p0, n, idx, s, &kind);
        cells[k] = ((int64_t)idx[2] * pb->ny + idx[1]) * pb->nx + idx[0];
        s_exit[k] = se;
        int crossed = sph_cross(pb, idx, kind);
        if (crossed == 1) { ret = k + 1; break; }
        if (crossed < 0) break;
        s = se;
    }
    unprep(&P);
    return ret;
}

/* Number of rays of the RAYS sampler (emitting cells x emitting bins x
 * viewers), or -1 if an emitting line lies outside the output grid. */
int64_t xo_ray_count(const xo_problem *pb, const xo_params *pr) {
    prep_t P;
    prep(&P, pb, pr);
    int64_t n = -1;
    if (rays_prep(&P) == 0) n = P.n_rcell * (int64_t)P.n_rbin * pr->n_theta * pr->n_phi;
    unprep(&P);
    return n;
}

/* Cell volumes (cm^3) of the spherical grid, natural order. */
int xo_cell_volumes(const xo_problem *pb, const xo_params *pr, double *vol) {
    prep_t P;
    prep(&P, pb, pr);
    if (pb->geometry == 1) memcpy(vol, P.vol, sizeof(double) * (size_t)P.ncell);
    else for (int64_t c = 0; c < P.ncell; c++) vol[c] = P.dx * P.dy * P.dz;
    unprep(&P);
    return 0;
}

/* Per-cell luminosity and packet quota as the transport sees them. */
int xo_emission(const xo_problem *pb, const xo_params *pr, double *Lc, int64_t *qoff) {
    prep_t P;
    prep(&P, pb, pr);
    int64_t nc = (int64_t)pb->nx * pb->ny * pb->nz;
    memcpy(Lc, P.Lc, sizeof(double) * (size_t)nc);
    memcpy(qoff, P.qoff, sizeof(int64_t) * (size_t)(nc + 1));
    unprep(&P);
    return 0;
}

/* tau_S and beta_S for every (cell, line) of a cell range (caller line order). */
int xo_tau_beta(const xo_problem *pb, int64_t c0, int64_t nc, double *tau, double *beta) {
    for (int64_t c = c0; c < c0 + nc; c++) {
        const double *n = pb->pops + c * pb->nlev;
        for (int32_t l = 0; l < pb->nline; l++) {
            double lam = pb->lambda_A[l] * 1e-8;
            double gl = pb->g[pb->lo[l]], gu = pb->g[pb->up[l]];
            double A = xo_einstein_A(lam, gl, gu, pb->f_lu[l]);
            double t = xo_tau_sobolev(A, gl, gu, lam, n[pb->lo[l]], n[pb->up[l]], pb->t);
            tau[(c - c0) * pb->nline + l] = t;
            if (beta) beta[(c - c0) * pb->nline + l] = xo_beta_sobolev(t);
        }
    }
    return 0;
}

/* Comoving frequency along a ray, for brute-force resonance checks. */
double xo_nu_cmf(double nu_lab, const double n[3], const double r[3], double s, double t) {
    double q[3] = {r[0] + s * n[0], r[1] + s * n[1], r[2] + s * n[2]};
    return nu_lab * (1.0 - dot3(n, q) / (XO_C * t));
}
