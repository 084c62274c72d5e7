/*
 * extrass.h - C ABI of the GB300 photoexcitation-rate transport library.
 *
 * The library computes photoexcitation rates by radiative transfer through a
 * 3D homologously expanding ejecta grid (van Baal & Jerkstrand, ExTraSS,
 * Sec. 2.3 "Radiative transfer" and Sec. 2.3.2 "Photoexcitation"), with the
 * per-cell, per-line estimator store split into Cartesian subdomains
 * (Sec. 2.4.1 "Domain decomposition").  All compute runs in CUDA kernels for
 * sm_103a; there is no CPU fallback.
 *
 * Conventions for every call:
 *   - Return 0 on success or a negative XT_E* code; xt_last_error() gives a
 *     message naming the offending argument.  Nothing traps; device-side loops
 *     are bounded and report overruns as status codes.
 *   - Array arguments are plain pointers that may point to host memory
 *     (pageable or pinned) or to device memory of the context's GPU; the
 *     library tells them apart with cudaPointerGetAttributes.  Inputs are only
 *     read during the call; outputs are written before the call returns (the
 *     call synchronises the context's stream).  The caller owns them.
 *   - Units are cgs; wavelengths are in Angstrom.  Floating point is FP64.
 *   - Cell index c = (iz * ny + iy) * nx + ix ("natural order").  Level index
 *     is global over ions: level i of ion z is level_off[z] + i.  Lines are
 *     addressed in the caller's order (the order given to load_atomic_data).
 *   - The context owns all device memory it allocates; xt_destroy frees it.
 *     A context is driven by one host thread at a time.
 */
#ifndef EXTRASS_H
#define EXTRASS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XT_OK 0
#define XT_EINVAL (-1)    /* bad argument (message names it) */
#define XT_ENOMEM (-2)    /* device allocation failed */
#define XT_ECUDA (-3)     /* a CUDA runtime call failed */
#define XT_ETIMEOUT (-4)  /* a bounded device loop hit its limit */
#define XT_ENOTCONV (-5)  /* an iterative solve did not converge */
#define XT_ESTATE (-6)    /* call made before the data it needs was loaded */

typedef struct xt_ctx xt_ctx;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (for example torch.cuda.current_stream().cuda_stream) or NULL for the
 * legacy default stream; every kernel of the context runs on it. */
int xt_create(xt_ctx **out, int device, void *cuda_stream);
void xt_destroy(xt_ctx *ctx);
const char *xt_last_error(const xt_ctx *ctx);

/* ---- grid (Sec. 2: snapshot, homologous v = r/t) ------------------------ */
#define XT_GEOM_CARTESIAN 0   /* the cube [-v_max t, v_max t]^3 of nx x ny x nz equal cells */
#define XT_GEOM_SPHERICAL 1   /* shells x polar sectors x azimuthal sectors (Sec. 2) */
typedef struct {
    int32_t nx, ny, nz;     /* cells per axis; the cube spans [-v_max t, v_max t]^3 */
    int32_t sx, sy, sz;     /* subdomains per axis (Sec. 2.4.1); must divide nx, ny, nz */
    double v_max;           /* cm/s */
    double t;               /* s since explosion */
    const double *rho;      /* [ncell] g/cm^3 (may be NULL) */
    const double *Te;       /* [ncell] K */
    const double *ne;       /* [ncell] cm^-3 */
    const double *L_cell;   /* [ncell] erg/s emitted in the flat-nu band (may be NULL) */
    const double *deposition; /* [ncell] erg/s/cm^3 non-thermal input (may be NULL) */
    double band_lo_A, band_hi_A;  /* emission band of L_cell, flat in frequency */
    /* Spherical grid (geometry = XT_GEOM_SPHERICAL; the paper's models are
     * spherical grids of radial shells, polar and azimuthal sectors, Sec. 2,
     * with subdomains that are azimuthal slices, Sec. 2.4.1): nx, ny, nz count
     * the cells in r, theta and phi, cell c = (iphi * ny + itheta) * nx + ir,
     * and sx, sy, sz block that index space as for the cube (phi slices:
     * sx = sy = 1).  r_edges [nx+1] velocities in cm/s, strictly increasing
     * from 0 to v_max (the shell radii are r_edges t); theta_edges [ny+1]
     * radians, strictly increasing from 0 to pi; phi_edges [nz+1] radians,
     * strictly increasing from 0 to 2 pi.  Host or device memory, read during
     * the call.  With XT_GEOM_CARTESIAN the three are ignored (may be NULL).
     * Every cell volume the readouts use (rates, the rate solve, line
     * emission) is then the spherical cell's, (r1^3 - r0^3) / 3 (cos theta0 -
     * cos theta1) (phi1 - phi0). */
    int32_t geometry;
    const double *r_edges, *theta_edges, *phi_edges;
} xt_grid_desc;
int init_grid(xt_ctx *ctx, const xt_grid_desc *g);

/* ---- atomic data (Sec. 2.2, 2.4 jagged level arrays) -------------------- */
typedef struct {
    int32_t n_ion;
    int32_t nline;
    const int32_t *level_off;   /* [n_ion+1] CSR offsets of each ion's levels */
    const double *E_level;      /* [nlev] erg above the ion's ground level */
    const double *g_level;      /* [nlev] statistical weights */
    const int32_t *lo, *up;     /* [nline] global lower / upper level (lo < up, same ion) */
    const double *lambda_A;     /* [nline] line wavelength, Angstrom */
    const double *f_lu;         /* [nline] absorption oscillator strength */
    const double *n_ion_density;/* [ncell*n_ion] cm^-3 (may be NULL) */
    const double *ups_down;     /* [nlev] sum_{j<u} Upsilon_ju; scatter mode only (may be NULL) */
    /* Photoionization (Sec. 2.3.1), all three NULL for none.  The lowest
     * pi_nlev[z] levels of ion z photoionize, with the hydrogenic cross
     * section of Eq. (sigma_OTSPI): sigma = 7.9e-18 cm^2 (lambda / lambda_ion)^3
     * (1 - E_u / chi_ion)^-1/2 / (charge + 1)^2 below the threshold wavelength
     * lambda_ion = h c / (chi_ion - E_u).  Photoionizing level k counts ion by
     * ion, lowest level first (k = sum_{z' < z} pi_nlev[z'] + i for level i of
     * ion z); at most XT_PI_MAX of them; every threshold chi_ion - E_u > 0. */
    const double *chi_ion;      /* [n_ion] erg, ionization energy from the ion's ground level */
    const int32_t *charge;      /* [n_ion] charge of the ion (0 neutral, 1 singly ionized, ...) */
    const int32_t *pi_nlev;     /* [n_ion] photoionizing levels of the ion (0..its level count) */
} xt_atom_desc;
#define XT_PI_MAX 256
int load_atomic_data(xt_ctx *ctx, const xt_atom_desc *a);

/* Level populations [ncell][nlev] in cm^-3 (natural cell order). */
int set_populations(xt_ctx *ctx, const double *pops);
int get_populations(xt_ctx *ctx, double *pops, size_t n_cap);

/* ---- A1: Sobolev optical depth and escape probability ------------------
 * tau_S, Eq. (tau_Sobolev) (App. A.1), and beta_S = (1 - e^-tau)/tau,
 * Eq. (beta_Sobolev), taken as 1 for tau <= 0 (empty lower level or
 * population inversion: no trapping), for cells [cell_begin, +n_cells) x all
 * lines, written [n_cells][nline] in the caller's line order.  beta may be
 * NULL. */
int get_sobolev_tau(xt_ctx *ctx, int64_t cell_begin, int64_t n_cells, double *tau, double *beta);

/* ---- A2-A6: transport (Secs. 2.3, 2.3.2, 2.4.1) ------------------------ */
#define XT_MODE_ATTEN 0     /* paper: attenuate by 1 - e^-tau at every line (default) */
#define XT_MODE_SCATTER 1   /* absorb-or-scatter with fluorescent re-emission */
#define XT_EMIT_BAND 0      /* flat-in-nu band emission with L_cell */
#define XT_EMIT_LINES 1     /* line emissivity A_ul dE beta N_u, Eq. (thin_emissivity) */
#define XT_PKT_FIELDS 11    /* per-packet record, see xt_transport_params.packet_records */
/* Pre-reduce the estimator increments (Sec. 2.3.2) per warp: lanes adding to
 * the same (cell, line) slot are summed and one FP64 atomic adds the sum
 * (attenuation mode with Monte Carlo packets, without photoionization; other
 * passes ignore the flag).  Off by default: one atomic per increment measured
 * faster on GB300.  Results differ only in the order of the additions. */
#define XT_FLAG_WARP_REDUCE 1
/* XT_SAMPLER_RAYS without photoionization: stage, per batch of rays of
 * consecutive bins of one cell, the frequency window of the sorted line list
 * that those rays can reach in shared memory (bulk copies; Sec. 2.3's rays all
 * start at their bin's frequency) and read the line records from there.
 * Off by default: with the whole line list resident in the 129 MB L2 it
 * measured 23 % slower at the paper-scale line density and 2 % slower with
 * 1e7 times thinner lines.  Results are the same. */
#define XT_FLAG_RAYS_STAGED 2

typedef struct {
    int64_t n_packets;      /* N of the whole emission (sets the per-cell quota) */
    int64_t packet_begin;   /* first packet id transported by this call */
    int64_t packet_count;   /* number of packets; <0 means all from packet_begin */
    uint64_t seed;          /* Philox4x64-10 key (seed, 0); counter (packet, draw, 0, 0) */
    int32_t mode;           /* XT_MODE_* */
    int32_t emission;       /* XT_EMIT_* */
    double tau_min;         /* lines are interaction points only above this tau (1e-4) */
    double e_cut;           /* stop below this fraction of the starting energy (1e-6) */
    int32_t n_theta, n_phi; /* viewing-direction bins (20, 20) */
    double spec_lam0_A;     /* first edge of the output grid */
    double spec_dlog;       /* bin edges lam0 (1 + dlog)^k (1e-3) */
    int32_t spec_nbins;
    int32_t accumulate;     /* 0: zero estimators, spectrum and ledger first */
    int64_t max_events;     /* per-packet event guard (XT_ETIMEOUT when hit) */
    int32_t subdomain_rounds; /* 0: the whole grid is one resident domain.  1: each
                             * subdomain of init_grid is a domain of its own; a packet
                             * that crosses into another subdomain is queued and
                             * carried on in the next round (Sec. 2.4.1 bundles) */
    int32_t flags;          /* XT_FLAG_* bits, 0 by default */
    /* Optional [packet_count][XT_PKT_FIELDS] doubles: fate (0 escaped,
     * 1 dropped below e_cut, 2 collisionally destroyed, 3 guard), events,
     * N_final, escaped lab energy, viewer, lambda bin, interactions, emitting
     * cell, N0, comoving emission frequency, final lab frequency. */
    double *packet_records;
    /* XT_SAMPLER_MC: n_packets Monte Carlo packets by the cells' integer quota.
     * XT_SAMPLER_RAYS (Sec. 2.3): from the middle of every emitting cell, for
     * every bin of the output grid (spec_lam0_A, spec_dlog, spec_nbins) that
     * holds emission, one ray towards every viewer, along the centre direction
     * of the viewer's (theta, phi) bin, carrying the cell's emission in the bin
     * times dOmega_k / 4 pi, at the bin's reddest feature (band emission: the
     * red edge of the bin's overlap with the band; line emission: the reddest
     * line in the bin, the ray starting past it).  No random numbers; ray r =
     * (emitting-cell rank, bin rank, viewer) row-major over cells with
     * emission in natural order, emitting bins in wavelength order and
     * viewers; n_packets is ignored and packet_begin / packet_count address
     * rays (xt_transport_stats.rays gives their number; packet_count = 0 only
     * counts them).  A ray whose cell has no emission in its bin is empty:
     * record fate 4, not traced.  Attenuation mode, without subdomain rounds,
     * with the estimator store on the device; every line must lie on the
     * output grid for line emission (XT_EINVAL otherwise). */
    int32_t sampler;
} xt_transport_params;
#define XT_SAMPLER_MC 0
#define XT_SAMPLER_RAYS 1

/* Ledger and timing of the last run_transport (photons/s and erg/s). */
typedef struct {
    double emitted_N, escaped_N, absorbed_N, dropped_N;
    double emitted_E, escaped_E, out_of_band_E;
    double events, tests, guard, thermal_E, interactions, abs_E_cmf, reemit_E_cmf;
    double transport_ms;    /* device time of the whole pass (clear, emission, trace, escape) */
    double zero_ms;         /* clearing the estimator store (overlaps the first emission) */
    double rounds;          /* trace rounds executed (1 per chunk without subdomain rounds) */
    double queued;          /* packets handed between subdomains */
    double emit_ms, trace_ms, escape_ms;   /* summed device time per kernel kind */
    double kernels;         /* kernels launched by this call */
    double photoionized_N;  /* photons absorbed by photoionization (Sec. 2.3.1) */
    double photoionized_E;  /* their energy at absorption (comoving), erg/s */
    double rays;            /* XT_SAMPLER_RAYS: rays of the whole enumeration */
} xt_transport_stats;

/* On a spherical grid (XT_GEOM_SPHERICAL) run_transport takes attenuation
 * mode with Monte Carlo packets or rays (XT_SAMPLER_RAYS: each ray starts at
 * the middle of its cell's r, theta and phi ranges), with photoionization
 * on every segment, without subdomain rounds, with the estimator store on the
 * device (dense or compact rows; run_transport_domain with phi-slice
 * domains); other passes return XT_EINVAL.
 * Packets start uniformly in their cell's volume (r^3, cos theta and phi
 * uniform) and walk from cell to cell through the shells' spheres, the polar
 * edges' cones (the plane z = 0 for theta = pi/2) and the azimuthal edges'
 * half-planes; every crossing is taken from the packet's emission point and
 * direction, so that a face met twice gives the same path length both times. */
int run_transport(xt_ctx *ctx, const xt_transport_params *p, xt_transport_stats *out);

/* Where the estimator store lives (Sec. 2.4.1: the photoexcitation store is
 * split by domain because the whole of it does not fit in one node's memory).
 * host_groups = 0 (default): on the device, ncell * nline doubles.  host_groups
 * = G > 0: in pinned host memory, in G groups of sz/G subdomain layers along z
 * (whole x-y layers of nz/G cells; G must divide sz); the device holds one
 * group's slab (ncell * nline / G doubles) at a time.  run_transport then
 * traces in rounds: every group with packets is staged (its slab from host
 * memory, zeros on its first visit in a pass), its packets traced until they
 * leave the group, escape or end, and the slab written back; trajectories and
 * results are those of the device-resident store.  get_estimators and
 * get_photoexcitation_rates stage the groups they read; solve_nlte with
 * estimator rates solves group by group, each group's slab staged (no graph
 * replay, no autotuning there); train_surrogate with estimator inputs
 * returns XT_ESTATE for a host-held store.
 * host_groups = XT_STORE_COMPACT_ROWS (-1): on the device, with rows only for
 * the cells that have populations (a cell without matter has no optical depth
 * and gets no estimator; 1.1e6 of the 2.1e6 cells of a 128^3 cube around a
 * sphere): the store shrinks by the empty cells' share; readouts give zeros
 * for the others.  The row map follows the populations of each pass.
 * Frees the current store (host and device); the next run_transport allocates. */
#define XT_STORE_COMPACT_ROWS (-1)
int set_estimator_store(xt_ctx *ctx, int32_t host_groups);

/* Raw estimators S [n_cells][nline] (photons/s absorbed, divided by f_corr),
 * cells [cell_begin, +n_cells), caller line order. */
int get_estimators(xt_ctx *ctx, int64_t cell_begin, int64_t n_cells, double *S);

/* ---- A7: rates (Sec. 2.3.2, Sec. 2.3.1 Gamma = N_abs / N_i) ------------
 * R_lu = S / (n_l V), R_ul = (g_l/g_u) R_lu (detailed balance), Jbar =
 * R_lu / B_lu with B_lu = 4 pi (pi e^2 / m_e c) f_lu / (h nu).  Each output
 * [n_cells][nline]; any may be NULL; slots with n_l = 0 give 0. */
int get_photoexcitation_rates(xt_ctx *ctx, int64_t cell_begin, int64_t n_cells,
                              double *R_lu, double *R_ul, double *Jbar);

/* ---- photoionization rates (Sec. 2.3.1) ---------------------------------
 * After an attenuation-mode run_transport with photoionization data loaded:
 * Gamma [n_cells][n_pi] (s^-1), Gamma_PI,k = N_abs,k / (n_k V), the photons
 * absorbed by photoionizing level k in the cell over the atoms in that level
 * (0 where n_k = 0), levels in the order of xt_atom_desc; heating [n_cells]
 * (erg/s), the absorbed photons' energy above their thresholds.  Either may be
 * NULL.  The same rules for host/device pointers as everywhere; XT_ESTATE
 * without a transport pass with photoionization. */
int get_photoionization_rates(xt_ctx *ctx, int64_t cell_begin, int64_t n_cells, double *Gamma,
                              double *heating);

/* ---- A5: spectrum (Secs. 2, 2.3) ----------------------------------------
 * kind 0: escaped lab-frame energy per (viewer, bin) [n_theta*n_phi][nbins], erg/s
 * kind 1: isotropic-equivalent L_lambda = 4 pi/dOmega_k E/dlambda, same shape, erg/s/A
 * kind 2: angle-summed L_lambda [nbins], erg/s/A */
int get_spectrum(xt_ctx *ctx, int32_t kind, double *out, size_t n_cap);

/* ---- A8: statistical-equilibrium level populations (Sec. 2.2, Sec. 2.3.2) --
 * For every (cell, ion): rates between the ion's levels held fixed (radiative
 * decay A_ul beta_S, photoexcitation R_lu and stimulated emission
 * (g_l/g_u) R_lu, collisions C_ul = 8.629e-6 Upsilon n_e/(g_u sqrt Te) and
 * C_lu by detailed balance for every pair, a non-thermal excitation term from
 * the deposition), equilibrium of every level with the equation of the ground
 * level replaced by sum n = n_z, solved as one linear system.  All systems go
 * through one persistent launch, longest first.
 *   XT_PREC_FP64     LU with partial pivoting in FP64 (the plain method).
 *   XT_PREC_FP32_IR  the system scaled by the warm start (columns) and row
 *                    maxima, LU in FP32, refined in FP64 (residual, update)
 *                    until the error every level keeps after the last
 *                    correction is below tol (relative): |d_k|, or d_k^2 /
 *                    |d_(k-1)| where the level's successive corrections d
 *                    contract by half or more.
 *   XT_PREC_TF32_IR  as XT_PREC_FP32_IR with the rank-nb trailing updates of
 *                    the blocked LU on the tensor cores (TF32 operands, FP32
 *                    accumulation); more refinement steps, same FP64 result.
 *   XT_PREC_BF16_IR  as XT_PREC_TF32_IR with BF16 operands (8-bit
 *                    significands): the factors are coarser, so refinement
 *                    takes more steps, and a system whose refinement does not
 *                    reach tol within max_iter steps is solved in FP64.
 * Rates: XT_RATES_ESTIMATORS uses the last transport pass (R_lu = S/(n_l V));
 * XT_RATES_JBAR illuminates every line with the external field
 * J_nu = jbar_W B_nu(jbar_TR), of which a Sobolev region absorbs the part
 * beta_S: R_lu = beta_S B_lu J_nu (the 1 - e^-tau absorbed fraction that the
 * Sec. 2.3.2 estimator counts).  Optical depths for beta_S
 * use the context's populations.  The warm start (scaling and first guess) is
 * the context's populations (XT_WARM_CURRENT), Boltzmann populations
 * (XT_WARM_LTE) or warm_in [ncell][nlev] (XT_WARM_GIVEN). */
#define XT_PREC_FP64 0
#define XT_PREC_FP32_IR 1
#define XT_PREC_TF32_IR 2   /* as FP32_IR, the trailing updates of the LU on the tensor cores (TF32) */
#define XT_PREC_BF16_IR 3   /* the same with BF16 operands */
#define XT_RATES_NONE 0
#define XT_RATES_ESTIMATORS 1
#define XT_RATES_JBAR 2
#define XT_WARM_CURRENT 0
#define XT_WARM_LTE 1
#define XT_WARM_GIVEN 2
#define XT_WARM_SURROGATE 3 /* the population surrogate's prediction (see below) */
#define XT_SE_OK 1          /* status bits per (cell, ion) */
#define XT_SE_FALLBACK 2    /* FP32 factor singular or refinement not converged; solved in FP64 */
#define XT_SE_SINGULAR 4    /* zero pivot in the FP64 factor */
#define XT_SE_NOCONV 8      /* Newton steps ran out (populations: the last iterate) */
typedef struct {
    int32_t precision;      /* XT_PREC_* */
    int32_t rates;          /* XT_RATES_* */
    int32_t warm;           /* XT_WARM_* */
    int32_t max_iter;       /* refinement steps (FP32_IR) */
    double tol;             /* refinement stop: max |dn| / n over kept levels */
    double jbar_W, jbar_TR; /* XT_RATES_JBAR */
    double eta_nt;          /* non-thermal excitation efficiency (0.5) */
    const int32_t *levels_used; /* [ncell*n_ion] levels kept per (cell, ion) (NULL: all) */
    const double *warm_in;  /* XT_WARM_GIVEN: [ncell][nlev] */
    const double *upsilon;  /* per ion, row-major [L_z][L_z] (entry [l][u], l < u),
                               concatenated over ions; required */
    int32_t use_graph;      /* replay the launch from a captured CUDA graph */
    int32_t autotune;       /* pick panel widths per level-count bucket by timing */
    /* Newton-Raphson on the optical depths (Sec. 2.2): newton_max = 0 solves the
     * linear system with beta_S from the context's populations; > 0 makes beta_S
     * a function of the solution and takes up to newton_max steps from the warm
     * start.  Each step factors the Jacobian (M plus every line's derivative of
     * its net downward flow through beta_S) in the chosen precision, with an
     * FP64 residual, for the correction d (refined until its last update is
     * below max(tol, newton_tol / 100) of every level's population: the fixed
     * point is set by the FP64 right-hand side, so the step needs no more).
     * With r = max |d_i| / n_i over
     * levels with n_i >= 1e-30 n_z: stop when r <= newton_tol; else every level
     * moves by the factor 1 + lam d_i / n_i kept within [1/newton_maxvar,
     * newton_maxvar], lam = 1 once r <= 0.1, before that 0.95, then 0.75, 0.5,
     * 0.25, 0.05 from steps 10, 35, 50, 90 on (Sec. 2.2).  Estimator rates stay
     * fixed per atom. */
    int32_t newton_max;
    double newton_tol;      /* 1e-6 */
    double newton_maxvar;   /* 10: largest change factor of a population per step */
} xt_nlte_params;
typedef struct {
    double systems, fp64_fallbacks, singular, max_iter_used, mean_iter;  /* iterations:
                               refinement steps, or Newton steps when newton_max > 0 */
    double solve_ms;        /* device time of the persistent launch */
    double assemble_flops, lu_flops;   /* algorithmic flop counts of the launch */
    int32_t panel_width[8]; /* chosen per bucket of 64 levels */
    double not_converged;   /* systems with XT_SE_NOCONV */
} xt_nlte_stats;
/* New populations into the context (and into pops_out [ncell][nlev] natural
 * order, levels beyond levels_used set to 0, when not NULL); status_out
 * [ncell*n_ion] (may be NULL). */
int solve_nlte(xt_ctx *ctx, const xt_nlte_params *p, double *pops_out, int32_t *status_out,
               xt_nlte_stats *stats);

/* ---- A9: population surrogate (no paper counterpart: it warm-starts A8) ----
 * A multilayer perceptron predicts log10(n_i / n_z) / 10 of every level of a
 * cell from log10 n_e, log10 Te, log10 of the deposition, per ion the mean
 * log10 Jbar of its lines in 32 log-lambda bins, and per ion log10 n_z / 10
 * (3 + 33 n_ion inputs: the 32 n_ion Jbar bins, then the n_ion densities; nlev
 * outputs).  Hidden layers GELU (tanh form), linear output, masked mean squared
 * error, Adam on FP32 master weights; every matrix product in BF16 on the
 * tensor cores with FP32 accumulation.  Weights are one flat FP32 vector:
 * W_1 [n_in][h], b_1, W_2, b_2, ..., W_out, b_out (W row-major [fan_in][fan_out]).
 * A bad prediction costs only refinement or Newton steps: solve_nlte refines (or falls
 * back to FP64) whatever the warm start.  Training (surrogate_train_step,
 * train_surrogate) runs in one persistent cooperative kernel per call (every
 * step of a call in one launch, one CTA per SM, tcgen05 BF16 products); its
 * grid barriers and MMA completions are waited on with bounded polls, after
 * which the call returns XT_ETIMEOUT.  Prediction uses BF16 products with FP32
 * accumulation (mma.sync).  At most 8 layers (n_sizes <= 9): XT_EINVAL. */
int surrogate_init(xt_ctx *ctx, const int32_t *sizes, int32_t n_sizes, uint64_t seed);
/* set != 0: load weights from flat; else copy them out.  n_cap in floats. */
int surrogate_weights(xt_ctx *ctx, int32_t set, float *flat, size_t n_cap);
/* One forward and backward pass on a batch: X [B][n_in], T and mask [B][n_out]
 * (FP32, host or device); update != 0 applies one Adam step (lr).  Gradients of
 * the flat parameter vector into grads_out (may be NULL), loss into loss_out. */
int surrogate_train_step(xt_ctx *ctx, const float *X, const float *T, const float *mask, int64_t B,
                         double lr, int32_t update, float *grads_out, double *loss_out);
int surrogate_predict(xt_ctx *ctx, const float *X, int64_t B, float *Y);
typedef struct {
    int32_t epochs, batch;
    double lr;
    int32_t n_hidden, n_layers;   /* network made on first use: 3 x 256 */
    uint64_t seed;
    int32_t rates;                /* how the Jbar inputs are formed (XT_RATES_*) */
    double jbar_W, jbar_TR;
    const int32_t *levels_used;   /* [ncell*n_ion] or NULL */
} xt_train_params;
typedef struct {
    double first_loss, last_loss, steps, samples, train_ms;
} xt_train_stats;
/* Train on every cell of the context: inputs from its grid and radiation
 * field, targets its current populations (the result of solve_nlte). */
int train_surrogate(xt_ctx *ctx, const xt_train_params *p, xt_train_stats *stats);

/* ---- A10: the coupled NLTE / transport loop -------------------------------
 * Sec. 2 alternates the NLTE solver and the ray tracing; Sec. 2.2 solves the
 * populations with the transport's photoexcitation rates held fixed; Sec.
 * 2.3.2 forms those rates from the estimators.  One outer step: a transport
 * pass (*transport, accumulate forced to 0) from the context's populations
 * n_k, solve_nlte (*nlte, rates forced to XT_RATES_ESTIMATORS, warm start the
 * current populations, so newton_max > 0 solves the optical depths with the
 * populations), then n_{k+1} = n_k^(1-alpha) s_k^alpha (alpha = 1: s_k), and
 * change = max |n_{k+1} - n_k| / n_k over levels with n >= floor n_z in either
 * iterate.  Stops when change <= tol or after max_outer steps; the context
 * keeps n_{k+1}.  Start populations: the context's (XT_WARM_CURRENT),
 * Boltzmann (XT_WARM_LTE, levels_used of *nlte), start_in [ncell][nlev]
 * natural order (XT_WARM_GIVEN), or the surrogate's prediction with its Jbar
 * inputs from nlte->jbar_W, jbar_TR (XT_WARM_SURROGATE).  Synchronous; the
 * transport keeps its seed every step, so a step is a deterministic map. */
typedef struct {
    const xt_transport_params *transport;
    const xt_nlte_params *nlte;
    int32_t start;          /* XT_WARM_* */
    const double *start_in; /* XT_WARM_GIVEN */
    double alpha;           /* 1 */
    double tol;             /* 1e-3 */
    double floor;           /* 1e-20 */
    int32_t max_outer;
} xt_coupled_params;
typedef struct {
    int32_t outer, converged;
    double last_change;
    double wall_ms;         /* host clock over the whole call, start included */
    double start_ms;        /* start populations (surrogate inference, Boltzmann) */
    double transport_ms, solve_ms, mix_ms;   /* device time summed over steps */
    double newton_steps;    /* mean Newton steps per system, summed over steps */
    double max_newton_steps, not_converged, fp64_fallbacks;
    double change[64];      /* change after each of the first 64 steps */
} xt_coupled_stats;
int run_coupled(xt_ctx *ctx, const xt_coupled_params *p, xt_coupled_stats *stats);

/* ---- numerical self-test (no paper counterpart: checks device primitives) --
 * GB300 runs FP64 arithmetic at about 1/64 of its FP32 rate, so the hot
 * transcendental and division steps are the library's own fixed-point routines
 * on the integer pipe.  This evaluates one of them for n inputs (host or device
 * arrays; y0, y1 and, when not NULL, r0, r1 hold n values each):
 *   kind 0: x[i] > 0, the attenuation factors of a line event: y0 = e^-x,
 *           y1 = 1 - e^-x; r0, r1 = CUDA's exp(-x), -expm1(-x).
 *   kind 1: 0 <= x[i] < 1 a multiple of 2^-53, the emission azimuth:
 *           y0 = sin(2 pi x), y1 = cos(2 pi x); r0, r1 = CUDA's sin, cos.
 *   kind 2: x holds n pairs (a, b) of positive normal numbers, the emission's
 *           quotients: y0 = a / b of the integer-pipe routine, r0 = CUDA's
 *           IEEE a / b; y1, r1 are set to 0.
 *   kind 3: x holds n pairs (u, v), multiples of 2^-53 in [0, 1), the
 *           isotropic emission direction with mu = 2u - 1, phi = 2 pi v:
 *           y0 = n_x, y1 = n_y, r0 = n_z; r1 is set to 0.
 * Runs on the current device, synchronously, with temporaries of its own.
 * XT_EINVAL for a NULL x, y0 or y1, n < 0 or an unknown kind. */
int xt_selftest_fixed(int32_t kind, const double *x, int64_t n, double *y0, double *y1,
                      double *r0, double *r1);

/* Check of the tensor-core path that the batched LU's trailing updates take
 * (tcgen05 MMA, kind::tf32, operands in shared memory, accumulator in TMEM):
 * D [128][N] = A B^T for A [128][32] and B [N][32] (host arrays, row-major,
 * FP32), with A and B rounded to TF32 (nearest, ties away from zero) and the
 * products summed in FP32 by the tensor core.  N a multiple of 16 in
 * [16, 256].  Runs one CTA on `device`, synchronously, with temporaries of its
 * own.  XT_EINVAL for a bad N or a NULL array; XT_ETIMEOUT if the MMA's
 * completion was not seen within its bounded wait. */
int xt_selftest_tc(int device, int N, const float *A, const float *B, float *D);

/* The same check for the BF16 leg (kind::f16 with BF16 operands): A and B
 * rounded to BF16 (nearest, ties to even), products summed in FP32.  Same
 * arguments, layout and errors as xt_selftest_tc. */
int xt_selftest_tc_bf16(int device, int N, const float *A, const float *B, float *D);

/* ---- transport without device allocation (no paper counterpart) -----------
 * For callers that cannot call cudaMalloc: programs whose device memory is
 * handed out once at start-up by another framework's allocator (a second
 * allocator would fragment or overrun its pool), or embedders held to a fixed
 * device-memory budget.  run_transport_noalloc does one attenuation-mode pass
 * (band emission, the whole grid one domain) like run_transport, but it makes
 * no device allocation: its working memory is a file-scope device array of
 * XT_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits, and it calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *   - The caller passes the inputs and the outputs.  pops, S and spec must be
 *     device memory; the other arrays may be host or device memory.
 *   - Limits: at most XT_NOALLOC_MAX_CELLS cells, XT_NOALLOC_MAX_LINES lines,
 *     2..65536 levels, 1..1024 cells per axis; larger sizes return XT_EINVAL
 *     with a message in errbuf.  Packets are traced in chunks of
 *     XT_NOALLOC_CHUNK, so n_packets is not limited.
 *   - On its first call on a device it looks up the device address of the
 *     array (cudaGetSymbolAddress, with that device current); make that first
 *     call before any stream capture starts.
 *   - Every call shares the one array (and fixed host staging buffers), which
 *     keeps the last call's contents; each call clears what must start at zero.
 *     Calls that overlap on the GPU, or run from several host threads at once,
 *     race with each other: issue them one after another.
 *   - Outputs: S [ncell][nline] (natural cell order, caller line order) gets the
 *     photoexcitation estimators, photons/s absorbed divided by f_corr, as
 *     get_estimators returns them; spec [n_theta*n_phi][spec_nbins] the escaped
 *     lab-frame energy per bin, as get_spectrum kind 0; `out` the ledger (the
 *     timing fields are 0).
 *   - The call is synchronous: it waits on `cuda_stream` after staging the
 *     inputs, after every chunk and at the end, and reads counters back to the
 *     host between chunks. */
#define XT_NOALLOC_SCRATCH_BYTES (32u << 20)
#define XT_NOALLOC_MAX_CELLS 65536
#define XT_NOALLOC_MAX_LINES 16384
#define XT_NOALLOC_CHUNK 131072
typedef struct {
    int32_t nx, ny, nz;
    double v_max, t;
    const double *L_cell;         /* [ncell] erg/s in the flat-nu band */
    double band_lo_A, band_hi_A;
    int32_t nlev, nline;
    const double *g_level;        /* [nlev] */
    const int32_t *lo, *up;       /* [nline] */
    const double *lambda_A, *f_lu;/* [nline] */
    const double *pops;           /* [ncell][nlev] device, natural order */
    int64_t n_packets;
    uint64_t seed;
    double tau_min, e_cut;
    int32_t n_theta, n_phi;
    double spec_lam0_A, spec_dlog;
    int32_t spec_nbins;
    int64_t max_events;
    double *S;                    /* out, device [ncell][nline] */
    double *spec;                 /* out, device [n_theta*n_phi][spec_nbins] */
} xt_noalloc_transport;
int run_transport_noalloc(const xt_noalloc_transport *a, void *cuda_stream,
                          xt_transport_stats *out, char *errbuf, size_t errlen);

/* ---- spatial decomposition across processes (Sec. 2.4.1) ------------------
 * One process per GPU owns a domain, the cells with z in [z_lo, z_hi) (whole
 * x-y layers), and holds the estimators, photoionization rates and spectrum
 * tallies that arise in it; packets that cross into another domain are handed
 * to that domain's process as bundles of packet states (the paper's managers
 * exchange bundles of rays between nodes, App. B).  One call: with emit != 0
 * the packets of [packet_begin, packet_begin + packet_count) of the
 * n_packets-packet emission whose emitting cell lies in the domain start
 * here; the n_in packets of bundle_in (from other domains) resume; every
 * packet is traced until it escapes, ends, or enters a cell outside the
 * domain, and those are written to bundle_out (XT_BUNDLE_FIELDS doubles each;
 * entry[XT_BUNDLE_CELL] holds the cell it entered, ix + 1024 iy + 1048576 iz,
 * which tells the caller the receiving domain).  *n_out is their number; if
 * it exceeds out_cap nothing is written past out_cap and XT_EINVAL is
 * returned (call again with a larger buffer after the same inputs: the pass
 * is deterministic).  accumulate works as in run_transport (0 on a domain's
 * first call of a pass, 1 on the calls that resume its bundles).  Attenuation
 * mode with Monte Carlo packets, or with rays (XT_SAMPLER_RAYS) on a
 * spherical grid, where a domain emits the rays of its own emitting cells;
 * the estimator store on the device, no packet records.  Results summed over the domains equal run_transport's on
 * the whole grid (up to the order of additions); a packet's trajectory does
 * not depend on the decomposition.  bundle_in and bundle_out may be host or
 * device memory.  An entry of bundle_in whose cell lies outside the grid, or
 * whose line cursor (entry[XT_BUNDLE_CELL + 1]) lies outside [0, nline], makes
 * the call return XT_EINVAL before anything is traced.  On a spherical grid
 * the domains are slices of whole azimuthal sectors (z is the phi index; the
 * paper's decomposition of its spherical grid, Sec. 2.4.1), phi wrapping
 * around, and a handed-on state carries the packet's path from its emission
 * point. */
#define XT_BUNDLE_FIELDS 24
#define XT_BUNDLE_CELL 17
int run_transport_domain(xt_ctx *ctx, const xt_transport_params *p, int32_t z_lo, int32_t z_hi,
                         int32_t emit, const double *bundle_in, int64_t n_in, double *bundle_out,
                         int64_t out_cap, int64_t *n_out, xt_transport_stats *out);

typedef struct {
    int64_t ncell, nlev, nline, n_ion;
    int64_t spec_views, spec_bins;
    int64_t store_bytes;    /* device bytes of the estimator store */
    int64_t n_pi;           /* photoionizing levels */
} xt_sizes;
int get_sizes(xt_ctx *ctx, xt_sizes *out);

#ifdef __cplusplus
}
#endif
#endif /* EXTRASS_H */
