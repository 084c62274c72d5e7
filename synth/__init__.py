"""Seeded synthetic inputs for the photoexcitation-transport workloads.

This module only *produces inputs*: grids, atomic models, starting level
populations and emission luminosities.  It holds none of the method's
arithmetic (no optical depths, escape probabilities, transport, estimators,
rates or rate-matrix algebra), so both the CPU oracle and the CUDA library
can consume what it writes without sharing any computation.

Workloads (all cgs, wavelengths in Angstrom):

* ``uniform_sphere`` - 16^3 Cartesian velocity cells of a homologous flow
  (v = r/t, v_max = 5000 km/s, t = 200 d), uniform density 1e-15 g/cm^3 inside
  |v| <= v_max, Te = 5000 K, ne = 1e7 cm^-3; one synthetic ion with 20 levels
  evenly spaced over 0-10 eV; 100 lines with log-uniform wavelengths in
  3000-10000 A and log-uniform oscillator strengths in 1e-4..1; uniform
  emissivity flat in frequency over 2900-10000 A; 1e5 packets.
* ``clumpy_onion`` - 64^3 cells, lognormal density clumps (sigma = 0.5,
  Gaussian correlation length 4 cells) in four onion zones
  (Fe-group / O / He / H), 10 synthetic ions of 50-200 levels, 1e5 lines
  (1000 A - 3 um, f in 1e-6..1), 1e8 packets, 8^3 subdomains.

The paper's explosion models (3D neutrino-driven models, the 1D-turned-3D
model and the public toy model it compares against) are not available; these
recipes stand in for their shapes and sizes (Section 3 of the paper: 17,100
zones, up to 100 levels per ion).
"""
from __future__ import annotations

import dataclasses
import numpy as np

# Physical constants (cgs).  Used only to express the input recipes (eV to erg,
# ion masses, Boltzmann starting populations), never for transport.
C_LIGHT = 2.99792458e10
H_PLANCK = 6.62607015e-27
K_BOLTZ = 1.380649e-16
EV = 1.602176634e-12
M_U = 1.66053906660e-24
DAY = 86400.0


@dataclasses.dataclass
class Workload:
    """Everything one transport pass (and the rate solves) consumes.

    Cell index c = (iz * ny + iy) * nx + ix ("natural" order).  Level indices
    are global: level ``level_off[z] + i`` is level i of ion z.  Lines are in
    generation order (unsorted); ``lo``/``up`` are global level indices.
    """
    name: str
    nx: int
    ny: int
    nz: int
    v_max: float          # cm/s; the cube spans [-v_max t, v_max t]^3
    t: float              # s since explosion
    rho: np.ndarray       # [ncell] g/cm^3
    Te: np.ndarray        # [ncell] K
    ne: np.ndarray        # [ncell] cm^-3
    deposition: np.ndarray  # [ncell] erg/s/cm^3 (non-thermal energy input)
    L_cell: np.ndarray    # [ncell] erg/s emitted by the cell (band emission)
    band_A: tuple         # (lambda_lo, lambda_hi) of the flat-in-nu emission band
    n_ion: int
    level_off: np.ndarray  # [n_ion+1] int32
    E_level: np.ndarray   # [nlev] erg above the ion's ground level
    g_level: np.ndarray   # [nlev] statistical weights
    ion_mass_u: np.ndarray  # [n_ion] mass numbers
    n_ion_density: np.ndarray  # [ncell, n_ion] cm^-3
    lo: np.ndarray        # [nline] int32 global lower level
    up: np.ndarray        # [nline] int32 global upper level
    lambda_A: np.ndarray  # [nline] line wavelength, Angstrom
    f_lu: np.ndarray      # [nline] absorption oscillator strength
    pops: np.ndarray      # [ncell, nlev] cm^-3 starting level populations
    upsilon_seed: int     # seed for collision strengths (see collision_strengths)
    n_packets: int
    seed: int
    subdomains: tuple     # (sx, sy, sz) number of subdomains per axis
    spec_band_A: tuple    # (lambda0, n_bins) of the 0.1 % log output grid
    meta: dict = dataclasses.field(default_factory=dict)
    upsilon: list = None          # per ion [L_z, L_z] collision strengths (entry [l, u], l < u)
    levels_used: np.ndarray = None  # [ncell, n_ion] levels kept per (cell, ion); None = all
    jbar_W: float = 0.0           # mean intensity model W B_nu(T_R) for the rate solves
    jbar_TR: float = 0.0
    # spherical grid (geometry "spherical"): cell edges in velocity (cm/s) and
    # angle; nx, ny, nz are then the radial, polar and azimuthal cell counts
    geometry: str = "cartesian"
    r_edges: np.ndarray = None
    theta_edges: np.ndarray = None
    phi_edges: np.ndarray = None
    # photoionization data (None: no photoionizing levels): per ion the
    # ionization energy from its ground level [erg], its charge, and how many of
    # its lowest levels photoionize
    chi_ion: np.ndarray = None
    charge: np.ndarray = None
    pi_nlev: np.ndarray = None

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nlev(self) -> int:
        return int(self.level_off[-1])

    @property
    def nline(self) -> int:
        return int(self.lo.shape[0])


def cell_centres(n: int, v_max: float) -> np.ndarray:
    """Velocity of the centres of n equal cells spanning [-v_max, v_max]."""
    return -v_max + (np.arange(n) + 0.5) * (2.0 * v_max / n)


def _speed_grid(n: int, v_max: float) -> np.ndarray:
    v = cell_centres(n, v_max)
    vz, vy, vx = np.meshgrid(v, v, v, indexing="ij")   # natural order: x fastest
    return np.sqrt(vx * vx + vy * vy + vz * vz).reshape(-1)


def lte_populations(n_ion_density, level_off, E_level, g_level, Te):
    """Boltzmann populations within each ion at the cell temperature.

    Starting populations for the transport-only workloads: n_i = n_z g_i
    exp(-E_i / k Te) / sum_j g_j exp(-E_j / k Te).
    """
    ncell, n_ion = n_ion_density.shape
    nlev = int(level_off[-1])
    pops = np.zeros((ncell, nlev))
    kT = K_BOLTZ * np.where(Te > 0, Te, 1.0)
    for z in range(n_ion):
        a, b = int(level_off[z]), int(level_off[z + 1])
        w = g_level[a:b][None, :] * np.exp(-E_level[a:b][None, :] / kT[:, None])
        pops[:, a:b] = n_ion_density[:, z:z + 1] * w / w.sum(axis=1, keepdims=True)
    return pops


def _synthetic_ion(rng, L, n_lines, lam_range, f_range, unique_pairs):
    """One synthetic ion: L levels evenly spaced over 0-10 eV, g = 1 + 2 (i mod 4),
    lines between random (l < u) pairs with log-uniform wavelength and f."""
    E = 10.0 * EV * np.arange(L) / (L - 1)
    g = 1.0 + 2.0 * (np.arange(L) % 4)
    iu, il = np.triu_indices(L, 1)[1], np.triu_indices(L, 1)[0]
    npairs = il.shape[0]
    if unique_pairs:
        pick = rng.choice(npairs, n_lines, replace=False)
    else:
        pick = rng.integers(0, npairs, n_lines)
    lo, up = il[pick], iu[pick]
    lam = 10.0 ** rng.uniform(np.log10(lam_range[0]), np.log10(lam_range[1]), n_lines)
    f = 10.0 ** rng.uniform(np.log10(f_range[0]), np.log10(f_range[1]), n_lines)
    return E, g, lo, up, lam, f


def collision_strengths(seed: int, level_off) -> list:
    """Effective collision strengths Upsilon for every level pair of every ion,
    log-uniform in [0.1, 10] (one seeded [L, L] upper-triangular array per ion;
    entry [l, u] with l < u)."""
    out = []
    for z in range(len(level_off) - 1):
        L = int(level_off[z + 1] - level_off[z])
        rng = np.random.default_rng([seed, 7919, z])
        ups = np.zeros((L, L))
        iu = np.triu_indices(L, 1)
        ups[iu] = 10.0 ** rng.uniform(-1.0, 1.0, iu[0].shape[0])
        out.append(ups)
    return out


def _spectrum_grid(lam_lo_emit, lam_hi_emit, v_max, dlog=1e-3):
    """0.1 % log wavelength grid wide enough for every Doppler-shifted escape."""
    b = v_max / C_LIGHT
    lam0 = lam_lo_emit * (1.0 - 1.5 * b)
    lam1 = lam_hi_emit * (1.0 + 1.5 * b)
    n_bins = int(np.ceil(np.log(lam1 / lam0) / np.log1p(dlog)))
    return (lam0, n_bins)


def uniform_sphere(seed: int = 0, n_packets: int = 100_000, n: int = 16,
                   n_lines: int = 100, n_levels: int = 20,
                   f_range=(1e-4, 1.0), subdomains=(1, 1, 1)) -> Workload:
    """Plain-method workload: uniform sphere in a 16^3 Cartesian velocity grid."""
    v_max, t = 5.0e8, 200.0 * DAY
    speed = _speed_grid(n, v_max)
    active = speed <= v_max
    ncell = n ** 3
    rng = np.random.default_rng(seed)
    E, g, lo, up, lam, f = _synthetic_ion(rng, n_levels, n_lines, (3000.0, 10000.0),
                                          f_range, unique_pairs=True)
    rho = np.where(active, 1e-15, 0.0)
    Te = np.full(ncell, 5000.0)
    ne = np.where(active, 1e7, 0.0)
    A = np.array([56.0])
    n_ion_density = (rho / (A[0] * M_U))[:, None].copy()
    level_off = np.array([0, n_levels], dtype=np.int32)
    pops = lte_populations(n_ion_density, level_off, E, g, Te)
    vol_active = active.astype(np.float64)
    L_cell = 1e40 * vol_active / vol_active.sum()
    deposition = L_cell / ((2.0 * v_max * t / n) ** 3)
    band = (2900.0, 10000.0)
    return Workload(
        name=f"uniform_sphere_{n}^3_{n_lines}lines_{n_packets}pk", nx=n, ny=n, nz=n,
        v_max=v_max, t=t, rho=rho, Te=Te, ne=ne, deposition=deposition, L_cell=L_cell,
        band_A=band, n_ion=1, level_off=level_off, E_level=E, g_level=g,
        ion_mass_u=A, n_ion_density=n_ion_density,
        lo=lo.astype(np.int32), up=up.astype(np.int32), lambda_A=lam, f_lu=f,
        pops=pops, upsilon_seed=seed, n_packets=n_packets, seed=seed,
        subdomains=tuple(subdomains), spec_band_A=_spectrum_grid(band[0], band[1], v_max),
        meta={"active_cells": int(active.sum())})


def gaussian_random_field(n: int, corr_len_cells: float, rng) -> np.ndarray:
    """Unit-variance periodic Gaussian random field on n^3 with correlation
    exp(-r^2 / (2 l^2)): white noise filtered by a Gaussian of width l/sqrt(2)."""
    w = rng.standard_normal((n, n, n))
    k = 2.0 * np.pi * np.fft.fftfreq(n)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    s = corr_len_cells / np.sqrt(2.0)
    filt = np.exp(-0.5 * (kx * kx + ky * ky + kz * kz) * s * s)
    field = np.real(np.fft.ifftn(np.fft.fftn(w) * filt))
    field -= field.mean()
    field /= field.std()
    return field.reshape(-1)   # natural order (x fastest)


ZONE_OF_ION = np.array([0, 0, 0, 1, 1, 2, 2, 3, 3, 3])   # Fe-group, O, He, H
MASS_OF_ZONE = np.array([56.0, 16.0, 4.0, 1.0])


def clumpy_onion(seed: int = 0, n_packets: int = 100_000_000, n: int = 64,
                 n_lines: int = 100_000, n_ion: int = 10, level_range=(50, 200),
                 subdomains=(8, 8, 8), lam_range=(1000.0, 30000.0),
                 f_range=(1e-6, 1.0), rho_mean=1e-15, sigma=0.5,
                 corr_len_cells=4.0, field_seed=None) -> Workload:
    """Paper-scale transport workload: onion zones with lognormal clumps.
    field_seed (default: seed) draws the clump field alone, so that two
    realizations can share the same atoms."""
    v_max, t = 5.0e8, 200.0 * DAY
    ncell = n ** 3
    speed = _speed_grid(n, v_max)
    active = speed <= v_max
    rng = np.random.default_rng(seed)
    zone = np.minimum((speed / v_max / 0.25).astype(np.int64), 3)
    grf = gaussian_random_field(n, corr_len_cells,
                                np.random.default_rng([seed if field_seed is None else field_seed, 1]))
    rho = np.where(active, rho_mean * np.exp(sigma * grf - 0.5 * sigma * sigma), 0.0)
    Te = np.full(ncell, 5000.0)
    ne = 1e7 * rho / rho_mean
    # number shares: native ions of the cell's zone share 97 %, the others 3 %
    ion_zone = ZONE_OF_ION[:n_ion] if n_ion == 10 else np.arange(n_ion) % 4
    A = MASS_OF_ZONE[ion_zone]
    share = np.zeros((ncell, n_ion))
    for zz in range(4):
        native = ion_zone == zz
        cells = zone == zz
        nn = int(native.sum())
        share[np.ix_(cells, native)] = 0.97 / nn
        share[np.ix_(cells, ~native)] = 0.03 / (n_ion - nn)
    mu = (share * A[None, :]).sum(axis=1)
    n_tot = np.where(active, rho / (mu * M_U), 0.0)
    n_ion_density = share * n_tot[:, None]
    # atoms
    Ls = rng.integers(level_range[0], level_range[1] + 1, n_ion)
    level_off = np.zeros(n_ion + 1, dtype=np.int32)
    level_off[1:] = np.cumsum(Ls)
    per_ion = np.full(n_ion, n_lines // n_ion)
    per_ion[: n_lines - per_ion.sum()] += 1
    Es, gs, los, ups, lams, fs = [], [], [], [], [], []
    for z in range(n_ion):
        E, g, lo, up, lam, f = _synthetic_ion(rng, int(Ls[z]), int(per_ion[z]), lam_range,
                                              f_range, unique_pairs=False)
        Es.append(E); gs.append(g)
        los.append(lo + level_off[z]); ups.append(up + level_off[z])
        lams.append(lam); fs.append(f)
    E = np.concatenate(Es); g = np.concatenate(gs)
    pops = lte_populations(n_ion_density, level_off, E, g, Te)
    L_cell = 1e40 * rho / rho.sum()
    deposition = L_cell / ((2.0 * v_max * t / n) ** 3)
    band = (lam_range[0] / (1.0 + 2.0 * v_max / C_LIGHT), lam_range[1])
    return Workload(
        name=f"clumpy_onion_{n}^3_{n_ion}ions_{n_lines}lines_{n_packets}pk",
        nx=n, ny=n, nz=n, v_max=v_max, t=t, rho=rho, Te=Te, ne=ne,
        deposition=deposition, L_cell=L_cell, band_A=band, n_ion=n_ion,
        level_off=level_off, E_level=E, g_level=g, ion_mass_u=A,
        n_ion_density=n_ion_density, lo=np.concatenate(los).astype(np.int32),
        up=np.concatenate(ups).astype(np.int32), lambda_A=np.concatenate(lams),
        f_lu=np.concatenate(fs), pops=pops, upsilon_seed=seed, n_packets=n_packets,
        seed=seed, subdomains=tuple(subdomains),
        spec_band_A=_spectrum_grid(band[0], band[1], v_max),
        meta={"active_cells": int(active.sum()), "levels_per_ion": Ls.tolist()})


def spherical_sphere(seed: int = 0, n_packets: int = 100_000, nr: int = 12, nth: int = 8,
                     nph: int = 12, n_lines: int = 100, n_levels: int = 20,
                     f_range=(1e-4, 1.0), subdomains=(1, 1, 4), clumps: bool = False) -> Workload:
    """The plain-method sphere on the paper's kind of grid: nr x nth x nph
    cells in (r, theta, phi) (Sec. 2: radial shells of equal velocity width,
    equal polar and azimuthal angles; the paper's validation model has 38 x 15
    x 30), every cell inside v_max; subdomains are phi slices (Sec. 2.4.1).
    Uniform density 1e-15 g/cm^3 (with clumps: the lognormal factor of the
    onion model drawn per cell), Te 5000 K, ne 1e7; the atoms and lines of
    uniform_sphere; band emission 2900-10000 A with L_cell proportional to the
    cell's volume (times its density with clumps)."""
    v_max, t = 5.0e8, 200.0 * DAY
    ncell = nr * nth * nph
    rng = np.random.default_rng(seed)
    E, g, lo, up, lam, f = _synthetic_ion(rng, n_levels, n_lines, (3000.0, 10000.0), f_range,
                                          unique_pairs=True)
    r_edges = np.linspace(0.0, v_max, nr + 1)
    th_edges = np.linspace(0.0, np.pi, nth + 1)
    ph_edges = np.linspace(0.0, 2.0 * np.pi, nph + 1)
    # natural order c = (iph * nth + ith) * nr + ir
    ir = np.tile(np.arange(nr), nth * nph)
    ith = np.tile(np.repeat(np.arange(nth), nr), nph)
    iph = np.repeat(np.arange(nph), nr * nth)
    vol = ((r_edges[ir + 1] ** 3 - r_edges[ir] ** 3) / 3.0 * (np.cos(th_edges[ith]) - np.cos(th_edges[ith + 1]))
           * (ph_edges[iph + 1] - ph_edges[iph]))
    fac = np.exp(0.5 * rng.standard_normal(ncell) - 0.125) if clumps else np.ones(ncell)
    rho = 1e-15 * fac
    Te = np.full(ncell, 5000.0)
    ne = 1e7 * fac
    A = np.array([56.0])
    n_ion_density = (rho / (A[0] * M_U))[:, None].copy()
    level_off = np.array([0, n_levels], dtype=np.int32)
    pops = lte_populations(n_ion_density, level_off, E, g, Te)
    L_cell = 1e40 * vol * fac / (vol * fac).sum()
    deposition = L_cell / (vol * t ** 3)
    band = (2900.0, 10000.0)
    return Workload(
        name=f"spherical_sphere_{nr}x{nth}x{nph}_{n_lines}lines_{n_packets}pk", nx=nr, ny=nth, nz=nph,
        v_max=v_max, t=t, rho=rho, Te=Te, ne=ne, deposition=deposition, L_cell=L_cell,
        band_A=band, n_ion=1, level_off=level_off, E_level=E, g_level=g,
        ion_mass_u=A, n_ion_density=n_ion_density,
        lo=lo.astype(np.int32), up=up.astype(np.int32), lambda_A=lam, f_lu=f,
        pops=pops, upsilon_seed=seed, n_packets=n_packets, seed=seed,
        subdomains=tuple(subdomains), spec_band_A=_spectrum_grid(band[0], band[1], v_max),
        meta={"active_cells": ncell}, geometry="spherical", r_edges=r_edges,
        theta_edges=th_edges, phi_edges=ph_edges)


def single_line_sphere(n: int = 16, n_packets: int = 100_000, seed: int = 3,
                       lam_A: float = 5000.0, f_lu: float = 1e-3,
                       n_scale: float = 1.0) -> Workload:
    """Two-level ion with one line inside a uniform sphere; ``n_scale`` rescales
    the ion density (n_scale -> 0 gives the optically thin limit)."""
    w = uniform_sphere(seed=seed, n_packets=n_packets, n=n, n_lines=1, n_levels=2)
    w.lambda_A = np.array([lam_A]); w.f_lu = np.array([f_lu])
    w.lo = np.array([0], np.int32); w.up = np.array([1], np.int32)
    w.n_ion_density = w.n_ion_density * n_scale
    w.pops = lte_populations(w.n_ion_density, w.level_off, w.E_level, w.g_level, w.Te)
    w.band_A = (lam_A * 0.9, lam_A * 1.1)
    w.spec_band_A = _spectrum_grid(w.band_A[0], w.band_A[1], w.v_max)
    w.name = f"single_line_sphere_{n}^3"
    return w


def nlte_batch(n: int = 64, seed: int = 0, n_ion: int = 10, L_max: int = 300,
               L_range=(20, 300), lines_per_level: int = 5) -> Workload:
    """Batched rate-solve workload: n^3 cells x n_ion ions; every (cell, ion)
    keeps its own number of levels, uniform in L_range (the ion models have
    L_max levels, 0-10 eV, g = 1 + 2 (i mod 4); each upper level has
    lines_per_level lines down to random lower levels, lambda log-uniform
    3000-10000 A, f log-uniform 1e-4..1; collision strengths log-uniform
    0.1-10 for every pair).  Te uniform 3000-10000 K per cell, n_e and ion
    densities lognormal, deposition lognormal.  The mean intensity stands in
    for the 16^3-sphere transport field: diluted Planck W B_nu(T_R) with
    T_R = 8000 K, W = 5.6e-5 (J_nu near 5000 A about 5e-9 erg/s/cm^2/Hz/sr).
    Starting populations: Boltzmann over the kept levels."""
    v_max, t = 5.0e8, 200.0 * DAY
    ncell = n ** 3
    rng = np.random.default_rng([seed, 3])
    Te = rng.uniform(3000.0, 10000.0, ncell)
    ne = 1e7 * np.exp(0.5 * rng.standard_normal(ncell))
    rho = np.full(ncell, 1e-15)
    n_ion_density = 1e6 * np.exp(0.5 * rng.standard_normal((ncell, n_ion)))
    deposition = 1e-14 * np.exp(0.5 * rng.standard_normal(ncell))
    levels_used = rng.integers(L_range[0], L_range[1] + 1, (ncell, n_ion)).astype(np.int32)
    level_off = (np.arange(n_ion + 1) * L_max).astype(np.int32)
    E1 = 10.0 * EV * np.arange(L_max) / (L_max - 1)
    g1 = 1.0 + 2.0 * (np.arange(L_max) % 4)
    los, ups_, lams, fs = [], [], [], []
    for z in range(n_ion):
        r = np.random.default_rng([seed, 11, z])
        u = np.repeat(np.arange(1, L_max), lines_per_level)
        lo = np.floor(r.random(u.shape[0]) * u).astype(np.int64)
        los.append(lo + level_off[z]); ups_.append(u + level_off[z])
        lams.append(10.0 ** r.uniform(np.log10(3000.0), 4.0, u.shape[0]))
        fs.append(10.0 ** r.uniform(-4.0, 0.0, u.shape[0]))
    E = np.tile(E1, n_ion); g = np.tile(g1, n_ion)
    pops = np.zeros((ncell, n_ion * L_max))
    kT = K_BOLTZ * Te
    base = g1[None, :] * np.exp(-E1[None, :] / kT[:, None])      # same levels in every ion
    csum = np.cumsum(base, axis=1)
    for z in range(n_ion):
        Lz = levels_used[:, z]
        norm = n_ion_density[:, z] / csum[np.arange(ncell), Lz - 1]
        blk = pops[:, level_off[z]:level_off[z + 1]]
        np.multiply(base, norm[:, None], out=blk)
        blk[np.arange(L_max)[None, :] >= Lz[:, None]] = 0.0
    w_ = Workload(
        name=f"nlte_batch_{n}^3x{n_ion}_L{L_range[0]}-{L_range[1]}", nx=n, ny=n, nz=n,
        v_max=v_max, t=t, rho=rho, Te=Te, ne=ne, deposition=deposition,
        L_cell=np.ones(ncell), band_A=(3000.0, 10000.0), n_ion=n_ion, level_off=level_off,
        E_level=E, g_level=g, ion_mass_u=np.full(n_ion, 56.0), n_ion_density=n_ion_density,
        lo=np.concatenate(los).astype(np.int32), up=np.concatenate(ups_).astype(np.int32),
        lambda_A=np.concatenate(lams), f_lu=np.concatenate(fs), pops=pops, upsilon_seed=seed,
        n_packets=0, seed=seed, subdomains=(1, 1, 1),
        spec_band_A=_spectrum_grid(3000.0, 10000.0, v_max), meta={},
        levels_used=levels_used, jbar_W=5.6e-5, jbar_TR=8000.0)
    w_.upsilon = collision_strengths(seed, level_off)
    return w_


def with_photoionization(w: Workload, chi_eV=None, charge=None, pi_nlev=9, seed=None) -> Workload:
    """Adds photoionization data to a workload (in place; returns it).

    Recipe (the paper's atomic data are not available): per ion an ionization
    energy chi_eV (default: uniform in 10.5-14 eV from ``seed``), a charge
    (default: ion index mod 3, i.e. neutral, singly and doubly ionized stages),
    and the lowest ``pi_nlev`` levels photoionizing (the ground level and the
    next eight by default, as the paper's on-the-spot treatment takes)."""
    rng = np.random.default_rng([w.seed if seed is None else seed, 4231])
    if chi_eV is None:
        chi_eV = rng.uniform(10.5, 14.0, w.n_ion)
    chi = np.broadcast_to(np.asarray(chi_eV, dtype=np.float64), (w.n_ion,)) * EV
    if charge is None:
        charge = np.arange(w.n_ion) % 3
    L = np.diff(w.level_off)
    w.chi_ion = np.ascontiguousarray(chi)
    w.charge = np.ascontiguousarray(np.broadcast_to(np.asarray(charge), (w.n_ion,)), dtype=np.int32)
    w.pi_nlev = np.minimum(np.broadcast_to(np.asarray(pi_nlev), (w.n_ion,)), L).astype(np.int32)
    return w


def pi_levels(w: Workload):
    """The photoionizing levels in their order (ion by ion, lowest first):
    global level index, ionization energy and charge of the level's ion."""
    lev, eion, ch = [], [], []
    for z in range(w.n_ion):
        for i in range(int(w.pi_nlev[z])):
            lev.append(int(w.level_off[z]) + i)
            eion.append(float(w.chi_ion[z]))
            ch.append(int(w.charge[z]))
    return (np.array(lev, dtype=np.int32), np.array(eion, dtype=np.float64),
            np.array(ch, dtype=np.int32))


def workload(name: str, **kw) -> Workload:
    if name == "uniform_sphere":
        return uniform_sphere(**kw)
    if name == "clumpy_onion":
        return clumpy_onion(**kw)
    raise KeyError(name)
