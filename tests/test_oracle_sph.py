"""Pins of the oracle on the spherical (r, theta, phi) grid (Sec. 2: the
paper's models are spherical grids of shells, polar and azimuthal sectors;
Sec. 2.4.1: phi slices as subdomains), against things other than itself (no
GPU).

- The cells tile the sphere: their volumes sum to 4/3 pi R^3.
- Optically thin line emission from a uniform sphere: every packet's lab
  wavelength follows the first-order Doppler shift of its emission point and
  direction, and their distribution is the parabolic profile of a uniformly
  emitting sphere, (3/4)(1 - x^2) in x = (lambda - lambda_l) c / (lambda_l
  v_max) (chi-square).
- Optically thin lines: the rates readout's mean intensity per radial shell
  equals the closed form J(r) of a uniformly emitting sphere (here the grid is
  the sphere, no voxelised edge), also where the absorbers' density changes
  from cell to cell (an event booked in the wrong cell would carry the wrong
  cell's population and break the per-cell mean intensity).
- The photon ledger closes.
- The walk alone (face solver and cell step): along random straight paths,
  every cell the oracle lists contains the middle of its path piece, the
  points just before and after each exit lie in the cell left and the cell
  entered, and a fine sampling of the path meets the cells in the same order
  (cell membership computed directly from r, theta and phi).
"""
import numpy as np
import pytest

import oracle
import synth

C = 2.99792458e10


def test_cells_tile_the_sphere():
    w = synth.spherical_sphere(nr=7, nth=5, nph=9)
    V = oracle.cell_volume(w)
    R = w.v_max * w.t
    assert V.sum() == pytest.approx(4.0 / 3.0 * np.pi * R ** 3, rel=1e-13)
    assert np.all(V > 0)


def test_thin_line_parabolic_profile():
    w = synth.spherical_sphere(n_packets=200_000, nr=10, nth=6, nph=8, n_lines=1, n_levels=2, seed=3)
    w.lambda_A = np.array([5000.0])
    w.f_lu = np.array([1e-3])
    w.pops = w.pops * 1e-30                               # no line can absorb
    w.pops[:, 1] = w.pops[:, 0]                           # upper level populated: it emits
    w.spec_band_A = synth._spectrum_grid(4800.0, 5200.0, w.v_max)
    o = oracle.transport(w, emission="lines", per_packet=True)
    pk = o["pkt"]
    assert o["ledger"]["events"] == 0 and np.all(pk[:, 0] == 0)
    lam = C / pk[:, 10] * 1e8
    x = (lam - 5000.0) / 5000.0 / (w.v_max / C)
    # first order in v/c: lambda_lab = lambda_l (1 - n.r / ct), |n.r| / ct <= v_max / c
    assert np.all(np.abs(x) <= 1.0 + 1e-9)
    edges = np.linspace(-1, 1, 41)
    cnt, _ = np.histogram(x, edges)
    F = lambda t: 0.75 * (t - t ** 3 / 3.0) + 0.5
    expct = len(x) * np.diff(F(edges))
    chi2 = np.sum((cnt - expct) ** 2 / expct) / len(cnt)
    assert 0.5 < chi2 < 1.6, chi2
    # a wrong volume weighting of the emission (e.g. uniform in r) or Doppler
    # sign moves the moments
    assert np.mean(x ** 2) == pytest.approx(0.2, abs=0.004)        # <x^2> of (3/4)(1 - x^2)
    assert abs(np.mean(x)) < 0.004


@pytest.mark.parametrize("clumps", [False, True])
def test_thin_sphere_mean_intensity(clumps):
    w = synth.spherical_sphere(n_packets=600_000, nr=16, nth=8, nph=12, n_lines=1000, n_levels=50,
                               seed=41, clumps=clumps)
    w.v_max = 5e7
    w.r_edges = w.r_edges * 0.1                           # the grid follows v_max
    V = oracle.cell_volume(w)
    w.L_cell = 1e40 * V / V.sum()                         # uniform emissivity
    nz = w.n_ion_density[:, 0]
    q = 0.97
    x = w.g_level * q ** np.arange(w.nlev)
    w.pops = nz[:, None] * (x / x.sum())[None, :]
    net = w.pops[0, w.lo] - w.g_level[w.lo] / w.g_level[w.up] * w.pops[0, w.up]
    tau_t = 10 ** np.random.default_rng(41).uniform(np.log10(5e-4), np.log10(2e-3), w.nline)
    w.f_lu = tau_t / (oracle.PI_E2_MC * w.lambda_A * 1e-8 * w.t * net)
    w.f_lu = w.f_lu * (1e-15 / w.rho.max())               # densest cell keeps tau < 2e-3 (clumps)
    # no Sobolev optical depth cut: in the thinnest cells of the clumpy model
    # the lines fall below the default 1e-4
    o = oracle.transport(w, tau_min=1e-12)
    _, _, J = oracle.rates(w, o["S"])
    R = w.v_max * w.t
    rc = 0.5 * (w.r_edges[:-1] + w.r_edges[1:]) * w.t
    ir = np.tile(np.arange(w.nx), w.ny * w.nz)
    r = rc[ir]
    dnu = C / (w.band_A[0] * 1e-8) - C / (w.band_A[1] * 1e-8)
    j = 1e40 / V.sum() / (4 * np.pi * dnu)
    J_exact = j * R / 2 * (1 + (R * R - r * r) / (2 * r * R) * np.log((R + r) / (R - r)))
    Jc = J.mean(axis=1)
    for a, b in [(0, 0.3), (0.3, 0.5), (0.5, 0.7), (0.7, 0.9)]:
        m = (r / R >= a) & (r / R < b)
        ratio = Jc[m].sum() / J_exact[m].sum()
        assert ratio == pytest.approx(1.0, abs=0.03), (a, b, ratio)
    if clumps:
        # the mean intensity does not follow the absorbers' density
        m = r / R < 0.8
        rel = Jc[m] / J_exact[m]
        cc = np.corrcoef(np.log(w.rho[m]), rel)[0, 1]
        assert abs(cc) < 0.2, cc


def test_ledger_closes():
    w = synth.spherical_sphere(n_packets=40_000, seed=9, clumps=True)
    w.pops = w.pops * 1e-3
    o = oracle.transport(w)
    L = o["ledger"]
    assert L["events"] > 10_000 and L["guard"] == 0
    assert L["esc_N"] + L["abs_N"] + L["drop_N"] == pytest.approx(L["emit_N"], rel=1e-13)


class _Domain:
    """One phi-slab domain traced by the oracle; sums what its calls tally."""

    def __init__(self, w, z_lo, z_hi):
        self.w, self.z_lo, self.z_hi = w, z_lo, z_hi
        self.S = self.spec = None
        self.ledger = {}

    def step(self, emit, bundle_in):
        import torch
        b = None if bundle_in is None else bundle_in.numpy()
        o = oracle.transport_domain(self.w, self.z_lo, self.z_hi, emit, b)
        self.S = o["S"] if self.S is None else self.S + o["S"]
        self.spec = o["spec"] if self.spec is None else self.spec + o["spec"]
        for k, v in o["ledger"].items():
            self.ledger[k] = self.ledger.get(k, 0.0) + v
        return torch.from_numpy(o["bundle"])

    def z_of(self, bundle):
        import torch
        return bundle[:, oracle.STATE_Z].to(torch.int64)


@pytest.mark.parametrize("world", [1, 3, 4])
def test_phi_slab_domains_sum_to_the_whole(world):
    """The paper's decomposition of the spherical grid (Sec. 2.4.1): each domain
    holds whole phi slices; a packet entering another domain's slices is handed
    on with its state (the path from its emission point included) and resumes
    there.  The domains' sums equal the single-domain pass; phi wraps around,
    and a straight ray crosses each slab boundary at most once."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2511_07539_gb300 import spatial
    w = synth.spherical_sphere(n_packets=20_000, seed=5, clumps=True)      # 12 phi slices
    w.pops = w.pops * 1e-3
    doms = [_Domain(w, *spatial.slab(r, w.nz, world)) for r in range(world)]
    rounds = spatial.run_local(doms, w.nz)
    assert (rounds == 0) == (world == 1) and rounds <= world - 1
    S, spec = sum(d.S for d in doms), sum(d.spec for d in doms)
    ref = oracle.transport(w)
    m = ref["S"] != 0
    assert np.array_equal(S != 0, m)
    assert np.max(np.abs(S[m] / ref["S"][m] - 1)) < 1e-12
    ms = ref["spec"] != 0
    assert np.array_equal(spec != 0, ms)
    assert np.max(np.abs(spec[ms] / ref["spec"][ms] - 1)) < 1e-12
    tot = {}
    for d in doms:
        for k, v in d.ledger.items():
            tot[k] = tot.get(k, 0.0) + v
    L = ref["ledger"]
    assert tot["events"] == L["events"] and tot["tests"] == L["tests"]
    for k in ("emit_N", "esc_N", "abs_N", "drop_N", "esc_E"):
        assert tot[k] == pytest.approx(L[k], rel=1e-12)


def _thin_single_line(w, lam_A=6000.0):
    w.lambda_A = np.array([lam_A])
    w.f_lu = np.array([1e-3])
    w.lo = np.array([0], np.int32)
    w.up = np.array([1], np.int32)
    w.pops = w.pops * 1e-30
    w.pops[:, 1] = w.pops[:, 0]
    return w


def test_thin_rays_on_the_spherical_grid():
    """The RAYS sampler on the spherical grid (Sec. 2.3), optically thin: every
    ray escapes into its own viewer, and the comoving energy per viewer is the
    emission times dOmega_k / 4 pi."""
    nt, nph = 6, 8
    w = synth.spherical_sphere(n_packets=1, seed=3, nr=6, nth=4, nph=6)
    w.pops = w.pops * 1e-30
    o = oracle.transport(w, sampler="rays", n_theta=nt, n_phi=nph, spec_dlog=0.01, per_packet=True)
    L = o["ledger"]
    assert L["events"] == 0
    assert L["emit_E"] == pytest.approx(w.L_cell.sum(), rel=1e-9)
    pk = o["pkt"]
    Ecmf = pk[:, 8] * 6.62607015e-27 * pk[:, 9]
    k = np.arange(o["n"]) % (nt * nph)
    per_view = np.bincount(k, weights=Ecmf, minlength=nt * nph)
    th = np.linspace(0.0, np.pi, nt + 1)
    dOm = np.repeat(2 * np.pi / nph * (np.cos(th[:-1]) - np.cos(th[1:])), nph)
    np.testing.assert_allclose(per_view, w.L_cell.sum() * dOm / (4 * np.pi), rtol=1e-10)
    assert np.array_equal(pk[:, 4], k.astype(float))


def test_single_line_rays_start_at_the_cell_middle():
    """One thin emission line, rays on the spherical grid: every ray's lab
    wavelength follows from the middle of its cell's r, theta and phi ranges and
    its viewer's direction by the first-order Doppler formula; the spectrum
    binned from that restatement equals the oracle's."""
    w = _thin_single_line(synth.spherical_sphere(n_packets=1, seed=7, nr=5, nth=4, nph=6, n_lines=1,
                                                 n_levels=2))
    nt, nph, dlog = 5, 8, 2e-4
    lam0 = 6000.0 * (1 - 0.03)
    nb = int(np.log(1.06 / 0.97) / np.log1p(dlog)) + 1
    w.spec_band_A = (lam0, nb)
    o = oracle.transport(w, sampler="rays", emission="lines", n_theta=nt, n_phi=nph, spec_dlog=dlog)
    nu_l = C / (6000.0 * 1e-8)
    spec = np.zeros((nt * nph, nb))
    Lc, _ = oracle.emission(w, n_packets=1, emission="lines")
    th = np.linspace(0.0, np.pi, nt + 1)
    w_k = np.repeat(2 * np.pi / nph * (np.cos(th[:-1]) - np.cos(th[1:])), nph) / (4 * np.pi)
    for c in np.nonzero(Lc > 0)[0]:
        ir, it_, ip_ = c % w.nx, (c // w.nx) % w.ny, c // (w.nx * w.ny)
        rm = 0.5 * (w.r_edges[ir] + w.r_edges[ir + 1]) * w.t
        tm = 0.5 * (w.theta_edges[it_] + w.theta_edges[it_ + 1])
        pm = 0.5 * (w.phi_edges[ip_] + w.phi_edges[ip_ + 1])
        r = rm * np.array([np.sin(tm) * np.cos(pm), np.sin(tm) * np.sin(pm), np.cos(tm)])
        for it in range(nt):
            for ip in range(nph):
                k = it * nph + ip
                tc, pc = np.pi * (it + 0.5) / nt, 2 * np.pi * (ip + 0.5) / nph
                n = np.array([np.sin(tc) * np.cos(pc), np.sin(tc) * np.sin(pc), np.cos(tc)])
                nu_lab = nu_l / (1 - n @ r / (C * w.t))
                b = int(np.floor(np.log(C / nu_lab * 1e8 / lam0) / np.log1p(dlog)))
                spec[k, b] += Lc[c] * w_k[k] * nu_lab / nu_l
    m = spec > 0
    assert np.array_equal(m, o["spec"] > 0)
    np.testing.assert_allclose(o["spec"][m], spec[m], rtol=1e-12)


H = 6.62607015e-27


def test_thin_sphere_photoionization_rates_on_the_spherical_grid():
    """Photoionization on every segment of the spherical walk (Sec. 2.3.1),
    optically thin: the rate of each photoionizing level per radial shell is the
    closed form of a uniformly emitting sphere, Gamma(r) = 4 pi J(r) sig c^3 /
    (3 h) (nu_th^-3 - nu_hi^-3) for the hydrogenic sigma = sig lambda^3 of
    Eq. sigma_OTSPI and a flat J_nu (the grid is the sphere itself)."""
    w = synth.spherical_sphere(n_packets=600_000, nr=16, nth=6, nph=8, n_lines=5, n_levels=20, seed=61,
                               subdomains=(1, 1, 4))
    w.v_max = 5e7
    w.r_edges = w.r_edges * 0.1
    w.f_lu = np.full(w.nline, 1e-30)                      # no line interacts
    synth.with_photoionization(w, chi_eV=6.0, charge=1, pi_nlev=8)
    w.pops = np.ones((w.ncell, 1)) * np.linspace(1.0, 2.0, w.nlev)[None, :]
    V = oracle.cell_volume(w)
    w.L_cell = 1e40 * V / V.sum()
    o = oracle.transport(w)
    G = oracle.pi_rates(w, o["S_pi"])
    lev, eion, ch = synth.pi_levels(w)
    R = w.v_max * w.t
    rc = 0.5 * (w.r_edges[:-1] + w.r_edges[1:]) * w.t
    r = rc[np.tile(np.arange(w.nx), w.ny * w.nz)]
    nu_lo, nu_hi = C / (w.band_A[1] * 1e-8), C / (w.band_A[0] * 1e-8)
    j = 1e40 / V.sum() / (4 * np.pi * (nu_hi - nu_lo))
    J = j * R / 2 * (1 + (R * R - r * r) / (2 * r * R) * np.log((R + r) / (R - r)))
    tested = 0
    for k in range(lev.shape[0]):
        nu_th = (eion[k] - w.E_level[lev[k]]) / H
        if nu_th >= nu_hi * (1 - 2 * w.v_max / C):
            assert np.all(G[:, k] == 0), k
            continue
        sig = oracle.sigma_pi(1.0, w.E_level[lev[k]], eion[k], int(ch[k]))
        want = 4 * np.pi * J * sig * C ** 3 / (3 * H) * (max(nu_th, nu_lo) ** -3 - nu_hi ** -3)
        for a, b in [(0, 0.4), (0.4, 0.6), (0.6, 0.8)]:
            m = (r / R >= a) & (r / R < b)
            ratio = G[m, k].sum() / want[m].sum()
            assert ratio == pytest.approx(1.0, abs=0.03), (k, a, b, ratio)
        tested += 1
    assert tested >= 3


def test_ledger_closes_with_photoionization_on_the_spherical_grid():
    w = synth.spherical_sphere(n_packets=30_000, seed=71, clumps=True)
    synth.with_photoionization(w, chi_eV=6.0, charge=0, pi_nlev=9)
    w.pops = w.pops * 1e-3
    o = oracle.transport(w)
    L = o["ledger"]
    assert L["pi_N"] > 0.05 * L["emit_N"] and L["abs_N"] > 0.05 * L["emit_N"] and L["events"] > 10_000
    assert L["esc_N"] + L["abs_N"] + L["pi_N"] + L["drop_N"] == pytest.approx(L["emit_N"], rel=1e-13)
    assert o["S_pi"].sum() == pytest.approx(L["pi_N"], rel=1e-12)


def _cell_of(w, p):
    """Natural index of the cell holding point p (cm), straight from the
    edges in r, theta and phi (-1 outside the outer sphere)."""
    r = float(np.sqrt(p @ p))
    if r >= w.r_edges[-1] * w.t:
        return -1
    th = float(np.arccos(np.clip(p[2] / r, -1.0, 1.0)))
    ph = float(np.arctan2(p[1], p[0])) % (2.0 * np.pi)
    ir = min(int(np.searchsorted(w.r_edges * w.t, r, side="right")) - 1, w.nx - 1)
    it = min(max(int(np.searchsorted(w.theta_edges, th, side="right")) - 1, 0), w.ny - 1)
    ip = min(max(int(np.searchsorted(w.phi_edges, ph, side="right")) - 1, 0), w.nz - 1)
    return (ip * w.ny + it) * w.nx + ir


@pytest.mark.parametrize("nr,nth,nph", [(6, 4, 6), (9, 7, 5), (5, 6, 1)])
def test_walk_against_cell_membership(nr, nth, nph):
    w = synth.spherical_sphere(n_packets=1, seed=3, nr=nr, nth=nth, nph=nph)
    rng = np.random.default_rng(nr * 100 + nth * 10 + nph)
    R = w.r_edges[-1] * w.t
    eps = 1e-9 * R
    for _ in range(150):
        # a point uniform in a random cell, a direction uniform on the sphere
        ir, it, ip = rng.integers(nr), rng.integers(nth), rng.integers(nph)
        r0, r1 = w.r_edges[ir] * w.t, w.r_edges[ir + 1] * w.t
        r = (r0 ** 3 + rng.random() * (r1 ** 3 - r0 ** 3)) ** (1.0 / 3.0)
        c0, c1 = np.cos(w.theta_edges[it]), np.cos(w.theta_edges[it + 1])
        mu = c0 + rng.random() * (c1 - c0)
        ph = w.phi_edges[ip] + rng.random() * (w.phi_edges[ip + 1] - w.phi_edges[ip])
        st = np.sqrt(1.0 - mu * mu)
        p0 = r * np.array([st * np.cos(ph), st * np.sin(ph), mu])
        u, v = rng.random(2)
        m = 2.0 * u - 1.0
        n = np.array([np.sqrt(1 - m * m) * np.cos(2 * np.pi * v), np.sqrt(1 - m * m) * np.sin(2 * np.pi * v), m])
        assert _cell_of(w, p0) == (ip * nth + it) * nr + ir
        out = oracle.sph_walk(w, p0, n, (ir, it, ip))
        assert out is not None
        cells, s_exit = out
        assert np.all(np.diff(s_exit) > 0) and s_exit[0] > 0
        s_prev = 0.0
        for k, (c, se) in enumerate(zip(cells, s_exit)):
            assert _cell_of(w, p0 + 0.5 * (s_prev + se) * n) == c
            assert _cell_of(w, p0 + (se - eps) * n) == c
            nxt = cells[k + 1] if k + 1 < len(cells) else -1
            assert _cell_of(w, p0 + (se + eps) * n) == nxt
            s_prev = se
        # a fine sampling meets the cells in the same order
        ss = np.linspace(0.0, s_exit[-1] * (1 - 1e-12), 4000)
        seen = [c for c in (_cell_of(w, p0 + s * n) for s in ss)]
        dedup = [seen[0]] + [b for a, b in zip(seen[:-1], seen[1:]) if b != a]
        it_cells = iter(cells.tolist())
        assert all(any(c == x for x in it_cells) for c in dedup)      # a subsequence, in order

