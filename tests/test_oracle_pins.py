"""Pins of the transport oracle against things other than itself (no GPU).

P1  Sobolev beta vs mpmath; tau vs the oscillator-strength form; Einstein A
    vs a textbook line (golden fixture).
P7  Philox4x64-10 vs numpy's independent Philox.
P4  single resonance: escaped N = N0 e^-tau and estimator N0 (1-e^-tau)/f_corr.
P5  event histories vs a brute-force restatement (bisection on the comoving
    frequency, cells by flooring the resonance point).
P2  optically thin line profile of the voxelised sphere vs the hat-box
    projection integrated by quadrature.
P3  optically thin estimator in a cell slab vs a 6-D quadrature of the
    mean-intensity integral; the rates readout's mean intensity in a thin
    uniform sphere vs the closed-form J(r) of a uniformly emitting sphere.
P6  photon ledger closure; comoving energy closure in scatter mode; the
    scatter-mode destruction probability of a single line.
A7  the mean intensity of the rates readout against the Einstein relation
    between A_ul (pinned above) and B_lu.
A5  spectrum normalisation (energy closure against the ledger) and isotropy.
"""
import os

import mpmath as mp
import numpy as np
import pytest

import oracle
import synth
from tests import oracle_brute as brute

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- P1
def test_beta_sobolev_vs_mpmath():
    L = oracle.lib()
    mp.mp.dps = 40
    worst = 0.0
    for tau in np.logspace(-12, 3, 301):
        exact = (1 - mp.exp(-mp.mpf(tau))) / mp.mpf(tau)
        got = L.xo_beta_sobolev(float(tau))
        worst = max(worst, abs(got - float(exact)) / float(exact))
    assert worst < 5e-16
    assert L.xo_beta_sobolev(0.0) == 1.0
    assert L.xo_beta_sobolev(-5.0) == 1.0 and L.xo_beta_sobolev(-1e4) == 1.0
    t = 1e-9
    assert abs(L.xo_beta_sobolev(t) - (1 - t / 2 + t * t / 6)) < 1e-16
    # large tau: beta -> 1/tau
    assert L.xo_beta_sobolev(1e6) == pytest.approx(1e-6, rel=1e-15)


def test_tau_sobolev_oscillator_strength_form():
    """Eq. (tau_Sobolev) written with A_ul equals the f-form
    (pi e^2/m_e c) f lambda t (n_l - g_l n_u/g_u), evaluated in mpmath."""
    L = oracle.lib()
    mp.mp.dps = 40
    rng = np.random.default_rng(1)
    e, me, c = mp.mpf("4.80320471e-10"), mp.mpf("9.1093837015e-28"), mp.mpf("2.99792458e10")
    for _ in range(200):
        lam = float(10 ** rng.uniform(3, 4.5)) * 1e-8
        f = float(10 ** rng.uniform(-6, 0))
        gl, gu = float(rng.integers(1, 9)), float(rng.integers(1, 9))
        nl, nu_ = float(10 ** rng.uniform(-5, 8)), float(10 ** rng.uniform(-5, 8))
        t = float(rng.uniform(1e6, 3e7))
        A = L.xo_einstein_A(lam, gl, gu, f)
        got = L.xo_tau_sobolev(A, gl, gu, lam, nl, nu_, t)
        exact = mp.pi * e * e / (me * c) * f * lam * t * (nl - gl * nu_ / gu)
        assert abs(got - float(exact)) <= 1e-13 * abs(float(exact)) + 1e-300
    # empty lower level: tau <= 0, so the line is never an interaction point
    A = L.xo_einstein_A(5e-5, 2.0, 4.0, 0.1)
    assert L.xo_tau_sobolev(A, 2.0, 4.0, 5e-5, 0.0, 1.0, 1e7) < 0
    assert L.xo_tau_sobolev(A, 2.0, 4.0, 5e-5, 0.0, 0.0, 1e7) == 0


def test_einstein_A_textbook_line():
    rows = np.loadtxt(os.path.join(HERE, "golden", "halpha_einstein_A.txt"), ndmin=2)
    L = oracle.lib()
    for lam, f, gl, gu, A_ref, tol in rows:
        A = L.xo_einstein_A(lam * 1e-8, gl, gu, f)
        assert A == pytest.approx(A_ref, rel=tol)


# ---------------------------------------------------------------- A7
def test_rates_mean_intensity_obeys_einstein_relation():
    """Jbar = R_lu / B_lu: with the B_lu the readout implies, B = R_lu / Jbar,
    the Einstein relation A_ul = (2 h nu^3 / c^2) (g_l / g_u) B_lu must give
    the A_ul of the oscillator-strength form (pinned against the textbook H
    alpha value above), so no factor of B_lu can be dropped unseen."""
    w = synth.uniform_sphere(n=4, n_packets=2000, n_lines=12, seed=3)
    S = np.random.default_rng(0).uniform(1.0, 2.0, (w.ncell, w.nline)) * 1e30
    R_lu, R_ul, J = oracle.rates(w, S)
    c = int(np.nonzero(w.rho > 0)[0][0])
    B = R_lu[c] / J[c]
    nu = 2.99792458e10 / (w.lambda_A * 1e-8)
    gl, gu = w.g_level[w.lo], w.g_level[w.up]
    A_rel = 2 * 6.62607015e-27 * nu ** 3 / 2.99792458e10 ** 2 * (gl / gu) * B
    L = oracle.lib()
    A_f = np.array([L.xo_einstein_A(lam * 1e-8, a, b, f)
                    for lam, a, b, f in zip(w.lambda_A, gl, gu, w.f_lu)])
    np.testing.assert_allclose(A_rel, A_f, rtol=1e-12)
    np.testing.assert_allclose(R_ul[c], (gl / gu) * R_lu[c], rtol=1e-15)
    assert np.all(R_lu[c] > 0)


def _thin_sphere(n=32, n_packets=1_000_000, n_lines=1000, v_max=5e7, q=0.97, seed=41):
    """Uniform sphere of optically thin lines (tau_S 5e-4..2e-3 in every active
    cell) with populations n_i ~ g_i q^i, so that f_corr = 1 - q^(u-l) spans
    0.03..0.8: a readout that divided by n_l instead of n_l - (g_l/g_u) n_u,
    or dropped the stimulated-emission correction, would be off by 1/f_corr.
    v_max = 500 km/s keeps the first-order Doppler terms (v/c) below 0.2 %."""
    w = synth.uniform_sphere(n=n, n_packets=n_packets, n_lines=n_lines, n_levels=50, seed=seed)
    w.v_max = v_max
    nz = w.n_ion_density[:, 0]
    x = w.g_level * q ** np.arange(w.nlev)
    w.pops = nz[:, None] * (x / x.sum())[None, :]
    c = int(np.nonzero(nz > 0)[0][0])
    net = w.pops[c, w.lo] - w.g_level[w.lo] / w.g_level[w.up] * w.pops[c, w.up]
    tau_t = 10 ** np.random.default_rng(seed).uniform(np.log10(5e-4), np.log10(2e-3), w.nline)
    w.f_lu = tau_t / (oracle.PI_E2_MC * w.lambda_A * 1e-8 * w.t * net)
    return w


def test_rates_thin_sphere_mean_intensity_closed_form():
    """P3 for the rates readout: in an optically thin uniform sphere with flat
    j_nu, Jbar = R_lu / B_lu with R_lu = S / (n_l V) must equal the
    mean intensity of a uniformly emitting sphere,
    J(r) = (j R / 2) [1 + (R^2 - r^2) / (2 r R) ln((R + r) / (R - r))],
    j = L_cell / (4 pi V dnu_band), to Monte Carlo error, in every radial
    shell and for every part of the line list.  This fixes the cell volume,
    the division by n_l and f_corr, and B_lu of the readout (the Einstein
    relation pin above fixes only the ratio of R_lu and Jbar)."""
    w = _thin_sphere()
    act = w.rho > 0
    tau, _ = oracle.tau_beta(w, int(np.nonzero(act)[0][0]), 1)
    assert 1e-4 < tau.min() and tau.max() < 3e-3            # thin, but interaction points
    o = oracle.transport(w)
    _, _, J = oracle.rates(w, o["S"])
    R = w.v_max * w.t
    xc = synth.cell_centres(w.nx, w.v_max) * w.t
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2).reshape(-1)
    c = 2.99792458e10
    dnu = c / (w.band_A[0] * 1e-8) - c / (w.band_A[1] * 1e-8)
    V = (2 * R / w.nx) ** 3
    j = w.L_cell[act][0] / V / (4 * np.pi * dnu)
    rr = np.clip(r, 1e-9 * R, (1 - 1e-9) * R)       # (cells outside the sphere are not compared)
    J_exact = j * R / 2 * (1 + (R * R - rr * rr) / (2 * rr * R) * np.log((R + rr) / (R - rr)))
    Jc = J.mean(axis=1)
    for a, b in [(0, 0.3), (0.3, 0.45), (0.45, 0.6), (0.6, 0.75), (0.75, 0.9)]:
        m = act & (r / R >= a) & (r / R < b)
        ratio = Jc[m].sum() / J_exact[m].sum()
        assert ratio == pytest.approx(1.0, abs=0.03), (a, b, ratio)
    # flat in frequency: every tenth of the line list (sorted by wavelength)
    # sees the same field in the inner sphere
    inner = act & (r < 0.75 * R)
    order = np.argsort(w.lambda_A)
    for part in np.array_split(order, 10):
        ratio = J[np.ix_(inner, part)].mean(axis=1).sum() / J_exact[inner].sum()
        assert ratio == pytest.approx(1.0, abs=0.05), ratio


# ---------------------------------------------------------------- P7
def test_philox_vs_numpy():
    rng = np.random.default_rng(5)
    for _ in range(500):
        ctr = [int(x) for x in rng.integers(0, 2 ** 63, 4, dtype=np.int64)]
        ctr[0] |= 1   # keep the 256-bit counter nonzero
        key = [int(x) for x in rng.integers(0, 2 ** 63, 2, dtype=np.int64)]
        mine = oracle.philox4x64_10(ctr, key)
        c256 = ctr[0] + (ctr[1] << 64) + (ctr[2] << 128) + (ctr[3] << 192)
        bg = np.random.Philox(counter=c256 - 1, key=key[0] + (key[1] << 64))
        assert np.array_equal(mine, bg.random_raw(4).astype(np.uint64))


def test_packet_quota_largest_remainder():
    rng = np.random.default_rng(2)
    for N in [1, 7, 1000, 123457]:
        L = rng.random(300) * (rng.random(300) > 0.3)
        q = oracle.packet_quota(L, N)
        n = np.diff(q)
        assert q[-1] == N and np.all(n >= 0)
        share = N * L / L.sum()
        assert np.all(np.abs(n - share) < 1.0)
        assert np.array_equal(q, brute.largest_remainder(list(L), N))


# ---------------------------------------------------------------- geometry helpers
def test_viewer_and_lambda_bins():
    L = oracle.lib()
    import ctypes as C

    def vb(n):
        a = np.ascontiguousarray(n, dtype=np.float64)
        return L.xo_viewer_bin(a.ctypes.data, 20, 20)
    assert vb([0, 0, 1]) // 20 == 0
    assert vb([0, 0, -1]) // 20 == 19
    assert vb([1, 0, 0]) == 10 * 20 + 0            # theta = pi/2 exactly, phi = 0
    assert vb([0, 1, 0]) % 20 == 5                  # phi = pi/2
    assert vb([0, -1, 0]) % 20 == 15                # phi = 3pi/2
    th = np.linspace(0, np.pi, 21)
    dOm = 2 * np.pi / 20 * (np.cos(th[:-1]) - np.cos(th[1:]))
    assert 20 * dOm.sum() == pytest.approx(4 * np.pi, rel=1e-14)
    lam0, dlog = 3000.0, 1e-3
    for k in [0, 1, 17, 999]:
        mid = lam0 * (1 + dlog) ** (k + 0.5)
        assert L.xo_lambda_bin(mid, lam0, dlog, 1000) == k
    assert L.xo_lambda_bin(lam0 * 0.999, lam0, dlog, 1000) == -1
    assert L.xo_lambda_bin(lam0 * (1 + dlog) ** 1000.5, lam0, dlog, 1000) == -1


def test_spectrum_normalisation_and_isotropy():
    """The binned spectrum holds every escaped erg (the ledger counts them on
    its own); L_lambda per viewer is 4 pi / dOmega_k E / dlambda, so the
    solid-angle average of the viewers' luminosities and the angle-summed
    L_lambda both integrate back to it; and a spherically symmetric source
    of isotropic emission lights every viewer in proportion to its solid angle
    (chi-square over the 400 viewers)."""
    w = synth.uniform_sphere(n_packets=40_000)
    o = oracle.transport(w)
    spec, led = o["spec"], o["ledger"]
    E = spec.sum()
    assert E == pytest.approx(led["esc_E"] - led["oob_E"], rel=1e-12)
    lam0, nb = w.spec_band_A
    L_k, L_tot, edges = oracle.spectrum_L_lambda(spec, lam0, 1e-3)
    dlam = np.diff(edges)
    th = np.linspace(0.0, np.pi, 21)
    dOm = np.repeat(2 * np.pi / 20 * (np.cos(th[:-1]) - np.cos(th[1:])), 20)
    assert (L_tot * dlam).sum() == pytest.approx(E, rel=1e-12)
    assert ((dOm / (4 * np.pi))[:, None] * L_k * dlam[None, :]).sum() == pytest.approx(E, rel=1e-12)
    # isotropy: energy per viewer against E dOmega_k / 4 pi, variance from the
    # packets' spread of energies
    Ek = spec.sum(axis=1)
    expect = E * dOm / (4 * np.pi)
    n_esc = 40_000 * (led["esc_N"] / led["emit_N"])       # escaped packets, about
    mean_e = E / n_esc
    chi2 = np.sum((Ek - expect) ** 2 / (expect * mean_e * 1.2))
    assert chi2 / 400 < 1.6, chi2 / 400


# ---------------------------------------------------------------- P4
@pytest.mark.parametrize("n_scale", [1e-9, 1e-7, 3e-6])
def test_single_resonance_exact(n_scale):
    w = synth.single_line_sphere(n=1, n_packets=4000, seed=11, n_scale=n_scale)
    nu_l = 2.99792458e10 / (w.lambda_A[0] * 1e-8)
    # emit just blueward of the line so that every packet meets it at once
    w.band_A = (2.99792458e10 / (nu_l * (1 + 2e-9)) * 1e8, 2.99792458e10 / (nu_l * (1 + 1e-9)) * 1e8)
    o = oracle.transport(w, per_packet=True)
    pk = o["pkt"]
    tau = brute.tau_f_form(w, 0, 0)
    assert tau > 1e-4
    lo, up = w.lo[0], w.up[0]
    fcorr = 1 - w.g_level[lo] * w.pops[0, up] / (w.g_level[up] * w.pops[0, lo])
    hit = pk[:, 1] == 1
    assert hit.mean() > 0.999
    esc = hit & (pk[:, 0] == 0)
    if np.exp(-tau) > 1e-5:
        assert esc.sum() == hit.sum()
        np.testing.assert_allclose(pk[esc, 2], pk[esc, 8] * np.exp(-tau), rtol=1e-13)
    S_exact = np.sum(pk[hit, 8] * (-np.expm1(-tau)) / fcorr)
    assert o["S"][0, 0] == pytest.approx(S_exact, rel=1e-12)


# ---------------------------------------------------------------- P5
def _scaled_sphere(n, n_lines, scale, seed, n_packets):
    w = synth.uniform_sphere(seed=seed, n_packets=n_packets, n=n, n_lines=n_lines)
    w.pops = w.pops * scale
    return w


@pytest.mark.parametrize("scale", [1e-6, 1e-4])
def test_event_histories_vs_brute_force(scale):
    w = _scaled_sphere(4, 150, scale, seed=4, n_packets=3000)
    qoff = brute.largest_remainder(list(w.L_cell), w.n_packets)
    Lc, q_or = oracle.emission(w)
    assert np.array_equal(q_or, qoff)
    n_checked = n_events = 0
    for p in range(0, w.n_packets, 19):
        o = oracle.transport(w, p_begin=p, p_end=p + 1, per_packet=True, sparse=True)
        ev, fate, N_fin, n_dir, nu_lab = brute.brute_packet(w, p, qoff)
        pk = o["pkt"][0]
        assert int(pk[1]) == len(ev), f"packet {p}"
        assert int(pk[0]) == fate
        assert pk[2] == pytest.approx(N_fin, rel=1e-11, abs=1e-300)
        got = {}
        for s, v in zip(o["S_slots"], o["S_values"]):
            got[int(s)] = v
        want = {}
        for cell, l, v in ev:
            want[cell * w.nline + l] = want.get(cell * w.nline + l, 0.0) + v
        assert set(got) == set(want), f"packet {p}"
        for k in want:
            assert got[k] == pytest.approx(want[k], rel=1e-11)
        if fate == 0:
            assert pk[10] == pytest.approx(nu_lab, rel=1e-14)
        n_checked += 1
        n_events += len(ev)
    assert n_checked > 100 and n_events > 60


# ---------------------------------------------------------------- P2
def _hatbox_expected(w, lam_l, edges, Lc, sub=12):
    """Expected escaped lab energy per wavelength bin for an optically thin
    line source: isotropic directions give z = n.r0 uniform on [-|r0|,|r0|]
    (Archimedes' hat-box theorem); lab energy = E0 / (1 - z/ct); lambda_lab =
    lambda_l (1 - z/ct).  Integrated over each emitting cell by a midpoint rule."""
    R = w.v_max * w.t
    d = 2 * R / w.nx
    ct = 2.99792458e10 * w.t
    zb = ct * (1 - edges / lam_l)            # descending in z
    za, zb_ = zb[1:], zb[:-1]                # bin k covers z in [za, zb_]
    g = (np.arange(sub) + 0.5) / sub
    out = np.zeros(len(edges) - 1)
    cells = np.nonzero(Lc > 0)[0]
    for c in cells:
        ix, iy, iz = c % w.nx, (c // w.nx) % w.ny, c // (w.nx * w.ny)
        x = -R + (ix + g) * d
        y = -R + (iy + g) * d
        zc = -R + (iz + g) * d
        X, Y, Z = np.meshgrid(x, y, zc, indexing="ij")
        r = np.sqrt(X * X + Y * Y + Z * Z).reshape(-1)
        lo = np.maximum(za[None, :], -r[:, None])
        hi = np.minimum(zb_[None, :], r[:, None])
        F = lambda z: -ct * np.log(1 - z / ct)
        val = np.where(hi > lo, (F(hi) - F(lo)) / (2 * r[:, None]), 0.0)
        out += Lc[c] * val.mean(axis=0)
    return out


def test_thin_line_profile_hatbox():
    w = synth.single_line_sphere(n=8, n_packets=400_000, seed=21, n_scale=1e-30)
    o = oracle.transport(w, emission="lines")
    Lc, _ = oracle.emission(w, emission="lines")
    lam0, nb = w.spec_band_A
    edges = lam0 * (1 + 1e-3) ** np.arange(nb + 1)
    spec = o["spec"].sum(axis=0)
    exp_ = _hatbox_expected(w, w.lambda_A[0], edges, Lc, sub=20)
    # no absorption: every packet escapes; total lab energy exactly sum E0/D
    assert o["ledger"]["events"] == 0
    assert spec.sum() == pytest.approx(exp_.sum(), rel=2e-3)
    # quadrature resolution check
    exp2 = _hatbox_expected(w, w.lambda_A[0], edges, Lc, sub=14)
    assert np.max(np.abs(exp2 - exp_)) < 1e-3 * exp_.max()
    m = exp_ > 1e-3 * exp_.max()
    E_pk = Lc.sum() / w.n_packets
    sig = np.sqrt(np.maximum(exp_, E_pk) * E_pk * 1.05)
    chi2 = np.sum(((spec - exp_)[m] / sig[m]) ** 2) / m.sum()
    assert 0.6 < chi2 < 1.5, chi2
    # a mistake in the Doppler sign or scale moves the profile by whole bins
    mean_mc = (spec * np.sqrt(edges[1:] * edges[:-1])).sum() / spec.sum()
    mean_ex = (exp_ * np.sqrt(edges[1:] * edges[:-1])).sum() / exp_.sum()
    assert mean_mc == pytest.approx(mean_ex, rel=2e-5)


# ---------------------------------------------------------------- P3
def _slab_workload(n=6, n_packets=600_000, tau_target=2e-3):
    w = synth.single_line_sphere(n=n, n_packets=n_packets, seed=33)
    ncell = n ** 3
    # matter everywhere, light only from the corner cell (0,0,0)
    w.n_ion_density = np.ones((ncell, 1)) * 1.0
    w.pops = synth.lte_populations(w.n_ion_density, w.level_off, w.E_level, w.g_level, w.Te)
    tau1 = brute.tau_f_form(w, 0, 0)
    w.pops = w.pops * (tau_target / tau1)
    w.L_cell = np.zeros(ncell)
    w.L_cell[0] = 1e38
    nu_l = 2.99792458e10 / (w.lambda_A[0] * 1e-8)
    w.band_A = (2.99792458e10 / (nu_l * 1.08) * 1e8, 2.99792458e10 / (nu_l * 0.999) * 1e8)
    return w


def test_thin_estimator_slab_quadrature():
    w = _slab_workload()
    n = w.nx
    o = oracle.transport(w)
    R = w.v_max * w.t
    d = 2 * R / n
    ct = 2.99792458e10 * w.t
    tau = brute.tau_f_form(w, 0, 0)
    lo, up = w.lo[0], w.up[0]
    fcorr = 1 - w.g_level[lo] * w.pops[0, up] / (w.g_level[up] * w.pops[0, lo])
    nu_l = 2.99792458e10 / (w.lambda_A[0] * 1e-8)
    nu_lo, nu_hi = 2.99792458e10 / (w.band_A[1] * 1e-8), 2.99792458e10 / (w.band_A[0] * 1e-8)
    xg, wg = np.polynomial.legendre.leggauss(5)
    xg = 0.5 * (xg + 1)
    wg = 0.5 * wg
    # source points (cell 0,0,0)
    S3 = np.stack(np.meshgrid(xg, xg, xg, indexing="ij"), -1).reshape(-1, 3)
    W3 = np.einsum("i,j,k->ijk", wg, wg, wg).reshape(-1)
    src = -R + S3 * d
    total_exp = total_mc = 0.0
    for iz in range(n):
        for iy in range(n):
            for ix in range(2, n):        # slab with a one-cell gap to the source
                tgt = -R + (np.array([ix, iy, iz]) + S3) * d
                diff = tgt[None, :, :] - src[:, None, :]
                s = np.linalg.norm(diff, axis=-1)
                nvec = diff / s[..., None]
                ndotr = np.einsum("ijk,ijk->ij", nvec, tgt[None, :, :].repeat(src.shape[0], 0))
                # the frequency the packet needs at emission must lie in the band
                D0ct = ct - np.einsum("ijk,ik->ij", nvec, src)
                nu0 = nu_l / (1 - s / D0ct)
                inband = (nu0 >= nu_lo) & (nu0 <= nu_hi)
                integrand = np.where(inband, 1.0 / (s * s * (ct - ndotr)), 0.0)
                I = np.einsum("i,j,ij->", W3, W3, integrand) * d ** 6
                c = (iz * n + iy) * n + ix
                total_exp += I
                total_mc += o["S"][c, 0]
    H = 6.62607015e-27
    Vs = d ** 3
    pref = w.L_cell[0] / (H * (nu_hi - nu_lo)) * (-np.expm1(-tau)) / fcorr / (4 * np.pi * Vs)
    total_exp *= pref
    # MC noise: each hit adds about N0 tau/f_corr
    N0 = w.L_cell[0] / w.n_packets / (H * nu_l)
    hit = N0 * (-np.expm1(-tau)) / fcorr
    sigma = np.sqrt(total_exp * hit)
    assert abs(total_mc - total_exp) < 4 * sigma, (total_mc, total_exp, sigma)
    assert abs(total_mc / total_exp - 1) < 0.02


# ---------------------------------------------------------------- P6
def test_ledgers_close():
    w = synth.uniform_sphere(n_packets=20_000)
    L = oracle.transport(w)["ledger"]
    assert (L["esc_N"] + L["abs_N"] + L["drop_N"]) == pytest.approx(L["emit_N"], rel=1e-13)
    assert L["emit_E"] == pytest.approx(1e40, rel=1e-12)
    Ls = oracle.transport(w, mode="scatter")["ledger"]
    assert Ls["interactions"] > 1000
    assert (Ls["reemit_E_cmf"] + Ls["thermal_E"]) == pytest.approx(Ls["abs_E_cmf"], rel=1e-13)


def test_scatter_channel_probability():
    """Scatter mode, one line: an interaction destroys the packet with
    probability C_ul / (C_ul + A_ul beta_S) and re-emits it in the line
    otherwise.  In a uniform sphere every cell has the same C, A and beta, so
    the destroyed fraction of all interactions is that probability within its
    binomial error (C and A beta written out from their definitions)."""
    w = synth.single_line_sphere(n=8, n_packets=60_000, f_lu=3e-3, n_scale=1.0)
    o = oracle.transport(w, mode="scatter", per_packet=True)
    pk = o["pkt"]
    fate, inter = pk[:, 0], pk[:, 6]
    n_int = float(inter.sum())
    n_destroyed = float((fate == 2).sum())
    c = int(np.nonzero(w.rho > 0)[0][0])
    g_l, g_u = w.g_level[0], w.g_level[1]
    n_l, n_u = w.pops[c, 0], w.pops[c, 1]
    lam = w.lambda_A[0] * 1e-8
    A = 8 * np.pi ** 2 * 4.80320471e-10 ** 2 / (9.1093837015e-28 * 2.99792458e10 * lam ** 2) * (g_l / g_u) * w.f_lu[0]
    K = np.pi * 4.80320471e-10 ** 2 / (9.1093837015e-28 * 2.99792458e10) * w.f_lu[0] * lam * w.t
    tau = K * (n_l - g_l / g_u * n_u)
    beta = -np.expm1(-tau) / tau
    ups = synth.collision_strengths(w.upsilon_seed, w.level_off)[0][0, 1]
    C = 8.629e-6 * w.ne[c] * ups / (g_u * np.sqrt(w.Te[c]))
    p = C / (C + A * beta)
    assert tau > 1.0 and 0.05 < p < 0.95, (tau, p)
    assert n_int > 2000
    sigma = np.sqrt(p * (1 - p) / n_int)
    assert abs(n_destroyed / n_int - p) < 4 * sigma, (n_destroyed / n_int, p, sigma)
