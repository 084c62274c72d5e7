"""Pins of the oracle's photoionization (Sec. 2.3.1, Eq. sigma_OTSPI) against
things other than itself (no GPU).

- The cross section against Kramers' hydrogenic bound-free cross section,
  written from the physical constants (Rybicki & Lightman, Sec. 10.5):
  sigma = (64 pi^4 m_e e^10 / (3 sqrt(3) c h^6)) Z^4 / (n^5 nu^3), for the
  levels n of a hydrogenic ion of charge Z - 1.
- One cell, one level: every packet's surviving photons N0 e^-tau with
  tau = sigma(lambda_emit) n l, l the path to the cube wall from an
  independent restatement of the emission (numpy's Philox); the absorbed
  photons and the heating they bring.
- Two levels share the absorption in proportion to sigma_i n_i.
- A threshold crossed in flight: the path length stops where the comoving
  frequency, found by bisection along the ray, reaches the threshold.
- Optically thin uniform sphere: Gamma_PI(r) = 4 pi J(r) sig c^3 / (3 h)
  (nu_th^-3 - nu_hi^-3) with the closed-form J(r) of a uniformly emitting
  sphere and sigma = sig lambda^3, to Monte Carlo error.
- The photon ledger closes with photoionization as a sink.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import oracle_brute as brute

C = 2.99792458e10
H = 6.62607015e-27
ME = 9.1093837015e-28
E_CH = 4.80320471e-10
EV = 1.602176634e-12


def test_sigma_pi_is_kramers_hydrogenic():
    K = 64 * np.pi ** 4 * ME * E_CH ** 10 / (3 * np.sqrt(3) * C * H ** 6)
    Ry = 2 * np.pi ** 2 * ME * E_CH ** 4 / H ** 2            # erg
    for Z in (1, 2, 3):
        E_ion = Z * Z * Ry
        for n in (1, 2, 3, 5):
            E_u = E_ion * (1 - 1 / n ** 2)
            nu_n = (E_ion - E_u) / H
            for x in (1.0, 1.3, 2.0, 5.0):                  # nu / nu_threshold
                nu = x * nu_n
                kram = K * Z ** 4 / (n ** 5 * nu ** 3)
                got = oracle.sigma_pi(C / nu, E_u, E_ion, Z - 1)
                # the paper's 7.9e-18 is Kramers' threshold value rounded
                assert got == pytest.approx(kram, rel=2e-3), (Z, n, x)


def _one_cell(n_packets=3000, band_over_threshold=(1.15, 1.35), n_pi=1, scale=1.0, seed=51):
    """One cell (the whole cube), a single ion whose lowest n_pi levels
    photoionize, lines too weak to interact; emission flat in nu within the
    given band in units of the lowest threshold frequency."""
    w = synth.uniform_sphere(n=1, n_packets=n_packets, n_lines=5, n_levels=8, seed=seed)
    w.f_lu = np.full(w.nline, 1e-30)
    synth.with_photoionization(w, chi_eV=6.0, charge=0, pi_nlev=n_pi)
    nu_th = (w.chi_ion[0] - w.E_level[0]) / H      # the highest threshold (ground level)
    w.band_A = (C / (nu_th * band_over_threshold[1]) * 1e8, C / (nu_th * band_over_threshold[0]) * 1e8)
    w.spec_band_A = synth._spectrum_grid(w.band_A[0], w.band_A[1], w.v_max)
    w.pops = np.full_like(w.pops, scale)
    return w


def _paths(w, ids):
    """Emission point, direction, comoving and lab frequency and the path to
    the cube wall of packets `ids` (one cell), restated with numpy's Philox."""
    R = w.v_max * w.t
    out = []
    nu_lo, nu_hi = C / (w.band_A[1] * 1e-8), C / (w.band_A[0] * 1e-8)
    for p in ids:
        u = brute.philox_uniforms(w.seed, p, 0)
        v = brute.philox_uniforms(w.seed, p, 1)
        r0 = -R + u[:3] * 2 * R
        mu = 2 * u[3] - 1
        ph = 2 * np.pi * v[0]
        st = np.sqrt(1 - mu * mu)
        nv = np.array([st * np.cos(ph), st * np.sin(ph), mu])
        with np.errstate(divide="ignore"):
            t = np.where(nv > 0, (R - r0) / nv, np.where(nv < 0, (-R - r0) / nv, np.inf))
        nu0 = nu_lo + v[1] * (nu_hi - nu_lo)
        nu_lab = nu0 / (1 - nv @ r0 / (C * w.t))
        out.append((r0, nv, nu0, nu_lab, float(t.min())))
    return out


def test_single_cell_attenuation_and_heating():
    w = _one_cell(scale=2.0)
    o = oracle.transport(w, per_packet=True)
    pk = o["pkt"]
    lev, eion, _ = synth.pi_levels(w)
    chi = eion[0] - w.E_level[lev[0]]
    tau = np.zeros(w.n_packets)
    for p, (r0, nv, nu0, nu_lab, ell) in enumerate(_paths(w, range(w.n_packets))):
        sig = oracle.sigma_pi(C / nu0, w.E_level[lev[0]], eion[0], 0)
        tau[p] = sig * ell * w.pops[0, lev[0]]
    assert 0.05 < np.median(tau) < 20
    alive = pk[:, 0] == 0
    np.testing.assert_allclose(pk[alive, 2], pk[alive, 8] * np.exp(-tau[alive]), rtol=1e-12)
    absorbed = pk[:, 8] * -np.expm1(-tau)
    # packets that fell below the energy cut lost their rest to the cut, not to photoionization
    dropped = pk[:, 0] == 1
    assert dropped.sum() < w.n_packets // 2
    want = absorbed[alive].sum()
    L = o["ledger"]
    assert o["S_pi"][0, 0] == pytest.approx(L["pi_N"], rel=1e-13)
    # dropped packets: the segment absorbed N0 (1 - e^-tau') for a tau' <= tau;
    # only the surviving packets are pinned exactly
    assert L["pi_N"] >= want * (1 - 1e-12)
    heat_alive = (absorbed * (H * pk[:, 9] - chi))[alive].sum()
    assert o["heat"][0] >= heat_alive * (1 - 1e-12)
    if not dropped.any():
        assert o["S_pi"][0, 0] == pytest.approx(want, rel=1e-12)
        assert o["heat"][0] == pytest.approx(heat_alive, rel=1e-12)


def test_single_cell_no_drops_exact():
    """Thin enough that no packet reaches the energy cut: the absorbed photons
    and the heating equal the per-packet closed forms summed."""
    w = _one_cell(scale=0.05)
    o = oracle.transport(w, per_packet=True)
    pk = o["pkt"]
    assert np.all(pk[:, 0] == 0)
    lev, eion, _ = synth.pi_levels(w)
    chi = eion[0] - w.E_level[lev[0]]
    tau = np.array([oracle.sigma_pi(C / nu0, w.E_level[lev[0]], eion[0], 0) * ell * w.pops[0, lev[0]]
                    for (_, _, nu0, _, ell) in _paths(w, range(w.n_packets))])
    absorbed = pk[:, 8] * -np.expm1(-tau)
    np.testing.assert_allclose(pk[:, 2], pk[:, 8] * np.exp(-tau), rtol=1e-12)
    assert o["S_pi"][0, 0] == pytest.approx(absorbed.sum(), rel=1e-12)
    assert o["heat"][0] == pytest.approx((absorbed * (H * pk[:, 9] - chi)).sum(), rel=1e-12)


def test_two_levels_share_by_optical_depth():
    """Two photoionizing levels above threshold along the whole path: their
    absorbed photons stand in the ratio sigma_1 n_1 / (sigma_2 n_2) at every
    segment, hence in total (the lambda^3 factors are common)."""
    w = _one_cell(n_pi=2, scale=0.3)
    w.pops[0, 1] = 0.7                            # n_1 != n_0
    o = oracle.transport(w)
    lev, eion, _ = synth.pi_levels(w)
    lam = 4000e-8
    s0 = oracle.sigma_pi(lam, w.E_level[lev[0]], eion[0], 0)
    s1 = oracle.sigma_pi(lam, w.E_level[lev[1]], eion[1], 0)
    ratio = o["S_pi"][0, 0] / o["S_pi"][0, 1]
    assert ratio == pytest.approx(s0 * w.pops[0, lev[0]] / (s1 * w.pops[0, lev[1]]), rel=1e-12)


def test_threshold_crossed_in_flight():
    """Emission just above threshold: the comoving frequency falls below it
    along most paths, and the path length that photoionizes stops there."""
    w = _one_cell(band_over_threshold=(1.0002, 1.012), scale=0.05, n_packets=600)
    w.v_max = 5e9                                  # a large Doppler shift across the cell
    o = oracle.transport(w, per_packet=True)
    pk = o["pkt"]
    lev, eion, _ = synth.pi_levels(w)
    chi = eion[0] - w.E_level[lev[0]]
    nu_th = chi / H
    crossed = 0
    for p, (r0, nv, nu0, nu_lab, ell) in enumerate(_paths(w, range(w.n_packets))):
        f = lambda s: oracle.lib().xo_nu_cmf(nu_lab, nv.ctypes.data, r0.ctypes.data, s, w.t) - nu_th
        if f(ell) < 0:                             # bisection for the crossing point
            a, b = 0.0, ell
            for _ in range(200):
                m = 0.5 * (a + b)
                a, b = (m, b) if f(m) > 0 else (a, m)
            ell_pi = 0.5 * (a + b)
            crossed += 1
        else:
            ell_pi = ell
        tau = oracle.sigma_pi(C / nu0, w.E_level[lev[0]], eion[0], 0) * ell_pi * w.pops[0, lev[0]]
        assert pk[p, 2] == pytest.approx(pk[p, 8] * np.exp(-tau), rel=1e-9), p
    assert crossed > w.n_packets // 3


def _thin_pi_sphere(n=32, n_packets=1_000_000, seed=61):
    w = synth.uniform_sphere(n=n, n_packets=n_packets, n_lines=5, n_levels=20, seed=seed)
    w.v_max = 5e7
    w.f_lu = np.full(w.nline, 1e-30)                # no line interacts
    synth.with_photoionization(w, chi_eV=6.0, charge=1, pi_nlev=8)
    act = w.rho > 0
    w.pops = np.where(act[:, None], 1.0, 0.0) * np.linspace(1.0, 2.0, w.nlev)[None, :]
    return w


def test_thin_sphere_rates_closed_form():
    w = _thin_pi_sphere()
    o = oracle.transport(w)
    G = oracle.pi_rates(w, o["S_pi"])
    lev, eion, ch = synth.pi_levels(w)
    act = w.rho > 0
    R = w.v_max * w.t
    xc = synth.cell_centres(w.nx, w.v_max) * w.t
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2).reshape(-1)
    nu_lo, nu_hi = C / (w.band_A[1] * 1e-8), C / (w.band_A[0] * 1e-8)
    V = (2 * R / w.nx) ** 3
    j = w.L_cell[act][0] / V / (4 * np.pi * (nu_hi - nu_lo))
    rr = np.clip(r, 1e-9 * R, (1 - 1e-9) * R)
    J = j * R / 2 * (1 + (R * R - rr * rr) / (2 * rr * R) * np.log((R + rr) / (R - rr)))
    tested = 0
    for k in range(lev.shape[0]):
        chi = eion[k] - w.E_level[lev[k]]
        nu_th = chi / H
        sig = oracle.sigma_pi(1.0, w.E_level[lev[k]], eion[k], int(ch[k]))   # sigma at lambda = 1 cm
        if nu_th >= nu_hi * (1 - 2 * w.v_max / C):
            assert np.all(G[:, k] == 0), k                # threshold above every photon
            continue
        lo = max(nu_th, nu_lo)
        want = 4 * np.pi * J * sig * C ** 3 / (3 * H) * (lo ** -3 - nu_hi ** -3)
        for a, b in [(0, 0.4), (0.4, 0.6), (0.6, 0.8)]:
            m = act & (r / R >= a) & (r / R < b)
            ratio = G[m, k].sum() / want[m].sum()
            assert ratio == pytest.approx(1.0, abs=0.03), (k, a, b, ratio)
        tested += 1
    assert tested >= 3


def test_ledger_closes_with_photoionization():
    w = synth.uniform_sphere(n=8, n_packets=30_000, seed=71)
    synth.with_photoionization(w, chi_eV=6.0, charge=0, pi_nlev=9)
    w.pops = w.pops * 1e-3
    o = oracle.transport(w)
    L = o["ledger"]
    assert L["pi_N"] > 0.1 * L["emit_N"] and L["abs_N"] > 0.1 * L["emit_N"] and L["events"] > 10_000
    assert L["esc_N"] + L["abs_N"] + L["pi_N"] + L["drop_N"] == pytest.approx(L["emit_N"], rel=1e-13)
    assert o["S_pi"].sum() == pytest.approx(L["pi_N"], rel=1e-12)
