"""The spherical (r, theta, phi) grid on the GPU against the oracle, through
the C ABI (needs a GPU).  The paper's models are spherical grids of radial
shells, polar and azimuthal sectors (Sec. 2), split into azimuthal slices as
subdomains (Sec. 2.4.1).  Bars as for the cube: per-packet histories identical
(fates, event counts and emitting cells exact), estimators relative 1e-10,
spectra 1e-9, rates 1e-10, populations of the coupled loop 1e-6."""
import numpy as np
import pytest

import oracle
import synth
from oracle import coupled

pytestmark = pytest.mark.gpu

S_TOL = 1e-10
SPEC_TOL = 1e-9


@pytest.fixture(scope="module")
def xt():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a GPU"
    import __graft_entry__ as g
    g.build()
    import paper_2511_07539_gb300 as xt
    return xt


def _ctx(xt):
    import torch
    return xt.Context(0, torch.cuda.current_stream().cuda_stream)


def _cmp_sparse(got, want, tol, what):
    mg, mw = got != 0, want != 0
    assert np.array_equal(mg, mw), f"{what}: support differs ({mg.sum()} vs {mw.sum()})"
    if mw.any():
        err = np.max(np.abs(got[mw] / want[mw] - 1))
        assert err < tol, f"{what}: max rel err {err}"


def _records(xt, ctx, w, **kw):
    n = w.n_packets if kw.get("packet_count", -1) < 0 else kw["packet_count"]
    rec = np.zeros((n, xt.XT_PKT_FIELDS))
    st = ctx.transport(w, packet_records=rec, **kw)
    return st, rec


def _cmp_records(rec, pk):
    assert np.array_equal(rec[:, 0], pk[:, 0]), "fates differ"
    assert np.array_equal(rec[:, 1], pk[:, 1]), "event counts differ"
    assert np.array_equal(rec[:, 7], pk[:, 7]), "emitting cells differ"
    assert np.all(np.abs(rec[:, 2] - pk[:, 2]) <= 1e-12 * np.abs(pk[:, 2]) + 1e-15 * pk[:, 8])
    np.testing.assert_allclose(rec[:, 8], pk[:, 8], rtol=1e-13)
    np.testing.assert_allclose(rec[:, 9], pk[:, 9], rtol=1e-15)
    # the lab frequency carries the emission point's last bits (cbrt, sincos)
    np.testing.assert_allclose(rec[:, 10], pk[:, 10], rtol=1e-14)
    esc = pk[:, 0] == 0
    assert np.array_equal(rec[esc, 4], pk[esc, 4]), "viewer bins differ"
    assert np.array_equal(rec[esc, 5], pk[esc, 5]), "wavelength bins differ"


def _cmp_ledger(st, L):
    assert st["events"] == L["events"] and st["tests"] == L["tests"]
    for k, kk in [("emitted_N", "emit_N"), ("escaped_N", "esc_N"), ("absorbed_N", "abs_N"),
                  ("dropped_N", "drop_N"), ("escaped_E", "esc_E"), ("emitted_E", "emit_E")]:
        assert st[k] == pytest.approx(L[kk], rel=1e-12), k
    assert st["guard"] == 0


@pytest.mark.parametrize("clumps", [False, True])
def test_band_emission_parity(xt, clumps):
    """12 x 8 x 12 cells in four phi slices, 100 lines, 1e5 packets: histories,
    estimators, spectrum, ledger and the rates readout (per-cell volumes)."""
    w = synth.spherical_sphere(n_packets=100_000, seed=7, clumps=clumps)
    with _ctx(xt) as ctx:
        ctx.load(w)
        st, rec = _records(xt, ctx, w)
        S = ctx.get_estimators()
        spec = ctx.get_spectrum(0)
        R_lu, R_ul, J = ctx.get_photoexcitation_rates()
    o = oracle.transport(w, per_packet=True)
    pk = o["pkt"]
    assert (pk[:, 0] == 0).sum() > 1000 and (pk[:, 0] == 1).sum() > 1000   # both fates occur
    _cmp_records(rec, pk)
    _cmp_sparse(S, o["S"], S_TOL, "estimators")
    _cmp_sparse(spec, o["spec"], SPEC_TOL, "spectrum")
    _cmp_ledger(st, o["ledger"])
    r_or = oracle.rates(w, o["S"])
    _cmp_sparse(R_lu, r_or[0], S_TOL, "R_lu")
    _cmp_sparse(R_ul, r_or[1], S_TOL, "R_ul")
    _cmp_sparse(J, r_or[2], S_TOL, "Jbar")


def test_line_emission_parity(xt):
    """Line emission A_ul dE beta_S n_u V per cell with the spherical cells'
    volumes (Eq. thin_emissivity)."""
    w = synth.spherical_sphere(n_packets=60_000, seed=11, nr=8, nth=6, nph=10, subdomains=(1, 1, 5))
    with _ctx(xt) as ctx:
        ctx.load(w)
        st, rec = _records(xt, ctx, w, emission=xt.XT_EMIT_LINES)
        S = ctx.get_estimators()
        spec = ctx.get_spectrum(0)
    o = oracle.transport(w, emission="lines", per_packet=True)
    _cmp_records(rec, o["pkt"])
    _cmp_sparse(S, o["S"], S_TOL, "estimators")
    _cmp_sparse(spec, o["spec"], SPEC_TOL, "spectrum")
    _cmp_ledger(st, o["ledger"])


@pytest.mark.parametrize("sd,compact", [((1, 1, 1), False), ((2, 2, 3), False), ((1, 1, 12), True)])
def test_store_layouts(xt, sd, compact):
    """The subdomain blocking of the store and its compact rows change nothing
    (cells without matter, here a quarter of the phi slices, get no rows)."""
    w = synth.spherical_sphere(n_packets=40_000, seed=13)
    empty = np.repeat(np.arange(w.nz) % 4 == 1, w.nx * w.ny)
    w.pops[empty] = 0.0
    w.n_ion_density[empty] = 0.0
    with _ctx(xt) as ctx:
        ctx.load(w, subdomains=sd)
        if compact:
            xt.set_estimator_store(ctx.h, xt.XT_STORE_COMPACT_ROWS)
        st, rec = _records(xt, ctx, w)
        S = ctx.get_estimators()
        st2 = ctx.transport(w)                    # a second pass clears through the slot log
        S2 = ctx.get_estimators()
    o = oracle.transport(w, per_packet=True)
    _cmp_records(rec, o["pkt"])
    _cmp_sparse(S, o["S"], S_TOL, "estimators")
    _cmp_sparse(S2, o["S"], S_TOL, "estimators, second pass")
    assert np.all(S[empty] == 0)
    assert st2["events"] == st["events"]


def test_single_phi_sector_and_equator(xt):
    """One azimuthal sector (no half-planes) and an odd number of polar
    sectors (no equatorial edge), then an even number (the plane z = 0)."""
    for nth in (5, 6):
        w = synth.spherical_sphere(n_packets=30_000, seed=17, nr=6, nth=nth, nph=1, subdomains=(1, 1, 1))
        with _ctx(xt) as ctx:
            ctx.load(w)
            st, rec = _records(xt, ctx, w)
            S = ctx.get_estimators()
        o = oracle.transport(w, per_packet=True)
        _cmp_records(rec, o["pkt"])
        _cmp_sparse(S, o["S"], S_TOL, f"estimators (nth {nth})")


def test_rejected_passes(xt):
    """What the spherical path does not take is refused (XT_EINVAL) before any
    work; bad edges are refused by init_grid."""
    w = synth.spherical_sphere(n_packets=1000, seed=1)
    with _ctx(xt) as ctx:
        ctx.load(w)
        for kw in [dict(mode=xt.XT_MODE_SCATTER), dict(subdomain_rounds=True)]:
            rc, _ = ctx.transport(w, check=False, **kw)
            assert rc == xt.XT_EINVAL, kw
        xt.set_estimator_store(ctx.h, 1)
        rc, _ = ctx.transport(w, check=False)
        assert rc == xt.XT_EINVAL
        xt.set_estimator_store(ctx.h, 0)
        ctx.transport(w)                          # still usable
        bad = [(w.r_edges[::-1].copy(), w.theta_edges, w.phi_edges),
               (w.r_edges, w.theta_edges * 0.5, w.phi_edges),
               (w.r_edges, w.theta_edges, w.phi_edges[:-1])]
        for e in bad:
            with pytest.raises((xt.XtError, ValueError)):
                xt.init_grid(ctx.h, w.nx, w.ny, w.nz, w.v_max, w.t, w.Te, w.ne, w.L_cell, w.band_A,
                             spherical_edges=e)


def test_paper_grid_sampled(xt):
    """The paper's grid (38 x 15 x 30 cells, Sec. 2) with 1e4 lines and 4e6
    packets in one launch: ledger closure, then packets sampled
    across the id range traced alone on both sides (their histories and
    estimators compared one by one)."""
    w = synth.spherical_sphere(n_packets=4_000_000, seed=23, nr=38, nth=15, nph=30, n_lines=10_000,
                               n_levels=200, subdomains=(1, 1, 30), clumps=True)
    w.pops = w.pops * 1e-6            # about 35 events per packet; 40 % escape
    with _ctx(xt) as ctx:
        ctx.load(w)
        st = ctx.transport(w)
        assert st["guard"] == 0 and st["events"] > 1e6
        assert st["escaped_N"] + st["absorbed_N"] + st["dropped_N"] == pytest.approx(st["emitted_N"], rel=1e-12)
        for b in (0, 1_234_567, 3_999_000):
            st_b, rec = _records(xt, ctx, w, packet_begin=b, packet_count=1000)
            S = ctx.get_estimators()
            o = oracle.transport(w, p_begin=b, p_end=b + 1000, per_packet=True, sparse=True)
            _cmp_records(rec, o["pkt"])
            slots, v = o["S_slots"], o["S_values"]
            got = S.ravel()[slots]
            assert np.all(np.abs(got / v - 1) < S_TOL)
            assert np.count_nonzero(S) == np.count_nonzero(v)


@pytest.mark.parametrize("precision", [0, 1])
def test_coupled_loop_vs_oracle(xt, precision):
    """The coupled NLTE / transport loop on a 6 x 4 x 6 spherical grid from
    Boltzmann populations: the same outer steps and populations as the
    oracle's loop (rates with the spherical cells' volumes)."""
    w = synth.spherical_sphere(n_packets=50_000, seed=4, nr=6, nth=4, nph=6, subdomains=(1, 1, 2))
    w.upsilon = synth.collision_strengths(4, w.level_off)
    with _ctx(xt) as ctx:
        ctx.load(w)
        st = xt.run_coupled(ctx.h, w.upsilon, w.n_packets, seed=w.seed, start=xt.XT_WARM_LTE,
                            tol=1e-4, precision=precision, newton_tol=1e-10,
                            spec_lam0_A=w.spec_band_A[0], spec_nbins=w.spec_band_A[1])
        got = np.zeros((w.ncell, w.nlev))
        xt.get_populations(ctx.h, got)
    ref, steps, hist = coupled.coupled_loop(w, tol=1e-4, newton_tol=1e-10)
    assert st["converged"] and steps == st["outer"], (st, hist)
    worst = 0.0
    nz = w.n_ion_density[:, :1]
    m = (ref >= 1e-30 * nz) & (nz > 0)
    worst = float(np.max(np.abs(got[m] / ref[m] - 1)))
    assert worst < 1e-6


@pytest.mark.parametrize("emission", ["band", "lines"])
def test_rays_on_the_spherical_grid(xt, emission):
    """The RAYS sampler on the spherical grid (Sec. 2.3, the paper's pass): rays
    from the middle of every emitting cell's r, theta and phi ranges, one per
    emitting bin and viewer; histories, estimators and spectrum against the
    oracle.  The 7 x 7 viewers share no direction with the cells' middles (a
    viewer centre at a cell's middle azimuth sends that cell's ray through the
    polar axis, where the next sector is a rounding matter on both sides; the
    paper's 20 x 20 viewers on its 38 x 15 x 30 grid share none either)."""
    w = synth.spherical_sphere(n_packets=1, seed=9, nr=6, nth=4, nph=6, subdomains=(1, 1, 3))
    kw = dict(sampler=xt.XT_SAMPLER_RAYS, n_theta=7, n_phi=7, spec_dlog=0.01)
    em = xt.XT_EMIT_BAND if emission == "band" else xt.XT_EMIT_LINES
    if emission == "lines":
        w.spec_band_A = synth._spectrum_grid(2800.0, 10500.0, w.v_max, dlog=0.01)
    with _ctx(xt) as ctx:
        ctx.load(w)
        st0 = ctx.transport(w, packet_count=0, emission=em, **kw)
        nr = int(st0["rays"])
        rec = np.zeros((nr, xt.XT_PKT_FIELDS))
        st = ctx.transport(w, packet_records=rec, emission=em, **kw)
        S = ctx.get_estimators()
        spec = ctx.get_spectrum(0)
    o = oracle.transport(w, sampler="rays", emission=emission, n_theta=7, n_phi=7, spec_dlog=0.01,
                         per_packet=True)
    assert o["n"] == nr and st["events"] > 1000
    pk = o["pkt"]
    assert np.array_equal(rec[:, 0], pk[:, 0]) and np.array_equal(rec[:, 1], pk[:, 1])
    assert np.array_equal(rec[:, 7], pk[:, 7])
    live = pk[:, 0] != 4
    np.testing.assert_allclose(rec[live, 8], pk[live, 8], rtol=1e-12)
    np.testing.assert_allclose(rec[live, 10], pk[live, 10], rtol=1e-13)
    _cmp_sparse(S, o["S"], S_TOL, "estimators")
    _cmp_sparse(spec, o["spec"], SPEC_TOL, "spectrum")
    L = o["ledger"]
    assert st["events"] == L["events"] and st["tests"] == L["tests"]
    assert st["emitted_E"] == pytest.approx(L["emit_E"], rel=1e-9)
