"""Photoionization on the GPU (Sec. 2.3.1, Eq. sigma_OTSPI) against the CPU
oracle, through the C ABI (needs a GB300).

Bars as for the line estimators: photoionization rates and heating relative
1e-10, line estimators 1e-10, spectra 1e-9, packet histories identical (fates
and event counts exact), ledger 1e-12."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


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


def _cmp(got, want, tol, what):
    mg, mw = got != 0, want != 0
    assert np.array_equal(mg, mw), f"{what}: support differs ({mg.sum()} vs {mw.sum()})"
    if mw.any():
        err = np.max(np.abs(got[mw] / want[mw] - 1))
        assert err < tol, f"{what}: max rel err {err}"


def _cmp_rates(got, want, what):
    """Photoionization rates: relative 1e-10, except where a level's rate in
    a cell comes only from path pieces that end at its threshold a hair after
    they start.  Such a piece's length is the distance to the point where the
    comoving frequency reaches the threshold, a difference of nearly equal
    frequencies that both sides form from positions rounded differently: its
    absolute error is about 1e-16 of the distance travelled, far below 1e-12
    of a whole cell's worth of the level's rate.  So each element must be
    within 1e-10 of itself or 1e-12 of the level's largest rate."""
    mg, mw = got != 0, want != 0
    scale = np.abs(want).max(axis=0, keepdims=True)
    ok = np.abs(got - want) <= np.maximum(TOL * np.abs(want), 1e-12 * scale)
    assert ok.all(), f"{what}: {np.count_nonzero(~ok)} elements off, worst rel " \
        f"{np.max(np.abs(got[mw] / want[mw] - 1))}"
    assert np.array_equal(mg & (want > 1e-12 * scale), mw & (want > 1e-12 * scale)), f"{what}: support"


def _check_pass(xt, ctx, w, **kw):
    n = w.n_packets
    rec = np.zeros((n, xt.XT_PKT_FIELDS))
    st = ctx.transport(w, packet_records=rec, **kw)
    o = oracle.transport(w, per_packet=True)
    pk = o["pkt"]
    assert np.array_equal(rec[:, 0], pk[:, 0]), "fates differ"
    assert np.array_equal(rec[:, 1], pk[:, 1]), "event counts differ"
    assert np.all(np.abs(rec[:, 2] - pk[:, 2]) <= 1e-12 * np.abs(pk[:, 2]) + 1e-15 * pk[:, 8])
    _cmp(ctx.get_estimators(), o["S"], TOL, "line estimators")
    G, heat = ctx.get_photoionization_rates()
    _cmp_rates(G, oracle.pi_rates(w, o["S_pi"]), "photoionization rates")
    np.testing.assert_allclose(heat, o["heat"], rtol=TOL, atol=1e-12 * np.abs(o["heat"]).max())
    _cmp(ctx.get_spectrum(0), o["spec"], 1e-9, "spectrum")
    L = o["ledger"]
    assert st["events"] == L["events"] and st["tests"] == L["tests"]
    # ledger sums: relative to the emission (a sum that cancels to ~0, such as
    # the lines' share when no line absorbs, keeps only rounding)
    tol = 1e-12 * st["emitted_N"]
    assert abs(st["photoionized_N"] - L["pi_N"]) <= tol
    assert st["photoionized_E"] == pytest.approx(L["pi_E"], rel=1e-12)
    assert abs(st["absorbed_N"] - L["abs_N"]) <= tol
    assert st["escaped_N"] + st["absorbed_N"] + st["photoionized_N"] + st["dropped_N"] == \
        pytest.approx(st["emitted_N"], rel=1e-12)
    return st, o


@pytest.mark.parametrize("sd,rounds", [((1, 1, 1), False), ((4, 4, 4), False), ((4, 2, 8), True)])
def test_sphere_with_photoionization(xt, sd, rounds):
    w = synth.uniform_sphere(n_packets=60_000, seed=71, subdomains=sd)
    synth.with_photoionization(w, chi_eV=6.0, charge=0, pi_nlev=9)
    w.pops = w.pops * 1e-3
    with _ctx(xt) as ctx:
        ctx.load(w)
        st, o = _check_pass(xt, ctx, w, subdomain_rounds=rounds)
        assert o["ledger"]["pi_N"] > 0.1 * o["ledger"]["emit_N"]
        if rounds:
            assert st["rounds"] > 1


def test_threshold_crossed_in_flight(xt):
    """One cell at a large velocity: the comoving frequency of most packets
    falls through the threshold inside the cell (the crossed-level path)."""
    w = synth.uniform_sphere(n=2, n_packets=20_000, n_lines=5, n_levels=8, seed=51)
    w.f_lu = np.full(w.nline, 1e-30)
    synth.with_photoionization(w, chi_eV=6.0, charge=1, pi_nlev=3)
    nu_th = (w.chi_ion[0] - w.E_level[0]) / 6.62607015e-27
    c = 2.99792458e10
    w.band_A = (c / (nu_th * 1.02) * 1e8, c / (nu_th * 0.995) * 1e8)
    w.spec_band_A = synth._spectrum_grid(w.band_A[0], w.band_A[1], w.v_max)
    w.v_max = 5e9
    w.pops = np.full_like(w.pops, 0.05)
    with _ctx(xt) as ctx:
        ctx.load(w)
        _check_pass(xt, ctx, w)


def test_onion_with_photoionization_subset(xt):
    """32^3 onion, 10 ions x 9 photoionizing levels (90), 1e4 lines: a packet
    subset, every photoionization rate and line estimator."""
    w = synth.clumpy_onion(n=32, n_lines=10_000, n_packets=2_000_000, subdomains=(4, 4, 4), seed=3)
    synth.with_photoionization(w)
    w.pops = w.pops * 1e-4
    with _ctx(xt) as ctx:
        ctx.load(w)
        p0, m = 700_001, 40_000
        st = ctx.transport(w, packet_begin=p0, packet_count=m)
        o = oracle.transport(w, p_begin=p0, p_end=p0 + m, sparse=False)
        _cmp(ctx.get_estimators(), o["S"], TOL, "line estimators")
        G, heat = ctx.get_photoionization_rates()
        _cmp_rates(G, oracle.pi_rates(w, o["S_pi"]), "photoionization rates")
        np.testing.assert_allclose(heat, o["heat"], rtol=TOL, atol=1e-12 * np.abs(o["heat"]).max())
        assert st["photoionized_N"] == pytest.approx(o["ledger"]["pi_N"], rel=1e-12)
        assert o["ledger"]["pi_N"] > 0


def test_scatter_mode_with_photoionization_is_refused(xt):
    w = synth.uniform_sphere(n=6, n_packets=1000, seed=72)
    synth.with_photoionization(w, chi_eV=6.0)
    with _ctx(xt) as ctx:
        ctx.load(w, with_scatter_data=oracle.upsilon_down_sums(w))
        with pytest.raises(xt.XtError) as e:
            ctx.transport(w, mode=xt.XT_MODE_SCATTER)
        assert e.value.code == xt.XT_EINVAL and "attenuation" in str(e.value)


def test_spherical_grid_with_photoionization(xt):
    """Photoionization on every segment of the spherical walk (the paper's
    grid): histories, rates, heating, estimators, spectrum and ledger against
    the oracle."""
    w = synth.spherical_sphere(n_packets=60_000, seed=71, clumps=True)
    synth.with_photoionization(w, chi_eV=6.0, charge=0, pi_nlev=9)
    w.pops = w.pops * 1e-3
    with _ctx(xt) as ctx:
        ctx.load(w)
        st, o = _check_pass(xt, ctx, w)
        assert o["ledger"]["pi_N"] > 0.05 * o["ledger"]["emit_N"]


def test_spherical_rays_with_photoionization(xt):
    """The RAYS sampler with photoionization on the spherical grid (7 x 7
    viewers: no viewer centre at a cell's middle direction)."""
    w = synth.spherical_sphere(n_packets=1, seed=72, nr=6, nth=4, nph=6, subdomains=(1, 1, 3))
    synth.with_photoionization(w, chi_eV=6.0, charge=0, pi_nlev=9)
    w.pops = w.pops * 1e-3
    kw = dict(n_theta=7, n_phi=7, spec_dlog=0.01)
    with _ctx(xt) as ctx:
        ctx.load(w)
        st = ctx.transport(w, sampler=xt.XT_SAMPLER_RAYS, **kw)
        G, heat = ctx.get_photoionization_rates()
        S = ctx.get_estimators()
    o = oracle.transport(w, sampler="rays", **kw)
    _cmp(S, o["S"], TOL, "line estimators")
    _cmp_rates(G, oracle.pi_rates(w, o["S_pi"]), "photoionization rates")
    np.testing.assert_allclose(heat, o["heat"], rtol=TOL, atol=1e-12 * np.abs(o["heat"]).max())
    L = o["ledger"]
    assert st["events"] == L["events"] and L["pi_N"] > 0.05 * L["emit_N"]
    assert abs(st["photoionized_N"] - L["pi_N"]) <= 1e-9 * st["emitted_N"]
