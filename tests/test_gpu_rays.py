"""The RAYS sampler on the GPU (Sec. 2.3: one ray per emitting cell, output
bin and viewer, from the middle of the cell) against the CPU oracle through
the C ABI (needs a GB300).  Bars as for Monte Carlo packets: histories
identical, estimators and rates 1e-10, spectra 1e-9.

Viewer grids here have no direction exactly diagonal between two axes (n_phi
not 4 times an odd number): such a ray from a cell centre reaches two walls at
the same distance, and which one it crosses first is decided by rounding."""
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


def _check(xt, ctx, w, emission="band", nt=9, nph=10, dlog=0.02, pi=False, **kw):
    em = xt.XT_EMIT_BAND if emission == "band" else xt.XT_EMIT_LINES
    n = oracle.ray_count(w, emission, nt, nph, dlog)
    rec = np.zeros((n, xt.XT_PKT_FIELDS))
    st = ctx.transport(w, sampler=xt.XT_SAMPLER_RAYS, emission=em, n_theta=nt, n_phi=nph,
                       spec_dlog=dlog, packet_records=rec, **kw)
    assert st["rays"] == n
    o = oracle.transport(w, sampler="rays", emission=emission, n_theta=nt, n_phi=nph,
                         spec_dlog=dlog, per_packet=True)
    pk = o["pkt"]
    assert np.array_equal(rec[:, 0], pk[:, 0]), "fates differ"
    assert np.array_equal(rec[:, 1], pk[:, 1]), "event counts differ"
    assert np.array_equal(rec[:, 7], pk[:, 7]), "cells differ"
    np.testing.assert_allclose(rec[:, 8], pk[:, 8], rtol=1e-13)
    assert np.all(np.abs(rec[:, 2] - pk[:, 2]) <= 1e-12 * np.abs(pk[:, 2]) + 1e-15 * pk[:, 8])
    esc = pk[:, 0] == 0
    assert np.array_equal(rec[esc, 4], pk[esc, 4]) and np.array_equal(rec[esc, 5], pk[esc, 5])
    _cmp(ctx.get_estimators(), o["S"], TOL, "estimators")
    _cmp(ctx.get_spectrum(0), o["spec"], 1e-9, "spectrum")
    if pi:
        G, heat = ctx.get_photoionization_rates()
        _cmp(G, oracle.pi_rates(w, o["S_pi"]), TOL, "photoionization rates")
    L = o["ledger"]
    assert st["events"] == L["events"] and st["tests"] == L["tests"]
    assert st["emitted_E"] == pytest.approx(L["emit_E"], rel=1e-9)     # sums over ~1e6 rays
    return st, o


@pytest.mark.parametrize("views,flags", [((9, 10), 0), ((6, 18), 0), ((9, 10), 2)])
def test_rays_band_emission(xt, views, flags):
    """flags 0: line records through L2; 2 (XT_FLAG_RAYS_STAGED): the line
    window of every batch of rays staged in shared memory."""
    w = synth.uniform_sphere(n=8, n_packets=1, seed=81)
    w.pops = w.pops * 1e-3
    with _ctx(xt) as ctx:
        ctx.load(w)
        st, o = _check(xt, ctx, w, nt=views[0], nph=views[1], flags=flags)
        assert o["ledger"]["events"] > 10_000


def test_rays_staged_window_at_paper_line_density(xt):
    """1e4 lines over 1000 A - 3 um on a 16^3 onion: each bin's window holds
    hundreds of line records; staged and unstaged passes give the oracle's
    estimators and spectrum."""
    w = synth.clumpy_onion(seed=5, n=16, n_packets=1, n_lines=10_000, level_range=(20, 40),
                           subdomains=(2, 2, 2))
    w.pops = w.pops * 1e-6
    with _ctx(xt) as ctx:
        ctx.load(w)
        for flags in (0, 2):
            _check(xt, ctx, w, nt=3, nph=6, dlog=0.05, flags=flags)


def test_rays_line_emission_with_photoionization(xt):
    w = synth.uniform_sphere(n=8, n_packets=1, seed=82)
    w.pops = w.pops * 1e-2
    synth.with_photoionization(w, chi_eV=6.0, charge=0, pi_nlev=9)
    with _ctx(xt) as ctx:
        ctx.load(w)
        st, o = _check(xt, ctx, w, emission="lines", dlog=0.005, pi=True)
        assert o["ledger"]["pi_N"] > 0 and o["ledger"]["events"] > 1000


def test_rays_subrange_accumulates_and_refusals(xt):
    w = synth.uniform_sphere(n=6, n_packets=1, seed=83)
    w.pops = w.pops * 1e-3
    kw = dict(n_theta=9, n_phi=10, spec_dlog=0.02)
    with _ctx(xt) as ctx:
        ctx.load(w)
        n = int(ctx.transport(w, sampler=xt.XT_SAMPLER_RAYS, packet_count=0, **kw)["rays"])
        assert n == oracle.ray_count(w, "band", 9, 10, 0.02)
        ctx.transport(w, sampler=xt.XT_SAMPLER_RAYS, packet_begin=0, packet_count=n // 3, **kw)
        ctx.transport(w, sampler=xt.XT_SAMPLER_RAYS, packet_begin=n // 3, accumulate=True, **kw)
        o = oracle.transport(w, sampler="rays", n_theta=9, n_phi=10, spec_dlog=0.02)
        _cmp(ctx.get_estimators(), o["S"], TOL, "split ray range")
        for bad in (dict(subdomain_rounds=True), dict(mode=xt.XT_MODE_SCATTER)):
            with pytest.raises(xt.XtError) as e:
                ctx.transport(w, sampler=xt.XT_SAMPLER_RAYS, **kw, **bad)
            assert e.value.code == xt.XT_EINVAL
        # a line off the output grid cannot be binned for line emission
        with pytest.raises(xt.XtError) as e:
            ctx.transport(w, sampler=xt.XT_SAMPLER_RAYS, emission=xt.XT_EMIT_LINES, n_theta=9,
                          n_phi=10, spec_dlog=0.02, spec_lam0_A=6000.0, spec_nbins=3)
        assert e.value.code == xt.XT_EINVAL and "outside" in str(e.value)
