"""GPU transport vs the CPU oracle, through the C ABI (needs a GB300).

Bars: estimators relative 1e-10 and spectra 1e-9 (FP64 transport; the only
freedom is the summation order of atomics and last-bit differences of the
math library), per-packet histories identical (fate and event counts exact,
photon counts relative 1e-12), Sobolev tau/beta relative 1e-13.
"""
import numpy as np
import pytest

import oracle
import synth

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
    # N_final of a dropped packet is a cancellation remainder (~2^-53 N0) where
    # CUDA's and glibc's expm1 may differ by one ulp: bound it against N0
    assert np.all(np.abs(rec[:, 2] - pk[:, 2]) <= 1e-12 * np.abs(pk[:, 2]) + 1e-15 * pk[:, 8])
    np.testing.assert_allclose(rec[:, 8], pk[:, 8], rtol=1e-13)
    np.testing.assert_allclose(rec[:, 9], pk[:, 9], rtol=1e-15)
    np.testing.assert_allclose(rec[:, 10], pk[:, 10], rtol=1e-14)
    esc = pk[:, 0] == 0
    assert np.array_equal(rec[esc, 4], pk[esc, 4]), "viewer bins differ"
    assert np.array_equal(rec[esc, 5], pk[esc, 5]), "wavelength bins differ"


def test_uniform_sphere_full(xt):
    """16^3 grid, 100 lines, 1e5 packets: estimators, spectrum, ledger, histories."""
    w = synth.uniform_sphere()
    with _ctx(xt) as ctx:
        ctx.load(w)
        st, rec = _records(xt, ctx, w)
        S = ctx.get_estimators()
        spec = ctx.get_spectrum(0)
        o = oracle.transport(w, per_packet=True)
        _cmp_records(rec, o["pkt"])
        _cmp_sparse(S, o["S"], S_TOL, "estimators")
        _cmp_sparse(spec, o["spec"], SPEC_TOL, "spectrum")
        L = o["ledger"]
        assert st["events"] == L["events"] and st["tests"] == L["tests"]
        for k, kk in [("emitted_N", "emit_N"), ("escaped_N", "esc_N"), ("absorbed_N", "abs_N"),
                      ("dropped_N", "drop_N"), ("escaped_E", "esc_E")]:
            assert st[k] == pytest.approx(L[kk], rel=1e-12)
        assert st["escaped_N"] + st["absorbed_N"] + st["dropped_N"] == pytest.approx(st["emitted_N"], rel=1e-13)


def test_sobolev_tau_beta_and_rates(xt):
    w = synth.uniform_sphere(n=8, n_packets=30_000, seed=2)
    w.pops = w.pops * np.linspace(1e-9, 1.0, w.ncell)[:, None]
    with _ctx(xt) as ctx:
        ctx.load(w)
        tau, beta = ctx.get_sobolev_tau()
        t_or, b_or = oracle.tau_beta(w)
        np.testing.assert_allclose(tau, t_or, rtol=1e-13, atol=0)
        np.testing.assert_allclose(beta, b_or, rtol=1e-13, atol=0)
        ctx.transport(w)
        R_lu, R_ul, J = ctx.get_photoexcitation_rates()
        o = oracle.transport(w)
        r_or = oracle.rates(w, o["S"])
        _cmp_sparse(R_lu, r_or[0], S_TOL, "R_lu")
        _cmp_sparse(R_ul, r_or[1], S_TOL, "R_ul")
        _cmp_sparse(J, r_or[2], S_TOL, "Jbar")
        # a cell sub-range through the same call
        R2, _, _ = ctx.get_photoexcitation_rates(100, 37, want=("R_lu",))
        assert np.array_equal(R2, R_lu[100:137])


@pytest.mark.parametrize("sd,rounds", [((1, 1, 1), False), ((2, 2, 2), False), ((4, 2, 8), True),
                                       ((16, 16, 16), True), ((2, 2, 2), True)])
def test_decomposition_invariance(xt, sd, rounds):
    """P9: the subdomain split of the store, and tracing each subdomain as a
    domain of its own with packets handed on between rounds, change no history."""
    w = synth.uniform_sphere(n_packets=40_000, seed=5)
    w.pops = w.pops * 1e-5
    with _ctx(xt) as ctx:
        ctx.load(w, subdomains=sd)
        st, rec = _records(xt, ctx, w, subdomain_rounds=rounds)
        if rounds and sd != (1, 1, 1):
            assert st["rounds"] > 1 and st["queued"] > 0
        S = ctx.get_estimators()
        o = oracle.transport(w, per_packet=True)
        _cmp_records(rec, o["pkt"])
        _cmp_sparse(S, o["S"], S_TOL, f"estimators sd={sd}")


def test_packet_subrange_and_accumulate(xt):
    w = synth.uniform_sphere(n_packets=50_000, seed=6)
    w.pops = w.pops * 1e-4
    with _ctx(xt) as ctx:
        ctx.load(w)
        ctx.transport(w, packet_begin=0, packet_count=17_001)
        ctx.transport(w, packet_begin=17_001, packet_count=50_000 - 17_001, accumulate=True)
        S = ctx.get_estimators()
        o = oracle.transport(w)
        _cmp_sparse(S, o["S"], S_TOL, "split run")
        _, rec = _records(xt, ctx, w, packet_begin=12_345, packet_count=999)
        o2 = oracle.transport(w, p_begin=12_345, p_end=12_345 + 999, per_packet=True)
        _cmp_records(rec, o2["pkt"])


def test_edge_cases(xt):
    # zero packets, one packet, odd grid with ragged subdomain blocks, empty matter
    w = synth.uniform_sphere(n=6, n_packets=1, seed=7, n_lines=30)
    with _ctx(xt) as ctx:
        ctx.load(w, subdomains=(3, 2, 1))
        st = ctx.transport(w, n_packets=0)
        assert st["emitted_N"] == 0 and ctx.get_estimators().sum() == 0
        _, rec = _records(xt, ctx, w)
        o = oracle.transport(w, per_packet=True)
        _cmp_records(rec, o["pkt"])
        w0 = synth.uniform_sphere(n=5, n_packets=5000, seed=8, n_lines=30)
        w0.pops = np.zeros_like(w0.pops)
        ctx.load(w0)
        st = ctx.transport(w0)
        assert st["events"] == 0 and st["escaped_N"] == pytest.approx(st["emitted_N"], rel=1e-13)
        o = oracle.transport(w0)
        _cmp_sparse(ctx.get_spectrum(0), o["spec"], SPEC_TOL, "empty-matter spectrum")
        # invalid arguments are reported, not trapped
        with pytest.raises(xt.XtError) as e:
            ctx.transport(w0, packet_begin=10, packet_count=w0.n_packets)
        assert e.value.code == xt.XT_EINVAL
        with pytest.raises(xt.XtError) as e:
            xt.init_grid(ctx.h, 5, 5, 5, w0.v_max, w0.t, w0.Te, w0.ne, w0.L_cell, w0.band_A,
                         subdomains=(2, 1, 1))
        assert e.value.code == xt.XT_EINVAL


@pytest.mark.parametrize("views", [(20, 20), (9, 14)])
def test_spectrum_normalisations_vs_oracle(xt, views):
    """get_spectrum kinds 1 and 2 (isotropic-equivalent L_lambda per viewer,
    4 pi / dOmega_k E / dlambda, and the angle-summed L_lambda) against the
    oracle's normalisation of its own binned energy, element by element."""
    nt, nph = views
    w = synth.uniform_sphere(n_packets=60_000, seed=31)
    w.pops = w.pops * 1e-3
    with _ctx(xt) as ctx:
        ctx.load(w)
        ctx.transport(w, n_theta=nt, n_phi=nph)
        L_k, L_tot = ctx.get_spectrum(1), ctx.get_spectrum(2)
        o = oracle.transport(w, n_theta=nt, n_phi=nph)
        Lk_o, Lt_o, _ = oracle.spectrum_L_lambda(o["spec"], w.spec_band_A[0], 1e-3, nt, nph)
        assert L_k.shape == Lk_o.shape and L_tot.shape == Lt_o.shape
        _cmp_sparse(L_k, Lk_o, SPEC_TOL, "L_lambda per viewer")
        _cmp_sparse(L_tot, Lt_o, SPEC_TOL, "angle-summed L_lambda")


@pytest.mark.parametrize("flags", [0, 1])
def test_warp_prereduction_of_estimators(xt, flags):
    """Few lines and thin: the lanes of a warp often add to the same (cell,
    line) slot at once.  With the warp pre-reduction (XT_FLAG_WARP_REDUCE) and
    without it (flags 0), the estimators equal the oracle's."""
    w = synth.uniform_sphere(n=6, n_packets=200_000, n_lines=12, n_levels=8, seed=35)
    w.lambda_A = np.linspace(5000.0, 5080.0, 12)     # every packet meets most lines
    w.band_A = (4990.0, 5100.0)
    w.spec_band_A = synth._spectrum_grid(w.band_A[0], w.band_A[1], w.v_max)
    w.pops = w.pops * 1e-3
    with _ctx(xt) as ctx:
        ctx.load(w)
        st = ctx.transport(w, flags=flags)
        o = oracle.transport(w)
        assert st["events"] == o["ledger"]["events"] > 200_000      # over ~1500 slots
        _cmp_sparse(ctx.get_estimators(), o["S"], S_TOL, f"estimators, flags {flags}")


def test_event_guard_reports_timeout(xt):
    w = synth.uniform_sphere(n=8, n_packets=2000, seed=9)
    w.pops = w.pops * 1e-5
    with _ctx(xt) as ctx:
        ctx.load(w)
        rc, st = ctx.transport(w, max_events=1, check=False)
        o = oracle.transport(w, max_events=1)
        assert rc == xt.XT_ETIMEOUT and st["guard"] == o["ledger"]["guard"] > 0


def test_line_emission(xt):
    w = synth.uniform_sphere(n=8, n_packets=30_000, seed=10)
    w.pops = w.pops * 1e-3
    with _ctx(xt) as ctx:
        ctx.load(w)
        _, rec = _records(xt, ctx, w, emission=xt.XT_EMIT_LINES)
        S = ctx.get_estimators()
        o = oracle.transport(w, emission="lines", per_packet=True)
        _cmp_records(rec, o["pkt"])
        _cmp_sparse(S, o["S"], S_TOL, "line-emission estimators")


@pytest.mark.parametrize("rounds", [False, True])
def test_scatter_mode(xt, rounds):
    w = synth.uniform_sphere(n_packets=40_000, seed=12, subdomains=(4, 4, 4))
    ups = oracle.upsilon_down_sums(w)
    with _ctx(xt) as ctx:
        ctx.load(w, with_scatter_data=ups)
        st, rec = _records(xt, ctx, w, mode=xt.XT_MODE_SCATTER, subdomain_rounds=rounds)
        S = ctx.get_estimators()
        spec = ctx.get_spectrum(0)
        o = oracle.transport(w, mode="scatter", per_packet=True)
        _cmp_records(rec, o["pkt"])
        assert np.array_equal(rec[:, 6], o["pkt"][:, 6]), "interaction counts differ"
        _cmp_sparse(S, o["S"], S_TOL, "scatter estimators")
        _cmp_sparse(spec, o["spec"], SPEC_TOL, "scatter spectrum")
        assert st["reemit_E_cmf"] + st["thermal_E"] == pytest.approx(st["abs_E_cmf"], rel=1e-13)


@pytest.fixture(scope="module")
def onion():
    return synth.clumpy_onion()


@pytest.mark.parametrize("rounds", [True, False])
def test_clumpy_onion_full_grid_packet_subset(xt, onion, rounds):
    """Paper-scale grid and line list (64^3 x 1e5 lines, 8^3 subdomains), a
    contiguous packet subset: every estimator slot the oracle touches, and
    nothing else in those cells.  rounds=False is the benchmark's path (the
    trace kernel emits its own packets, the whole grid one domain)."""
    w = onion
    with _ctx(xt) as ctx:
        ctx.load(w)
        p0, m = (61_234_567, 60_000) if rounds else (17_000_001, 60_000)
        st, rec = _records(xt, ctx, w, packet_begin=p0, packet_count=m, subdomain_rounds=rounds)
        assert (st["rounds"] > 1) == rounds
        o = oracle.transport(w, p_begin=p0, p_end=p0 + m, per_packet=True)
        _cmp_records(rec, o["pkt"])
        slots, vals = o["S_slots"], o["S_values"]
        cells = np.unique(slots // w.nline)
        # read back windows of at most 64 consecutive cells around the touched ones
        k = 0
        while k < len(cells):
            lo_c = int(cells[k])
            hi_c = lo_c + 64
            k = int(np.searchsorted(cells, hi_c))
            S = ctx.get_estimators(lo_c, hi_c - lo_c if hi_c <= w.ncell else w.ncell - lo_c)
            want = np.zeros_like(S)
            sel = (slots // w.nline >= lo_c) & (slots // w.nline < lo_c + S.shape[0])
            want.reshape(-1)[slots[sel] - lo_c * w.nline] = vals[sel]
            _cmp_sparse(S, want, S_TOL, "onion estimators")


def test_clumpy_onion_full_run_sampled(xt, onion):
    """The full 1e8-packet pass in the benchmark's launch configuration:
    sampled packet histories vs the oracle one by one, and the ledger closes."""
    w = onion
    with _ctx(xt) as ctx:
        ctx.load(w)
        import torch
        rec = torch.zeros((w.n_packets, xt.XT_PKT_FIELDS), dtype=torch.float64, device="cuda")
        st = ctx.transport(w, packet_records=rec)
        assert st["escaped_N"] + st["absorbed_N"] + st["dropped_N"] == pytest.approx(st["emitted_N"], rel=1e-12)
        rng = np.random.default_rng(0)
        ids = np.sort(rng.choice(w.n_packets, 300, replace=False))
        got = rec[torch.as_tensor(ids, device="cuda")].cpu().numpy()
        for i, p in enumerate(ids):
            o = oracle.transport(w, p_begin=int(p), p_end=int(p) + 1, per_packet=True, sparse=True)
            _cmp_records(got[i:i + 1], o["pkt"])


def test_consecutive_passes_clear_the_store(xt):
    """Back-to-back passes on one context: each pass clears what the previous
    one wrote (the touched-slot log, or the whole store after a log overflow,
    which the first pass here provokes with > 4.2e6 events)."""
    w = synth.uniform_sphere(n_packets=800_000, seed=14, n_lines=180)
    w.v_max = 3e9                   # 10 % of c: many resonances per packet
    w.pops = w.pops * 3e-7          # thin lines: packets survive many events
    with _ctx(xt) as ctx:
        ctx.load(w)
        for k, seed in enumerate((14, 15, 16, 17)):
            st = ctx.transport(w, seed=seed)
            S = ctx.get_estimators()
            o = oracle.transport(w, seed=seed)
            assert st["events"] == o["ledger"]["events"]
            if k == 0:
                assert st["events"] > 4.4e6
            _cmp_sparse(S, o["S"], S_TOL, f"pass with seed {seed}")


def test_host_streamed_store_matches_device_store(xt):
    """The estimator store held in host memory in 2 and 4 groups of subdomain
    z-layers (one group on the device at a time, packets traced group by group
    in rounds) gives the estimators, rates, spectrum and ledger of the
    device-resident store, on two passes in a row and after switching back."""
    w = synth.clumpy_onion(seed=2, n=16, n_packets=200_000, n_lines=2000, level_range=(20, 50),
                           subdomains=(2, 2, 4))
    with _ctx(xt) as ctx:
        ctx.load(w)
        st0 = ctx.transport(w)
        S0 = ctx.get_estimators()
        R0 = ctx.get_photoexcitation_rates(want=("R_lu",))[0]
        spec0 = ctx.get_spectrum(0)
        assert st0["events"] > 10_000
        for groups in (2, 4, 0):
            xt.set_estimator_store(ctx.h, groups)
            for _ in range(2):
                st = ctx.transport(w)
                assert st["events"] == st0["events"] and st["tests"] == st0["tests"]
                assert st["escaped_N"] == pytest.approx(st0["escaped_N"], rel=1e-12)
                if groups:
                    assert st["rounds"] >= groups
                _cmp_sparse(ctx.get_estimators(), S0, S_TOL, f"estimators, {groups} groups")
                _cmp_sparse(ctx.get_photoexcitation_rates(want=("R_lu",))[0], R0, S_TOL, "rates")
                _cmp_sparse(ctx.get_spectrum(0), spec0, SPEC_TOL, "spectrum")
            # a cell range that spans two groups
            part = ctx.get_estimators(1000, 3000)
            _cmp_sparse(part, S0[1000:4000], S_TOL, "estimator range")


def test_compact_rows_store_matches_dense(xt):
    """XT_STORE_COMPACT_ROWS holds estimator rows only for cells with
    populations (here the 2176 cells of the sphere, of 4096): estimators,
    rates and an estimator-rate solve equal the dense store's, on passes in
    a row and after the cells with populations change."""
    w = synth.uniform_sphere(n_packets=60_000, seed=41)
    w.pops = w.pops * 1e-3
    ups = synth.collision_strengths(w.upsilon_seed, w.level_off)
    res = {}
    for mode in (0, xt.XT_STORE_COMPACT_ROWS):
        with _ctx(xt) as ctx:
            ctx.load(w)
            xt.set_estimator_store(ctx.h, mode)
            out = []
            for seed in (41, 42):
                st = ctx.transport(w, seed=seed)
                out.append((st["events"], ctx.get_estimators(), ctx.get_photoexcitation_rates()[2]))
            sz = xt.get_sizes(ctx.h)["store_bytes"]
            p = np.zeros((w.ncell, w.nlev))
            xt.solve_nlte(ctx.h, ups, precision=0, rates=xt.XT_RATES_ESTIMATORS, warm=xt.XT_WARM_CURRENT,
                          pops_out=p)
            # fewer cells with populations: a new row map
            pops2 = w.pops.copy()
            pops2[: w.ncell // 2] = 0.0
            ctx.set_populations(pops2)
            st2 = ctx.transport(w, seed=43)
            res[mode] = (out, sz, p, st2["events"], ctx.get_estimators())
    (o0, sz0, p0, e0, S0), (o1, sz1, p1, e1, S1) = res[0], res[xt.XT_STORE_COMPACT_ROWS]
    assert sz1 == 2176 * w.nline * 8 and sz0 == w.ncell * w.nline * 8
    for a, b in zip(o0, o1):
        assert a[0] == b[0]
        _cmp_sparse(b[1], a[1], S_TOL, "compact estimators")
        _cmp_sparse(b[2], a[2], S_TOL, "compact Jbar")
    np.testing.assert_allclose(p1, p0, rtol=1e-10)
    assert e0 == e1
    _cmp_sparse(S1, S0, S_TOL, "compact estimators after a new row map")
