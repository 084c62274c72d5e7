"""run_transport_noalloc: the transport pass for callers that cannot call
cudaMalloc (programs whose device memory is handed out once by another
framework's allocator, or that must stay within a fixed device-memory budget).
Through the C ABI, two calls in a row, each checked against run_transport on
the same inputs, within the estimator and spectrum tolerances of the other GPU
tests; then a pass of more than two packet chunks, which reuses the fixed
packet pool chunk after chunk.  This file is collected last."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

S_TOL = 1e-10
SPEC_TOL = 1e-9


def _cmp(got, want, tol, what):
    mg, mw = got != 0, want != 0
    assert np.array_equal(mg, mw), f"{what}: support differs"
    if mw.any():
        err = np.max(np.abs(got[mw] / want[mw] - 1))
        assert err < tol, f"{what}: max rel err {err}"


def _setup():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a GPU"
    import __graft_entry__ as g
    g.build()
    import paper_2511_07539_gb300 as xt
    return torch, xt


def _noalloc(xt, w, pops, S, spec, n_packets, seed, stream):
    return xt.run_transport_noalloc(
        w.nx, w.ny, w.nz, w.v_max, w.t, w.L_cell, w.band_A, w.g_level, w.lo, w.up,
        w.lambda_A, w.f_lu, pops, S, spec, n_packets, seed=seed,
        spec_lam0_A=w.spec_band_A[0], spec_nbins=w.spec_band_A[1], stream=stream)


def test_noalloc_transport_matches_run_transport():
    torch, xt = _setup()
    w = synth.uniform_sphere(n=12, n_packets=60_000, n_lines=80, seed=21)
    w.pops = w.pops * 1e-4
    stream = torch.cuda.current_stream().cuda_stream
    pops = torch.as_tensor(w.pops, device="cuda").contiguous()
    views, nb = 400, w.spec_band_A[1]
    S = torch.zeros((w.ncell, w.nline), dtype=torch.float64, device="cuda")
    spec = torch.zeros((views, nb), dtype=torch.float64, device="cuda")
    ctx = xt.Context(0, stream)
    try:
        ctx.load(w, subdomains=(1, 1, 1))
        for seed in (21, 22):
            st = _noalloc(xt, w, pops, S, spec, w.n_packets, seed, stream)
            ref = ctx.transport(w, seed=seed)
            assert st["events"] == ref["events"] > 0
            assert st["emitted_N"] == pytest.approx(ref["emitted_N"], rel=1e-13)
            _cmp(S.cpu().numpy(), ctx.get_estimators(), S_TOL, f"estimators, seed {seed}")
            _cmp(spec.cpu().numpy(), ctx.get_spectrum(0), SPEC_TOL, f"spectrum, seed {seed}")
        # sizes beyond the fixed scratch are refused with a message
        with pytest.raises(xt.XtError) as e:
            big = np.ones(70 * 70 * 70)
            S_big = torch.zeros(70 * 70 * 70 * w.nline, dtype=torch.float64, device="cuda")
            p_big = torch.zeros(70 * 70 * 70 * w.nlev, dtype=torch.float64, device="cuda")
            xt.run_transport_noalloc(70, 70, 70, w.v_max, w.t, big, w.band_A, w.g_level, w.lo,
                                     w.up, w.lambda_A, w.f_lu, p_big, S_big, spec, 10,
                                     spec_nbins=nb, stream=stream)
        assert e.value.code == xt.XT_EINVAL and "exceed" in str(e.value)
        # an output tensor smaller than the call would write is refused before the call
        with pytest.raises(ValueError):
            xt.run_transport_noalloc(w.nx, w.ny, w.nz, w.v_max, w.t, w.L_cell, w.band_A,
                                     w.g_level, w.lo, w.up, w.lambda_A, w.f_lu, pops, S,
                                     spec[:1], 10, spec_nbins=nb, stream=stream)
    finally:
        ctx.close()


def test_noalloc_transport_over_several_chunks():
    """300,000 packets: three chunks of at most XT_NOALLOC_CHUNK (131,072)
    packets through the one fixed pool, counters reset and escapes tallied per
    chunk; the result equals run_transport's single pass."""
    torch, xt = _setup()
    w = synth.uniform_sphere(n=12, n_packets=300_000, n_lines=80, seed=23)
    w.pops = w.pops * 1e-4
    stream = torch.cuda.current_stream().cuda_stream
    pops = torch.as_tensor(w.pops, device="cuda").contiguous()
    S = torch.zeros((w.ncell, w.nline), dtype=torch.float64, device="cuda")
    spec = torch.zeros((400, w.spec_band_A[1]), dtype=torch.float64, device="cuda")
    ctx = xt.Context(0, stream)
    try:
        ctx.load(w, subdomains=(1, 1, 1))
        st = _noalloc(xt, w, pops, S, spec, w.n_packets, 23, stream)
        assert w.n_packets > 2 * 131_072
        ref = ctx.transport(w, seed=23)
        assert st["events"] == ref["events"] > 0 and st["tests"] == ref["tests"]
        assert st["escaped_N"] == pytest.approx(ref["escaped_N"], rel=1e-12)
        _cmp(S.cpu().numpy(), ctx.get_estimators(), S_TOL, "estimators, three chunks")
        _cmp(spec.cpu().numpy(), ctx.get_spectrum(0), SPEC_TOL, "spectrum, three chunks")
    finally:
        ctx.close()
