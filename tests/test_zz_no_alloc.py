"""run_transport_noalloc: the transport pass for callers that cannot call
cudaMalloc (inside a stream capture, under another framework's fixed device
memory budget).  Through the C ABI, two calls in a row, each checked against
run_transport on the same inputs, within the estimator and spectrum
tolerances of the other GPU tests.  This file is collected last."""
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


def test_noalloc_transport_matches_run_transport():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a GPU"
    import __graft_entry__ as g
    g.build()
    import paper_2511_07539_gb300 as xt

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
            st = xt.run_transport_noalloc(
                w.nx, w.ny, w.nz, w.v_max, w.t, w.L_cell, w.band_A, w.g_level, w.lo, w.up,
                w.lambda_A, w.f_lu, pops, S, spec, w.n_packets, seed=seed,
                spec_lam0_A=w.spec_band_A[0], spec_nbins=nb, stream=stream)
            ref = ctx.transport(w, seed=seed)
            assert st["events"] == ref["events"] > 0
            assert st["emitted_N"] == pytest.approx(ref["emitted_N"], rel=1e-13)
            _cmp(S.cpu().numpy(), ctx.get_estimators(), S_TOL, f"estimators, seed {seed}")
            _cmp(spec.cpu().numpy(), ctx.get_spectrum(0), SPEC_TOL, f"spectrum, seed {seed}")
        # sizes beyond the fixed scratch are refused with a message
        with pytest.raises(xt.XtError) as e:
            big = np.ones(70 * 70 * 70)
            xt.run_transport_noalloc(70, 70, 70, w.v_max, w.t, big, w.band_A, w.g_level, w.lo,
                                     w.up, w.lambda_A, w.f_lu, pops, S, spec, 10, stream=stream)
        assert e.value.code == xt.XT_EINVAL and "exceed" in str(e.value)
    finally:
        ctx.close()
