"""Spatial decomposition (Sec. 2.4.1) on the GPU through the C ABI: the
domains of run_transport_domain, each on a context of its own, driven in one
process by the bundle-exchange driver (run_local: the domains step in
lockstep; bundles of packet states go from context to context on the
device).  The sums over the domains equal one run_transport of the whole
grid: estimators and photoionization rates 1e-10, spectrum 1e-9, events and
tests exact."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xt():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a GPU"
    import __graft_entry__ as g
    g.build()
    import paper_2511_07539_gb300 as xt
    return xt


def _cmp(got, want, tol, what):
    mg, mw = got != 0, want != 0
    assert np.array_equal(mg, mw), f"{what}: support differs ({mg.sum()} vs {mw.sum()})"
    if mw.any():
        err = np.max(np.abs(got[mw] / want[mw] - 1))
        assert err < tol, f"{what}: max rel err {err}"


@pytest.mark.parametrize("world,pi", [(2, False), (4, True)])
def test_domains_sum_to_the_whole_grid(xt, world, pi):
    import torch
    from paper_2511_07539_gb300 import spatial
    w = synth.clumpy_onion(seed=2, n=16, n_packets=400_000, n_lines=2000, level_range=(20, 50),
                           subdomains=(2, 2, 4))
    if pi:
        synth.with_photoionization(w)
    w.pops = w.pops * 1e-3
    stream = torch.cuda.current_stream().cuda_stream
    kw = dict(n_packets=w.n_packets, seed=w.seed, spec_lam0_A=w.spec_band_A[0],
              spec_nbins=w.spec_band_A[1])
    ref = xt.Context(0, stream)
    ref.load(w)
    st = ref.transport(w)
    S_ref, spec_ref = ref.get_estimators(), ref.get_spectrum(0)
    G_ref = ref.get_photoionization_rates()[0] if pi else None
    ref.close()
    ctxs, trs = [], []
    for r in range(world):
        c = xt.Context(0, stream)
        c.load(w)
        ctxs.append(c)
        trs.append(spatial.LibDomainTracer(c, *spatial.slab(r, w.nz, world), **kw))
    rounds = spatial.run_local(trs, w.nz)
    assert 1 <= rounds <= world - 1
    S = np.zeros_like(S_ref)
    spec = np.zeros_like(spec_ref)
    G = np.zeros_like(G_ref) if pi else None
    ev = tests = 0.0
    nxy = w.nx * w.ny
    for r, (c, t) in enumerate(zip(ctxs, trs)):
        z0, z1 = spatial.slab(r, w.nz, world)
        S[z0 * nxy:z1 * nxy] = c.get_estimators(z0 * nxy, (z1 - z0) * nxy)
        spec += c.get_spectrum(0)
        if pi:
            G[z0 * nxy:z1 * nxy] = c.get_photoionization_rates(z0 * nxy, (z1 - z0) * nxy)[0]
        # a domain's store holds nothing outside its cells
        if z0 > 0:
            assert not c.get_estimators(0, z0 * nxy).any()
        ev += t.stats[-1]["events"]              # a domain's ledger accumulates over its calls
        tests += t.stats[-1]["tests"]
        c.close()
    assert ev == st["events"] and tests == st["tests"]
    _cmp(S, S_ref, 1e-10, "estimators")
    _cmp(spec, spec_ref, 1e-9, "spectrum")
    if pi:
        _cmp(G, G_ref, 1e-10, "photoionization rates")


@pytest.mark.parametrize("world,pi", [(3, False), (4, True)])
def test_phi_slab_domains_on_the_spherical_grid(xt, world, pi):
    """The paper's decomposition of its spherical grid (Sec. 2.4.1): domains of
    whole phi slices (the azimuthal index is the grid's third), packets handed
    on with their path from the emission point; phi wraps around.  The sums
    over the domains equal one run_transport of the whole grid."""
    import torch
    from paper_2511_07539_gb300 import spatial
    w = synth.spherical_sphere(n_packets=200_000, seed=5, clumps=True)      # 12 phi slices
    if pi:
        synth.with_photoionization(w)
    w.pops = w.pops * 1e-3
    stream = torch.cuda.current_stream().cuda_stream
    kw = dict(n_packets=w.n_packets, seed=w.seed, spec_lam0_A=w.spec_band_A[0],
              spec_nbins=w.spec_band_A[1])
    ref = xt.Context(0, stream)
    ref.load(w)
    st = ref.transport(w)
    S_ref, spec_ref = ref.get_estimators(), ref.get_spectrum(0)
    G_ref = ref.get_photoionization_rates()[0] if pi else None
    ref.close()
    ctxs, trs = [], []
    for r in range(world):
        c = xt.Context(0, stream)
        c.load(w)
        ctxs.append(c)
        trs.append(spatial.LibDomainTracer(c, *spatial.slab(r, w.nz, world), **kw))
    rounds = spatial.run_local(trs, w.nz)
    assert 1 <= rounds <= world - 1
    S = np.zeros_like(S_ref)
    spec = np.zeros_like(spec_ref)
    G = np.zeros_like(G_ref) if pi else None
    ev = tests = 0.0
    nxy = w.nx * w.ny
    for r, (c, t) in enumerate(zip(ctxs, trs)):
        z0, z1 = spatial.slab(r, w.nz, world)
        S[z0 * nxy:z1 * nxy] = c.get_estimators(z0 * nxy, (z1 - z0) * nxy)
        spec += c.get_spectrum(0)
        if pi:
            G[z0 * nxy:z1 * nxy] = c.get_photoionization_rates(z0 * nxy, (z1 - z0) * nxy)[0]
        ev += t.stats[-1]["events"]
        tests += t.stats[-1]["tests"]
        c.close()
    assert ev == st["events"] and tests == st["tests"]
    _cmp(S, S_ref, 1e-10, "estimators")
    _cmp(spec, spec_ref, 1e-9, "spectrum")
    if pi:
        _cmp(G, G_ref, 1e-10, "photoionization rates")


@pytest.mark.parametrize("pi", [False, True])
def test_rays_across_phi_slab_domains(xt, pi):
    """The paper's own configuration (Secs. 2.3, 2.4.1): the RAYS sampler on
    the spherical grid with domains of whole phi slices; a domain emits the
    rays of its cells (a contiguous range of the cells' blocks of ray ids) and
    hands on those that enter another domain.  The sums over the domains equal
    one run_transport of the whole grid with the same rays."""
    import torch
    from paper_2511_07539_gb300 import spatial
    w = synth.spherical_sphere(n_packets=1, seed=72, nr=6, nth=4, nph=6, subdomains=(1, 1, 3))
    if pi:
        synth.with_photoionization(w, chi_eV=6.0, charge=0, pi_nlev=9)
    w.pops = w.pops * 1e-3
    stream = torch.cuda.current_stream().cuda_stream
    kw = dict(n_packets=1, seed=w.seed, spec_lam0_A=w.spec_band_A[0], spec_nbins=w.spec_band_A[1],
              sampler=xt.XT_SAMPLER_RAYS, n_theta=7, n_phi=7, spec_dlog=0.01)
    ref = xt.Context(0, stream)
    ref.load(w)
    st = xt.run_transport(ref.h, **kw)
    S_ref, spec_ref = ref.get_estimators(), ref.get_spectrum(0)
    G_ref = ref.get_photoionization_rates()[0] if pi else None
    ref.close()
    world = 3
    ctxs, trs = [], []
    for r in range(world):
        c = xt.Context(0, stream)
        c.load(w)
        ctxs.append(c)
        trs.append(spatial.LibDomainTracer(c, *spatial.slab(r, w.nz, world), **kw))
    rounds = spatial.run_local(trs, w.nz)
    assert 1 <= rounds <= world - 1
    S = np.zeros_like(S_ref)
    spec = np.zeros_like(spec_ref)
    G = np.zeros_like(G_ref) if pi else None
    ev = tests = emitted = 0.0
    nxy = w.nx * w.ny
    for r, (c, t) in enumerate(zip(ctxs, trs)):
        z0, z1 = spatial.slab(r, w.nz, world)
        S[z0 * nxy:z1 * nxy] = c.get_estimators(z0 * nxy, (z1 - z0) * nxy)
        spec += c.get_spectrum(0)
        if pi:
            G[z0 * nxy:z1 * nxy] = c.get_photoionization_rates(z0 * nxy, (z1 - z0) * nxy)[0]
        ev += t.stats[-1]["events"]
        tests += t.stats[-1]["tests"]
        emitted += t.stats[-1]["emitted_E"]
        c.close()
    assert st["rays"] > 0 and st["events"] > 1000
    assert ev == st["events"] and tests == st["tests"]
    assert abs(emitted / st["emitted_E"] - 1) < 1e-12
    _cmp(S, S_ref, 1e-10, "estimators")
    _cmp(spec, spec_ref, 1e-9, "spectrum")
    if pi:
        assert (G_ref > 0).any()
        _cmp(G, G_ref, 1e-10, "photoionization rates")


def test_rays_domains_refused_on_the_cube(xt):
    """Domains take rays on the spherical grid only (the cube's domain path
    emits through the packet pool, which has no ray form)."""
    import torch
    w = synth.clumpy_onion(seed=2, n=8, n_packets=1000, n_lines=200, level_range=(20, 30),
                           subdomains=(2, 2, 2))
    with xt.Context(0, torch.cuda.current_stream().cuda_stream) as ctx:
        ctx.load(w)
        with pytest.raises(xt.XtError) as e:
            xt.run_transport_domain(ctx.h, 0, 4, True, n_packets=1, seed=1, spec_lam0_A=w.spec_band_A[0],
                                    spec_nbins=w.spec_band_A[1], sampler=xt.XT_SAMPLER_RAYS)
        assert e.value.code == xt.XT_EINVAL


def test_malformed_bundle_is_refused(xt):
    """A received state whose cell lies outside the grid, or whose line cursor
    lies outside the line list, is refused (XT_EINVAL) before it is traced."""
    import torch
    w = synth.spherical_sphere(n_packets=2_000, seed=5)
    with xt.Context(0, torch.cuda.current_stream().cuda_stream) as ctx:
        ctx.load(w)
        for cell, cursor in [(float(1 << 30), 0.0), (float(w.nx | (w.ny << 10)), 0.0),
                             (0.0, float(w.nline + 1)), (-1.0, 0.0)]:
            b = np.zeros((1, xt.XT_BUNDLE_FIELDS))
            b[0, xt.XT_BUNDLE_CELL] = cell
            b[0, xt.XT_BUNDLE_CELL + 1] = cursor
            with pytest.raises(xt.XtError) as e:
                xt.run_transport_domain(ctx.h, 0, w.nz, False, bundle_in=b, n_packets=w.n_packets,
                                        seed=w.seed, spec_lam0_A=w.spec_band_A[0],
                                        spec_nbins=w.spec_band_A[1])
            assert e.value.code == xt.XT_EINVAL
