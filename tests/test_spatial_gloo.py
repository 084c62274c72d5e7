"""Spatial decomposition across processes (Sec. 2.4.1): the bundle-exchange
driver of paper_2511_07539_gb300.spatial run as two gloo ranks on the CPU,
with the oracle tracing each rank's domain (packets resumed from the states
other ranks hand over): Monte Carlo packets on the cube, and rays on the
spherical grid in phi slices (the paper's configuration).  The sums over the
domains equal the single-domain oracle pass: estimators, photoionization,
spectrum and ledger; every packet keeps its trajectory whatever the
decomposition."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    import synth
    w = synth.uniform_sphere(n=8, n_packets=20_000, seed=3)
    synth.with_photoionization(w, chi_eV=6.0, charge=0, pi_nlev=9)
    w.pops = w.pops * 1e-3
    return w


def _ray_workload():
    import synth
    w = synth.spherical_sphere(n_packets=1, seed=72, nr=6, nth=4, nph=6, subdomains=(1, 1, 3))
    synth.with_photoionization(w, chi_eV=6.0, charge=0, pi_nlev=9)
    w.pops = w.pops * 1e-3
    return w


RAY_KW = dict(sampler="rays", n_theta=7, n_phi=7, spec_dlog=0.01)


class OracleTracer:
    """A domain traced by the CPU oracle; sums what the domain's calls tally."""

    def __init__(self, w, z_lo, z_hi, **kw):
        self.w, self.z_lo, self.z_hi, self.kw = w, z_lo, z_hi, kw
        self.S = self.spec = self.S_pi = self.heat = None
        self.ledger = {}
        self.calls = 0

    def step(self, emit, bundle_in):
        import oracle
        b = None if bundle_in is None else bundle_in.numpy()
        o = oracle.transport_domain(self.w, self.z_lo, self.z_hi, emit, b, **self.kw)
        for k in ("S", "spec", "S_pi", "heat"):
            cur = getattr(self, k)
            setattr(self, k, o[k] if cur is None else cur + o[k])
        for k, v in o["ledger"].items():
            self.ledger[k] = self.ledger.get(k, 0.0) + v
        self.calls += 1
        return torch.from_numpy(o["bundle"])

    def z_of(self, bundle):
        import oracle
        return bundle[:, oracle.STATE_Z].to(torch.int64)


def _compare(S, spec, S_pi, heat, ledger, w, **kw):
    import oracle
    ref = oracle.transport(w, **kw)
    m = ref["S"] != 0
    assert np.array_equal(S != 0, m)
    assert np.max(np.abs(S[m] / ref["S"][m] - 1)) < 1e-12
    ms = ref["spec"] != 0
    assert np.array_equal(spec != 0, ms)
    assert np.max(np.abs(spec[ms] / ref["spec"][ms] - 1)) < 1e-12
    mp_ = ref["S_pi"] != 0
    assert np.array_equal(S_pi != 0, mp_)
    assert mp_.any()
    assert np.max(np.abs(S_pi[mp_] / ref["S_pi"][mp_] - 1)) < 1e-12
    np.testing.assert_allclose(heat, ref["heat"], rtol=1e-12, atol=1e-12 * np.abs(ref["heat"]).max())
    L = ref["ledger"]
    assert ledger["events"] == L["events"] and ledger["tests"] == L["tests"]
    for k in ("emit_N", "esc_N", "abs_N", "drop_N", "pi_N", "esc_E"):
        assert ledger[k] == pytest.approx(L[k], rel=1e-12)


def _rank(rank, world, port, q, rays=False):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2511_07539_gb300 import spatial
    w = _ray_workload() if rays else _workload()
    z_lo, z_hi = spatial.slab(rank, w.nz, world)
    tr = OracleTracer(w, z_lo, z_hi, **(RAY_KW if rays else {}))
    rounds = spatial.run_distributed(tr, rank, world, w.nz, dist)
    sums = []
    for a in (tr.S, tr.spec, tr.S_pi, tr.heat):
        t = torch.from_numpy(np.ascontiguousarray(a))
        dist.all_reduce(t)
        sums.append(t.numpy())
    keys = sorted(tr.ledger)
    lt = torch.tensor([tr.ledger[k] for k in keys], dtype=torch.float64)
    dist.all_reduce(lt)
    q.put((rank, rounds, tr.calls, sums if rank == 0 else None, dict(zip(keys, lt.tolist()))))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("rays", [False, True])
def test_two_gloo_ranks_exchange_bundles(rays):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q, rays)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted([q.get(timeout=300) for _ in range(2)], key=lambda g: g[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert got[0][1] == got[1][1] >= 1                  # both ranks saw the same rounds
    S, spec, S_pi, heat = got[0][3]
    sys.path.insert(0, ROOT)
    if rays:
        _compare(S, spec, S_pi, heat, got[0][4], _ray_workload(), **RAY_KW)
    else:
        _compare(S, spec, S_pi, heat, got[0][4], _workload())


@pytest.mark.parametrize("world", [1, 4])
def test_local_lockstep_domains(world):
    """All domains in one process (the driver's run_local), 1 and 4 slabs."""
    sys.path.insert(0, ROOT)
    from paper_2511_07539_gb300 import spatial
    w = _workload()
    trs = [OracleTracer(w, *spatial.slab(r, w.nz, world)) for r in range(world)]
    rounds = spatial.run_local(trs, w.nz)
    # a straight ray crosses each slab boundary at most once
    assert (rounds == 0) == (world == 1) and rounds <= world - 1
    tot = {}
    for t in trs:
        for k, v in t.ledger.items():
            tot[k] = tot.get(k, 0.0) + v
    _compare(sum(t.S for t in trs), sum(t.spec for t in trs), sum(t.S_pi for t in trs),
             sum(t.heat for t in trs), tot, w)


def test_local_lockstep_ray_domains():
    """Rays on the spherical grid in 3 phi-slab domains, all in one process."""
    sys.path.insert(0, ROOT)
    from paper_2511_07539_gb300 import spatial
    w = _ray_workload()
    trs = [OracleTracer(w, *spatial.slab(r, w.nz, 3), **RAY_KW) for r in range(3)]
    rounds = spatial.run_local(trs, w.nz)
    assert 1 <= rounds
    tot = {}
    for t in trs:
        for k, v in t.ledger.items():
            tot[k] = tot.get(k, 0.0) + v
    _compare(sum(t.S for t in trs), sum(t.spec for t in trs), sum(t.S_pi for t in trs),
             sum(t.heat for t in trs), tot, w, **RAY_KW)
