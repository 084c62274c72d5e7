"""Spatial decomposition of one transport pass across processes (Sec. 2.4.1).

Each process owns a domain of whole x-y layers (z slabs of equal thickness),
emits the packets of its own cells, traces them until they end or cross into
another process's cells, and hands those over as bundles of packet states
(the paper's managers exchange bundles of rays between nodes, App. B).
Rounds of trace-and-exchange go on until no packet is in flight anywhere.
Estimators, photoionization rates and spectrum tallies stay with the domain
where they arise; the pass's results are the sums over the domains.

The driver only routes bundles: tracing is done by a tracer object with
  step(emit, bundle_in) -> bundle_out   (packet states, rows of floats)
  z_of(bundle) -> z layer of the cell each packet entered
of which LibDomainTracer drives the CUDA library (run_transport_domain).
Exchange runs over torch.distributed (NCCL between GPUs; any backend with
send/recv), or in one process over all domains in lockstep (run_local).
"""
from __future__ import annotations

import numpy as np


def owner(z, nz, world):
    """Domain of z layer z: world slabs of nz / world layers."""
    return z // (nz // world)


def slab(rank, nz, world):
    """The z layers [z_lo, z_hi) of domain `rank`."""
    h = nz // world
    return rank * h, (rank + 1) * h


class LibDomainTracer:
    """A process's domain traced by the CUDA library: run_transport_domain on
    the context `ctx` (grid, atoms and populations loaded), transport keyword
    arguments as for run_transport (n_packets, seed, spectrum grid, sampler:
    rays take domains on the spherical grid ...).  Bundles stay on the device
    (torch tensors)."""

    def __init__(self, ctx, z_lo, z_hi, device="cuda", **kw):
        import torch
        import paper_2511_07539_gb300 as xt
        self.xt, self.torch = xt, torch
        self.ctx, self.z_lo, self.z_hi, self.kw, self.device = ctx, z_lo, z_hi, kw, device
        self.first = True
        self.cap = 1 << 16
        self.stats = []

    def step(self, emit, bundle_in):
        xt, torch = self.xt, self.torch
        if bundle_in is not None and bundle_in.shape[0] == 0:
            bundle_in = None
        while True:
            out = torch.empty((self.cap, xt.XT_BUNDLE_FIELDS), dtype=torch.float64, device=self.device)
            st, n = xt.run_transport_domain(self.ctx.h, self.z_lo, self.z_hi, emit, bundle_in, out,
                                            accumulate=not self.first, **self.kw)
            if n <= self.cap:
                break
            # too small: the call is deterministic, so run it again with room
            # for all (a pass's first call clears the store, later calls add)
            self.cap = 2 * n
            if self.first:
                continue
            raise RuntimeError("bundle buffer too small after the domain's first call")
        self.first = False
        self.stats.append(st)
        return out[:n]

    def z_of(self, bundle):
        xt = self.xt
        return bundle[:, xt.XT_BUNDLE_CELL].to(self.torch.int64) >> 20


def _route(tracer, bundle, nz, world):
    """Split a bundle by receiving domain: list of world bundles."""
    import torch
    if bundle.shape[0] == 0:
        return [bundle[:0] for _ in range(world)]
    dest = owner(tracer.z_of(bundle), nz, world)
    order = torch.argsort(dest, stable=True)
    counts = torch.bincount(dest, minlength=world).tolist()
    return list(torch.split(bundle[order], counts))


def run_distributed(tracer, rank, world, nz, dist, max_rounds=1 << 20):
    """This process's part of a pass: returns the rounds of exchange.  Every
    process calls it with its own tracer; dist is torch.distributed with an
    initialised default group."""
    import torch
    out = tracer.step(True, None)
    for rnd in range(max_rounds):
        parts = _route(tracer, out, nz, world)
        counts = torch.tensor([p.shape[0] for p in parts], dtype=torch.int64, device=out.device)
        allc = [torch.zeros_like(counts) for _ in range(world)]
        dist.all_gather(allc, counts)
        M = torch.stack(allc).cpu()                   # M[src, dst] packets in flight
        if int(M.sum()) == 0:
            return rnd
        ops, recv = [], []
        for q in range(world):
            if q == rank:
                continue
            if parts[q].shape[0]:
                ops.append(dist.isend(parts[q].contiguous(), q))
            n = int(M[q, rank])
            if n:
                buf = torch.empty((n, out.shape[1]), dtype=out.dtype, device=out.device)
                recv.append(buf)
                ops.append(dist.irecv(buf, q))
        for op in ops:
            op.wait()
        bundle_in = torch.cat(recv) if recv else out[:0]
        out = tracer.step(False, bundle_in)
    raise RuntimeError("spatial decomposition: packets still in flight after max_rounds")


def run_local(tracers, nz, max_rounds=1 << 20):
    """All domains in one process, in lockstep (one GPU, or tests): returns
    the rounds of exchange."""
    import torch
    world = len(tracers)
    outs = [t.step(True, None) for t in tracers]
    for rnd in range(max_rounds):
        parts = [_route(t, o, nz, world) for t, o in zip(tracers, outs)]
        if sum(p.shape[0] for ps in parts for p in ps) == 0:
            return rnd
        outs = [tracers[r].step(False, torch.cat([parts[q][r] for q in range(world)]))
                for r in range(world)]
    raise RuntimeError("spatial decomposition: packets still in flight after max_rounds")
