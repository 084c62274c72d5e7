"""Benchmark: packet-line interactions per second of one transport pass.

A step is one full transport pass (estimator store cleared, emission of every
packet, the resonance event loop with estimator accumulation, spectrum
tallies) over the paper-scale workload: 64^3 cells with lognormal clumps in
four onion zones, 10 synthetic ions of 50-200 levels, 1e5 lines, 1e8 packets,
8^3 subdomains.  The metric counts resonance events with tau_S > 1e-4.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 launch with torch.distributed.run: each rank is an independent
replica over its own packet range (no data-path collective; weak scaling).
``--impl reference`` times the CPU oracle on the host cores on a bounded
packet sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "packet-line interactions/s"
UNIT = "interactions/s"
BYTES_PER_EVENT = 32          # n_l, n_u reads (16 B) + estimator read-modify-write (16 B)
# per packet of the fused pass: the cell's packet energies read (16 B), and the
# direction, lab frequency and id written for the escape tallies (40 B)
BYTES_PER_PACKET = 56
# DRAM bytes (read + write) per event of the attenuation trace kernel (which
# emits its own packets), from an ncu capture of this kernel version on the
# 32^3 onion case (829.96 + 496.58 MB over 7,813,774 events;
# profiles/k_trace_onion32_full.md); the bench's launch is too large to
# capture with many passes, and its traffic is taken as proportional to its
# events.
TRACE_DRAM_BYTES_PER_EVENT = (829.959680e6 + 496.577536e6) / 7813774
# FP64 thread instructions (DFMA + DMUL + DADD) per event of the same kernel and
# capture, and the share of cycles its FP64 pipe was busy: GB300 issues FP64
# arithmetic to 2 lanes per SM and cycle, so the event loop is bound by that
# pipe long before HBM.
TRACE_FP64_OPS_PER_EVENT = 3075609.776316 * (16.308496 + 18.950921 + 22.362010) / 7813774
TRACE_FP64_PIPE_BUSY = 0.58324374
FP64_LANES_PER_SM_CYCLE = 2


# the host arrays a context load uploads
E2E_INPUTS = ("Te", "ne", "L_cell", "rho", "deposition", "level_off", "E_level", "g_level", "lo",
              "up", "lambda_A", "f_lu", "n_ion_density", "pops")


def _pinned_inputs(w):
    """A shallow copy of the workload whose uploaded arrays live in pinned
    (page-locked) host memory, in the dtypes the binding passes through."""
    import copy
    import torch
    wp = copy.copy(w)
    ints = ("level_off", "lo", "up")
    for k in E2E_INPUTS:
        a = getattr(w, k)
        if a is None:
            continue
        a = np.ascontiguousarray(a, dtype=np.int32 if k in ints else np.float64)
        t = torch.empty(a.shape, dtype=torch.int32 if k in ints else torch.float64, pin_memory=True)
        t.numpy()[...] = a
        setattr(wp, k, t.numpy())
    return wp


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def make_workload(args):
    import synth
    if args.workload == "onion":
        return synth.clumpy_onion(n_packets=args.packets)
    if args.workload == "onion-small":     # profiling case: 32^3 x 1e4 lines (2.6 GB store)
        return synth.clumpy_onion(n=32, n_lines=10_000, n_packets=min(args.packets, 4_000_000),
                                  subdomains=(4, 4, 4))
    if args.workload == "sphere":
        return synth.uniform_sphere(n_packets=min(args.packets, 100_000))
    if args.workload == "onion-thin":      # the event loop's regime: ~35 events per packet
        return thin_onion(min(args.packets, THIN_PACKETS))
    raise SystemExit(f"unknown workload {args.workload}")


THIN_POP_SCALE = 1e-7       # every population of the 64^3 onion scaled down
THIN_PACKETS = 20_000_000


def thin_onion(n_packets=THIN_PACKETS):
    """The 64^3 x 1e5-line onion with every level population scaled by 1e-7:
    the lines are 1e7 times thinner, so a packet meets ~300 resonances and
    ~35 interaction points (tau_S > 1e-4) before it leaves or drops below the
    energy cut, instead of ~3 and ~2 at the paper-scale densities."""
    import synth
    w = synth.clumpy_onion(n_packets=n_packets)
    w.pops = w.pops * THIN_POP_SCALE
    w.name = w.name + f"_pops_x{THIN_POP_SCALE:g}"
    return w


def thin_bench(local, stream_ptr, passes=3):
    """The attenuation pass on the thin-line onion (the event loop dominates):
    events/s and the trace kernel's algorithmic HBM rate at 32 B per event."""
    import torch
    import paper_2511_07539_gb300 as xt
    w = thin_onion()
    peaks, _ = _measured_peaks()
    ctx = xt.Context(local, stream_ptr)
    ctx.load(w)
    ctx.transport(w)
    sts = [ctx.transport(w) for _ in range(passes)]
    torch.cuda.synchronize()
    ctx.close()
    ev = float(np.mean([s["events"] for s in sts]))
    tr = float(np.mean([s["trace_ms"] for s in sts]))
    dev = float(np.mean([s["transport_ms"] for s in sts]))
    ach = BYTES_PER_EVENT * ev / (tr * 1e-3) / 1e9
    return {"workload": w.name, "packets": w.n_packets, "events_per_pass": ev,
            "tests_per_pass": float(np.mean([s["tests"] for s in sts])),
            "events_per_packet": ev / w.n_packets, "pass_device_ms": dev, "trace_ms": tr,
            "value": ev / (dev * 1e-3), "unit": UNIT,
            "trace_GB_per_s": ach, "frac_hbm": ach / peaks["hbm_gbs"]}


def rays_bench(local, stream_ptr):
    """The RAYS sampler (Sec. 2.3) on the 32^3 onion with the paper-scale line
    list (1e5 lines): rays from every cell centre for every 1 % bin of the
    band and 10 x 10 viewers, with each batch's line window staged in shared
    memory (XT_FLAG_RAYS_STAGED) and with the line list read through L2
    (default), at the paper-scale line density and with 1e7 times thinner
    lines."""
    import torch
    import paper_2511_07539_gb300 as xt
    import synth
    w = synth.clumpy_onion(n=32, n_packets=1, subdomains=(4, 4, 4))
    ctx = xt.Context(local, stream_ptr)
    kw = dict(sampler=xt.XT_SAMPLER_RAYS, n_theta=10, n_phi=10, spec_dlog=1e-2)
    out = {"workload": w.name + "_rays_10x10_viewers_1pc_bins"}
    for dens, scale in (("paper_density", 1.0), ("thin_lines", THIN_POP_SCALE)):
        ctx.load(w, pops=w.pops * scale)
        res = {}
        for name, flags in (("staged", xt.XT_FLAG_RAYS_STAGED), ("unstaged", 0)):
            ctx.transport(w, flags=flags, **kw)
            st = min((ctx.transport(w, flags=flags, **kw) for _ in range(2)), key=lambda x: x["trace_ms"])
            res[name] = {"trace_ms": st["trace_ms"], "rays": st["rays"], "events": st["events"],
                         "tests": st["tests"], "rays_per_s": st["rays"] / (st["trace_ms"] * 1e-3),
                         "events_per_s": st["events"] / (st["trace_ms"] * 1e-3)}
        res["speedup_staged"] = res["unstaged"]["trace_ms"] / res["staged"]["trace_ms"]
        out[dens] = res
    ctx.close()
    torch.cuda.synchronize()
    return out


SPH_POP_SCALE = 1e-6


def paper_sphere(n_packets=20_000_000):
    """The paper's spherical grid (38 x 15 x 30 zones in r, theta, phi; Sec.
    2) in 30 azimuthal slices, lognormal clumps, one ion of 200 levels with 1e4
    lines, level populations scaled by 1e-6 (about 35 interaction points per
    packet, 40 % of the packets escape)."""
    import synth
    w = synth.spherical_sphere(n_packets=n_packets, seed=23, nr=38, nth=15, nph=30, n_lines=10_000,
                               n_levels=200, subdomains=(1, 1, 30), clumps=True)
    w.pops = w.pops * SPH_POP_SCALE
    w.name = w.name + f"_pops_x{SPH_POP_SCALE:g}"
    return w


def sph_bench(local, stream_ptr, passes=3, n_packets=20_000_000):
    """The attenuation pass on the paper's spherical grid: events/s and the
    trace kernel's algorithmic HBM rate at 32 B per event."""
    import torch
    import paper_2511_07539_gb300 as xt
    w = paper_sphere(n_packets)
    peaks, _ = _measured_peaks()
    ctx = xt.Context(local, stream_ptr)
    ctx.load(w)
    ctx.transport(w)
    sts = [ctx.transport(w) for _ in range(passes)]
    torch.cuda.synchronize()
    ctx.close()
    ev = float(np.mean([s["events"] for s in sts]))
    tr = float(np.mean([s["trace_ms"] for s in sts]))
    dev = float(np.mean([s["transport_ms"] for s in sts]))
    ach = BYTES_PER_EVENT * ev / (tr * 1e-3) / 1e9
    return {"workload": w.name, "packets": w.n_packets, "cells": w.ncell, "events_per_pass": ev,
            "tests_per_pass": float(np.mean([s["tests"] for s in sts])),
            "events_per_packet": ev / w.n_packets, "pass_device_ms": dev, "trace_ms": tr,
            "value": ev / (dev * 1e-3), "unit": UNIT, "packets_per_s": w.n_packets / (dev * 1e-3),
            "trace_GB_per_s": ach, "frac_hbm": ach / peaks["hbm_gbs"], "kernel": "k_trace_sph"}


def paper_rays_bench(local, stream_ptr, steps=1):
    """The paper's radiative-transfer pass at its own scale (Sec. 2.3, the ray
    count of its validation pass): the RAYS sampler on the 38 x 15 x 30
    spherical grid of paper_sphere(), band emission over 400-15000 A on the 0.1 %
    output grid from 400 A (3626 emitting bins) and 20 x 20 viewers: 17,100 x
    3626 x 400 = 2.48e10 rays per pass.  One warm-up pass, then `steps` timed."""
    import torch
    import paper_2511_07539_gb300 as xt
    w = paper_sphere(1)
    w.band_A = (400.0, 15000.0)
    nb = int(np.ceil(np.log(15000.0 * (1.0 + 1.5 * w.v_max / 2.99792458e10) / 400.0) / np.log1p(1e-3)))
    kw = dict(sampler=xt.XT_SAMPLER_RAYS, n_theta=20, n_phi=20, spec_lam0_A=400.0, spec_dlog=1e-3,
              spec_nbins=nb, seed=w.seed)
    ctx = xt.Context(local, stream_ptr)
    ctx.load(w)
    xt.run_transport(ctx.h, 1, **kw)
    sts = [xt.run_transport(ctx.h, 1, **kw) for _ in range(steps)]
    torch.cuda.synchronize()
    ctx.close()
    st = min(sts, key=lambda x: x["transport_ms"])
    return {"workload": w.name.replace("_1pk", "_rays") + "_band_400-15000A_0.1pc_bins_20x20_viewers",
            "rays": st["rays"], "events": st["events"], "tests": st["tests"],
            "pass_device_ms": st["transport_ms"], "trace_ms": st["trace_ms"],
            "rays_per_s": st["rays"] / (st["transport_ms"] * 1e-3),
            "events_per_s": st["events"] / (st["transport_ms"] * 1e-3),
            "trace_launches": st["rounds"], "escaped_E_over_emitted": st["escaped_E"] / st["emitted_E"]}


def cfg5_bench(local, stream_ptr, packets=1_000_000_000):
    """The full-loop scale (128^3 cells, 10 ions, 2e4 lines, 1e9 packets, 4^3
    subdomains) on one GPU: the dense FP64 store (336 GB) does not fit the
    device, the store with rows for the cells with matter only (1.1e6 of 2.1e6)
    does.  Times one transport pass and the estimator-rate solve of every
    (cell, ion) that follows it (one outer step of the coupled loop)."""
    import torch
    import paper_2511_07539_gb300 as xt
    import synth
    t0 = time.perf_counter()
    w = synth.clumpy_onion(n=128, n_lines=20_000, n_packets=packets, subdomains=(4, 4, 4))
    ups = synth.collision_strengths(w.upsilon_seed, w.level_off)
    gen_s = time.perf_counter() - t0
    ctx = xt.Context(local, stream_ptr)
    ctx.load(w)
    xt.set_estimator_store(ctx.h, xt.XT_STORE_COMPACT_ROWS)
    st0 = ctx.transport(w)                    # allocations, row map
    torch.cuda.synchronize()
    st = ctx.transport(w)
    sz = xt.get_sizes(ctx.h)
    sol = xt.solve_nlte(ctx.h, ups, precision=xt.XT_PREC_FP32_IR, rates=xt.XT_RATES_ESTIMATORS,
                        warm=xt.XT_WARM_CURRENT)
    free, total = torch.cuda.mem_get_info()
    ctx.close()
    return {"workload": w.name, "cells": w.ncell, "cells_with_matter": int((w.rho > 0).sum()),
            "lines": w.nline, "packets": packets, "generate_s": gen_s,
            "store_GB": sz["store_bytes"] / 1e9, "dense_store_GB": w.ncell * w.nline * 8 / 1e9,
            "transport_ms": st["transport_ms"], "events": st["events"],
            "events_per_s": st["events"] / (st["transport_ms"] * 1e-3),
            "first_pass_ms": st0["transport_ms"], "solve_ms": sol["solve_ms"], "systems": sol["systems"],
            "fp64_fallbacks": sol["fp64_fallbacks"], "device_GB_free_after": free / 1e9}


def cfg5_loop_bench(local, stream_ptr, packets=1_000_000_000):
    """A10 at the full-loop scale: the coupled loop to a relative population
    change <= 1e-3 on 128^3 cells (1.1e6 with matter; 10 ions of 20-60 levels,
    2e4 lines, 1e9 packets per pass, 4^3 subdomains, the estimator store with
    rows for the cells with matter only), the plain loop (FP64 factors from
    Boltzmann populations) against the fast one (FP32 factors with FP64
    refinement from the surrogate's prediction).  The surrogate is trained
    beforehand, outside the timing, on the converged populations of a 32^3
    realization with the same atoms.  Both loops timed by the host clock around
    the whole run_coupled call."""
    import torch
    import paper_2511_07539_gb300 as xt
    import synth
    kw = dict(seed=1, n_lines=20_000, level_range=(20, 60), subdomains=(4, 4, 4))
    A = synth.clumpy_onion(n=32, n_packets=2_000_000, **kw)
    B = synth.clumpy_onion(n=128, n_packets=packets, field_seed=2, **kw)
    for k in ("level_off", "E_level", "g_level", "lo", "up", "lambda_A", "f_lu"):
        assert np.array_equal(getattr(A, k), getattr(B, k)), k      # the same atoms
    ups = synth.collision_strengths(A.upsilon_seed, A.level_off)
    common = dict(tol=1e-3, jbar_W=5.6e-5, jbar_TR=8000.0, spec_lam0_A=B.spec_band_A[0],
                  spec_nbins=B.spec_band_A[1], seed=B.seed)
    ctx = xt.Context(local, stream_ptr)
    ctx.load(A)
    t0 = time.perf_counter()
    stA = xt.run_coupled(ctx.h, ups, A.n_packets, start=xt.XT_WARM_LTE, precision=xt.XT_PREC_FP32_IR,
                         **common)
    tr = xt.train_surrogate(ctx.h, epochs=60, batch=128, lr=2e-3, rates=xt.XT_RATES_JBAR,
                            jbar_W=5.6e-5, jbar_TR=8000.0)
    prep_s = time.perf_counter() - t0
    res, pops = {}, {}
    for name, start, prec in (("plain_fp64", xt.XT_WARM_LTE, xt.XT_PREC_FP64),
                              ("surrogate_mixed", xt.XT_WARM_SURROGATE, xt.XT_PREC_FP32_IR)):
        ctx.load(B)
        xt.set_estimator_store(ctx.h, xt.XT_STORE_COMPACT_ROWS)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        st = xt.run_coupled(ctx.h, ups, B.n_packets, start=start, precision=prec, max_outer=30, **common)
        torch.cuda.synchronize()
        host_s = time.perf_counter() - t1
        p = np.zeros((B.ncell, B.nlev))
        xt.get_populations(ctx.h, p)
        pops[name] = p
        res[name] = {k: st[k] for k in ("outer", "converged", "wall_ms", "start_ms", "transport_ms",
                                        "solve_ms", "newton_steps", "max_newton_steps", "not_converged",
                                        "change")}
        res[name]["host_s"] = host_s
    sz = xt.get_sizes(ctx.h)
    free, _ = torch.cuda.mem_get_info()
    ctx.close()
    nz = np.repeat(B.n_ion_density, np.diff(B.level_off), axis=1)
    ref = pops["plain_fp64"]
    sig = (ref >= 1e-20 * nz) & (nz > 0)
    dev = float(np.max(np.abs(pops["surrogate_mixed"][sig] / ref[sig] - 1)))
    return {"workload": B.name + " (clump field 2; surrogate trained on a 32^3 realization)",
            "cells": B.ncell, "cells_with_matter": int((B.rho > 0).sum()), "systems": B.ncell * B.n_ion,
            "store_GB": sz["store_bytes"] / 1e9, "device_GB_free_after": free / 1e9, "tol": 1e-3, **res,
            "max_rel_dev_vs_plain": dev,
            "speedup_surrogate_mixed_vs_plain": res["plain_fp64"]["wall_ms"] / res["surrogate_mixed"]["wall_ms"],
            "training": {"outer_32": stA["outer"], "last_loss": tr["last_loss"], "steps": tr["steps"],
                         "train_ms": tr["train_ms"], "prep_s": prep_s}}


def collision_sphere(n_packets=20_000_000):
    """A 16^3 sphere whose 12 lines lie within 5000-5080 A and whose band is
    4990-5100 A: every packet meets most lines, so the lanes of a warp often
    add to the same (cell, line) estimator slot at once."""
    import synth
    w = synth.uniform_sphere(n=16, n_packets=n_packets, n_lines=12, n_levels=8, seed=35)
    w.lambda_A = np.linspace(5000.0, 5080.0, 12)
    w.band_A = (4990.0, 5100.0)
    w.spec_band_A = synth._spectrum_grid(w.band_A[0], w.band_A[1], w.v_max)
    w.pops = w.pops * 1e-3
    w.name = "collision_sphere_16^3_12lines"
    return w


def prereduce_bench(local, stream_ptr, w_main):
    """The trace kernel with the warp pre-reduction of estimator increments
    (XT_FLAG_WARP_REDUCE) and without it (default), on the paper-scale onion,
    its thin-line variant and a workload whose lanes often share a slot."""
    import paper_2511_07539_gb300 as xt
    out = {}
    for name, w in (("onion", w_main), ("thin_lines", thin_onion()), ("collisions", collision_sphere())):
        ctx = xt.Context(local, stream_ptr)
        ctx.load(w)
        res = {}
        for flags in (xt.XT_FLAG_WARP_REDUCE, 0, xt.XT_FLAG_WARP_REDUCE, 0):
            ctx.transport(w, flags=flags)
            ms = min(ctx.transport(w, flags=flags)["trace_ms"] for _ in range(2))
            key = "reduce" if flags else "no_reduce"
            res[key] = min(ms, res.get(key, ms))
        st = ctx.transport(w)
        ctx.close()
        out[name] = {"trace_ms_reduce": res["reduce"], "trace_ms_no_reduce": res["no_reduce"],
                     "events": st["events"], "ratio": res["no_reduce"] / res["reduce"]}
    return out


def workload_config(w, world):
    """The `config` object of both arms' lines: the workload by name and size."""
    store_gb = w.ncell * w.nline * 8 / 1e9          # dense estimator store, FP64
    l2 = (f"inputs larger than L2: estimator store ({store_gb:.1f} GB) cleared every step"
          if store_gb > 0.129 else
          f"inputs within L2 (estimator store {store_gb * 1e3:.1f} MB): a test case, not a bench line")
    return {"workload": w.name, "cells": w.ncell, "lines": w.nline, "levels": w.nlev,
            "packets_per_gpu": w.n_packets, "subdomains": list(w.subdomains),
            "mode": "attenuation", "l2": l2, "parallelism": f"replicas{world}"}


def replica_seed(base_seed, rank):
    """Seed of rank `rank`'s replica: every rank transports its own packets."""
    return base_seed + 1000003 * rank


def reduce_over_ranks(ms, ev, dist=None, device="cuda"):
    """(largest time, summed events) over the ranks of the default process
    group (this rank's own values without one)."""
    import torch
    t = torch.tensor([ms, ev], dtype=torch.float64, device=device)
    if dist is not None:
        tm = t.clone()
        dist.all_reduce(tm[0:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(tm[1:2], op=dist.ReduceOp.SUM)
        t = tm
    return float(t[0]), float(t[1])


def _oracle_on_cores(w, seconds, chunk, seed, cores):
    """The oracle, as it stands, on `cores` host threads at once (the C code
    runs with the interpreter lock released), each transporting random
    contiguous `chunk`-packet ranges of the workload until `seconds` have
    passed; estimators are not kept (the same arithmetic runs).  Returns
    (events, packets, seconds, per-chunk seconds)."""
    import concurrent.futures as cf
    import oracle
    oracle.build()
    oracle.transport(w, p_begin=0, p_end=10, estimators=False)     # warm (build, load)
    t0 = time.perf_counter()

    def work(k):
        rng = np.random.default_rng([seed, k])
        ev, npk, times = 0.0, 0, []
        while time.perf_counter() - t0 < seconds:
            p0 = int(rng.integers(0, max(1, w.n_packets - chunk)))
            t1 = time.perf_counter()
            o = oracle.transport(w, p_begin=p0, p_end=min(p0 + chunk, w.n_packets), estimators=False)
            times.append(time.perf_counter() - t1)
            ev += o["ledger"]["events"]
            npk += chunk
        return ev, npk, times

    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        res = list(ex.map(work, range(cores)))
    dt = time.perf_counter() - t0
    return (sum(r[0] for r in res), sum(r[1] for r in res), dt, [t for r in res for t in r[2]])


def cpu_baseline(w, seconds=12.0):
    """The oracle, as it stands, on every host core over a bounded packet sample."""
    cores = os.cpu_count() or 1
    events, n_pk, dt, _ = _oracle_on_cores(w, seconds, 20_000, 123, cores)
    return {"value": events / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_pk} packets in 20000-packet random contiguous ranges of the "
                      f"{w.n_packets}-packet workload, the serial C oracle on {cores} host "
                      f"threads at once, {dt:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = make_workload(args)
    cores = os.cpu_count() or 1
    per_step = []
    events = 0.0
    n_pk = 0
    for s in range(args.warmup + args.steps):
        # one step: the oracle on every host core for a bounded time
        ev, npk, dt, _ = _oracle_on_cores(w, 6.0, 20_000, 7 + s, cores)
        if s >= args.warmup:
            per_step.append(dt)
            events += ev
            n_pk += npk
    T = sum(per_step)
    v = events / T
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": workload_config(w, world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n_pk} packets, 20000-packet random contiguous ranges "
                                       f"on {cores} host threads, about 6 s per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def nlte_bench(local, stream_ptr, n=64):
    """A8 on the batched rate-solve workload (n^3 cells x 10 ions, 20-300
    levels each; n = 64: 2.6e6 systems): FP32 LU + FP64 refinement, TF32 and
    BF16 LU updates on the tensor cores + FP64 refinement, and the plain FP64
    LU, each on every system and timed; the mixed, TF32 and BF16 results'
    deviation from the FP64 one on the (n/2)^3 sub-batch (1/8 of the systems)."""
    import paper_2511_07539_gb300 as xt
    import synth
    out = {}
    w = synth.nlte_batch(n=n)
    kw = dict(rates=xt.XT_RATES_JBAR, warm=xt.XT_WARM_CURRENT, jbar_W=w.jbar_W,
              jbar_TR=w.jbar_TR, levels_used=w.levels_used)
    ctx = xt.Context(local, stream_ptr)
    ctx.load(w)
    xt.solve_nlte(ctx.h, w.upsilon, precision=xt.XT_PREC_FP32_IR, autotune=True, use_graph=True, **kw)
    best = None
    for _ in range(3):
        xt.set_populations(ctx.h, w.pops)
        st = xt.solve_nlte(ctx.h, w.upsilon, precision=xt.XT_PREC_FP32_IR, use_graph=True, **kw)
        best = st if best is None or st["solve_ms"] < best["solve_ms"] else best
    out["mixed"] = {"systems": best["systems"], "solve_ms": best["solve_ms"],
                    "lu_tflops": best["lu_flops"] / (best["solve_ms"] * 1e-3) / 1e12,
                    "fp64_fallbacks": best["fp64_fallbacks"], "mean_refinements": best["mean_iter"],
                    "max_refinements": best["max_iter_used"], "panel_width": best["panel_width"]}
    # the same with the LU's trailing updates on the tensor cores, TF32 and BF16
    def tensor_leg(prec):
        xt.set_populations(ctx.h, w.pops)
        xt.solve_nlte(ctx.h, w.upsilon, precision=prec, autotune=True, use_graph=True, **kw)
        tb = None
        for _ in range(2):
            xt.set_populations(ctx.h, w.pops)
            st = xt.solve_nlte(ctx.h, w.upsilon, precision=prec, use_graph=True, **kw)
            tb = st if tb is None or st["solve_ms"] < tb["solve_ms"] else tb
        return {"solve_ms": tb["solve_ms"], "fp64_fallbacks": tb["fp64_fallbacks"],
                "mean_refinements": tb["mean_iter"], "max_refinements": tb["max_iter_used"],
                "panel_width": tb["panel_width"]}
    out["tf32"] = tensor_leg(xt.XT_PREC_TF32_IR)
    out["bf16"] = tensor_leg(xt.XT_PREC_BF16_IR)
    # the plain FP64 LU on the whole batch, timed
    xt.set_populations(ctx.h, w.pops)
    st64f = xt.solve_nlte(ctx.h, w.upsilon, precision=xt.XT_PREC_FP64, **kw)
    out["fp64"] = {"systems": st64f["systems"], "solve_ms": st64f["solve_ms"],
                   "lu_tflops": st64f["lu_flops"] / (st64f["solve_ms"] * 1e-3) / 1e12,
                   "singular": st64f["singular"]}
    ctx.close()
    del w
    ws = synth.nlte_batch(n=max(n // 2, 1))
    kws = dict(rates=xt.XT_RATES_JBAR, warm=xt.XT_WARM_CURRENT, jbar_W=ws.jbar_W,
               jbar_TR=ws.jbar_TR, levels_used=ws.levels_used)
    ctx = xt.Context(local, stream_ptr)
    ctx.load(ws)
    p64 = np.zeros((ws.ncell, ws.nlev))
    st64 = xt.solve_nlte(ctx.h, ws.upsilon, precision=xt.XT_PREC_FP64, pops_out=p64, **kws)
    xt.set_populations(ctx.h, ws.pops)
    p32 = np.zeros_like(p64)
    st32 = xt.solve_nlte(ctx.h, ws.upsilon, precision=xt.XT_PREC_FP32_IR, pops_out=p32,
                         autotune=True, **kws)
    xt.set_populations(ctx.h, ws.pops)
    ptf = np.zeros_like(p64)
    xt.solve_nlte(ctx.h, ws.upsilon, precision=xt.XT_PREC_TF32_IR, pops_out=ptf, autotune=True, **kws)
    xt.set_populations(ctx.h, ws.pops)
    pbf = np.zeros_like(p64)
    xt.solve_nlte(ctx.h, ws.upsilon, precision=xt.XT_PREC_BF16_IR, pops_out=pbf, autotune=True, **kws)
    ctx.close()
    nz = np.repeat(ws.n_ion_density, np.diff(ws.level_off), axis=1)
    sig = p64 >= 1e-30 * nz
    err = float(np.max(np.abs(p32[sig] / p64[sig] - 1)))
    out["deviation_subbatch"] = {"systems": st64["systems"], "fp64_ms": st64["solve_ms"],
                                 "mixed_ms": st32["solve_ms"]}
    out["max_rel_dev_mixed_vs_fp64"] = err
    out["max_rel_dev_tf32_vs_fp64"] = float(np.max(np.abs(ptf[sig] / p64[sig] - 1)))
    out["max_rel_dev_bf16_vs_fp64"] = float(np.max(np.abs(pbf[sig] / p64[sig] - 1)))
    out["speedup_vs_fp64"] = out["fp64"]["solve_ms"] / best["solve_ms"]
    out["speedup_tf32_vs_fp64"] = out["fp64"]["solve_ms"] / out["tf32"]["solve_ms"]
    out["speedup_bf16_vs_fp64"] = out["fp64"]["solve_ms"] / out["bf16"]["solve_ms"]
    return out


def train_bench(local, stream_ptr, epochs=60):
    """A9 training alone: the surrogate (4 layers: 333 -> 256 -> 256 -> 256 ->
    406) on the 32^3 onion's populations (10 ions of 20-60 levels, J_ext
    rates), batch 128, `epochs` passes over the 17,152 cells with matter, all
    steps in launches of the fused training kernel.  Timed twice, the second
    continuing from the first's weights; the faster is reported."""
    import paper_2511_07539_gb300 as xt
    import synth
    w = synth.clumpy_onion(n=32, n_packets=2_000_000, seed=1, n_lines=5000, level_range=(20, 60),
                           subdomains=(4, 4, 4))
    ctx = xt.Context(local, stream_ptr)
    ctx.load(w)
    runs = [xt.train_surrogate(ctx.h, epochs=epochs, batch=128, lr=2e-3, rates=xt.XT_RATES_JBAR,
                               jbar_W=5.6e-5, jbar_TR=8000.0) for _ in range(2)]
    ctx.close()
    tr = min(runs, key=lambda r: r["train_ms"])
    return {"workload": w.name + " surrogate 333-256-256-256-406, batch 128", "epochs": epochs,
            "steps": tr["steps"], "train_ms": tr["train_ms"], "us_per_step": tr["train_ms"] * 1e3 / tr["steps"],
            "first_loss": runs[0]["first_loss"], "last_loss": runs[0]["last_loss"]}


def coupled_bench(local, stream_ptr, n=32):
    """A10: the coupled loop to a relative population change <= 1e-3 on a
    clumpy onion of n^3 cells (10 ions of 20-60 levels, 5000 lines, 2e6
    packets per pass): the plain loop (Newton steps factored in FP64 from
    Boltzmann populations) against the fast one (FP32 factors with FP64
    refinement, Newton from the surrogate's prediction).  The surrogate is
    trained beforehand, and outside the timing, on the converged populations of
    another clump realization with the same atoms.  Both loops are timed by the
    host clock around the whole run_coupled call (start populations included)."""
    import paper_2511_07539_gb300 as xt
    import synth
    kw_w = dict(seed=1, n=n, n_packets=2_000_000, n_lines=5000, level_range=(20, 60),
                subdomains=(4, 4, 4))
    A = synth.clumpy_onion(**kw_w)
    B = synth.clumpy_onion(field_seed=2, **kw_w)
    ups = synth.collision_strengths(A.upsilon_seed, A.level_off)
    common = dict(tol=1e-3, jbar_W=5.6e-5, jbar_TR=8000.0, spec_lam0_A=A.spec_band_A[0],
                  spec_nbins=A.spec_band_A[1], seed=A.seed)
    ctx = xt.Context(local, stream_ptr)
    ctx.load(A)
    stA = xt.run_coupled(ctx.h, ups, A.n_packets, start=xt.XT_WARM_LTE,
                         precision=xt.XT_PREC_FP32_IR, **common)
    tr = xt.train_surrogate(ctx.h, epochs=60, batch=128, lr=2e-3, rates=xt.XT_RATES_JBAR,
                            jbar_W=5.6e-5, jbar_TR=8000.0)
    ctx.load(B)
    xt.run_coupled(ctx.h, ups, B.n_packets, start=xt.XT_WARM_LTE, max_outer=1,
                   precision=xt.XT_PREC_FP32_IR, **common)           # warm-up (buffers)
    res, pops = {}, {}
    for name, start, prec in (("plain_fp64", xt.XT_WARM_LTE, xt.XT_PREC_FP64),
                              ("surrogate_mixed", xt.XT_WARM_SURROGATE, xt.XT_PREC_FP32_IR),
                              ("lte_mixed", xt.XT_WARM_LTE, xt.XT_PREC_FP32_IR)):
        ctx.load(B)
        st = xt.run_coupled(ctx.h, ups, B.n_packets, start=start, precision=prec, **common)
        p = np.zeros((B.ncell, B.nlev))
        xt.get_populations(ctx.h, p)
        pops[name] = p
        res[name] = {k: st[k] for k in ("outer", "converged", "wall_ms", "start_ms",
                                        "transport_ms", "solve_ms", "newton_steps",
                                        "max_newton_steps", "not_converged", "change")}
    ctx.close()
    nz = np.repeat(B.n_ion_density, np.diff(B.level_off), axis=1)
    ref = pops["plain_fp64"]
    sig = (ref >= 1e-20 * nz) & (nz > 0)
    dev = {k: float(np.max(np.abs(v[sig] / ref[sig] - 1))) for k, v in pops.items() if k != "plain_fp64"}
    return {"workload": B.name + " (clump field 2; surrogate trained on clump field 1)",
            "tol": 1e-3, **res, "max_rel_dev_vs_plain": dev,
            "speedup_surrogate_mixed_vs_plain": res["plain_fp64"]["wall_ms"] / res["surrogate_mixed"]["wall_ms"],
            "training": {"realization_1_outer": stA["outer"], "first_loss": tr["first_loss"],
                         "last_loss": tr["last_loss"], "steps": tr["steps"],
                         "train_ms": tr["train_ms"]}}


def scatter_rates_bench(local, stream_ptr):
    """A3b and A7 on the 32^3 onion (1e4 lines, 4e6 packets, 2.6 GB store):
    scatter-mode passes (interaction = the whole packet absorbed with
    probability 1 - e^-tau, re-emitted in a down-line or destroyed), and the
    rates R_lu = S / (n_l V) of the whole store written to device memory."""
    import torch
    import paper_2511_07539_gb300 as xt
    import synth
    w = synth.clumpy_onion(n=32, n_lines=10_000, n_packets=4_000_000, subdomains=(4, 4, 4))
    ups = synth.collision_strengths(w.upsilon_seed, w.level_off)
    ups_down = np.concatenate([u.sum(axis=0) for u in ups])   # sum_{j<u} Upsilon_ju per level
    stream = torch.cuda.current_stream()
    ctx = xt.Context(local, stream_ptr)
    ctx.load(w, with_scatter_data=ups_down)
    out = {"workload": w.name}
    kw = dict(mode=xt.XT_MODE_SCATTER, seed=w.seed)
    for _ in range(2):
        ctx.transport(w, **kw)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sts = [ctx.transport(w, **kw) for _ in range(3)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 3
    out["scatter"] = {"ms_per_pass": ms, "events_per_s": sts[-1]["events"] / (ms * 1e-3),
                      "interactions_per_s": sts[-1]["interactions"] / (ms * 1e-3),
                      "packets_per_s": w.n_packets / (ms * 1e-3),
                      "interactions_per_packet": sts[-1]["interactions"] / w.n_packets,
                      "launches_per_pass": float(sts[-1]["kernels"])}
    # rates of every (cell, line) of an attenuation pass's store, device to device
    ctx.transport(w, seed=w.seed)
    R = torch.empty((w.ncell, w.nline), dtype=torch.float64, device="cuda")
    xt.get_photoexcitation_rates(ctx.h, R_lu=R, want=("R_lu",))
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        xt.get_photoexcitation_rates(ctx.h, R_lu=R, want=("R_lu",))
    e1.record(stream)
    torch.cuda.synchronize()
    ms_r = e0.elapsed_time(e1) / 3
    elems = w.ncell * w.nline
    # algorithmic bytes per (cell, line): the estimator read, the rate written
    out["rates"] = {"ms": ms_r, "elements": elems, "GB_per_s": 16 * elems / (ms_r * 1e-3) / 1e9,
                    "bytes_per_element": 16}
    ctx.close()
    return out


def stream_bench(local, stream_ptr, groups=8, packets=100_000_000):
    """The estimator store held in pinned host memory and streamed through the
    device by groups of subdomain z-layers, against the device-resident store,
    on the 64^3 onion with 1e4 lines (21 GB store; 8 groups of 2.6 GB)."""
    import paper_2511_07539_gb300 as xt
    import synth
    w = synth.clumpy_onion(n_lines=10_000, n_packets=packets)
    ctx = xt.Context(local, stream_ptr)
    ctx.load(w)
    out = {"workload": w.name, "groups": groups}
    for name, g in (("resident", 0), ("host_streamed", groups)):
        xt.set_estimator_store(ctx.h, g)
        ctx.transport(w)                                   # warm-up (allocations)
        best = None
        for _ in range(2):
            st = ctx.transport(w)
            best = st if best is None or st["transport_ms"] < best["transport_ms"] else best
        out[name] = {"value": best["events"] / (best["transport_ms"] * 1e-3), "unit": UNIT,
                     "ms_per_pass": best["transport_ms"], "launches": best["rounds"],
                     "store_bytes": float(w.ncell) * w.nline * 8}
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--packets", type=int, default=100_000_000)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="onion",
                    choices=["onion", "onion-small", "onion-thin", "sphere"])
    ap.add_argument("--no-thin", action="store_true", help="skip the thin-line measurement")
    ap.add_argument("--no-rays", action="store_true", help="skip the RAYS-sampler measurement")
    ap.add_argument("--no-sph", action="store_true", help="skip the spherical-grid measurement")
    ap.add_argument("--only-sph", action="store_true", help="print the spherical-grid object alone")
    ap.add_argument("--sph-packets", type=int, default=20_000_000)
    ap.add_argument("--prereduce", action="store_true",
                    help="also time the trace kernel with and without the warp pre-reduction")
    ap.add_argument("--no-nlte", action="store_true", help="skip the rate-solve measurement")
    ap.add_argument("--no-coupled", action="store_true", help="skip the coupled-loop measurement")
    ap.add_argument("--only-coupled", action="store_true", help="print the coupled-loop object alone")
    ap.add_argument("--coupled-n", type=int, default=32)
    ap.add_argument("--only-train", action="store_true", help="print the surrogate-training object alone")
    ap.add_argument("--train-epochs", type=int, default=60)
    ap.add_argument("--no-stream", action="store_true", help="skip the host-streamed store measurement")
    ap.add_argument("--no-scatter", action="store_true",
                    help="skip the scatter-mode and rates measurement")
    ap.add_argument("--only-scatter", action="store_true",
                    help="print the scatter-mode and rates object alone")
    ap.add_argument("--only-nlte", action="store_true", help="print the rate-solve object alone")
    ap.add_argument("--only-cfg5", action="store_true",
                    help="print the 128^3 full-loop-scale object alone (a pass and a solve)")
    ap.add_argument("--only-paper-rays", action="store_true",
                    help="print the paper's full RAYS pass on its spherical grid alone (2.48e10 rays)")
    ap.add_argument("--only-cfg5-loop", action="store_true",
                    help="print the 128^3 coupled-loop object alone (plain vs surrogate + mixed)")
    ap.add_argument("--nlte-n", type=int, default=64)
    ap.add_argument("--nlte-precision", default="fp32", choices=["fp32", "tf32", "bf16", "fp64"],
                    help="with --only-nlte --nlte-once: the factor precision of that launch")
    ap.add_argument("--nlte-once", action="store_true",
                    help="with --only-nlte: one plain mixed-precision launch (profiling case)")
    ap.add_argument("--rounds-steps", type=int, default=1,
                    help="extra timed passes with subdomain rounds (0 to skip)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    assert torch.cuda.is_available(), "bench needs a GPU"
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    import __graft_entry__ as g
    if rank == 0:
        g.build()
    barrier()
    g.build()
    import paper_2511_07539_gb300 as xt

    if args.only_nlte and args.nlte_once:
        import synth
        w = synth.nlte_batch(n=args.nlte_n)
        ctx = xt.Context(local, torch.cuda.current_stream().cuda_stream)
        ctx.load(w)
        prec = {"fp32": xt.XT_PREC_FP32_IR, "tf32": xt.XT_PREC_TF32_IR, "bf16": xt.XT_PREC_BF16_IR, "fp64": xt.XT_PREC_FP64}[args.nlte_precision]
        st = xt.solve_nlte(ctx.h, w.upsilon, precision=prec, rates=xt.XT_RATES_JBAR,
                           jbar_W=w.jbar_W, jbar_TR=w.jbar_TR, levels_used=w.levels_used)
        ctx.close()
        print(json.dumps({"nlte_once": st}), flush=True)
        return
    if args.only_nlte:
        if rank == 0:
            print(json.dumps({"nlte": nlte_bench(local, torch.cuda.current_stream().cuda_stream,
                                                 args.nlte_n)}), flush=True)
        return
    if args.only_cfg5:
        if rank == 0:
            print(json.dumps({"cfg5": cfg5_bench(local, torch.cuda.current_stream().cuda_stream)}),
                  flush=True)
        return
    if args.only_paper_rays:
        if rank == 0:
            print(json.dumps({"paper_rays": paper_rays_bench(local, torch.cuda.current_stream().cuda_stream)}),
                  flush=True)
        return
    if args.only_cfg5_loop:
        if rank == 0:
            print(json.dumps({"cfg5_loop": cfg5_loop_bench(local, torch.cuda.current_stream().cuda_stream)}),
                  flush=True)
        return
    if args.only_sph:
        if rank == 0:
            print(json.dumps({"spherical": sph_bench(local, torch.cuda.current_stream().cuda_stream,
                                                     n_packets=args.sph_packets)}), flush=True)
        return
    if args.only_scatter:
        if rank == 0:
            print(json.dumps({"scatter_rates": scatter_rates_bench(
                local, torch.cuda.current_stream().cuda_stream)}), flush=True)
        return
    if args.only_train:
        if rank == 0:
            print(json.dumps({"train": train_bench(local, torch.cuda.current_stream().cuda_stream,
                                                   args.train_epochs)}), flush=True)
        return
    if args.only_coupled:
        if rank == 0:
            print(json.dumps({"coupled": coupled_bench(local, torch.cuda.current_stream().cuda_stream,
                                                       args.coupled_n)}), flush=True)
        return

    w = make_workload(args)
    stream = torch.cuda.current_stream()
    ctx = xt.Context(local, stream.cuda_stream)
    ctx.load(w)
    # each rank transports its own replica of the emission (independent packets)
    seed = replica_seed(w.seed, rank)
    kw = dict(seed=seed)

    for _ in range(args.warmup):
        ctx.transport(w, **kw)
    torch.cuda.synchronize()
    barrier()
    stats = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(ctx.transport(w, **kw))
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    ev = sum(s["events"] for s in stats)
    kern_ms = float(np.mean([s["transport_ms"] for s in stats]))
    zero_ms = float(np.mean([s["zero_ms"] for s in stats]))
    emit_ms = float(np.mean([s["emit_ms"] for s in stats]))
    trace_ms = float(np.mean([s["trace_ms"] for s in stats]))
    escape_ms = float(np.mean([s["escape_ms"] for s in stats]))
    trace_launches = float(np.mean([s["rounds"] for s in stats]))
    ms_max, ev_all = reduce_over_ranks(ms, ev, dist)
    launches = int(sum(s["kernels"] for s in stats))
    value = ev_all / (ms_max * 1e-3)

    # the same pass with every subdomain a domain of its own (Sec. 2.4.1 bundles)
    rounds = None
    if args.rounds_steps > 0:
        ctx.transport(w, subdomain_rounds=True, **kw)
        rs = []
        for _ in range(args.rounds_steps):
            r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            st_r = ctx.transport(w, subdomain_rounds=True, **kw)
            r1.record(stream)
            torch.cuda.synchronize()
            rs.append(r0.elapsed_time(r1))
        rounds = {"value": st_r["events"] / (min(rs) * 1e-3), "unit": UNIT,
                  "ms_per_step": min(rs), "rounds": st_r["rounds"], "queued": st_r["queued"],
                  "subdomains": list(w.subdomains)}

    # end to end through the public API with host buffers: upload every input
    # from pinned host memory, transport, read the spectrum back
    e2e_ms = []
    h2d = d2h = 0
    ev_e2e = 0.0
    spec = np.zeros(1)
    wp = _pinned_inputs(w) if args.e2e_steps > 0 else w
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.load(wp)                    # host arrays -> device (grid, atoms, populations)
        st = ctx.transport(wp, **kw)
        spec = ctx.get_spectrum(0)      # device -> host
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        ev_e2e = st["events"]
    h2d = sum(getattr(wp, k).nbytes for k in E2E_INPUTS if getattr(wp, k) is not None)
    d2h = spec.nbytes + 18 * 8
    e2e_val = ev_e2e / (min(e2e_ms) * 1e-3) if e2e_ms else None

    peaks, src = _measured_peaks()
    # dominant kernel: the trace loop; its device time per launch from CUDA
    # events on the launching stream inside the library
    achieved = BYTES_PER_EVENT * (ev / len(stats)) / (trace_ms * 1e-3) / 1e9
    # the FP64 pipe beside it: thread instructions per second against the
    # pipe's lane rate at the maximum SM clock
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp64_peak = FP64_LANES_PER_SM_CYCLE * sms * peaks.get("sm_max_mhz", 2070.0) * 1e6
    fp64_ach = TRACE_FP64_OPS_PER_EVENT * (ev / len(stats)) / (trace_ms * 1e-3)
    # a second view: the per-packet bytes of the fused pass beside the events'
    wp_b = BYTES_PER_EVENT * (ev / len(stats)) + BYTES_PER_PACKET * w.n_packets
    with_packets = {"bytes_per_event": BYTES_PER_EVENT, "bytes_per_packet": BYTES_PER_PACKET,
                    "achieved": wp_b / (trace_ms * 1e-3) / 1e9,
                    "frac": wp_b / (trace_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
    fp64 = {"ops_per_event": TRACE_FP64_OPS_PER_EVENT, "achieved": fp64_ach, "peak": fp64_peak,
            "unit": "FP64 thread instructions/s", "frac": fp64_ach / fp64_peak,
            "pipe_busy_ncu": TRACE_FP64_PIPE_BUSY,
            "source": "ops per event and pipe busy from ncu on the 32^3 onion; peak = 2 lanes "
                      "x SMs x max SM clock"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, world),
        "events_per_step": ev / len(stats),
        "tests_per_step": float(np.mean([s["tests"] for s in stats])),
        "packets_per_s": w.n_packets * world / (ms_max * 1e-3 / args.steps),
        "pass_device_ms": kern_ms, "store_clear_ms": zero_ms, "emit_ms": emit_ms,
        "trace_ms": trace_ms, "escape_ms": escape_ms, "trace_launches_per_pass": trace_launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                     "traffic": TRACE_DRAM_BYTES_PER_EVENT * ev / len(stats),
                     "traffic_source": "ncu dram bytes per event on the 32^3 onion, scaled by events",
                     "peak_source": src, "kernel": "k_trace",
                     "bytes_per_unit": BYTES_PER_EVENT, "unit_counted": "event",
                     "fp64": fp64, "with_packets": with_packets},
        "clocks": clk.summary(),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": min(e2e_ms) if e2e_ms else None},
        "subdomain_rounds": rounds,
        "gpu_launches": launches,
    }
    ctx.close()
    if rank == 0 and not args.no_thin and args.workload == "onion":
        line["thin_lines"] = thin_bench(local, stream.cuda_stream)
    if rank == 0 and not args.no_rays and args.workload == "onion":
        line["rays"] = rays_bench(local, stream.cuda_stream)
    if rank == 0 and not args.no_sph and args.workload == "onion":
        line["spherical"] = sph_bench(local, stream.cuda_stream, n_packets=args.sph_packets)
    if rank == 0 and args.prereduce and args.workload == "onion":
        line["prereduce"] = prereduce_bench(local, stream.cuda_stream, w)
    if rank == 0 and not args.no_nlte and args.workload == "onion":
        line["nlte"] = nlte_bench(local, stream.cuda_stream, args.nlte_n)
    if rank == 0 and not args.no_coupled and args.workload == "onion":
        line["coupled"] = coupled_bench(local, stream.cuda_stream, args.coupled_n)
    if rank == 0 and not args.no_stream and args.workload == "onion":
        line["stream"] = stream_bench(local, stream.cuda_stream)
    if rank == 0 and not args.no_scatter and args.workload == "onion":
        line["scatter_rates"] = scatter_rates_bench(local, stream.cuda_stream)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
