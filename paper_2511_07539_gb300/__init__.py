"""GB300-native photoexcitation-rate transport (ExTraSS method, Secs. 2.3-2.4).

Thin Python binding of the C-ABI library ``libextrass.so`` (declared in
``include/extrass.h``).  The functions here only marshal arguments: every step
of the computation runs in the library's CUDA kernels.  There is no CPU
fallback; if the library has not been built, importing the binding raises.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); they are passed to the library as plain pointers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libextrass.so")

XT_OK, XT_EINVAL, XT_ENOMEM, XT_ECUDA, XT_ETIMEOUT, XT_ENOTCONV, XT_ESTATE = 0, -1, -2, -3, -4, -5, -6
XT_MODE_ATTEN, XT_MODE_SCATTER = 0, 1
XT_EMIT_BAND, XT_EMIT_LINES = 0, 1
XT_PKT_FIELDS = 11
XT_FLAG_WARP_REDUCE = 1
XT_FLAG_RAYS_STAGED = 2
XT_STORE_COMPACT_ROWS = -1
XT_SAMPLER_MC, XT_SAMPLER_RAYS = 0, 1
XT_GEOM_CARTESIAN, XT_GEOM_SPHERICAL = 0, 1
PKT_FIELDS = ["fate", "events", "N_final", "esc_E", "viewer", "lbin", "interactions", "cell",
              "N0", "nu_cmf0", "nu_lab"]


class XtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("sx", C.c_int32), ("sy", C.c_int32), ("sz", C.c_int32),
                ("v_max", C.c_double), ("t", C.c_double),
                ("rho", C.c_void_p), ("Te", C.c_void_p), ("ne", C.c_void_p),
                ("L_cell", C.c_void_p), ("deposition", C.c_void_p),
                ("band_lo_A", C.c_double), ("band_hi_A", C.c_double),
                ("geometry", C.c_int32), ("r_edges", C.c_void_p), ("theta_edges", C.c_void_p),
                ("phi_edges", C.c_void_p)]


class AtomDesc(C.Structure):
    _fields_ = [("n_ion", C.c_int32), ("nline", C.c_int32),
                ("level_off", C.c_void_p), ("E_level", C.c_void_p), ("g_level", C.c_void_p),
                ("lo", C.c_void_p), ("up", C.c_void_p), ("lambda_A", C.c_void_p),
                ("f_lu", C.c_void_p), ("n_ion_density", C.c_void_p), ("ups_down", C.c_void_p),
                ("chi_ion", C.c_void_p), ("charge", C.c_void_p), ("pi_nlev", C.c_void_p)]


class TransportParams(C.Structure):
    _fields_ = [("n_packets", C.c_int64), ("packet_begin", C.c_int64),
                ("packet_count", C.c_int64), ("seed", C.c_uint64),
                ("mode", C.c_int32), ("emission", C.c_int32),
                ("tau_min", C.c_double), ("e_cut", C.c_double),
                ("n_theta", C.c_int32), ("n_phi", C.c_int32),
                ("spec_lam0_A", C.c_double), ("spec_dlog", C.c_double),
                ("spec_nbins", C.c_int32), ("accumulate", C.c_int32),
                ("max_events", C.c_int64), ("subdomain_rounds", C.c_int32), ("flags", C.c_int32),
                ("packet_records", C.c_void_p), ("sampler", C.c_int32)]


STATS_FIELDS = ["emitted_N", "escaped_N", "absorbed_N", "dropped_N", "emitted_E", "escaped_E",
                "out_of_band_E", "events", "tests", "guard", "thermal_E", "interactions",
                "abs_E_cmf", "reemit_E_cmf", "transport_ms", "zero_ms", "rounds", "queued",
                "emit_ms", "trace_ms", "escape_ms", "kernels", "photoionized_N", "photoionized_E",
                "rays"]


class TransportStats(C.Structure):
    _fields_ = [(f, C.c_double) for f in STATS_FIELDS]

    def as_dict(self):
        return {f: getattr(self, f) for f in STATS_FIELDS}


class NoallocTransport(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("v_max", C.c_double), ("t", C.c_double), ("L_cell", C.c_void_p),
                ("band_lo_A", C.c_double), ("band_hi_A", C.c_double),
                ("nlev", C.c_int32), ("nline", C.c_int32), ("g_level", C.c_void_p),
                ("lo", C.c_void_p), ("up", C.c_void_p), ("lambda_A", C.c_void_p),
                ("f_lu", C.c_void_p), ("pops", C.c_void_p), ("n_packets", C.c_int64),
                ("seed", C.c_uint64), ("tau_min", C.c_double), ("e_cut", C.c_double),
                ("n_theta", C.c_int32), ("n_phi", C.c_int32), ("spec_lam0_A", C.c_double),
                ("spec_dlog", C.c_double), ("spec_nbins", C.c_int32), ("max_events", C.c_int64),
                ("S", C.c_void_p), ("spec", C.c_void_p)]


XT_PREC_FP64, XT_PREC_FP32_IR, XT_PREC_TF32_IR, XT_PREC_BF16_IR = 0, 1, 2, 3
XT_RATES_NONE, XT_RATES_ESTIMATORS, XT_RATES_JBAR = 0, 1, 2
XT_WARM_CURRENT, XT_WARM_LTE, XT_WARM_GIVEN = 0, 1, 2
XT_SE_OK, XT_SE_FALLBACK, XT_SE_SINGULAR, XT_SE_NOCONV = 1, 2, 4, 8
XT_WARM_SURROGATE = 3


class TrainParams(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_double),
                ("n_hidden", C.c_int32), ("n_layers", C.c_int32), ("seed", C.c_uint64),
                ("rates", C.c_int32), ("jbar_W", C.c_double), ("jbar_TR", C.c_double),
                ("levels_used", C.c_void_p)]


class TrainStats(C.Structure):
    _fields_ = [(f, C.c_double) for f in ["first_loss", "last_loss", "steps", "samples", "train_ms"]]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class NlteParams(C.Structure):
    _fields_ = [("precision", C.c_int32), ("rates", C.c_int32), ("warm", C.c_int32),
                ("max_iter", C.c_int32), ("tol", C.c_double), ("jbar_W", C.c_double),
                ("jbar_TR", C.c_double), ("eta_nt", C.c_double), ("levels_used", C.c_void_p),
                ("warm_in", C.c_void_p), ("upsilon", C.c_void_p), ("use_graph", C.c_int32),
                ("autotune", C.c_int32), ("newton_max", C.c_int32), ("newton_tol", C.c_double),
                ("newton_maxvar", C.c_double)]


NLTE_STATS = ["systems", "fp64_fallbacks", "singular", "max_iter_used", "mean_iter", "solve_ms",
              "assemble_flops", "lu_flops"]


class NlteStats(C.Structure):
    _fields_ = ([(f, C.c_double) for f in NLTE_STATS] + [("panel_width", C.c_int32 * 8)] +
                [("not_converged", C.c_double)])

    def as_dict(self):
        d = {f: getattr(self, f) for f in NLTE_STATS}
        d["panel_width"] = list(self.panel_width)
        d["not_converged"] = self.not_converged
        return d


class Sizes(C.Structure):
    _fields_ = [(f, C.c_int64) for f in
                ["ncell", "nlev", "nline", "n_ion", "spec_views", "spec_bins", "store_bytes", "n_pi"]]


_lib = None


def lib():
    """Load libextrass.so (built by __graft_entry__.build() or build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} missing "
                              "(run python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "xt_create": ([C.POINTER(vp), C.c_int, vp], C.c_int),
            "xt_destroy": ([vp], None),
            "xt_last_error": ([vp], C.c_char_p),
            "init_grid": ([vp, vp], C.c_int),
            "load_atomic_data": ([vp, vp], C.c_int),
            "set_populations": ([vp, vp], C.c_int),
            "get_populations": ([vp, vp, C.c_size_t], C.c_int),
            "get_sobolev_tau": ([vp, i64, i64, vp, vp], C.c_int),
            "run_transport": ([vp, vp, vp], C.c_int),
            "get_estimators": ([vp, i64, i64, vp], C.c_int),
            "get_photoexcitation_rates": ([vp, i64, i64, vp, vp, vp], C.c_int),
            "get_photoionization_rates": ([vp, i64, i64, vp, vp], C.c_int),
            "get_spectrum": ([vp, i32, vp, C.c_size_t], C.c_int),
            "get_sizes": ([vp, vp], C.c_int),
            "xt_selftest_fixed": ([i32, vp, i64, vp, vp, vp, vp], C.c_int),
            "xt_selftest_tc": ([C.c_int, C.c_int, vp, vp, vp], C.c_int),
            "xt_selftest_tc_bf16": ([C.c_int, C.c_int, vp, vp, vp], C.c_int),
            "run_transport_noalloc": ([vp, vp, vp, C.c_char_p, C.c_size_t], C.c_int),
            "run_transport_domain": ([vp, vp, i32, i32, i32, vp, i64, vp, i64, vp, vp], C.c_int),
            "solve_nlte": ([vp, vp, vp, vp, vp], C.c_int),
            "surrogate_init": ([vp, vp, i32, C.c_uint64], C.c_int),
            "surrogate_weights": ([vp, i32, vp, C.c_size_t], C.c_int),
            "surrogate_train_step": ([vp, vp, vp, vp, i64, C.c_double, i32, vp, vp], C.c_int),
            "surrogate_predict": ([vp, vp, i64, vp], C.c_int),
            "train_surrogate": ([vp, vp, vp], C.c_int),
            "run_coupled": ([vp, vp, vp], C.c_int),
            "set_estimator_store": ([vp, i32], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _ptr(a):
    """Plain pointer of a numpy array or torch tensor (None stays None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _check_device_f64(name, a, n):
    """`a` must be a contiguous float64 CUDA tensor of exactly n elements."""
    import torch
    if not isinstance(a, torch.Tensor) or a.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor")
    if a.dtype != torch.float64 or not a.is_contiguous():
        raise ValueError(f"{name} must be contiguous float64")
    if a.numel() != n:
        raise ValueError(f"{name} has {a.numel()} elements, {n} required")


def _check_records(rec, n):
    """Packet records: [n][XT_PKT_FIELDS] contiguous float64 (host or device)."""
    if rec is None:
        return
    if hasattr(rec, "data_ptr"):
        import torch
        ok = rec.dtype == torch.float64 and rec.is_contiguous() and rec.numel() == n * XT_PKT_FIELDS
    else:
        ok = (isinstance(rec, np.ndarray) and rec.dtype == np.float64 and rec.flags.c_contiguous
              and rec.size == n * XT_PKT_FIELDS)
    if not ok:
        raise ValueError(f"packet_records must be contiguous float64 with {n} x {XT_PKT_FIELDS} elements")


def _f64(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(ctx, rc):
    if rc != XT_OK:
        msg = lib().xt_last_error(ctx).decode() if ctx else "xt_create failed"
        raise XtError(rc, msg)


# ---- C-ABI functions under their own names ---------------------------------
def xt_create(device=0, stream=None):
    h = C.c_void_p()
    _check(None, lib().xt_create(C.byref(h), int(device), stream))
    return h


def xt_destroy(ctx):
    lib().xt_destroy(ctx)


def xt_last_error(ctx):
    return lib().xt_last_error(ctx).decode()


def init_grid(ctx, nx, ny, nz, v_max, t, Te, ne, L_cell=None, band_A=(0.0, 0.0), rho=None,
              deposition=None, subdomains=(1, 1, 1), spherical_edges=None):
    """spherical_edges = (r_edges [nx+1] cm/s, theta_edges [ny+1], phi_edges
    [nz+1] radians) selects the spherical grid; None the cube."""
    keep = [_f64(x) for x in (rho, Te, ne, L_cell, deposition)]
    geom, edges = XT_GEOM_CARTESIAN, [None, None, None]
    if spherical_edges is not None:
        geom = XT_GEOM_SPHERICAL
        edges = [_f64(e) for e in spherical_edges]
        for e, n_, what in zip(edges, (nx, ny, nz), ("r_edges", "theta_edges", "phi_edges")):
            if e.size != n_ + 1:
                raise ValueError(f"init_grid: {what} needs {n_ + 1} entries, got {e.size}")
    d = GridDesc(nx, ny, nz, *subdomains, v_max, t, *[_ptr(x) for x in keep], *band_A, geom,
                 *[_ptr(e) for e in edges])
    _check(ctx, lib().init_grid(ctx, C.byref(d)))


def load_atomic_data(ctx, level_off, E_level, g_level, lo, up, lambda_A, f_lu,
                     n_ion_density=None, ups_down=None, chi_ion=None, charge=None, pi_nlev=None):
    lo_, up_, off_ = _i32(lo), _i32(up), _i32(level_off)
    fl = [_f64(x) for x in (E_level, g_level, lambda_A, f_lu, n_ion_density, ups_down, chi_ion)]
    ch_, np_ = (_i32(charge) if charge is not None else None), (_i32(pi_nlev) if pi_nlev is not None else None)
    d = AtomDesc(len(off_) - 1, len(lo_), _ptr(off_), _ptr(fl[0]), _ptr(fl[1]), _ptr(lo_),
                 _ptr(up_), _ptr(fl[2]), _ptr(fl[3]), _ptr(fl[4]), _ptr(fl[5]), _ptr(fl[6]),
                 _ptr(ch_), _ptr(np_))
    _check(ctx, lib().load_atomic_data(ctx, C.byref(d)))


def set_populations(ctx, pops):
    p = _f64(pops)
    _check(ctx, lib().set_populations(ctx, _ptr(p)))


def get_sizes(ctx):
    s = Sizes()
    _check(ctx, lib().get_sizes(ctx, C.byref(s)))
    return {f: getattr(s, f) for f, _ in Sizes._fields_}


def get_populations(ctx, out=None):
    sz = get_sizes(ctx)
    if out is None:
        out = np.zeros((sz["ncell"], sz["nlev"]))
    _check(ctx, lib().get_populations(ctx, _ptr(out), int(np.prod(out.shape))))
    return out


def get_sobolev_tau(ctx, cell_begin=0, n_cells=None, tau=None, beta=None, want_beta=True):
    sz = get_sizes(ctx)
    n_cells = sz["ncell"] - cell_begin if n_cells is None else n_cells
    if tau is None:
        tau = np.zeros((n_cells, sz["nline"]))
    if beta is None and want_beta:
        beta = np.zeros((n_cells, sz["nline"]))
    _check(ctx, lib().get_sobolev_tau(ctx, cell_begin, n_cells, _ptr(tau), _ptr(beta)))
    return tau, beta


def set_estimator_store(ctx, host_groups=0):
    """Device-resident store (0) or a pinned host store in host_groups groups of
    subdomain z-layers, one group staged on the device at a time."""
    _check(ctx, lib().set_estimator_store(ctx, int(host_groups)))


def run_transport(ctx, n_packets, seed=0, packet_begin=0, packet_count=-1, mode=XT_MODE_ATTEN,
                  emission=XT_EMIT_BAND, tau_min=1e-4, e_cut=1e-6, n_theta=20, n_phi=20,
                  spec_lam0_A=1000.0, spec_dlog=1e-3, spec_nbins=1, accumulate=False,
                  max_events=1_000_000, subdomain_rounds=False, packet_records=None, check=True,
                  flags=0, sampler=XT_SAMPLER_MC):
    def params(count, rec):
        return TransportParams(int(n_packets), int(packet_begin), int(count), int(seed), int(mode),
                               int(emission), tau_min, e_cut, n_theta, n_phi, spec_lam0_A, spec_dlog,
                               int(spec_nbins), int(bool(accumulate)), int(max_events),
                               int(bool(subdomain_rounds)), int(flags), _ptr(rec), int(sampler))
    if packet_records is not None:
        total = int(n_packets)
        if sampler == XT_SAMPLER_RAYS and packet_count < 0:      # the number of rays first
            st0 = TransportStats()
            _check(ctx, lib().run_transport(ctx, C.byref(params(0, None)), C.byref(st0)))
            total = int(st0.rays)
        _check_records(packet_records, total - int(packet_begin) if packet_count < 0
                       else int(packet_count))
    p = params(packet_count, packet_records)
    st = TransportStats()
    rc = lib().run_transport(ctx, C.byref(p), C.byref(st))
    if check:
        _check(ctx, rc)
    return st.as_dict() if check else (rc, st.as_dict())


XT_BUNDLE_FIELDS, XT_BUNDLE_CELL = 24, 17


def run_transport_domain(ctx, z_lo, z_hi, emit, bundle_in=None, bundle_out=None, n_packets=0, seed=0,
                         tau_min=1e-4, e_cut=1e-6, n_theta=20, n_phi=20, spec_lam0_A=1000.0,
                         spec_dlog=1e-3, spec_nbins=1, accumulate=False, max_events=1_000_000,
                         flags=0, sampler=None):
    """One call of a process's domain (see include/extrass.h): returns
    (stats, n_out); the leaving packets' states are in bundle_out[:n_out]
    (a [cap, XT_BUNDLE_FIELDS] float64 array or tensor, host or device)."""
    n_in = 0 if bundle_in is None else int(bundle_in.shape[0])
    cap = 0 if bundle_out is None else int(bundle_out.shape[0])
    for name, b in (("bundle_in", bundle_in), ("bundle_out", bundle_out)):
        if b is not None and (b.ndim != 2 or b.shape[1] != XT_BUNDLE_FIELDS):
            raise ValueError(f"{name} must have shape [n, {XT_BUNDLE_FIELDS}]")
    p = TransportParams(int(n_packets), 0, -1, int(seed), XT_MODE_ATTEN, XT_EMIT_BAND, tau_min, e_cut,
                        int(n_theta), int(n_phi), spec_lam0_A, spec_dlog, int(spec_nbins),
                        int(bool(accumulate)), int(max_events), 0, int(flags), None,
                        XT_SAMPLER_MC if sampler is None else int(sampler))
    st = TransportStats()
    n_out = C.c_int64()
    rc = lib().run_transport_domain(ctx, C.byref(p), int(z_lo), int(z_hi), int(bool(emit)),
                                    _ptr(bundle_in) if n_in else None, n_in,
                                    _ptr(bundle_out) if cap else None, cap, C.byref(n_out), C.byref(st))
    if rc != XT_OK and not (rc == XT_EINVAL and n_out.value > cap):
        _check(ctx, rc)
    return st.as_dict(), int(n_out.value)


def get_estimators(ctx, cell_begin=0, n_cells=None, out=None):
    sz = get_sizes(ctx)
    n_cells = sz["ncell"] - cell_begin if n_cells is None else n_cells
    if out is None:
        out = np.zeros((n_cells, sz["nline"]))
    _check(ctx, lib().get_estimators(ctx, cell_begin, n_cells, _ptr(out)))
    return out


def get_photoexcitation_rates(ctx, cell_begin=0, n_cells=None, R_lu=None, R_ul=None, Jbar=None,
                              want=("R_lu", "R_ul", "Jbar")):
    sz = get_sizes(ctx)
    n_cells = sz["ncell"] - cell_begin if n_cells is None else n_cells
    shape = (n_cells, sz["nline"])
    if R_lu is None and "R_lu" in want:
        R_lu = np.zeros(shape)
    if R_ul is None and "R_ul" in want:
        R_ul = np.zeros(shape)
    if Jbar is None and "Jbar" in want:
        Jbar = np.zeros(shape)
    _check(ctx, lib().get_photoexcitation_rates(ctx, cell_begin, n_cells, _ptr(R_lu), _ptr(R_ul),
                                                _ptr(Jbar)))
    return R_lu, R_ul, Jbar


def get_photoionization_rates(ctx, cell_begin=0, n_cells=None, Gamma=None, heating=None,
                              want=("Gamma", "heating")):
    """Photoionization rates [n_cells, n_pi] (s^-1) and heating [n_cells] (erg/s)
    of the last attenuation pass (Sec. 2.3.1)."""
    sz = get_sizes(ctx)
    n_cells = sz["ncell"] - cell_begin if n_cells is None else n_cells
    if Gamma is None and "Gamma" in want:
        Gamma = np.zeros((n_cells, sz["n_pi"]))
    if heating is None and "heating" in want:
        heating = np.zeros(n_cells)
    _check(ctx, lib().get_photoionization_rates(ctx, cell_begin, n_cells, _ptr(Gamma), _ptr(heating)))
    return Gamma, heating


def solve_nlte(ctx, upsilon, precision=XT_PREC_FP32_IR, rates=XT_RATES_ESTIMATORS,
               warm=XT_WARM_CURRENT, max_iter=8, tol=1e-10, jbar_W=0.0, jbar_TR=0.0, eta_nt=0.5,
               levels_used=None, warm_in=None, use_graph=False, autotune=False, pops_out=None,
               status_out=None, check=True, newton_max=0, newton_tol=1e-6, newton_maxvar=10.0):
    """A8: statistical-equilibrium populations of every (cell, ion); the new
    populations replace the context's.  upsilon: per-ion [L_z, L_z] arrays (a
    list, concatenated here) or one flat array."""
    if isinstance(upsilon, (list, tuple)):
        upsilon = np.concatenate([np.ascontiguousarray(u, dtype=np.float64).ravel() for u in upsilon])
    ups = _f64(upsilon)
    lu = _i32(levels_used) if levels_used is not None else None
    wi = _f64(warm_in) if warm_in is not None else None
    p = NlteParams(int(precision), int(rates), int(warm), int(max_iter), float(tol), float(jbar_W),
                   float(jbar_TR), float(eta_nt), _ptr(lu), _ptr(wi), _ptr(ups), int(bool(use_graph)),
                   int(bool(autotune)), int(newton_max), float(newton_tol), float(newton_maxvar))
    st = NlteStats()
    rc = lib().solve_nlte(ctx, C.byref(p), _ptr(pops_out), _ptr(status_out), C.byref(st))
    if check:
        _check(ctx, rc)
        return st.as_dict()
    return rc, st.as_dict()


class CoupledParams(C.Structure):
    _fields_ = [("transport", C.c_void_p), ("nlte", C.c_void_p), ("start", C.c_int32),
                ("start_in", C.c_void_p), ("alpha", C.c_double), ("tol", C.c_double),
                ("floor", C.c_double), ("max_outer", C.c_int32)]


COUPLED_STATS = ["last_change", "wall_ms", "start_ms", "transport_ms", "solve_ms", "mix_ms",
                 "newton_steps", "max_newton_steps", "not_converged", "fp64_fallbacks"]


class CoupledStats(C.Structure):
    _fields_ = ([("outer", C.c_int32), ("converged", C.c_int32)] +
                [(f, C.c_double) for f in COUPLED_STATS] + [("change", C.c_double * 64)])

    def as_dict(self):
        d = {"outer": self.outer, "converged": bool(self.converged)}
        d.update({f: getattr(self, f) for f in COUPLED_STATS})
        d["change"] = list(self.change)[: min(self.outer, 64)]
        return d


def run_coupled(ctx, upsilon, n_packets, seed=0, start=XT_WARM_LTE, start_in=None, alpha=1.0,
                tol=1e-3, floor=1e-20, max_outer=30, precision=XT_PREC_FP32_IR, newton_max=150,
                newton_tol=1e-6, newton_maxvar=10.0, max_iter=8, ir_tol=1e-10, jbar_W=0.0,
                jbar_TR=0.0, eta_nt=0.5, levels_used=None, use_graph=False, emission=XT_EMIT_BAND,
                tau_min=1e-4, e_cut=1e-6, spec_lam0_A=1000.0, spec_dlog=1e-3, spec_nbins=1,
                max_events=1_000_000, subdomain_rounds=False, check=True, sampler=XT_SAMPLER_MC,
                n_theta=20, n_phi=20):
    """A10: the coupled loop (see include/extrass.h, run_coupled).  The paper's
    loop: emission=XT_EMIT_LINES (the lines emit from the current populations)
    with sampler=XT_SAMPLER_RAYS."""
    if isinstance(upsilon, (list, tuple)):
        upsilon = np.concatenate([np.ascontiguousarray(u, dtype=np.float64).ravel() for u in upsilon])
    ups = _f64(upsilon)
    lu = _i32(levels_used) if levels_used is not None else None
    si = _f64(start_in) if start_in is not None else None
    tp = TransportParams(int(n_packets), 0, -1, int(seed), XT_MODE_ATTEN, int(emission), tau_min, e_cut,
                         int(n_theta), int(n_phi), spec_lam0_A, spec_dlog, int(spec_nbins), 0,
                         int(max_events), int(bool(subdomain_rounds)), 0, None, int(sampler))
    np_ = NlteParams(int(precision), XT_RATES_ESTIMATORS, XT_WARM_CURRENT, int(max_iter), float(ir_tol),
                     float(jbar_W), float(jbar_TR), float(eta_nt), _ptr(lu), None, _ptr(ups),
                     int(bool(use_graph)), 0, int(newton_max), float(newton_tol), float(newton_maxvar))
    p = CoupledParams(C.addressof(tp), C.addressof(np_), int(start), _ptr(si), float(alpha), float(tol),
                      float(floor), int(max_outer))
    st = CoupledStats()
    rc = lib().run_coupled(ctx, C.byref(p), C.byref(st))
    if check:
        _check(ctx, rc)
        return st.as_dict()
    return rc, st.as_dict()


def _f32(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.float32)


def surrogate_init(ctx, sizes, seed=0):
    s = np.ascontiguousarray(sizes, dtype=np.int32)
    _check(ctx, lib().surrogate_init(ctx, _ptr(s), len(s), int(seed)))


def surrogate_weights(ctx, flat=None, n=None):
    """Set the flat FP32 weights (flat given) or return them (n floats)."""
    if flat is not None:
        f = _f32(flat)
        _check(ctx, lib().surrogate_weights(ctx, 1, _ptr(f), int(f.size)))
        return f
    out = np.zeros(n, dtype=np.float32)
    _check(ctx, lib().surrogate_weights(ctx, 0, _ptr(out), int(n)))
    return out


def surrogate_train_step(ctx, X, T, mask, lr=1e-3, update=True, n_param=None):
    X, T, mask = _f32(X), _f32(T), _f32(mask)
    grads = np.zeros(n_param, dtype=np.float32) if n_param else None
    loss = C.c_double()
    _check(ctx, lib().surrogate_train_step(ctx, _ptr(X), _ptr(T), _ptr(mask), int(X.shape[0]),
                                           float(lr), int(bool(update)), _ptr(grads), C.byref(loss)))
    return loss.value, grads


def surrogate_predict(ctx, X, n_out):
    X = _f32(X)
    Y = np.zeros((X.shape[0], n_out), dtype=np.float32)
    _check(ctx, lib().surrogate_predict(ctx, _ptr(X), int(X.shape[0]), _ptr(Y)))
    return Y


def train_surrogate(ctx, epochs=20, batch=256, lr=1e-3, n_hidden=256, n_layers=3, seed=0,
                    rates=XT_RATES_JBAR, jbar_W=0.0, jbar_TR=0.0, levels_used=None):
    lu = _i32(levels_used) if levels_used is not None else None
    p = TrainParams(int(epochs), int(batch), float(lr), int(n_hidden), int(n_layers), int(seed),
                    int(rates), float(jbar_W), float(jbar_TR), _ptr(lu))
    st = TrainStats()
    _check(ctx, lib().train_surrogate(ctx, C.byref(p), C.byref(st)))
    return st.as_dict()


def get_spectrum(ctx, kind=0, out=None):
    sz = get_sizes(ctx)
    if out is None:
        out = np.zeros(sz["spec_bins"]) if kind == 2 else np.zeros((sz["spec_views"], sz["spec_bins"]))
    _check(ctx, lib().get_spectrum(ctx, int(kind), _ptr(out), int(np.prod(out.shape))))
    return out


def xt_selftest_fixed(kind, x):
    """Device fixed-point primitives (kind 0: e^-x, 1 - e^-x; kind 1: sin, cos
    of 2 pi x) and CUDA's exp/expm1 or sin/cos beside them; kind 2: x of shape
    (n, 2), the quotient a / b and CUDA's; kind 3: x of shape (n, 2), the
    emission direction (n_x, n_y, n_z) for mu = 2u - 1, phi = 2 pi v."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    if kind >= 2 and (x.ndim != 2 or x.shape[1] != 2):
        raise ValueError("kinds 2 and 3 take pairs, shape (n, 2)")
    out = [np.zeros(n) for _ in range(4)]
    rc = lib().xt_selftest_fixed(int(kind), _ptr(x), n, *[_ptr(o) for o in out])
    if rc != XT_OK:
        raise XtError(rc, "xt_selftest_fixed failed")
    return out



def xt_selftest_tc(A, B, device=0, bf16=False):
    """D = A B^T on the tensor cores (TF32 inputs, or BF16 with bf16=True; FP32
    accumulation): A [128][32], B [N][32] float32, N a multiple of 16 in
    [16, 256]; returns D [128][N]."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    if A.shape != (128, 32) or B.ndim != 2 or B.shape[1] != 32:
        raise ValueError("xt_selftest_tc: A must be [128][32] and B [N][32]")
    D = np.zeros((128, B.shape[0]), dtype=np.float32)
    fn = lib().xt_selftest_tc_bf16 if bf16 else lib().xt_selftest_tc
    rc = fn(int(device), int(B.shape[0]), _ptr(A), _ptr(B), _ptr(D))
    if rc != XT_OK:
        raise XtError(rc, "xt_selftest_tc failed")
    return D


def xt_selftest_tc_bf16(A, B, device=0):
    """xt_selftest_tc with the operands rounded to BF16 (kind::f16)."""
    return xt_selftest_tc(A, B, device, bf16=True)

def run_transport_noalloc(nx, ny, nz, v_max, t, L_cell, band_A, g_level, lo, up, lambda_A, f_lu,
                          pops, S, spec, n_packets, seed=0, tau_min=1e-4, e_cut=1e-6, n_theta=20,
                          n_phi=20, spec_lam0_A=1000.0, spec_dlog=1e-3, spec_nbins=1,
                          max_events=1_000_000, stream=None):
    """One attenuation-mode pass that makes no device allocation (see
    include/extrass.h).  pops, S and spec must be contiguous float64 CUDA
    tensors of ncell*nlev, ncell*nline and n_theta*n_phi*spec_nbins elements;
    the library cannot check the sizes of caller buffers, so they are checked
    here (ValueError)."""
    keep = [_f64(L_cell), _f64(g_level), _i32(lo), _i32(up), _f64(lambda_A), _f64(f_lu)]
    ncell, nlev, nline = int(nx) * int(ny) * int(nz), len(keep[1]), len(keep[2])
    if len(keep[0]) != ncell:
        raise ValueError(f"L_cell has {len(keep[0])} entries, the grid {ncell} cells")
    for name, a in (("up", keep[3]), ("lambda_A", keep[4]), ("f_lu", keep[5])):
        if len(a) != nline:
            raise ValueError(f"{name} has {len(a)} entries, lo has {nline}")
    for name, a, n in (("pops", pops, ncell * nlev), ("S", S, ncell * nline),
                       ("spec", spec, int(n_theta) * int(n_phi) * int(spec_nbins))):
        _check_device_f64(name, a, n)
    a = NoallocTransport(nx, ny, nz, v_max, t, _ptr(keep[0]), band_A[0], band_A[1],
                         int(len(keep[1])), int(len(keep[2])), _ptr(keep[1]), _ptr(keep[2]),
                         _ptr(keep[3]), _ptr(keep[4]), _ptr(keep[5]), _ptr(pops), int(n_packets),
                         int(seed), tau_min, e_cut, n_theta, n_phi, spec_lam0_A, spec_dlog,
                         int(spec_nbins), int(max_events), _ptr(S), _ptr(spec))
    st = TransportStats()
    err = C.create_string_buffer(512)
    rc = lib().run_transport_noalloc(C.byref(a), stream, C.byref(st), err, 512)
    if rc != XT_OK:
        raise XtError(rc, err.value.decode())
    return st.as_dict()


# ---- convenience --------------------------------------------------------------
class Context:
    """Owns one library context; methods mirror the C-ABI calls."""

    def __init__(self, device=0, stream=None):
        self.h = xt_create(device, stream)

    def close(self):
        if self.h is not None:
            xt_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, w, subdomains=None, pops=None, with_scatter_data=None):
        """init_grid + load_atomic_data + set_populations from a workload object
        (attributes as produced by the input generator)."""
        sd = tuple(subdomains) if subdomains is not None else tuple(w.subdomains)
        edges = None
        if getattr(w, "geometry", "cartesian") == "spherical":
            edges = (w.r_edges, w.theta_edges, w.phi_edges)
        init_grid(self.h, w.nx, w.ny, w.nz, w.v_max, w.t, w.Te, w.ne, w.L_cell, w.band_A,
                  rho=w.rho, deposition=w.deposition, subdomains=sd, spherical_edges=edges)
        load_atomic_data(self.h, w.level_off, w.E_level, w.g_level, w.lo, w.up, w.lambda_A,
                         w.f_lu, n_ion_density=w.n_ion_density, ups_down=with_scatter_data,
                         chi_ion=getattr(w, "chi_ion", None), charge=getattr(w, "charge", None),
                         pi_nlev=getattr(w, "pi_nlev", None))
        set_populations(self.h, w.pops if pops is None else pops)

    def transport(self, w, **kw):
        kw.setdefault("n_packets", w.n_packets)
        kw.setdefault("seed", w.seed)
        kw.setdefault("spec_lam0_A", w.spec_band_A[0])
        kw.setdefault("spec_nbins", w.spec_band_A[1])
        return run_transport(self.h, **kw)

    def __getattr__(self, name):
        f = globals().get(name)
        if callable(f) and name in _CTX_FUNCS:
            return lambda *a, **k: f(self.h, *a, **k)
        raise AttributeError(name)


_CTX_FUNCS = {"init_grid", "load_atomic_data", "set_populations", "get_populations", "solve_nlte",
              "get_sobolev_tau", "run_transport", "get_estimators", "get_photoexcitation_rates",
              "get_spectrum", "get_sizes", "run_coupled", "set_estimator_store",
              "get_photoionization_rates"}
