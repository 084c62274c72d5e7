"""CPU oracle for the photoexcitation-rate transport and the rate solves.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The product path (the
CUDA library and its Python binding) never imports, links or executes it, and
the oracle imports nothing from the product.  The two share no code: the only
common module is the seeded input generator ``synth``, which holds none of the
method's arithmetic.

Parts:
  transport.c  serial C: Philox4x64-10, Sobolev tau/beta, packet emission,
               the segment/resonance event loop (attenuation and scatter
               modes), estimators, spectrum tallies (Secs. 2, 2.3, 2.3.2,
               App. A.1).
  this file    ctypes binding; A7 rates from estimators (Sec. 2.3.2: a
               photoexcitation rate per line and cell, photodeexcitation from
               detailed balance); photoionization rates (Sec. 2.3.1);
               spectrum normalisation (Sec. 2.3).
  nlte.py      statistical-equilibrium rate matrices and their FP64 solve.
  mlp.py       FP64 MLP forward/backward/Adam for the surrogate.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

C_LIGHT = 2.99792458e10
H_PLANCK = 6.62607015e-27
PI_E2_MC = np.pi * 4.80320471e-10 ** 2 / (9.1093837015e-28 * 2.99792458e10)

LEDGER = ["emit_N", "esc_N", "abs_N", "drop_N", "emit_E", "esc_E", "oob_E", "events",
          "tests", "guard", "thermal_E", "interactions", "abs_E_cmf", "reemit_E_cmf",
          "pi_N", "pi_E"]
PKT_FIELDS = ["fate", "events", "N_final", "esc_E", "viewer", "lbin", "interactions", "cell",
              "N0", "nu_cmf0", "nu_lab"]


def build(force: bool = False) -> str:
    """Compile transport.c with gcc (no FMA contraction) into oracle/_build."""
    src = os.path.join(_HERE, "transport.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Problem(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("v_max", C.c_double), ("t", C.c_double),
                ("L_cell", C.c_void_p), ("band_lo_A", C.c_double), ("band_hi_A", C.c_double),
                ("nlev", C.c_int32), ("nline", C.c_int32),
                ("g", C.c_void_p), ("E_level", C.c_void_p), ("pops", C.c_void_p),
                ("lo", C.c_void_p), ("up", C.c_void_p),
                ("lambda_A", C.c_void_p), ("f_lu", C.c_void_p),
                ("ne", C.c_void_p), ("Te", C.c_void_p), ("ups_down", C.c_void_p),
                ("geometry", C.c_int32), ("r_edges", C.c_void_p), ("th_edges", C.c_void_p),
                ("ph_edges", C.c_void_p),
                ("n_pi", C.c_int32), ("pi_level", C.c_void_p), ("pi_Eion", C.c_void_p),
                ("pi_charge", C.c_void_p)]


class _Params(C.Structure):
    _fields_ = [("n_packets", C.c_int64), ("p_begin", C.c_int64), ("p_end", C.c_int64),
                ("seed", C.c_uint64), ("mode", C.c_int32), ("emission_mode", C.c_int32),
                ("tau_min", C.c_double), ("e_cut", C.c_double),
                ("n_theta", C.c_int32), ("n_phi", C.c_int32),
                ("spec_lam0_A", C.c_double), ("spec_dlog", C.c_double),
                ("spec_nbins", C.c_int32), ("max_events", C.c_int64), ("sampler", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d = C.c_double
        _lib.xo_tau_sobolev.restype = d
        _lib.xo_tau_sobolev.argtypes = [d] * 7
        _lib.xo_beta_sobolev.restype = d
        _lib.xo_beta_sobolev.argtypes = [d]
        _lib.xo_einstein_A.restype = d
        _lib.xo_einstein_A.argtypes = [d] * 4
        _lib.xo_viewer_bin.restype = C.c_int32
        _lib.xo_viewer_bin.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
        _lib.xo_lambda_bin.restype = C.c_int64
        _lib.xo_lambda_bin.argtypes = [d, d, d, C.c_int32]
        _lib.xo_nu_cmf.restype = d
        _lib.xo_nu_cmf.argtypes = [d, C.c_void_p, C.c_void_p, d, d]
        _lib.xo_transport.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                      C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.xo_sigma_pi.restype = d
        _lib.xo_sigma_pi.argtypes = [d, d, d, C.c_int32]
        _lib.xo_emission.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.xo_transport_domain.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                             C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.xo_cell_volumes.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.xo_ray_count.restype = C.c_int64
        _lib.xo_ray_count.argtypes = [C.c_void_p, C.c_void_p]
        _lib.xo_sph_walk.restype = C.c_int64
        _lib.xo_sph_walk.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_int64, C.c_void_p, C.c_void_p]
        _lib.xo_tau_beta.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]
        _lib.xo_packet_quota.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p]
        _lib.xo_philox4x64_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ci32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class _Keep:
    """Holds the arrays a _Problem points at for the lifetime of a call."""

    def __init__(self, w, ups_down=None):
        self.arrs = dict(L=_c64(w.L_cell), g=_c64(w.g_level), E=_c64(w.E_level),
                         pops=_c64(w.pops), lo=_ci32(w.lo), up=_ci32(w.up),
                         lam=_c64(w.lambda_A), f=_c64(w.f_lu), ne=_c64(w.ne), Te=_c64(w.Te),
                         ups=_c64(ups_down if ups_down is not None else np.zeros(w.nlev)))
        a = self.arrs
        self.sph = getattr(w, "geometry", "cartesian") == "spherical"
        if self.sph:
            a.update(re=_c64(w.r_edges), te=_c64(w.theta_edges), pe=_c64(w.phi_edges))
        self.n_pi = 0
        if getattr(w, "pi_nlev", None) is not None:
            import synth
            lev, eion, ch = synth.pi_levels(w)
            a.update(pi_lev=_ci32(lev), pi_eion=_c64(eion), pi_ch=_ci32(ch))
            self.n_pi = int(lev.shape[0])
        self.pb = _Problem(w.nx, w.ny, w.nz, w.v_max, w.t, _ptr(a["L"]), w.band_A[0],
                           w.band_A[1], w.nlev, w.nline, _ptr(a["g"]), _ptr(a["E"]),
                           _ptr(a["pops"]), _ptr(a["lo"]), _ptr(a["up"]), _ptr(a["lam"]),
                           _ptr(a["f"]), _ptr(a["ne"]), _ptr(a["Te"]), _ptr(a["ups"]),
                           1 if self.sph else 0, _ptr(a.get("re")), _ptr(a.get("te")), _ptr(a.get("pe")),
                           self.n_pi, _ptr(a.get("pi_lev")), _ptr(a.get("pi_eion")),
                           _ptr(a.get("pi_ch")))


def upsilon_down_sums(w) -> np.ndarray:
    """sum_{j<u} Upsilon_ju for every level (collisional de-excitation weight)."""
    import synth
    out = np.zeros(w.nlev)
    for z, ups in enumerate(synth.collision_strengths(w.upsilon_seed, w.level_off)):
        out[w.level_off[z]:w.level_off[z + 1]] = ups.sum(axis=0)
    return out


def _params(w, N, p_begin, p_end, seed, mode, emission, tau_min, e_cut, n_theta, n_phi, spec_dlog,
            max_events, sampler):
    lam0, nbins = w.spec_band_A
    return _Params(N, p_begin, p_end, w.seed if seed is None else seed,
                   0 if mode == "atten" else 1, 0 if emission == "band" else 1,
                   tau_min, e_cut, n_theta, n_phi, lam0, spec_dlog, nbins, max_events,
                   1 if sampler == "rays" else 0)


def sph_walk(w, p0, n, idx0, max_cells=10_000):
    """The spherical grid's walk alone (test entry): the natural indices of
    the cells a straight path from p0 (cm, inside cell idx0 = (ir, ith, iph))
    along the unit vector n crosses, and the path length at which it leaves
    each; None if the path does not leave the outer sphere within max_cells."""
    keep = _Keep(w)
    pr = _params(w, 0, 0, 0, 0, "atten", "band", 1e-4, 1e-6, 20, 20, 1e-3, 1, "mc")
    p0 = np.ascontiguousarray(p0, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    i0 = np.ascontiguousarray(idx0, dtype=np.int32)
    cells = np.zeros(max_cells, dtype=np.int64)
    s_exit = np.zeros(max_cells)
    k = lib().xo_sph_walk(C.byref(keep.pb), C.byref(pr), _ptr(p0), _ptr(n), _ptr(i0), max_cells,
                          _ptr(cells), _ptr(s_exit))
    if k < 0:
        return None
    return cells[:k], s_exit[:k]


def ray_count(w, emission="band", n_theta=20, n_phi=20, spec_dlog=1e-3):
    """Rays of the RAYS sampler: emitting cells x emitting wavelength bins x viewers."""
    keep = _Keep(w)
    pr = _params(w, 0, 0, 0, 0, "atten", emission, 1e-4, 1e-6, n_theta, n_phi, spec_dlog, 1, "rays")
    n = lib().xo_ray_count(C.byref(keep.pb), C.byref(pr))
    if n < 0:
        raise ValueError("an emitting line lies outside the output wavelength grid")
    return int(n)


def transport(w, p_begin=0, p_end=None, n_packets=None, seed=None, mode="atten",
              emission="band", tau_min=1e-4, e_cut=1e-6, n_theta=20, n_phi=20,
              spec_dlog=1e-3, max_events=1_000_000, per_packet=False, sparse=None,
              rec_cap=None, sampler="mc", estimators=True):
    """Run packets [p_begin, p_end) of the workload's emission through the grid.

    Returns S [ncell, nline] (photons/s absorbed, divided by f_corr; natural
    cell order, the workload's line order), spec [n_theta*n_phi, n_bins]
    (escaped lab-frame energy, erg/s), the photon/energy ledger and, if asked,
    per-packet records.  With ``sparse`` (default: when the dense store would
    exceed 2 GB) S is returned as summed (cell, line, value) records instead;
    estimators=False keeps no estimators (S is None; the same arithmetic
    runs, and no shared state of the C code is touched, so calls on disjoint
    packet ranges may run in parallel threads).
    A workload with photoionization data (attenuation mode) also gives S_pi
    [ncell, n_pi] (photons/s absorbed per photoionizing level) and heat
    [ncell] (erg/s of photon energy above the thresholds)."""
    if sampler == "rays":
        N = ray_count(w, emission, n_theta, n_phi, spec_dlog)
    else:
        N = w.n_packets if n_packets is None else n_packets
    p_end = N if p_end is None else p_end
    keep = _Keep(w, upsilon_down_sums(w) if mode == "scatter" else None)
    if keep.n_pi and mode != "atten":
        raise ValueError("photoionization is part of the attenuation mode only")
    if keep.sph and mode != "atten":
        raise ValueError("the spherical grid: attenuation mode")
    S_pi = np.zeros((w.ncell, keep.n_pi)) if keep.n_pi else None
    heat = np.zeros(w.ncell) if keep.n_pi else None
    lam0, nbins = w.spec_band_A
    pr = _params(w, N, p_begin, p_end, seed, mode, emission, tau_min, e_cut, n_theta, n_phi,
                 spec_dlog, max_events, sampler)
    if not estimators:
        sparse = False
    elif sparse is None:
        sparse = w.ncell * w.nline * 8 > 2e9
    S = None if (sparse or not estimators) else np.zeros((w.ncell, w.nline))
    spec = np.zeros((n_theta * n_phi, nbins))
    ledger = np.zeros(20)
    pkt = np.zeros((p_end - p_begin, len(PKT_FIELDS))) if per_packet else None
    rec = None
    nrec = np.zeros(1, dtype=np.int64)
    if sparse:
        cap = rec_cap if rec_cap is not None else max(1024, 64 * (p_end - p_begin))
        rec = np.zeros(cap, dtype=[("cell", np.int64), ("line", np.int64), ("value", np.float64)])
    rc = lib().xo_transport(C.byref(keep.pb), C.byref(pr), _ptr(S), _ptr(spec), _ptr(ledger),
                            _ptr(pkt), _ptr(rec), 0 if rec is None else rec.shape[0], _ptr(nrec),
                            _ptr(S_pi), _ptr(heat))
    if rc == -2:
        raise ValueError("an emitting line lies outside the output wavelength grid")
    if rc != 0:
        raise RuntimeError(f"oracle record buffer too small ({nrec[0]} records)")
    out = dict(S=S, spec=spec, ledger=dict(zip(LEDGER, ledger[:len(LEDGER)].tolist())), n=N)
    if keep.n_pi:
        out["S_pi"], out["heat"] = S_pi, heat
    if sparse:
        r = rec[: nrec[0]]
        key = r["cell"] * w.nline + r["line"]
        uk, inv = np.unique(key, return_inverse=True)
        val = np.zeros(uk.shape[0])
        np.add.at(val, inv, r["value"])
        out["S_slots"] = uk
        out["S_values"] = val
    if per_packet:
        out["pkt"] = pkt
    return out


STATE_FIELDS = 21          # doubles per packet state handed between domains
STATE_Z = 4                # the z index of the cell the packet entered


def transport_domain(w, z_lo, z_hi, emit, bundle_in=None, n_theta=20, n_phi=20, spec_dlog=1e-3,
                     tau_min=1e-4, e_cut=1e-6, seed=None, max_events=1_000_000, sampler="mc"):
    """One domain of a spatial decomposition (Sec. 2.4.1): the cells with z in
    [z_lo, z_hi).  With emit, the workload's packets (or, sampler="rays", its
    rays) emitted in the domain start; the packets of bundle_in (states from
    other domains, [n, STATE_FIELDS]) resume.  Returns S [ncell, nline] (only
    the domain's cells written), spec, ledger, S_pi and heat (with
    photoionization data), and the states of the packets that entered another
    domain's cells."""
    keep = _Keep(w)
    lam0, nbins = w.spec_band_A
    N = ray_count(w, "band", n_theta, n_phi, spec_dlog) if sampler == "rays" else w.n_packets
    pr = _params(w, N, 0, N, seed, "atten", "band", tau_min, e_cut, n_theta, n_phi, spec_dlog,
                 max_events, sampler)
    S = np.zeros((w.ncell, w.nline))
    spec = np.zeros((n_theta * n_phi, nbins))
    ledger = np.zeros(20)
    S_pi = np.zeros((w.ncell, keep.n_pi)) if keep.n_pi else None
    heat = np.zeros(w.ncell) if keep.n_pi else None
    bin_ = np.zeros((0, STATE_FIELDS)) if bundle_in is None else np.ascontiguousarray(bundle_in, dtype=np.float64)
    cap = max(1024, 4 * bin_.shape[0], w.n_packets // 2)
    while True:
        out = np.zeros((cap, STATE_FIELDS))
        n_out = np.zeros(1, dtype=np.int64)
        S[:] = 0.0; spec[:] = 0.0; ledger[:] = 0.0
        if S_pi is not None:
            S_pi[:] = 0.0; heat[:] = 0.0
        rc = lib().xo_transport_domain(C.byref(keep.pb), C.byref(pr), int(z_lo), int(z_hi), int(bool(emit)),
                                       _ptr(bin_), bin_.shape[0], _ptr(out), cap, _ptr(n_out), _ptr(S),
                                       _ptr(spec), _ptr(ledger), _ptr(S_pi), _ptr(heat))
        if rc == 0:
            break
        if rc == -2:
            raise ValueError("an emitting line lies outside the output wavelength grid")
        cap = int(n_out[0])
    res = dict(S=S, spec=spec, ledger=dict(zip(LEDGER, ledger[:len(LEDGER)].tolist())),
               bundle=out[: int(n_out[0])])
    if keep.n_pi:
        res["S_pi"], res["heat"] = S_pi, heat
    return res


def emission(w, n_packets=None, emission="band"):
    """Cell luminosities and the largest-remainder packet quota prefix."""
    keep = _Keep(w)
    N = w.n_packets if n_packets is None else n_packets
    pr = _Params(N, 0, 0, 0, 0, 0 if emission == "band" else 1, 1e-4, 1e-6, 20, 20, 1.0, 1e-3,
                 1, 1, 0)
    Lc = np.zeros(w.ncell)
    qoff = np.zeros(w.ncell + 1, dtype=np.int64)
    lib().xo_emission(C.byref(keep.pb), C.byref(pr), _ptr(Lc), _ptr(qoff))
    return Lc, qoff


def packet_quota(L, N):
    L = _c64(L)
    q = np.zeros(L.shape[0] + 1, dtype=np.int64)
    lib().xo_packet_quota(_ptr(L), L.shape[0], N, _ptr(q))
    return q


def tau_beta(w, c0=0, nc=None):
    """Sobolev tau and beta for cells [c0, c0+nc) x all lines (workload line order)."""
    nc = w.ncell - c0 if nc is None else nc
    keep = _Keep(w)
    tau = np.zeros((nc, w.nline))
    beta = np.zeros((nc, w.nline))
    lib().xo_tau_beta(C.byref(keep.pb), c0, nc, _ptr(tau), _ptr(beta))
    return tau, beta


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    o = np.zeros(4, dtype=np.uint64)
    lib().xo_philox4x64_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def cell_volume(w):
    """Cell volume: one number for the Cartesian cube, per cell [ncell] for the
    spherical grid ((r1^3 - r0^3)/3 (cos theta0 - cos theta1)(phi1 - phi0))."""
    if getattr(w, "geometry", "cartesian") == "spherical":
        keep = _Keep(w)
        pr = _params(w, 0, 0, 0, 0, "atten", "band", 1e-4, 1e-6, 20, 20, 1e-3, 1, "mc")
        v = np.zeros(w.ncell)
        lib().xo_cell_volumes(C.byref(keep.pb), C.byref(pr), _ptr(v))
        return v
    return (2.0 * w.v_max * w.t / w.nx) * (2.0 * w.v_max * w.t / w.ny) * (2.0 * w.v_max * w.t / w.nz)


def rates(w, S):
    """Photoexcitation rates from the estimators (A7).

    R_lu = S / (n_l V) [s^-1] (Sec. 2.3.2: photons absorbed per line and cell
    over the number of lower-level atoms, as Gamma = N_abs / N_i in Sec. 2.3.1),
    R_ul = (g_l/g_u) R_lu (photodeexcitation by detailed balance), and the mean
    intensity Jbar = R_lu / B_lu with B_lu = 4 pi (pi e^2 / m_e c) f_lu / (h nu).
    Slots with n_l = 0 give 0."""
    V = cell_volume(w)
    V = V[:, None] if np.ndim(V) else V
    n_l = w.pops[:, w.lo]
    with np.errstate(divide="ignore", invalid="ignore"):
        R_lu = np.where(n_l > 0, S / (n_l * V), 0.0)
    gr = w.g_level[w.lo] / w.g_level[w.up]
    R_ul = R_lu * gr[None, :]
    nu = C_LIGHT / (w.lambda_A * 1e-8)
    B_lu = 4.0 * np.pi * PI_E2_MC * w.f_lu / (H_PLANCK * nu)
    Jbar = R_lu / B_lu[None, :]
    return R_lu, R_ul, Jbar


def pi_rates(w, S_pi):
    """Photoionization rates Gamma_PI,i = N_abs,i / (n_i V) [s^-1] of every
    photoionizing level and cell (Sec. 2.3.1: photons absorbed by the level
    over the number of atoms in it); levels with n_i = 0 give 0."""
    import synth
    lev, _, _ = synth.pi_levels(w)
    V = cell_volume(w)
    N_i = w.pops[:, lev] * (V[:, None] if np.ndim(V) else V)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(N_i > 0, S_pi / N_i, 0.0)


def sigma_pi(lambda_cm, E_u, E_ion, charge):
    """Eq. (sigma_OTSPI), the oracle's hydrogenic cross section [cm^2]."""
    return lib().xo_sigma_pi(float(lambda_cm), float(E_u), float(E_ion), int(charge))


def spectrum_L_lambda(spec, lam0, dlog, n_theta=20, n_phi=20):
    """Isotropic-equivalent L_lambda per viewer, 4 pi / dOmega_k * E_bin / dlambda
    [erg/s/A], and the angle-summed L_lambda = sum_k E_bin / dlambda (Sec. 2.3:
    the solid angle of each viewing direction is accounted for in the output)."""
    nb = spec.shape[1]
    edges = lam0 * (1.0 + dlog) ** np.arange(nb + 1)
    dlam = np.diff(edges)
    th = np.linspace(0.0, np.pi, n_theta + 1)
    dphi = 2.0 * np.pi / n_phi
    dOm = np.repeat(dphi * (np.cos(th[:-1]) - np.cos(th[1:])), n_phi)
    L_k = 4.0 * np.pi / dOm[:, None] * spec / dlam[None, :]
    L_tot = spec.sum(axis=0) / dlam
    return L_k, L_tot, edges
