"""Oracle for the statistical-equilibrium (NLTE level population) solve.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): used by tests, the smoke
check and the benchmark's CPU baseline, never by the product path.

For one ion in one cell, with L levels (Sec. 2.2: level populations from the
rates between all levels, with photoexcitation rates from the radiative
transfer held fixed; Sec. 2.3.2: photodeexcitation from detailed balance):

  rates i -> j (per atom, s^-1), P[i, j]:
    radiative decay     u -> l : A_ul beta_S(tau_ul)          (Eq. beta_Sobolev)
    photoexcitation     l -> u : R_lu from the estimators, or beta_S B_lu J_ext for a
                                 given external field J_ext (reading: the part of an
                                 outside field a Sobolev region absorbs, the quantity
                                 the Sec. 2.3.2 estimator counts, 1 - e^-tau per photon)
    stimulated emission u -> l : R_ul = (g_l / g_u) R_lu
    collisions (every pair)    : C_ul = 8.629e-6 Upsilon n_e / (g_u sqrt(Te)),
                                 C_lu = C_ul (g_u / g_l) exp(-(E_u - E_l) / k Te)
    non-thermal excitation 0 -> u : eta D Upsilon_0u / (n_z sum_u' Upsilon_0u' dE_0u')
  equilibrium: sum_j n_j P[j, i] - n_i sum_j P[i, j] = 0 for every level i,
  with the equation of level 0 replaced by sum_i n_i = n_z.

The system is solved with LAPACK (numpy.linalg.solve) in FP64.  The
collisional and non-thermal forms are the documented stand-ins for the
paper's SUMO collision data and Spencer-Fano deposition (readings Q11).
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 2.99792458e10
H_PLANCK = 6.62607015e-27
K_BOLTZ = 1.380649e-16
PI_E2_MC = np.pi * 4.80320471e-10 ** 2 / (9.1093837015e-28 * 2.99792458e10)
EIGHT_PI2_E2_MC = 8.0 * np.pi ** 2 * 4.80320471e-10 ** 2 / (9.1093837015e-28 * 2.99792458e10)
CCOLL = 8.629e-6


def einstein_A(lam_cm, g_l, g_u, f_lu):
    """A_ul = 8 pi^2 e^2 / (m_e c lambda^2) (g_l/g_u) f_lu."""
    return EIGHT_PI2_E2_MC / (lam_cm * lam_cm) * (g_l / g_u) * f_lu


def sobolev_tau(lam_cm, f_lu, g_l, g_u, n_l, n_u, t):
    """Eq. (tau_Sobolev) in its oscillator-strength form."""
    return PI_E2_MC * f_lu * lam_cm * t * (n_l - (g_l / g_u) * n_u)


def sobolev_beta(tau):
    """Eq. (beta_Sobolev) for tau > 0; 1 for tau <= 0 (no trapping)."""
    tau = np.asarray(tau, dtype=np.float64)
    out = np.ones_like(tau)
    pos = tau > 0
    out[pos] = -np.expm1(-tau[pos]) / tau[pos]
    return out


def planck_nu(nu, T):
    x = H_PLANCK * nu / (K_BOLTZ * T)
    return 2.0 * H_PLANCK * nu ** 3 / C_LIGHT ** 2 / np.expm1(x)


def rate_matrix(E, g, lo, up, lam_A, f_lu, ups, Te, ne, n_z, dep, t, pops_beta,
                R_lu=None, jbar=None, eta=0.5):
    """Rates P[i, j] (i -> j) of one ion with L = len(E) levels.

    lo, up index this ion's levels; ups is the [L, L] Upsilon matrix (entry
    [l, u], l < u).  beta comes from pops_beta (the populations the optical
    depths are evaluated with).  R_lu is given per line, or computed as B_lu
    jbar(nu) when jbar (a function of frequency) is given."""
    L = E.shape[0]
    P = np.zeros((L, L))
    lam = lam_A * 1e-8
    nu = C_LIGHT / lam
    gl, gu = g[lo], g[up]
    A = einstein_A(lam, gl, gu, f_lu)
    tau = sobolev_tau(lam, f_lu, gl, gu, pops_beta[lo], pops_beta[up], t)
    beta = sobolev_beta(tau)
    if R_lu is None:
        R_lu = np.zeros_like(lam) if jbar is None else beta * 4.0 * np.pi * PI_E2_MC * f_lu / (H_PLANCK * nu) * jbar(nu)
    R_ul = (gl / gu) * R_lu
    np.add.at(P, (up, lo), A * beta + R_ul)
    np.add.at(P, (lo, up), R_lu)
    iu = np.triu_indices(L, 1)
    Y = ups[iu]
    l_, u_ = iu
    C_ul = CCOLL * Y * ne / (g[u_] * np.sqrt(Te))
    C_lu = C_ul * (g[u_] / g[l_]) * np.exp(-(E[u_] - E[l_]) / (K_BOLTZ * Te))
    P[u_, l_] += C_ul
    P[l_, u_] += C_lu
    if dep > 0 and n_z > 0 and L > 1:
        Y0 = ups[0, 1:]
        denom = n_z * np.sum(Y0 * (E[1:] - E[0]))
        if denom > 0:
            P[0, 1:] += eta * dep * Y0 / denom
    return P


def se_system(P, n_z):
    """Matrix and right-hand side of statistical equilibrium, equation of level 0
    replaced by the number conservation sum n = n_z."""
    L = P.shape[0]
    M = P.T.copy()
    np.fill_diagonal(M, 0.0)
    M[np.arange(L), np.arange(L)] = -P.sum(axis=1) + np.diag(P)
    M[0, :] = 1.0
    b = np.zeros(L)
    b[0] = n_z
    return M, b


def solve_se(P, n_z):
    M, b = se_system(P, n_z)
    return np.linalg.solve(M, b)


def lte(E, g, Te, n_z):
    w = g * np.exp(-(E - E[0]) / (K_BOLTZ * Te))
    return n_z * w / w.sum()


def ion_view(w, z, L=None):
    """Levels, lines and collision strengths of ion z (first L levels)."""
    a, b = int(w.level_off[z]), int(w.level_off[z + 1])
    L = b - a if L is None else int(L)
    sel = (w.lo >= a) & (w.up < a + L) & (w.up >= a)
    return dict(E=w.E_level[a:a + L], g=w.g_level[a:a + L], lo=w.lo[sel] - a, up=w.up[sel] - a,
                lam=w.lambda_A[sel], f=w.f_lu[sel], line_index=np.nonzero(sel)[0],
                ups=w.upsilon[z][:L, :L], off=a, L=L)


def system(w, c, z, pops_beta=None, R_lu_lines=None, eta=0.5):
    """Rates P and the equilibrium populations of ion z in cell c.

    L = w.levels_used[c, z] when given.  beta from pops_beta (default: the
    workload's populations).  Photoexcitation from R_lu_lines (per workload
    line, e.g. from the estimators) or from the workload's Jbar model."""
    L = None if w.levels_used is None else int(w.levels_used[c, z])
    v = ion_view(w, z, L)
    pb = (w.pops[c] if pops_beta is None else pops_beta)[v["off"]:v["off"] + v["L"]]
    jbar = None
    R = None
    if R_lu_lines is not None:
        R = R_lu_lines[v["line_index"]]
    elif w.jbar_W > 0:
        jbar = lambda nu: w.jbar_W * planck_nu(nu, w.jbar_TR)
    n_z = float(w.n_ion_density[c, z])
    P = rate_matrix(v["E"], v["g"], v["lo"], v["up"], v["lam"], v["f"], v["ups"], float(w.Te[c]),
                    float(w.ne[c]), n_z, float(w.deposition[c]), w.t, pb, R_lu=R, jbar=jbar,
                    eta=eta)
    return P, n_z, v



def sobolev_beta_deriv(tau):
    """d beta_S / d tau = (tau e^-tau - (1 - e^-tau)) / tau^2 for tau > 0, with
    the limit -1/2 as tau -> 0+; 0 for tau <= 0, where beta_S = 1."""
    tau = np.asarray(tau, dtype=np.float64)
    out = np.zeros_like(tau)
    pos = tau > 1e-8
    out[pos] = (tau[pos] * np.exp(-tau[pos]) + np.expm1(-tau[pos])) / tau[pos] ** 2
    out[(tau > 0) & ~pos] = -0.5
    return out


def newton_damping(it):
    """Damping of Newton step it (0-based), Sec. 2.2."""
    return 0.95 if it < 10 else 0.75 if it < 35 else 0.5 if it < 50 else 0.25 if it < 90 else 0.05


def newton_se(w, c, z, n0=None, R_lu_lines=None, tol=1e-6, max_iter=150, max_var=10.0,
              floor=1e-30, eta=0.5):
    """Populations of ion z in cell c that are consistent with their own Sobolev
    optical depths (Sec. 2.2: Newton-Raphson on the rate equations with the
    photoexcitation rates of the transport held fixed per atom).

    G(n) = M(beta(n)) n - b.  The Jacobian is M plus, for every line, the
    derivative of its net downward flow F = A beta n_u - beta B_lu J_ext
    (n_l - g_l/g_u n_u) through beta (J_ext: the external-field model; with
    estimator rates R_lu is fixed per atom and only A beta n_u depends on
    beta): dF/dn_l = beta' K (A n_u - B_lu J_ext net), dF/dn_u = -g_l/g_u times
    that; F enters row l with +, row u with - (row 0 is sum n = n_z).

    With d = J^-1 (-G) and r = max |d_i| / n_i over the levels with
    n_i >= floor n_z: stop when r <= tol; otherwise every level moves by the
    factor 1 + lam d_i / n_i, kept within [1/max_var, max_var] (Sec. 2.2 bounds
    the variation of the populations between two steps; readings: a factor 10,
    which also keeps them positive), lam = 1 once r <= 0.1 and the damping of
    the step before that (Sec. 2.2: 0.95, then 0.75, 0.5, 0.25 and 0.05 from
    steps 10, 35, 50 and 90 on).  Returns (n, steps); steps = -1 when max_iter
    ran out."""
    L = None if w.levels_used is None else int(w.levels_used[c, z])
    v = ion_view(w, z, L)
    L = v["L"]
    off = v["off"]
    n = (w.pops[c][off:off + L] if n0 is None else np.asarray(n0, dtype=np.float64)).copy()
    lo, up, g = v["lo"], v["up"], v["g"]
    lam_cm = v["lam"] * 1e-8
    A = einstein_A(lam_cm, g[lo], g[up], v["f"])
    K = PI_E2_MC * v["f"] * lam_cm * w.t
    gr = g[lo] / g[up]
    BJ = np.zeros_like(A)
    if R_lu_lines is None and w.jbar_W > 0:
        nu = C_LIGHT / lam_cm
        BJ = 4.0 * np.pi * PI_E2_MC * v["f"] / (H_PLANCK * nu) * w.jbar_W * planck_nu(nu, w.jbar_TR)
    n_z = float(w.n_ion_density[c, z])
    n = np.maximum(n, 1e-280 * n_z)
    for it in range(max_iter):
        pops = w.pops[c].copy()
        pops[off:off + L] = n
        P, n_z, _ = system(w, c, z, pops_beta=pops, R_lu_lines=R_lu_lines, eta=eta)
        M, b = se_system(P, n_z)
        G = M @ n - b
        J = M.copy()
        net = n[lo] - gr * n[up]
        t = sobolev_beta_deriv(K * net) * K * (A * n[up] - BJ * net)
        for k in range(lo.shape[0]):
            l, u = lo[k], up[k]
            if l != 0:
                J[l, l] += t[k]
                J[l, u] -= gr[k] * t[k]
            if u != 0:
                J[u, l] -= t[k]
                J[u, u] += gr[k] * t[k]
        d = np.linalg.solve(J, -G)
        sig = n >= floor * n_z
        r = float(np.max(np.abs(d[sig]) / n[sig])) if sig.any() else 0.0
        lam = 1.0 if r <= 0.1 else newton_damping(it)
        n = n * np.clip(1.0 + lam * d / n, 1.0 / max_var, max_var)
        if r <= tol:
            return n, it + 1
    return n, -1
