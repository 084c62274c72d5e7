"""Oracle of the coupled NLTE / radiative-transfer loop.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

One outer step (Sec. 2: the NLTE solver and the ray tracing alternate; the
photoexcitation rates of a transport pass are held fixed while the level
populations are solved, Sec. 2.2, and feed the next pass, Sec. 2.3.2):

  1. line emission from the current populations n_k (Eq. thin_emissivity:
     A_ul dE_ul beta_S N_u per line and cell), packets through the grid with
     the same seed every step (common random numbers, so the step is a
     deterministic map of n_k);
  2. R_lu = S / (n_l V) from the estimators, R_ul by detailed balance;
  3. per cell and ion the equilibrium populations s_k with these rates and
     beta_S from n_k (lagged one step);
  4. n_{k+1} = n_k^(1 - alpha) s_k^alpha (geometric under-relaxation; the
     paper damps its own population updates, Sec. 2.2), alpha = 1 undamped.

The loop stops when max |n_{k+1} - n_k| / n_k <= tol over every level with
n >= floor * n_z in either iterate (reading: levels below 1e-20 of their ion
carry no emission or optical depth that matters and may keep falling by
orders of magnitude).
"""
from __future__ import annotations

import copy

import numpy as np

from . import nlte, rates, transport


def relax(old, new, alpha):
    """n_old^(1-alpha) n_new^alpha; where either side is 0, or alpha = 1, the new
    value."""
    out = new.copy()
    if alpha == 1.0:
        return out
    m = (old > 0) & (new > 0)
    out[m] = np.exp((1.0 - alpha) * np.log(old[m]) + alpha * np.log(new[m]))
    return out


def max_change(old, new, w, floor):
    """max |new - old| / old over levels with max(old, new) >= floor n_z."""
    nz_lev = np.zeros_like(old)
    for z in range(w.n_ion):
        a, b = int(w.level_off[z]), int(w.level_off[z + 1])
        nz_lev[:, a:b] = w.n_ion_density[:, z:z + 1]
    sig = (np.maximum(old, new) >= floor * nz_lev) & (nz_lev > 0) & (old > 0)
    if not sig.any():
        return 0.0
    return float(np.max(np.abs(new[sig] - old[sig]) / old[sig]))


def solve_all(w, R_lu, eta=0.5, newton=False, newton_tol=1e-6):
    """Equilibrium populations of every (cell, ion) with matter, photoexcitation
    R_lu [ncell, nline]; beta_S from w.pops (lagged), or, with newton, from the
    populations themselves (nlte.newton_se started at w.pops)."""
    out = np.zeros_like(w.pops)
    for c in np.nonzero(w.n_ion_density.sum(axis=1) > 0)[0]:
        for z in range(w.n_ion):
            if w.n_ion_density[c, z] <= 0:
                continue
            if newton:
                L = None if w.levels_used is None else int(w.levels_used[c, z])
                v = nlte.ion_view(w, z, L)
                n, _ = nlte.newton_se(w, c, z, R_lu_lines=R_lu[c], tol=newton_tol, eta=eta)
                out[c, v["off"]:v["off"] + v["L"]] = n
                continue
            P, n_z, v = nlte.system(w, c, z, R_lu_lines=R_lu[c], eta=eta)
            out[c, v["off"]:v["off"] + v["L"]] = nlte.solve_se(P, n_z)
    return out


def outer_step(w, n_packets=None, seed=None, alpha=1.0, eta=0.5, tau_min=1e-4, emission="band",
               newton=True, newton_tol=1e-6, sampler="mc", n_theta=20, n_phi=20, spec_dlog=1e-3):
    """One outer step from w.pops; returns (relaxed populations, solved s_k)."""
    o = transport(w, n_packets=n_packets, seed=seed, emission=emission, tau_min=tau_min,
                  sampler=sampler, n_theta=n_theta, n_phi=n_phi, spec_dlog=spec_dlog)
    R_lu = rates(w, o["S"])[0]
    s = solve_all(w, R_lu, eta=eta, newton=newton, newton_tol=newton_tol)
    return relax(w.pops, s, alpha), s


def coupled_loop(w, n_packets=None, seed=None, alpha=1.0, tol=1e-3, floor=1e-20,
                 max_outer=60, eta=0.5, tau_min=1e-4, emission="band", newton=True,
                 newton_tol=1e-6, sampler="mc", n_theta=20, n_phi=20, spec_dlog=1e-3):
    """Runs outer steps from w.pops until the change is <= tol.  Returns
    (populations, steps, history of changes); steps = -1 if max_outer ran out.
    emission="lines" with sampler="rays" is the paper's loop: the lines emit
    from the current populations (Eq. thin_emissivity), traced as the paper's
    rays (Sec. 2.3), so that a step is a smooth map of the populations."""
    w = copy.copy(w)
    hist = []
    for k in range(max_outer):
        n_new, _ = outer_step(w, n_packets, seed, alpha, eta, tau_min, emission, newton,
                              newton_tol, sampler, n_theta, n_phi, spec_dlog)
        ch = max_change(w.pops, n_new, w, floor)
        hist.append(ch)
        w.pops = n_new
        if ch <= tol:
            return w.pops, k + 1, hist
    return w.pops, -1, hist
