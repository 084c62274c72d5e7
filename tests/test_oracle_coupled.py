"""Pins of the oracle's Newton solve on the optical depths and of the coupled
NLTE / transport loop (CPU only)."""
import numpy as np
from scipy.optimize import brentq

import synth
from oracle import coupled, nlte

EV = 1.602176634e-12


def _two_level(f, n=4, n_packets=2000, seed=0):
    w = synth.uniform_sphere(seed=seed, n=n, n_packets=n_packets, n_lines=1, n_levels=2,
                             f_range=(f, f))
    w.upsilon = synth.collision_strengths(seed, w.level_off)
    return w


def _two_level_rates(w, c):
    """Collisional and non-thermal rates of the two-level ion in cell c, written
    out from their definitions (Sec. 2.2 rate terms)."""
    g0, g1 = w.g_level
    dE = w.E_level[1] - w.E_level[0]
    Te, ne, nz = w.Te[c], w.ne[c], w.n_ion_density[c, 0]
    ups = w.upsilon[0][0, 1]
    C10 = 8.629e-6 * ups * ne / (g1 * np.sqrt(Te))
    C01 = C10 * (g1 / g0) * np.exp(-dE / (1.380649e-16 * Te))
    NT = 0.5 * w.deposition[c] / (nz * dE)          # eta D Upsilon_01 / (n_z Upsilon_01 dE)
    lam = w.lambda_A[0] * 1e-8
    A = 8 * np.pi ** 2 * 4.80320471e-10 ** 2 / (9.1093837015e-28 * 2.99792458e10 * lam ** 2) * (g0 / g1) * w.f_lu[0]
    K = np.pi * 4.80320471e-10 ** 2 / (9.1093837015e-28 * 2.99792458e10) * w.f_lu[0] * lam * w.t
    return C10, C01, NT, A, K, g0, g1, nz


def test_thin_two_level_loop_is_the_closed_form():
    """Lines far below tau_min: no photoexcitation, beta_S -> 1, and the loop's
    populations are the two-level balance n1/n0 = (C01 + NT) / (C10 + A)."""
    w = _two_level(1e-14)
    n, steps, hist = coupled.coupled_loop(w, tol=1e-9, newton=True)
    assert steps > 0, hist
    for c in np.nonzero(w.rho > 0)[0][::5]:
        C10, C01, NT, A, K, g0, g1, nz = _two_level_rates(w, c)
        r = (C01 + NT) / (C10 + A)
        np.testing.assert_allclose(n[c], [nz / (1 + r), nz * r / (1 + r)], rtol=1e-8)


def test_thick_two_level_newton_is_the_scalar_root():
    """An optically thick line with no photoexcitation: the populations solve the
    scalar balance n1 (A beta_S(tau(n)) + C10) = n0 (C01 + NT), n0 + n1 = n_z,
    tau = K (n0 - g0/g1 n1); found here by bracketing (Brent), independent of
    the Newton iteration and its Jacobian."""
    w = _two_level(0.5)
    R0 = np.zeros(w.nline)
    for c in np.nonzero(w.rho > 0)[0][::50]:
        C10, C01, NT, A, K, g0, g1, nz = _two_level_rates(w, c)

        def f(x):
            tau = K * ((nz - x) - g0 / g1 * x)
            beta = -np.expm1(-tau) / tau if tau > 0 else 1.0
            return x * (A * beta + C10) - (nz - x) * (C01 + NT)
        x = brentq(f, 0.0, nz * g1 / (g0 + g1) * (1 - 1e-12), xtol=1e-300, rtol=1e-14)
        n, steps = nlte.newton_se(w, c, 0, R_lu_lines=R0, tol=1e-12)
        assert steps > 0
        assert K * (n[0] - g0 / g1 * n[1]) > 1e3          # the line is thick
        np.testing.assert_allclose(n, [nz - x, x], rtol=1e-9)


def test_newton_matches_the_lagged_linear_solve_at_its_fixed_point():
    """At the Newton solution, the linear solve with beta_S from the solution
    returns the solution (estimator-like rates fixed per atom)."""
    w = synth.nlte_batch(n=2, seed=7, L_range=(20, 40))
    for c, z in ((0, 0), (3, 4), (7, 9)):
        n, steps = nlte.newton_se(w, c, z, tol=1e-12)
        assert steps > 0
        pops = w.pops[c].copy()
        L = int(w.levels_used[c, z])
        off = int(w.level_off[z])
        pops[off:off + L] = n
        P, nz, _ = nlte.system(w, c, z, pops_beta=pops)
        np.testing.assert_allclose(nlte.solve_se(P, nz), n, rtol=1e-8)


def test_coupled_loop_converges_to_a_fixed_point():
    """The loop on the 16^3-sphere ion (small packet count): converged, and one
    more outer step moves no population by more than the tolerance."""
    w = synth.uniform_sphere(seed=2, n=6, n_packets=20_000)
    w.upsilon = synth.collision_strengths(2, w.level_off)
    n, steps, hist = coupled.coupled_loop(w, tol=1e-4, newton=True)
    assert steps > 0, hist
    import copy
    w2 = copy.copy(w)
    w2.pops = n
    n2, _ = coupled.outer_step(w2)
    assert coupled.max_change(n, n2, w2, 1e-20) <= 1e-4


def test_relax_and_change():
    old = np.array([[1.0, 4.0, 0.0]])
    new = np.array([[4.0, 1.0, 2.0]])
    np.testing.assert_allclose(coupled.relax(old, new, 0.5), [[2.0, 2.0, 2.0]])
    assert np.array_equal(coupled.relax(old, new, 1.0), new)
