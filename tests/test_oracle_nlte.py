"""Pins of the statistical-equilibrium oracle (no GPU).

P8  3-level closed form (Cramer's rule); exact rational solve (sympy) of a
    5-level system; collisions alone give Boltzmann populations; radiative
    rates alone in a Planck field at T with thin lines give Boltzmann
    populations at T (this pins A_ul, B_lu, R_ul = (g_l/g_u) R_lu together).
"""
import numpy as np
import pytest
import sympy as sp

from oracle import nlte

K = 1.380649e-16
H = 6.62607015e-27
C = 2.99792458e10


def test_three_level_cramer():
    rng = np.random.default_rng(0)
    for _ in range(20):
        P = rng.uniform(0.1, 10.0, (3, 3)) * 10.0 ** rng.uniform(-3, 3, (3, 3))
        np.fill_diagonal(P, 0.0)
        nz = 7.0
        n = nlte.solve_se(P, nz)
        # rows 1, 2: sum_j n_j P[j,i] - n_i sum_j P[i,j] = 0 ; row 0: n0+n1+n2 = nz
        out = P.sum(axis=1)
        A = np.array([[1.0, 1.0, 1.0],
                      [P[0, 1], -out[1], P[2, 1]],
                      [P[0, 2], P[1, 2], -out[2]]])
        b = np.array([nz, 0.0, 0.0])
        D = np.linalg.det(A)
        x = []
        for k in range(3):
            Ak = A.copy()
            Ak[:, k] = b
            x.append(np.linalg.det(Ak) / D)
        np.testing.assert_allclose(n, x, rtol=1e-12)


def test_five_level_exact_rational():
    rng = np.random.default_rng(1)
    L = 5
    Pq = [[sp.Rational(0) if i == j else sp.Rational(int(rng.integers(1, 1000)), int(rng.integers(1, 100)))
           for j in range(L)] for i in range(L)]
    nz = sp.Rational(3)
    M = sp.zeros(L, L)
    for i in range(L):
        for j in range(L):
            if i != j:
                M[i, j] = Pq[j][i]
        M[i, i] = -sum(Pq[i][j] for j in range(L) if j != i)
    for j in range(L):
        M[0, j] = 1
    b = sp.zeros(L, 1)
    b[0] = nz
    exact = M.LUsolve(b)
    P = np.array([[float(Pq[i][j]) for j in range(L)] for i in range(L)])
    n = nlte.solve_se(P, float(nz))
    np.testing.assert_allclose(n, [float(v) for v in exact], rtol=1e-13)


def test_collisions_alone_give_boltzmann():
    rng = np.random.default_rng(2)
    L = 12
    E = np.sort(rng.uniform(0, 8, L)) * 1.602176634e-12
    E[0] = 0.0
    g = rng.integers(1, 9, L).astype(float)
    ups = np.triu(10 ** rng.uniform(-1, 1, (L, L)), 1)
    Te = 6000.0
    P = nlte.rate_matrix(E, g, np.zeros(0, int), np.zeros(0, int), np.zeros(0), np.zeros(0), ups,
                         Te, 1e7, 1e5, 0.0, 1.7e7, np.zeros(L))
    n = nlte.solve_se(P, 1e5)
    boltz = g * np.exp(-E / (K * Te))
    np.testing.assert_allclose(n, 1e5 * boltz / boltz.sum(), rtol=1e-10)


def test_thin_lines_in_planck_field_give_boltzmann():
    T = 7000.0
    lam = np.array([4000.0, 6500.0, 9000.0])         # lines 0-1, 1-2, 0-2 energies consistent
    nu = C / (lam * 1e-8)
    E = np.array([0.0, H * nu[0], H * nu[0] + H * nu[1]])
    nu02 = (E[2] - E[0]) / H
    lam[2] = C / nu02 * 1e8
    g = np.array([2.0, 4.0, 6.0])
    lo, up = np.array([0, 1, 0]), np.array([1, 2, 2])
    f = np.array([0.3, 0.1, 0.05])
    # tau = 0 (empty beta populations): beta = 1; no collisions, no deposition
    P = nlte.rate_matrix(E, g, lo, up, lam, f, np.zeros((3, 3)), T, 0.0, 1.0, 0.0, 1.7e7,
                         np.zeros(3), jbar=lambda x: nlte.planck_nu(x, T))
    n = nlte.solve_se(P, 1.0)
    boltz = g * np.exp(-E / (K * T))
    np.testing.assert_allclose(n, boltz / boltz.sum(), rtol=1e-10)



def test_external_field_absorption_closed_form():
    """Net photoexcitations per volume of an isotropic external field J_nu in a
    homologous flow: every photon that crosses the resonance is absorbed with
    probability 1 - e^-tau, and the resonance sweeps d nu / ds = nu / (c t), so
    n_l R_lu - n_u R_ul = 4 pi J_nu (1 - e^-tau) / (h c t), whatever f_lu and
    the populations (Sobolev geometry, Sec. 2.3.2 absorbed fraction)."""
    E = np.array([0.0, 3e-12])
    g = np.array([2.0, 4.0])
    lo, up = np.array([0]), np.array([1])
    ups = np.zeros((2, 2))
    t = 100 * 86400.0
    J = 3e-9
    for f, nl, nu_ in ((1e-3, 1.0, 0.1), (0.5, 1e4, 7.0), (0.2, 1e8, 1e7)):
        lam_A = np.array([6000.0])
        pops = np.array([nl, nu_])
        P = nlte.rate_matrix(E, g, lo, up, lam_A, np.array([f]), ups, 5000.0, 0.0, 1.0, 0.0, t,
                             pops, jbar=lambda nu: np.full_like(nu, J))
        tau = nlte.sobolev_tau(lam_A * 1e-8, f, 2.0, 4.0, nl, nu_, t)[0]
        A = nlte.einstein_A(lam_A * 1e-8, 2.0, 4.0, f)[0]
        net_up = nl * P[0, 1] - nu_ * (P[1, 0] - A * nlte.sobolev_beta(tau))
        expect = 4 * np.pi * J * -np.expm1(-tau) / (nlte.H_PLANCK * nlte.C_LIGHT * t)
        assert np.isclose(net_up, expect, rtol=1e-10), (f, nl, nu_, net_up, expect)
