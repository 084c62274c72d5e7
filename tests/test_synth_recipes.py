"""The seeded input generators against the recipes they state (no GPU):
the clump field, the onion zones and shares, the normalisations, the batch of
rate systems."""
import numpy as np
import pytest

import synth

C_LIGHT = 2.99792458e10


def test_gaussian_random_field_recipe():
    """Unit variance, zero mean, correlation exp(-r^2 / (2 l^2)) along the axes
    (averaged over eight realisations: one 64^3 field with l = 4 scatters its
    lag-8 correlation by about 0.035)."""
    n, ell = 64, 4.0
    corr = {lag: [] for lag in (1, 2, 4, 8)}
    for seed in range(8):
        g = synth.gaussian_random_field(n, ell, np.random.default_rng(seed)).reshape(n, n, n)
        assert abs(g.mean()) < 1e-12 and g.std() == pytest.approx(1.0, rel=1e-12)
        for lag in corr:
            corr[lag].append(np.mean([np.mean(g * np.roll(g, lag, axis=a)) for a in range(3)]))
    for lag, tol in ((1, 0.003), (2, 0.008), (4, 0.02), (8, 0.04)):
        assert np.mean(corr[lag]) == pytest.approx(np.exp(-lag * lag / (2 * ell * ell)), abs=tol), lag


def test_clumpy_onion_recipe():
    w = synth.clumpy_onion(n=32, n_lines=2000, n_packets=1000)
    n = w.nx
    c = (np.arange(n) + 0.5) / n * 2 - 1                     # cell centres in units of v_max t
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    v = np.sqrt(x * x + y * y + z * z).reshape(-1)
    active = v <= 1.0
    assert np.array_equal(w.rho > 0, active)
    # lognormal clumps: log(rho / rho_mean) = sigma g - sigma^2 / 2 with sigma = 0.5
    lr = np.log(w.rho[active] / 1e-15)
    assert (lr + 0.125).std() == pytest.approx(0.5, rel=0.05)
    assert np.mean(w.rho[active]) / 1e-15 == pytest.approx(1.0, abs=0.08)
    np.testing.assert_allclose(w.ne[active], 1e7 * w.rho[active] / 1e-15, rtol=1e-14)
    assert w.L_cell.sum() == pytest.approx(1e40, rel=1e-12)
    np.testing.assert_allclose(w.L_cell[active] / w.rho[active],
                               (w.L_cell[active] / w.rho[active])[0], rtol=1e-12)
    # onion zones: native ions hold 97 % of the atoms of their zone
    zone = np.minimum((v / 0.25).astype(int), 3)
    ion_zone = np.array([0, 0, 0, 1, 1, 2, 2, 3, 3, 3])
    frac = w.n_ion_density[active] / w.n_ion_density[active].sum(axis=1, keepdims=True)
    for zz in range(4):
        sel = zone[active] == zz
        assert frac[sel][:, ion_zone == zz].sum(axis=1) == pytest.approx(0.97, rel=1e-12)
    # mass: sum_z n_z A_z m_u = rho
    m = (w.n_ion_density[active] * w.ion_mass_u[None, :]).sum(axis=1) * 1.66053906660e-24
    np.testing.assert_allclose(m, w.rho[active], rtol=1e-12)
    # atoms: 10 ions of 50-200 levels, lines within 1000 A - 3 um
    Ls = np.diff(w.level_off)
    assert w.n_ion == 10 and Ls.min() >= 50 and Ls.max() <= 200
    assert w.lambda_A.min() >= 1000.0 and w.lambda_A.max() <= 30000.0 and w.lambda_A.size == 2000
    assert np.all(w.lo < w.up)
    # the emission band's blue edge leaves every line its full resonance cone
    assert w.band_A[0] == pytest.approx(1000.0 / (1 + 2 * 5.0e8 / C_LIGHT), rel=1e-14)


def test_nlte_batch_recipe():
    w = synth.nlte_batch(n=8, seed=2)
    lu = w.levels_used
    assert lu.shape == (512, 10) and lu.min() >= 20 and lu.max() <= 300
    assert np.mean(lu) == pytest.approx(160, rel=0.05)         # uniform 20..300
    assert w.Te.min() >= 3000.0 and w.Te.max() <= 10000.0
    # the populations it carries are normalised per ion
    for z in range(w.n_ion):
        a, b = int(w.level_off[z]), int(w.level_off[z + 1])
        np.testing.assert_allclose(w.pops[:, a:b].sum(axis=1), w.n_ion_density[:, z], rtol=1e-12)
