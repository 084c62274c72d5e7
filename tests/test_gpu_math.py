"""The library's fixed-point device primitives against mpmath and against
CUDA's own functions (needs a GPU): e^-tau and 1 - e^-tau of every line event,
sin and cos of every emission azimuth."""
import mpmath as mp
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
EPS = 2.220446049250313e-16


@pytest.fixture(scope="module")
def xt():
    import __graft_entry__ as g
    g.build()
    import paper_2511_07539_gb300 as xt
    return xt


def test_expneg_accuracy(xt):
    rng = np.random.default_rng(0)
    ln2 = np.log(2.0)
    tau = np.concatenate([10 ** rng.uniform(-4, np.log10(708), 40000),
                          ln2 * np.arange(1, 1000), ln2 * np.arange(1, 200) * (1 + 2 * EPS),
                          ln2 * np.arange(1, 200) * (1 - 2 * EPS),
                          [1e-4, 0.6931471805599452, 0.6931471805599453, 0.6931471805599454,
                           37.4, 38.0, 708.9, 709.0, 800.0, 1e6]])
    ex, ome, rex, rome = xt.xt_selftest_fixed(0, tau)
    mp.mp.dps = 40
    idx = np.concatenate([np.arange(0, tau.shape[0], 7), np.arange(tau.shape[0] - 12, tau.shape[0])])
    for i in idx:
        t = mp.mpf(float(tau[i]))
        te = mp.e ** (-t)
        if tau[i] < 708:
            assert abs(ex[i] - te) <= 0.6 * EPS * te, (tau[i], ex[i])
        else:
            assert ex[i] == 0.0 or abs(ex[i] - te) <= 1e-300
        assert abs(ome[i] - (1 - te)) <= 8 * EPS * (1 - te), (tau[i], ome[i])
    ok = tau < 700
    np.testing.assert_allclose(ex[ok], rex[ok], rtol=4 * EPS, atol=0)
    np.testing.assert_allclose(ome, rome, rtol=10 * EPS, atol=0)
    assert np.all(ex[tau >= 709] == 0) and np.all(ome[tau >= 709] == 1)


def test_sincos_2pi_accuracy(xt):
    rng = np.random.default_rng(1)
    U = np.concatenate([rng.integers(0, 2 ** 53, 40000, dtype=np.int64),
                        np.arange(0, 2 ** 53, 2 ** 47, dtype=np.int64),      # octant edges and j steps
                        np.array([1, 2 ** 50 - 1, 2 ** 50, 2 ** 50 + 1, 2 ** 53 - 1], dtype=np.int64)])
    u = U.astype(np.float64) * 2.0 ** -53
    assert np.array_equal((u * 2.0 ** 53).astype(np.int64), U)
    s, c, rs, rc = xt.xt_selftest_fixed(1, u)
    mp.mp.dps = 40
    # Q63 fixed point: an absolute error of a few 2^-63 (far below one ulp of
    # 1; direction components enter the geometry with absolute meaning) on top
    # of the final rounding to double
    for i in range(0, U.shape[0], 5):
        phi = 2 * mp.pi * mp.mpf(int(U[i])) / mp.mpf(2) ** 53
        for got, ref in ((s[i], mp.sin(phi)), (c[i], mp.cos(phi))):
            err = abs(got - ref)
            assert err <= 0.5 * EPS * abs(ref) + 4e-18, (U[i], got)
    # CUDA sin/cos of the double 2 pi u (rounded angle): a few ulp apart at most
    assert np.max(np.abs(s - rs)) < 8 * EPS and np.max(np.abs(c - rc)) < 8 * EPS
    np.testing.assert_allclose(s * s + c * c, 1.0, rtol=0, atol=4 * EPS)
