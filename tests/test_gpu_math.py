"""The library's fixed-point e^-tau / 1 - e^-tau (used for every line event)
against mpmath and against CUDA's exp / expm1 (needs a GPU)."""
import mpmath as mp
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
EPS = 2.220446049250313e-16


def test_expneg_accuracy():
    import __graft_entry__ as g
    g.build()
    import paper_2511_07539_gb300 as xt
    rng = np.random.default_rng(0)
    ln2 = np.log(2.0)
    tau = np.concatenate([10 ** rng.uniform(-4, np.log10(708), 40000),
                          ln2 * np.arange(1, 1000), ln2 * np.arange(1, 200) * (1 + 2 * EPS),
                          ln2 * np.arange(1, 200) * (1 - 2 * EPS),
                          [1e-4, 0.6931471805599452, 0.6931471805599453, 0.6931471805599454,
                           37.4, 38.0, 708.9, 709.0, 800.0, 1e6]])
    ex, ome, rex, rome = xt.xt_selftest_expneg(tau)
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
