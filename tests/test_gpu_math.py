"""The library's fixed-point device primitives against mpmath and against
CUDA's own functions (needs a GPU): e^-tau and 1 - e^-tau of every line event,
sin and cos of every emission azimuth, the emission's quotients and its
direction."""
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


def _ulps(got, ref):
    """Distance in units in the last place of ref (positive doubles)."""
    return np.abs(got - ref) / np.spacing(np.abs(ref))


def test_integer_pipe_quotient(xt):
    """The emission's quotients (lab frequency, photon number, wall spacing
    d / |n_k|) on the integer pipe: within 0.51 ulp of the exact quotient, and
    CUDA's correctly rounded division agrees to one ulp at most, mostly exactly."""
    rng = np.random.default_rng(2)
    a = 10 ** rng.uniform(-30, 30, 60000)
    b = 10 ** rng.uniform(-30, 30, 60000)
    one_m = np.nextafter(2.0, 0.0)                                   # significand all ones
    sa = np.array([1.0, 1.0, 3.0, 1.5, one_m, one_m, 1.0, np.nextafter(1.0, 2.0), 7.0, 1e15, 1e43])
    sb = np.array([1.0, one_m, 1.5, 3.0, one_m, 1.0, np.nextafter(1.0, 2.0), 1.0, 2.0 ** 40, 0.97,
                   3e15])
    # the emission's ranges: nu_cmf / D, E0/h / nu_cmf, d / |n_k|
    nu = 10 ** rng.uniform(14, 15.6, 20000)
    D = 1.0 + rng.uniform(-0.03, 0.03, 20000)
    nk = 10 ** rng.uniform(-20, 0, 20000)
    A = np.concatenate([a, sa, nu, 1e43 * rng.uniform(0.5, 2, 20000), np.full(20000, 2.4e13)])
    B = np.concatenate([b, sb, D, nu, nk])
    q, _, ref, _ = xt.xt_selftest_fixed(2, np.stack([A, B], axis=1))
    u = _ulps(q, ref)
    assert u.max() <= 1.0, (A[u.argmax()], B[u.argmax()], q[u.argmax()], ref[u.argmax()])
    assert np.mean(u == 0) > 0.98
    exact_q = [0, 2, 3, 4, 5, 7, 8]                                   # representable quotients
    np.testing.assert_array_equal(q[60000 + np.array(exact_q)], (sa / sb)[exact_q])
    mp.mp.dps = 40
    for i in np.concatenate([np.nonzero(u > 0)[0][:200], np.arange(0, A.size, 97)]):
        exact = mp.mpf(float(A[i])) / mp.mpf(float(B[i]))
        assert abs(q[i] - exact) <= 0.51 * np.spacing(q[i]), (A[i], B[i])


def test_integer_pipe_direction(xt):
    """The isotropic emission direction from the integer pipe: n_z = 2u - 1
    exactly; n_x, n_y = sqrt(1 - mu^2) (cos, sin)(2 pi v) from the exact
    106-bit 1 - mu^2, within about half an ulp plus the Q63 angle error of the
    exact values, and a unit vector."""
    rng = np.random.default_rng(3)
    U = np.concatenate([rng.integers(0, 2 ** 53, 30000, dtype=np.int64),
                        np.array([0, 1, 2, 2 ** 10, 2 ** 30, 2 ** 52 - 1, 2 ** 52, 2 ** 52 + 1,
                                  2 ** 53 - 2 ** 20, 2 ** 53 - 1], dtype=np.int64)])
    V = np.concatenate([rng.integers(0, 2 ** 53, 30000, dtype=np.int64),
                        np.array([0, 1, 2 ** 50, 2 ** 51, 3 * 2 ** 50, 2 ** 52, 5 * 2 ** 50,
                                  3 * 2 ** 51, 7 * 2 ** 50, 2 ** 53 - 1], dtype=np.int64)])
    u = U.astype(np.float64) * 2.0 ** -53
    v = V.astype(np.float64) * 2.0 ** -53
    nx, ny, nz = xt.xt_selftest_fixed(3, np.stack([u, v], axis=1))[:3]
    mu = (2 * U - 2 ** 53).astype(np.float64) * 2.0 ** -53             # exact
    np.testing.assert_array_equal(nz, mu)
    assert nx[-10] == 0.0 and ny[-10] == 0.0 and nz[-10] == -1.0       # U = 0: mu = -1
    np.testing.assert_allclose(nx * nx + ny * ny + nz * nz, 1.0, rtol=0, atol=4 * EPS)
    mp.mp.dps = 50
    for i in np.concatenate([np.arange(0, U.size, 7), np.arange(U.size - 10, U.size)]):
        m = 2 * mp.mpf(int(U[i])) / mp.mpf(2) ** 53 - 1
        st = mp.sqrt(1 - m * m)
        phi = 2 * mp.pi * mp.mpf(int(V[i])) / mp.mpf(2) ** 53
        for got, ref in ((nx[i], st * mp.cos(phi)), (ny[i], st * mp.sin(phi))):
            assert abs(got - ref) <= 0.6 * EPS * abs(ref) + 5e-18 * st, (U[i], V[i], got)
    # beside the plain double formula sqrt(1 - mu mu) (cos, sin) of the rounded
    # angle: apart only by that formula's own rounding and cancellation
    st = np.sqrt(1.0 - mu * mu)
    ok = np.abs(mu) < 0.999
    assert np.max(np.abs(nx - st * np.cos(2 * np.pi * v))[ok]) < 8 * EPS
    assert np.max(np.abs(ny - st * np.sin(2 * np.pi * v))[ok]) < 8 * EPS
