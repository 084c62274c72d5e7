"""The library's integer-pipe routines (fixexp.cuh: the quotient, the
emission direction, e^-tau and 1 - e^-tau, sin/cos of the azimuth, Sobolev
beta and its derivative, the scaled rounding to FP32 of the rate solve; and
the Philox generator of philox.cuh; the packet quota of quota.h; the line
order of linesort.h; the ray hand-out order of raysched.h) compiled
for the host from the same source and
checked against mpmath on the CPU, so that they are pinned without a GPU.
On the device the FP32 seeds of the two Newton-Raphson iterations come from
rcp/rsqrt.approx instead of the correctly rounded host operations; the bounds
below hold for either seed.  (The same routines run on the GB300 in
test_gpu_math.py.)"""
import ctypes as C
import os
import shutil
import subprocess

import mpmath as mp
import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2511_07539_gb300", "csrc")
EPS = 2.220446049250313e-16


@pytest.fixture(scope="module")
def fx(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    so = str(tmp_path_factory.mktemp("fixmath") / "fixmath_host.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off", "-I", HERE,
                    "-I", CSRC, os.path.join(HERE, "fixmath_host.cpp"), "-o", so], check=True)
    return C.CDLL(so)


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _call(lib, name, ins, nout):
    n = ins[0].shape[0]
    outs = [np.zeros(n) for _ in range(nout)]
    getattr(lib, name)(*[_p(a) for a in ins], *[_p(o) for o in outs], C.c_long(n))
    return outs


def test_quotient(fx):
    rng = np.random.default_rng(4)
    a = 10 ** rng.uniform(-300, 300, 50000)
    b = 10 ** rng.uniform(-300, 300, 50000)
    keep = np.abs(np.log10(a) - np.log10(b)) < 300         # quotient in the normal range
    a, b = a[keep], b[keep]
    (q,) = _call(fx, "h_div_pos", [a, b], 1)
    ulp = np.abs(q - a / b) / np.spacing(a / b)
    assert ulp.max() <= 1.0 and np.mean(ulp == 0) > 0.98
    mp.mp.dps = 40
    for i in np.concatenate([np.nonzero(ulp > 0)[0][:100], np.arange(0, a.size, 211)]):
        exact = mp.mpf(float(a[i])) / mp.mpf(float(b[i]))
        assert abs(q[i] - exact) <= 0.51 * np.spacing(q[i]), (a[i], b[i])


def test_exponential(fx):
    rng = np.random.default_rng(5)
    ln2 = np.log(2.0)
    tau = np.concatenate([10 ** rng.uniform(-4, np.log10(700), 20000), ln2 * np.arange(1, 300),
                          ln2 * np.arange(1, 300) * (1 + 2 * EPS), [0.6931471805599453, 1e-4]])
    ex, ome = _call(fx, "h_expneg", [tau], 2)
    mp.mp.dps = 40
    for i in range(0, tau.size, 13):
        te = mp.e ** (-mp.mpf(float(tau[i])))
        assert abs(ex[i] - te) <= 0.6 * EPS * te, tau[i]
        assert abs(ome[i] - (1 - te)) <= 8 * EPS * (1 - te), tau[i]


def test_azimuth_and_direction(fx):
    rng = np.random.default_rng(6)
    U = np.concatenate([rng.integers(0, 2 ** 53, 20000, dtype=np.int64),
                        np.array([0, 1, 2 ** 50, 2 ** 52, 2 ** 53 - 1], dtype=np.int64)]).astype(np.uint64)
    V = rng.integers(0, 2 ** 53, U.size, dtype=np.int64).astype(np.uint64)
    s, c = _call(fx, "h_sincos", [V], 2)
    nx, ny, nz = _call(fx, "h_isotropic", [U, V], 3)
    mu = (2 * U.astype(np.int64) - 2 ** 53).astype(np.float64) * 2.0 ** -53
    np.testing.assert_array_equal(nz, mu)
    np.testing.assert_allclose(nx * nx + ny * ny + nz * nz, 1.0, rtol=0, atol=4 * EPS)
    mp.mp.dps = 50
    for i in np.concatenate([np.arange(0, U.size, 17), np.arange(U.size - 5, U.size)]):
        phi = 2 * mp.pi * mp.mpf(int(V[i])) / mp.mpf(2) ** 53
        for got, ref in ((s[i], mp.sin(phi)), (c[i], mp.cos(phi))):
            assert abs(got - ref) <= 0.5 * EPS * abs(ref) + 4e-18, (V[i], got)
        m = 2 * mp.mpf(int(U[i])) / mp.mpf(2) ** 53 - 1
        st = mp.sqrt(1 - m * m)
        for got, ref in ((nx[i], st * mp.cos(phi)), (ny[i], st * mp.sin(phi))):
            assert abs(got - ref) <= 0.6 * EPS * abs(ref) + 5e-18 * st, (U[i], V[i], got)


def test_sobolev_beta_and_derivative(fx):
    rng = np.random.default_rng(7)
    tau = np.concatenate([10 ** rng.uniform(-20, 4, 5000), [0.0, -1.0, 2.0 ** -10,
                          np.nextafter(2.0 ** -10, 0), 1e-300, 709.0, 800.0, 1e6]])
    beta, dbeta = _call(fx, "h_beta", [tau], 2)
    assert beta[-8] == 1.0 and dbeta[-8] == 0.0 and beta[-7] == 1.0 and dbeta[-7] == 0.0
    mp.mp.dps = 50
    for i in range(tau.size):
        t = mp.mpf(float(tau[i]))
        if t <= 0:
            continue
        b = -mp.expm1(-t) / t
        if t < mp.mpf("1e-3"):      # the closed form cancels: its Taylor series
            db = mp.fsum(k * (-t) ** (k - 1) * (-1) / mp.factorial(k + 1) for k in range(1, 40))
        else:
            db = (t * mp.exp(-t) + mp.expm1(-t)) / (t * t)
        assert abs(beta[i] - b) <= 3 * EPS * b, (tau[i], beta[i])
        # the derivative's numerator cancels to about tau^2 / 2 for small tau:
        # a relative error up to ~2 / tau ulp just above the series range
        bound = 4 * EPS if tau[i] < 2.0 ** -10 else 4 * EPS * max(1.0, 2.0 / float(tau[i]))
        assert abs(dbeta[i] - db) <= bound * abs(db), (tau[i], dbeta[i], float(db))


def test_scaled_rounding_to_fp32(fx):
    """w 2^k rounded to FP32 with integer operations equals the correctly
    rounded conversion (to nearest even, subnormals kept) bit for bit."""
    rng = np.random.default_rng(8)
    n = 200000
    w = rng.choice([-1.0, 1.0], n) * 10 ** rng.uniform(-300, 300, n)
    ew = np.frexp(w)[1] - 1
    k = rng.integers(-200, 80, n) - ew                       # results from 2^-200 to 2^80
    k = k.astype(np.int32)
    # ties and the subnormal boundary: 24- and 25-bit significands near 2^-126 and 2^-149
    m = rng.integers(2 ** 24, 2 ** 25, 2000).astype(np.float64)
    w2 = np.concatenate([m, -m]) * 2.0 ** -24
    k2 = rng.integers(-160, -120, w2.size).astype(np.int32)
    w, k = np.concatenate([w, w2]), np.concatenate([k, k2])
    out = np.zeros(w.size, dtype=np.float32)
    fx.h_scaled_f32(_p(w), _p(k), _p(out), C.c_long(w.size))
    with np.errstate(over="ignore", under="ignore"):
        ref = np.ldexp(w, k).astype(np.float32)
    np.testing.assert_array_equal(out.view(np.uint32), ref.view(np.uint32))


def test_philox_vs_numpy(fx):
    """The CUDA side's Philox4x64-10 against numpy's independent Philox (which
    increments its counter before use), and u = (x >> 11) 2^-53 exactly."""
    rng = np.random.default_rng(9)
    n = 300
    ctr = rng.integers(0, 2 ** 63, (n, 4), dtype=np.int64).astype(np.uint64)
    ctr[:, 0] |= np.uint64(1)                    # nonzero 256-bit counter
    key = rng.integers(0, 2 ** 63, (n, 2), dtype=np.int64).astype(np.uint64)
    out = np.zeros((n, 4), dtype=np.uint64)
    fx.h_philox(_p(ctr), _p(key), _p(out), C.c_long(n))
    for i in range(n):
        c = [int(x) for x in ctr[i]]
        c256 = c[0] + (c[1] << 64) + (c[2] << 128) + (c[3] << 192)
        bg = np.random.Philox(counter=c256 - 1, key=int(key[i, 0]) + (int(key[i, 1]) << 64))
        assert np.array_equal(out[i], bg.random_raw(4).astype(np.uint64)), i
    x = np.concatenate([out.ravel(), np.array([0, 2 ** 11 - 1, 2 ** 11, 2 ** 64 - 1], dtype=np.uint64)])
    u = np.zeros(x.size)
    fx.h_u01(_p(x), _p(u), C.c_long(x.size))
    np.testing.assert_array_equal(u, (x >> np.uint64(11)).astype(np.float64) * 2.0 ** -53)


def test_line_order_is_a_stable_descending_frequency_sort(fx):
    """The library's line order (a radix sort of the frequencies' bit
    patterns) equals a stable sort by descending frequency: numpy's stable
    argsort of -nu, with many ties, one line, none, and frequencies spanning
    many binades."""
    rng = np.random.default_rng(12)
    cases = [np.zeros(0), np.array([3.0e15]),
             2.99792458e18 / (1000.0 + rng.integers(0, 50, 20_000) * 0.5),    # many equal wavelengths
             10.0 ** rng.uniform(10, 20, 100_003),                           # many binades
             np.full(777, 5.0e14)]
    for nu in cases:
        nu = np.ascontiguousarray(nu, dtype=np.float64)
        order = np.zeros(len(nu), dtype=np.int32)
        fx.h_linesort(_p(nu), C.c_int(len(nu)), _p(order))
        np.testing.assert_array_equal(order, np.argsort(-nu, kind="stable"))


@pytest.mark.parametrize("p_begin,n,nbin,nview", [(0, 3 * 5 * 7, 5, 7), (11, 3 * 5 * 7, 5, 7),
                                                   (35, 70, 5, 7), (0, 40, 40, 1), (3, 1, 5, 7),
                                                   (0, 0, 5, 7), (123, 4 * 36 * 49 + 17, 36, 49)])
def test_ray_hand_out_order_is_a_bijection(fx, p_begin, n, nbin, nview):
    """The refill's ray order permutes each launch's id range onto itself
    (every ray traced once), takes a whole block's ids viewer by viewer and bin
    after bin, and leaves the ids of blocks the range cuts in order."""
    out = np.zeros(n, dtype=np.int64)
    fx.h_rayids(C.c_int64(p_begin), C.c_int64(n), C.c_int64(nbin), C.c_int64(nview), _p(out))
    ids = np.arange(p_begin, p_begin + n)
    np.testing.assert_array_equal(np.sort(out), ids)
    per = nbin * nview
    for v, p in zip(ids, out):
        lo = (v // per) * per
        if nview > 1 and lo >= p_begin and lo + per <= p_begin + n:
            rem = v - lo
            assert p == lo + (rem % nbin) * nview + rem // nbin       # bin fastest, then viewer
        else:
            assert p == v


def test_packet_quota_matches_the_oracle(fx):
    """The library's largest-remainder quota (a selection of the largest
    remainders, ties to the lower cell) equals the oracle's (pinned by brute
    force) exactly, ties and empty cells included."""
    import oracle
    rng = np.random.default_rng(10)
    for N in [1, 7, 1000, 123457, 100_000_000]:
        for kind in range(3):
            L = rng.random(5000) * (rng.random(5000) > 0.3)
            if kind == 1:
                L = np.round(L * 4) / 4                  # many equal remainders
            if kind == 2:
                L[:] = 0.0
                L[rng.integers(0, 5000, 7)] = 1.0
            q = np.zeros(L.size + 1, dtype=np.int64)
            fx.h_quota(_p(L), C.c_long(L.size), C.c_long(N), _p(q))
            np.testing.assert_array_equal(q, oracle.packet_quota(L, N))
