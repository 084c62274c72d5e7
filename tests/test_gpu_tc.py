"""The tensor-core path of the batched LU (tcgen05 MMA, kind::tf32 and
kind::f16 with BF16 operands, operands in shared memory, accumulator in TMEM)
against numpy (needs a GPU): D = A B^T with A and B rounded to TF32 (nearest,
ties away from zero) or BF16 (nearest, ties to even) equals the float64
product of the rounded operands to FP32 accumulation error."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xt():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a GPU"
    import __graft_entry__ as g
    g.build()
    import paper_2511_07539_gb300 as xt
    return xt


def tf32(x):
    """Round float32 to TF32 (10 mantissa bits), nearest, ties away from zero."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32)


def bf16(x):
    """Round float32 to BF16 (7 stored mantissa bits), nearest, ties to even."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32)


def test_bf16_rounding_helper():
    """The test's own BF16 rounding: ties go to the even neighbour."""
    one = np.float32(1.0)
    tie_down = np.array([0x3F808000], np.uint32).view(np.float32)     # 1 + 2^-8: between 1 and 1 + 2^-7
    tie_up = np.array([0x3F818000], np.uint32).view(np.float32)       # 1 + 3 * 2^-8
    assert bf16(tie_down)[0] == one
    assert bf16(tie_up)[0] == np.float32(1 + 2 ** -6)
    assert bf16(np.float32(1 + 2 ** -7))[0] == np.float32(1 + 2 ** -7)


@pytest.mark.parametrize("N", [16, 48, 128, 256])
def test_bf16_gemm_vs_numpy(xt, N):
    rng = np.random.default_rng(100 + N)
    A = rng.standard_normal((128, 32)).astype(np.float32)
    B = rng.standard_normal((N, 32)).astype(np.float32)
    A[7] = 0.0
    B[:, 30] = -0.5
    D = xt.xt_selftest_tc_bf16(A, B)
    ref = bf16(A).astype(np.float64) @ bf16(B).astype(np.float64).T
    scale = np.abs(bf16(A)).astype(np.float64) @ np.abs(bf16(B)).astype(np.float64).T
    assert np.all(np.isfinite(D))
    err = np.abs(D - ref) / np.maximum(scale, 1e-30)
    assert err.max() < 2e-6, err.max()
    # BF16 is what the tensor core sees: the TF32-rounded product differs more
    assert np.abs(tf32(A).astype(np.float64) @ tf32(B).astype(np.float64).T - ref).max() > 1e-3


def test_bf16_gemm_rows_and_columns_are_not_mixed(xt):
    """Unit vectors in BF16: each K element sits at its own 2-byte slot of the
    16-bit layout, so a wrong chunk or element offset moves the entries."""
    A = np.zeros((128, 32), np.float32)
    B = np.zeros((80, 32), np.float32)
    for r in range(128):
        A[r, (5 * r + 1) % 32] = float(r % 16 + 1)
    for n in range(80):
        B[n, (7 * n) % 32] = float(2 ** -(n % 5))
    D = xt.xt_selftest_tc_bf16(A, B)
    np.testing.assert_array_equal(D, (A.astype(np.float64) @ B.astype(np.float64).T).astype(np.float32))


@pytest.mark.parametrize("N", [16, 48, 128, 256])
def test_tf32_gemm_vs_numpy(xt, N):
    rng = np.random.default_rng(N)
    A = rng.standard_normal((128, 32)).astype(np.float32)
    B = rng.standard_normal((N, 32)).astype(np.float32)
    A[5] = 0.0                       # a zero row and an exactly representable column
    B[:, 3] = 0.25
    D = xt.xt_selftest_tc(A, B)
    ref = tf32(A).astype(np.float64) @ tf32(B).astype(np.float64).T
    scale = np.abs(tf32(A)).astype(np.float64) @ np.abs(tf32(B)).astype(np.float64).T
    assert np.all(np.isfinite(D))
    err = np.abs(D - ref) / np.maximum(scale, 1e-30)
    assert err.max() < 2e-6, err.max()
    # the rounding to TF32 is what the tensor core sees: the unrounded product differs more
    assert np.abs(A.astype(np.float64) @ B.astype(np.float64).T - ref).max() > 1e-4


def test_tf32_gemm_rows_and_columns_are_not_mixed(xt):
    """Unit vectors pick single entries: a transposed or shifted operand layout
    would move them."""
    A = np.zeros((128, 32), np.float32)
    B = np.zeros((64, 32), np.float32)
    for r in range(128):
        A[r, r % 32] = r + 1
    for n in range(64):
        B[n, (3 * n) % 32] = 1.0 / (n + 1)
    D = xt.xt_selftest_tc(A, B)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    np.testing.assert_allclose(D, ref, rtol=2e-3, atol=0)


def _solve(xt, w, prec, **kw):
    import torch
    with xt.Context(0, torch.cuda.current_stream().cuda_stream) as ctx:
        ctx.load(w)
        pops = np.zeros((w.ncell, w.nlev))
        st = xt.solve_nlte(ctx.h, w.upsilon, precision=prec, rates=xt.XT_RATES_JBAR,
                           warm=xt.XT_WARM_CURRENT, jbar_W=w.jbar_W, jbar_TR=w.jbar_TR,
                           levels_used=w.levels_used, pops_out=pops, **kw)
    return pops, st


def test_tensor_core_trailing_updates_in_the_rate_solve(xt):
    """The TF32 leg of the batched solve (trailing updates of the LU on the
    tensor cores) on systems of 250-300 levels (several 128-row tiles and two
    column chunks per update): no system falls back to FP64, the refinement
    converges in a few steps, and the populations agree with the FP32 leg's."""
    import synth
    w = synth.nlte_batch(n=3, seed=2, L_range=(250, 300))
    p32, s32 = _solve(xt, w, xt.XT_PREC_FP32_IR)
    ptc, stc = _solve(xt, w, xt.XT_PREC_TF32_IR)
    assert stc["fp64_fallbacks"] == 0 and stc["singular"] == 0, stc
    assert stc["mean_iter"] <= 4.0 and stc["max_iter_used"] <= 8, stc
    assert list(stc["panel_width"])[4:] == [32, 32, 32, 32]
    nz = np.repeat(w.n_ion_density, np.diff(w.level_off), axis=1)
    sig = (p32 >= 1e-30 * nz) & (nz > 0)
    assert np.max(np.abs(ptc[sig] / p32[sig] - 1)) < 1e-8


def test_bf16_trailing_updates_in_the_rate_solve(xt):
    """The BF16 leg: the same systems with the trailing updates' operands in
    BF16.  The factors are coarser, so the FP64 refinement takes more steps;
    a system it does not bring below tol within max_iter goes to the FP64
    solve.  Either way every population reaches the FP32 leg's to 1e-8."""
    import synth
    w = synth.nlte_batch(n=3, seed=2, L_range=(250, 300))
    p32, s32 = _solve(xt, w, xt.XT_PREC_FP32_IR, max_iter=16)
    pbf, sbf = _solve(xt, w, xt.XT_PREC_BF16_IR, max_iter=16)
    ptc, stc = _solve(xt, w, xt.XT_PREC_TF32_IR, max_iter=16)
    assert sbf["singular"] == 0, sbf
    nsys = w.ncell * (len(w.level_off) - 1)
    # the BF16 factors are coarser than the TF32 ones: more refinement steps
    assert sbf["mean_iter"] > stc["mean_iter"], (sbf, stc)
    assert sbf["fp64_fallbacks"] < 0.5 * nsys, sbf
    nz = np.repeat(w.n_ion_density, np.diff(w.level_off), axis=1)
    sig = (p32 >= 1e-30 * nz) & (nz > 0)
    assert np.max(np.abs(pbf[sig] / p32[sig] - 1)) < 1e-8
