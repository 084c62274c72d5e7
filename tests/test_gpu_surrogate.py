"""A9 population surrogate on the GPU (needs a GPU): BF16 tensor-core forward
and backward vs the FP64 oracle (P10: cosine >= 0.999, relative norm error
<= 1e-2 on the gradients), training lowers the loss, and the trained network
as warm start of the rate solves versus the Boltzmann warm start."""
import numpy as np
import pytest

import synth
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xt():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a GPU"
    import __graft_entry__ as g
    g.build()
    import paper_2511_07539_gb300 as xt
    return xt


def _ctx(xt):
    import torch
    return xt.Context(0, torch.cuda.current_stream().cuda_stream)


def _bf16(a):
    """Round float32 values to bfloat16 (nearest even) and back."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_gradients_vs_fp64_oracle(xt):
    rng = np.random.default_rng(0)
    sizes = [35, 64, 64, 64, 40]
    flat = np.concatenate([np.concatenate([rng.standard_normal(a * b) * np.sqrt(2.0 / a),
                                           rng.standard_normal(b) * 0.1])
                           for a, b in zip(sizes[:-1], sizes[1:])]).astype(np.float32)
    B = 96
    X = rng.standard_normal((B, 35)).astype(np.float32)
    T = rng.standard_normal((B, 40)).astype(np.float32)
    M = (rng.random((B, 40)) > 0.25).astype(np.float32)
    with _ctx(xt) as ctx:
        xt.surrogate_init(ctx.h, sizes)
        xt.surrogate_weights(ctx.h, flat)
        loss, g = xt.surrogate_train_step(ctx.h, X, T, M, update=False, n_param=flat.size)
        Y = xt.surrogate_predict(ctx.h, X, 40)
    # oracle with BF16-rounded weights and inputs (biases stay FP32 on the GPU)
    params = mlp.unflatten(flat.astype(np.float64), sizes)
    params = [(_bf16(W), b) for W, b in params]
    y, _ = mlp.forward(params, _bf16(X))
    l_o, g_o = mlp.loss_and_grads(params, _bf16(X), T.astype(np.float64), M.astype(np.float64))
    go = np.concatenate([np.concatenate([gW.ravel(), gb.ravel()]) for gW, gb in g_o])
    assert np.linalg.norm(Y - y) / np.linalg.norm(y) < 1e-2
    assert abs(loss - l_o) / l_o < 1e-2
    cos = float(g @ go / (np.linalg.norm(g) * np.linalg.norm(go)))
    rel = float(np.linalg.norm(g - go) / np.linalg.norm(go))
    assert cos >= 0.999 and rel <= 1e-2, (cos, rel)
    # every layer, not only the total
    o = 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        n = a * b + b
        gl, gol = g[o:o + n], go[o:o + n]
        assert np.linalg.norm(gl - gol) / np.linalg.norm(gol) < 2e-2
        o += n


@pytest.mark.parametrize("sizes,B", [([35, 50, 7], 37), ([17, 129, 33, 300], 130)])
def test_gradients_ragged_shapes(xt, sizes, B):
    """The fused kernel pads every row to 16 elements and the batch to tiles
    of 128: layer sizes and batches that fill neither (a second batch tile of
    2 rows; 129 inputs, whose last weight row and the bias row spill into a
    second 128-row tile; a 300-wide K in two chunks) give the FP64 oracle's
    gradients."""
    rng = np.random.default_rng(7)
    flat = np.concatenate([np.concatenate([rng.standard_normal(a * b) * np.sqrt(2.0 / a),
                                           rng.standard_normal(b) * 0.1])
                           for a, b in zip(sizes[:-1], sizes[1:])]).astype(np.float32)
    nin, nout = sizes[0], sizes[-1]
    X = rng.standard_normal((B, nin)).astype(np.float32)
    T = rng.standard_normal((B, nout)).astype(np.float32)
    M = (rng.random((B, nout)) > 0.3).astype(np.float32)
    with _ctx(xt) as ctx:
        xt.surrogate_init(ctx.h, sizes)
        xt.surrogate_weights(ctx.h, flat)
        loss, g = xt.surrogate_train_step(ctx.h, X, T, M, update=False, n_param=flat.size)
    params = [(_bf16(W), b) for W, b in mlp.unflatten(flat.astype(np.float64), sizes)]
    l_o, g_o = mlp.loss_and_grads(params, _bf16(X), T.astype(np.float64), M.astype(np.float64))
    go = np.concatenate([np.concatenate([gW.ravel(), gb.ravel()]) for gW, gb in g_o])
    assert abs(loss - l_o) / l_o < 1e-2
    o = 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        n = a * b + b
        gl, gol = g[o:o + n], go[o:o + n]
        cos = float(gl @ gol / (np.linalg.norm(gl) * np.linalg.norm(gol)))
        assert cos >= 0.999 and np.linalg.norm(gl - gol) / np.linalg.norm(gol) < 2e-2, (a, b, cos)
        # the bias part alone (the row of ones)
        bl, bol = gl[a * b:], gol[a * b:]
        assert np.linalg.norm(bl - bol) / np.linalg.norm(bol) < 2e-2, (a, b)
        o += n


def test_training_lowers_the_loss(xt):
    rng = np.random.default_rng(1)
    sizes = [16, 64, 64, 8]
    W = rng.standard_normal((16, 8))
    X = rng.standard_normal((512, 16)).astype(np.float32)
    T = np.tanh(X @ W / 4).astype(np.float32)
    M = np.ones_like(T)
    with _ctx(xt) as ctx:
        xt.surrogate_init(ctx.h, sizes, seed=3)
        l0, _ = xt.surrogate_train_step(ctx.h, X, T, M, lr=3e-3, update=True)
        for _ in range(300):
            l, _ = xt.surrogate_train_step(ctx.h, X, T, M, lr=3e-3, update=True)
    assert l < 0.05 * l0, (l0, l)


def test_surrogate_warm_start_gains(xt):
    """Trained on the solved populations of one clumpy ejecta realization, the
    network warm-starts the Newton solves (optical depths from the
    populations) of a second realization with the same atoms and new clumps:
    the result is the same and the solves take far fewer Newton steps than
    from Boltzmann populations."""
    kw_w = dict(seed=1, n=12, n_packets=1000, n_lines=2000, level_range=(20, 50),
                subdomains=(2, 2, 2))
    train = synth.clumpy_onion(**kw_w)
    test = synth.clumpy_onion(field_seed=2, **kw_w)
    ups = synth.collision_strengths(train.upsilon_seed, train.level_off)
    kw = dict(rates=xt.XT_RATES_JBAR, jbar_W=5.6e-5, jbar_TR=8000.0, newton_max=100,
              newton_tol=1e-8)
    with _ctx(xt) as ctx:
        ctx.load(train)
        s0 = xt.solve_nlte(ctx.h, ups, precision=xt.XT_PREC_FP64, warm=xt.XT_WARM_LTE, **kw)
        assert s0["not_converged"] == 0
        st = xt.train_surrogate(ctx.h, epochs=500, batch=128, lr=2e-3, rates=xt.XT_RATES_JBAR,
                                jbar_W=5.6e-5, jbar_TR=8000.0)
        assert st["last_loss"] < 0.02 * st["first_loss"], st
        ref = np.zeros((test.ncell, test.nlev))
        # the second realization in the same context: grid and atoms reloaded, network kept
        ctx.load(test)
        xt.solve_nlte(ctx.h, ups, precision=xt.XT_PREC_FP64, warm=xt.XT_WARM_LTE, pops_out=ref, **kw)
        res = {}
        for warm in (xt.XT_WARM_LTE, xt.XT_WARM_SURROGATE):
            out = np.zeros_like(ref)
            s = xt.solve_nlte(ctx.h, ups, precision=xt.XT_PREC_FP32_IR, warm=warm,
                              pops_out=out, **kw)
            assert s["not_converged"] == 0
            m = ref > 1e-30 * ref.max()
            assert np.max(np.abs(out[m] / ref[m] - 1)) < 1e-6
            res[warm] = (s["mean_iter"], s["solve_ms"])
    print("mean Newton steps, solve ms", res, "training", st)
    assert res[xt.XT_WARM_SURROGATE][0] < 0.6 * res[xt.XT_WARM_LTE][0], res
