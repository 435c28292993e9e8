"""The surrogate network's CUDA kernels against the FP64 oracle: gradients (relative 1e-4),
Adam updates, FP32 vs BF16 inference, determinism, and learning a separable problem."""
import numpy as np
import pytest

import paper_2411_18370_b300 as ft
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

D, W = 9, 128


@pytest.fixture(scope="module")
def ctx():
    c = ft.create(0)
    yield c
    c.close()


def _batch(B, seed):
    g = np.random.default_rng(seed)
    X = g.standard_normal((B, D)).astype(np.float32)
    y = (X[:, 0] + 0.5 * X[:, 1] - 0.3 * X[:, 2] + 0.2 * g.standard_normal(B) > 0).astype(np.float32)
    return X, y


def test_gradient_matches_fp64_backprop(ctx):
    net = ft.MLP(ctx, D, W, seed=3)
    theta = net.get_params()
    X, y = _batch(256, 1)
    loss, g = net.loss_grad(X, y)
    l_or, g_or = omlp.loss_and_grad(theta.astype(np.float64), X, y, D, W)
    assert abs(loss - l_or) < 1e-5 * abs(l_or) + 1e-7
    scale = np.abs(g_or).max()
    err = np.abs(g.astype(np.float64) - g_or)
    assert np.all(err <= 1e-4 * np.abs(g_or) + 1e-6 * scale), float((err / (np.abs(g_or) + 1e-6 * scale)).max())
    net.close()


def test_adam_step_matches_oracle(ctx):
    net = ft.MLP(ctx, D, W, seed=4)
    th0 = net.get_params().astype(np.float64)
    X, y = _batch(128, 2)
    m = np.zeros_like(th0)
    v = np.zeros_like(th0)
    th = th0.copy()
    for t in (1, 2, 3):
        _, g = net.loss_grad(X, y)
        net.adam_step(1e-3)
        th, m, v = omlp.adam_step(th, g.astype(np.float64), m, v, t, 1e-3)
        got = net.get_params().astype(np.float64)
        assert np.all(np.abs(got - th) <= 1e-6 + 1e-5 * np.abs(th))
    net.close()


def test_training_learns_and_is_deterministic(ctx):
    X, y = _batch(8192, 5)
    nets = []
    for _ in range(2):
        net = ft.MLP(ctx, D, W, seed=11)
        hist = net.train(X, y, batch=512, epochs=8, lr=2e-3, seed=21)
        nets.append(net)
    assert hist[-1] < 0.5 * hist[0]
    assert np.array_equal(nets[0].get_params(), nets[1].get_params())
    Xt, yt = _batch(4096, 6)
    p32 = nets[0].predict(Xt, bf16=False)
    p16 = nets[0].predict(Xt, bf16=True)
    assert np.mean((p32 > 0.5) == (yt > 0.5)) > 0.9
    assert np.max(np.abs(p32 - p16)) < 0.05
    p_or = omlp.predict(nets[0].get_params().astype(np.float64), Xt, D, W)
    assert np.max(np.abs(p32 - p_or)) < 1e-5
    for n in nets:
        n.close()


@pytest.mark.parametrize("d,w,n", [(D, W, 1000), (13, 128, 4096), (40, 64, 300), (9, 48, 129)])
def test_bf16_inference_on_tensor_cores(ctx, d, w, n):
    """BF16 inference with each hidden layer one tcgen05.mma product of 128 samples (FP32
    accumulators in tensor memory) against (a) the same BF16 inference on the CUDA cores and
    (b) the FP64 oracle.  Both BF16 paths round inputs, weights and activations to BF16 and sum
    in FP32, so they differ only by summation order (an activation near a BF16 rounding
    boundary can round the other way): at most 5e-3 in p, 5e-4 on average.  Against the FP64
    network the BF16 roundings (unit roundoff 2^-8 per layer) allow 0.05, the tolerance of the
    BF16 path.  Sample counts that are not a multiple of 128 leave a ragged last tile."""
    net = ft.MLP(ctx, d, w, seed=5 + d)
    g = np.random.default_rng(d * 100 + w)
    X = g.standard_normal((4096, d)).astype(np.float32)
    y = (X[:, 0] - 0.7 * X[:, 1] + 0.3 * g.standard_normal(4096) > 0).astype(np.float32)
    net.train(X, y, batch=512, epochs=3, lr=2e-3, seed=7)
    Xt = g.standard_normal((n, d)).astype(np.float32)
    p_tc = net.predict(Xt, bf16=True)
    p_cc = net.predict(Xt, bf16=True, tensor_cores=False)
    p_or = omlp.predict(net.get_params().astype(np.float64), Xt, d, w)
    assert np.all(np.isfinite(p_tc)) and np.all((p_tc >= 0) & (p_tc <= 1))
    diff = np.abs(p_tc.astype(np.float64) - p_cc)
    assert diff.max() < 5e-3 and diff.mean() < 5e-4, (diff.max(), diff.mean())
    assert np.max(np.abs(p_tc - p_or)) < 0.05
    # device input and output take the same path
    import torch

    p_dev = net.predict(torch.from_numpy(Xt).cuda(), bf16=True).cpu().numpy()
    assert np.array_equal(p_dev, p_tc)
    net.close()


def test_tensor_core_inference_many_tiles_per_group(ctx):
    """Enough samples that every SM's four tile groups loop over several 128-sample tiles
    (the bias stored back into the accumulator columns after each layer carries from one
    tile to the next), with a ragged last tile: the same probabilities as the CUDA-core BF16
    path up to summation order, and the FP64 oracle within the BF16 tolerance on a sample."""
    import torch

    d, w = 13, 128
    net = ft.MLP(ctx, d, w, seed=11)
    g = np.random.default_rng(17)
    X = g.standard_normal((4096, d)).astype(np.float32)
    y = (X[:, 0] - 0.4 * X[:, 3] + 0.3 * g.standard_normal(4096) > 0).astype(np.float32)
    net.train(X, y, batch=512, epochs=2, lr=2e-3, seed=5)
    n = 4 * 148 * 128 * 3 + 77
    Xt = torch.randn(n, d, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    p_tc = net.predict(Xt, bf16=True).cpu().numpy().astype(np.float64)
    p_cc = net.predict(Xt, bf16=True, tensor_cores=False).cpu().numpy().astype(np.float64)
    diff = np.abs(p_tc - p_cc)
    assert diff.max() < 5e-3 and diff.mean() < 5e-4, (diff.max(), diff.mean())
    idx = np.random.default_rng(1).choice(n, 2000, replace=False)
    p_or = omlp.predict(net.get_params().astype(np.float64), Xt.cpu().numpy()[idx], d, w)
    assert np.max(np.abs(p_tc[idx] - p_or)) < 0.05
    net.close()
