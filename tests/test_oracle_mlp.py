"""Pins of the FP64 reference of the warm-start network (CPU)."""
import numpy as np
import pytest

import synth
from oracle import mlp


def _data(B=40, seed=1):
    X = synth.normal(seed, 1, B * 64).reshape(B, 64)
    T = synth.normal(seed, 2, B * 3).reshape(B, 3)
    return X, T


def test_parameter_count():
    assert mlp.N_PARAMS == 12675


def test_gradient_against_central_differences():
    theta = mlp.init_params(3)
    X, T = _data()
    L, g = mlp.loss_and_grad(theta, X, T)
    rng_idx = (synth.uniform(4, 1, 60) * mlp.N_PARAMS).astype(int)
    h = 1e-6
    for i in rng_idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, T)[0] - mlp.loss_and_grad(tm, X, T)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9)


def test_all_units_active_is_a_product_of_matrices():
    """With large positive biases every ReLU passes: the network is affine,
    y = W4 (W3 (W2 (W1 x + b1) + b2) + b3) + b4."""
    theta = mlp.init_params(5)
    P = mlp.unpack(theta)
    for b in ("b1", "b2", "b3"):
        P[b][:] = 1e3
    P["W2"] = np.abs(P["W2"])   # positive inputs stay positive after layer 1
    P["W3"] = np.abs(P["W3"])
    theta = mlp.pack(P)
    X, _ = _data(10, 6)
    y, _ = mlp.forward(theta, X)
    ref = np.matmul(np.matmul(np.matmul(np.matmul(X, P["W1"].T) + P["b1"], P["W2"].T) + P["b2"],
                              P["W3"].T) + P["b3"], P["W4"].T) + P["b4"]
    np.testing.assert_allclose(y, ref, rtol=1e-12)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    v = synth.normal(7, 1, 5000) * 10 ** (synth.uniform(7, 2, 5000) * 6 - 3)
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.to_bf16(v), ref)


def test_features_against_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    p, _ = synth.torus(1500, seed=2, noise=0.002)
    X = mlp.features(p)
    p64 = p.astype(np.float64)
    _, nb = spatial.cKDTree(p64).query(p64, k=17)
    c = p64.mean(0)
    R = np.sqrt(((p64 - c) ** 2).sum(1).mean())
    for i in range(0, 1500, 37):
        js = [j for j in nb[i] if j != i][:16]
        o = p64[js] - p64[i]
        s = np.sqrt((o * o).sum(1).mean())
        np.testing.assert_allclose(X[i, :48], (o / s).ravel(), atol=1e-6)
        np.testing.assert_allclose(X[i, 48:51], (p64[i] - c) / R, atol=1e-12)
        assert np.all(X[i, 51:] == 0)
