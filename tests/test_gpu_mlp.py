"""The warm-start network's CUDA kernels (tensor-core forward and backward,
Adam, patch features) against the FP64 reference in oracle/mlp.py."""
import numpy as np
import pytest

import synth
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture
def torch():
    return pytest.importorskip("torch")


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_features_match_reference(dwglib):
    p, _ = synth.torus(3000, seed=4, noise=0.002)
    h = dwglib.dwg_create(p)
    try:
        X = np.zeros((len(p), 64), np.float32)
        dwglib.dwg_mlp_features(h, X)
    finally:
        dwglib.dwg_destroy(h)
    ref = mlp.features(p)
    close = np.all(np.abs(X - ref) <= 1e-5 + 1e-5 * np.abs(ref), axis=1)
    assert close.mean() >= 0.999, close.mean()


@pytest.mark.parametrize("B", [1, 15, 16, 64, 127, 128, 129, 1000, 4097, 200003])
def test_forward_matches_bf16_reference(dwglib, torch, B):
    """The tcgen05 forward: single rows, partial and whole 128-row tiles, and
    more tiles than the persistent grid has CTAs."""
    theta = mlp.init_params(1)
    X = synth.normal(2, 1, B * 64).reshape(B, 64)
    Y = torch.zeros((B, 3), dtype=torch.float32, device="cuda")
    dwglib.dwg_mlp_forward(_dev(torch, theta), _dev(torch, X), Y)
    ref, _ = mlp.forward(theta.astype(np.float32), X.astype(np.float32), bf16=True)
    err = np.abs(Y.cpu().numpy() - ref)
    assert err.max() <= 2e-2 * max(1.0, np.abs(ref).max()), err.max()


@pytest.mark.parametrize("B", [16, 300, 5000])
def test_gradient_matches_bf16_reference(dwglib, torch, B):
    theta = mlp.init_params(3)
    X = synth.normal(4, 1, B * 64).reshape(B, 64)
    T = synth.normal(4, 2, B * 3).reshape(B, 3)
    grad = torch.zeros(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = dwglib.dwg_mlp_grad(_dev(torch, theta), _dev(torch, X), _dev(torch, T), grad)
    L, g = mlp.loss_and_grad(theta.astype(np.float32), X.astype(np.float32),
                             T.astype(np.float32), bf16=True)
    assert loss == pytest.approx(L, rel=1e-2)
    gg = grad.cpu().numpy()
    for name, (o, k) in _slices().items():
        ref = g[o:o + k]
        assert np.abs(gg[o:o + k] - ref).max() <= 3e-2 * np.abs(ref).max() + 1e-7, name


def _slices():
    out, o = {}, 0
    for name, shape in mlp.SIZES:
        k = int(np.prod(shape))
        out[name] = (o, k)
        o += k
    return out


def test_adam_training_reduces_the_loss(dwglib, torch):
    B = 4096
    X = synth.normal(5, 1, B * 64).reshape(B, 64)
    Wt = synth.normal(5, 3, 64 * 3).reshape(64, 3) / 8
    T = np.tanh(X @ Wt)
    P = _dev(torch, mlp.init_params(7))
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    g = torch.zeros_like(P)
    dX, dT = _dev(torch, X), _dev(torch, T)
    first = dwglib.dwg_mlp_grad(P, dX, dT, g)
    for step in range(1, 301):
        dwglib.dwg_mlp_grad(P, dX, dT, g)
        dwglib.dwg_mlp_adam(P, g, m, v, step, 3e-3)
    last = dwglib.dwg_mlp_grad(P, dX, dT, g)
    assert last < 0.2 * first, (first, last)


def test_learned_init_is_the_normalised_network_output(dwglib, torch):
    p, _ = synth.sphere(2000, seed=6)
    theta = mlp.init_params(8).astype(np.float32)
    h = dwglib.dwg_create(p)
    try:
        X = np.zeros((len(p), 64), np.float32)
        dwglib.dwg_mlp_features(h, X)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_LEARNED, 1, theta)
        n0 = np.zeros((len(p), 3), np.float32)
        dwglib.dwg_get_normals(h, n0)
    finally:
        dwglib.dwg_destroy(h)
    Y = torch.zeros((len(p), 3), dtype=torch.float32, device="cuda")
    dwglib.dwg_mlp_forward(_dev(torch, theta), _dev(torch, X), Y)
    y = Y.cpu().numpy()
    ref = y / np.linalg.norm(y, axis=1, keepdims=True)
    np.testing.assert_allclose(n0, ref, atol=1e-6)


@pytest.mark.parametrize("shape", ["sphere", "ellipsoid"])
def test_shipped_warm_start_converges_in_fewer_iterations(dwglib, shape):
    """What the trained network gains over the method without it: from the
    shipped weights the orientation reaches the same final agreement with
    the analytic normals in at most half the iterations of random normals
    (mean-change rule, same tolerance)."""
    from paper_2405_13839_gb300 import train_init
    params = np.load(train_init.DEFAULT_WEIGHTS).astype(np.float32)
    n = 40000
    if shape == "sphere":
        p, nt = synth.sphere(n, seed=21)
    else:
        q, nt = synth.ellipsoid_points(n, [1.0, 0.6, 0.35], seed=22, stream=71)
        p = q.astype(np.float32)
    res = {}
    for init in ("random", "learned"):
        h = dwglib.dwg_create(p)
        try:
            dwglib.dwg_set_params(h, 1, 0.5 * 2.0 / np.sqrt(n), 10.0, 100, 0.1)
            dwglib.dwg_set_update(h, 7, 10, dwglib.DWG_UPDATE_LEVELSET)
            dwglib.dwg_set_convergence(h, dwglib.DWG_CONV_MEAN)
            if init == "learned":
                dwglib.dwg_set_init(h, dwglib.DWG_INIT_LEARNED, 1, params)
            else:
                dwglib.dwg_set_init(h, dwglib.DWG_INIT_RANDOM, 1)
            out = np.zeros((n, 3), np.float32)
            rc, it = dwglib.dwg_orient(h, out)
        finally:
            dwglib.dwg_destroy(h)
        d = np.sum(out * nt, axis=1)
        res[init] = (rc, it, float(np.mean(np.sign(d.sum()) * d > 0)))
    assert res["learned"][0] == dwglib.DWG_OK and res["random"][0] == dwglib.DWG_OK, res
    assert res["learned"][2] >= 0.999 and res["learned"][2] >= res["random"][2] - 1e-4, res
    assert 2 * res["learned"][1] <= res["random"][1], res
