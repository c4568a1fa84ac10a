"""The modified Poisson kernel (Sec. 5.2, "Poisson Kernels"): clamp radii,
evaluation and orientation of the CUDA library against the FP64 oracle,
through the C ABI.

Tolerances as for the softened kernel (w: 1e-5, relative above 1; grad w: 1e-5
relative plus 16 ulp of S_g, the sum of the gradient terms' magnitudes with
rho_j = max(|p_j - q|, delta_j)).  Both sides decide "inside the radius" in
float32 the same way, so the gradient's jump at |p_j - q| = delta_j cannot
split them.  Radii: FP64 on both sides from the same float32 points, equal
to the float32 rounding (relative 1e-6), except where the k-th and (k+1)-th
neighbours tie in float32 only (at most 0.1 % of the points)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def s_g_clamp(points, normals, weights, queries, delta):
    p = np.asarray(points, np.float64)
    m = np.asarray(weights, np.float64)[:, None] * np.asarray(normals, np.float64) / (4 * np.pi)
    mn = np.linalg.norm(m, axis=1)
    out = np.zeros(len(queries))
    for i0 in range(0, len(queries), 256):
        q = np.asarray(queries[i0:i0 + 256], np.float64)
        r2 = ((p[None, :, :] - q[:, None, :]) ** 2).sum(-1)
        rho2 = np.maximum(r2, delta[None, :] ** 2)
        out[i0:i0 + 256] = 4 * (mn[None, :] * rho2 ** -1.5).sum(1)
    return out


def check_wg(w, g, wo, go, sg):
    # w is 1e-5 absolute, relative where |w| > 1 (a query inside a heavy
    # source's radius sees |m| / delta^2, thousands for a one-point cloud)
    dw = np.abs(w - wo) / np.maximum(1.0, np.abs(wo))
    assert dw.max() <= 1e-5, f"max |dw| {dw.max():.3e}"
    gn = np.linalg.norm(go, axis=1)
    tol = 1e-5 * np.maximum(1.0, gn) + 16 * U32 * sg
    dg = np.abs(g - go).max(axis=1)
    bad = dg > tol
    assert not bad.any(), f"{bad.sum()} gradients off; worst ratio {(dg / tol).max():.3f}"


def _torus(n, seed):
    p, nt = synth.torus(n, seed=seed, noise=0.003)
    area = 4 * np.pi ** 2 * 0.3
    return p, nt, np.full(n, area / n, np.float32)


@pytest.mark.parametrize("k,vmin,vmax", [(10, 0.0, 0.0), (10, 0.02, 0.05), (4, 0.001, 0.3),
                                         (10, 0.2, 0.3), (31, 1e-4, 0.01)])
def test_clamp_radii_match_oracle(dwglib, oracle_mod, k, vmin, vmax):
    p, _, _ = _torus(6000, 1)
    h = dwglib.dwg_create(p)
    try:
        d = np.zeros(len(p), np.float32)
        dwglib.dwg_set_regularization(h, dwglib.DWG_REG_CLAMP, k, vmin, vmax, d)
    finally:
        dwglib.dwg_destroy(h)
    if vmin == 0.0 and vmax == 0.0:
        ext = float(np.max(p.max(axis=0).astype(np.float64) - p.min(axis=0)))
        vmin, vmax = 0.0015 * ext, 0.015 * ext
    ref = oracle_mod.clamp_radii(p, k, vmin, vmax)
    bad = np.abs(d - ref) > 1e-6 * ref
    assert bad.mean() <= 1e-3, (bad.sum(), np.max(np.abs(d / ref - 1)))
    assert np.all(d >= np.float32(vmin) * (1 - 1e-6)) and np.all(d <= np.float32(vmax) * (1 + 1e-6))


@pytest.mark.parametrize("n", [1, 33, 1000, 4097])
@pytest.mark.parametrize("kernel,lam", [(0, 0.0), (1, 10.0), (1, 100.0)])
def test_clamp_eval_matches_oracle(dwglib, oracle_mod, n, kernel, lam):
    p, _, a = _torus(n, n)
    n0 = synth.random_unit_normals(n, seed=3).astype(np.float32)
    vmin, vmax = 0.01, 0.08
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, kernel, 0.01, lam, 30, 0.1)
        dwglib.dwg_set_regularization(h, dwglib.DWG_REG_CLAMP, 10, vmin, vmax)
        dwglib.dwg_set_normals(h, n0)
        # the points, random queries, queries close to (inside the radius of) points
        q = np.vstack([p, synth.uniform_box(257, [-1.5, -1.5, -0.6], [1.5, 1.5, 0.6], seed=5),
                       p[: min(n, 50)] + np.float32(3e-3)]).astype(np.float32)
        w = np.zeros(len(q), np.float32)
        g = np.zeros((len(q), 3), np.float32)
        dwglib.dwg_eval_gwn(h, q, w, g)
        w2 = np.zeros(len(q), np.float32)
        dwglib.dwg_eval_gwn(h, q, w2, None)
    finally:
        dwglib.dwg_destroy(h)
    delta = oracle_mod.clamp_radii(p, 10, vmin, vmax)
    wo, go = oracle_mod.gwn(p, n0, a, q, kernel=kernel, lam=lam, delta=delta)
    check_wg(w, g, wo, go, s_g_clamp(p, n0, a, q, delta))
    assert np.max(np.abs(w2 - wo) / np.maximum(1.0, np.abs(wo))) <= 1e-5


def test_clamp_with_duplicates(dwglib, oracle_mod):
    p, _, a = _torus(600, 7)
    p = np.vstack([p, p[10:13], p[10:11]]).astype(np.float32)
    a = np.append(a, a[:4]).astype(np.float32)
    n0 = synth.random_unit_normals(len(p), seed=8).astype(np.float32)
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_regularization(h, dwglib.DWG_REG_CLAMP, 10, 0.02, 0.2)
        dwglib.dwg_set_normals(h, n0)
        w = np.zeros(len(p), np.float32)
        g = np.zeros((len(p), 3), np.float32)
        dwglib.dwg_eval_gwn(h, p, w, g)
        dwglib.dwg_set_update(h, 5, 10, dwglib.DWG_UPDATE_LEVELSET)
        ws = np.zeros(len(p), np.float32)
        gs = np.zeros((len(p), 3), np.float32)
        dwglib.dwg_step(h, ws, gs)
    finally:
        dwglib.dwg_destroy(h)
    delta = oracle_mod.clamp_radii(p, 10, 0.02, 0.2)
    wo, go = oracle_mod.gwn(p, n0, a, p, delta=delta)
    sg = s_g_clamp(p, n0, a, p, delta)
    check_wg(w, g, wo, go, sg)
    check_wg(ws, gs, wo, go, sg)


def _agreement(n, nt):
    d = np.sum(n * nt, axis=1)
    return float(np.mean((1.0 if d.sum() >= 0 else -1.0) * d > 0))


@pytest.mark.parametrize("kernel,lam", [(0, 0.0), (1, 10.0)])
def test_clamp_orientation_matches_oracle(dwglib, oracle_mod, kernel, lam):
    n = 1500
    p, nt, a = _torus(n, 11)
    n0 = synth.random_unit_normals(n, seed=2).astype(np.float32)
    vmin, vmax = 0.01, 0.1
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, kernel, 0.01, lam, 40, 0.5)
        dwglib.dwg_set_update(h, 5, 10, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_convergence(h, dwglib.DWG_CONV_MEAN)
        dwglib.dwg_set_regularization(h, dwglib.DWG_REG_CLAMP, 10, vmin, vmax)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, n0)
        out = np.zeros((n, 3), np.float32)
        rc, iters = dwglib.dwg_orient(h, out)
    finally:
        dwglib.dwg_destroy(h)
    delta = oracle_mod.clamp_radii(p, 10, vmin, vmax)
    r = oracle_mod.orient(p, a, n0, oracle_mod.params(kernel=kernel, lam=lam, depth=5,
                                                      max_iters=40, tol=0.5, rule=1,
                                                      delta=delta))
    assert _agreement(out, r["normals"]) >= 0.999
    assert abs(iters - r["iters"]) <= 3, (iters, r["iters"])
    assert _agreement(out, nt) >= 0.99


def test_switching_back_to_softening_is_exact(dwglib):
    p, _, a = _torus(3000, 12)
    n0 = synth.random_unit_normals(len(p), seed=4).astype(np.float32)
    q = synth.uniform_box(300, [-1.5] * 3, [1.5] * 3, seed=6)
    res = []
    for clamp_first in (False, True):
        h = dwglib.dwg_create(p)
        try:
            dwglib.dwg_set_weights(h, a)
            dwglib.dwg_set_params(h, 0, 0.02, 0.0, 30, 0.1)
            dwglib.dwg_set_normals(h, n0)
            if clamp_first:
                dwglib.dwg_set_regularization(h, dwglib.DWG_REG_CLAMP, 10, 0.01, 0.1)
                dwglib.dwg_eval_gwn(h, q, np.zeros(len(q), np.float32))
                dwglib.dwg_set_regularization(h, dwglib.DWG_REG_SOFTEN)
            w = np.zeros(len(q), np.float32)
            g = np.zeros((len(q), 3), np.float32)
            dwglib.dwg_eval_gwn(h, q, w, g)
            res.append((w, g))
        finally:
            dwglib.dwg_destroy(h)
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_clamp_refusals(dwglib):
    p, _, _ = _torus(2000, 13)
    h = dwglib.dwg_create(p)
    try:
        for args in ((0, 0.01, 0.1), (32, 0.01, 0.1), (10, 0.1, 0.01), (10, -1.0, 0.1)):
            with pytest.raises(dwglib.DWGError) as e:
                dwglib.dwg_set_regularization(h, dwglib.DWG_REG_CLAMP, *args)
            assert e.value.code == dwglib.DWG_ERR_INVALID, args
        dwglib.dwg_set_regularization(h, dwglib.DWG_REG_CLAMP, 10, 0.01, 0.1)
        with pytest.raises(dwglib.DWGError) as e:
            dwglib.dwg_autotune(h, dwglib.DWG_TUNE_SHAPES)
        assert e.value.code == dwglib.DWG_ERR_STATE
    finally:
        dwglib.dwg_destroy(h)
    hb = dwglib.dwg_create_batch(np.vstack([p, p + 3]).astype(np.float32),
                                 np.array([0, len(p), 2 * len(p)], np.int64))
    try:
        with pytest.raises(dwglib.DWGError) as e:
            dwglib.dwg_set_regularization(hb, dwglib.DWG_REG_CLAMP, 10, 0.01, 0.1)
        assert e.value.code == dwglib.DWG_ERR_STATE
    finally:
        dwglib.dwg_destroy(hb)


@pytest.mark.parametrize("group", [0, 1])
@pytest.mark.parametrize("grad,kernel,lam", [(True, 1, 30.0), (False, 1, 30.0), (True, 0, 0.0)])
def test_clamp_tree_walk_matches_oracle_tree(dwglib, oracle_mod, group, grad, kernel, lam):
    """Barnes-Hut with the modified kernel at arbitrary queries: the per-query
    walk (with either test form set: arbitrary queries have no group lists,
    and the modified kernel's fallback is the per-query walk) against the
    oracle's per-query tree with the same radii and opening rule."""
    n = 30000
    p, _, a = _torus(n, 17)
    n0 = synth.random_unit_normals(n, seed=5).astype(np.float32)
    vmin, vmax = 0.005, 0.05
    q = np.vstack([p[:4096], synth.uniform_box(2048, [-1.4, -1.4, -0.5], [1.4, 1.4, 0.5],
                                                seed=9)]).astype(np.float32)
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, kernel, 0.01, lam, 30, 0.1)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.4)
        dwglib.dwg_set_tuning(h, tree_leaf=32, tree_group=group)
        dwglib.dwg_set_regularization(h, dwglib.DWG_REG_CLAMP, 10, vmin, vmax)
        dwglib.dwg_set_normals(h, n0)
        w = np.zeros(len(q), np.float32)
        g = np.zeros((len(q), 3), np.float32) if grad else None
        dwglib.dwg_eval_gwn(h, q, w, g)
    finally:
        dwglib.dwg_destroy(h)
    delta = oracle_mod.clamp_radii(p, 10, vmin, vmax)
    beta = float(1.0 / np.float32(0.4))
    out = oracle_mod.tree_gwn(p, n0, a, q, kernel=kernel, lam=lam, beta=beta, bucket=32,
                              delta=delta, grad=grad)
    wo, go = (out if grad else (out, None))
    dw = np.abs(w - wo) / np.maximum(1.0, np.abs(wo))
    assert dw.max() <= 1e-5, dw.max()
    if grad:
        sg = s_g_clamp(p, n0, a, q, delta)
        tol = 1e-5 * np.maximum(1.0, np.linalg.norm(go, axis=1)) + 16 * U32 * sg
        assert np.all(np.abs(g - go).max(axis=1) <= tol)


@pytest.mark.parametrize("kernel,lam,leaf", [(1, 30.0, 32), (0, 0.0, 16)])
def test_clamp_group_lists_step_matches_oracle_group_tree(dwglib, oracle_mod, kernel, lam, leaf):
    """One iteration on the Barnes-Hut path with the group test and the
    modified kernel evaluates the group lists (w and grad w at the points, in
    Morton order, 64 per group): the oracle's group tree with the same radii
    on the Morton-ordered points."""
    n = 20000
    p, _, a = _torus(n, 23)
    nrm = synth.random_unit_normals(n, seed=13).astype(np.float32)
    vmin, vmax = 0.005, 0.05
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, kernel, 0.01, lam, 30, 0.1)
        dwglib.dwg_set_update(h, 6, 10, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.5)
        dwglib.dwg_set_tuning(h, tree_group=1, tree_leaf=leaf)
        dwglib.dwg_set_regularization(h, dwglib.DWG_REG_CLAMP, 10, vmin, vmax)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, nrm)
        w = np.zeros(n, np.float32)
        g = np.zeros((n, 3), np.float32)
        dwglib.dwg_step(h, w, g)
    finally:
        dwglib.dwg_destroy(h)
    delta = oracle_mod.clamp_radii(p, 10, vmin, vmax)
    order = oracle_mod.morton_order(p)
    wo_s, go_s = oracle_mod.tree_gwn_group(p, nrm, a, p[order], kernel=kernel, lam=lam,
                                           beta=2.0, bucket=leaf, group=64, delta=delta)
    wo = np.empty(n)
    go = np.empty((n, 3))
    wo[order] = wo_s
    go[order] = go_s
    sel = np.arange(0, n, 7)
    check_wg(w[sel], g[sel], wo[sel], go[sel], s_g_clamp(p, nrm, a, p[sel], delta))


def test_clamp_tree_orientation(dwglib, oracle_mod):
    """The whole iteration on the Barnes-Hut path with the modified kernel
    orients the torus."""
    n = 40000
    p, nt, a = _torus(n, 19)
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, 1, 0.01, 30.0, 60, 0.5)
        dwglib.dwg_set_update(h, 7, 10, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_convergence(h, dwglib.DWG_CONV_MEAN)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.5)
        dwglib.dwg_set_regularization(h, dwglib.DWG_REG_CLAMP, 10, 0.0, 0.0)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_RANDOM, 3)
        out = np.zeros((n, 3), np.float32)
        rc, it = dwglib.dwg_orient(h, out)
        st = dwglib.dwg_get_stats(h)
    finally:
        dwglib.dwg_destroy(h)
    assert rc == dwglib.DWG_OK, it
    assert _agreement(out, nt) >= 0.99
    assert st["interactions"] > 0
