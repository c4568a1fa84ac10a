"""Autotuner and the tunable settings it chooses between.

Every compiled evaluator shape must give the oracle's w and grad w (the
shape only changes the order of the FP32 additions); every Barnes-Hut leaf
size must make the oracle's opening decisions (the oracle's tree with the
same leaf size); the tuner must respect its error budget, apply what it
reports, and read its cache."""
import os

import numpy as np
import pytest

import synth
from test_gpu_parity import check_wg, make_cloud, s_g

pytestmark = pytest.mark.gpu

SHAPES_GRAD = [(2, 128), (1, 128), (3, 128), (1, 256), (2, 256)]
SHAPES_W = [(4, 128), (2, 128), (3, 128), (6, 128), (2, 256), (3, 256), (4, 256), (1, 128),
            (1, 256), (2, 64)]


@pytest.fixture
def handle(dwglib):
    made = []

    def make(points):
        h = dwglib.dwg_create(points)
        made.append(h)
        return h

    yield make
    for h in made:
        dwglib.dwg_destroy(h)


@pytest.mark.parametrize("kernel,lam", [(0, 0.0), (1, 10.0)])
@pytest.mark.parametrize("shape", SHAPES_GRAD)
def test_every_gradient_shape_matches_oracle(dwglib, oracle_mod, handle, shape, kernel, lam):
    n = 3001  # several query tiles of every shape and a ragged tail
    p, _, a, eps = make_cloud(n, seed=21)
    nrm = synth.random_unit_normals(n, seed=22).astype(np.float32)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_ALLPAIRS, 0.5)
    dwglib.dwg_set_tuning(h, points_pairs=shape[0], points_threads=shape[1])
    assert dwglib.dwg_get_tuning(h)["points_pairs"] == shape[0]
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, nrm)
    w = np.zeros(n, np.float32)
    g = np.zeros((n, 3), np.float32)
    dwglib.dwg_step(h, w, g)
    wo, go = oracle_mod.gwn(p, nrm, a, p, kernel=kernel, eps=eps, lam=lam)
    check_wg(w, g, wo, go, s_g(p, nrm, a, p, eps))


@pytest.mark.parametrize("kernel,lam", [(0, 0.0), (1, 10.0)])
@pytest.mark.parametrize("shape", SHAPES_W)
def test_every_w_shape_matches_oracle(dwglib, oracle_mod, handle, shape, kernel, lam):
    """The w-only evaluator (the one the level-set step runs at the leaf
    corners), through dwg_eval_gwn without a gradient output: 7,001 queries
    span several tiles of every shape and end in a ragged tile."""
    n = 2500
    p, _, a, eps = make_cloud(n, seed=31, kind="sphere")
    nrm = synth.random_unit_normals(n, seed=32).astype(np.float32)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_ALLPAIRS, 0.5)
    dwglib.dwg_set_tuning(h, corners_pairs=shape[0], corners_threads=shape[1])
    dwglib.dwg_set_normals(h, nrm)
    q = np.vstack([p, synth.uniform_box(7001 - n, [-1.3] * 3, [1.3] * 3, seed=34)])
    q = np.ascontiguousarray(q, dtype=np.float32)
    w = np.zeros(len(q), np.float32)
    dwglib.dwg_eval_gwn(h, q, w)
    wo = oracle_mod.gwn(p, nrm, a, q, kernel=kernel, eps=eps, lam=lam, grad=False)
    assert np.abs(w - wo).max() <= 1e-5
    # and one level-set step with this shape runs and reports finite values
    dwglib.dwg_set_update(h, 5, 10, dwglib.DWG_UPDATE_LEVELSET)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, nrm)
    iso, stat = dwglib.dwg_step(h)
    assert np.isfinite(iso) and np.isfinite(stat)


@pytest.mark.parametrize("leaf", [16, 32, 64, 128])
def test_tree_leaf_sizes_match_oracle_tree(dwglib, oracle_mod, handle, leaf):
    n = 30000
    p, _ = synth.torus(n, seed=5, noise=0.004)
    a = np.full(n, 4 * np.pi ** 2 * 0.3 / n, np.float32)
    nrm = synth.random_unit_normals(n, seed=6).astype(np.float32)
    eps = synth.default_eps(4 * np.pi ** 2 * 0.3, n)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, 0, eps, 0.0, 30, 0.1)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.5)
    dwglib.dwg_set_tuning(h, tree_leaf=leaf, tree_group=0)
    dwglib.dwg_set_normals(h, nrm)
    sel = np.unique((synth.uniform(8, leaf, 1200) * n).astype(np.int64))
    q = np.vstack([p[sel], synth.uniform_box(300, [-1.5, -1.5, -0.6], [1.5, 1.5, 0.6],
                                             seed=leaf)]).astype(np.float32)
    w = np.zeros(len(q), np.float32)
    g = np.zeros((len(q), 3), np.float32)
    dwglib.dwg_eval_gwn(h, q, w, g)
    cnt_gpu = dwglib.dwg_get_stats(h)["interactions_eval"]
    wo, go, cnt = oracle_mod.tree_gwn(p, nrm, a, q, eps=eps, beta=2.0, bucket=leaf,
                                      want_count=True)
    check_wg(w, g, wo, go, s_g(p, nrm, a, q, eps))
    assert cnt_gpu == cnt.sum() + len(sel)


def test_set_tuning_rejects_unknown_settings(dwglib, handle):
    p, _ = synth.sphere(500, seed=1)
    h = handle(p)
    for bad in (dict(points_pairs=5), dict(corners_threads=64), dict(tree_leaf=24),
                dict(theta=0.0), dict(path=dwglib.DWG_PATH_AUTO), dict(tree_group=2)):
        with pytest.raises(dwglib.DWGError) as e:
            dwglib.dwg_set_tuning(h, **bad)
        assert e.value.code == dwglib.DWG_ERR_INVALID, bad


def test_autotune_shapes_applies_a_compiled_shape(dwglib, oracle_mod, handle, tmp_path):
    n = 20000
    p, _, a, eps = make_cloud(n, seed=41)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, 0, eps, 0.0, 30, 0.1)
    dwglib.dwg_set_update(h, 6, 10, dwglib.DWG_UPDATE_LEVELSET)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_ALLPAIRS, 0.5)
    cache = str(tmp_path / "tune.jsonl")
    t = dwglib.dwg_autotune(h, dwglib.DWG_TUNE_SHAPES, 1e-3, cache)
    assert (t["points_pairs"], t["points_threads"]) in SHAPES_GRAD
    assert (t["corners_pairs"], t["corners_threads"]) in SHAPES_W
    assert t["path"] == dwglib.DWG_PATH_ALLPAIRS and t["from_cache"] == 0
    assert t["ms_points"] > 0 and t["ms_corners"] > 0
    assert dwglib.dwg_get_tuning(h)["corners_pairs"] == t["corners_pairs"]
    # results after tuning still match the oracle
    nrm = synth.random_unit_normals(n, seed=42).astype(np.float32)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, nrm)
    w = np.zeros(n, np.float32)
    g = np.zeros((n, 3), np.float32)
    dwglib.dwg_step(h, w, g)
    sel = np.arange(0, n, 37)
    wo, go = oracle_mod.gwn(p, nrm, a, p[sel], eps=eps)
    check_wg(w[sel], g[sel], wo, go, s_g(p, nrm, a, p[sel], eps))
    # a second handle on the same problem takes the cached result
    h2 = handle(p)
    dwglib.dwg_set_weights(h2, a)
    dwglib.dwg_set_params(h2, 0, eps, 0.0, 30, 0.1)
    dwglib.dwg_set_update(h2, 6, 10, dwglib.DWG_UPDATE_LEVELSET)
    dwglib.dwg_set_tree(h2, dwglib.DWG_PATH_ALLPAIRS, 0.5)
    t2 = dwglib.dwg_autotune(h2, dwglib.DWG_TUNE_SHAPES, 1e-3, cache)
    assert t2["from_cache"] == 1
    for k in ("points_pairs", "points_threads", "corners_pairs", "corners_threads"):
        assert t2[k] == t[k]
    assert len(open(cache).read().strip().splitlines()) == 1


@pytest.mark.parametrize("budget", [1e-2, 3e-3])
def test_autotune_tree_meets_the_error_budget(dwglib, oracle_mod, handle, budget):
    n = 60000
    p, _ = synth.torus(n, seed=7, noise=0.003)
    area = 4 * np.pi ** 2 * 0.3
    a = np.full(n, area / n, np.float32)
    eps = synth.default_eps(area, n)
    nrm = synth.random_unit_normals(n, seed=8).astype(np.float32)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, 0, eps, 0.0, 30, 0.1)
    dwglib.dwg_set_update(h, 7, 10, dwglib.DWG_UPDATE_LEVELSET)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.5)
    dwglib.dwg_set_normals(h, nrm)
    t = dwglib.dwg_autotune(h, dwglib.DWG_TUNE_TREE, budget, None)
    assert t["path"] == dwglib.DWG_PATH_TREE
    assert t["tree_leaf"] in (16, 32, 64, 128)
    assert 0.2 <= t["theta"] <= 0.9
    assert t["w_err"] <= budget
    # the applied settings are the oracle tree's, and the far field stays
    # near the budget on fresh queries (the budget was met on a sample)
    sel = np.unique((synth.uniform(9, 1, 1500) * n).astype(np.int64))
    q = p[sel]
    w = np.zeros(len(q), np.float32)
    dwglib.dwg_eval_gwn(h, q, w)
    beta = float(np.float32(1) / np.float32(t["theta"]))
    if t["tree_group"]:
        wt = oracle_mod.tree_gwn_group(p, nrm, a, q, eps=eps, beta=beta, bucket=t["tree_leaf"],
                                       group=64, grad=False)
    else:
        wt = oracle_mod.tree_gwn(p, nrm, a, q, eps=eps, beta=beta, bucket=t["tree_leaf"],
                                 grad=False)
    assert np.abs(w - wt).max() <= 1e-5
    we = oracle_mod.gwn(p, nrm, a, q, eps=eps, grad=False)
    assert np.abs(w - we).max() <= 4 * budget


def test_autotune_auto_path_picks_a_path_and_orients(dwglib, handle):
    n = 40000
    p, nt = synth.torus(n, seed=2)
    area = 4 * np.pi ** 2 * 0.3
    h = handle(p)
    dwglib.dwg_set_weights(h, np.full(n, area / n, np.float32))
    dwglib.dwg_set_params(h, 1, synth.default_eps(area, n), 10.0, 40, 0.1)
    dwglib.dwg_set_update(h, 7, 10, dwglib.DWG_UPDATE_LEVELSET)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_AUTO, 0.5)
    t = dwglib.dwg_autotune(h, dwglib.DWG_TUNE_SHAPES | dwglib.DWG_TUNE_TREE, 1e-3, None)
    assert t["path"] in (dwglib.DWG_PATH_ALLPAIRS, dwglib.DWG_PATH_TREE)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_RANDOM, 1)
    out = np.zeros((n, 3), np.float32)
    dwglib.dwg_orient(h, out)
    d = np.sum(out * nt, axis=1)
    assert np.mean(np.sign(d.sum()) * d > 0) >= 0.999


def test_autotune_tree_rejects_an_unreachable_budget(dwglib, handle):
    """A first-order far field cannot reach 1e-9 at any opening angle down to
    0.2: on the tree path the tuner reports it instead of choosing one."""
    n = 20000
    p, _ = synth.torus(n, seed=3)
    h = handle(p)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.5)
    before = dwglib.dwg_get_tuning(h)
    with pytest.raises(dwglib.DWGError) as e:
        dwglib.dwg_autotune(h, dwglib.DWG_TUNE_TREE, 1e-9, None)
    assert e.value.code == dwglib.DWG_ERR_INVALID
    assert dwglib.dwg_get_tuning(h) == before


def test_autotune_relative_budget_scales_with_the_weights(dwglib, handle):
    """DWG_TUNE_RELATIVE: the budget follows the winding number's scale
    estimated from the spacing, so with a_i = 1 (w inside about n / area)
    and a_i = area / n (w inside about 1) the tuner picks the same settings."""
    n = 30000
    p, nt = synth.sphere(n, seed=11)
    res = []
    for a in (np.ones(n, np.float32), np.full(n, 4 * np.pi / n, np.float32)):
        h = handle(p)
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.5)
        dwglib.dwg_set_normals(h, nt.astype(np.float32))
        t = dwglib.dwg_autotune(h, dwglib.DWG_TUNE_TREE | dwglib.DWG_TUNE_RELATIVE, 0.02, None)
        res.append(t)
        scale = float(a[0]) * n / (4 * np.pi)  # w inside for this weighting
        assert t["w_err"] <= 0.05 * scale, (t, scale)
    assert (res[0]["tree_leaf"], res[0]["theta"], res[0]["tree_group"]) == \
        (res[1]["tree_leaf"], res[1]["theta"], res[1]["tree_group"])
