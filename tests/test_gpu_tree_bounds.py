"""The library's Barnes-Hut far field (Sec. 5.2, "Octree Traversal") against
the exact FP64 sum of the oracle, within the a-priori first-order bound.

The tree the library built is read back (dwg_get_tree) and checked against
the points: every node's area and centre recomputed from its range, its
radius bounding every point's distance from the centre, the traversal
records holding the float centres and the opening radius of the paper's
test (beta r; with the modified kernel max(beta r, r + the node's largest
clamp radius)).  Then, per query,

  |w_gpu - w_exact| <= sum over the far nodes of oracle.far_field_bound + tol,
  |g_gpu - g_exact| <= the same for the gradient + tol,

with the far nodes those of the opening test applied to the verified tree in
FP64 (nodes on the test's boundary counted as far: opening them can only
lower the bound), and tol the exact path's rounding allowance.  This holds
for the per-query walk and, because a node far from a group's box is far
from each of its queries, for the group form and its interaction lists.
For the per-query walk the GPU also matches, to the exact path's tolerance,
the FP64 value of that decomposition (leaves opened point by point, far
nodes as one dipole), which pins every opening decision up to the
boundary nodes' bounds."""
import json

import numpy as np
import pytest

import synth
import bh_check
from test_gpu_parity import s_g, U32
from test_gpu_clamp import s_g_clamp
from test_gpu_tree import _term_sums

pytestmark = pytest.mark.gpu

AREA = 4 * np.pi ** 2 * 0.3


def _cloud(n, seed):
    p, _ = synth.torus(n, seed=seed, noise=0.004)
    a = np.full(n, AREA / n, np.float32)
    nrm = synth.random_unit_normals(n, seed=seed + 1).astype(np.float32)
    return p, a, nrm


def _queries(p, n, seed):
    sel = np.unique((synth.uniform(7, seed, min(n, 1500)) * n).astype(np.int64))
    box = synth.uniform_box(500, [-1.5, -1.5, -0.6], [1.5, 1.5, 0.6], seed=seed)
    return np.vstack([p[sel], box]).astype(np.float32)


def _tree_checks(dwglib, h, p, a, q, beta, lam, eps, delta=None):
    T = dwglib.dwg_get_tree(h, len(p))
    bh_check.verify_tree(T, p, a)
    bh_check.verify_records(T, beta, delta, rtol=1e-6 if delta is None else 1e-5)
    far, amb, leaves = bh_check.walk(T, q, beta, delta)
    bw, bg = bh_check.far_bound(T, q, far, lam=lam, eps=eps)
    return T, far, amb, leaves, bw, bg


def _assert_within(w, g, we, ge, bw, bg, tol_w, tol_g, what):
    ew = np.abs(w - we)
    bad = ew > bw + tol_w
    assert not bad.any(), f"{what}: {bad.sum()} w beyond the bound; worst " \
                          f"{(ew / (bw + tol_w)).max():.3f}"
    if g is not None:
        eg = np.linalg.norm(g - ge, axis=1)
        bad = eg > bg + tol_g
        assert not bad.any(), f"{what}: {bad.sum()} grad beyond the bound; worst " \
                              f"{(eg / (bg + tol_g)).max():.3f}"


@pytest.mark.parametrize("kernel,lam,theta,leaf", [(0, 0.0, 0.5, 16), (0, 0.0, 1 / 2.3, 32),
                                                   (1, 10.0, 0.5, 16), (1, 100.0, 0.5, 32),
                                                   (1, 100.0, 0.7, 64)])
@pytest.mark.parametrize("group", [0, 1])
def test_tree_eval_within_the_bound_of_the_exact_sum(dwglib, oracle_mod, kernel, lam, theta,
                                                     leaf, group):
    n = 40000
    p, a, nrm = _cloud(n, 41 + leaf)
    eps = synth.default_eps(AREA, n)
    q = _queries(p, n, 43)
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, theta)
        dwglib.dwg_set_tuning(h, tree_group=group, tree_leaf=leaf)
        dwglib.dwg_set_normals(h, nrm)
        w = np.zeros(len(q), np.float32)
        g = np.zeros((len(q), 3), np.float32)
        dwglib.dwg_eval_gwn(h, q, w, g)
        beta = float(np.float32(1) / np.float32(theta))
        T, far, amb, leaves, bw, bg = _tree_checks(dwglib, h, p, a, q, beta, lam, eps)
    finally:
        dwglib.dwg_destroy(h)
    we, ge = oracle_mod.gwn(p, nrm, a, q, kernel=kernel, eps=eps, lam=lam)
    sg = s_g(p, nrm, a, q, eps)
    tol_g = 1e-5 * np.maximum(1.0, np.linalg.norm(ge, axis=1)) + 16 * U32 * sg
    _assert_within(w, g, we, ge, bw, bg, 1e-5, tol_g, "tree vs exact")
    assert len(far[0]) > 10 * len(q)   # the far field carries the sum
    if group == 0:
        # the per-query walk equals the FP64 value of its decomposition
        wv, gv = bh_check.decomposition_value(T, p, nrm, a, q, far, leaves, kernel=kernel,
                                              lam=lam, eps=eps)
        ab_w, ab_g = bh_check.far_bound(T, q, amb, lam=lam, eps=eps)
        _assert_within(w, g, wv, gv, ab_w, ab_g, 1e-5, tol_g, "tree vs its decomposition")


@pytest.mark.parametrize("kernel,lam,leaf", [(1, 30.0, 32), (0, 0.0, 16)])
def test_clamped_tree_within_the_bound_of_the_exact_sum(dwglib, oracle_mod, kernel, lam, leaf):
    """The modified kernel of Sec. 5.2: a node opens unless the query is
    beyond both beta r and r + its largest clamp radius, so a far node's
    terms are unclamped and the unsoftened bound applies."""
    n = 40000
    p, a, nrm = _cloud(n, 51)
    vmin, vmax = 0.005, 0.05
    q = _queries(p, n, 53)
    theta = 0.4
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, kernel, 0.01, lam, 30, 0.1)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, theta)
        dwglib.dwg_set_tuning(h, tree_leaf=leaf, tree_group=0)
        d_gpu = np.zeros(n, np.float32)
        dwglib.dwg_set_regularization(h, dwglib.DWG_REG_CLAMP, 10, vmin, vmax, d_gpu)
        dwglib.dwg_set_normals(h, nrm)
        w = np.zeros(len(q), np.float32)
        g = np.zeros((len(q), 3), np.float32)
        dwglib.dwg_eval_gwn(h, q, w, g)
        delta = oracle_mod.clamp_radii(p, 10, vmin, vmax)
        assert np.mean(np.abs(d_gpu - delta) > 1e-6 * delta) <= 1e-3
        beta = float(np.float32(1) / np.float32(theta))
        T, far, amb, leaves, bw, bg = _tree_checks(dwglib, h, p, a, q, beta, lam, 0.0, delta)
    finally:
        dwglib.dwg_destroy(h)
    we, ge = oracle_mod.gwn(p, nrm, a, q, kernel=kernel, lam=lam, delta=delta)
    sg = s_g_clamp(p, nrm, a, q, delta)
    tol_w = 1e-5 * np.maximum(1.0, np.abs(we))
    tol_g = 1e-5 * np.maximum(1.0, np.linalg.norm(ge, axis=1)) + 16 * U32 * sg
    _assert_within(w, g, we, ge, bw, bg, tol_w, tol_g, "clamped tree vs exact")
    wv, gv = bh_check.decomposition_value(T, p, nrm, a, q, far, leaves, kernel=kernel, lam=lam,
                                          delta=delta)
    ab_w, ab_g = bh_check.far_bound(T, q, amb, lam=lam)
    _assert_within(w, g, wv, gv, ab_w, ab_g, tol_w, tol_g, "clamped tree vs its decomposition")


@pytest.mark.parametrize("kernel,lam,leaf", [(0, 0.0, 16), (1, 10.0, 32), (1, 100.0, 64)])
def test_group_lists_step_within_the_bound(dwglib, oracle_mod, kernel, lam, leaf):
    """One iteration with the group test evaluates the interaction lists at
    the points: w and grad w at every 7th point within the bound."""
    n = 40000
    p, a, nrm = _cloud(n, 61)
    eps = synth.default_eps(AREA, n)
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
        dwglib.dwg_set_update(h, 6, 10, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.5)
        dwglib.dwg_set_tuning(h, tree_group=1, tree_leaf=leaf)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, nrm)
        w = np.zeros(n, np.float32)
        g = np.zeros((n, 3), np.float32)
        dwglib.dwg_step(h, w, g)
        sel = np.arange(0, n, 7)
        q = p[sel]
        T, far, amb, leaves, bw, bg = _tree_checks(dwglib, h, p, a, q, 2.0, lam, eps)
    finally:
        dwglib.dwg_destroy(h)
    we, ge = oracle_mod.gwn(p, nrm, a, q, kernel=kernel, eps=eps, lam=lam)
    sg = s_g(p, nrm, a, q, eps)
    tol_g = 1e-5 * np.maximum(1.0, np.linalg.norm(ge, axis=1)) + 16 * U32 * sg
    _assert_within(w[sel], g[sel], we, ge, bw, bg, 1e-5, tol_g, "group lists vs exact")


@pytest.mark.parametrize("group", [0, 1])
def test_full_size_metaballs_within_the_bound(dwglib, oracle_mod, group):
    """The 1,000,000-point metaballs workload in the benchmark's Barnes-Hut
    configuration (screened lambda 100, leaf 32, opening angle 0.4): with
    the group test, one step's interaction lists at 8 sampled groups of 64
    Morton-consecutive points; with the per-query test, dwg_eval_gwn at the
    same points.  a_i = 1 makes the terms large (w inside ~ n / area): the
    rounding allowance is 160 u sum |t| (flushes of at most 128 FP32
    additions folded into two-sums)."""
    W = synth.workload_metaballs1m()
    p, a, eps = W["points"], W["weights"], W["eps"]
    n = len(p)
    nrm = synth.random_unit_normals(n, seed=1).astype(np.float32)
    order = oracle_mod.morton_order(p)
    groups = np.unique((synth.uniform(4, 9, 8) * (n // 64)).astype(np.int64))
    idx = np.concatenate([order[64 * gi:64 * gi + 64] for gi in groups])
    q = p[idx]
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, 1, eps, 100.0, 30, 0.1)
        dwglib.dwg_set_update(h, 9, 10, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.4)
        dwglib.dwg_set_tuning(h, tree_group=group, tree_leaf=32)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, nrm)
        if group:
            w = np.zeros(n, np.float32)
            g = np.zeros((n, 3), np.float32)
            dwglib.dwg_step(h, w, g)
            w, g = w[idx], g[idx]
        else:
            w = np.zeros(len(q), np.float32)
            g = np.zeros((len(q), 3), np.float32)
            dwglib.dwg_eval_gwn(h, q, w, g)
        beta = float(np.float32(1) / np.float32(0.4))
        T, far, amb, leaves, bw, bg = _tree_checks(dwglib, h, p, a, q, beta, 100.0, eps)
    finally:
        dwglib.dwg_destroy(h)
    we, ge = oracle_mod.gwn(p, nrm, a, q, kernel=1, eps=eps, lam=100.0)
    scale = float(np.median(np.abs(we)))
    ew = np.abs(w - we) / scale
    eg = np.linalg.norm(g - ge, axis=1) / np.maximum(np.linalg.norm(ge, axis=1), 1e-30)
    print(json.dumps({"tree_error": "metaballs-1m", "test": "group lists" if group else
                      "per query", "theta": 0.4, "leaf": 32, "lambda": 100.0,
                      "w_rel_to_median_w": {"max": float(ew.max()),
                                            "p99": float(np.percentile(ew, 99)),
                                            "median": float(np.median(ew))},
                      "grad_rel": {"max": float(eg.max()), "p99": float(np.percentile(eg, 99)),
                                   "median": float(np.median(eg))},
                      "error_over_bound_max": float((np.abs(w - we) / bw).max())}))
    sw, sg = _term_sums(p, nrm, a, q, eps)
    _assert_within(w, g, we, ge, bw, bg, 160 * U32 * sw, 160 * U32 * sg * np.sqrt(3),
                   "metaballs tree vs exact")
    if group == 0:
        wv, gv = bh_check.decomposition_value(T, p, nrm, a, q, far, leaves, kernel=1,
                                              lam=100.0, eps=eps)
        ab_w, ab_g = bh_check.far_bound(T, q, amb, lam=100.0, eps=eps)
        _assert_within(w, g, wv, gv, ab_w, ab_g, 160 * U32 * sw, 160 * U32 * sg * np.sqrt(3),
                       "metaballs tree vs its decomposition")
