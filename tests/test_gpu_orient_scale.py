"""Whole orientations (Algorithm 1) of the CUDA library against the FP64
oracle's, from the same initial normals, at sizes where the oracle still
finishes in about a minute: per-point sign agreement up to one global flip,
iteration counts, and the convergence statistics of Sec. 5.1 and Fig. 6."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

AREA = 4 * np.pi ** 2 * 0.3


def _flip_agreement(a, b):
    d = np.sum(np.asarray(a, np.float64) * np.asarray(b, np.float64), axis=1)
    s = 1.0 if d.sum() >= 0 else -1.0
    return float(np.mean(s * d > 0))


def test_top1_plateau_matches_the_oracle(dwglib, oracle_mod):
    """5,000-point torus with 0.5 % noise, depth 6: both sides settle (all
    normals agree with the analytic ones, mean change far below the chord of
    0.1 deg) while the top-1 % statistic stays at a few tenths of a degree;
    the two sides' final normals agree point by point."""
    n, depth = 5000, 6
    p, nt = synth.torus(n, seed=0, noise=0.005)
    a = np.full(n, AREA / n, np.float32)
    eps = synth.default_eps(AREA, n)
    n0 = synth.random_unit_normals(n, seed=1).astype(np.float32)
    prm = oracle_mod.params(eps=eps, depth=depth, max_iters=1, tol=0.1)
    cur = n0.astype(np.float64)
    top_o = []
    for _ in range(25):
        r = oracle_mod.iterate(p, a, cur, prm)
        top_o.append(oracle_mod.top1_mean(r["dtheta"]))
        cur = r["normals"]
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, 0, eps, 0.0, 25, 0.1)
        dwglib.dwg_set_update(h, depth, 10, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_ALLPAIRS, 0.5)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, n0)
        top_g = [dwglib.dwg_step(h)[1] for _ in range(25)]
        out = np.zeros((n, 3), np.float32)
        dwglib.dwg_get_normals(h, out)
    finally:
        dwglib.dwg_destroy(h)
    assert _flip_agreement(out, nt) == 1.0
    assert _flip_agreement(out, cur) >= 0.999
    for top in (top_o, top_g):
        assert 0.2 <= min(top[18:]) and max(top[18:]) <= 2.0, top[18:]


def test_orientation_matches_the_oracle_at_20k_points(dwglib, oracle_mod):
    """20,000-point torus with 0.25 % noise, depth 6, from the same random
    normals to the Fig. 6 rule: both sides converge, at nearby iterations,
    and give the same sign at >= 99.9 % of the
    points after one global flip (both agree with the analytic normals).
    At 0.5 % noise the noise reaches the point spacing and about 0.5 % of
    the points keep switching between two states on both sides (reading 8),
    so the stopping iteration and those points' phase are not unique."""
    n, depth = 20000, 6
    p, nt = synth.torus(n, seed=3, noise=0.0025)
    a = np.full(n, AREA / n, np.float32)
    eps = synth.default_eps(AREA, n)
    n0 = synth.random_unit_normals(n, seed=4).astype(np.float32)
    r = oracle_mod.orient(p, a, n0, oracle_mod.params(eps=eps, depth=depth, max_iters=60,
                                                      tol=0.1, rule=1))
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, 0, eps, 0.0, 60, 0.1)
        dwglib.dwg_set_update(h, depth, 10, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_convergence(h, dwglib.DWG_CONV_MEAN)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_ALLPAIRS, 0.5)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, n0)
        out = np.zeros((n, 3), np.float32)
        rc, iters = dwglib.dwg_orient(h, out)
    finally:
        dwglib.dwg_destroy(h)
    assert r["converged"] and rc == dwglib.DWG_OK
    # the transient (top-1 % statistic at 60-90 deg for about 30 iterations
    # on the oracle) is sensitive to rounding: the stopping points agree to
    # a quarter of the oracle's count
    assert abs(iters - r["iters"]) <= max(5, r["iters"] // 4), (iters, r["iters"])
    assert _flip_agreement(out, r["normals"]) >= 0.999
    assert _flip_agreement(out, nt) >= 0.999 and _flip_agreement(r["normals"], nt) >= 0.999


def test_mixed_component_matches_the_oracle(dwglib, oracle_mod):
    """The two-sphere case of test_oracle_orient: B heals alone and stays
    mixed beside a consistently oriented A, on the GPU as on the oracle."""
    from test_oracle_orient import mixed_component_runs, _two_spheres
    ref = mixed_component_runs(oracle_mod)
    pa, na, aa, pb, nb, ab, nb0 = _two_spheres()
    runs = {"B alone": (pb, ab, nb0),
            "A outward": (np.vstack([pa, pb]), np.concatenate([aa, ab]), np.vstack([na, nb0])),
            "A inward": (np.vstack([pa, pb]), np.concatenate([aa, ab]), np.vstack([-na, nb0]))}
    for name, (P, A, N0) in runs.items():
        P = P.astype(np.float32)
        h = dwglib.dwg_create(P)
        try:
            dwglib.dwg_set_weights(h, A.astype(np.float32))
            dwglib.dwg_set_params(h, 0, 0.5 * np.sqrt(A.sum() / len(P)), 0.0, 15, 0.1)
            dwglib.dwg_set_update(h, 6, 10, dwglib.DWG_UPDATE_LEVELSET)
            dwglib.dwg_set_tree(h, dwglib.DWG_PATH_ALLPAIRS, 0.5)
            dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, N0.astype(np.float32))
            for _ in range(15):
                dwglib.dwg_step(h)
            out = np.zeros((len(P), 3), np.float32)
            dwglib.dwg_get_normals(h, out)
        finally:
            dwglib.dwg_destroy(h)
        frac = float(np.mean(np.sum(out[-1500:] * nb, axis=1) > 0))
        assert abs(frac - ref[name][0]) <= 0.05, (name, frac, ref[name][0])
        d = np.sum(out.astype(np.float64) * ref[name][2], axis=1)
        assert np.mean(d > 0) >= 0.99, name


def _per_primitive(out, nt, lab):
    d = np.sum(np.asarray(out, np.float64) * nt, axis=1)
    s = np.where(np.bincount(lab, weights=d) >= 0, 1.0, -1.0)[lab]
    return float(np.mean(s * d > 0))


def test_union_plateau_is_not_the_far_field(dwglib):
    """A union of 40 random tori and ellipsoids, 300,000 points, no noise,
    depth 8, screened lambda 100, 100 iterations from random normals: the
    exact all-pairs path orients no better than the Barnes-Hut path at the
    paper's opening angle (1 / 2.3), and both end well below one orientation
    per shape -- the mixed components of the two-sphere test, not the far
    field and not the noise.  (Which of the two ends a little higher varies
    with the rounding of the terms: the plateau's trajectory is chaotic.)"""
    n = 300_000
    p, nt, lab = synth.union_of_shapes(n, seed=0, noise=0.0, labels=True)
    eps = 0.5 * float((p.max(0) - p.min(0)).max()) / np.sqrt(n)
    res = {}
    for path in (dwglib.DWG_PATH_ALLPAIRS, dwglib.DWG_PATH_TREE):
        h = dwglib.dwg_create(p)
        try:
            dwglib.dwg_set_weights(h, np.ones(n, np.float32))
            dwglib.dwg_set_params(h, 1, eps, 100.0, 100, 0.1)
            dwglib.dwg_set_update(h, 8, 10, dwglib.DWG_UPDATE_LEVELSET)
            dwglib.dwg_set_tree(h, path, 1 / 2.3)
            if path == dwglib.DWG_PATH_TREE:
                dwglib.dwg_set_tuning(h, tree_group=0, tree_leaf=16)
            dwglib.dwg_set_init(h, dwglib.DWG_INIT_RANDOM, 1)
            for _ in range(100):
                dwglib.dwg_step(h)
            out = np.zeros((n, 3), np.float32)
            dwglib.dwg_get_normals(h, out)
        finally:
            dwglib.dwg_destroy(h)
        res[path] = _per_primitive(out, nt, lab)
    exact, tree = res[dwglib.DWG_PATH_ALLPAIRS], res[dwglib.DWG_PATH_TREE]
    assert exact < 0.99 and tree < 0.99, res
    assert exact <= tree + 0.02, res
