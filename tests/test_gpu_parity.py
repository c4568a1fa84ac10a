"""CUDA library vs the FP64 oracle, element by element, through the C ABI.

Tolerances (FP32 terms, compensated sums):
  w:      |dw| <= 1e-5                                   (exact path)
  grad w: |dg|_inf <= 1e-5 max(1, |g|) + 16 * 2^-24 * S_g, S_g = 4 sum_j |m_j| rho_j^-3,
          a bound on the sum of the gradient terms' magnitudes (forward-error
          allowance of FP32 arithmetic on a sum whose terms cancel).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def s_g(points, normals, weights, queries, eps):
    p = np.asarray(points, np.float64)
    m = np.asarray(weights, np.float64)[:, None] * np.asarray(normals, np.float64) / (4 * np.pi)
    mn = np.linalg.norm(m, axis=1)
    out = np.zeros(len(queries))
    for i0 in range(0, len(queries), 256):
        q = np.asarray(queries[i0:i0 + 256], np.float64)
        d2 = ((p[None, :, :] - q[:, None, :]) ** 2).sum(-1) + eps * eps
        out[i0:i0 + 256] = 4 * (mn[None, :] * d2 ** -1.5).sum(1)
    return out


def check_wg(w, g, wo, go, sg):
    dw = np.abs(w - wo)
    assert dw.max() <= 1e-5, f"max |dw| {dw.max():.3e}"
    gn = np.linalg.norm(go, axis=1)
    tol = 1e-5 * np.maximum(1.0, gn) + 16 * U32 * sg
    dg = np.abs(g - go).max(axis=1)
    bad = dg > tol
    assert not bad.any(), f"{bad.sum()} gradients off; worst ratio {(dg / tol).max():.3f}"


def make_cloud(n, seed, kind="torus"):
    if kind == "torus":
        p, nt = synth.torus(n, seed=seed, noise=0.005)
        area = 4 * np.pi ** 2 * 0.3
    elif kind == "sphere":
        p, nt = synth.sphere(n, seed=seed)
        area = 4 * np.pi
    else:
        p = synth.uniform_box(n, [-1] * 3, [1] * 3, seed=seed)
        nt = synth.random_unit_normals(n, seed=seed + 1)
        area = 4.0 * n ** (1 / 3)
    a = np.full(n, area / max(n, 1), dtype=np.float32)
    return p, nt, a, synth.default_eps(area, max(n, 1))


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


# ----------------------------------------------------------------------------
# evaluation (Eq. 2/3, Eq. 5)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 200, 1000, 4097])
@pytest.mark.parametrize("kernel,lam", [(0, 0.0), (1, 10.0), (1, 100.0)])
def test_eval_at_points_and_queries(dwglib, oracle_mod, handle, n, kernel, lam):
    p, _, a, eps = make_cloud(n, seed=n, kind="torus")
    n0 = synth.random_unit_normals(n, seed=3).astype(np.float32)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
    dwglib.dwg_set_normals(h, n0)
    q = np.vstack([p, synth.uniform_box(257, [-1.5, -1.5, -0.6], [1.5, 1.5, 0.6], seed=5),
                   p[:1] + np.float32(1e-3)]).astype(np.float32)
    w = np.zeros(len(q), np.float32)
    g = np.zeros((len(q), 3), np.float32)
    dwglib.dwg_eval_gwn(h, q, w, g)
    wo, go = oracle_mod.gwn(p, n0, a, q, kernel=kernel, eps=eps, lam=lam)
    check_wg(w, g, wo, go, s_g(p, n0, a, q, eps))
    # w only
    w2 = np.zeros(len(q), np.float32)
    dwglib.dwg_eval_gwn(h, q, w2, None)
    assert np.max(np.abs(w2 - wo)) <= 1e-5


def test_eval_duplicates_and_coincident_queries(dwglib, oracle_mod, handle):
    p, _, a, eps = make_cloud(500, seed=7, kind="sphere")
    p = np.vstack([p, p[10:13], p[10:11]]).astype(np.float32)   # exact duplicates
    a = np.append(a, a[:4]).astype(np.float32)
    n0 = synth.random_unit_normals(len(p), seed=8).astype(np.float32)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, 0, eps, 0.0, 30, 0.1)
    dwglib.dwg_set_normals(h, n0)
    w = np.zeros(len(p), np.float32)
    g = np.zeros((len(p), 3), np.float32)
    dwglib.dwg_eval_gwn(h, p, w, g)
    wo, go = oracle_mod.gwn(p, n0, a, p, eps=eps)
    check_wg(w, g, wo, go, s_g(p, n0, a, p, eps))
    # and through one iteration, where the queries are the sorted sources
    dwglib.dwg_set_update(h, 5, 10, dwglib.DWG_UPDATE_LEVELSET)
    ws = np.zeros(len(p), np.float32)
    gs = np.zeros((len(p), 3), np.float32)
    dwglib.dwg_step(h, ws, gs)
    check_wg(ws, gs, wo, go, s_g(p, n0, a, p, eps))


def test_eval_torus_100k_sampled(dwglib, oracle_mod, handle):
    """The 100,000-point torus (0.5 % noise) at its full size, through the same
    kernels and launch shapes as an orientation step; the oracle checks a
    seeded sample of 1,500 points."""
    W = synth.workload_torus100k()
    p, a, eps = W["points"], W["weights"], W["eps"]
    n = len(p)
    n0 = synth.random_unit_normals(n, seed=1).astype(np.float32)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_ALLPAIRS, 0.5)
    for kernel, lam in ((0, 0.0), (1, 10.0)):
        dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
        dwglib.dwg_set_update(h, 8, 10, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, n0)
        w = np.zeros(n, np.float32)
        g = np.zeros((n, 3), np.float32)
        dwglib.dwg_step(h, w, g)
        idx = np.unique((synth.uniform(9, 1, 1500) * n).astype(np.int64))
        wo, go = oracle_mod.gwn(p, n0, a, p[idx], kernel=kernel, eps=eps, lam=lam)
        check_wg(w[idx], g[idx], wo, go, s_g(p, n0, a, p[idx], eps))


# ----------------------------------------------------------------------------
# octree discretisation (integer work: bit-exact)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,depth", [(1, 3), (33, 4), (2000, 6), (20000, 8)])
def test_leaves_and_corners_bit_exact(dwglib, oracle_mod, handle, n, depth):
    p, _, _, _ = make_cloud(n, seed=11, kind="torus")
    h = handle(p)
    dwglib.dwg_set_update(h, depth, 10, dwglib.DWG_UPDATE_LEVELSET)
    L = dwglib.dwg_get_leaves(h)
    Lo = oracle_mod.octree_leaves(p, depth)
    order = np.lexsort((Lo[:, 3], Lo[:, 2], Lo[:, 1], Lo[:, 0]))
    np.testing.assert_array_equal(L, Lo[order])
    K = dwglib.dwg_get_corners(h)
    np.testing.assert_array_equal(K, oracle_mod.corner_keys(Lo, depth))


# ----------------------------------------------------------------------------
# k nearest points
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,k", [(5, 10), (1000, 10), (30000, 10), (3000, 32), (3000, 1)])
def test_knn(dwglib, oracle_mod, handle, n, k):
    p = synth.uniform_box(n, [-1] * 3, [1] * 3, seed=n)
    q = synth.uniform_box(700, [-1.3] * 3, [1.3] * 3, seed=n + 1)
    h = handle(p)
    idx = np.zeros((len(q), k), np.int64)
    dwglib.dwg_knn(h, q, k, idx)
    ref = oracle_mod.knn(p, q, k)
    mism = idx != ref
    if mism.any():
        # only where float32 distances cannot tell the candidates apart
        p64, q64 = p.astype(np.float64), q.astype(np.float64)
        for i, t in zip(*np.nonzero(mism)):
            da = np.linalg.norm(p64[idx[i, t]] - q64[i])
            db = np.linalg.norm(p64[ref[i, t]] - q64[i])
            assert abs(da - db) <= 1e-6 * max(da, db), (i, t, da, db)


def test_knn_ties_by_index(dwglib, handle):
    p = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                  [2, 0, 0]], dtype=np.float32)[::-1].copy()
    h = handle(p)
    idx = np.zeros((1, 3), np.int64)
    dwglib.dwg_knn(h, np.zeros((1, 3), np.float32), 3, idx)
    np.testing.assert_array_equal(idx[0], [1, 2, 3])


# ----------------------------------------------------------------------------
# one iteration and the full loop
# ----------------------------------------------------------------------------
def angle(a, b):
    c = np.cross(a, b)
    return np.arctan2(np.linalg.norm(c, axis=1), np.sum(a * b, axis=1))


@pytest.mark.parametrize("kernel,lam", [(0, 0.0), (1, 10.0)])
def test_one_step_levelset(dwglib, oracle_mod, handle, kernel, lam):
    W = synth.workload_sphere2k()
    p, a, eps = W["points"], W["weights"], W["eps"]
    n = len(p)
    n0 = synth.random_unit_normals(n, seed=1).astype(np.float32)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
    dwglib.dwg_set_update(h, 6, 10, dwglib.DWG_UPDATE_LEVELSET)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, n0)
    w = np.zeros(n, np.float32)
    g = np.zeros((n, 3), np.float32)
    dth = np.zeros(n, np.float32)
    iso, stat = dwglib.dwg_step(h, w, g, dth)
    prm = oracle_mod.params(kernel=kernel, lam=lam, eps=eps, depth=6)
    r = oracle_mod.iterate(p, a, n0, prm)
    check_wg(w, g, r["w"], r["g"], s_g(p, n0, a, p, eps))
    assert iso == pytest.approx(r["iso"], abs=1e-6)
    n1 = np.zeros((n, 3), np.float32)
    dwglib.dwg_get_normals(h, n1)
    ang = angle(n1.astype(np.float64), r["normals"])
    # the update is continuous in the corner values except where a face's
    # 10th neighbour is nearly tied; nearly all points agree to 1e-3 rad
    assert np.mean(ang < 1e-3) >= 0.99, np.sort(ang)[-10:]
    assert np.mean(ang < 1e-1) >= 0.999
    same = ang < 1e-3
    assert np.max(np.abs(dth[same] - r["dtheta"][same])) < 0.06


def test_one_step_direct(dwglib, oracle_mod, handle):
    W = synth.workload_sphere2k()
    p, a, eps = W["points"], W["weights"], W["eps"]
    n = len(p)
    n0 = synth.random_unit_normals(n, seed=2).astype(np.float32)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, 0, eps, 0.0, 30, 0.1)
    dwglib.dwg_set_update(h, 6, 10, dwglib.DWG_UPDATE_DIRECT)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, n0)
    dth = np.zeros(n, np.float32)
    iso, stat = dwglib.dwg_step(h, None, None, dth)
    r = oracle_mod.iterate(p, a, n0, oracle_mod.params(eps=eps, mode=oracle_mod.MODE_DIRECT))
    n1 = np.zeros((n, 3), np.float32)
    dwglib.dwg_get_normals(h, n1)
    ang = angle(n1.astype(np.float64), r["normals"])
    assert ang.max() < 1e-4, ang.max()
    assert stat == pytest.approx(oracle_mod.top1_mean(r["dtheta"]), abs=1e-3)


def test_random_init_follows_the_generator_definition(dwglib, handle):
    p, _, _, _ = make_cloud(3000, seed=4, kind="box")
    h = handle(p)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_RANDOM, 123)
    out = np.zeros((3000, 3), np.float32)
    dwglib.dwg_get_normals(h, out)
    np.testing.assert_allclose(out, synth.random_unit_normals(3000, seed=123), atol=2e-6)


def agreement(n, nt):
    d = np.sum(n * nt, axis=1)
    s = 1.0 if d.sum() >= 0 else -1.0
    return float(np.mean(s * d > 0))


def test_orient_sphere_matches_oracle_and_analytic(dwglib, oracle_mod, handle):
    W = synth.workload_sphere2k()
    p, a, eps = W["points"], W["weights"], W["eps"]
    n = len(p)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, 0, eps, 0.0, 40, 0.1)
    dwglib.dwg_set_update(h, 6, 10, dwglib.DWG_UPDATE_LEVELSET)
    n0 = synth.random_unit_normals(n, seed=1).astype(np.float32)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, n0)
    out = np.zeros((n, 3), np.float32)
    rc, iters = dwglib.dwg_orient(h, out)
    r = oracle_mod.orient(p, a, n0, oracle_mod.params(eps=eps, depth=6, max_iters=40))
    assert agreement(out, W["normals_true"]) == 1.0
    assert agreement(out, r["normals"]) >= 0.999
    assert rc == dwglib.DWG_OK and abs(iters - r["iters"]) <= 3, (iters, r["iters"])
    tr = dwglib.dwg_get_trace(h)
    assert len(tr["stat"]) == iters and tr["stat"][-1] <= 0.1
    # deterministic: a second run gives the same bits
    out2 = np.zeros_like(out)
    dwglib.dwg_orient(h, out2)
    assert np.array_equal(out, out2)


def test_orient_mean_change_rule_matches_oracle(dwglib, oracle_mod, handle):
    """DWG_CONV_MEAN stops at the oracle's iteration (mean |n_new - n_old| <=
    chord of tol) and gives its normals."""
    n = 1200
    p, nt = synth.torus(n, seed=4)
    area = 4 * np.pi ** 2 * 0.3
    a = np.full(n, area / n, np.float32)
    eps = synth.default_eps(area, n)
    n0 = synth.random_unit_normals(n, seed=2).astype(np.float32)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, 1, eps, 10.0, 40, 0.5)
    dwglib.dwg_set_update(h, 5, 10, dwglib.DWG_UPDATE_LEVELSET)
    dwglib.dwg_set_convergence(h, dwglib.DWG_CONV_MEAN)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, n0)
    out = np.zeros((n, 3), np.float32)
    rc, iters = dwglib.dwg_orient(h, out)
    r = oracle_mod.orient(p, a, n0, oracle_mod.params(kernel=1, lam=10.0, eps=eps, depth=5,
                                                      max_iters=40, tol=0.5, rule=1))
    assert r["converged"] and rc == dwglib.DWG_OK
    assert abs(iters - r["iters"]) <= 2, (iters, r["iters"])
    assert agreement(out, r["normals"]) >= 0.995
    tr = dwglib.dwg_get_trace(h)
    chord = 2 * np.sin(np.radians(0.5) / 2)
    assert tr["mean_dn"][-1] <= chord and np.all(tr["mean_dn"][:-1] > chord)
    with pytest.raises(dwglib.DWGError):
        dwglib.dwg_set_convergence(h, 7)


def test_orient_torus_agrees_with_analytic(dwglib, handle):
    n = 20000
    p, nt = synth.torus(n, seed=0)
    area = 4 * np.pi ** 2 * 0.3
    h = handle(p)
    dwglib.dwg_set_weights(h, np.full(n, area / n, np.float32))
    dwglib.dwg_set_params(h, 1, synth.default_eps(area, n), 10.0, 40, 0.1)
    dwglib.dwg_set_update(h, 7, 10, dwglib.DWG_UPDATE_LEVELSET)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_RANDOM, 1)
    out = np.zeros((n, 3), np.float32)
    rc, iters = dwglib.dwg_orient(h, out)
    assert agreement(out, nt) >= 0.999, (agreement(out, nt), iters)


# ----------------------------------------------------------------------------
# error paths
# ----------------------------------------------------------------------------
def test_error_paths(dwglib, handle):
    with pytest.raises(dwglib.DWGError) as e:
        dwglib.dwg_create(np.array([[0, 0, np.nan]], np.float32))
    assert e.value.code == dwglib.DWG_ERR_NONFINITE
    with pytest.raises(dwglib.DWGError) as e:
        dwglib.dwg_create(np.zeros((0, 3), np.float32))
    assert e.value.code == dwglib.DWG_ERR_INVALID
    h = handle(synth.uniform_box(10, [0] * 3, [1] * 3, seed=1))
    for args in ((5, 0.1, 0.0, 10, 0.1), (0, 0.0, 0.0, 10, 0.1), (0, 0.1, -1.0, 10, 0.1),
                 (0, 0.1, 0.0, 0, 0.1), (0, 0.1, 0.0, 10, 0.0)):
        with pytest.raises(dwglib.DWGError) as e:
            dwglib.dwg_set_params(h, *args)
        assert e.value.code == dwglib.DWG_ERR_INVALID
    with pytest.raises(dwglib.DWGError):
        dwglib.dwg_set_update(h, 0, 10, 0)
    with pytest.raises(dwglib.DWGError):
        dwglib.dwg_set_normals(h, np.zeros((10, 3), np.float32))
    # the handle still works after the errors
    out = np.zeros((10, 3), np.float32)
    dwglib.dwg_set_update(h, 3, 10, 0)
    dwglib.dwg_orient(h, out)
    assert np.all(np.isfinite(out))


@pytest.mark.parametrize("n", [1, 99, 101, 5000, 300001])
def test_select_statistic_equals_oracle_on_the_same_changes(dwglib, oracle_mod, handle, n):
    """The convergence statistic of a step (multi-CTA radix select, FP64 sums
    in a fixed order) against the oracle's mean of the ceil(n/100) largest of
    the same float32 changes: equal to rounding of the FP64 sum."""
    p, _, a, eps = make_cloud(n, seed=n % 97 + 3, kind="box")
    n0 = synth.random_unit_normals(n, seed=5).astype(np.float32)
    h = handle(p)
    dwglib.dwg_set_params(h, 0, max(eps, 1e-3), 0.0, 30, 0.1)
    dwglib.dwg_set_update(h, 3, 10, dwglib.DWG_UPDATE_DIRECT)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.5)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, n0)
    dth = np.zeros(n, np.float32)
    iso, stat = dwglib.dwg_step(h, None, None, dth)
    ref = oracle_mod.top1_mean(dth.astype(np.float64))
    assert stat == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_checkpoint_resume_is_bit_exact(dwglib, handle):
    """The iteration's state is the normals: stopping after 8 iterations,
    reading the normals and orienting 8 more from them gives the normals of
    16 iterations in one run, bit for bit (deterministic sums and
    order-independent fixed-point scatter)."""
    n = 3000
    p, _ = synth.torus(n, seed=8, noise=0.003)
    area = 4 * np.pi ** 2 * 0.3
    eps = synth.default_eps(area, n)
    n0 = synth.random_unit_normals(n, seed=9).astype(np.float32)
    outs, totals = [], []
    for caps in ((16,), (8, 8)):
        h = handle(p)
        dwglib.dwg_set_weights(h, np.full(n, area / n, np.float32))
        dwglib.dwg_set_update(h, 6, 10, dwglib.DWG_UPDATE_LEVELSET)
        start, total = n0, 0
        for cap in caps:
            dwglib.dwg_set_params(h, 1, eps, 10.0, cap, 1e-6)  # tol met only at an exact fixed point
            dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, start)
            out = np.zeros((n, 3), np.float32)
            rc, it = dwglib.dwg_orient(h, out)
            assert 1 <= it <= cap
            total += it
            start = out
        outs.append(out)
        totals.append(total)
    assert totals[0] >= 9 and totals[1] == totals[0]  # the split run resumed mid-way
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("kind,n,depth,k", [("torus", 20000, 7, 10), ("box", 6000, 6, 10),
                                            ("torus", 20000, 8, 7), ("sphere", 3000, 9, 10),
                                            ("cluster", 12000, 6, 10)])
def test_knn_cell_lists_equal_the_tree_search(dwglib, handle, kind, n, depth, k):
    """The per-leaf candidate lists (knn_lists = 1) return exactly the tree
    search's k nearest points: identical normals and iteration counts.  The
    cluster case (4,000 points in a ball of radius 0.02 on a sphere) has
    cells with more than 256 candidates, which keep the tree search."""
    if kind == "cluster":
        p, _, a, eps = make_cloud(n - 4000, seed=21, kind="sphere")
        c = synth.uniform_box(4000, [-0.02] * 3, [0.02] * 3, seed=23) + np.float32([1.0, 0, 0])
        p = np.vstack([p, c]).astype(np.float32)
        a = np.full(n, 4 * np.pi / n, np.float32)
    else:
        p, _, a, eps = make_cloud(n, seed=21, kind=kind)
    n0 = synth.random_unit_normals(n, seed=22).astype(np.float32)
    res = []
    for lists in (1, 0):
        h = handle(p)
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, 1, eps, 10.0, 12, 0.1)
        dwglib.dwg_set_update(h, depth, k, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_tuning(h, knn_lists=lists)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, n0)
        out = np.zeros((n, 3), np.float32)
        rc, it = dwglib.dwg_orient(h, out)
        res.append((it, out))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])


def test_wait_limit_reports_timeout_and_the_handle_stays_usable(dwglib, handle):
    """Failure detection without a fault: a device-side wait that nothing
    completes gives up after its poll limit, the host sees DWG_ERR_TIMEOUT,
    and the same handle then evaluates and orients exactly as before."""
    p, _, a, eps = make_cloud(2000, seed=41, kind="sphere")
    n0 = synth.random_unit_normals(2000, seed=42).astype(np.float32)
    q = synth.uniform_box(300, [-1.5] * 3, [1.5] * 3, seed=43)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, 0, eps, 0.0, 30, 0.1)
    dwglib.dwg_set_normals(h, n0)
    w0 = np.zeros(len(q), np.float32)
    dwglib.dwg_eval_gwn(h, q, w0)
    for polls in (1, 1024):
        with pytest.raises(dwglib.DWGError) as e:
            dwglib.dwg_selfcheck_wait(h, polls)
        assert e.value.code == dwglib.DWG_ERR_TIMEOUT
    w1 = np.zeros(len(q), np.float32)
    dwglib.dwg_eval_gwn(h, q, w1)
    assert np.array_equal(w0, w1)
    dwglib.dwg_set_update(h, 6, 10, dwglib.DWG_UPDATE_LEVELSET)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, n0)
    rc, it = dwglib.dwg_orient(h, np.zeros((2000, 3), np.float32))
    assert rc in (dwglib.DWG_OK, dwglib.DWG_NOT_CONVERGED) and it >= 1
    with pytest.raises(dwglib.DWGError) as e:
        dwglib.dwg_selfcheck_wait(h, 0)
    assert e.value.code == dwglib.DWG_ERR_INVALID


def test_fp32_microbenchmarks_are_near_the_derived_issue_rate(dwglib):
    """The measured packed-FMA rate is within 25 % of SMs x 128 lanes x the
    SM clock (the derived peak of the evaluators' roofline) at any clock the
    GPU runs at, MUFU rsqrt is at most an eighth of it (16 per SM per clock)
    and MUFU ex2 at most a quarter."""
    torch = pytest.importorskip("torch")
    ffma, rsq, ex2 = dwglib.dwg_measure_fp32_peaks(0)
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    assert ffma > 0 and rsq > 0
    per_sm_clk = ffma / sms  # lane operations per SM per second
    # between 1.0 and 2.2 GHz of 128 lanes
    assert 0.75 * 128 * 1.0e9 <= per_sm_clk <= 1.05 * 128 * 2.2e9, per_sm_clk
    assert rsq <= ffma / 8 * 1.10, (rsq, ffma)
    assert 0 < ex2 <= ffma / 4 * 1.10, (ex2, ffma)
    with pytest.raises(dwglib.DWGError) as e:
        dwglib.dwg_measure_fp32_peaks(999)
    assert e.value.code == dwglib.DWG_ERR_INVALID
