"""Barnes-Hut path of the CUDA library against the oracle's Barnes-Hut
(Sec. 5.2): same bucket tree (bit-exact Morton order), same node data
(double sums in the same order), same float32 opening test, so the two make
identical far/near decisions (checked through the evaluation counts); values
agree to the exact path's tolerances."""
import numpy as np
import pytest

import synth
from test_gpu_parity import check_wg, s_g, agreement

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("n", [1, 33, 1000, 5000, 40000])
@pytest.mark.parametrize("kernel,lam,theta", [(0, 0.0, 0.5), (0, 0.0, 1 / 2.3), (1, 10.0, 0.5)])
def test_tree_eval_matches_oracle_tree(dwglib, oracle_mod, handle, n, kernel, lam, theta):
    p, _ = synth.torus(n, seed=n + 3, noise=0.004)
    a = np.full(n, 4 * np.pi ** 2 * 0.3 / n, np.float32)
    nrm = synth.random_unit_normals(n, seed=n).astype(np.float32)
    eps = synth.default_eps(4 * np.pi ** 2 * 0.3, n)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, theta)
    dwglib.dwg_set_tuning(h, tree_group=0)  # the per-query test of Sec. 5.2
    dwglib.dwg_set_normals(h, nrm)
    sel = np.unique((synth.uniform(7, n, min(n, 1500)) * n).astype(np.int64))
    q = np.vstack([p[sel], synth.uniform_box(500, [-1.5, -1.5, -0.6], [1.5, 1.5, 0.6],
                                             seed=n)]).astype(np.float32)
    w = np.zeros(len(q), np.float32)
    g = np.zeros((len(q), 3), np.float32)
    dwglib.dwg_eval_gwn(h, q, w, g)
    cnt_gpu = dwglib.dwg_get_stats(h)["interactions_eval"]
    wo, go, cnt = oracle_mod.tree_gwn(p, nrm, a, q, kernel=kernel, eps=eps, lam=lam,
                                      beta=float(np.float32(1) / np.float32(theta)),
                                      want_count=True)
    check_wg(w, g, wo, go, s_g(p, nrm, a, q, eps))
    # identical opening decisions; the library also counts the query's own
    # point (it adds zero and is removed from the gradient afterwards)
    own = len(sel)
    assert cnt_gpu == cnt.sum() + own


def test_tree_with_tiny_opening_angle_is_exact(dwglib, oracle_mod, handle):
    n = 20000
    p, _ = synth.torus(n, seed=1, noise=0.003)
    a = np.full(n, 4 * np.pi ** 2 * 0.3 / n, np.float32)
    nrm = synth.random_unit_normals(n, seed=2).astype(np.float32)
    eps = synth.default_eps(4 * np.pi ** 2 * 0.3, n)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, 0, eps, 0.0, 30, 0.1)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 1e-3)
    dwglib.dwg_set_normals(h, nrm)
    q = p[::40].copy()
    w = np.zeros(len(q), np.float32)
    g = np.zeros((len(q), 3), np.float32)
    dwglib.dwg_eval_gwn(h, q, w, g)
    wo, go = oracle_mod.gwn(p, nrm, a, q, eps=eps)
    check_wg(w, g, wo, go, s_g(p, nrm, a, q, eps))


def test_tree_orientation_torus(dwglib, handle):
    n = 60000
    p, nt = synth.torus(n, seed=0)
    area = 4 * np.pi ** 2 * 0.3
    h = handle(p)
    dwglib.dwg_set_weights(h, np.full(n, area / n, np.float32))
    dwglib.dwg_set_params(h, 1, synth.default_eps(area, n), 10.0, 40, 0.1)
    dwglib.dwg_set_update(h, 7, 10, dwglib.DWG_UPDATE_LEVELSET)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.5)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_RANDOM, 1)
    out = np.zeros((n, 3), np.float32)
    rc, iters = dwglib.dwg_orient(h, out)
    assert agreement(out, nt) >= 0.999, (agreement(out, nt), iters)
    st = dwglib.dwg_get_stats(h)
    # the far field does the work of many points
    assert st["interactions"] < 0.5 * iters * (n * n + st["n_corners"] * n)


@pytest.mark.parametrize("n", [1, 33, 1000, 5000, 40000])
@pytest.mark.parametrize("kernel,lam,theta,leaf", [(0, 0.0, 0.5, 16), (0, 0.0, 1 / 2.3, 32),
                                                   (1, 10.0, 0.5, 16), (1, 100.0, 0.7, 64)])
def test_group_tree_matches_oracle_group_tree(dwglib, oracle_mod, handle, n, kernel, lam, theta,
                                              leaf):
    """Group form of the opening test (64 consecutive queries share the test
    against their bounding box): the oracle's group tree makes the same
    decisions (equal evaluation counts) and the values agree to the exact
    path's tolerances."""
    p, _ = synth.torus(n, seed=n + 5, noise=0.004)
    a = np.full(n, 4 * np.pi ** 2 * 0.3 / n, np.float32)
    nrm = synth.random_unit_normals(n, seed=n + 1).astype(np.float32)
    eps = synth.default_eps(4 * np.pi ** 2 * 0.3, n)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, theta)
    dwglib.dwg_set_tuning(h, tree_group=1, tree_leaf=leaf)
    dwglib.dwg_set_normals(h, nrm)
    # Morton-ordered points (compact groups) then scattered box queries
    order = oracle_mod.morton_order(p)
    sel = order[::max(1, n // 1500)]
    q = np.vstack([p[sel], synth.uniform_box(500, [-1.5, -1.5, -0.6], [1.5, 1.5, 0.6],
                                             seed=n + 2)]).astype(np.float32)
    w = np.zeros(len(q), np.float32)
    g = np.zeros((len(q), 3), np.float32)
    dwglib.dwg_eval_gwn(h, q, w, g)
    cnt_gpu = dwglib.dwg_get_stats(h)["interactions_eval"]
    beta = float(np.float32(1) / np.float32(theta))
    wo, go, cnt = oracle_mod.tree_gwn_group(p, nrm, a, q, kernel=kernel, eps=eps, lam=lam,
                                            beta=beta, bucket=leaf, group=64, want_count=True)
    check_wg(w, g, wo, go, s_g(p, nrm, a, q, eps))
    assert cnt_gpu == cnt.sum() + len(sel)


def test_group_tree_within_the_per_query_error_bound(dwglib, oracle_mod, handle):
    """Plain kernel: |w_group - w_exact| <= the per-query first-order bound
    (the group test only opens more nodes) plus the exact path's 1e-5."""
    n = 30000
    p, nt = synth.torus(n, seed=9, noise=0.003)
    a = np.full(n, 4 * np.pi ** 2 * 0.3 / n, np.float32)
    eps = synth.default_eps(4 * np.pi ** 2 * 0.3, n)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, 0, eps, 0.0, 30, 0.1)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.5)
    dwglib.dwg_set_tuning(h, tree_group=1)
    nrm = nt.astype(np.float32)
    dwglib.dwg_set_normals(h, nrm)
    q = p[oracle_mod.morton_order(p)[::20]]
    w = np.zeros(len(q), np.float32)
    dwglib.dwg_eval_gwn(h, q, w)
    we = oracle_mod.gwn(p, nrm, a, q, eps=eps, grad=False)
    _, bnd = oracle_mod.tree_gwn(p, nrm, a, q, eps=eps, beta=2.0, grad=False, want_bound=True)
    assert np.all(np.abs(w - we) <= bnd + 1e-5)


@pytest.mark.parametrize("group", [0, 1])
def test_tree_orientation_torus_both_tests(dwglib, handle, group):
    n = 60000
    p, nt = synth.torus(n, seed=0)
    area = 4 * np.pi ** 2 * 0.3
    h = handle(p)
    dwglib.dwg_set_weights(h, np.full(n, area / n, np.float32))
    dwglib.dwg_set_params(h, 1, synth.default_eps(area, n), 10.0, 40, 0.1)
    dwglib.dwg_set_update(h, 7, 10, dwglib.DWG_UPDATE_LEVELSET)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.5)
    dwglib.dwg_set_tuning(h, tree_group=group)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_RANDOM, 1)
    out = np.zeros((n, 3), np.float32)
    rc, iters = dwglib.dwg_orient(h, out)
    assert agreement(out, nt) >= 0.999, (agreement(out, nt), iters)


@pytest.mark.parametrize("kernel,lam,leaf", [(0, 0.0, 16), (1, 10.0, 32), (1, 100.0, 64)])
def test_group_lists_step_matches_oracle_group_tree(dwglib, oracle_mod, handle, kernel, lam,
                                                    leaf):
    """One iteration on the Barnes-Hut path with the group test evaluates the
    interaction lists built once per cloud (w and grad w at the points, in
    Morton order, 64 per group): the values are the oracle's group tree on
    the Morton-ordered points."""
    n = 20000
    p, _ = synth.torus(n, seed=12, noise=0.004)
    area = 4 * np.pi ** 2 * 0.3
    a = np.full(n, area / n, np.float32)
    eps = synth.default_eps(area, n)
    nrm = synth.random_unit_normals(n, seed=13).astype(np.float32)
    h = handle(p)
    dwglib.dwg_set_weights(h, a)
    dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
    dwglib.dwg_set_update(h, 6, 10, dwglib.DWG_UPDATE_LEVELSET)
    dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.5)
    dwglib.dwg_set_tuning(h, tree_group=1, tree_leaf=leaf)
    dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, nrm)
    w = np.zeros(n, np.float32)
    g = np.zeros((n, 3), np.float32)
    for rep in range(2):  # the second step reuses the lists with new normals
        dwglib.dwg_step(h, w, g)
        order = oracle_mod.morton_order(p)
        wo_s, go_s = oracle_mod.tree_gwn_group(p, nrm, a, p[order], kernel=kernel, eps=eps,
                                               lam=lam, beta=2.0, bucket=leaf, group=64)
        wo = np.empty(n)
        go = np.empty((n, 3))
        wo[order] = wo_s
        go[order] = go_s
        sel = np.arange(0, n, 7)
        check_wg(w[sel], g[sel], wo[sel], go[sel], s_g(p, nrm, a, p[sel], eps))
        nrm = np.zeros((n, 3), np.float32)
        dwglib.dwg_get_normals(h, nrm)


def _term_sums(points, normals, weights, queries, eps, chunk=16):
    """Per query: sum_j |m_j| rho_j^-2 (bounds sum |w terms|) and
    4 sum_j |m_j| rho_j^-3 (bounds sum |grad terms|), m = a n / 4 pi."""
    p = np.asarray(points, np.float64)
    mn = np.abs(np.asarray(weights, np.float64)) * np.linalg.norm(
        np.asarray(normals, np.float64), axis=1) / (4 * np.pi)
    sw = np.zeros(len(queries))
    sg = np.zeros(len(queries))
    for i0 in range(0, len(queries), chunk):
        q = np.asarray(queries[i0:i0 + chunk], np.float64)
        d2 = ((p[None, :, :] - q[:, None, :]) ** 2).sum(-1) + eps * eps
        sw[i0:i0 + chunk] = (mn[None, :] / d2).sum(1)
        sg[i0:i0 + chunk] = 4 * (mn[None, :] * d2 ** -1.5).sum(1)
    return sw, sg


def test_full_size_metaballs_step_matches_oracle_on_sampled_groups(dwglib, oracle_mod):
    """The 1,000,000-point metaballs workload in the launch configuration the
    benchmark times (screened lambda 100, depth 9, leaf 32, opening angle
    0.4, group test, lists): w and grad w of one step at 8 sampled groups of
    64 Morton-consecutive points against the oracle's group tree on the same
    groups.  a_i = 1 makes the terms large (w inside ~ n / area), so the
    tolerance is the FP32 forward-error bound of the sums: flushes of at most
    128 plain FP32 additions folded into two-sums, 160 u sum |t|."""
    W = synth.workload_metaballs1m()
    p, a, eps = W["points"], W["weights"], W["eps"]
    n = len(p)
    nrm = synth.random_unit_normals(n, seed=1).astype(np.float32)
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, 1, eps, 100.0, 30, 0.1)
        dwglib.dwg_set_update(h, 9, 10, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.4)
        dwglib.dwg_set_tuning(h, tree_group=1, tree_leaf=32)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, nrm)
        w = np.zeros(n, np.float32)
        g = np.zeros((n, 3), np.float32)
        dwglib.dwg_step(h, w, g)
    finally:
        dwglib.dwg_destroy(h)
    order = oracle_mod.morton_order(p)
    groups = np.unique((synth.uniform(4, 9, 8) * (n // 64)).astype(np.int64))
    idx = np.concatenate([order[64 * gi:64 * gi + 64] for gi in groups])
    beta = float(np.float32(1) / np.float32(0.4))
    wo, go = oracle_mod.tree_gwn_group(p, nrm, a, p[idx], kernel=1, eps=eps, lam=100.0,
                                       beta=beta, bucket=32, group=64)
    sw, sg = _term_sums(p, nrm, a, p[idx], eps)
    u = 2.0 ** -24
    assert np.all(np.abs(w[idx] - wo) <= 160 * u * sw)
    assert np.all(np.abs(g[idx] - go).max(axis=1) <= 160 * u * sg)
