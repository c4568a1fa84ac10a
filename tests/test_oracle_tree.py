"""Pins of the oracle's Barnes-Hut far field (Sec. 5.2), CPU only."""
import numpy as np
import pytest

import synth


def cloud(n, seed, consistent=False):
    p, nt = synth.torus(n, seed=seed, noise=0.003)
    nrm = nt if consistent else synth.random_unit_normals(n, seed=seed + 1)
    a = np.full(n, 4 * np.pi ** 2 * 0.3 / n)
    return p, nrm, a


def test_morton_order_is_sorted_interleaved_codes(oracle_mod):
    p, _, _ = cloud(3000, 1)
    c = oracle_mod.cells(p, 21).astype(np.uint64)
    key = np.zeros(len(p), dtype=np.uint64)
    for b in range(21):
        for ax in range(3):
            key |= ((c[:, ax] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + ax)
    ref = np.lexsort((np.arange(len(p)), key))
    np.testing.assert_array_equal(oracle_mod.morton_order(p), ref)


def test_tree_never_far_is_the_exact_sum(oracle_mod):
    p, nrm, a = cloud(2000, 2)
    q = np.vstack([p[:100], synth.uniform_box(100, [-1.4] * 3, [1.4] * 3, seed=3)])
    for kernel, lam in ((0, 0.0), (1, 10.0)):
        we, ge = oracle_mod.gwn(p, nrm, a, q, kernel=kernel, eps=0.01, lam=lam)
        w, g, cnt = oracle_mod.tree_gwn(p, nrm, a, q, kernel=kernel, eps=0.01, lam=lam,
                                        beta=1e7, want_count=True)
        np.testing.assert_allclose(w, we, atol=1e-13)
        np.testing.assert_allclose(g, ge, atol=1e-10 * np.abs(ge).max())
        # every source evaluated once, the query's own point skipped
        np.testing.assert_array_equal(cnt, [len(p) - 1] * 100 + [len(p)] * 100)


@pytest.mark.parametrize("beta", [2.0, 2.3, 4.0])
@pytest.mark.parametrize("consistent", [False, True])
def test_tree_error_within_first_order_bound(oracle_mod, beta, consistent):
    """|w_tree - w_exact| <= sum over far nodes of A r / (2 pi (d - r)^3): the
    Taylor remainder of replacing a node's dipoles by one at its centre."""
    p, nrm, a = cloud(4000, 5, consistent)
    q = np.vstack([p[::20], synth.uniform_box(200, [-1.4] * 3, [1.4] * 3, seed=6)])
    eps = 0.005
    we = oracle_mod.gwn(p, nrm, a, q, eps=eps, grad=False)
    w, cnt, bnd = oracle_mod.tree_gwn(p, nrm, a, q, eps=eps, beta=beta, grad=False,
                                      want_count=True, want_bound=True)
    assert np.all(np.abs(w - we) <= bnd + 1e-12)
    assert cnt.mean() < len(p)  # the far field does replace points


def test_tree_error_shrinks_with_the_opening_angle(oracle_mod):
    p, nrm, a = cloud(4000, 7, True)
    q = p[::10]
    we = oracle_mod.gwn(p, nrm, a, q, eps=0.005, grad=False)
    errs = [np.abs(oracle_mod.tree_gwn(p, nrm, a, q, eps=0.005, beta=b, grad=False) - we).mean()
            for b in (2.0, 4.0, 8.0)]
    assert errs[0] > errs[1] > errs[2]


def test_group_of_one_is_the_per_query_tree(oracle_mod):
    """With one query per group the box is the query itself: the group test
    is then the per-query test, decisions and values identical."""
    p, nrm, a = cloud(3000, 11)
    q = np.vstack([p[::15], synth.uniform_box(150, [-1.4] * 3, [1.4] * 3, seed=12)])
    for kernel, lam in ((0, 0.0), (1, 10.0)):
        w1, g1, c1 = oracle_mod.tree_gwn(p, nrm, a, q, kernel=kernel, eps=0.004, lam=lam,
                                         beta=2.0, want_count=True)
        w2, g2, c2 = oracle_mod.tree_gwn_group(p, nrm, a, q, kernel=kernel, eps=0.004, lam=lam,
                                               beta=2.0, group=1, want_count=True)
        np.testing.assert_array_equal(c1, c2)
        np.testing.assert_allclose(w2, w1, rtol=0, atol=1e-13)
        np.testing.assert_allclose(g2, g1, rtol=0, atol=1e-10 * np.abs(g1).max())


@pytest.mark.parametrize("group", [8, 64])
@pytest.mark.parametrize("consistent", [False, True])
def test_group_tree_is_within_the_per_query_bound(oracle_mod, group, consistent):
    """Far for a group's box implies far for each of its queries, and a
    node's first-order bound is at least its children's sum: the group form
    stays within each query's per-query bound and never evaluates fewer
    terms."""
    p, nrm, a = cloud(4000, 13, consistent)
    order = oracle_mod.morton_order(p)
    q = p[order][::7]  # Morton-ordered queries, as the library groups them
    eps = 0.005
    we = oracle_mod.gwn(p, nrm, a, q, eps=eps, grad=False)
    _, cq, bnd = oracle_mod.tree_gwn(p, nrm, a, q, eps=eps, beta=2.0, grad=False,
                                     want_count=True, want_bound=True)
    wg, cg = oracle_mod.tree_gwn_group(p, nrm, a, q, eps=eps, beta=2.0, group=group,
                                       grad=False, want_count=True)
    assert np.all(np.abs(wg - we) <= bnd + 1e-12)
    assert np.all(cg >= cq)
    assert cg.mean() < len(p)


def test_group_tree_never_far_is_the_exact_sum(oracle_mod):
    p, nrm, a = cloud(1500, 14)
    q = p[::9]
    we, ge = oracle_mod.gwn(p, nrm, a, q, eps=0.01)
    w, g = oracle_mod.tree_gwn_group(p, nrm, a, q, eps=0.01, beta=1e7, group=32)
    np.testing.assert_allclose(w, we, atol=1e-13)
    np.testing.assert_allclose(g, ge, atol=1e-10 * np.abs(ge).max())
