"""Pins of the far-field error bound of the Barnes-Hut traversal (Sec. 5.2,
"Octree Traversal") for the plain kernel (Eq. 2/3), the screened kernel
(Eq. 5), softened or not, and of the tree checker that applies it
(tests/bh_check.py).  CPU only.

The bound (oracle.far_field_bound) is the mean-value remainder of replacing
a node's sources by one dipole: (mass / 4 pi) r times the norm of the
kernel's second (for w) or third (for grad w) derivative at the nearest
distance.  Pinned here against: the closed forms of the plain kernel; the
oracle's own gradient (itself pinned by finite differences) for a single
source, where the radial direction attains the norms; random clusters,
where it must hold; and one off-centre source at a small r / d, where it is
attained to first order (so a wrong constant fails)."""
import numpy as np
import pytest

import synth
import bh_check

LAMS = [0.0, 10.0, 100.0]


def test_plain_norms_are_the_closed_forms(oracle_mod):
    rho = np.array([0.01, 0.3, 1.0, 7.0])
    H, T = oracle_mod.kernel_derivative_norms(rho, 0.0)
    np.testing.assert_allclose(H, 2 / rho ** 3, rtol=1e-15)
    np.testing.assert_allclose(T, 6 / rho ** 4, rtol=1e-15)
    bw, bg = oracle_mod.far_field_bound(3.0, 0.2, 1.1)
    np.testing.assert_allclose(bw, 3.0 * 0.2 / (2 * np.pi * 0.9 ** 3), rtol=1e-15)
    np.testing.assert_allclose(bg, 3 * 3.0 * 0.2 / (2 * np.pi * 0.9 ** 4), rtol=1e-15)
    assert np.isinf(oracle_mod.far_field_bound(1.0, 1.0, 1.0)[0])


@pytest.mark.parametrize("lam", LAMS)
def test_norms_decrease_and_the_radial_direction_attains_the_third(oracle_mod, lam):
    rho = np.geomspace(1e-3, 30.0, 4000)
    H, T = oracle_mod.kernel_derivative_norms(rho, lam)
    assert np.all(np.diff(H) < 0) and np.all(np.diff(T) < 0)
    u = np.sqrt(lam) * rho
    g3 = np.exp(-u) * (6 + 6 * u + 3 * u * u + u ** 3) / rho ** 4
    np.testing.assert_allclose(T, g3, rtol=1e-14)


def _single(p, n, a, q, lam, eps, oracle_mod):
    return oracle_mod.gwn(np.array([p]), np.array([n]), np.array([a]), np.array([q]),
                          kernel=1 if lam > 0 else 0, eps=eps, lam=lam)


@pytest.mark.parametrize("lam", LAMS)
@pytest.mark.parametrize("eps", [0.0, 0.05])
def test_norms_against_the_oracle_gradient(oracle_mod, lam, eps):
    """grad_q t = Hess(p - q) m: with m along p - q its length is the radial
    eigenvalue (the Hessian norm); its derivative along the same direction,
    by central differences of the oracle's gradient, is the third
    derivative's norm; random directions never exceed either."""
    rng = np.random.default_rng(1)
    a = 4 * np.pi  # m = n
    for rho in (0.2, 0.7, 1.5):
        x = rng.normal(size=3)
        x /= np.linalg.norm(x)
        q = np.array([0.1, -0.2, 0.3])
        p = q + rho * x
        rs = np.sqrt(rho * rho + eps * eps)
        H, T = oracle_mod.kernel_derivative_norms(rs, lam)
        _, g = _single(p, x, a, q, lam, eps, oracle_mod)
        if eps == 0.0:
            np.testing.assert_allclose(np.linalg.norm(g), H, rtol=1e-12)
            h = 1e-5 * rho
            _, gp = _single(p, x, a, q + h * x, lam, eps, oracle_mod)
            _, gm = _single(p, x, a, q - h * x, lam, eps, oracle_mod)
            dg = (gp - gm) / (2 * h)
            np.testing.assert_allclose(np.linalg.norm(dg), T, rtol=1e-6)
        for _ in range(200):
            m = rng.normal(size=3)
            m /= np.linalg.norm(m)
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            _, g = _single(p, m, a, q, lam, eps, oracle_mod)
            assert np.linalg.norm(g) <= H * (1 + 1e-12)
            h = 1e-5 * rho
            _, gp = _single(p, m, a, q + h * u, lam, eps, oracle_mod)
            _, gm = _single(p, m, a, q - h * u, lam, eps, oracle_mod)
            assert np.linalg.norm((gp - gm) / (2 * h)) <= T * (1 + 1e-6)


def _cluster_error(oracle_mod, P, N, A, c, q, lam, eps):
    we, ge = oracle_mod.gwn(P, N, A, q[None], kernel=1 if lam > 0 else 0, eps=eps, lam=lam)
    M = (A[:, None] * N).sum(0)
    Mn = np.linalg.norm(M)
    wd, gd = oracle_mod.gwn(c[None], (M / Mn)[None], np.array([Mn]), q[None],
                            kernel=1 if lam > 0 else 0, eps=eps, lam=lam)
    return abs(we[0] - wd[0]), np.linalg.norm(ge[0] - gd[0])


@pytest.mark.parametrize("lam", LAMS)
@pytest.mark.parametrize("eps", [0.0, 0.02])
@pytest.mark.parametrize("centroid", [True, False])
def test_bound_holds_on_random_clusters(oracle_mod, lam, eps, centroid):
    rng = np.random.default_rng(7 + int(lam) + int(centroid))
    worst = 0.0
    for t in range(300):
        k = int(rng.integers(1, 40))
        r0 = 10 ** rng.uniform(-2, -0.5)
        P = rng.normal(size=(k, 3))
        P *= (r0 * rng.uniform(0, 1, k) ** (1 / 3) / np.linalg.norm(P, axis=1))[:, None]
        N = rng.normal(size=(k, 3))
        N /= np.linalg.norm(N, axis=1)[:, None]
        A = rng.uniform(0.1, 2.0, k)
        c = (A[:, None] * P).sum(0) / A.sum() if centroid else rng.normal(size=3) * r0 * 0.3
        r = np.linalg.norm(P - c, axis=1).max()
        dirn = rng.normal(size=3)
        dirn /= np.linalg.norm(dirn)
        d = r * rng.uniform(1.05, 20.0)
        q = c + d * dirn
        ew, eg = _cluster_error(oracle_mod, P, N, A, c, q, lam, eps)
        bw, bg = oracle_mod.far_field_bound(A.sum(), r, d, lam=lam, eps=eps)
        assert ew <= bw * (1 + 1e-9) + 1e-15, (t, ew, bw)
        assert eg <= bg * (1 + 1e-9) + 1e-15, (t, eg, bg)
        worst = max(worst, ew / bw)
    assert worst > 0.01  # the bound is not vacuous on these clusters


@pytest.mark.parametrize("lam", LAMS)
def test_bound_is_attained_by_one_offset_source(oracle_mod, lam):
    """One source at c + r x, normal x, query on the far side along -x: to
    first order in r / d the error is r times the norms."""
    x = np.array([0.0, 0.6, 0.8])
    c = np.array([0.2, 0.1, -0.3])
    for d in (0.5, 2.0):
        r = 1e-6 * d
        q = c - d * x
        ew, eg = _cluster_error(oracle_mod, np.array([c + r * x]), np.array([x]),
                                np.array([1.3]), c, q, lam, 0.0)
        bw, bg = oracle_mod.far_field_bound(1.3, r, d, lam=lam)
        assert 0.999 <= ew / bw <= 1.0, ew / bw
        assert 0.999 <= eg / bg <= 1.0, eg / bg


def _torus(n, seed):
    p, nt = synth.torus(n, seed=seed, noise=0.003)
    a = np.full(n, 4 * np.pi ** 2 * 0.3 / n)
    return p, nt, a


@pytest.mark.parametrize("kernel,lam,clamp", [(0, 0.0, False), (1, 10.0, False),
                                              (1, 100.0, False), (1, 30.0, True),
                                              (0, 0.0, True)])
@pytest.mark.parametrize("beta,leaf", [(2.0, 16), (2.5, 32)])
def test_walk_bound_holds_on_a_valid_tree(oracle_mod, kernel, lam, clamp, beta, leaf):
    """On a valid hierarchy (built here, verified), each query's decomposition
    under the opening test, evaluated in FP64, is within the summed bound of
    the exact sum; with the modified kernel the opening radius also covers
    r + the node's largest clamp radius, so a far node's terms are unclamped."""
    n = 4000
    p, _, a = _torus(n, 21)
    nrm = synth.random_unit_normals(n, seed=22)
    q = np.vstack([p[::13], synth.uniform_box(150, [-1.4] * 3, [1.4] * 3, seed=23)])
    eps = 0.0 if clamp else 0.004
    delta = oracle_mod.clamp_radii(p, 10, 0.005, 0.05) if clamp else None
    T = bh_check.build_reference_tree(p, a, leaf, beta, delta)
    bh_check.verify_tree(T, p, a)
    bh_check.verify_records(T, beta, delta)
    far, amb, leaves = bh_check.walk(T, q, beta, delta)
    bw, bg = bh_check.far_bound(T, q, far, lam=lam, eps=eps)
    wv, gv = bh_check.decomposition_value(T, p, nrm, a, q, far, leaves, kernel=kernel, lam=lam,
                                          eps=eps, delta=delta)
    we, ge = oracle_mod.gwn(p, nrm, a, q, kernel=kernel, eps=eps, lam=lam, delta=delta)
    assert np.all(np.abs(wv - we) <= bw + 1e-12)
    assert np.all(np.linalg.norm(gv - ge, axis=1) <= bg + 1e-9)
    assert len(far[0]) > len(q)          # the far field is used
    assert np.median(np.abs(wv - we) / np.maximum(bw, 1e-300)) < 0.5
    # every point is covered exactly once per query: far nodes + opened leaves
    counts = np.zeros(len(q))
    nleaf = T["nodes"] // 2
    lev = np.floor(np.log2(far[1])).astype(np.int64)
    span = 1 << (int(np.log2(nleaf)) - lev)
    first = far[1] * span - nleaf
    cnt_far = np.minimum((first + span) * leaf, n) - np.minimum(first * leaf, n)
    np.add.at(counts, far[0], cnt_far)
    lb = leaves[1] - nleaf
    np.add.at(counts, leaves[0], np.minimum((lb + 1) * leaf, n) - np.minimum(lb * leaf, n))
    np.testing.assert_array_equal(counts, n)


def test_verify_tree_catches_broken_hierarchies(oracle_mod):
    n = 3000
    p, _, a = _torus(n, 31)
    a = a * (1 + 0.5 * synth.uniform(3, 1, n))   # unequal weights
    T = bh_check.build_reference_tree(p, a, 16, 2.0)
    bh_check.verify_tree(T, p, a)
    nleaf = T["nodes"] // 2
    bad = []
    t = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in T.items()}
    t["radius"][nleaf + 5] *= 0.9                 # a leaf radius too small
    bad.append(t)
    t = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in T.items()}
    t["radius"][3] *= 0.99                        # an inner radius too small
    bad.append(t)
    t = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in T.items()}
    t["centre"][nleaf + 7, 1] += 1e-6             # a centre moved
    bad.append(t)
    t = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in T.items()}
    t["perm"][[0, 100]] = t["perm"][[100, 0]]     # two points in the wrong leaves
    bad.append(t)
    t = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in T.items()}
    t["area"][nleaf + 2] *= 1.001                 # an area off
    bad.append(t)
    for t in bad:
        with pytest.raises(AssertionError):
            bh_check.verify_tree(t, p, a)
