"""Pins of the oracle's modified Poisson kernel and its clamp radii (Sec. 5.2,
"Poisson Kernels"): closed forms of a single source and of the sphere's
centre, finite differences on each side of the radius, the plain kernel
outside every radius, and lattice values of delta_i."""
import math

import numpy as np
import pytest

import oracle
import synth


def test_single_source_inside_and_outside():
    p = np.array([[0.1, -0.2, 0.3]])
    n = np.array([[0.6, 0.0, 0.8]])
    a = np.array([2.0])
    m = a[0] * n[0] / (4 * math.pi)
    delta = np.array([0.5])
    q_in = np.array([[0.2, 0.0, 0.1]])        # |d| = 0.3 < 0.5
    q_out = np.array([[1.0, 0.4, -0.2]])
    for lam, kern in ((0.0, oracle.KERNEL_PLAIN), (30.0, oracle.KERNEL_SCREENED)):
        s = math.sqrt(lam)
        F = math.exp(-s * 0.5) * (1 + s * 0.5)
        w, g = oracle.gwn(p, n, a, q_in, kernel=kern, lam=lam, delta=delta)
        d = p[0] - q_in[0]
        assert abs(w[0] - F * (m @ d) / 0.125) < 1e-15
        np.testing.assert_allclose(g[0], -F * m / 0.125, rtol=1e-14)
        # outside every radius: the unsoftened kernel
        w1, g1 = oracle.gwn(p, n, a, q_out, kernel=kern, lam=lam, delta=delta)
        w2, g2 = oracle.gwn(p, n, a, q_out, kernel=kern, lam=lam, eps=0.0)
        assert w1[0] == w2[0] and np.array_equal(g1, g2)


def test_sphere_centre_closed_form():
    """Unit sphere, a_j = 4 pi / N, outward normals, every delta_j = 1.25 > 1:
    at the centre each term is <m_j, n_j> / delta^3, so w(0) = 1 / delta^3 for
    any sampling (and F(delta) times that when screened)."""
    _, nt = synth.sphere(3000, seed=3)
    p = nt  # FP64 points exactly on the sphere
    a = np.full(len(p), 4 * math.pi / len(p))
    delta = np.full(len(p), 1.25)
    w = oracle.gwn(p, nt, a, np.zeros((1, 3)), delta=delta, grad=False)
    assert abs(w[0] - 1.25 ** -3) < 1e-12
    lam = 4.0
    w = oracle.gwn(p, nt, a, np.zeros((1, 3)), kernel=oracle.KERNEL_SCREENED, lam=lam,
                   delta=delta, grad=False)
    F = math.exp(-2 * 1.25) * (1 + 2 * 1.25)
    assert abs(w[0] - F * 1.25 ** -3) < 1e-12


@pytest.mark.parametrize("lam", [0.0, 20.0])
def test_gradient_is_the_derivative_on_each_side(lam):
    p = synth.uniform_box(40, [-1] * 3, [1] * 3, seed=4).astype(np.float64)
    n = synth.random_unit_normals(40, seed=5)
    a = synth.uniform(6, 0, 40) + 0.5
    delta = 0.2 + 0.3 * synth.uniform(7, 0, 40)
    q = synth.uniform_box(60, [-1.2] * 3, [1.2] * 3, seed=8).astype(np.float64)
    kern = oracle.KERNEL_SCREENED if lam > 0 else oracle.KERNEL_PLAIN
    w, g = oracle.gwn(p, n, a, q, kernel=kern, lam=lam, delta=delta)
    h = 1e-6
    r = np.linalg.norm(p[None, :, :] - q[:, None, :], axis=2)
    far_from_edges = np.all(np.abs(r - delta[None, :]) > 1e-3, axis=1)
    assert far_from_edges.sum() > 30
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        wp = oracle.gwn(p, n, a, q + e, kernel=kern, lam=lam, delta=delta, grad=False)
        wm = oracle.gwn(p, n, a, q - e, kernel=kern, lam=lam, delta=delta, grad=False)
        fd = (wp - wm) / (2 * h)
        err = np.abs(fd - g[:, k])[far_from_edges]
        assert err.max() <= 1e-6 * max(1.0, np.abs(g[:, k]).max()), err.max()


def test_value_is_continuous_across_the_radius():
    p = np.array([[0.0, 0.0, 0.0]])
    n = np.array([[0.0, 0.0, 1.0]])
    delta = np.array([0.25])
    zs = np.array([0.25 - 1e-7, 0.25 + 1e-7])
    q = np.c_[np.zeros(2), np.zeros(2), -zs]
    w = oracle.gwn(p, n, np.ones(1), q, delta=delta, grad=False)
    assert abs(w[0] - w[1]) < 1e-5 * abs(w[0])


def test_clamp_radii_on_a_square_lattice():
    h = 0.0625
    g = np.stack(np.meshgrid(np.arange(9), np.arange(9), indexing="ij"), -1).reshape(-1, 2)
    p = np.c_[g * h, np.zeros(len(g))].astype(np.float32)
    centre = np.all(g == 4, axis=1)
    # 10 nearest other points of an interior node: 4 at h, 4 at h sqrt 2, 2 at 2h
    d = oracle.clamp_radii(p, 10, 0.5 * h, 3 * h)
    assert abs(d[centre][0] - (4 * h + 4 * math.sqrt(2) * h + 4 * h) / 10) < 1e-15
    d = oracle.clamp_radii(p, 10, 0.5 * h, 1.5 * h)
    assert abs(d[centre][0] - (4 * h + 4 * math.sqrt(2) * h) / 8) < 1e-15
    d = oracle.clamp_radii(p, 10, 3 * h, 4 * h)      # nothing in range: mean clamped up
    assert d[centre][0] == float(np.float32(3 * h))
    d = oracle.clamp_radii(p, 10, 0.1 * h, 0.5 * h)  # nothing in range: mean clamped down
    assert d[centre][0] == float(np.float32(0.5 * h))


def test_clamp_radii_skip_self_keep_copies():
    p = np.array([[0, 0, 0], [0, 0, 0], [1, 0, 0], [0, 2, 0]], np.float32)
    d = oracle.clamp_radii(p, 2, 0.5, 10.0)
    # point 0: nearest others are the copy (0, filtered out) and (1,0,0)
    assert d[0] == 1.0 and d[1] == 1.0
    # point 2: both copies at distance 1
    assert d[2] == 1.0


def _cloud(n=3000, seed=31):
    p, nt = synth.torus(n, seed=seed, noise=0.002)
    a = np.full(n, 4 * np.pi ** 2 * 0.3 / n)
    delta = oracle.clamp_radii(p, 10, 0.01, 0.1)
    q = np.vstack([p[:300], synth.uniform_box(200, [-1.4, -1.4, -0.5], [1.4, 1.4, 0.5], seed=seed)])
    return p, nt, a, delta, q


@pytest.mark.parametrize("lam", [0.0, 30.0])
def test_tree_with_every_node_open_is_the_exact_sum(lam):
    p, nt, a, delta, q = _cloud()
    kern = oracle.KERNEL_SCREENED if lam else oracle.KERNEL_PLAIN
    w0, g0 = oracle.gwn(p, nt, a, q, kernel=kern, lam=lam, delta=delta)
    w1, g1 = oracle.tree_gwn(p, nt, a, q, kernel=kern, lam=lam, beta=1e9, bucket=16, delta=delta)
    np.testing.assert_allclose(w1, w0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(g1, g0, rtol=1e-11, atol=1e-9)


def test_radii_larger_than_the_cloud_open_every_node():
    """With every delta beyond the cloud's size no node can be far (the opening
    radius is at least r + max delta), whatever beta: the exact sum again."""
    p, nt, a, _, q = _cloud(1500)
    big = np.full(len(p), 10.0)
    w0 = oracle.gwn(p, nt, a, q, delta=big, grad=False)
    w1, cnt = oracle.tree_gwn(p, nt, a, q, beta=2.0, bucket=16, delta=big, grad=False,
                              want_count=True)
    np.testing.assert_allclose(w1, w0, rtol=1e-12, atol=1e-12)
    q_in = np.all(np.isin(q, p), axis=1)
    assert np.all(cnt[~q_in] == len(p))


def test_tree_error_within_the_first_order_bound():
    """Far nodes hold no point within its radius of the query, so the plain
    kernel's far field is the unsoftened dipole and the first-order bound
    A r / (2 pi (d - r)^3) holds for the modified kernel too."""
    p, nt, a, delta, q = _cloud()
    w0 = oracle.gwn(p, nt, a, q, delta=delta, grad=False)
    for beta in (2.0, 3.0):
        w1, bnd = oracle.tree_gwn(p, nt, a, q, beta=beta, bucket=16, delta=delta, grad=False,
                                  want_bound=True)
        assert np.all(np.abs(w1 - w0) <= bnd + 1e-9 * (1 + np.abs(w0))), beta


def test_group_of_one_equals_the_per_query_test():
    p, nt, a, delta, q = _cloud(2000)
    w1, g1, c1 = oracle.tree_gwn(p, nt, a, q, kernel=oracle.KERNEL_SCREENED, lam=30.0, beta=2.5,
                                 bucket=32, delta=delta, want_count=True)
    w2, g2, c2 = oracle.tree_gwn_group(p, nt, a, q, kernel=oracle.KERNEL_SCREENED, lam=30.0,
                                       beta=2.5, bucket=32, group=1, delta=delta, want_count=True)
    assert np.array_equal(c1, c2)
    np.testing.assert_allclose(w2, w1, rtol=1e-12, atol=1e-12)
