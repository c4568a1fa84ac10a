"""Pins of the oracle's PCA and Gauss-map initial normals (Sec. 5.1, "Normal
Initialization") against closed forms, an independent construction (SVD of
the neighbourhood found by a full sort) and invariants."""
import numpy as np
import pytest

import oracle
import synth


def _rot(seed):
    q, r = np.linalg.qr(synth.normal(seed, 3, 9).reshape(3, 3))
    return q * np.sign(np.diag(r))


def test_pca_on_a_plane_is_the_plane_normal():
    R = _rot(1)
    uv = synth.uniform(2, 0, 2 * 400).reshape(400, 2) * 2 - 1
    p = (np.c_[uv, np.zeros(400)] @ R.T + [0.3, -0.2, 0.1]).astype(np.float32)
    n, gap = oracle.pca_normals(p)
    # float32 rounding of the points tilts the plane by ~1e-7 per neighbourhood
    assert np.max(1 - np.abs(n @ R[:, 2])) < 1e-10
    assert np.median(gap) > 0.1


def test_pca_on_a_vertical_plane_points_toward_plus_x():
    """n_z = 0 exactly: the sign rule falls through to n_y = 0, then n_x > 0."""
    g = np.stack(np.meshgrid(np.arange(6), np.arange(6), indexing="ij"), -1).reshape(-1, 2)
    p = np.c_[np.full(36, 2.0), g * 0.25].astype(np.float32)
    n, _ = oracle.pca_normals(p)
    np.testing.assert_allclose(n, np.tile([1.0, 0.0, 0.0], (36, 1)), atol=1e-12)


def test_pca_sign_rule():
    p, _ = synth.torus(2000, seed=3, noise=0.002)
    n, _ = oracle.pca_normals(p)
    p64 = p.astype(np.float64)
    c = 0.5 * (p64.min(axis=0) + p64.max(axis=0))
    assert np.all(np.sum(n * (p64 - c), axis=1) >= 0)


def test_pca_on_an_ellipsoid_is_the_outward_normal():
    """A convex cloud around its box centre: PCA lines with the Gauss-map
    side are the outward normals up to the O(h) tilt of the fit."""
    p, nt = synth.ellipsoid_points(20000, (1.0, 0.6, 0.4), seed=3, stream=2)
    p = np.ascontiguousarray(p, np.float32)
    n, _ = oracle.pca_normals(p)
    assert np.min(np.sum(n * nt, axis=1)) > 0.95


def test_pca_on_a_sphere_is_radial():
    p = synth.fibonacci_sphere(20000)[0]
    n, _ = oracle.pca_normals(p)
    r = p / np.linalg.norm(p, axis=1, keepdims=True)
    cosang = np.abs(np.sum(n * r, axis=1))
    # neighbourhood radius h ~ 0.04: the tilt is O(h^2)
    assert cosang.min() > 1 - 1e-3


def test_pca_equals_smallest_singular_vector_of_the_sorted_neighbourhood():
    """Independent route: neighbours by a full lexicographic sort of (distance,
    index), the line as the last right singular vector of the centred
    neighbourhood matrix."""
    p = synth.add_noise(synth.sphere(60, seed=4)[0], 0.05, seed=5)
    n, gap = oracle.pca_normals(p, k=10)
    p64 = p.astype(np.float64)
    for i in range(len(p)):
        d2 = np.sum((p64 - p64[i]) ** 2, axis=1)
        nb = np.lexsort((np.arange(len(p)), d2))[:10]
        X = p64[nb] - p64[i]
        X = X - X.mean(axis=0)
        v = np.linalg.svd(X)[2][-1]
        assert abs(abs(np.dot(v, n[i])) - 1) < 1e-10 / max(gap[i], 1e-3), i


def test_pca_rotation_and_translation_equivariance():
    p, _ = synth.torus(1500, seed=6, noise=0.001)
    R = _rot(7)
    q = (p.astype(np.float64) @ R.T + [1.0, 2.0, -3.0]).astype(np.float32)
    a, ga = oracle.pca_normals(p)
    b, gb = oracle.pca_normals(q)
    ok = (ga > 0.1) & (gb > 0.1)
    assert ok.mean() > 0.9
    cosang = np.abs(np.sum((a @ R.T) * b, axis=1))
    assert np.all(cosang[ok] > 1 - 1e-6)


def test_pca_zero_covariance_is_nan():
    p = np.r_[np.zeros((12, 3)), synth.uniform_box(50, [1] * 3, [2] * 3, seed=8)].astype(np.float32)
    n, gap = oracle.pca_normals(p)
    assert np.all(np.isnan(n[:12])) and np.all(gap[:12] == 0)
    assert not np.any(np.isnan(n[12:]))


def test_pca_fewer_points_than_k():
    p = synth.uniform_box(5, [0] * 3, [1] * 3, seed=9)
    n, _ = oracle.pca_normals(p)
    assert n.shape == (5, 3) and np.allclose(np.linalg.norm(n, axis=1), 1)


def test_gauss_map_of_axis_points():
    e = np.eye(3)
    p = (np.r_[e, -e] * 1.5 + [0.5, 0.25, -2.0]).astype(np.float32)
    n = oracle.gauss_map_normals(p)
    np.testing.assert_array_equal(n, np.r_[e, -e])


def test_gauss_map_of_a_symmetric_sphere_is_the_analytic_normal():
    h = synth.fibonacci_sphere(1000)[0].astype(np.float64)
    p = np.r_[h, -h, [[2.0, 0, 0], [-2.0, 0, 0]]].astype(np.float32)  # box centre exactly 0
    n = oracle.gauss_map_normals(p)
    r = p.astype(np.float64) / np.linalg.norm(p.astype(np.float64), axis=1, keepdims=True)
    np.testing.assert_allclose(n, r, atol=1e-15)


def test_gauss_map_translation_invariance_and_centre_point():
    g = np.stack(np.meshgrid(*[np.arange(-3, 4)] * 3, indexing="ij"), -1).reshape(-1, 3)
    p = (g * 0.125).astype(np.float32)
    a = oracle.gauss_map_normals(p)
    b = oracle.gauss_map_normals(p + np.float32(4.0))
    centre = np.all(g == 0, axis=1)
    assert np.all(np.isnan(a[centre])) and np.all(np.isnan(b[centre]))
    np.testing.assert_array_equal(a[~centre], b[~centre])


def test_gauss_map_centre_is_the_bounding_box_centre_not_the_centroid():
    p = np.r_[np.eye(3), -np.eye(3), [[0.9, 0.9, 0.9]] * 5].astype(np.float32)
    n = oracle.gauss_map_normals(p)
    p64 = p.astype(np.float64)
    np.testing.assert_allclose(n, p64 / np.linalg.norm(p64, axis=1, keepdims=True), atol=1e-15)
