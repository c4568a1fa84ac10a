"""Pins of the oracle's local-Voronoi area weights (Sec. 5.1, "Computing Area
Weights"): lattice closed forms, the cell areas of a full 2D Voronoi diagram
(scipy/Qhull), an independent polar integral for the disk-cut cells,
invariants, and the total area of a sphere."""
import math

import numpy as np
import pytest

import oracle
import synth


def _rot(seed):
    q, r = np.linalg.qr(synth.normal(seed, 3, 9).reshape(3, 3))
    return q * np.sign(np.diag(r))


def _embed(uv, seed, shift=(0.2, -0.4, 0.7)):
    R = _rot(seed)
    return (np.c_[uv, np.zeros(len(uv))] @ R.T + shift).astype(np.float32)


def test_square_lattice_interior_cells_are_h_squared():
    h = 0.0625  # exact in float32
    g = np.stack(np.meshgrid(np.arange(12), np.arange(12), indexing="ij"), -1).reshape(-1, 2)
    p = np.c_[g * h, np.zeros(len(g))].astype(np.float32)
    a = oracle.voronoi_weights(p)
    inner = np.all((g >= 3) & (g <= 8), axis=1)
    np.testing.assert_allclose(a[inner], h * h, rtol=1e-12)


def test_hexagonal_lattice_interior_cells():
    h = 0.05
    i, j = np.meshgrid(np.arange(14), np.arange(14), indexing="ij")
    uv = np.stack([h * (i + 0.5 * (j % 2)), h * (math.sqrt(3) / 2) * j], -1).reshape(-1, 2)
    p = _embed(uv, 3)
    a = oracle.voronoi_weights(p)
    ij = np.stack([i, j], -1).reshape(-1, 2)
    inner = np.all((ij >= 4) & (ij <= 9), axis=1)
    # float32 positions: relative rounding ~1e-7 of coordinates of size ~1
    np.testing.assert_allclose(a[inner], (math.sqrt(3) / 2) * h * h, rtol=2e-4)


def test_bounded_cells_match_a_full_voronoi_diagram():
    scipy_spatial = pytest.importorskip("scipy.spatial")
    uv = synth.uniform(4, 0, 2 * 600).reshape(600, 2)
    p = _embed(uv, 5)
    a = oracle.voronoi_weights(p)
    # the oracle's plane frame is the embedding's plane: compare in 2D
    uv32 = ((p.astype(np.float64) - [0.2, -0.4, 0.7]) @ _rot(5))[:, :2]
    vor = scipy_spatial.Voronoi(uv32)
    checked = 0
    idx = oracle.knn(p, p, 16)
    for i in range(len(p)):
        reg = vor.regions[vor.point_region[i]]
        if not reg or -1 in reg:
            continue
        V = vor.vertices[reg]
        nb = [j for j in idx[i] if j != i][:15]
        R = 0.5 * np.max(np.linalg.norm(uv32[nb] - uv32[i], axis=1))
        if np.max(np.linalg.norm(V - uv32[i], axis=1)) >= R:
            continue  # cut by the disk
        # every Voronoi neighbour must be among the 15 nearest points
        vn = set(np.r_[vor.ridge_points[np.any(vor.ridge_points == i, axis=1)].ravel()]) - {i}
        if not vn <= set(nb):
            continue
        area = scipy_spatial.ConvexHull(V).volume
        assert abs(a[i] - area) <= 1e-6 * area, (i, a[i], area)
        checked += 1
    assert checked > 300


def test_disk_cut_cells_match_a_polar_integral():
    """Points on the hull of their neighbourhood: area = integral over the
    direction phi of min(rho(phi), R)^2 / 2, rho the distance to the cell
    boundary (the cell is star-shaped about its seed)."""
    uv = synth.uniform(6, 0, 2 * 60).reshape(60, 2)
    p = np.c_[uv, np.zeros(60)].astype(np.float32)
    a = oracle.voronoi_weights(p)
    idx = oracle.knn(p, p, 16)
    P = p[:, :2].astype(np.float64)
    phi = (np.arange(200000) + 0.5) * (2 * math.pi / 200000)
    u = np.stack([np.cos(phi), np.sin(phi)], 1)
    hull_like = 0
    for i in range(0, 60, 3):
        nb = [j for j in idx[i] if j != i][:15]
        q = P[nb] - P[i]
        R = 0.5 * np.max(np.linalg.norm(q, axis=1))
        dots = u @ q.T
        with np.errstate(divide="ignore"):
            t = np.where(dots > 0, 0.5 * np.sum(q * q, axis=1) / dots, np.inf)
        rho = np.minimum(t.min(axis=1), R)
        area = 0.5 * np.mean(rho ** 2) * 2 * math.pi
        hull_like += int(np.any(t.min(axis=1) > R))
        assert abs(a[i] - area) <= 1e-6 * area, (i, a[i], area)
    assert hull_like >= 3


def test_scale_rotation_translation():
    p, _ = synth.torus(1200, seed=7, noise=0.0)
    a = oracle.voronoi_weights(p)
    R = _rot(8)
    q = (p.astype(np.float64) @ R.T * 2.0 + [3, -1, 2]).astype(np.float32)
    b = oracle.voronoi_weights(q)
    rel = np.abs(b / (4 * a) - 1)
    assert np.median(rel) < 1e-5 and np.mean(rel < 1e-3) > 0.99


def test_sphere_total_area():
    p = synth.fibonacci_sphere(20000)[0]
    a = oracle.voronoi_weights(p)
    assert abs(a.sum() / (4 * math.pi) - 1) < 5e-3
    assert a.min() > 0


def test_coincident_copies_and_degenerate_neighbourhoods():
    p = np.r_[np.zeros((17, 3)), synth.uniform_box(200, [1] * 3, [2] * 3, seed=9)].astype(np.float32)
    p[17:, 2] = 1.5  # a planar patch away from the 17 copies
    a = oracle.voronoi_weights(p)
    good = a[17:]
    assert np.all(good > 0)
    np.testing.assert_allclose(a[:17], good.mean(), rtol=1e-12)


def test_single_point_and_copies_take_the_default_weight():
    assert np.array_equal(oracle.voronoi_weights(np.zeros((1, 3), np.float32)), [1.0])
    assert np.array_equal(oracle.voronoi_weights(np.zeros((4, 3), np.float32)), np.ones(4))
