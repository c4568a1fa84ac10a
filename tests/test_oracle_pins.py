"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, invariants, finite differences, library routines, analytic
shapes).  CPU only."""
import math

import numpy as np
import pytest

import synth


def _rot(seed):
    q = synth.normal(seed, 11, 4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


# ----------------------------------------------------------------------------
# Eq. 2/3 and Eq. 5: closed forms at the centre of a sphere
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("eps", [0.0, 0.04, 0.3])
def test_sphere_centre_plain(oracle_mod, eps):
    """a = 4 pi / N, outward normals on the unit sphere: every term equals
    rho^-3 / N, so w(0) = (1 + eps^2)^-3/2 for ANY sampling, and
    grad w(0) = (3 rho^-5 - rho^-3) * mean(p)."""
    n = 777
    _, u = synth.sphere(n, seed=4)   # float64 unit directions: points and normals
    a = np.full(n, 4 * np.pi / n)
    w, g = oracle_mod.gwn(u, u, a, np.zeros((1, 3)), eps=eps)
    rho = math.sqrt(1 + eps * eps)
    assert w[0] == pytest.approx(rho ** -3, rel=1e-13)
    np.testing.assert_allclose(g[0], (3 * rho ** -5 - rho ** -3) * u.mean(0), rtol=1e-10,
                               atol=1e-15)


@pytest.mark.parametrize("lam", [10.0, 100.0])
def test_sphere_centre_screened(oracle_mod, lam):
    """Eq. 5 at the centre: w = exp(-s rho)(1 + s rho) rho^-3, s = sqrt(lambda)."""
    n = 500
    _, nt = synth.sphere(n, seed=9)
    a = np.full(n, 4 * np.pi / n)
    eps = 0.05
    w, g = oracle_mod.gwn(nt, nt, a, np.zeros((1, 3)), kernel=1, eps=eps, lam=lam)
    s = math.sqrt(lam)
    rho = math.sqrt(1 + eps * eps)
    F = math.exp(-s * rho) * (1 + s * rho)
    assert w[0] == pytest.approx(F * rho ** -3, rel=1e-12)
    coef = F * (3 * rho ** -5 - rho ** -3) + s * s * math.exp(-s * rho) * rho ** -3
    np.testing.assert_allclose(g[0], coef * nt.mean(0), rtol=1e-9, atol=1e-15)


def test_screened_lambda_zero_is_plain(oracle_mod):
    p, nt = synth.torus(300, seed=2)
    n0 = synth.random_unit_normals(300, seed=3)
    a = np.full(300, 0.01)
    q = synth.uniform_box(50, [-1.5] * 3, [1.5] * 3, seed=4)
    w0, g0 = oracle_mod.gwn(p, n0, a, q, kernel=0, eps=0.02)
    w1, g1 = oracle_mod.gwn(p, n0, a, q, kernel=1, eps=0.02, lam=0.0)
    assert np.array_equal(w0, w1) and np.array_equal(g0, g1)


# ----------------------------------------------------------------------------
# continuum limits on a densely sampled sphere (Sec. 3: w = 1 inside, 0 outside)
# ----------------------------------------------------------------------------
def test_sphere_inside_outside_and_surface(oracle_mod):
    n = 20000
    p, u = synth.fibonacci_sphere(n)
    a = np.full(n, 4 * np.pi / n)
    h = math.sqrt(4 * np.pi / n)
    eps = 0.1 * h
    q = np.array([[0.3, 0.2, 0.1], [-0.5, 0.1, 0.4], [0.0, 0.0, 2.0], [1.5, -1.0, 0.5]])
    w = oracle_mod.gwn(p, u, a, q, eps=eps, grad=False)
    np.testing.assert_allclose(w[:2], 1.0, atol=1e-3)
    np.testing.assert_allclose(w[2:], 0.0, atol=1e-3)
    # on the surface (self term skipped): 1/2 for the plain kernel, and
    # (1 - e^{-2s}) / (2s) - e^{-2s} / 2 for the screened one (R = 1)
    ws = oracle_mod.gwn(p, u, a, p[::97], eps=eps, grad=False)
    np.testing.assert_allclose(ws, 0.5, atol=1e-2)
    for lam in (10.0, 100.0):
        s = math.sqrt(lam)
        ref = (1 - math.exp(-2 * s)) / (2 * s) - math.exp(-2 * s) / 2
        wl = oracle_mod.gwn(p, u, a, p[::97], kernel=1, eps=eps, lam=lam, grad=False)
        np.testing.assert_allclose(wl, ref, atol=1e-2)


# ----------------------------------------------------------------------------
# gradient: central finite differences of w
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("kernel,lam", [(0, 0.0), (1, 10.0), (1, 100.0)])
def test_gradient_finite_differences(oracle_mod, kernel, lam):
    p, _ = synth.torus(400, seed=1, noise=0.01)
    n0 = synth.random_unit_normals(400, seed=2)
    a = np.full(400, 4 * np.pi ** 2 * 0.3 / 400)
    q = synth.uniform_box(20, [-1.4, -1.4, -0.5], [1.4, 1.4, 0.5], seed=3).astype(np.float64)
    eps = 0.03
    _, g = oracle_mod.gwn(p, n0, a, q, kernel=kernel, eps=eps, lam=lam)
    hstep = 1e-5
    fd = np.zeros_like(g)
    for k in range(3):
        e = np.zeros(3)
        e[k] = hstep
        wp = oracle_mod.gwn(p, n0, a, q + e, kernel=kernel, eps=eps, lam=lam, grad=False)
        wm = oracle_mod.gwn(p, n0, a, q - e, kernel=kernel, eps=eps, lam=lam, grad=False)
        fd[:, k] = (wp - wm) / (2 * hstep)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())


# ----------------------------------------------------------------------------
# invariants
# ----------------------------------------------------------------------------
def test_linearity_in_normals(oracle_mod):
    p, _ = synth.sphere(300, seed=5)
    n0 = synth.random_unit_normals(300, seed=6)
    a = np.full(300, 0.04)
    q = synth.uniform_box(40, [-1.2] * 3, [1.2] * 3, seed=7)
    w, g = oracle_mod.gwn(p, n0, a, q, eps=0.05)
    wn, gn = oracle_mod.gwn(p, -n0, a, q, eps=0.05)
    assert np.array_equal(wn, -w) and np.array_equal(gn, -g)
    # flipping one normal changes the sums by exactly twice its term
    n1 = n0.copy()
    n1[17] = -n1[17]
    w1, g1 = oracle_mod.gwn(p, n1, a, q, eps=0.05)
    wt, gt = oracle_mod.gwn(p[17:18], n0[17:18], a[17:18], q, eps=0.05)
    np.testing.assert_allclose(w - w1, 2 * wt, atol=1e-13)
    np.testing.assert_allclose(g - g1, 2 * gt, atol=1e-12)


def test_rotation_translation_equivariance(oracle_mod):
    p, _ = synth.torus(300, seed=8)
    p = p.astype(np.float64)
    n0 = synth.random_unit_normals(300, seed=9)
    a = np.full(300, 0.02)
    q = synth.uniform_box(30, [-1.3] * 3, [1.3] * 3, seed=10).astype(np.float64)
    R = _rot(3)
    t = np.array([0.7, -2.1, 0.35])
    for kernel, lam in ((0, 0.0), (1, 25.0)):
        w, g = oracle_mod.gwn(p, n0, a, q, kernel=kernel, eps=0.02, lam=lam)
        w2, g2 = oracle_mod.gwn(p @ R.T + t, n0 @ R.T, a, q @ R.T + t, kernel=kernel, eps=0.02,
                                lam=lam)
        np.testing.assert_allclose(w2, w, atol=1e-10)
        np.testing.assert_allclose(g2, g @ R.T, atol=1e-9 * np.abs(g).max())


def test_coincident_source_is_skipped(oracle_mod):
    p, _ = synth.sphere(100, seed=11)
    p = p.astype(np.float64)
    n0 = synth.random_unit_normals(100, seed=12)
    a = np.full(100, 0.1)
    # duplicate point 5 as point 100; query at that location
    p2 = np.vstack([p, p[5:6]])
    n2 = np.vstack([n0, n0[40:41]])
    a2 = np.append(a, 0.3)
    w, g = oracle_mod.gwn(p2, n2, a2, p[5:6], eps=0.01)
    keep = [j for j in range(101) if j not in (5, 100)]
    wr, gr = oracle_mod.gwn(p2[keep], n2[keep], a2[keep], p[5:6], eps=0.01)
    assert w[0] == wr[0] and np.array_equal(g, gr)


# ----------------------------------------------------------------------------
# Sec. 5.1 convergence measure: mean of the largest 1 %
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 7, 99, 100, 101, 1000, 12345])
def test_top1_mean_against_sort(oracle_mod, n):
    v = 180 * synth.uniform(3, n, n)
    k = -(-n // 100)
    ref = np.sort(v)[::-1][:k].mean()
    assert oracle_mod.top1_mean(v) == pytest.approx(ref, rel=1e-14)
    # ties: the mean of the k largest is unique whatever the order
    v2 = np.round(v / 30) * 30
    assert oracle_mod.top1_mean(v2) == pytest.approx(np.sort(v2)[::-1][:k].mean(), rel=1e-14)


# ----------------------------------------------------------------------------
# Sec. 5.1 octree around the cloud
# ----------------------------------------------------------------------------
def test_cube_and_cells(oracle_mod):
    p = np.array([[0.0, 0.0, 0.0], [2.0, 1.0, 0.5], [1.0, 0.25, 0.25]], dtype=np.float32)
    c = oracle_mod.cube(p, 3)
    # extent 2 -> edge 2.25, centred on (1, 0.5, 0.25)
    assert c["L"] == 2.25
    np.testing.assert_array_equal(c["lo"], [1 - 1.125, 0.5 - 1.125, 0.25 - 1.125])
    cl = oracle_mod.cells(p, 3)
    # cell = floor((x - lo) * 8 / 2.25)
    ref = np.floor((p.astype(np.float64) - c["lo"]) * (8 / 2.25)).astype(np.int64)
    np.testing.assert_array_equal(cl, ref)


@pytest.mark.parametrize("depth", [1, 3, 5])
def test_octree_leaves_partition_the_cube(oracle_mod, depth):
    p, _ = synth.torus(700, seed=5, noise=0.01)
    L = oracle_mod.octree_leaves(p, depth)
    # leaves tile the root cube: volumes add up to 1
    assert np.sum(8.0 ** (-L[:, 0])) == pytest.approx(1.0, abs=1e-12)
    # non-empty leaves are exactly the distinct depth-d cells of the points
    ne = L[L[:, 4] == 1]
    assert np.all(ne[:, 0] == depth)
    cells = {tuple(c) for c in oracle_mod.cells(p, depth)}
    assert {tuple(r) for r in ne[:, 1:4]} == cells
    # empty leaves contain no point, and every empty leaf's parent holds points
    for lev, ix, iy, iz, _ in L[L[:, 4] == 0]:
        sh = depth - lev
        inside = [c for c in cells if (c[0] >> sh, c[1] >> sh, c[2] >> sh) == (ix, iy, iz)]
        assert not inside
        par = [c for c in cells
               if (c[0] >> (sh + 1), c[1] >> (sh + 1), c[2] >> (sh + 1)) == (ix >> 1, iy >> 1, iz >> 1)]
        assert par


def test_corner_set(oracle_mod):
    d = 4
    p, _ = synth.sphere(500, seed=6)
    L = oracle_mod.octree_leaves(p, d)
    K = oracle_mod.corner_keys(L, d)
    S1 = 2 ** d + 1
    ref = set()
    for lev, ix, iy, iz, _ in L:
        s = 2 ** (d - lev)
        for v in range(8):
            X = (ix + (v & 1)) * s
            Y = (iy + ((v >> 1) & 1)) * s
            Z = (iz + ((v >> 2) & 1)) * s
            ref.add((X * S1 + Y) * S1 + Z)
    assert list(K) == sorted(ref)


# ----------------------------------------------------------------------------
# level-set faces (Alg. 1, Marching Cubes step)
# ----------------------------------------------------------------------------
def _all_leaf_faces(oracle_mod, p, depth, field, iso):
    L = oracle_mod.octree_leaves(p, depth)
    K = oracle_mod.corner_keys(L, depth)
    cb = oracle_mod.cube(p, depth)
    X = oracle_mod.corner_positions(K, depth, cb)
    return oracle_mod.faces(L, depth, cb, K, field(X), iso), cb


def test_faces_of_a_linear_field_tile_the_plane(oracle_mod):
    """For a linear field the piecewise-linear interpolant is exact: the faces
    tile the plane's section of the root cube, all oriented along +grad."""
    p, _ = synth.sphere(400, seed=7)
    gdir = np.array([0.3, -0.5, 0.8])
    gdir /= np.linalg.norm(gdir)
    F, cb = _all_leaf_faces(oracle_mod, p, 4, lambda X: X @ gdir, 0.1)
    A = F[:, :3]
    C = F[:, 3:]
    areas = np.linalg.norm(A, axis=1)
    assert np.all(A @ gdir >= areas * (1 - 1e-9))          # oriented along +grad
    np.testing.assert_allclose(C @ gdir, 0.1, atol=1e-6)    # centroids on the plane
    # total area equals the area of the plane section of the cube, computed
    # independently by Monte Carlo-free exact polygon clipping (sum of the
    # section of each finest cell is not needed: use the cube's section)
    lo, Lc = cb["lo"], cb["L"]
    area = _plane_cube_section_area(gdir, 0.1, lo, Lc)
    assert A.sum(0) @ gdir == pytest.approx(area, rel=1e-6)


def _plane_cube_section_area(nv, c, lo, L):
    """Area of {x : n.x = c} inside the axis-aligned cube [lo, lo + L]^3 by
    clipping a large square in the plane against the six faces."""
    u = np.cross(nv, [1.0, 0.0, 0.0] if abs(nv[0]) < 0.9 else [0.0, 1.0, 0.0])
    u /= np.linalg.norm(u)
    v = np.cross(nv, u)
    o = nv * c
    Rr = 10 * L + np.linalg.norm(lo)
    poly = [o + Rr * (su * u + sv * v) for su, sv in ((-1, -1), (1, -1), (1, 1), (-1, 1))]
    for ax in range(3):
        for side, bound in ((1, lo[ax]), (-1, lo[ax] + L)):
            out = []
            for i in range(len(poly)):
                P, Q = poly[i], poly[(i + 1) % len(poly)]
                fp, fq = side * (P[ax] - bound), side * (Q[ax] - bound)
                if fp >= 0:
                    out.append(P)
                if (fp >= 0) != (fq >= 0):
                    out.append(P + (Q - P) * (fp / (fp - fq)))
            poly = out
    s = np.zeros(3)
    for i in range(len(poly)):
        s += np.cross(poly[i], poly[(i + 1) % len(poly)])
    return 0.5 * abs(s @ nv)


def test_faces_of_a_sphere_field(oracle_mod):
    """w = |x - c|^2 at iso r^2: faces approximate the sphere, oriented outward
    (toward increasing w), total area -> 4 pi r^2."""
    # points filling the cube make every leaf a finest cell (a uniform grid)
    p = synth.uniform_box(40000, [-1] * 3, [1] * 3, seed=8)
    c0 = np.array([0.05, -0.02, 0.01])
    r = 0.6
    F, _ = _all_leaf_faces(oracle_mod, p, 4, lambda X: ((X - c0) ** 2).sum(1), r * r)
    A, C = F[:, :3], F[:, 3:]
    radial = (C - c0) / np.linalg.norm(C - c0, axis=1, keepdims=True)
    assert np.all(np.sum(A * radial, axis=1) > 0)
    np.testing.assert_allclose(np.linalg.norm(C - c0, axis=1), r, atol=0.02)
    tot = np.linalg.norm(A, axis=1).sum()
    assert tot == pytest.approx(4 * np.pi * r * r, rel=0.05)
    # closed surface: the vector areas cancel
    assert np.linalg.norm(A.sum(0)) < 1e-9 * tot


# ----------------------------------------------------------------------------
# k nearest points (Eq. 7's face-to-point assignment)
# ----------------------------------------------------------------------------
def test_knn_against_kdtree(oracle_mod):
    spatial = pytest.importorskip("scipy.spatial")
    p = synth.uniform_box(3000, [-1] * 3, [1] * 3, seed=1).astype(np.float64)
    q = synth.uniform_box(500, [-1.2] * 3, [1.2] * 3, seed=2).astype(np.float64)
    idx = oracle_mod.knn(p, q, 10)
    d, ref = spatial.cKDTree(p).query(q, k=10)
    np.testing.assert_array_equal(idx, ref)


def test_knn_ties_go_to_smaller_index(oracle_mod):
    # a query equidistant from all points of a regular grid patch
    p = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                  [2, 0, 0]], dtype=np.float64)
    idx = oracle_mod.knn(p[::-1].copy(), np.zeros((1, 3)), 3)
    # reversed order: indices 1..6 are the unit points; the three smallest win
    np.testing.assert_array_equal(idx[0], [1, 2, 3])
    idx = oracle_mod.knn(p[:2], np.zeros((1, 3)), 4)
    np.testing.assert_array_equal(idx[0], [0, 1, -1, -1])


# ----------------------------------------------------------------------------
# Eq. 7 scatter and the normal-change measure
# ----------------------------------------------------------------------------
def test_scatter_single_face(oracle_mod):
    p = synth.uniform_box(50, [-1] * 3, [1] * 3, seed=3).astype(np.float64)
    n_old = synth.random_unit_normals(50, seed=4)
    A = np.array([0.2, -0.1, 0.4])
    c = np.array([0.1, 0.2, -0.3])
    face = np.concatenate([A, c])[None, :]
    out = oracle_mod.scatter_normals(p, face, 10, n_old)
    near = set(np.argsort(np.linalg.norm(p - c, axis=1))[:10])
    for j in range(50):
        if j in near:
            np.testing.assert_allclose(out[j], -A / np.linalg.norm(A), atol=1e-15)
        else:
            np.testing.assert_array_equal(out[j], n_old[j])


def test_direct_step_and_dtheta(oracle_mod):
    p, _ = synth.sphere(300, seed=13)
    a = np.full(300, 4 * np.pi / 300)
    n0 = synth.random_unit_normals(300, seed=14)
    prm = oracle_mod.params(eps=0.05, mode=oracle_mod.MODE_DIRECT)
    r = oracle_mod.iterate(p, a, n0, prm)
    g = r["g"]
    np.testing.assert_allclose(r["normals"], -g / np.linalg.norm(g, axis=1, keepdims=True),
                               atol=1e-15)
    ang = np.degrees(np.arccos(np.clip(np.sum(n0 * r["normals"], axis=1), -1, 1)))
    np.testing.assert_allclose(r["dtheta"], ang, atol=1e-6)
    assert r["iso"] == pytest.approx(r["w"].mean(), rel=1e-14)


def test_oracle_rounding_against_extended_precision(oracle_mod):
    """Precision check (not an independent pin: the same definition, Eq. 2/3/5
    and their gradients, evaluated in numpy's extended long double): on 150
    points the FP64 oracle's w and grad w agree to 1e-12 of the sum of the
    terms' magnitudes, for the plain and the screened kernel."""
    import math
    if np.finfo(np.longdouble).eps >= np.finfo(np.float64).eps:
        pytest.skip("long double is no wider than double here")
    p = synth.uniform_box(150, [-1] * 3, [1] * 3, seed=71).astype(np.float64)
    nrm = synth.random_unit_normals(150, seed=72)
    a = synth.uniform(73, 0, 150) + 0.5
    q = synth.uniform_box(40, [-1.3] * 3, [1.3] * 3, seed=74).astype(np.float64)
    eps = 0.05
    L = np.longdouble
    for lam in (0.0, 25.0):
        kern = oracle_mod.KERNEL_SCREENED if lam else oracle_mod.KERNEL_PLAIN
        w, g = oracle_mod.gwn(p, nrm, a, q, kernel=kern, eps=eps, lam=lam)
        s = np.sqrt(L(lam))
        for i in range(len(q)):
            d = p.astype(L) - q[i].astype(L)
            m = a.astype(L)[:, None] * nrm.astype(L) / (L(4) * L(math.pi))
            rho2 = np.sum(d * d, axis=1) + L(eps) * L(eps)
            rho = np.sqrt(rho2)
            phi = np.sum(m * d, axis=1) / (rho2 * rho)
            E = np.exp(-s * rho)
            F = E * (1 + s * rho) if lam else np.ones_like(rho)
            t = F * phi
            gphi = -m / (rho2 * rho)[:, None] + 3 * (phi / rho2)[:, None] * d
            gt = F[:, None] * gphi + ((phi * s * s * E)[:, None] * d if lam else 0)
            assert abs(w[i] - float(t.sum())) <= 1e-12 * float(np.abs(t).sum())
            tol = 1e-12 * float(np.abs(gt).sum(axis=0).max())
            assert np.max(np.abs(g[i] - gt.sum(axis=0).astype(np.float64))) <= tol
