"""FP64 CPU oracle for the Diffusing Winding Gradients iteration.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg are the only callers.  The CUDA library never
imports or links this package, and this package never imports the CUDA
library.

The arithmetic lives in ``dwg_oracle.c`` (plain C, double precision, OpenMP
over independent outputs); this module compiles it with gcc and wraps each
entry point with numpy arrays.  Section and equation numbers refer to the
paper (Diffusing Winding Gradients, arXiv 2405.13839).

Parity status: every function here is pinned by tests against closed forms,
invariants, library routines or analytic shapes (tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dwg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libdwg_oracle.so")
_lock = threading.Lock()
_lib = None

KERNEL_PLAIN = 0
KERNEL_SCREENED = 1
MODE_LEVELSET = 0
MODE_DIRECT = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("eps", ctypes.c_double),
                ("lmbda", ctypes.c_double), ("depth", ctypes.c_int),
                ("knn", ctypes.c_int), ("mode", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("tol", ctypes.c_double), ("rule", ctypes.c_int),
                ("delta", ctypes.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.dwgo_gwn.argtypes = [i64, P, P, P, i64, P, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, P, P, P]
            lib.dwgo_cube.argtypes = [i64, P, ctypes.c_int, P]
            lib.dwgo_cells.argtypes = [i64, P, ctypes.c_int, P]
            lib.dwgo_octree.argtypes = [i64, P, ctypes.c_int, P, i64]
            lib.dwgo_octree.restype = i64
            lib.dwgo_corners.argtypes = [i64, P, ctypes.c_int, P, i64]
            lib.dwgo_corners.restype = i64
            lib.dwgo_corner_positions.argtypes = [i64, P, ctypes.c_int, P, P]
            lib.dwgo_faces.argtypes = [i64, P, ctypes.c_int, P, i64, P, P, ctypes.c_double,
                                       P, i64]
            lib.dwgo_faces.restype = i64
            lib.dwgo_knn.argtypes = [i64, P, i64, P, ctypes.c_int, P]
            lib.dwgo_set_threads.argtypes = [ctypes.c_int]
            lib.dwgo_set_threads.restype = ctypes.c_int
            lib.dwgo_top1_mean.argtypes = [i64, P]
            lib.dwgo_top1_mean.restype = ctypes.c_double
            lib.dwgo_scatter_normals.argtypes = [i64, P, i64, P, ctypes.c_int, P, P]
            lib.dwgo_iterate.argtypes = [i64, P, P, P, ctypes.POINTER(_Params), P, P, P, P, P]
            lib.dwgo_iterate.restype = i64
            lib.dwgo_orient.argtypes = [i64, P, P, P, ctypes.POINTER(_Params), P,
                                        ctypes.POINTER(ctypes.c_int), P, P]
            lib.dwgo_orient.restype = ctypes.c_int
            lib.dwgo_morton_order.argtypes = [i64, P, P]
            lib.dwgo_tree_gwn.argtypes = [i64, P, P, P, i64, P, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int, P, P,
                                          P, P, P]
            lib.dwgo_tree_gwn_group.argtypes = [i64, P, P, P, i64, P, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_int, ctypes.c_int, P,
                                                P, P, P]
            _lib = lib
    return _lib


def _d(x, shape_last=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape_last is not None:
        a = a.reshape(-1, shape_last)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def gwn(points, normals, weights, queries, kernel=KERNEL_PLAIN, eps=0.0, lam=0.0,
        grad=True, delta=None):
    """w and grad w at queries (Eq. 2/3; Eq. 5 when kernel is screened).
    delta: per-source radii of the modified kernel (Sec. 5.2), which then
    replaces the softening eps."""
    lib = _load()
    p = _d(points, 3)
    nn = _d(normals, 3)
    a = _d(weights).ravel()
    q = _d(queries, 3)
    dl = None if delta is None else _d(delta).ravel()
    w = np.zeros(len(q))
    g = np.zeros((len(q), 3)) if grad else None
    lib.dwgo_gwn(len(p), _ptr(p), _ptr(nn), _ptr(a), len(q), _ptr(q), int(kernel),
                 float(eps), float(lam), _ptr(dl) if dl is not None else None, _ptr(w),
                 _ptr(g) if grad else None)
    return (w, g) if grad else w


def cube(points, depth):
    lib = _load()
    p = _d(points, 3)
    out = np.zeros(6)
    lib.dwgo_cube(len(p), _ptr(p), int(depth), _ptr(out))
    return dict(lo=out[:3].copy(), L=out[3], h=out[4], inv_h=out[5])


def cells(points, depth):
    lib = _load()
    p = _d(points, 3)
    out = np.zeros((len(p), 3), dtype=np.int64)
    lib.dwgo_cells(len(p), _ptr(p), int(depth), _ptr(out))
    return out


def octree_leaves(points, depth):
    """Leaves (level, ix, iy, iz, nonempty) of the depth-d octree (Sec. 5.1)."""
    lib = _load()
    p = _d(points, 3)
    nl = lib.dwgo_octree(len(p), _ptr(p), int(depth), None, 0)
    out = np.zeros((nl, 5), dtype=np.int64)
    lib.dwgo_octree(len(p), _ptr(p), int(depth), _ptr(out), nl)
    return out


def corner_keys(leaves, depth):
    lib = _load()
    L = np.ascontiguousarray(leaves, dtype=np.int64)
    nc = lib.dwgo_corners(len(L), _ptr(L), int(depth), None, 0)
    out = np.zeros(nc, dtype=np.int64)
    lib.dwgo_corners(len(L), _ptr(L), int(depth), _ptr(out), nc)
    return out


def corner_positions(keys, depth, cube_info):
    lib = _load()
    k = np.ascontiguousarray(keys, dtype=np.int64)
    c = np.array(list(cube_info["lo"]) + [cube_info["L"], cube_info["h"], cube_info["inv_h"]])
    out = np.zeros((len(k), 3))
    lib.dwgo_corner_positions(len(k), _ptr(k), int(depth), _ptr(c), _ptr(out))
    return out


def faces(leaves, depth, cube_info, keys, wc, iso):
    """Level-set faces: rows (area vector xyz, centroid xyz)."""
    lib = _load()
    L = np.ascontiguousarray(leaves, dtype=np.int64)
    k = np.ascontiguousarray(keys, dtype=np.int64)
    w = _d(wc).ravel()
    c = np.array(list(cube_info["lo"]) + [cube_info["L"], cube_info["h"], cube_info["inv_h"]])
    nf = lib.dwgo_faces(len(L), _ptr(L), int(depth), _ptr(c), len(k), _ptr(k), _ptr(w),
                        float(iso), None, 0)
    out = np.zeros((nf, 6))
    lib.dwgo_faces(len(L), _ptr(L), int(depth), _ptr(c), len(k), _ptr(k), _ptr(w),
                   float(iso), _ptr(out), nf)
    return out


def set_threads(n):
    """OpenMP threads of the oracle's parallel loops (n <= 0: the default);
    returns the count in effect."""
    return _load().dwgo_set_threads(int(n))


def knn(points, queries, k):
    lib = _load()
    p = _d(points, 3)
    q = _d(queries, 3)
    out = np.zeros((len(q), k), dtype=np.int64)
    lib.dwgo_knn(len(p), _ptr(p), len(q), _ptr(q), int(k), _ptr(out))
    return out


def top1_mean(values):
    lib = _load()
    v = _d(values).ravel()
    return lib.dwgo_top1_mean(len(v), _ptr(v))


def scatter_normals(points, face_rows, k, n_old):
    lib = _load()
    p = _d(points, 3)
    f = _d(face_rows, 6)
    no = _d(n_old, 3)
    out = np.zeros_like(no)
    lib.dwgo_scatter_normals(len(p), _ptr(p), len(f), _ptr(f), int(k), _ptr(no), _ptr(out))
    return out


def params(kernel=KERNEL_PLAIN, eps=0.0, lam=0.0, depth=6, knn=10, mode=MODE_LEVELSET,
           max_iters=30, tol=0.1, rule=0, delta=None):
    """delta: per-point radii of the modified kernel (Sec. 5.2) or None."""
    dl = None if delta is None else _d(delta).ravel()
    prm = _Params(int(kernel), float(eps), float(lam), int(depth), int(knn), int(mode),
                  int(max_iters), float(tol), int(rule), dl.ctypes.data if dl is not None else None)
    prm._delta_keep = dl  # the struct points into this array
    return prm


def iterate(points, weights, n_old, prm):
    """One iteration of Algorithm 1 from normals n_old."""
    lib = _load()
    p = _d(points, 3)
    a = _d(weights).ravel()
    no = _d(n_old, 3)
    nn = np.zeros_like(no)
    dth = np.zeros(len(p))
    wp = np.zeros(len(p))
    gp = np.zeros((len(p), 3))
    iso = ctypes.c_double()
    nf = lib.dwgo_iterate(len(p), _ptr(p), _ptr(a), _ptr(no), ctypes.byref(prm), _ptr(nn),
                          _ptr(dth), _ptr(wp), _ptr(gp), ctypes.byref(iso))
    return dict(normals=nn, dtheta=dth, w=wp, g=gp, iso=iso.value, faces=nf)


def orient(points, weights, n0, prm):
    """Algorithm 1 to convergence (or prm.max_iters)."""
    lib = _load()
    p = _d(points, 3)
    a = _d(weights).ravel()
    n0 = _d(n0, 3)
    out = np.zeros_like(n0)
    it = ctypes.c_int()
    ti = np.zeros(max(prm.max_iters, 1))
    ts = np.zeros(max(prm.max_iters, 1))
    conv = lib.dwgo_orient(len(p), _ptr(p), _ptr(a), _ptr(n0), ctypes.byref(prm), _ptr(out),
                           ctypes.byref(it), _ptr(ti), _ptr(ts))
    k = it.value
    return dict(normals=out, iters=k, converged=bool(conv), iso=ti[:k].copy(),
                stat=ts[:k].copy())


def morton_order(points):
    """Input indices in Morton order of the root cube (21 bits per axis)."""
    lib = _load()
    p = _d(points, 3)
    out = np.zeros(len(p), dtype=np.int64)
    lib.dwgo_morton_order(len(p), _ptr(p), _ptr(out))
    return out


def tree_gwn(points, normals, weights, queries, kernel=KERNEL_PLAIN, eps=0.0, lam=0.0,
             beta=2.0, bucket=16, grad=True, want_count=False, want_bound=False, delta=None):
    """Barnes-Hut w (and grad w) at queries (Sec. 5.2); optional per-query
    evaluation counts and first-order error bounds.  delta: per-point radii
    of the modified kernel (Sec. 5.2; eps unused then), which also widen the
    opening radius to r + max delta."""
    lib = _load()
    p = _d(points, 3)
    nn = _d(normals, 3)
    a = _d(weights).ravel()
    q = _d(queries, 3)
    dl = None if delta is None else _d(delta).ravel()
    w = np.zeros(len(q))
    g = np.zeros((len(q), 3)) if grad else None
    cnt = np.zeros(len(q)) if want_count else None
    bnd = np.zeros(len(q)) if want_bound else None
    lib.dwgo_tree_gwn(len(p), _ptr(p), _ptr(nn), _ptr(a), len(q), _ptr(q), int(kernel),
                      float(eps), float(lam), float(beta), int(bucket),
                      _ptr(dl) if dl is not None else None, _ptr(w),
                      _ptr(g) if grad else None, _ptr(cnt) if want_count else None,
                      _ptr(bnd) if want_bound else None)
    out = [w]
    if grad:
        out.append(g)
    if want_count:
        out.append(cnt)
    if want_bound:
        out.append(bnd)
    return tuple(out) if len(out) > 1 else w


def tree_gwn_group(points, normals, weights, queries, kernel=KERNEL_PLAIN, eps=0.0, lam=0.0,
                   beta=2.0, bucket=16, group=64, grad=True, want_count=False, delta=None):
    """Barnes-Hut w (and grad w) with the opening test applied to groups of
    `group` consecutive queries (a conservative form of Sec. 5.2's test);
    optional per-query evaluation counts."""
    lib = _load()
    p = _d(points, 3)
    nn = _d(normals, 3)
    a = _d(weights).ravel()
    q = _d(queries, 3)
    w = np.zeros(len(q))
    g = np.zeros((len(q), 3)) if grad else None
    cnt = np.zeros(len(q)) if want_count else None
    dl = None if delta is None else _d(delta).ravel()
    lib.dwgo_tree_gwn_group(len(p), _ptr(p), _ptr(nn), _ptr(a), len(q), _ptr(q), int(kernel),
                            float(eps), float(lam), float(beta), int(bucket), int(group),
                            _ptr(dl) if dl is not None else None,
                            _ptr(w), _ptr(g) if grad else None,
                            _ptr(cnt) if want_count else None)
    out = [w]
    if grad:
        out.append(g)
    if want_count:
        out.append(cnt)
    return tuple(out) if len(out) > 1 else w


def kernel_derivative_norms(rho, lam=0.0):
    """Operator norms of the second and third derivative tensors of the
    potential whose negative directional derivative is the term of Eq. 2/3
    (lam = 0) or Eq. 5 (lam > 0), at distance rho.

    With G(rho) = exp(-s rho) / rho, s = sqrt(lam), a source's term is
    t(q) = -<m, grad G(p - q)>: grad G(x) = -F(rho) x / rho^3 with
    F = exp(-s rho)(1 + s rho), the factor of Eq. 5 (F = 1 for lam = 0), and
    grad_q t = Hess G(p - q) m.  For a radial function with derivatives
    G1, G2, G3 (first to third) the Hessian has eigenvalues G2 (radial) and
    G1 / rho (tangential, twice); the third-derivative tensor is
    a xh xh xh + b (delta_ij xh_k + delta_ik xh_j + delta_jk xh_i), xh the unit
    direction, with b = (G2 - G1 / rho) / rho and a = G3 - 3 G2 / rho +
    3 G1 / rho^2.  As a symmetric trilinear form its norm is the largest
    |T(u, u, u)| over unit u, i.e. the maximum over c = xh.u in [0, 1] of
    |a c^3 + 3 b c|: at c = 1 (|G3|) or at c^2 = -b / a.  Here, with
    u = s rho and e = exp(-u):
      G2 = e (2 + 2u + u^2) / rho^3,  G1 / rho = -e (1 + u) / rho^3,
      G3 = -e (6 + 6u + 3u^2 + u^3) / rho^4,
      b = e (3 + 3u + u^2) / rho^4,   a = -e (15 + 15u + 6u^2 + u^3) / rho^4.
    Both norms decrease with rho.  Softening (the regulariser of Sec. 3, read
    as rho^2 = |x|^2 + eps^2) makes the potential the restriction of the 4D
    radial function G(|(x, eps)|) to a hyperplane, so the same norms at
    rho = sqrt(|x|^2 + eps^2) bound it.
    Returns (hessian_norm, third_norm) as arrays."""
    rho = np.asarray(rho, np.float64)
    s = math.sqrt(max(lam, 0.0))
    u = s * rho
    e = np.exp(-u)
    g2 = e * (2 + 2 * u + u * u) / rho ** 3
    g1r = e * (1 + u) / rho ** 3                  # |G1| / rho
    g3 = e * (6 + 6 * u + 3 * u * u + u ** 3) / rho ** 4
    b = e * (3 + 3 * u + u * u) / rho ** 4
    a = -e * (15 + 15 * u + 6 * u * u + u ** 3) / rho ** 4
    c2 = np.clip(-b / a, 0.0, 1.0)
    inner = np.abs(np.sqrt(c2) * (a * c2 + 3 * b))
    return np.maximum(g2, g1r), np.maximum(g3, inner)


def far_field_bound(mass, r, d, lam=0.0, eps=0.0):
    """First-order remainder bound of the Barnes-Hut far field (Sec. 5.2,
    "Octree Traversal"): a node whose sources p_j lie within r of the point c
    where its dipole sum M = sum m_j is placed, at distance d > r from the
    query, is replaced by one term at c.  By the mean-value theorem on each
    source's term the error is at most
      |dw|      <= (mass / 4 pi) r H(rho0),
      |d grad|  <= (mass / 4 pi) r T(rho0),
    with mass = sum_j a_j |n_j| (so sum |m_j| = mass / 4 pi), H and T the
    norms of kernel_derivative_norms at the nearest distance any segment
    [c, p_j] comes to the query, rho0 = sqrt((d - r)^2 + eps^2).  For
    lam = 0 and eps = 0 these are A r / (2 pi (d - r)^3) and
    3 A r / (2 pi (d - r)^4).  The bound needs no property of c beyond
    |p_j - c| <= r.  Returns (w_bound, grad_bound); infinite where d <= r."""
    mass = np.asarray(mass, np.float64)
    r = np.asarray(r, np.float64)
    d = np.asarray(d, np.float64)
    gap = d - r
    ok = gap > 0
    rho0 = np.sqrt(np.where(ok, gap, 1.0) ** 2 + eps * eps)
    H, T = kernel_derivative_norms(rho0, lam)
    k = mass * r / (4 * np.pi)
    return (np.where(ok, k * H, np.inf), np.where(ok, k * T, np.inf))


# ----------------------------------------------------------------------------
# Initial normals (Sec. 5.1, "Normal Initialization")
# ----------------------------------------------------------------------------
PCA_K = 10


def pca_normals(points, k=PCA_K):
    """PCA initialisation: for each point, the eigenvector of the smallest
    eigenvalue of the covariance of its k nearest input points (the point
    itself included; brute force in FP64, ties by the smaller index), taken
    on the offsets from the point.  PCA gives a line; the direction chosen
    points away from the bounding-box centre c (n . (p - c) > 0, the side of
    the Gauss map, which is centred the same way), and where that product is
    zero the one with n_z > 0 (n_y > 0 where n_z = 0, then n_x > 0).

    Returns (normals (n, 3) float64, gap (n,) float64): gap is the relative
    eigen-gap (lambda_2 - lambda_1) / lambda_3 that bounds how well the
    eigenvector is determined.  Rows whose covariance is zero are NaN with
    gap 0 (the library keeps its random normal there)."""
    p = _d(points, 3)
    kk = min(int(k), len(p))
    idx = knn(p, p, kk)
    d = p[idx] - p[:, None, :]
    e = d - d.mean(axis=1, keepdims=True)
    C = np.einsum("nki,nkj->nij", e, e) / kk
    lam, V = np.linalg.eigh(C)
    n = V[:, :, 0].copy()
    c = 0.5 * (p.min(axis=0) + p.max(axis=0))
    side = np.sum(n * (p - c), axis=1)
    axis_rule = (n[:, 2] < 0) | ((n[:, 2] == 0) & ((n[:, 1] < 0) | ((n[:, 1] == 0) & (n[:, 0] < 0))))
    flip = np.where(side != 0.0, side < 0.0, axis_rule)
    n[flip] *= -1.0
    zero = ~np.any(C != 0.0, axis=(1, 2))
    n[zero] = np.nan
    with np.errstate(divide="ignore", invalid="ignore"):
        gap = np.where(lam[:, 2] > 0, (lam[:, 1] - lam[:, 0]) / lam[:, 2], 0.0)
    return n, gap


def gauss_map_normals(points):
    """Gauss-map initialisation: n_i = (p_i - c) / |p_i - c| in FP64, c the
    centre of the bounding box of the (float32) points.  Rows at c are NaN."""
    p = _d(points, 3)
    c = 0.5 * (p.min(axis=0) + p.max(axis=0))
    d = p - c
    l = np.sqrt(np.sum(d * d, axis=1))
    with np.errstate(divide="ignore", invalid="ignore"):
        n = d / l[:, None]
    n[l == 0] = np.nan
    return n


# ----------------------------------------------------------------------------
# Area weights a_i (Sec. 5.1, "Computing Area Weights")
# ----------------------------------------------------------------------------
VORONOI_M = 15


def _clip_halfplane(poly, a, b):
    """Convex polygon (list of 2D points, counter-clockwise) intersected with
    the half-plane a . x <= b."""
    out = []
    k = len(poly)
    for t in range(k):
        P, Q = poly[t], poly[(t + 1) % k]
        fp, fq = a @ P - b, a @ Q - b
        if fp <= 0:
            out.append(P)
        if (fp < 0 < fq) or (fq < 0 < fp):
            out.append(P + (fp / (fp - fq)) * (Q - P))
    return out


def _disk_polygon_area(poly, R):
    """Area of (convex polygon containing the origin) intersected with the
    disk of radius R about the origin: per edge, the triangle (0, A, B) cut by
    the circle, its inside part as triangles and its outside parts as circular
    sectors."""
    def cross(u, v):
        return u[0] * v[1] - u[1] * v[0]

    def sector(u, v):
        return 0.5 * R * R * math.atan2(cross(u, v), u @ v)

    total = 0.0
    k = len(poly)
    for t in range(k):
        A, B = poly[t], poly[(t + 1) % k]
        D = B - A
        a, b, c = D @ D, A @ D, A @ A - R * R
        disc = b * b - a * c
        if a == 0.0:
            continue
        if disc <= 0.0:
            total += sector(A, B)
            continue
        s = math.sqrt(disc)
        t1, t2 = (-b - s) / a, (-b + s) / a
        s1, s2 = min(max(t1, 0.0), 1.0), min(max(t2, 0.0), 1.0)
        P1, P2 = A + s1 * D, A + s2 * D
        total += sector(A, P1) + 0.5 * cross(P1, P2) + sector(P2, B)
    return total


def voronoi_weights(points, m=VORONOI_M):
    """Local-Voronoi area weights, the paper's approximation of geodesic
    Voronoi areas.  For each point p_i:
      1. its m nearest other points (brute force in FP64, ties by the smaller
         index; p_i itself is left out by index, coincident copies stay);
      2. the tangent plane at p_i: normal = smallest-eigenvalue eigenvector of
         the covariance of p_i and those neighbours;
      3. the neighbours' offsets projected onto the plane (any orthonormal
         basis: the area does not depend on it);
      4. the 2D Voronoi cell of the origin among the projected seeds (seeds
         that project onto the origin impose nothing), cut to the disk of
         radius R_i = half the largest projected neighbour distance, which
         bounds the cells of points on the hull of their neighbourhood;
      5. a_i = its area.
    A neighbourhood with no extent (zero area) takes the mean of the positive
    areas, or 1 (the paper's default weight) when there are none.  Returns
    float64 (n,)."""
    p = _d(points, 3)
    n = len(p)
    kk = min(int(m) + 1, n)
    idx = knn(p, p, kk)
    out = np.zeros(n)
    for i in range(n):
        nb = [j for j in idx[i] if j != i][: kk - 1]
        d = p[nb] - p[i]
        X = np.vstack([np.zeros(3), d])
        X = X - X.mean(axis=0)
        C = X.T @ X / len(X)
        if not np.any(C != 0.0):
            continue
        nrm = np.linalg.eigh(C)[1][:, 0]
        ax = np.zeros(3)
        ax[int(np.argmin(np.abs(nrm)))] = 1.0
        e1 = np.cross(nrm, ax)
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(nrm, e1)
        q = np.stack([d @ e1, d @ e2], axis=1)
        r = np.sqrt(np.sum(q * q, axis=1))
        R = 0.5 * r.max()
        if not R > 0.0:
            continue
        poly = [np.array(v, float) for v in ((-R, -R), (R, -R), (R, R), (-R, R))]
        for j in range(len(q)):
            if r[j] > 0.0:
                poly = _clip_halfplane(poly, q[j], 0.5 * r[j] * r[j])
        out[i] = _disk_polygon_area(poly, R) if len(poly) >= 3 else 0.0
    good = out > 0.0
    if not good.all():
        # none positive (one point, or copies of one): the default a_i = 1
        out[~good] = out[good].mean() if good.any() else 1.0
    return out


# ----------------------------------------------------------------------------
# Clamp radii of the modified Poisson kernel (Sec. 5.2, "Poisson Kernels")
# ----------------------------------------------------------------------------
def clamp_radii(points, k=10, vmin=0.0015, vmax=0.015):
    """delta_i = mean distance from p_i to those of its k nearest other points
    (ties by the smaller index) whose distance lies in [vmin, vmax]; if none
    does, the mean of all k distances clamped to [vmin, vmax].  Distances in
    FP64 from the float32 points; vmin and vmax as float32 values."""
    p = _d(points, 3)
    n = len(p)
    kk = min(int(k) + 1, n)
    idx = knn(p, p, kk)
    lo, hi = float(np.float32(vmin)), float(np.float32(vmax))
    out = np.zeros(n)
    for i in range(n):
        nb = [j for j in idx[i] if j != i][: kk - 1]
        if not nb:
            out[i] = lo
            continue
        d = np.sqrt(np.sum((p[nb] - p[i]) ** 2, axis=1))
        sel = d[(d >= lo) & (d <= hi)]
        out[i] = sel.mean() if len(sel) else min(max(d.mean(), lo), hi)
    return out
