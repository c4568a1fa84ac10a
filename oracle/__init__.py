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
                ("max_iters", ctypes.c_int), ("tol", ctypes.c_double), ("rule", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.dwgo_gwn.argtypes = [i64, P, P, P, i64, P, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, P, P]
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
                                          P, P]
            lib.dwgo_tree_gwn_group.argtypes = [i64, P, P, P, i64, P, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_int, ctypes.c_int, P,
                                                P, P]
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
        grad=True):
    """w and grad w at queries (Eq. 2/3; Eq. 5 when kernel is screened)."""
    lib = _load()
    p = _d(points, 3)
    nn = _d(normals, 3)
    a = _d(weights).ravel()
    q = _d(queries, 3)
    w = np.zeros(len(q))
    g = np.zeros((len(q), 3)) if grad else None
    lib.dwgo_gwn(len(p), _ptr(p), _ptr(nn), _ptr(a), len(q), _ptr(q), int(kernel),
                 float(eps), float(lam), _ptr(w), _ptr(g) if grad else None)
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
           max_iters=30, tol=0.1, rule=0):
    return _Params(int(kernel), float(eps), float(lam), int(depth), int(knn), int(mode),
                   int(max_iters), float(tol), int(rule))


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
             beta=2.0, bucket=16, grad=True, want_count=False, want_bound=False):
    """Barnes-Hut w (and grad w) at queries (Sec. 5.2); optional per-query
    evaluation counts and first-order error bounds."""
    lib = _load()
    p = _d(points, 3)
    nn = _d(normals, 3)
    a = _d(weights).ravel()
    q = _d(queries, 3)
    w = np.zeros(len(q))
    g = np.zeros((len(q), 3)) if grad else None
    cnt = np.zeros(len(q)) if want_count else None
    bnd = np.zeros(len(q)) if want_bound else None
    lib.dwgo_tree_gwn(len(p), _ptr(p), _ptr(nn), _ptr(a), len(q), _ptr(q), int(kernel),
                      float(eps), float(lam), float(beta), int(bucket), _ptr(w),
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
                   beta=2.0, bucket=16, group=64, grad=True, want_count=False):
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
    lib.dwgo_tree_gwn_group(len(p), _ptr(p), _ptr(nn), _ptr(a), len(q), _ptr(q), int(kernel),
                            float(eps), float(lam), float(beta), int(bucket), int(group),
                            _ptr(w), _ptr(g) if grad else None,
                            _ptr(cnt) if want_count else None)
    out = [w]
    if grad:
        out.append(g)
    if want_count:
        out.append(cnt)
    return tuple(out) if len(out) > 1 else w
