"""ctypes binding of libdwg.so: the C ABI of include/dwg.h, one Python function
per C function with the same name.

The binding only marshals arguments: arrays may be numpy arrays (host) or
torch tensors (host or CUDA); their data pointers are passed straight to the
library, which tells host from device memory itself.  Every computation runs
in the library's CUDA kernels.  If libdwg.so is missing, importing this
module raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

DWG_OK = 0
DWG_NOT_CONVERGED = 1
DWG_ERR_INVALID = -1
DWG_ERR_CUDA = -2
DWG_ERR_OOM = -3
DWG_ERR_NONFINITE = -4
DWG_ERR_TIMEOUT = -5
DWG_ERR_STATE = -6
DWG_KERNEL_PLAIN = 0
DWG_KERNEL_SCREENED = 1
DWG_UPDATE_LEVELSET = 0
DWG_UPDATE_DIRECT = 1
DWG_INIT_RANDOM = 0
DWG_INIT_GIVEN = 1
DWG_INIT_LEARNED = 2
DWG_INIT_PCA = 3
DWG_INIT_GAUSS = 4
DWG_REG_SOFTEN = 0
DWG_REG_CLAMP = 1
MLP_PARAMS = 12675
DWG_CONV_TOP1 = 0
DWG_CONV_MEAN = 1
DWG_MAX_BATCH_LANES = 16
DWG_PATH_AUTO = 0
DWG_PATH_ALLPAIRS = 1
DWG_PATH_TREE = 2

_NAMES = {v: k for k, v in dict(
    DWG_ERR_INVALID=-1, DWG_ERR_CUDA=-2, DWG_ERR_OOM=-3, DWG_ERR_NONFINITE=-4,
    DWG_ERR_TIMEOUT=-5, DWG_ERR_STATE=-6).items()}


class DWGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class dwg_stats(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("n_corners", ctypes.c_int64), ("iters", ctypes.c_int),
                ("converged", ctypes.c_int), ("faces_last", ctypes.c_int64),
                ("iso_last", ctypes.c_double), ("stat_last", ctypes.c_double),
                ("interactions", ctypes.c_double), ("ms_orient", ctypes.c_double),
                ("interactions_eval", ctypes.c_double),
                ("interactions_points_step", ctypes.c_double),
                ("interactions_corners_step", ctypes.c_double),
                ("kernels_per_iteration", ctypes.c_int),
                ("knn_deferred_last", ctypes.c_int)]


class dwg_tuning(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("points_pairs", ctypes.c_int),
                ("points_threads", ctypes.c_int), ("corners_pairs", ctypes.c_int),
                ("corners_threads", ctypes.c_int), ("tree_leaf", ctypes.c_int),
                ("theta", ctypes.c_float), ("tree_group", ctypes.c_int),
                ("knn_lists", ctypes.c_int), ("w_err", ctypes.c_double),
                ("ms_points", ctypes.c_double), ("ms_corners", ctypes.c_double),
                ("from_cache", ctypes.c_int)]


DWG_TUNE_SHAPES = 1
DWG_TUNE_TREE = 2
DWG_TUNE_RELATIVE = 4


def lib_path() -> str:
    return _build.LIB


def _load() -> ctypes.CDLL:
    if not os.path.exists(_build.LIB):
        raise ImportError(
            f"libdwg.so not built ({_build.LIB}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I = ctypes.c_int
    F = ctypes.c_float
    H = ctypes.c_void_p
    sig = {
        "dwg_create": ([P, I64, ctypes.POINTER(H)], I),
        "dwg_destroy": ([H], None),
        "dwg_last_error": ([H], ctypes.c_char_p),
        "dwg_set_stream": ([H, P], I),
        "dwg_set_params": ([H, I, F, F, I, F], I),
        "dwg_set_update": ([H, I, I, I], I),
        "dwg_set_convergence": ([H, I], I),
        "dwg_set_compensation": ([H, I], I),
        "dwg_set_batch_mode": ([H, I], I),
        "dwg_set_knn_budget": ([H, I], I),
        "dwg_set_weights": ([H, P], I),
        "dwg_voronoi_weights": ([H, I, P], I),
        "dwg_selfcheck_wait": ([H, I], I),
        "dwg_extract_level_set": ([H, P, I64, ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_double)],
                                  I),
        "dwg_measure_fp32_peaks": ([I, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)], I),
        "dwg_set_regularization": ([H, I, I, F, F, P], I),
        "dwg_set_tree": ([H, I, F], I),
        "dwg_create_batch": ([P, P, I, ctypes.POINTER(H)], I),
        "dwg_orient_batch": ([H, P, P], I),
        "dwg_set_init": ([H, I, ctypes.c_uint64, P], I),
        "dwg_orient": ([H, P, ctypes.POINTER(I)], I),
        "dwg_step": ([H, P, P, P, ctypes.POINTER(ctypes.c_double),
                      ctypes.POINTER(ctypes.c_double)], I),
        "dwg_get_normals": ([H, P], I),
        "dwg_set_normals": ([H, P], I),
        "dwg_eval_gwn": ([H, P, I64, P, P], I),
        "dwg_get_stats": ([H, ctypes.POINTER(dwg_stats)], I),
        "dwg_get_trace": ([H, P, P, P, P, I, ctypes.POINTER(I)], I),
        "dwg_get_leaves": ([H, P, I64, ctypes.POINTER(I64)], I),
        "dwg_get_corners": ([H, P, I64, ctypes.POINTER(I64)], I),
        "dwg_get_tree": ([H, I64, ctypes.POINTER(I64), ctypes.POINTER(I), P, P, P, P, P], I),
        "dwg_knn": ([H, P, I64, I, P], I),
        "dwg_profile_step": ([H, P, I, ctypes.POINTER(I)], I),
        "dwg_eval_w_noalloc": ([P, P, P, I64, P, I64, I, F, F, P, P], I),
        "dwg_mlp_features": ([H, P], I),
        "dwg_mlp_forward": ([P, P, I64, P, P], I),
        "dwg_mlp_grad": ([P, P, P, I64, P, ctypes.POINTER(ctypes.c_double), P], I),
        "dwg_mlp_adam": ([P, P, P, P, I, F, P], I),
        "dwg_autotune": ([H, I, ctypes.c_double, ctypes.c_char_p, ctypes.POINTER(dwg_tuning)], I),
        "dwg_get_tuning": ([H, ctypes.POINTER(dwg_tuning)], I),
        "dwg_set_tuning": ([H, ctypes.POINTER(dwg_tuning)], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


# ----------------------------------------------------------------------------
# marshalling helpers
# ----------------------------------------------------------------------------
def _ptr(a):
    """Data pointer of a contiguous numpy array or torch tensor (or None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check_f32(a, cols=None, name="array"):
    dt = getattr(a, "dtype", None)
    ok = dt == np.float32 or str(dt) == "torch.float32"
    if not ok:
        raise TypeError(f"{name} must be float32, got {dt}")
    if cols is not None and (a.ndim != 2 or a.shape[1] != cols):
        raise ValueError(f"{name} must have shape (n, {cols})")


def _raise(h, rc):
    if rc < 0:
        msg = _lib.dwg_last_error(h)
        raise DWGError(rc, msg.decode() if msg else "")
    return rc


def _like(ref, shape, dtype=np.float32):
    """Output buffer on the same side (host/device) as ref."""
    if isinstance(ref, np.ndarray):
        return np.empty(shape, dtype=dtype)
    import torch
    tdt = {np.float32: torch.float32, np.int64: torch.int64}[dtype]
    return torch.empty(shape, dtype=tdt, device=ref.device)


# ----------------------------------------------------------------------------
# the ABI, one function per C entry point
# ----------------------------------------------------------------------------
def dwg_create(points):
    """Handle for a float32 (n, 3) cloud (numpy, or torch on host or GPU)."""
    _check_f32(points, 3, "points")
    h = ctypes.c_void_p()
    rc = _lib.dwg_create(_ptr(points), int(points.shape[0]), ctypes.byref(h))
    _raise(None, rc)
    return h


def dwg_create_batch(points, offsets):
    """Batch handle for concatenated clouds; offsets int64 (n_clouds + 1)."""
    _check_f32(points, 3, "points")
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    h = ctypes.c_void_p()
    rc = _lib.dwg_create_batch(_ptr(points), off.ctypes.data, len(off) - 1, ctypes.byref(h))
    _raise(None, rc)
    return h


def dwg_orient_batch(h, normals_out, n_clouds):
    """Orients every cloud; returns (rc, iterations per cloud)."""
    it = np.zeros(n_clouds, dtype=np.int32)
    rc = _lib.dwg_orient_batch(h, _ptr(normals_out), it.ctypes.data)
    _raise(h, rc)
    return rc, it


def dwg_destroy(h):
    _lib.dwg_destroy(h)


def dwg_last_error(h=None):
    m = _lib.dwg_last_error(h)
    return m.decode() if m else ""


def dwg_set_stream(h, stream):
    """stream: a cudaStream_t as int (e.g. torch.cuda.current_stream().cuda_stream) or None."""
    return _raise(h, _lib.dwg_set_stream(h, stream))


def dwg_set_params(h, kernel, eps, screening, max_iters, tol):
    return _raise(h, _lib.dwg_set_params(h, int(kernel), float(eps), float(screening),
                                         int(max_iters), float(tol)))


def dwg_set_convergence(h, rule):
    return _raise(h, _lib.dwg_set_convergence(h, int(rule)))


def dwg_set_batch_mode(h, lanes):
    """Batch handles: lanes >= 1 batched phases (one launch per phase over a
    lane's clouds, lanes concurrent; default 1), 0 one graph branch per
    cloud."""
    return _raise(h, _lib.dwg_set_batch_mode(h, int(lanes)))


def dwg_set_knn_budget(h, budget):
    """Node visits and distances after which a face's kNN search is handed
    to a block (default 16384); -1: never.  The results do not change."""
    return _raise(h, _lib.dwg_set_knn_budget(h, int(budget)))


def dwg_set_compensation(h, on):
    """1: two-sum fold of the all-pairs tile sums (default); 0: plain FP32."""
    return _raise(h, _lib.dwg_set_compensation(h, int(on)))


def dwg_set_update(h, depth, knn=10, mode=DWG_UPDATE_LEVELSET):
    return _raise(h, _lib.dwg_set_update(h, int(depth), int(knn), int(mode)))


def dwg_set_tree(h, path, theta=0.5):
    return _raise(h, _lib.dwg_set_tree(h, int(path), float(theta)))


def dwg_set_weights(h, a):
    _check_f32(a, None, "weights")
    return _raise(h, _lib.dwg_set_weights(h, _ptr(a)))


def dwg_set_regularization(h, mode, k=10, vmin=0.0, vmax=0.0, delta_out=None):
    """DWG_REG_SOFTEN, or DWG_REG_CLAMP (the modified kernel of Sec. 5.2 with
    radii from the k nearest points filtered to [vmin, vmax]; 0, 0 = the
    paper's values times the largest bounding-box extent).  delta_out
    (float32 (n,), host or device) receives the radii."""
    if delta_out is not None:
        _check_f32(delta_out, None, "delta_out")
    return _raise(h, _lib.dwg_set_regularization(h, int(mode), int(k), float(vmin), float(vmax),
                                                 _ptr(delta_out)))


def dwg_measure_fp32_peaks(device=0):
    """(packed-FMA FP32 lane operations per second, MUFU rsqrt per second,
    MUFU ex2 per second)."""
    f = ctypes.c_double()
    r = ctypes.c_double()
    e = ctypes.c_double()
    _raise(None, _lib.dwg_measure_fp32_peaks(int(device), ctypes.byref(f), ctypes.byref(r),
                                             ctypes.byref(e)))
    return f.value, r.value, e.value


def dwg_extract_level_set(h, tri_out=None):
    """The level set of the current normals as triangles.  Returns (count,
    iso); with tri_out (float32 (cap, 9), host or device) fills it when
    count <= cap."""
    cnt = ctypes.c_int64()
    iso = ctypes.c_double()
    cap = 0 if tri_out is None else int(tri_out.shape[0])
    if tri_out is not None:
        _check_f32(tri_out, 9, "tri_out")
    _raise(h, _lib.dwg_extract_level_set(h, _ptr(tri_out), cap, ctypes.byref(cnt),
                                         ctypes.byref(iso)))
    return cnt.value, iso.value


def dwg_selfcheck_wait(h, polls=1024):
    """Exercise the device-side wait limit; raises DWGError(DWG_ERR_TIMEOUT)."""
    return _raise(h, _lib.dwg_selfcheck_wait(h, int(polls)))


def dwg_voronoi_weights(h, m=15, a_out=None):
    """Local-Voronoi area weights of the m nearest points, installed as the
    handle's a_i; a_out (float32 (n,), host or device) receives them."""
    if a_out is not None:
        _check_f32(a_out, None, "a_out")
    return _raise(h, _lib.dwg_voronoi_weights(h, int(m), _ptr(a_out)))


def dwg_set_init(h, mode, seed=1, normals=None):
    """normals: (n, 3) initial normals for DWG_INIT_GIVEN, or the flat float32
    network parameters (12,675) for DWG_INIT_LEARNED; None for DWG_INIT_RANDOM,
    DWG_INIT_PCA and DWG_INIT_GAUSS (seed: their random fallback)."""
    if normals is not None:
        _check_f32(normals, 3 if mode == DWG_INIT_GIVEN else None, "normals")
    return _raise(h, _lib.dwg_set_init(h, int(mode), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                       _ptr(normals)))


def dwg_orient(h, normals_out):
    """Runs Algorithm 1; fills normals_out (float32 (n, 3)).  Returns (rc, iters)."""
    it = ctypes.c_int()
    rc = _lib.dwg_orient(h, _ptr(normals_out), ctypes.byref(it))
    _raise(h, rc)
    return rc, it.value


def dwg_step(h, w_out=None, grad_out=None, dtheta_out=None):
    """One iteration.  Returns (iso, stat)."""
    iso = ctypes.c_double()
    st = ctypes.c_double()
    rc = _lib.dwg_step(h, _ptr(w_out), _ptr(grad_out), _ptr(dtheta_out), ctypes.byref(iso),
                       ctypes.byref(st))
    _raise(h, rc)
    return iso.value, st.value


def dwg_get_normals(h, normals_out):
    return _raise(h, _lib.dwg_get_normals(h, _ptr(normals_out)))


def dwg_set_normals(h, normals):
    _check_f32(normals, 3, "normals")
    return _raise(h, _lib.dwg_set_normals(h, _ptr(normals)))


def dwg_eval_gwn(h, queries, w_out, grad_out=None):
    _check_f32(queries, 3, "queries")
    return _raise(h, _lib.dwg_eval_gwn(h, _ptr(queries), int(queries.shape[0]), _ptr(w_out),
                                       _ptr(grad_out)))


def dwg_get_stats(h):
    s = dwg_stats()
    _raise(h, _lib.dwg_get_stats(h, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in dwg_stats._fields_}


def dwg_get_trace(h, cap=100000):
    cnt = ctypes.c_int()
    _raise(h, _lib.dwg_get_trace(h, None, None, None, None, 0, ctypes.byref(cnt)))
    k = cnt.value
    iso = np.zeros(k)
    stat = np.zeros(k)
    dn = np.zeros(k)
    faces = np.zeros(k, dtype=np.int64)
    _raise(h, _lib.dwg_get_trace(h, iso.ctypes.data, stat.ctypes.data, dn.ctypes.data,
                                 faces.ctypes.data, k, ctypes.byref(cnt)))
    return dict(iso=iso, stat=stat, mean_dn=dn, faces=faces)


def dwg_get_leaves(h):
    cnt = ctypes.c_int64()
    _raise(h, _lib.dwg_get_leaves(h, None, 0, ctypes.byref(cnt)))
    out = np.zeros((cnt.value, 5), dtype=np.int64)
    _raise(h, _lib.dwg_get_leaves(h, out.ctypes.data, cnt.value, ctypes.byref(cnt)))
    return out


def dwg_get_corners(h):
    cnt = ctypes.c_int64()
    _raise(h, _lib.dwg_get_corners(h, None, 0, ctypes.byref(cnt)))
    out = np.zeros(cnt.value, dtype=np.int64)
    _raise(h, _lib.dwg_get_corners(h, out.ctypes.data, cnt.value, ctypes.byref(cnt)))
    return out


def dwg_get_tree(h, n):
    """The Barnes-Hut hierarchy as built (dict of numpy arrays: perm, area,
    centre, radius, record; leaf size and node count); n = number of points."""
    nodes = ctypes.c_int64()
    leaf = ctypes.c_int()
    _raise(h, _lib.dwg_get_tree(h, 0, ctypes.byref(nodes), ctypes.byref(leaf), None, None, None,
                                None, None))
    nn = nodes.value
    perm = np.zeros(n, np.int64)
    area = np.zeros(nn)
    centre = np.zeros((nn, 3))
    radius = np.zeros(nn)
    record = np.zeros((nn, 4), np.float32)
    _raise(h, _lib.dwg_get_tree(h, nn, ctypes.byref(nodes), ctypes.byref(leaf), perm.ctypes.data,
                                area.ctypes.data, centre.ctypes.data, radius.ctypes.data,
                                record.ctypes.data))
    return dict(nodes=nn, leaf=leaf.value, perm=perm, area=area, centre=centre, radius=radius,
                record=record)


def dwg_knn(h, queries, k, idx_out):
    _check_f32(queries, 3, "queries")
    return _raise(h, _lib.dwg_knn(h, _ptr(queries), int(queries.shape[0]), int(k),
                                  _ptr(idx_out)))


PROFILE_KERNELS = ["eval_points", "reduce_points", "iso", "eval_corners", "reduce_corners",
                   "mc_faces", "knn_scatter", "normal_update", "select"]


def dwg_profile_step(h):
    """Per-kernel device milliseconds of one iteration (dict by kernel name)."""
    ms = np.zeros(16, dtype=np.float32)
    cnt = ctypes.c_int()
    _raise(h, _lib.dwg_profile_step(h, ms.ctypes.data, 16, ctypes.byref(cnt)))
    return {k: float(ms[i]) for i, k in enumerate(PROFILE_KERNELS[:cnt.value])}


def dwg_eval_w_noalloc(points, normals, weights, queries, w_out, kernel=DWG_KERNEL_PLAIN,
                       eps=1e-3, screening=0.0, stream=None):
    """w at queries without any device allocation (all arrays CUDA tensors of
    one device; the library refuses host memory and other devices' memory)."""
    _check_f32(points, 3, "points")
    _check_f32(normals, 3, "normals")
    _check_f32(queries, 3, "queries")
    _check_f32(w_out, None, "w_out")
    n, m = int(points.shape[0]), int(queries.shape[0])
    if int(normals.shape[0]) != n:
        raise ValueError(f"normals has {int(normals.shape[0])} rows, points has {n}")
    if w_out.ndim != 1 or int(w_out.shape[0]) != m:
        raise ValueError(f"w_out must have shape ({m},), got {tuple(w_out.shape)}")
    arrays = [points, normals, queries, w_out]
    if weights is not None:
        _check_f32(weights, None, "weights")
        if weights.ndim != 1 or int(weights.shape[0]) != n:
            raise ValueError(f"weights must have shape ({n},), got {tuple(weights.shape)}")
        arrays.append(weights)
    devices = {str(getattr(a, "device", "cpu")) for a in arrays}
    if len(devices) != 1:
        raise ValueError(f"all arrays must be on one device, got {sorted(devices)}")
    rc = _lib.dwg_eval_w_noalloc(_ptr(points), _ptr(normals), _ptr(weights),
                                 int(points.shape[0]), _ptr(queries), int(queries.shape[0]),
                                 int(kernel), float(eps), float(screening), _ptr(w_out), stream)
    return _raise(None, rc)


def dwg_mlp_features(h, X_out):
    """Patch feature rows (n, 64) of the handle's points, input order."""
    return _raise(h, _lib.dwg_mlp_features(h, _ptr(X_out)))


def dwg_mlp_forward(params, X, Y, stream=None):
    return _raise(None, _lib.dwg_mlp_forward(_ptr(params), _ptr(X), int(X.shape[0]), _ptr(Y),
                                              stream))


def dwg_mlp_grad(params, X, T, grad, stream=None):
    """Fills grad (12,675) with the gradient of the mean squared error; returns the loss."""
    loss = ctypes.c_double()
    _raise(None, _lib.dwg_mlp_grad(_ptr(params), _ptr(X), _ptr(T), int(X.shape[0]), _ptr(grad),
                                   ctypes.byref(loss), stream))
    return loss.value


def dwg_mlp_adam(params, grad, m, v, step, lr, stream=None):
    return _raise(None, _lib.dwg_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step),
                                          float(lr), stream))


def _tuning_dict(t):
    return {name: getattr(t, name) for name, _ in dwg_tuning._fields_}


def dwg_autotune(h, what=DWG_TUNE_SHAPES | DWG_TUNE_TREE, w_budget=1e-3, cache_path=None):
    """Measure and apply the fastest settings (dict of dwg_tuning's fields)."""
    t = dwg_tuning()
    cp = None if cache_path is None else os.fsencode(cache_path)
    _raise(h, _lib.dwg_autotune(h, int(what), float(w_budget), cp, ctypes.byref(t)))
    return _tuning_dict(t)


def dwg_get_tuning(h):
    t = dwg_tuning()
    _raise(h, _lib.dwg_get_tuning(h, ctypes.byref(t)))
    return _tuning_dict(t)


def dwg_set_tuning(h, **settings):
    """Apply settings; fields not given keep their current values."""
    t = dwg_tuning()
    _raise(h, _lib.dwg_get_tuning(h, ctypes.byref(t)))
    for k, v in settings.items():
        if k not in dict(dwg_tuning._fields_):
            raise KeyError(k)
        setattr(t, k, v)
    return _raise(h, _lib.dwg_set_tuning(h, ctypes.byref(t)))
