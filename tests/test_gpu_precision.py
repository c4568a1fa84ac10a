"""Error of each output of the exact all-pairs evaluator against the FP64
oracle, with and without the two-sum fold of the tile sums
(dwg_set_compensation), on the 2,000-point sphere and the 100,000-point
noisy torus, plain kernel (Eq. 2/3) and screened kernel (Eq. 5, lambda 10 and
100), w and grad w at every input point.

Each case prints one JSON line (run pytest with -s to see them): max, 99th
percentile and median of |dw|, of |dg| (Euclidean) and of |dg| / |g_64|.
The assertions are the stated tolerances of the compensated path (|dw| <=
1e-5; |dg|_inf <= 1e-5 max(1, |g|) + 16 u S_g) and that the fold does not
lose accuracy against plain FP32 addition of the same tile sums."""
import json

import numpy as np
import pytest

import synth
from test_gpu_parity import s_g, U32

pytestmark = pytest.mark.gpu


def _stats(x):
    return {"max": float(np.max(x)), "p99": float(np.percentile(x, 99)),
            "median": float(np.median(x))}


def _workloads():
    S = synth.workload_sphere2k()
    T = synth.workload_torus100k()
    return [("sphere-2k", S), ("torus-100k", T)]


@pytest.mark.parametrize("name", ["sphere-2k", "torus-100k"])
@pytest.mark.parametrize("kernel,lam", [(0, 0.0), (1, 10.0), (1, 100.0)])
def test_precision_against_fp64(dwglib, oracle_mod, name, kernel, lam):
    W = dict(_workloads())[name]
    p, a, eps = W["points"], W["weights"], W["eps"]
    n = len(p)
    nrm = synth.random_unit_normals(n, seed=1).astype(np.float32)
    w64, g64 = oracle_mod.gwn(p, nrm, a, p, kernel=kernel, eps=eps, lam=lam)
    gn = np.linalg.norm(g64, axis=1)
    h = dwglib.dwg_create(p)
    res = {}
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_ALLPAIRS, 0.5)
        dwglib.dwg_set_normals(h, nrm)
        for comp in (1, 0):
            dwglib.dwg_set_compensation(h, comp)
            w = np.zeros(n, np.float32)
            g = np.zeros((n, 3), np.float32)
            dwglib.dwg_eval_gwn(h, p, w, g)
            dw = np.abs(w.astype(np.float64) - w64)
            dg = np.linalg.norm(g.astype(np.float64) - g64, axis=1)
            res[comp] = (w, g, dw, dg)
            print(json.dumps({"precision": name, "kernel": "plain" if kernel == 0 else
                              f"screened lambda={lam:g}", "two_sum_fold": bool(comp),
                              "w_abs": _stats(dw), "grad_abs": _stats(dg),
                              "grad_rel": _stats(dg / np.maximum(gn, 1e-30)),
                              "w_scale_median": float(np.median(np.abs(w64))),
                              "grad_scale_median": float(np.median(gn))}))
    finally:
        dwglib.dwg_destroy(h)
    w, g, dw, dg = res[1]
    assert dw.max() <= 1e-5
    sel = np.arange(0, n, 1 if n <= 10000 else 10)
    tol = 1e-5 * np.maximum(1.0, gn[sel]) + 16 * U32 * s_g(p, nrm, a, p[sel], eps)
    assert np.all(np.abs(g[sel] - g64[sel]).max(axis=1) <= tol)
    # the fold never loses accuracy in aggregate (allow rounding noise)
    assert np.mean(res[1][2]) <= np.mean(res[0][2]) * 1.05 + 1e-12
    assert np.mean(res[1][3]) <= np.mean(res[0][3]) * 1.05 + 1e-12
