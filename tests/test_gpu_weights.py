"""Local-Voronoi area weights (Sec. 5.1, "Computing Area Weights"): the CUDA
library against the FP64 oracle, through the C ABI.

Both sides compute the cell in FP64 from the same float32 points, so the
areas agree to the float32 rounding of the result (relative 1e-6 asserted).
A neighbourhood whose m-th and (m+1)-th nearest points are equally far in
float32 but not in FP64 may differ; at most 0.1 % of the points may."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _weights(dwglib, p, m=15):
    h = dwglib.dwg_create(p)
    try:
        a = np.zeros(len(p), np.float32)
        dwglib.dwg_voronoi_weights(h, m, a)
    finally:
        dwglib.dwg_destroy(h)
    return a


def _uneven_sphere(n, seed):
    """Unit sphere, the lower hemisphere sampled ten times more sparsely."""
    p, nt = synth.sphere(n, seed=seed)
    keep = (p[:, 2] >= 0) | (synth.uniform(seed, 77, n) < 0.1)
    return np.ascontiguousarray(p[keep]), nt[keep]


def _cases():
    tor, _ = synth.torus(6000, seed=2, noise=0.001)
    sph, _ = _uneven_sphere(12000, 3)
    h = 0.0625
    g = np.stack(np.meshgrid(np.arange(20), np.arange(20), indexing="ij"), -1).reshape(-1, 2)
    lat = np.c_[g * h, np.zeros(len(g))].astype(np.float32)
    return {"torus": tor, "uneven-sphere": sph, "lattice": lat}


@pytest.mark.parametrize("kind", ["torus", "uneven-sphere", "lattice"])
@pytest.mark.parametrize("m", [15, 8, 31])
def test_voronoi_weights_match_oracle(dwglib, oracle_mod, kind, m):
    p = _cases()[kind]
    a = _weights(dwglib, p, m)
    ref = oracle_mod.voronoi_weights(p, m)
    assert np.all(a > 0)
    bad = np.abs(a - ref) > 1e-6 * ref
    assert bad.mean() <= 1e-3, (bad.sum(), np.max(np.abs(a / ref - 1)))


def test_lattice_interior_is_exact(dwglib):
    h = 0.0625
    g = np.stack(np.meshgrid(np.arange(16), np.arange(16), indexing="ij"), -1).reshape(-1, 2)
    p = np.c_[g * h, np.zeros(len(g))].astype(np.float32)
    a = _weights(dwglib, p)
    inner = np.all((g >= 3) & (g <= 12), axis=1)
    np.testing.assert_array_equal(a[inner], np.float32(h * h))


def test_weights_are_installed(dwglib):
    """dwg_eval_gwn after dwg_voronoi_weights equals dwg_eval_gwn after
    dwg_set_weights with the same values."""
    p, nt = _uneven_sphere(6000, 4)
    q = synth.uniform_box(500, [-1.5] * 3, [1.5] * 3, seed=5)
    res = []
    for use_set in (False, True):
        h = dwglib.dwg_create(p)
        try:
            a = np.zeros(len(p), np.float32)
            dwglib.dwg_voronoi_weights(h, 15, a)
            if use_set:
                dwglib.dwg_set_weights(h, np.ones(len(p), np.float32))
                dwglib.dwg_set_weights(h, a)
            dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, nt.astype(np.float32))
            dwglib.dwg_get_normals(h, np.zeros_like(p))
            w = np.zeros(len(q), np.float32)
            dwglib.dwg_eval_gwn(h, q, w)
            res.append(w)
        finally:
            dwglib.dwg_destroy(h)
    np.testing.assert_array_equal(res[0], res[1])


def test_voronoi_weights_correct_uneven_sampling(dwglib):
    """Inside an unevenly sampled unit sphere with its analytic normals the
    winding number is 1 only if a_i follows the sampling density: with
    Voronoi weights it is within 5 % (the FP64 oracle gives 3.0 %: tangent-plane
    cells of the sparse half miss some area), with uniform weights it is off
    by far more (0.45)."""
    p, nt = _uneven_sphere(40000, 6)
    n = len(p)
    q = (synth.uniform_box(400, [-0.5] * 3, [0.5] * 3, seed=7)).astype(np.float32)
    out = {}
    for name in ("uniform", "voronoi"):
        h = dwglib.dwg_create(p)
        try:
            if name == "voronoi":
                a = np.zeros(n, np.float32)
                dwglib.dwg_voronoi_weights(h, 15, a)
                assert abs(a.sum() / (4 * math.pi) - 1) < 0.04, a.sum()
            else:
                dwglib.dwg_set_weights(h, np.full(n, 4 * math.pi / n, np.float32))
            dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, nt.astype(np.float32))
            dwglib.dwg_get_normals(h, np.zeros_like(p))
            w = np.zeros(len(q), np.float32)
            dwglib.dwg_eval_gwn(h, q, w)
            out[name] = w
        finally:
            dwglib.dwg_destroy(h)
    assert np.max(np.abs(out["voronoi"] - 1)) < 0.05, np.max(np.abs(out["voronoi"] - 1))
    assert np.max(np.abs(out["uniform"] - 1)) > 0.1


def test_batch_voronoi_weights_equal_singles(dwglib):
    clouds = [synth.sphere(3000, seed=1)[0], synth.torus(5000, seed=2)[0],
              synth.sphere(500, seed=3, center=(2, 0, 0))[0]]
    off = np.cumsum([0] + [len(c) for c in clouds]).astype(np.int64)
    P = np.ascontiguousarray(np.vstack(clouds))
    hb = dwglib.dwg_create_batch(P, off)
    try:
        a = np.zeros(len(P), np.float32)
        dwglib.dwg_voronoi_weights(hb, 15, a)
    finally:
        dwglib.dwg_destroy(hb)
    for c, pc in enumerate(clouds):
        np.testing.assert_array_equal(a[off[c]:off[c + 1]], _weights(dwglib, pc))


def test_voronoi_weights_reject_bad_m(dwglib):
    p = synth.sphere(100, seed=1)[0]
    h = dwglib.dwg_create(p)
    try:
        for m in (2, 32):
            with pytest.raises(dwglib.DWGError) as e:
                dwglib.dwg_voronoi_weights(h, m)
            assert e.value.code == dwglib.DWG_ERR_INVALID
    finally:
        dwglib.dwg_destroy(h)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17])
def test_tiny_clouds(dwglib, oracle_mod, n):
    """Voronoi weights, clamp radii, PCA and Gauss-map starts and the level set
    on clouds of a few points: finite, positive, the oracle's values."""
    p = synth.uniform_box(n, [-1] * 3, [1] * 3, seed=60 + n)
    h = dwglib.dwg_create(p)
    try:
        a = np.zeros(n, np.float32)
        dwglib.dwg_voronoi_weights(h, 15, a)
        d = np.zeros(n, np.float32)
        dwglib.dwg_set_regularization(h, dwglib.DWG_REG_CLAMP, 10, 0.01, 0.5, d)
        dwglib.dwg_set_regularization(h, dwglib.DWG_REG_SOFTEN)
        nrm = np.zeros((n, 3), np.float32)
        for mode in (dwglib.DWG_INIT_PCA, dwglib.DWG_INIT_GAUSS):
            dwglib.dwg_set_init(h, mode, 3)
            dwglib.dwg_get_normals(h, nrm)
            assert np.allclose(np.linalg.norm(nrm, axis=1), 1, atol=1e-5)
        dwglib.dwg_set_update(h, 4, 10, dwglib.DWG_UPDATE_LEVELSET)
        cnt, iso = dwglib.dwg_extract_level_set(h)
        assert cnt >= 0 and np.isfinite(iso)
    finally:
        dwglib.dwg_destroy(h)
    np.testing.assert_allclose(a, oracle_mod.voronoi_weights(p), rtol=1e-6)
    np.testing.assert_allclose(d, oracle_mod.clamp_radii(p, 10, 0.01, 0.5), rtol=1e-6)
