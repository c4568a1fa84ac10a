"""PCA and Gauss-map initial normals (Sec. 5.1, "Normal Initialization"):
the CUDA library against the FP64 oracle, through the C ABI.

Tolerances: the Gauss map is the same FP64 expression on both sides rounded
to float32, so the two agree to one float32 ulp.  The PCA line is an FP64
eigenvector (Jacobi rotations on the GPU, LAPACK in the oracle): where the
relative eigen-gap is at least 1e-3 the two lines differ by far less than
the float32 rounding of the result (1 - |cos| <= 1e-10 is asserted after
renormalising the float32 output in FP64); the direction rule
(n . (p - c) > 0) is compared where that product is above 1e-6 |p - c|.  Neighbourhoods
whose 10th and 11th nearest points are equally far in float32 but not in
FP64 may differ; at most 0.1 % of the points are allowed to."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _init(dwglib, p, mode, seed=5):
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_init(h, mode, seed)
        out = np.zeros((len(p), 3), np.float32)
        dwglib.dwg_get_normals(h, out)
    finally:
        dwglib.dwg_destroy(h)
    return out


def _clouds():
    tor, _ = synth.torus(20000, seed=1, noise=0.002)
    ell, _ = synth.ellipsoid_points(8000, (0.9, 0.5, 0.3), seed=2, stream=3)
    box = synth.uniform_box(5000, [-1] * 3, [1] * 3, seed=3)
    return {"torus": tor, "ellipsoid": np.ascontiguousarray(ell, np.float32), "box": box}


@pytest.mark.parametrize("kind", ["torus", "ellipsoid", "box"])
def test_pca_matches_oracle(dwglib, oracle_mod, kind):
    p = _clouds()[kind]
    out = _init(dwglib, p, dwglib.DWG_INIT_PCA)
    ref, gap = oracle_mod.pca_normals(p)
    assert np.allclose(np.linalg.norm(out, axis=1), 1, atol=1e-6)
    ok = gap >= 1e-3
    assert ok.mean() > 0.5
    o = out.astype(np.float64)
    o /= np.linalg.norm(o, axis=1, keepdims=True)  # float32 rounding moves |out| by ~1e-7
    cos = np.abs(np.sum(o * ref, axis=1))
    bad_line = ok & (1 - cos > 1e-10)
    p64 = p.astype(np.float64)
    rel = p64 - 0.5 * (p64.min(axis=0) + p64.max(axis=0))
    side_ref = np.sum(ref * rel, axis=1)
    sided = ok & (np.abs(side_ref) > 1e-6 * np.linalg.norm(rel, axis=1))
    bad_sign = sided & (np.sign(np.sum(o * rel, axis=1)) != np.sign(side_ref))
    assert (bad_line | bad_sign).mean() <= 1e-3, ((bad_line).sum(), bad_sign.sum())


def test_pca_degenerate_neighbourhoods_keep_the_random_normal(dwglib, oracle_mod):
    """Twelve coincident points: zero covariance, the random draw stays."""
    rest = synth.uniform_box(500, [-1] * 3, [1] * 3, seed=6)
    p = np.r_[np.full((12, 3), 0.25, np.float32), rest]
    out = _init(dwglib, p, dwglib.DWG_INIT_PCA, seed=77)
    ref, _ = oracle_mod.pca_normals(p)
    assert np.all(np.isnan(ref[:12])) and not np.any(np.isnan(ref[12:]))
    rnd = synth.random_unit_normals(len(p), seed=77)
    np.testing.assert_allclose(out[:12], rnd[:12], atol=2e-6)
    cos = np.abs(np.sum(out[12:].astype(np.float64) * ref[12:], axis=1))
    assert np.mean(1 - cos <= 1e-6) > 0.99


@pytest.mark.parametrize("shift", [0.0, 3.5])
def test_gauss_map_matches_oracle(dwglib, oracle_mod, shift):
    p, _ = synth.torus(30000, seed=9, noise=0.003)
    p = (p + np.float32(shift)).astype(np.float32)
    out = _init(dwglib, p, dwglib.DWG_INIT_GAUSS)
    ref = oracle_mod.gauss_map_normals(p)
    assert not np.any(np.isnan(ref))
    assert np.max(np.abs(out - ref)) <= 2.0 ** -24


def test_gauss_map_point_at_the_centre_keeps_the_random_normal(dwglib, oracle_mod):
    e = np.eye(3, dtype=np.float32)
    p = np.r_[e, -e, np.zeros((1, 3), np.float32), 0.5 * e].astype(np.float32)
    out = _init(dwglib, p, dwglib.DWG_INIT_GAUSS, seed=31)
    ref = oracle_mod.gauss_map_normals(p)
    assert np.all(np.isnan(ref[6]))
    np.testing.assert_allclose(out[6], synth.random_unit_normals(len(p), seed=31)[6], atol=2e-6)
    keep = np.arange(len(p)) != 6
    np.testing.assert_array_equal(out[keep], ref[keep].astype(np.float32))


def _orient_mean_rule(dwglib, p, mode, depth=7):
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_update(h, depth, 10, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_convergence(h, dwglib.DWG_CONV_MEAN)
        dwglib.dwg_set_init(h, mode, 1)
        out = np.zeros_like(p)
        rc, it = dwglib.dwg_orient(h, out)
    finally:
        dwglib.dwg_destroy(h)
    return rc, it, out


@pytest.mark.parametrize("mode", [4, 3])
def test_star_shaped_cloud_starts_oriented(dwglib, mode):
    """Gauss map (4) and PCA (3) on a sphere off the origin: the start is
    already consistent (both take the side away from the box centre), so the
    mean-change rule is met within a few iterations, normals outward."""
    p, nt = synth.sphere(20000, seed=12, center=(0.3, -0.1, 0.2))
    rc, it, out = _orient_mean_rule(dwglib, p, mode)
    assert rc == dwglib.DWG_OK
    d = np.sum(out * nt, axis=1)
    # every normal outward; the level-set normals scatter by a few degrees
    assert np.all(d > 0) and np.median(d) > 0.99 and np.mean(d > 0.9) >= 0.99
    assert it <= 6, it


def test_pca_init_orients_an_ellipsoid_faster_than_random(dwglib):
    p, nt = synth.ellipsoid_points(20000, (1.0, 0.6, 0.4), seed=13, stream=4)
    p = np.ascontiguousarray(p, np.float32)
    res = {}
    for mode in (dwglib.DWG_INIT_RANDOM, dwglib.DWG_INIT_PCA):
        h = dwglib.dwg_create(p)
        try:
            dwglib.dwg_set_update(h, 7, 10, dwglib.DWG_UPDATE_LEVELSET)
            dwglib.dwg_set_convergence(h, dwglib.DWG_CONV_MEAN)
            dwglib.dwg_set_init(h, mode, 1)
            out = np.zeros_like(p)
            rc, it = dwglib.dwg_orient(h, out)
        finally:
            dwglib.dwg_destroy(h)
        d = np.sum(out * nt, axis=1)
        res[mode] = (rc, it, float(np.mean(np.sign(d.sum()) * d > 0)))
    assert res[dwglib.DWG_INIT_PCA][0] == dwglib.DWG_OK, res
    assert res[dwglib.DWG_INIT_PCA][2] >= 0.999, res
    assert res[dwglib.DWG_INIT_PCA][1] < res[dwglib.DWG_INIT_RANDOM][1], res
