"""The extracted level set (dwg_extract_level_set): the CUDA library's
triangles against the FP64 oracle's level-set faces on the same octree.

The oracle gives one face per cut tetrahedron (vector area toward
increasing w, centroid); the library splits a four-point face into two
triangles on the same edge points.  Sums that do not depend on the split
must agree: the total area, and the enclosed volume by the divergence
theorem (sum of c . A / 3 over planar faces equals sum of v0 . (v1 x v2) / 6
over their triangles).  Tolerance: relative 2e-5, the float32 rounding of
the edge points (w itself differs by ~1e-7 between FP32 and FP64)."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _tri_sums(T):
    v0, v1, v2 = T[:, 0:3].astype(np.float64), T[:, 3:6].astype(np.float64), T[:, 6:9].astype(np.float64)
    cr = np.cross(v1 - v0, v2 - v0)
    area = 0.5 * np.linalg.norm(cr, axis=1).sum()
    vol = np.einsum("ij,ij->i", v0, np.cross(v1, v2)).sum() / 6.0
    return area, vol, cr, (v0 + v1 + v2) / 3.0


@pytest.mark.parametrize("n,depth,kernel,lam", [(4000, 6, 0, 0.0), (6000, 7, 1, 10.0)])
def test_level_set_matches_oracle_faces(dwglib, oracle_mod, n, depth, kernel, lam):
    p, nt = synth.sphere(n, seed=3)
    a = np.full(n, 4 * math.pi / n, np.float32)
    eps = synth.default_eps(4 * math.pi, n)
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_weights(h, a)
        dwglib.dwg_set_params(h, kernel, eps, lam, 30, 0.1)
        dwglib.dwg_set_update(h, depth, 10, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_ALLPAIRS, 0.5)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, nt.astype(np.float32))
        cnt, iso = dwglib.dwg_extract_level_set(h)
        T = np.full((cnt, 9), np.nan, np.float32)
        cnt2, iso2 = dwglib.dwg_extract_level_set(h, T)
    finally:
        dwglib.dwg_destroy(h)
    assert cnt == cnt2 and iso == iso2 and not np.isnan(T).any()
    L = oracle_mod.octree_leaves(p, depth)
    K = oracle_mod.corner_keys(L, depth)
    cb = oracle_mod.cube(p, depth)
    X = oracle_mod.corner_positions(K, depth, cb)
    wc = oracle_mod.gwn(p, nt, a, X, kernel=kernel, eps=eps, lam=lam, grad=False)
    wp = oracle_mod.gwn(p, nt, a, p, kernel=kernel, eps=eps, lam=lam, grad=False)
    iso_o = wp.mean()
    F = oracle_mod.faces(L, depth, cb, K, wc, iso_o)
    assert abs(iso - iso_o) <= 1e-6 * max(1.0, abs(iso_o))
    assert len(F) <= cnt <= 2 * len(F)
    area, vol, cr, cen = _tri_sums(T)
    area_o = np.linalg.norm(F[:, :3], axis=1).sum()
    vol_o = -np.einsum("ij,ij->i", F[:, 3:6], F[:, :3]).sum() / 3.0  # faces point inward
    assert abs(area / area_o - 1) <= 2e-5, (area, area_o)
    assert abs(vol / vol_o - 1) <= 2e-5, (vol, vol_o)
    # wound outward: the normals point away from the sphere's centre
    out = np.einsum("ij,ij->i", cr, cen) > 0
    assert out.mean() >= 0.999


def test_level_set_count_only_and_small_cap(dwglib):
    p, nt = synth.sphere(3000, seed=4)
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_update(h, 6, 10, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, nt.astype(np.float32))
        cnt, _ = dwglib.dwg_extract_level_set(h)
        assert cnt > 100
        T = np.full((cnt - 1, 9), 7.0, np.float32)
        cnt2, _ = dwglib.dwg_extract_level_set(h, T)
        assert cnt2 == cnt and np.all(T == 7.0)
    finally:
        dwglib.dwg_destroy(h)


def test_level_set_after_orientation_on_both_paths(dwglib, torch):
    """Orient a torus from its analytic normals on the Barnes-Hut path in the
    DIRECT update mode (no octree during the iterations: the extraction
    builds it) and on the exact path in the level-set mode, extract both
    surfaces into device memory: total areas within 1 % of each other, the
    enclosed volume the torus's, 2 pi^2 R r^2, within 5 %."""
    n = 100_000
    p, nt = synth.torus(n, seed=5, noise=0.001)
    area_t = 4 * math.pi ** 2 * 0.3
    a = np.full(n, area_t / n, np.float32)
    eps = synth.default_eps(area_t, n)
    res = {}
    for path in (dwglib.DWG_PATH_TREE, dwglib.DWG_PATH_ALLPAIRS):
        h = dwglib.dwg_create(p)
        try:
            dwglib.dwg_set_weights(h, a)
            dwglib.dwg_set_params(h, 0, eps, 0.0, 40, 0.1)
            mode = (dwglib.DWG_UPDATE_DIRECT if path == dwglib.DWG_PATH_TREE
                    else dwglib.DWG_UPDATE_LEVELSET)
            dwglib.dwg_set_update(h, 7, 10, mode)
            dwglib.dwg_set_tree(h, path, 0.4)
            dwglib.dwg_set_convergence(h, dwglib.DWG_CONV_MEAN)
            dwglib.dwg_set_init(h, dwglib.DWG_INIT_GIVEN, 0, nt.astype(np.float32))
            dwglib.dwg_orient(h, np.zeros((n, 3), np.float32))
            cnt, _ = dwglib.dwg_extract_level_set(h)
            T = torch.empty((cnt, 9), dtype=torch.float32, device="cuda")
            dwglib.dwg_extract_level_set(h, T)
            res[path] = _tri_sums(T.cpu().numpy())
        finally:
            dwglib.dwg_destroy(h)
    at, vt = res[dwglib.DWG_PATH_TREE][:2]
    ae, ve = res[dwglib.DWG_PATH_ALLPAIRS][:2]
    assert abs(at / ae - 1) <= 0.01, (at, ae)
    vol_true = 2 * math.pi ** 2 * 1.0 * 0.3 ** 2
    assert abs(abs(ve) / vol_true - 1) <= 0.05, (ve, vol_true)
    assert abs(abs(vt) / vol_true - 1) <= 0.05, (vt, vol_true)


@pytest.fixture
def torch():
    return pytest.importorskip("torch")
