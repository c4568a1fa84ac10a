"""Batched orientation (one handle, many clouds): every cloud's result must be
bit-identical to orienting that cloud alone with the same parameters."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _clouds():
    specs = [("sphere", 1500, 0), ("torus", 4000, 1), ("sphere", 700, 2), ("torus", 9000, 3),
             ("sphere", 33, 4)]
    pts, offs = [], [0]
    for kind, n, s in specs:
        p = synth.sphere(n, seed=s)[0] if kind == "sphere" else synth.torus(n, seed=s)[0]
        pts.append(p)
        offs.append(offs[-1] + n)
    return np.ascontiguousarray(np.vstack(pts)), np.array(offs, np.int64)


@pytest.mark.parametrize("path,init,knn,phases", [(1, 0, 10, 4), (2, 0, 10, 4), (1, 3, 10, 4),
                                                  (2, 4, 10, 4), (2, 0, 10, 1), (1, 0, 10, 3),
                                                  (2, 0, 10, 0), (2, 0, 12, 4)])
def test_batch_equals_singles(dwglib, path, init, knn, phases):
    """init: DWG_INIT_RANDOM (0), DWG_INIT_PCA (3), DWG_INIT_GAUSS (4).  With
    k = 10 every phase of an iteration is one launch over the clouds of a
    lane (phases = lanes); with another k, or phases = 0, the clouds' chains
    run as graph branches."""
    P, off = _clouds()
    nc = len(off) - 1
    hb = dwglib.dwg_create_batch(P, off)
    try:
        dwglib.dwg_set_batch_mode(hb, phases)
        if knn != 10:   # one depth for every cloud then (the singles take it too)
            dwglib.dwg_set_update(hb, 6, knn, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_tree(hb, path, 0.5)
        dwglib.dwg_set_init(hb, init, 11)
        out = np.zeros_like(P)
        rc, iters = dwglib.dwg_orient_batch(hb, out, nc)
        st = dwglib.dwg_get_stats(hb)
    finally:
        dwglib.dwg_destroy(hb)
    assert st["n_points"] == len(P)
    for c in range(nc):
        p = np.ascontiguousarray(P[off[c]:off[c + 1]])
        n = len(p)
        h = dwglib.dwg_create(p)
        try:
            depth = min(10, max(5, int(round(0.5 * np.log2(max(n, 2)))))) if knn == 10 else 6
            dwglib.dwg_set_update(h, depth, knn, dwglib.DWG_UPDATE_LEVELSET)
            dwglib.dwg_set_tree(h, path, 0.5)
            dwglib.dwg_set_init(h, init, 11 + c)
            o = np.zeros_like(p)
            rc1, it1 = dwglib.dwg_orient(h, o)
        finally:
            dwglib.dwg_destroy(h)
        assert it1 == iters[c], (c, it1, iters[c])
        assert np.array_equal(o, out[off[c]:off[c + 1]]), c


def test_batch_orients_every_cloud(dwglib):
    P, off = _clouds()
    nts = []
    for kind, n, s in [("sphere", 1500, 0), ("torus", 4000, 1), ("sphere", 700, 2),
                       ("torus", 9000, 3), ("sphere", 33, 4)]:
        nts.append(synth.sphere(n, seed=s)[1] if kind == "sphere" else synth.torus(n, seed=s)[1])
    hb = dwglib.dwg_create_batch(P, off)
    try:
        dwglib.dwg_set_params(hb, 1, 0.01, 10.0, 40, 0.1)   # screened, one eps for all
        out = np.zeros_like(P)
        rc, iters = dwglib.dwg_orient_batch(hb, out, len(off) - 1)
    finally:
        dwglib.dwg_destroy(hb)
    for c in range(4):  # the 33-point cloud is too sparse to judge
        o = out[off[c]:off[c + 1]]
        d = np.sum(o * nts[c], axis=1)
        s = 1.0 if d.sum() >= 0 else -1.0
        assert np.mean(s * d > 0) >= 0.99, (c, np.mean(s * d > 0), iters)


def test_batch_handle_rejects_single_calls(dwglib):
    P, off = _clouds()
    hb = dwglib.dwg_create_batch(P, off)
    try:
        with pytest.raises(dwglib.DWGError) as e:
            dwglib.dwg_orient(hb, np.zeros_like(P))
        assert e.value.code == dwglib.DWG_ERR_STATE
    finally:
        dwglib.dwg_destroy(hb)
    with pytest.raises(dwglib.DWGError):
        dwglib.dwg_create_batch(P, np.array([0, 10, 10, len(P)], np.int64))


def test_batch_autotune_per_cloud_then_orient(dwglib):
    """The tuner on a batch handle tunes every cloud (relative budget) and
    the batch still orients every cloud."""
    P, off = _clouds()
    nts = []
    for kind, n, s in [("sphere", 1500, 0), ("torus", 4000, 1), ("sphere", 700, 2),
                       ("torus", 9000, 3), ("sphere", 33, 4)]:
        nts.append(synth.sphere(n, seed=s)[1] if kind == "sphere" else synth.torus(n, seed=s)[1])
    hb = dwglib.dwg_create_batch(P, off)
    try:
        dwglib.dwg_set_params(hb, 1, 0.0, 10.0, 40, 0.1)
        dwglib.dwg_set_tree(hb, dwglib.DWG_PATH_TREE, 0.5)
        t = dwglib.dwg_autotune(hb, dwglib.DWG_TUNE_TREE | dwglib.DWG_TUNE_RELATIVE, 0.025, None)
        assert t["path"] == dwglib.DWG_PATH_TREE and t["tree_leaf"] in (16, 32, 64, 128)
        assert dwglib.dwg_get_tuning(hb)["theta"] == t["theta"]
        out = np.zeros_like(P)
        dwglib.dwg_orient_batch(hb, out, len(off) - 1)
    finally:
        dwglib.dwg_destroy(hb)
    for c in range(4):
        o = out[off[c]:off[c + 1]]
        d = np.sum(o * nts[c], axis=1)
        s = 1.0 if d.sum() >= 0 else -1.0
        assert np.mean(s * d > 0) >= 0.99, (c, np.mean(s * d > 0))


def _kernels_per_iteration(dwglib, clouds, path, lanes):
    P = np.ascontiguousarray(np.vstack(clouds))
    off = np.cumsum([0] + [len(c) for c in clouds]).astype(np.int64)
    hb = dwglib.dwg_create_batch(P, off)
    try:
        dwglib.dwg_set_batch_mode(hb, lanes)
        dwglib.dwg_set_params(hb, 1, 0.0, 10.0, 2, 0.1)
        dwglib.dwg_set_tree(hb, path, 0.5)
        dwglib.dwg_orient_batch(hb, np.zeros_like(P), len(clouds))
        return dwglib.dwg_get_stats(hb)["kernels_per_iteration"]
    finally:
        dwglib.dwg_destroy(hb)


@pytest.mark.parametrize("path", [1, 2])
def test_launches_per_iteration_do_not_grow_with_the_clouds(dwglib, path):
    """Every phase of a batched iteration is one launch over a lane's clouds:
    the iteration graph has as many kernel launches for 16 clouds as for 4
    (the tree levels of the moments follow each lane's largest cloud; the
    large cloud has a lane of its own in both batches)."""
    big = synth.torus(20000, seed=7)[0]
    small = [synth.sphere(2000, seed=20 + i)[0] for i in range(15)]
    k1 = _kernels_per_iteration(dwglib, [big] + small, path, 1)
    assert k1 < 4 * 15     # a few dozen phases, not a chain per cloud
    k4 = _kernels_per_iteration(dwglib, [big] + small[:3], path, 4)
    k16 = _kernels_per_iteration(dwglib, [big] + small, path, 4)
    assert k4 == k16, (k4, k16)
    assert k16 <= 4 * k1, (k1, k16)
