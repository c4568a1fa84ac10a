"""The kNN scatter hands a face whose own tree search runs long to a block of
threads (dwg_set_knn_budget).  The k points a face reaches, and so every sum
of the update, must not depend on which of the two finished its search."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _two_steps(dwglib, p, budget, depth=7):
    h = dwglib.dwg_create(p)
    try:
        dwglib.dwg_set_params(h, 1, 0.5 * 2.0 / np.sqrt(len(p)), 10.0, 50, 0.1)
        dwglib.dwg_set_update(h, depth, 10, dwglib.DWG_UPDATE_LEVELSET)
        dwglib.dwg_set_tree(h, dwglib.DWG_PATH_TREE, 0.5)
        dwglib.dwg_set_knn_budget(h, budget)
        dwglib.dwg_set_init(h, dwglib.DWG_INIT_RANDOM, 5)
        deferred = []
        for _ in range(2):
            dwglib.dwg_step(h)
            deferred.append(dwglib.dwg_get_stats(h)["knn_deferred_last"])
        out = np.zeros_like(p)
        dwglib.dwg_get_normals(h, out)
    finally:
        dwglib.dwg_destroy(h)
    return out, deferred


def test_deferred_searches_reach_the_same_points(dwglib):
    """A 40,000-point sphere from random normals: the first level sets cross
    cells far from the points, whose faces have no candidate list.  Budget 0
    hands every such face to a block, -1 none, the default the long ones:
    the normals after two iterations are the same bits."""
    p, _ = synth.sphere(40_000, seed=3)
    alone, d_alone = _two_steps(dwglib, p, -1)
    blocks, d_blocks = _two_steps(dwglib, p, 0)
    default, _ = _two_steps(dwglib, p, 16384)
    assert d_alone == [0, 0]
    assert d_blocks[0] > 0, d_blocks          # the block path ran
    assert np.array_equal(alone, blocks)
    assert np.array_equal(alone, default)


def test_deferred_searches_in_a_batch(dwglib):
    """The batched phases (one launch per phase over all clouds) defer the
    same way: budget 0 and -1 orient every cloud to the same bits."""
    clouds = [synth.sphere(20_000, seed=4)[0], synth.torus(30_000, seed=5)[0],
              synth.sphere(3_000, seed=6)[0]]
    P = np.ascontiguousarray(np.vstack(clouds))
    off = np.cumsum([0] + [len(c) for c in clouds]).astype(np.int64)
    outs = []
    for budget in (-1, 0):
        hb = dwglib.dwg_create_batch(P, off)
        try:
            dwglib.dwg_set_params(hb, 1, 0.0, 10.0, 4, 0.1)
            dwglib.dwg_set_tree(hb, dwglib.DWG_PATH_TREE, 0.5)
            dwglib.dwg_set_knn_budget(hb, budget)
            dwglib.dwg_set_init(hb, dwglib.DWG_INIT_RANDOM, 9)
            out = np.zeros_like(P)
            dwglib.dwg_orient_batch(hb, out, len(clouds))
            outs.append(out)
        finally:
            dwglib.dwg_destroy(hb)
    assert np.array_equal(outs[0], outs[1])


def test_budget_is_checked(dwglib):
    p, _ = synth.sphere(500, seed=1)
    h = dwglib.dwg_create(p)
    try:
        with pytest.raises(dwglib.DWGError) as e:
            dwglib.dwg_set_knn_budget(h, -2)
        assert e.value.code == dwglib.DWG_ERR_INVALID
    finally:
        dwglib.dwg_destroy(h)
