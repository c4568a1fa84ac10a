"""Sharding independent clouds over ranks: the assignment covers every cloud
once and balances the work; with two gloo ranks on the CPU, each rank's
results for its clouds assemble into the single-process layout."""
import os
import socket

import numpy as np
import pytest

import synth
from paper_2405_13839_gb300 import shard


def test_assignment_covers_every_cloud_once_and_balances():
    u = synth.uniform(0, 700, 64)
    sizes = np.round(np.exp(np.log(5e3) + u * (np.log(5e5) - np.log(5e3)))).astype(np.int64)
    for world in (1, 2, 3, 8):
        parts = shard.assign(sizes, world)
        flat = sorted(c for p in parts for c in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(shard.cloud_cost(int(sizes[c])) for c in p) for p in parts]
        # greedy LPT: no rank exceeds the mean by more than the largest cloud
        assert max(loads) <= sum(loads) / world + max(shard.cloud_cost(int(s)) for s in sizes)
    assert shard.assign([10, 20], 1) == [[0, 1]]


def test_sub_batch_keeps_each_cloud():
    P = np.arange(30, dtype=np.float32).reshape(10, 3)
    off = np.array([0, 2, 5, 10])
    pts, so = shard.sub_batch(P, off, [2, 0])
    np.testing.assert_array_equal(so, [0, 5, 7])
    np.testing.assert_array_equal(pts[:5], P[5:10])
    np.testing.assert_array_equal(pts[5:], P[0:2])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, sizes, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        off = np.zeros(len(sizes) + 1, dtype=np.int64)
        off[1:] = np.cumsum(sizes)
        mine = shard.assign(sizes, world)[rank]
        # a stand-in per-cloud result: each cloud's normals from its own seed
        local = np.vstack([synth.random_unit_normals(int(sizes[c]), seed=c) for c in mine]
                          ).astype(np.float32) if mine else np.zeros((0, 3), np.float32)
        full = shard.gather_normals(local, mine, off, int(off[-1]))
        q.put((rank, mine, full))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_assemble_the_single_process_layout():
    mp = pytest.importorskip("torch.multiprocessing")
    sizes = np.array([300, 1200, 50, 700, 900, 10], dtype=np.int64)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref = np.vstack([synth.random_unit_normals(int(n), seed=c) for c, n in enumerate(sizes)]
                    ).astype(np.float32)
    owned = sorted(c for _, mine, _ in res for c in mine)
    assert owned == list(range(len(sizes)))
    for _, mine, full in res:
        np.testing.assert_array_equal(full, ref)
