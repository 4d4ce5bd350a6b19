"""Multi-rank path of the periodic Fourier-block solve on CPU (gloo,
world size 2): each rank solves its contiguous Fourier-index range, the
sorted parts are gathered and merged, and the result equals the unsharded
spectrum (values and block map).  Per-rank compute is the oracle's block
route here (no GPU); on GPUs it is fock_circulant_eig_range."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1702_00339_gb300 import shard


def test_j_range_partitions():
    for n in (1, 5, 24, 1000):
        for w in (1, 2, 3, 8):
            rs = [shard.j_range(n, r, w) for r in range(w)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(w - 1))
            assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1


def test_merge_orders_by_value_then_block():
    ev, blk = shard.merge([([1.0, 2.0, np.inf], [0, 0, 0]), ([1.0, 1.5], [3, 3])])
    assert ev.tolist() == [1.0, 1.0, 1.5, 2.0, np.inf] and blk.tolist() == [0, 3, 3, 0, 0]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import blocks, dense
    from tests import _cases
    p = _cases.periodic_3d_small(L=(3, 2, 4), n0=4, R=8)
    H, S = dense.build(p)
    _, per, _ = blocks.periodic_eigs(p, H, S)

    def solve_range(j0, j1):
        ev = np.concatenate([per[j] for j in range(j0, j1)]) if j1 > j0 else np.zeros(0)
        bl = np.concatenate([[j] * p.m0 for j in range(j0, j1)]).astype(np.int32) if j1 > j0 else np.zeros(0, np.int32)
        o = np.lexsort((bl, ev))
        return ev[o], bl[o]

    ev, blk = shard.solve_sharded(solve_range, p.ncell)
    if rank == 0:
        np.save(out, np.stack([ev, blk.astype(float)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_merge_equals_unsharded(tmp_path):
    out = str(tmp_path / "merged.npy")
    port = 29500 + os.getpid() % 1000
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    merged = np.load(out)
    from oracle import blocks, dense
    from tests import _cases
    p = _cases.periodic_3d_small(L=(3, 2, 4), n0=4, R=8)
    H, S = dense.build(p)
    ev, per, _ = blocks.periodic_eigs(p, H, S)
    bl = np.concatenate([[j] * p.m0 for j in range(p.ncell)])
    flat = np.concatenate(list(per))
    o = np.lexsort((bl, flat))
    assert np.array_equal(merged[0], flat[o]) and np.array_equal(merged[1], bl[o].astype(float))
    assert np.array_equal(np.sort(merged[0]), ev)
