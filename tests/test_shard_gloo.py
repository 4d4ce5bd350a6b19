"""Multi-rank path of the periodic Fourier-block solve on CPU (gloo,
world sizes 2 and 3, ranges of unequal and zero length): each rank solves its contiguous Fourier-index range, the
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


def _problem(which):
    from tests import _cases
    if which == "3d":
        return _cases.periodic_3d_small(L=(3, 2, 4), n0=4, R=8)
    if which == "chain5":
        return _cases.periodic_chain_small(L=5, n0=6, n_perp=12, m0=4, R=8)
    return _cases.periodic_chain_small(L=2, n0=6, n_perp=12, m0=4, R=8)      # "chain2"


def _worker(rank, world, port, out, which="3d"):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import blocks, dense
    p = _problem(which)
    H, S = dense.build(p)
    _, per = blocks.periodic_eigs(p, H, S)

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


@pytest.mark.parametrize("world,which", [(2, "3d"), (3, "chain5"), (3, "chain2")])
def test_gloo_merge_equals_unsharded(tmp_path, world, which):
    """Two ranks on a 3D lattice; three ranks on 5 blocks (ranges of 2, 2, 1)
    and on 2 blocks (one rank with an empty range)."""
    out = str(tmp_path / "merged.npy")
    port = 29500 + (os.getpid() * 7 + 31 * world + len(which)) % 2000
    mp.spawn(_worker, args=(world, port, out, which), nprocs=world, join=True)
    merged = np.load(out)
    from oracle import blocks, dense
    p = _problem(which)
    H, S = dense.build(p)
    ev, per = blocks.periodic_eigs(p, H, S)
    bl = np.concatenate([[j] * p.m0 for j in range(p.ncell)])
    flat = np.concatenate(list(per))
    o = np.lexsort((bl, flat))
    assert np.array_equal(merged[0], flat[o]) and np.array_equal(merged[1], bl[o].astype(float))
    assert np.array_equal(np.sort(merged[0]), ev)
