"""Sharding one build over ranks by occupied column blocks (host logic).

The paper distributes occupied orbitals over MPI ranks (Sec. III B); here rank
g owns a contiguous block I_g of occupied columns.  These CPU tests check the
partition and, with two gloo ranks, that gathering the column blocks gives the
one-rank K and E bit for bit.  Each rank's block is computed by the FP64
oracle (a column needs only the pairs (i, j) of its own i, so a column subset
is exact) -- on the GPU the same host logic drives the library's column-block
mode (tests/test_gpu_shard.py).
"""
import os
import socket

import numpy as np
import pytest

from paper_1708_05353_gb300 import shard

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("nocc,world", [(1, 1), (7, 2), (20, 3), (601, 8), (660, 8), (5, 8), (241, 4)])
def test_blocks_cover_in_order_and_balance(nocc, world):
    b = shard.column_blocks(nocc, world)
    assert len(b) == world
    assert b[0][0] == 0 and b[-1][1] == nocc
    for (a0, a1), (b0, b1) in zip(b, b[1:]):
        assert a1 == b0 and a0 <= a1
    costs = [shard.block_cost(nocc, c0, c1) for c0, c1 in b if c1 > c0]
    if nocc >= world:
        assert all(c1 > c0 for c0, c1 in b)
        # a block's cost grows with its width alone, so the largest cost is
        # smallest when no block is wider than ceil(nocc / world)
        assert max(costs) <= shard.block_cost(nocc, 0, -(-nocc // world))


def test_pairs_touching_counts_by_enumeration():
    n = 23
    for c0, c1 in [(0, 5), (3, 9), (20, 23), (0, 23), (11, 12)]:
        brute = sum(1 for i in range(n) for j in range(i, n) if c0 <= i < c1 or c0 <= j < c1)
        assert shard.pairs_touching(n, c0, c1) == brute


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from oracle import fmm
    from oracle import tree as otree
    from paper_1708_05353_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = inputs.small_sp(natom=8, nocc=6, spacing=3.0, depth=3)
        tr = otree.build_tree(s.basis, 3, 8.0)
        blocks = shard.column_blocks(s.nocc, world)
        c0, c1 = blocks[rank]
        Kt = torch.full((s.nocc, s.basis.nao), float("nan"), dtype=torch.float64)   # rows = columns of K
        Kb, _ = fmm.farfield(s, L=2, tree=tr, i_subset=list(range(c0, c1)))
        Kt[c0:c1] = torch.from_numpy(np.ascontiguousarray(Kb.T))
        shard.gather_columns(Kt, blocks, rank)
        K = Kt.numpy().T
        E = -0.5 * float(np.sum(s.C * K))
        out.put((rank, K.copy(), E))
    finally:
        dist.destroy_process_group()


def test_gathered_blocks_equal_one_rank_gloo_world2():
    from oracle import fmm
    from oracle import tree as otree
    from paper_1708_05353_gb300 import inputs
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get() for _ in range(2)]
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    s = inputs.small_sp(natom=8, nocc=6, spacing=3.0, depth=3)
    Kref, Eref = fmm.farfield(s, L=2, tree=otree.build_tree(s.basis, 3, 8.0))
    for rank, K, E in got:
        assert np.array_equal(K, Kref), rank
        assert E == -0.5 * float(np.sum(s.C * Kref))
        assert abs(E - Eref) <= 1e-14 * abs(Eref)
