"""One far-field exchange build sharded over several GPUs by occupied columns.

The paper's implementation distributes batches of occupied orbitals over MPI
ranks (Sec. III B).  Here each rank g owns a contiguous block I_g of occupied
columns i and computes K^ff_{r,i} for i in I_g: steps (a)-(d) on every
occupied pair (i, j) that touches I_g, step (e) on the block's columns
(occk_set_column_block).  Nothing is exchanged until the end, when the K
blocks are gathered (all_gather over NCCL on GPUs, gloo on CPU) and the
energy is formed from the gathered K with the reduction order of the
unsharded call (occk_exchange_energy), so K and E equal the one-GPU result
bit for bit.

The blocks balance an estimate of each rank's work: the stored pairs i <= j
that touch the block (steps (a)-(d)) plus the block's columns times all j
(step (e)).  Marshalling and collectives only; every step of the build runs
in the library's kernels.
"""
from __future__ import annotations


def pairs_touching(nocc: int, c0: int, c1: int) -> int:
    """Stored pairs i <= j with i or j in [c0, c1)."""
    if c1 <= c0:
        return 0
    with_i = sum(nocc - i for i in range(c0, c1))        # i in the block, j >= i
    return with_i + c0 * (c1 - c0)                       # i < c0, j in the block


def block_cost(nocc: int, c0: int, c1: int) -> int:
    return pairs_touching(nocc, c0, c1) + (c1 - c0) * nocc


def column_blocks(nocc: int, world: int) -> list:
    """Contiguous blocks [c0, c1) of the occupied columns, one per rank,
    covering 0..nocc-1 in order, with balanced block_cost (the largest block
    cost is minimised by bisection on a common bound).  Ranks beyond nocc get
    empty blocks."""
    if world <= 1:
        return [(0, nocc)]

    def split(bound):
        out, c0 = [], 0
        while c0 < nocc and len(out) < world:
            c1 = c0 + 1
            while c1 < nocc and block_cost(nocc, c0, c1 + 1) <= bound:
                c1 += 1
            out.append((c0, c1))
            c0 = c1
        return out, c0 >= nocc

    lo, hi = 0, block_cost(nocc, 0, nocc)
    best = None
    while lo <= hi:
        mid = (lo + hi) // 2
        blocks, ok = split(mid)
        if ok:
            best, hi = blocks, mid - 1
        else:
            lo = mid + 1
    blocks = list(best)
    while len(blocks) < world:
        blocks.append((nocc, nocc))
    return blocks


def gather_columns(Kt, blocks, rank, group=None):
    """All-gather of column blocks.  Kt is the transposed (row = column i)
    view of a column-major K, [nocc, nao] contiguous: rank `rank` holds valid
    rows blocks[rank]; on return every rank holds all rows.  Works on CUDA
    tensors (NCCL) and CPU tensors (gloo)."""
    import torch
    import torch.distributed as dist
    world = len(blocks)
    if world <= 1:
        return Kt
    bmax = max(c1 - c0 for c0, c1 in blocks)
    c0, c1 = blocks[rank]
    send = torch.zeros((bmax, Kt.shape[1]), dtype=Kt.dtype, device=Kt.device)
    if c1 > c0:
        send[:c1 - c0].copy_(Kt[c0:c1])
    parts = [torch.empty_like(send) for _ in range(world)]
    dist.all_gather(parts, send, group=group)
    for g, (a, b) in enumerate(blocks):
        if g != rank and b > a:
            Kt[a:b].copy_(parts[g][:b - a])
    return Kt


def farfield_K_sharded(ctx, tree, C, blocks, rank, prec="fp64", K=None, Ex=None, group=None, stream=None):
    """One far-field build shared by the ranks of `group`: this rank computes
    its column block, the blocks are gathered, and E is formed from the whole
    K.  C: [nao, nocc] float64 CUDA (column-major view); K, Ex as in
    occk.farfield_K (K must be column-major).  Returns (K, Ex)."""
    import torch
    from . import occk
    nao, nocc = C.shape
    if K is None:
        K = occk.empty_fortran(nao, nocc, torch.float64, C.device)
    if Ex is None:
        Ex = torch.empty((), dtype=torch.float64, device=C.device)
    c0, c1 = blocks[rank]
    if c1 > c0:
        ctx.set_column_block(c0, c1)
        try:
            occk.farfield_K(ctx, tree, C, prec=prec, K=K, Ex=Ex, stream=stream)
        finally:
            ctx.set_column_block(0, 0)
    gather_columns(K.t(), blocks, rank, group)
    occk.exchange_energy(ctx, C, K, Ex, stream=stream)
    return K, Ex
