"""Grid decomposition over ranks: the task decomposition of Section 2.3.1 (Fig. 5).

The unit of work is the brick (a batch of grid points, Section 2.3.2).  Bricks are dealt to
ranks as contiguous slabs along the first lattice vector, with slab boundaries placed so that
every rank gets about the same cost (Section 2.3.1 gives each process a near-equal share of
the grid work; cost per brick from the library's per-brick atom-image counts, so the
slabs adapt to vacuum and to dense regions instead of cutting the cell into equal widths).
Each rank restricts its handle to its bricks (gint_select_bricks) and computes partial
results; then
  * H (the sparse block buffer) is summed onto the rank that owns each block: contiguous
    ranges of atom rows with about equal numbers of values (a stand-in for the 2-D
    block-cyclic layout the eigensolver wants, Section 2.4), one reduce per owner;
  * F, the stress and E are summed over all ranks (one all-reduce each);
  * rho needs no exchange: each rank owns the grid points of its slab.
The collectives are torch.distributed calls (NCCL on GPUs, gloo on CPU ranks), on tensors in
place.  This module holds partition and reduction logic only: every number comes from the
kernels (or, in tests, from the oracle).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def bricks_per_axis(grid: Sequence[int], brick: Sequence[int]) -> Tuple[int, int, int]:
    """nb_i = ceil(n_i / B_i): the brick grid (brick b = (b0 nb1 + b1) nb2 + b2)."""
    return tuple(int(-(-int(n) // int(b))) for n, b in zip(grid, brick))


def brick_costs(loads: np.ndarray) -> np.ndarray:
    """Relative cost of each brick from its atom-image count n: n (n + 1), the pair count that
    the per-brick contraction scales with (empty bricks cost nothing here)."""
    n = np.asarray(loads, dtype=np.float64)
    return n * (n + 1.0)


def partition_slabs(costs: np.ndarray, nb: Sequence[int], n_ranks: int) -> List[np.ndarray]:
    """Brick ids of each rank: contiguous slabs of whole b0-planes with about equal summed cost.

    Plane boundaries are put where the running cost crosses k / n_ranks of the total (at least
    one plane per rank while planes last).  Returns n_ranks sorted int64 arrays covering every
    brick exactly once (a rank may get none when there are fewer planes than ranks)."""
    nb0, nb1, nb2 = (int(x) for x in nb)
    costs = np.asarray(costs, dtype=np.float64).reshape(nb0, nb1 * nb2)
    plane = costs.sum(1)
    total = float(plane.sum())
    cum = np.concatenate([[0.0], np.cumsum(plane)])
    cuts = [0]
    for k in range(1, n_ranks):
        target = total * k / n_ranks
        c = int(np.searchsorted(cum, target, side="left"))
        # the plane whose running cost is closest to the target
        if c > 0 and abs(cum[c - 1] - target) <= abs(cum[min(c, nb0)] - target):
            c -= 1
        c = max(c, cuts[-1] + 1) if cuts[-1] < nb0 else nb0
        cuts.append(min(c, nb0))
    cuts.append(nb0)
    per_plane = nb1 * nb2
    return [np.arange(cuts[r] * per_plane, cuts[r + 1] * per_plane, dtype=np.int64) for r in range(n_ranks)]


def brick_point_mask(ids: np.ndarray, grid: Sequence[int], brick: Sequence[int]) -> np.ndarray:
    """Boolean grid array [n1][n2][n3]: the points covered by the bricks `ids`."""
    n = np.array(grid, dtype=np.int64)
    B = np.array(brick, dtype=np.int64)
    nb = bricks_per_axis(grid, brick)
    mask = np.zeros(tuple(n), dtype=bool)
    ids = np.asarray(ids, dtype=np.int64)
    b0 = ids // (nb[1] * nb[2])
    b1 = (ids // nb[2]) % nb[1]
    b2 = ids % nb[2]
    for x, y, z in zip(b0, b1, b2):
        mask[x * B[0]:(x + 1) * B[0], y * B[1]:(y + 1) * B[1], z * B[2]:(z + 1) * B[2]] = True
    return mask


def row_owner_segments(blocks: np.ndarray, offsets: np.ndarray, n_atoms: int, n_ranks: int) -> List[Tuple[int, int]]:
    """[v0, v1) value ranges of the block buffer owned by each rank: contiguous atom-row ranges
    (blocks are sorted by their row atom I) with about equal numbers of values."""
    blocks = np.asarray(blocks, dtype=np.int64)
    offsets = np.asarray(offsets, dtype=np.int64)
    # first block of every atom row, then the value offset where each row starts
    first = np.searchsorted(blocks[:, 0], np.arange(n_atoms + 1), side="left")
    row_val = offsets[first]
    total = int(offsets[-1])
    segs, start_atom = [], 0
    for r in range(n_ranks):
        if r == n_ranks - 1:
            end_atom = n_atoms
        else:
            end_atom = int(np.searchsorted(row_val, total * (r + 1) / n_ranks, side="left"))
            end_atom = min(max(end_atom, start_atom), n_atoms)
        segs.append((int(row_val[start_atom]), int(row_val[end_atom])))
        start_atom = end_atom
    return segs


def reduce_to_owners(H, segments: Sequence[Tuple[int, int]], group=None):
    """Sum each owner's segment of the partial block buffers onto that owner (one reduce per
    owner rank, in place).  After the call rank r's H[v0:v1] holds the full values of its
    segment; other values of H are partial sums and must not be used."""
    import torch.distributed as dist
    for r, (v0, v1) in enumerate(segments):
        if v1 > v0:
            dist.reduce(H[v0:v1], dst=r, op=dist.ReduceOp.SUM, group=group)
    return H


def allreduce_sum(*tensors, group=None):
    """In-place sums over the ranks (forces, stress, energy)."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


def sharded_step(g, rank: int, n_ranks: int, V, D, group=None):
    """One decomposed H^V + rho + force/stress step on this rank's slab of handle `g`.

    Returns (H, (v0, v1), rho, F, sigma, E): H holds the full values of this rank's owner
    segment [v0, v1); rho is written on this rank's bricks only; F, sigma and E are the
    totals over all ranks.  Every rank must call it (collectives inside when n_ranks > 1;
    a single rank needs no process group)."""
    loads = g.brick_loads()
    nb = bricks_per_axis(g.grid, g.info()["brick"])
    ids = partition_slabs(brick_costs(loads), nb, n_ranks)[rank]
    g.select_bricks(ids)
    H = g.vlocal(V)
    rho = g.rho(D)
    F, sigma, _, E = g.force_stress(V, D)
    blocks, offsets = g.pattern()
    segs = row_owner_segments(blocks, offsets, g.n_atoms, n_ranks)
    if n_ranks > 1:
        reduce_to_owners(H, segs, group)
        allreduce_sum(F, sigma, E, group=group)
    return H, segs[rank], rho, F, sigma, E
