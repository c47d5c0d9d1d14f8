"""Grid decomposition over ranks (Section 2.3.1, Fig. 5) on CPU: the slab partition by cost,
the owner segments of the block buffer, and a world-size-2 gloo run in which each rank takes
its slab's partial H^V, rho and forces from the oracle's sums restricted to its grid points,
reduces H onto the owners of its atom rows and sums F, the stress and E.  The results equal
the single-rank oracle results to FP64 summation order.  The same partition drives the GPU
library (gint_select_bricks); the GPU side is checked on one GPU in test_gpu_shard.py."""
import os
import socket

import numpy as np
import pytest

import synth
from paper_2409_09399_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_every_brick_once_and_balances_cost():
    nb = (12, 5, 4)
    rng = np.random.default_rng(0)
    # a slab-and-vacuum profile: heavy planes in the middle of a1, empty ones at the ends
    prof = np.exp(-((np.arange(nb[0]) - 6.5) / 2.5) ** 2)
    costs = (prof[:, None, None] * (1.0 + rng.random(nb))).reshape(-1)
    costs[costs < 0.05] = 0.0
    for n_ranks in (1, 2, 3, 4, 12, 15):
        parts = shard.partition_slabs(costs, nb, n_ranks)
        assert len(parts) == n_ranks
        allids = np.concatenate(parts)
        assert np.array_equal(np.sort(allids), np.arange(np.prod(nb)))
        per_plane = nb[1] * nb[2]
        for p in parts:  # contiguous whole planes
            if p.size:
                assert p[0] % per_plane == 0 and p.size % per_plane == 0
                assert np.array_equal(p, np.arange(p[0], p[0] + p.size))
        if 1 < n_ranks <= 4:
            share = np.array([costs[p].sum() for p in parts]) / costs.sum()
            plane_max = (costs.reshape(nb[0], -1).sum(1) / costs.sum()).max()
            # balanced to within one plane of the ideal share
            assert np.all(np.abs(share - 1.0 / n_ranks) <= plane_max + 1e-12), share


def test_owner_segments_tile_the_block_buffer():
    blocks = np.array([[0, 0, 0, 0, 0], [0, 1, 0, 0, 0], [1, 0, 0, 0, 0], [1, 1, 0, 0, 0], [1, 2, 0, 0, 0],
                       [2, 1, 0, 0, 0], [2, 2, 0, 0, 0]])
    nw = np.array([4, 2, 3])
    sizes = nw[blocks[:, 0]] * nw[blocks[:, 1]]
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    for n_ranks in (1, 2, 3, 5):
        segs = shard.row_owner_segments(blocks, offsets, 3, n_ranks)
        assert segs[0][0] == 0 and segs[-1][1] == offsets[-1]
        for (a0, a1), (b0, b1) in zip(segs, segs[1:]):
            assert a1 == b0 and a0 <= a1
        row_starts = set(offsets[np.searchsorted(blocks[:, 0], np.arange(4))].tolist())
        assert all(v0 in row_starts and v1 in row_starts for v0, v1 in segs)  # whole atom rows


def test_brick_point_mask_matches_brick_numbering():
    grid, brick = (7, 5, 9), (3, 2, 4)
    nb = shard.bricks_per_axis(grid, brick)
    assert nb == (3, 3, 3)
    total = np.zeros(grid, dtype=int)
    for b in range(int(np.prod(nb))):
        m = shard.brick_point_mask([b], grid, brick)
        b0, b1, b2 = b // (nb[1] * nb[2]), (b // nb[2]) % nb[1], b % nb[2]
        idx = np.argwhere(m)
        assert idx[:, 0].min() == b0 * brick[0] and idx[:, 1].min() == b1 * brick[1] and idx[:, 2].min() == b2 * brick[2]
        total += m
    assert np.all(total == 1)


def _system():
    return synth.diamond(grid=(18, 18, 18), species=synth.make_species("O", "SZP"))


def _host_loads(s, brick):
    """Atom images near each brick (brick-centre distance below rc + half the brick diagonal)."""
    nb = shard.bricks_per_axis(s.grid, brick)
    B, n = np.array(brick), np.array(s.grid)
    ids = np.arange(int(np.prod(nb)))
    bc = np.stack([ids // (nb[1] * nb[2]), (ids // nb[2]) % nb[1], ids % nb[2]], 1)
    fc = (bc * B + 0.5 * (B - 1)) / n
    half = 0.5 * np.sum(np.linalg.norm((B / n)[:, None] * s.cell, axis=1))
    fa = np.linalg.solve(s.cell.T, s.pos.T).T
    loads = np.zeros(len(ids))
    t = np.arange(-3, 4)
    T = np.stack(np.meshgrid(t, t, t, indexing="ij"), -1).reshape(-1, 3)
    for f in fa:
        d = np.linalg.norm(((fc[:, None, :] - f[None, None, :] - T[None]) @ s.cell), axis=2)
        loads += (d < 7.0 + half).sum(1)
    return loads


def _rank_main(rank, ws, port, out):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(ws),
                       "RANK": str(rank), "OMP_NUM_THREADS": "4"})
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        s = _system()
        brick = (6, 6, 6)
        o = oracle.Oracle(s)
        V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
        D = o.d_fill()
        nb = shard.bricks_per_axis(s.grid, brick)
        parts = shard.partition_slabs(shard.brick_costs(_host_loads(s, brick)), nb, ws)
        mask = shard.brick_point_mask(parts[rank], s.grid, brick)
        # this rank's partial results (the sums of Eq. 2-5 over its slab's grid points)
        H = torch.from_numpy(o.vlocal_masked(V, mask))
        F, W = o.force_masked(V, D, mask)
        F = torch.from_numpy(F)
        sigma = torch.from_numpy(-W.sum(0) / o.omega)
        pts = np.argwhere(mask)
        rho_slab = o.rho_points(D, pts)
        E = torch.tensor([float(np.sum(V[mask].reshape(-1) * rho_slab)) * o.dV], dtype=torch.float64)
        segs = shard.row_owner_segments(o.blocks, o.offsets, s.n_atoms, ws)
        shard.reduce_to_owners(H, segs)
        shard.allreduce_sum(F, sigma, E)
        # single-rank references
        H_ref = o.vlocal(V)
        F_ref, W_ref = o.force(V, D)
        rho_ref = o.rho(D)
        E_ref = o.energy(V, D)
        v0, v1 = segs[rank]
        eH = float(np.max(np.abs(H.numpy()[v0:v1] - H_ref[v0:v1]), initial=0.0)) / float(np.max(np.abs(H_ref)))
        eF = float(np.max(np.abs(F.numpy() - F_ref))) / max(1.0, float(np.max(np.abs(F_ref))))
        eS = float(np.max(np.abs(sigma.numpy() - (-W_ref.sum(0) / o.omega))))
        eR = float(np.max(np.abs(rho_slab - rho_ref[mask])))
        # E = sum V rho dV cancels heavily (V and rho change sign): relative to sum |V rho| dV
        eE = abs(float(E[0]) - E_ref) / (float(np.sum(np.abs(V * rho_ref))) * o.dV)
        out.put((rank, len(parts[rank]), v1 - v0, eH, eF, eS, eR, eE))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_rank_results():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    ws, port = 2, _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [out.get(timeout=600) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert sum(r[1] for r in res) == 27 and all(r[1] > 0 for r in res)  # every brick dealt once
    assert all(r[2] > 0 for r in res)  # each rank owns part of H
    for rank, nbk, nval, eH, eF, eS, eR, eE in res:
        print(f"rank {rank}: {nbk} bricks, {nval} H values owned: H {eH:.1e} F {eF:.1e} sigma {eS:.1e} "
              f"rho {eR:.1e} E {eE:.1e}")
        assert eH < 1e-13 and eF < 1e-12 and eS < 1e-12 and eR == 0.0 and eE < 1e-12
