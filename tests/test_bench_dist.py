"""bench.py's cross-rank timing on CPU: two gloo ranks (one process each)."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(ws),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ws_env, rank_env, local_env = bench.dist_env()
        # per-rank step times differ; every rank must see the slowest one
        t_max = bench.max_over_ranks(100.0 + 25.0 * rank, ws_env, "cpu")
        out.put((rank_env, local_env, ws_env, t_max, bench.whole_job_rate(1000, 4, ws_env, t_max)))
    finally:
        dist.destroy_process_group()


def test_one_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_rate(1000, 4, 1, 2000.0) == pytest.approx(2000.0)


def test_two_gloo_ranks_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    ws, port = 2, _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and [r[1] for r in res] == [0, 1]
    for _, _, ws_env, t_max, rate in res:
        assert ws_env == 2 and t_max == 125.0
        # 1000 units per rank and step, 4 steps, 2 ranks, 125 ms
        assert rate == pytest.approx(1000 * 4 * 2 / 0.125)
