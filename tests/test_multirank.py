"""The multi-rank bench path on CPU: two gloo ranks (127.0.0.1) check the Philox
counter ranges of the ranks are disjoint, the whole-job rate takes the slowest
rank, and the Monte Carlo sums of the ranks add up (no GPU)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        steps, n = 25, 1 << 20
        lo = bench.rank_offset(rank)
        ranges = [None] * world
        dist.all_gather_object(ranges, (lo, lo + steps * n))
        step_ms = 2.0 + rank  # the second rank is slower
        value, t_max = bench.job_rate(step_ms, n, world, dist)

        class Acc:
            sum_w, sum_w2, n_acc, n_try = 1.5 * (rank + 1), 0.25 * (rank + 1), n, n + 10 * rank
        mc = bench.merge_acc(Acc, world, dist)
        if rank == 0:
            out.put((ranges, value, t_max, mc))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    ranges, value, t_max, mc = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (a0, a1), (b0, b1) = ranges
    assert a1 <= b0 or b1 <= a0                      # disjoint counters
    assert t_max == 3.0                              # the slowest rank
    assert value == pytest.approx(2 * (1 << 20) / 3.0e-3)
    assert mc == {"sum_w": 4.5, "sum_w2": 0.75, "n_acc": 2 << 20, "n_try": (2 << 20) + 10}


def test_issue_roofline_arithmetic():
    """The issue-rate roofline: instructions per point x points / time against 152 x 4 x clock."""
    import bench
    r = bench.issue_roofline("udx_epvegg", "k_ps", 0.222, 2 ** 20)
    assert r["peak"] == pytest.approx(152 * 4 * 2.07)
    per_point = bench.WARP_INSTRUCTIONS_PER_POINT[("udx_epvegg", "k_ps")]
    assert r["achieved"] == pytest.approx(per_point * 2 ** 20 / 0.222e-3 / 1e9)
    assert 0.5 < r["frac"] < 0.8
    assert bench.issue_roofline("uux_epem", "k_ps", 0.1, 65536) is None
