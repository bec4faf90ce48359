"""Host logic of bench.py on CPU: the N > 1 path on two gloo ranks, and the
clock record.

Block PLHR on one problem does not shard here (one GPU per box), so N ranks
run N replicas and the reported time is the maximum over the ranks, taken
between barriers.  These tests run that reduction and the barrier as two
processes over gloo, check that the reference arm does no work on ranks
other than 0, and parse nvidia-smi samples into the clock summary."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        w, r, _ = bench._dist()
        bench._barrier(w)
        # per-rank step times; every rank must report the slowest
        m = bench._max_over_ranks(1.25 + 0.5 * r, w)
        bench._barrier(w)
        q.put((r, w, m))
    finally:
        dist.destroy_process_group()


def test_replica_time_is_the_maximum_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    assert got == [(0, 2, 1.75), (1, 2, 1.75)]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.5, 1) == 3.5
    bench._barrier(1)


def test_reference_arm_returns_without_work_on_other_ranks():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup = 1, 0

    # rank 1 of 2 prints nothing and runs no oracle
    assert bench.run_reference(Args(), 2, 1, 1) is None


def test_clock_summary_parses_samples_and_throttle_reasons():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 950.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1001.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line", "0, [N/A], 2070, 0, 0x0, a, b, c, d"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    assert bench.ClockSampler(0).summary()["sm_mhz"] is None
