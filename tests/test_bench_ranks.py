"""The benchmark's multi-rank logic on CPU: two `gloo` ranks (as torchrun
starts them: RANK, WORLD_SIZE, MASTER_ADDR/PORT in the environment).  Each
rank runs its own replica of the workload (replicas only, no data-path
collective); the timed region is the slowest rank's and the rate is the
whole job's.  The reference arm runs on rank 0 alone."""
import argparse
import importlib.util
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    bench = _bench()
    args = argparse.Namespace(impl="reference", gpus=world, steps=0, warmup=0)
    r, w, local, dist = bench.dist_setup(args)
    assert (r, w, local) == (rank, world, rank) and dist is not None
    # rank r took r + 1 seconds: every rank sees the slowest one
    t_max = bench.slowest_rank_time(float(rank + 1), dist, "cpu")
    rate = bench.whole_job_rate(1000, 10, w, t_max)
    # the reference arm prints on rank 0 only; other ranks return at once
    if rank != 0:
        bench.run_reference(args, r, w)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t_max, rate))


def test_two_gloo_ranks_time_the_slowest_and_count_all_particles():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(out.get(timeout=10) for _ in range(world))
    assert [g[0] for g in got] == [0, 1]
    for _, t_max, rate in got:
        assert t_max == 2.0
        assert rate == 1000 * 10 * 2 / 2.0


def test_single_rank_needs_no_process_group():
    bench = _bench()
    args = argparse.Namespace(impl="reference", gpus=1, steps=0, warmup=0)
    env = {k: os.environ.pop(k) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_setup(args) == (0, 1, 0, None)
    finally:
        os.environ.update(env)
    assert bench.slowest_rank_time(1.5, None, "cpu") == 1.5
    assert bench.whole_job_rate(100, 10, 1, 2.0) == 500.0


def test_timed_region_is_whole_graph_replays():
    """The benchmark times whole graphs whatever --steps is: the graph length
    divides the step count, and the untimed alignment leaves the step counter
    on a graph (thermo) boundary."""
    bench = _bench()
    for steps, g in ((20, 20), (1000, 100), (150, 75), (7, 7), (101, 1), (300, 100), (1, 1)):
        assert bench.graph_len(steps) == g
        assert steps % g == 0 and g <= 100
    for step in (0, 1, 99, 100, 1234):
        for g in (1, 20, 100):
            a = bench.align_steps(step + g, g)
            assert (step + g + a) % g == 0 and 0 <= a < g
