"""The benchmark's multi-rank logic on CPU (gloo, world size 2).

With N GPUs every rank evaluates its own independent cloud; the only
cross-rank operations are a barrier and an all-reduce(MAX) of the elapsed
time, and the whole-job throughput is the points of all ranks over the
slowest rank's time.  These run here on two CPU processes.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2308_00292_gb300 import inputs
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        cfg = inputs.CONFIGS["laplace3d_clustered_n1e7"]
        ms_local = 10.0 + 5.0 * rank
        dist.barrier()
        ms = bench.max_over_ranks(ms_local, dist, "cpu")
        value = bench.job_throughput(1000, world, ms)
        # each rank's cloud is its own: different seeds, different points
        seed = bench.rank_seed(cfg, rank)
        x, _ = inputs.make("uniform_cube", 8, seed)
        out[rank] = (ms, value, seed, float(x[0, 0]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_weak_throughput():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert set(res) == {0, 1}
    # every rank sees the slowest rank's time
    assert res[0][0] == res[1][0] == 15.0
    # whole-job points/s = (points per rank x ranks) / slowest time
    assert res[0][1] == pytest.approx(2 * 1000 / 15e-3)
    # independent replicas: distinct seeds and points
    assert res[0][2] != res[1][2]
    assert res[0][3] != res[1][3]


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    import bench

    def boom(*a, **k):
        raise AssertionError("rank 1 must not run the oracle")

    monkeypatch.setattr(bench, "cpu_baseline", boom)

    class A:
        config = "laplace3d_clustered_n1e7"
        cpu_sample = 1000
        steps = 1
        warmup = 3
        gpus = 2

    bench.run_reference(A, rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(10_000_000, 1, 122.0) == pytest.approx(1e7 / 0.122)
