"""The N > 1 path of the benchmark on CPU: two gloo ranks.

Every rank runs its own independent batch (weak scaling, no data-path collective): the job's time
is the slowest rank's (a max all-reduce), its throughput the units of all ranks over that time,
each rank draws its own seeded inputs, and only rank 0 reports."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.rank_env()
        ms = 10.0 + 5.0 * r                               # rank 1 is the slower one
        job_ms = bench.max_over_ranks(ms, w, "cpu")
        rate = bench.job_rate(1000, w, job_ms)
        # per-rank inputs: the rank's seed offset gives it its own batch
        d = synth.batch_stencils(64, seed=20230810 + r)
        first = float(d["x"][0, 0])
        t = torch.tensor([first], dtype=torch.float64)
        gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(w)]
        dist.all_gather(gathered, t)
        out[r] = (w, r, local, job_ms, rate, [float(g.item()) for g in gathered])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_aggregate_throughput():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r, (w, rr, local, job_ms, rate, firsts) in res.items():
        assert (w, rr, local) == (2, r, r)
        assert job_ms == 15.0                    # the slowest rank's time, on every rank
        assert rate == pytest.approx(2 * 1000 / 15e-3)
        assert firsts[0] != firsts[1]           # each rank has its own batch
    assert res[0][5] == res[1][5]


def test_single_process_defaults(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.rank_env() == (1, 0, 0)
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_rate(1000, 1, 10.0) == pytest.approx(1e5)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.run_reference(None) is None       # no work and no output on the other ranks
    assert capsys.readouterr().out == ""
