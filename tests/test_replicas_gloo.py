"""Multi-GPU path (replicas, no collective on the data path), exercised with
two gloo ranks on the CPU: the bench's cross-rank reduction takes the
slowest rank's time and the sum of the ranks' work, every rank solves its
own seeded problem, and only rank 0 runs the reference arm."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dev_ms = [100.0, 250.0][rank]
    e2e = [1.0, 3.0][rank]
    evals = [1000.0, 3000.0][rank]
    e2e_evals = [10.0, 30.0][rank]
    r = bench.reduce_ranks(torch, dist, "cpu", dev_ms, e2e, evals, e2e_evals)
    w = bench.WORKLOADS["chain100"]
    p = bench._problem(w, seed=rank)
    out.put((rank, r, float(p.s[0])))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict()
    for _ in procs:
        rank, r, s0 = q.get(timeout=120)
        got[rank] = (r, s0)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        assert got[rank][0] == (250.0, 3.0, 4000.0, 40.0)   # max time, summed work, on every rank
    assert got[0][1] != got[1][1]                            # each rank solves its own replica


def test_reference_arm_prints_only_on_rank_zero(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    class A:
        workload, cpu_gens, warmup, steps, gpus = "chain100", 1, 0, 1, 2
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
