"""The multi-process side of bench.py on CPU (gloo, world size 2): ranks run
independent replicas of the fit and only exchange their timings, the slowest
rank's time setting the job's throughput."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    b = _bench()
    w, r, lr = b.dist_env()
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=r, world_size=w)
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is slower
        ms_max = b.max_over_ranks(ms, w)
        out[rank] = (w, r, lr, ms_max, b.job_throughput(w, 1000, 4, ms_max))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for rank in (0, 1):
        w, r, lr, ms_max, value = res[rank]
        assert (w, r, lr) == (2, rank, rank)
        assert ms_max == 15.0
        # 2 ranks x 1000 units x 4 steps in 15 ms
        assert value == pytest.approx(2 * 1000 * 4 / 0.015)


def test_single_rank_is_identity():
    b = _bench()
    assert b.max_over_ranks(3.25, 1) == 3.25
    assert b.job_throughput(1, 60, 2, 1.0) == pytest.approx(120000.0)
