"""Host logic of bench.py's multi-rank (torchrun) path on CPU: two gloo ranks
with different local timings agree on the slowest rank's time and on the
whole-job rate; non-zero ranks of the reference arm exit without work."""
import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

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


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        local_s = [1.5, 2.5][rank]
        t = b.max_over_ranks(local_s, dist, "cpu")
        dist.barrier()
        q.put((rank, t, b.job_rate(100, world, t)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, rate in out:
        assert t == 2.5
        assert rate == pytest.approx(2 * 100 / 2.5)


def test_single_process_needs_no_group():
    b = _bench()
    assert b.max_over_ranks(3.0) == 3.0
    assert b.job_rate(400, 1, 0.5) == 800.0


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    b = _bench()
    monkeypatch.setenv("RANK", "1")

    class A:
        gpus, steps, warmup = 2, 3, 3
    assert b.run_reference(A()) is None
    assert capsys.readouterr().out == ""
