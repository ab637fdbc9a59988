"""The replica path of the benchmark on CPU: two gloo ranks (no GPU) aggregate their timings the
way the GPU ranks do under torchrun — job time = the slowest rank, throughput = all ranks' steps."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_2501_03061_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert replicas.env() == (world, rank, rank)
        job_s, value = replicas.job_throughput(1.0 + rank, steps=3)
        out.put((rank, job_s, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_steps():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, job_s, value in res:
        assert job_s == pytest.approx(2.0)          # rank 1 took 2 s
        assert value == pytest.approx(2 * 3 / 2.0)  # 6 steps in 2 s


def test_single_process_needs_no_process_group():
    from paper_2501_03061_gb300 import replicas
    assert replicas.job_throughput(0.5, steps=2) == (0.5, 4.0)


def test_reference_arm_prints_on_rank_zero_only(capsys, monkeypatch):
    """Under torchrun the reference arm runs on rank 0 alone; other ranks exit without output."""
    import importlib.util
    path = os.path.join(os.path.dirname(__file__), "..", "bench.py")
    spec = importlib.util.spec_from_file_location("bench_mod", path)
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(type("A", (), {"warmup": 0, "steps": 1})())
    assert capsys.readouterr().out == ""
