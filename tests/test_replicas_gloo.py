"""The N > 1 host logic of the benchmark (paper_2608_15764_gb300.replicas)
over a world of two gloo ranks on the CPU: rank 0's choice reaches every rank,
the job's interval is the maximum over ranks, per-rank result triples (with
64-bit XORs above 2^63) arrive intact and in rank order, and the whole-job
throughput counts every rank's bytes."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

from paper_2608_15764_gb300 import replicas  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        choice = replicas.broadcast_choice(7 if rank == 0 else 3, dist)
        tmax = replicas.max_over_ranks(10.0 + rank, dist, device="cpu")
        xor = (0xF000_0000_0000_0001 + rank) if rank else 0xFFFF_FFFF_FFFF_FFFF
        got = replicas.gather_results(0xFFFF_FFF0 + rank, xor, 1 << 40, dist, device="cpu")
        dist.barrier()
        q.put((rank, choice, tmax, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, choice, tmax, got = q.get(timeout=120)
        out[rank] = (choice, tmax, got)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = [(0xFFFF_FFF0, 0xFFFF_FFFF_FFFF_FFFF, 1 << 40), (0xFFFF_FFF1, 0xF000_0000_0000_0002, 1 << 40)]
    for rank in (0, 1):
        choice, tmax, got = out[rank]
        assert choice == 7
        assert tmax == 11.0
        assert got == want


def test_single_process_defaults():
    assert replicas.broadcast_choice(5) == 5
    assert replicas.max_over_ranks(2.5) == 2.5
    assert replicas.gather_results(1, 2, 3) == [(1, 2, 3)]


def test_job_throughput_counts_every_rank():
    # 2 ranks x 4 GiB x 10 steps in 12 ms (slowest rank)
    assert replicas.job_gbs(4 << 30, 10, 2, 12.0) == pytest.approx(2 * (4 << 30) * 10 / 12e6)
    with pytest.raises(ValueError):
        replicas.job_gbs(1, 1, 1, 0.0)


def test_env_rank_defaults(monkeypatch):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench._dist() == (0, 1, 0)
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench._dist() == (1, 2, 1)


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the oracle arm; other ranks exit 0 and
    print nothing."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
