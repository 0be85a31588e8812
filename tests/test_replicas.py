"""Host-side logic of the multi-GPU bench (independent replicas, one per
rank): the job's step time is the MAX over ranks, the value counts every
rank's solves, only rank 0 prints, the reference arm runs on rank 0 alone.
World size 2 over gloo on the CPU (no GPU involved)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import bench
    w, r, loc = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    ms = bench.job_ms(10.0 + 5.0 * rank, dist, device="cpu")      # rank 1 is slower
    ref = bench.reference_arm(type("A", (), {"steps": 1, "warmup": 0})(), w, r) if r == 1 else None
    out.put((r, w, loc, ms, bench.job_value(w, ms), ref))
    dist.destroy_process_group()


def test_two_replicas_over_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, w, loc, ms, value, ref) in enumerate(res):
        assert (r, w, loc) == (rank, 2, rank)
        assert ms == 15.0                                  # the slowest rank's time
        assert value == pytest.approx(2 * 8 / 15e-3)       # both replicas' solves
    assert res[1][5] is None                               # reference arm: rank 0 only


def test_single_process_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.job_ms(12.5) == 12.5
    assert bench.job_value(1, 25.0) == pytest.approx(320.0)
