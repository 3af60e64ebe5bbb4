"""The multi-GPU form is independent replicas (one RVE per rank, no data-path
collective); its host logic runs here as world-size-2 gloo process groups on the CPU:
the whole-job totals (slowest rank's time, summed voxel-iterations), distinct seeded
realizations per rank, and the reference arm's other ranks exiting without work."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [1.25, 2.5][rank]
        vox = [3.0e9, 5.0e9][rank]
        t, v = bench.job_totals(secs, vox, world, device="cpu")
        from paper_1504_07499_gb300 import inputs as I
        sl = I.generate_spheres(bench.replica_seed(rank), 20, 0.2)
        dist.barrier()
        q.put((rank, t, v, sl.spheres.tolist()))
    finally:
        dist.destroy_process_group()


def test_job_totals_and_replicas_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        r, t, v, sph = q.get(timeout=120)
        out[r] = (t, v, sph)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        t, v, _ = out[r]
        assert t == 2.5                     # the slowest rank's time
        assert v == 8.0e9                   # every rank's voxel-iterations
    assert out[0][2] != out[1][2]           # independent realizations (seed 3000 + rank)


def test_single_rank_totals_are_local():
    assert bench.job_totals(1.5, 7.0, 1) == (1.5, 7.0)
    assert bench.replica_seed(0) == bench.SEED and bench.replica_seed(3) == bench.SEED + 3


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup, gpus = 1, 0, 2

    bench.run_reference(Args())             # returns at once: no oracle work, no output
    assert capsys.readouterr().out == ""
