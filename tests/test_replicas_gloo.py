"""The multi-rank bench path on CPU: two gloo ranks, as torchrun would start them on two GPUs.
Each rank works on its own seeded cube (no data-path collective); the only collective is the
max over ranks of the timed region, and the job value counts every rank's pixels."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_1201_2025_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench._dist() == (ws, rank, rank)
    ms = [0.7, 1.9][rank]  # the ranks' own timed regions
    got = bench.max_over_ranks(ms, ws, "cpu")
    cube = synth.make_scene(12, 12, 16, rank, n_anom=2, margin=2).cube  # the per-rank seed, small
    sig = float(cube.sum())
    sigs = [None] * ws
    dist.all_gather_object(sigs, sig)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, got, bench.job_value(ws, got), sigs))


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import bench
    for rank, got, value, sigs in res:
        assert got == 1.9                      # the slowest rank's time
        assert value == bench.job_value(2, 1.9) == 2 * bench.job_value(1, 1.9)
        assert sigs[0] != sigs[1]              # each rank has its own cube


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.job_value(1, 1.0) == pytest.approx(3 * bench.H * bench.W / 1e3)
