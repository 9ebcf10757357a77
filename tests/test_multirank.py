"""Host logic of the replicas run (bench.py under torchrun): world_size-2
gloo process groups on the CPU.  Each rank solves its own instance; the
whole-job line takes the slowest rank's time and the updates of all ranks,
and the reference arm prints from rank 0 only."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    ms, upd = bench.reduce_over_ranks(dist, 10.0 + 5.0 * rank, 1000 * (rank + 1), "cpu")
    out[rank] = (ms, upd)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo():
    world, port = 2, free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == (15.0, 3000.0)


def test_reduce_without_process_group_is_identity():
    assert bench.reduce_over_ranks(None, 7.5, 42, "cpu") == (7.5, 42.0)


class A:
    ng, np, box, rc, rtol, steps, warmup, pm_steps = 16, 8, 16.0, 1.0, 1e-8, 1, 1, 0


def test_ranks_solve_different_instances():
    p0, p1 = bench.particles(A, 0), bench.particles(A, 1)
    assert p0.shape == p1.shape and not np.array_equal(p0, p1)


def test_reference_arm_prints_from_rank_0_only():
    for rank in (1, 0):
        buf = io.StringIO()
        with redirect_stdout(buf):
            bench.run_reference(A, rank, 2)
        txt = buf.getvalue().strip()
        if rank == 1:
            assert txt == ""
        else:
            line = json.loads(txt.splitlines()[-1])
            assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
            assert line["cpu_baseline"]["kind"] == "oracle"
