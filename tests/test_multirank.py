"""Host logic of the multi-GPU benchmark path (replicas only: one independent box per rank,
no data-path collective) on CPU with the gloo backend, world size 2."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    t_ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)  # rank 1 is the slow one
    q.put((rank, t_ms, bench.aggregate_rate(world, 1000, 4, t_ms)))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_rate():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]           # both ranks see the slowest rank's time
    assert out[0][2] == pytest.approx(2 * 1000 * 4 / 15e-3)  # all ranks' atoms / max time
    assert torch is not None


def test_reference_arm_runs_on_rank0_only():
    sys.path.insert(0, ROOT)
    import bench
    args = SimpleNamespace(workload="cu131k", steps=1, warmup=0, gpus=2)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, 2, 1)  # rank 1 of 2: exits without work or output
    assert buf.getvalue() == ""
