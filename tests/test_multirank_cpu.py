"""The N > 1 path of bench.py on CPU with the gloo backend (world size 2):
every rank solves its own replica (no collective on the data path); the
timing takes the max over ranks and the work the sum; the reference arm
runs on rank 0 only."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    try:
        _work(rank, world, port, q)
    except BaseException as e:  # report instead of leaving the peer waiting
        q.put((rank, None, None, f"error: {e!r}"))
        raise


def _work(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    cpu = torch.device("cpu")
    t_max = bench.reduce_over_ranks(10.0 + 5.0 * rank, "max", cpu)
    w_sum = bench.reduce_over_ranks(100.0 * (rank + 1), "sum", cpu)
    # the reference arm prints only on rank 0 (a tiny workload)
    import contextlib
    import io
    buf = io.StringIO()

    class A:
        side, stencil, steps, warmup, tol, band, band_n = 6, 7, 1, 1, 1e-8, 0, 0
        variant, max_iter, gpus = "exblas", 1000, 2

    with contextlib.redirect_stdout(buf):
        bench.reference_arm(A, rank, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t_max, w_sum, buf.getvalue()))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    errors = [o[3] for o in out if o[1] is None]
    assert not errors, errors
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [15.0, 15.0]  # max of the per-rank times
    assert [o[2] for o in out] == [300.0, 300.0]  # sum of the per-rank work
    assert '"impl": "reference"' in out[0][3] and out[1][3] == ""
