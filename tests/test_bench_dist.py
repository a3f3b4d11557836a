"""Multi-rank logic of bench.py on the CPU (gloo, world size 2): the job time
is the maximum over ranks, and the reference arm runs on rank 0 only."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_setup(world)
    assert (r, w) == (rank, world) and dist.get_backend() == "gloo"
    bench.barrier(w)
    out[rank] = bench.reduce_max(1.5 + rank, w)

    class A:
        steps, warmup, ref_budget, gpus = 1, 0, 1e-6, 2
    out[world + rank] = 0.0 if bench.reference_arm(A(), r) is None else 1.0
    dist.destroy_process_group()


def test_max_over_ranks_and_rank0_reference():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Array("d", 2 * world)
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert list(out[:world]) == [2.5, 2.5]
    assert list(out[world:]) == [1.0, 0.0]

