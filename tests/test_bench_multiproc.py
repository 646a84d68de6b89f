"""Host side of the multi-process bench path on CPU: two gloo ranks (the
replicas of `bench.py --gpus 2` under torchrun) agree on the max-over-ranks
timing, pass the barriers, and only rank 0 runs the reference arm."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "TOMO_BENCH_BACKEND": "gloo"})
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_init()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    t = bench.max_over_ranks(w, 1.5 + rank)
    bench.barrier(w)

    class Args:
        steps, warmup, gpus = 1, 0, world

    # ranks other than 0 return at once without touching the oracle
    ran = False
    if rank != 0:
        bench.run_reference(Args, w, r)
        ran = True
    out.put((rank, t, ran))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_max_and_barrier():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    assert all(t == 2.5 for _, t, _ in res)
    assert res[1][2] is True
