"""Replica mode on CPU: the bench's rank plumbing over gloo, world size 2.

With several GPUs, each rank runs an independent box (no data-path
collective); the only collectives are the timing reductions: the job's
throughput is the units of all ranks over the slowest rank's time. The
reference arm runs on rank 0 alone.
"""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    class Args:
        impl = "ours"

    r, w, _ = bench.dist_setup(Args())
    assert dist.get_backend() == "gloo"
    # rank 0: 100 units in 2 s; rank 1: 300 units in 4 s -> 400 units / 4 s
    units, secs = (100.0, 2.0) if r == 0 else (300.0, 4.0)
    thr = bench.replica_throughput(units, secs, w)
    m = bench.dist_max(float(r + 1), w)
    bench.barrier(w)
    # the reference arm: ranks other than 0 return without work
    skipped = bench.run_reference(None, r, w) is None if r != 0 else True
    out.put((r, w, thr, m, skipped))
    dist.destroy_process_group()


def test_replica_throughput_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1]
    for r, w, thr, m, skipped in res:
        assert w == 2
        assert thr == 100.0
        assert m == 2.0
        assert skipped
