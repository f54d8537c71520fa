"""The multi-GPU form of the benchmark is replicas only: every rank solves its
own copy of the pair, and the whole-job figure is all ranks' pairs over the
slowest rank's time. Its host side (the reduction over ranks, rank-0-only
output of the reference arm, the environment it reads) runs here as two gloo
processes on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        # rank r took 10 + r ms for 1000 (r + 1) pairs, e2e 20 + 3 r ms for 500 pairs
        got = bench.reduce_over_ranks(dist, 10.0 + r, 1000.0 * (r + 1), 20.0 + 3 * r, 500.0, "cpu")
        out.put((r, w, local, got))
    finally:
        dist.destroy_process_group()


def test_reduction_over_two_ranks():
    mp = torch.multiprocessing.get_context("spawn")
    out = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, local, got in res:
        assert w == 2 and local == r
        # the slowest rank's times, the sum of all ranks' pairs, on every rank
        assert got == (11.0, 3000.0, 23.0, 1000.0)


def test_single_process_reduction_is_the_identity():
    import bench
    assert bench.reduce_over_ranks(None, 5.0, 7.0, 9.0, 11.0, "cpu") == (5.0, 7.0, 9.0, 11.0)


def test_reference_arm_prints_on_rank_zero_only(capsys):
    import bench
    args = bench.argparse.Namespace(steps=1, warmup=0, impl="reference")
    bench.run_reference(args, 2, 1)   # rank 1 of 2: returns without work or output
    assert capsys.readouterr().out == ""
