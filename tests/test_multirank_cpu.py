"""The N>1 path of bench.py on CPU: two gloo ranks, the job time is the
maximum over ranks, and the reference arm runs on rank 0 only."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank], world, device="cpu")
        out[rank] = got
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == [2.0, 10.0] and out[1] == [2.0, 10.0]


def test_reference_arm_other_ranks_do_nothing(capsys):
    import argparse

    import bench
    bench.run_reference(argparse.Namespace(steps=1, warmup=3), rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks([3, 4], 1) == [3.0, 4.0]
