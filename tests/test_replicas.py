"""The N>1 path of bench.py on CPU: two gloo ranks (replicas only; no data-path collective).

The timing helpers must synchronise the ranks and report the slowest rank's time, and the
reference arm's non-zero ranks must leave without work."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    # slowest rank's time
    out[rank] = bench.max_over_ranks(world, 10.0 * (rank + 1), None)
    dist.destroy_process_group()


def test_two_gloo_ranks_max_over_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {0: 20.0, 1: 20.0}


def _reference_rank(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    called = []
    bench.oracle_apply_fn = lambda case, step, n: (lambda: called.append(1), 1000, "stand-in")   # stand-in step
    import argparse
    args = argparse.Namespace(impl="reference", gpus=world, steps=2, warmup=3, case="strut20", state_step=1,
                              sample_cells=8)
    rc = bench.run_reference(args)
    out[rank] = (rc, len(called))


def test_reference_arm_other_ranks_do_no_work():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_reference_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == (0, 5) and out[1] == (0, 0)
