"""The benchmark's multi-process path on CPU: two gloo ranks.

The hot path does not shard (one solver per GPU, no exchange), so `bench.py --gpus N` runs N
independent replicas: each rank times its own steps, the ranks meet at barriers around the
timed region, and rank 0 reports the slowest rank's time.  These tests run the benchmark's own
process-group helpers in two CPU processes over gloo, and the reference arm's rank rule
(rank 0 alone runs the oracle, the other ranks exit without work).
"""
import importlib.util
import os
import socket

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    bench = _bench()
    w, r, _ = bench.dist_setup(None)
    assert (w, r) == (world, rank)
    bench.barrier(w)
    out[rank] = bench.max_over_ranks(10.0 + 5.0 * rank, w)   # the slowest rank's time wins
    # the reference arm: only rank 0 does (and prints) anything
    class A:
        steps, warmup, n, gpus = 1, 0, 64, world
    called = []
    bench.oracle_sample = lambda **kw: called.append(kw) or (1.0, 1, 1.0, 1)
    bench.run_reference(A, w, r)
    out[100 + rank] = len(called)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == 15.0
    assert res[100] == 1 and res[101] == 0
