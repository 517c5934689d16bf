"""Multi-rank bench plumbing on CPU: world_size 2 over gloo (barrier, max over ranks, replicas).

The embedding shards as independent problems (one graph per rank, no collective on the data
path); the only cross-rank operations are the barrier around the timed region and the max of
the per-rank times, which these tests exercise without a GPU.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    d = bench.Dist("gloo")
    d.barrier()
    m = d.max(float(10 * rank + 1))
    ref = None
    if rank == 0:
        class A:  # a tiny reference-arm configuration
            shape, knn, K, tol, precision, seed = "square", 8, 2, 1e-5, "fp32", 1
            n = 1000
            cpu_sample_n = 600
            steps, warmup = 1, 0
        ref = bench.run_reference(A, d)
    else:
        ref = bench.run_reference(type("A", (), {"shape": "square", "knn": 8, "K": 2, "tol": 1e-5,
                                                 "precision": "fp32", "seed": 1, "n": 1000,
                                                 "cpu_sample_n": 600, "steps": 1, "warmup": 0}), d)
    d.barrier()
    d.close()
    q.put((rank, m, ref))


def test_world2_max_and_reference_on_rank0_only():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = {}
    for _ in ps:
        r, m, ref = q.get(timeout=300)
        out[r] = (m, ref)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 11.0
    assert out[0][1]["impl"] == "reference" and out[0][1]["value"] > 0
    assert out[1][1] is None
