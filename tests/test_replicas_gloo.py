"""The multi-GPU form of the benchmark is replicas only (one independent
decomposition per rank, no collective on the data path).  Its host logic runs
here as two gloo ranks on the CPU: each rank draws its own seeded workload, the
timing barrier completes, and the max-over-ranks time reaches every rank."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        cfg = dict(bench.CFG)
        cfg.update(n_per=60, k=4, oversample=4, epochs=2)
        host = bench.make_inputs(cfg, rank)
        bench.dist_barrier(world)
        t_max = bench.dist_max(1.5 + rank, world)
        q.put((rank, t_max, int(host["G_XA"].nnz), float(host["V0"].sum()),
               host["perm"].shape))
    finally:
        dist.destroy_process_group()


def test_two_replicas_on_gloo():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, nnz0, v0, sh0), (r1, t1, nnz1, v1, sh1) = res
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 2.5                       # the max over ranks on every rank
    assert sh0 == sh1 == (2, 60)                 # same shapes of work per rank
    assert (nnz0, v0) != (nnz1, v1)              # each rank its own seeded workload
    assert np.isfinite(v0) and np.isfinite(v1)
