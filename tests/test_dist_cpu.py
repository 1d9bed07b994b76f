"""The multi-rank bench path on CPU with the gloo backend (world size 2): each rank gets
its own view of the shared grid (weak scaling, no data exchanged) and the step time is
the maximum over ranks."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    from paper_2103_14645_gb300 import synth
    sc = synth.make_scene("tiny")
    cams = bench.rank_cameras(sc, rank)
    t = bench.reduce_max(1.5 + rank, torch.device("cpu"))
    v = bench.whole_job_mrays(ws, 640000, t)
    q.put((rank, np.asarray(cams["c2w"]).tolist(), int(cams["W"][0]), t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, cam0, w0, t0, v0), (r1, cam1, w1, t1, v1) = res
    assert (r0, r1) == (0, 1)
    assert cam0 != cam1                  # each rank renders its own view
    assert w1 == 800
    assert t0 == t1 == 2.5               # the slowest rank decides the step time
    assert v0 == v1 == pytest.approx(2 * 640000 / 2.5e-3 / 1e6)
