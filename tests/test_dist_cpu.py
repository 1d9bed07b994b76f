"""The multi-rank paths on CPU with the gloo backend (world size 2): the bench's forward
shards (each rank gets its own view of the shared grid, weak scaling, no data exchanged;
the step time is the maximum over ranks) and the exchange step of data-parallel
fine-tuning (gradients summed over the ranks, atlas gradients over touched blocks only)."""
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


class _TorchBlockOps:
    """CPU stand-ins for the library's touched / gather / scatter kernels (the kernels
    themselves are checked against these on the GPU)."""

    @staticmethod
    def touched(g):
        import torch
        return (g.reshape(g.shape[0], -1) != 0).any(1).to(torch.int32)

    @staticmethod
    def gather(g, idx):
        return g.reshape(g.shape[0], -1)[idx.long()].clone()

    @staticmethod
    def scatter(p, idx, g):
        g.reshape(g.shape[0], -1).index_copy_(0, idx.long(), p)


def _exchange_worker(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from paper_2103_14645_gb300 import renderer
    gm = torch.arange(883, dtype=torch.float32) * (rank + 1)
    ga = torch.zeros((6, 2, 2, 2, 8), dtype=torch.float32)
    touched = [(0, 2), (2, 5)][rank]
    for b in touched:
        ga[b] = torch.arange(64, dtype=torch.float32).reshape(2, 2, 2, 8) + 100 * (rank + 1) + b
    n = renderer.allreduce_gradients(gm, ga, ops=_TorchBlockOps)
    q.put((rank, n, gm.numpy().copy(), ga.numpy().copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gradient_exchange_over_touched_blocks():
    """dL/dPhi is summed; the atlas gradient is summed over the union of the touched blocks
    (rank 0 touched 0 and 2, rank 1 touched 2 and 5) and stays zero elsewhere, the same on
    both ranks."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    base = np.arange(64, dtype=np.float32).reshape(2, 2, 2, 8)
    want = np.zeros((6, 2, 2, 2, 8), np.float32)
    for rank, blocks in ((0, (0, 2)), (1, (2, 5))):
        for b in blocks:
            want[b] += base + 100 * (rank + 1) + b
    for rank, n, gm, ga in res:
        assert n == 3
        np.testing.assert_array_equal(gm, np.arange(883, dtype=np.float32) * 3)
        np.testing.assert_array_equal(ga, want)
