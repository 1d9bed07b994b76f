"""The density-probe skip inside an occupied block, replayed on the CPU in binary32.

Inside a block the march probes the nearest voxel of sample k. A non-zero probe value D
says that no voxel of the block within Chebyshev distance D - 1 of it, in the cone of
the ray's direction octant, has density; the march then jumps to k + max(1, ceil(q)),
q = (D - 1 - eps) / m (biased down), m = max_i |d_i| and eps bounding the rounding of
the lattice. This test builds blocks with random voxels and with thin planes of density
(the case where a ray runs beside a surface), computes the one-sided distance map by
brute force, replays the probe loop along random rays with the kernel's binary32
arithmetic, and checks that every sample it jumps over has a nearest voxel without
density -- so the composited samples are exactly those of a sample-by-sample march."""

import numpy as np
import pytest

F = np.float32


def _cone_distance(occ, octant, cap=255):
    n = occ.shape[0]
    cells = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)   # (z, y, x)
    q = cells[occ.reshape(-1)]
    out = np.full(n ** 3, cap, np.int64)
    if len(q):
        diff = q[None] - cells[:, None]
        sign = np.array([-1 if (octant >> 2) & 1 else 1, -1 if (octant >> 1) & 1 else 1, -1 if octant & 1 else 1])
        ok = ((diff * sign) >= 0).all(-1)
        out = np.minimum(np.where(ok, np.abs(diff).max(-1), cap).min(1), cap)
    return out.reshape(occ.shape)


def _block(rng, B, kind):
    occ = np.zeros((B, B, B), bool)
    if kind == "random":
        occ = rng.uniform(size=(B, B, B)) < 0.03
    else:                                               # a thin plane of density, random orientation
        axis = int(rng.integers(0, 3))
        idx = [slice(None)] * 3
        idx[axis] = int(rng.integers(0, B))
        occ[tuple(idx)] = True
    return occ


@pytest.mark.parametrize("kind,seed", [("random", 1), ("plane", 2), ("plane", 3)])
def test_skipped_samples_are_empty(kind, seed):
    rng = np.random.default_rng(seed)
    B, N = 16, 16                                       # one block filling the grid
    occ = _block(rng, B, kind)
    maps = [_cone_distance(occ, o) for o in range(8)]
    checked_skips = 0
    for _ in range(400):
        d = rng.normal(size=3)
        if rng.uniform() < 0.5:                         # nearly parallel to an axis plane
            d[rng.integers(0, 3)] *= 10.0 ** rng.uniform(-4, -1)
        d = (d / np.linalg.norm(d)).astype(F)
        o = rng.uniform(0.5, N - 0.5, 3).astype(F)     # ray starts inside the grid
        t0 = F(0.0)
        tf = np.inf
        for i in range(3):
            if d[i] != 0:
                ta, tb = F(F(-o[i]) / d[i]), F(F(F(N) - o[i]) / d[i])
                tf = min(tf, max(ta, tb))
        t1 = F(tf)
        octant = int(d[0] < 0) | int(d[1] < 0) << 1 | int(d[2] < 0) << 2
        vmap = maps[octant]
        m = F(max(abs(float(x)) for x in d))
        skip_inv_m = F(F(1.0 - 1.0 / 1048576.0) / m)
        skip_eps = F(F(max(float(t1), float(N))) * F(1.0 / 524288.0))

        def nearest(k):
            t = F(t0 + F(F(k) + F(0.5)))
            if not t < t1:
                return None
            u = [F(o[i] + F(t * d[i])) for i in range(3)]
            return tuple(min(max(int(np.floor(x)), 0), N - 1) for x in u)   # (x, y, z)

        k = 0
        while True:
            v = nearest(k)
            if v is None:
                break
            D = int(vmap[v[2], v[1], v[0]])
            if D == 0:
                k += 1
                continue
            q = F(F(F(D) - F(1.0) - skip_eps) * skip_inv_m)
            step = max(1, int(np.ceil(q)))
            for j in range(k + 1, k + step):
                w = nearest(j)
                if w is None:
                    break
                assert not occ[w[2], w[1], w[0]], (o, d, k, j, D)
                checked_skips += 1
            k += step
    assert checked_skips > 1000
