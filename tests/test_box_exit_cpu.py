"""The march's unconfirmed block exits, replayed on the CPU in binary32.

A block (or empty box) run ends at the first lattice sample whose nearest voxel leaves
the box. The kernel estimates that index from the ray/face distance and, when the real
crossing is at least a margin away from every integer, takes the estimate without
checking samples on the lattice. This test replays that arithmetic with numpy float32
(one rounding per operation, as the kernel's binary32 control arithmetic does), with the
reciprocal of each direction component perturbed by up to 2 ulp (the error bound of the
approximate reciprocal the kernel uses), on random rays and on rays built so that a face
crossing falls within 1e-3 samples of a lattice point, and on rays whose first face
crossing comes before the second sample (an estimate K in (0, 1), where the fraction
1 - K of K < 1/2 is rounded). Whenever the estimate is taken it must equal the first
index found by stepping the lattice one sample at a time."""

import numpy as np
import pytest

F = np.float32
INF = F(np.inf)


def _ulp_perturb(x: np.float32, rng, max_ulp=2):
    steps = int(rng.integers(-max_ulp, max_ulp + 1))
    for _ in range(abs(steps)):
        x = np.nextafter(x, INF if steps > 0 else -INF, dtype=F)
    return x


def _lattice_t(t0, k):
    return F(t0 + F(F(k) + F(0.5)))


def _in_box(o, d, t0, t1, k, lo, hi):
    t = _lattice_t(t0, k)
    if not t < t1:
        return False
    for i in range(3):
        u = F(o[i] + F(t * d[i]))
        if not (u >= lo[i] and u < hi[i]):
            return False
    return True


def _exit_margin(d, t1, N):
    dmin = min([abs(float(x)) for x in d if x != 0], default=np.inf)
    tm = max(float(t1), 1.0)
    lat = (2 * tm + (N + 1) / dmin) / 16777216.0
    return F(4.0 * (tm / 1048576.0 + lat + tm / 16777216.0))


def _estimate(o, d, inv_d, t0, t1, lo, hi):
    te = t1
    for i in range(3):
        if d[i] > 0:
            te = min(te, F(F(hi[i] - o[i]) * inv_d[i]))
        elif d[i] < 0:
            te = min(te, F(F(lo[i] - o[i]) * inv_d[i]))
    K = F(F(te - t0) - F(0.5))
    n = F(np.ceil(K))
    return n, F(n - K)


def _case(rng, N, B, mode):
    d = rng.normal(size=3)
    if rng.uniform() < 0.3:                     # near an axis or a face plane
        d[rng.integers(0, 3)] *= 10.0 ** rng.uniform(-6, -1)
    d = (d / np.linalg.norm(d)).astype(F)
    t0 = F(0.0)
    k = int(rng.integers(0, 4 * N))
    o = rng.uniform(0, N, 3).astype(F)
    if mode == "near_start":
        # the ray starts inside the grid and crosses a face of its first block at
        # t = K + 1/2 with K in (0, 1), mostly below 1/2
        i = int(np.argmax(np.abs(d)))
        k = 0
        K = rng.uniform(0.0, 0.5) if rng.uniform() < 0.75 else rng.uniform(0.5, 1.0)
        b = int(rng.integers(1, N // B - 1))
        face = b * B + (B if d[i] > 0 else 0)
        o[i] = F(face - (K + 0.5) * float(d[i]))
        for j in range(3):
            if j != i:
                o[j] = F(rng.uniform(B, N - B))
    elif mode == "adversarial":
        # put the crossing of one face of the block of sample k within 1e-3 of a lattice index
        i = int(np.argmax(np.abs(d)))
        kt = k + int(rng.integers(1, 3 * B))
        eps = rng.uniform(-1e-3, 1e-3)
        t_cross = kt + 0.5 + eps
        u_k = rng.uniform(B, N - B)
        face = np.floor(u_k / B) * B + (B if d[i] > 0 else 0)
        o[i] = F(face - t_cross * float(d[i]))
        for j in range(3):
            if j != i:
                o[j] = F(rng.uniform(B, N - B) - (k + 0.5) * float(d[j]))
    # the ray's extent in the grid [0, N]^3 (slabs), as the kernel clips it
    tn, tf = -np.inf, np.inf
    for i in range(3):
        if d[i] != 0:
            ta, tb = F(F(-o[i]) / d[i]), F(F(F(N) - o[i]) / d[i])
            tn, tf = max(tn, min(ta, tb)), min(tf, max(ta, tb))
        elif not (0 <= o[i] <= N):
            return None
    t0, t1 = F(max(tn, 0.0)), F(tf)
    if not t0 < t1:
        return None
    # the box: the block of sample k (or a one-sided box of blocks around it)
    t = _lattice_t(t0, k)
    if not t < t1:
        return None
    lo, hi = [0.0] * 3, [0.0] * 3
    D1 = int(rng.integers(0, 3)) if rng.uniform() < 0.5 else 0
    for i in range(3):
        u = F(o[i] + F(t * d[i]))
        b = min(max(int(np.floor(u)), 0), N - 1) // B
        bl, bh = (b - D1, b) if d[i] < 0 else (b, b + D1)
        L, H = bl * B, (bh + 1) * B
        lo[i] = -INF if L <= 0 else F(L)
        hi[i] = INF if H >= N else F(H)
    if not _in_box(o, d, t0, t1, k, lo, hi):
        return None
    return o, d, t0, t1, k, lo, hi


@pytest.mark.parametrize("N,B,n_cases,mode", [(64, 8, 1500, "random"), (256, 32, 1500, "random"),
                                              (1024, 32, 1500, "adversarial"), (2048, 32, 1000, "adversarial"),
                                              (1024, 32, 1500, "near_start")])
def test_unconfirmed_exit_matches_the_lattice(N, B, n_cases, mode):
    rng = np.random.default_rng(N + {"random": 0, "adversarial": 7, "near_start": 13}[mode])
    kmax = 4 * N + 16
    taken = checked = below_half = 0
    while checked < n_cases:
        c = _case(rng, N, B, mode)
        if c is None:
            continue
        o, d, t0, t1, k, lo, hi = c
        checked += 1
        inv_d = [_ulp_perturb(F(F(1.0) / d[i]), rng) if d[i] != 0 else INF for i in range(3)]
        n, fr = _estimate(o, d, inv_d, t0, t1, lo, hi)
        m = _exit_margin(d, t1, N)
        if not (n >= k + 1 and n < kmax and fr >= m and fr < 1 - m):
            continue
        taken += 1
        if mode == "near_start":
            below_half += bool(n == 1 and F(1) - fr < F(0.5))
        exact = k + 1
        while exact < kmax and _in_box(o, d, t0, t1, exact, lo, hi):
            exact += 1
        assert n == exact, (o, d, t0, t1, k, lo, hi, n, exact)
    assert taken > n_cases // 2          # the estimate is taken in most cases
    if mode == "near_start":
        assert below_half > n_cases // 4    # and often with a rounded fraction (K < 1/2)
