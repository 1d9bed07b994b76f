"""Pins of the oracle's bake (Sec. 5.3-5.4) to closed forms, invariants and a brute force
through an independent route (scipy's Gaussian density), on CPU.

The bake evaluates an analytic field that stands in for the trained network:
density = sum of isotropic Gaussian blobs (centre, std, peak), channel c (diffuse RGB and
4 features) = 0.5 + 0.5 sin(w_c . x + phi_c). Alpha = 1 - exp(-sigma v) at voxel centres;
macroblocks whose maximum alpha is below tau_alpha = 0.005 are culled; kept voxels average
16 samples at Gaussian offsets (std v / sqrt 12, here given in voxel units) and store
8-bit codes (density as sigma / sigma_max)."""
import math

import numpy as np
import pytest

import oracle

TAU = 0.005


def _quant(x):
    return np.clip(np.floor(np.asarray(x, np.float64) * 255.0 + 0.5), 0, 255).astype(np.int64)


def _near_boundary(x, eps=1e-6):
    f = np.asarray(x, np.float64) * 255.0
    return np.abs(f - np.floor(f) - 0.5) < eps * np.maximum(1.0, np.abs(f))


def _flat_blob(peak):
    # s = 1e4 world units over a grid of extent 2: the density varies by < 1e-7 relative.
    return np.array([[0.0, 0.0, 0.0, 1e4, peak]], np.float32)


def _still_colors(phis):
    c = np.zeros((7, 4), np.float32)
    c[:, 3] = phis
    return c


def test_bake_alpha_threshold_closed_form():
    """A constant density sigma: every block is kept iff 1 - exp(-sigma v) >= tau_alpha,
    i.e. sigma >= -ln(1 - tau_alpha) / v; kept blocks are numbered in raster order, and
    the density code is round(255 sigma / sigma_max)."""
    N, B, extent = 16, 4, 2.0
    v = extent / N
    s_tau = -math.log1p(-TAU) / v
    jit = np.zeros((16, 3), np.float32)
    sigma_max = s_tau * 1.001 * 255.0 / 100.2
    ind, atl, _ = oracle.bake(N, B, (-1, -1, -1), extent, sigma_max, _flat_blob(s_tau * 1.001), _still_colors(np.zeros(7)), jit)
    assert (ind.ravel() == np.arange(64)).all()
    assert (atl[..., 0] == 100).all()
    ind, atl, _ = oracle.bake(N, B, (-1, -1, -1), extent, sigma_max, _flat_blob(s_tau * 0.999), _still_colors(np.zeros(7)), jit)
    assert (ind == -1).all() and atl.shape[0] == 0


def test_bake_density_code_saturates():
    N, B = 8, 4
    ind, atl, _ = oracle.bake(N, B, (-1, -1, -1), 2.0, 10.0, _flat_blob(15.0), _still_colors(np.zeros(7)),
                              np.zeros((16, 3), np.float32))
    assert (ind >= 0).all() and (atl[..., 0] == 255).all()


def test_bake_constant_channels_in_channel_order():
    """w_c = 0: channel c is the constant 0.5 + 0.5 sin(phi_c), stored in atlas slot 1 + c
    (diffuse RGB, then the 4 features), whatever the jitter."""
    phis = np.array([math.pi / 6, -math.pi / 2, math.pi / 2, 0.0, 1.0, -2.0, 3.0], np.float32)
    jit = np.random.default_rng(1).normal(size=(16, 3)).astype(np.float32) / math.sqrt(12)
    ind, atl, _ = oracle.bake(8, 4, (-1, -1, -1), 2.0, 40.0, _flat_blob(30.0), _still_colors(phis), jit)
    want = _quant(0.5 + 0.5 * np.sin(phis.astype(np.float64)))
    assert want[0] == 191 and want[1] == 0 and want[2] == 255
    for c in range(7):
        assert (atl[..., 1 + c] == want[c]).all()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_bake_jitter_average_closed_form(axis):
    """Jitter offsets in +/- pairs and a channel varying along one axis only:
    mean over the pairs of sin(a + w j v) = sin(a) * mean cos(w j v), so the stored value
    is 0.5 + 0.5 sin(w x_centre + phi) * mean cos(w j_axis v). Pins the voxel centre (+1/2),
    the jitter scale (voxel units times v), the axis each offset moves along, the 16-sample
    average and the atlas layout [slot][z][y][x]."""
    N, B, extent = 16, 4, 2.0
    v = extent / N
    rng = np.random.default_rng(7 + axis)
    half = rng.normal(size=(8, 3)) / math.sqrt(12)
    jit = np.concatenate([half, -half]).astype(np.float32)
    w = 5.0
    colors = np.zeros((7, 4), np.float32)
    colors[0, axis] = w
    colors[0, 3] = 0.3
    bmin = np.array([-1.0, -0.75, -1.25], np.float32)
    ind, atl, _ = oracle.bake(N, B, bmin, extent, 40.0, _flat_blob(30.0), colors, jit)
    G = N // B
    assert (ind.ravel() == np.arange(G ** 3)).all()
    dense = atl[..., 1].reshape(G, G, G, B, B, B).transpose(0, 3, 1, 4, 2, 5).reshape(N, N, N)  # [z, y, x]
    jv = jit[:, axis].astype(np.float64)
    cmean = np.mean(np.cos(w * jv * v))
    i = np.arange(N)
    xc = float(bmin[axis]) + (i + 0.5) * v
    val = 0.5 + 0.5 * np.sin(w * xc + float(np.float32(0.3))) * cmean
    want = _quant(val)
    ok = ~_near_boundary(val)
    got = np.moveaxis(dense, 2 - axis, 0)           # the varying axis first
    assert ok.sum() >= N - 1
    for k in np.nonzero(ok)[0]:
        assert (got[k] == want[k]).all(), (axis, k)


def _scipy_sigma(blobs, pts):
    from scipy.stats import multivariate_normal
    acc = np.zeros(pts.shape[0])
    for c0, c1, c2, s, peak in blobs.astype(np.float64):
        norm = (2 * math.pi * s * s) ** 1.5
        acc += peak * norm * multivariate_normal(mean=[c0, c1, c2], cov=s * s * np.eye(3)).pdf(pts)
    return acc


def test_bake_brute_force_scipy_density():
    """Random blobs on a 16^3 grid of 4^3 blocks: the kept-block set (max alpha at voxel
    centres >= tau) and the density codes (16 jittered samples averaged) equal a brute force
    whose density comes from scipy's multivariate normal pdf; the colour channels of blocks
    never culled are in [0, 255] and the culled blocks' maxima are below tau."""
    pytest.importorskip("scipy")
    N, B, extent, sigma_max = 16, 4, 2.0, 60.0
    v = extent / N
    G = N // B
    rng = np.random.default_rng(11)
    blobs = np.zeros((5, 5), np.float32)
    blobs[:, :3] = rng.uniform(-0.7, 0.7, (5, 3))
    blobs[:, 3] = rng.uniform(0.08, 0.2, 5)
    blobs[:, 4] = rng.uniform(5, 40, 5)
    jit = (rng.normal(size=(16, 3)) / math.sqrt(12)).astype(np.float32)
    bmin = np.array([-1, -1, -1], np.float32)
    ind, atl, amax = oracle.bake(N, B, bmin, extent, sigma_max, blobs, np.zeros((7, 4), np.float32), jit)
    zz, yy, xx = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    centres = np.stack([xx, yy, zz], -1).reshape(-1, 3) + 0.5
    alpha = -np.expm1(-_scipy_sigma(blobs, -1.0 + centres * v) * v).reshape(N, N, N)
    bmax = alpha.reshape(G, B, G, B, G, B).max(axis=(1, 3, 5))
    np.testing.assert_allclose(amax, bmax, rtol=1e-9, atol=1e-15)
    assert 0 < (bmax >= TAU).sum() < G ** 3
    assert np.abs(bmax - TAU).min() > 1e-9
    assert ((ind >= 0) == (bmax >= TAU)).all()
    kept = np.argwhere(ind >= 0)                     # raster order (z, y, x)
    assert (ind[tuple(kept.T)] == np.arange(kept.shape[0])).all()
    sig = np.zeros(N ** 3)
    for j in jit.astype(np.float64):
        sig += _scipy_sigma(blobs, -1.0 + (centres + j) * v)
    sig = (sig / 16.0 / np.float32(sigma_max)).reshape(N, N, N)
    for slot, (bz, by, bx) in enumerate(kept):
        ref = sig[bz * B:(bz + 1) * B, by * B:(by + 1) * B, bx * B:(bx + 1) * B]
        ok = ~_near_boundary(ref)
        assert ok.mean() > 0.99
        assert (atl[slot, ..., 0][ok] == _quant(ref)[ok]).all()
    assert (atl[..., 1:] == 128).all()               # w = 0, phi = 0: 0.5 -> round(127.5) = 128


def test_bake_max_blocks_overflow_raises():
    with pytest.raises(oracle.OracleError):
        oracle.bake(8, 4, (-1, -1, -1), 2.0, 40.0, _flat_blob(30.0), _still_colors(np.zeros(7)),
                    np.zeros((16, 3), np.float32), max_blocks=3)


def test_bake_blocks_agrees_with_whole_bake():
    """The per-block entry (used for sampled checks of large bakes) returns the whole
    bake's block maxima and, for kept blocks, its atlas content; its raw values round to
    the stored codes."""
    N, B = 32, 8
    rng = np.random.default_rng(5)
    blobs = np.zeros((6, 5), np.float32)
    blobs[:, :3] = rng.uniform(-0.6, 0.6, (6, 3))
    blobs[:, 3] = rng.uniform(0.05, 0.2, 6)
    blobs[:, 4] = rng.uniform(5, 40, 6)
    colors = np.zeros((7, 4), np.float32)
    colors[:, :3] = rng.uniform(-6, 6, (7, 3))
    colors[:, 3] = rng.uniform(0, 6.28, 7)
    jit = (rng.normal(size=(16, 3)) / math.sqrt(12)).astype(np.float32)
    ind, atl, amax = oracle.bake(N, B, (-1, -1, -1), 2.0, 50.0, blobs, colors, jit)
    blocks = np.arange((N // B) ** 3)
    a2, content, raw = oracle.bake_blocks(N, B, (-1, -1, -1), 2.0, 50.0, blobs, colors, jit, blocks)
    np.testing.assert_array_equal(a2, amax.ravel())
    kept = ind.ravel() >= 0
    np.testing.assert_array_equal(content[kept], atl[ind.ravel()[kept]])
    np.testing.assert_array_equal(content, _quant(raw / 255.0))


def test_bake_alpha_codes_closed_form():
    """With alpha codes, a constant density sigma stores round(255 (1 - exp(-sigma v))) in
    channel 0 (the viewer's alpha texture, App. A); the culling and the other channels are
    unchanged."""
    N, B, extent = 16, 4, 2.0
    v = extent / N
    jit = np.random.default_rng(3).normal(size=(16, 3)).astype(np.float32) / math.sqrt(12)
    args = (N, B, (-1, -1, -1), extent, 40.0, _flat_blob(3.0), _still_colors(np.full(7, 0.7)), jit)
    ind_s, atl_s, _ = oracle.bake(*args)
    ind_a, atl_a, _ = oracle.bake(*args, alpha_codes=True)
    want = int(math.floor(255.0 * -math.expm1(-3.0 * v) + 0.5))
    assert want == 80
    assert (atl_a[..., 0] == want).all()
    np.testing.assert_array_equal(ind_a, ind_s)
    np.testing.assert_array_equal(atl_a[..., 1:], atl_s[..., 1:])
