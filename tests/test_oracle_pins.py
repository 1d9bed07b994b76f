"""Pins for the FP64 oracle against facts the paper and the mathematics fix.

None of these retypes the oracle: each checks a closed form (uniform slab, two-sample
ray, early-exit count), an invariant (weights sum to 1 - T, slot permutation,
zero-density blocks), a library routine (torch float64 linear layers, scipy trilinear
interpolation) or a brute-force evaluation on a tiny grid. A plausible mistake in the
oracle (dropped transmittance factor, wrong alpha sign, transposed weight, off-by-one
in the sample lattice, wrong trilinear corner) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2103_14645_gb300 import synth
from tests import helpers

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pix(scene, cam=0):
    return synth.all_pixels(scene.cameras[cam:cam + 1])


# --------------------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------------------

def test_empty_grid_returns_background():
    """No occupied block: every ray returns the background exactly (Eq. 2 with no samples)."""
    sc = synth.make_scene("tiny")
    sc.ind[:] = -1
    out = oracle.render_rays(sc, _pix(sc), trace_cap=4)
    assert np.array_equal(out["rgb"], np.tile(np.asarray(sc.bg), (out["rgb"].shape[0], 1)))
    assert (out["counts"] == 0).all()
    assert (out["aux"] == 0).all()


def test_uniform_slab_transmittance():
    """Axis ray through M voxels of uniform density: T = exp(-sigma L), C_d = c (1 - T)."""
    q = 200
    col = np.array([100, 150, 200, 10, 20, 30, 40])
    sc = helpers.slab_scene(z_range=(4, 6), q=q, color=col, sigma_max_vox=1.0)
    out = oracle.render_rays(sc, np.array([[0, 0, 0]]), trace_cap=8)
    sigma_delta = q / 255.0 * 1.0
    T = math.exp(-2 * sigma_delta)
    cd = col[:3] / 255.0 * (1 - T)
    v = col[3:] / 255.0 * (1 - T)
    np.testing.assert_allclose(out["aux"][0, :3], cd, rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["aux"][0, 3:7], v, rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["aux"][0, 7], 1 - T, rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["rgb"][0], cd + T * np.asarray(sc.bg), rtol=0, atol=1e-14)
    # the ray enters block row bz=1 (z in [4,8)) at u_z = 7.5: 4 samples there, 2 composited
    assert out["counts"][0].tolist() == [4, 2]
    N = sc.N
    assert out["trace"][0, :2].tolist() == [(5 * N + 5) * N + 5, (4 * N + 5) * N + 5]


def test_two_sample_ray_by_hand():
    """Two voxels of different density along the ray: w1 = 1 - e^-a, w2 = e^-a (1 - e^-b)."""
    col = np.array([255, 0, 51, 0, 0, 0, 255])
    sc = helpers.slab_scene(z_range=(4, 6), per_voxel_q=(51, 204), color=col, sigma_max_vox=2.0)
    out = oracle.render_rays(sc, np.array([[0, 0, 0]]))
    a = 204 / 255.0 * 2.0    # voxel z=5 is met first (the ray travels towards -z)
    b = 51 / 255.0 * 2.0
    w1 = 1 - math.exp(-a)
    w2 = math.exp(-a) * (1 - math.exp(-b))
    T = math.exp(-a - b)
    expect = np.array([w1 + w2, 0.0, 0.2 * (w1 + w2)]) + T * 1.0
    np.testing.assert_allclose(out["rgb"][0], expect, rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["aux"][0, 6], w1 + w2, rtol=0, atol=1e-14)


def test_early_exit_after_crossing_sample():
    """Opaque slab with sigma*delta = 1 per sample: marching stops after the first sample
    where the optical depth exceeds ln(1000), i.e. after floor(ln 1000) + 1 = 7 samples."""
    sc = helpers.slab_scene(z_range=(2, 14), q=255, sigma_max_vox=1.0)
    out = oracle.render_rays(sc, np.array([[0, 0, 0]]), trace_cap=16)
    n_active = math.floor(math.log(1000.0)) + 1
    assert out["counts"][0, 1] == n_active
    # block row bz=3 (z 12..15) is entered at u_z=15.5: 2 non-composited samples first
    assert out["counts"][0, 0] == 2 + n_active
    np.testing.assert_allclose(1 - out["aux"][0, 7], math.exp(-n_active), rtol=1e-12)


def test_zero_weights_residual_is_half():
    """W = 0, b = 0: sigmoid(0) = 1/2 is added only where a sample was composited."""
    sc = synth.make_scene("tiny")
    w = np.zeros(synth.MLP_NPARAM, np.float32)
    out = oracle.render_rays(sc, _pix(sc), mlp=w)
    act = out["counts"][:, 1] > 0
    assert act.any() and (~act).any()
    T = 1 - out["aux"][:, 7]
    np.testing.assert_allclose(out["rgb"][act], out["aux"][act, :3] + 0.5 + T[act, None], atol=1e-14)
    np.testing.assert_array_equal(out["rgb"][~act], np.ones(((~act).sum(), 3)))


def test_saturated_bias_gives_diffuse_plus_background():
    sc = synth.make_scene("tiny")
    out = oracle.render_rays(sc, _pix(sc), mlp=helpers.silent_mlp())
    T = 1 - out["aux"][:, 7]
    np.testing.assert_allclose(out["rgb"], out["aux"][:, :3] + T[:, None] * 1.0, rtol=0, atol=1e-14)


# --------------------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------------------

def test_weights_sum_to_opacity():
    """Sum_k w_k = 1 - T_final <= 1: with every block stored and every colour value 1,
    C_d equals the opacity (corners in empty blocks would read 0)."""
    sc0 = synth.make_scene("gauss64")
    ind, atlas = helpers.dense_to_blocks(helpers.blocks_to_dense(sc0), sc0.B, keep_empty=True)
    sc = synth.custom_scene(sc0.N, sc0.B, ind, atlas, sc0.sigma_max, sc0.mlp, sc0.cameras)
    val = np.ones(sc.atlas.shape, np.float64)
    out = oracle.render_rays(sc, _pix(sc), val=val)
    acc = out["aux"][:, 7]
    assert (acc >= 0).all() and (acc <= 1).all()
    for c in range(7):
        np.testing.assert_allclose(out["aux"][:, c], acc, rtol=0, atol=1e-12)
    assert (out["counts"][:, 1] > 0).mean() > 0.3


def test_colours_bounded_by_opacity():
    sc = synth.make_scene("gauss64")
    out = oracle.render_rays(sc, _pix(sc))
    acc = out["aux"][:, 7]
    assert (out["aux"][:, :7] <= acc[:, None] + 1e-12).all()
    assert (out["aux"][:, :7] >= 0).all()


def test_atlas_slot_permutation_invariance():
    """The indirection grid is the only link from space to atlas slots (Sec. 5.1)."""
    sc = synth.make_scene("tiny")
    ref = oracle.render_rays(sc, _pix(sc), trace_cap=64)
    perm = np.random.default_rng(3).permutation(sc.nb)
    inv = np.argsort(perm)
    sc2 = synth.custom_scene(sc.N, sc.B, np.where(sc.ind >= 0, inv[np.maximum(sc.ind, 0)], -1),
                             sc.atlas[perm], sc.sigma_max, sc.mlp, sc.cameras)
    out = oracle.render_rays(sc2, _pix(sc2), trace_cap=64)
    for k in ("rgb", "aux", "counts", "trace"):
        assert np.array_equal(ref[k], out[k]), k


def test_zero_density_blocks_equal_empty_blocks():
    """Storing an all-zero block changes the step count only, never the image."""
    sc = synth.make_scene("tiny")
    dense = helpers.blocks_to_dense(sc)
    ind_all, atlas_all = helpers.dense_to_blocks(dense, sc.B, keep_empty=True)
    # stored-but-zero blocks must also have zero colour to match "empty reads 0"
    sc_all = synth.custom_scene(sc.N, sc.B, ind_all, atlas_all, sc.sigma_max, sc.mlp, sc.cameras)
    a = oracle.render_rays(sc, _pix(sc), trace_cap=64)
    b = oracle.render_rays(sc_all, _pix(sc_all), trace_cap=64)
    assert np.array_equal(a["rgb"], b["rgb"])
    assert np.array_equal(a["trace"], b["trace"])
    assert np.array_equal(a["counts"][:, 1], b["counts"][:, 1])
    assert (b["counts"][:, 0] >= a["counts"][:, 0]).all() and (b["counts"][:, 0] > a["counts"][:, 0]).any()


# --------------------------------------------------------------------------------------
# library routines
# --------------------------------------------------------------------------------------

def _torch_mlp(w, x):
    w = torch.as_tensor(np.asarray(w, np.float64))
    x = torch.as_tensor(np.asarray(x, np.float64))
    o = 0
    W1 = w[o:o + 16 * 34].reshape(16, 34); o += 16 * 34
    b1 = w[o:o + 16]; o += 16
    W2 = w[o:o + 256].reshape(16, 16); o += 256
    b2 = w[o:o + 16]; o += 16
    W3 = w[o:o + 48].reshape(3, 16); o += 48
    b3 = w[o:o + 3]
    F = torch.nn.functional
    h = F.relu(F.linear(x, W1, b1))
    h = F.relu(F.linear(h, W2, b2))
    return torch.sigmoid(F.linear(h, W3, b3)).numpy()


def test_mlp_matches_torch_float64():
    rng = np.random.default_rng(11)
    w = rng.normal(size=synth.MLP_NPARAM)
    x = rng.normal(size=(257, 34))
    np.testing.assert_allclose(oracle.mlp_eval(w, x), _torch_mlp(w, x), rtol=0, atol=1e-14)


def test_mlp_input_layout():
    """Input = [C_d(3), V(4), d(3), sin(2^l d)(3), cos(2^l d)(3) for l = 0..3] (34)."""
    rng = np.random.default_rng(12)
    cd, v = rng.uniform(size=3), rng.uniform(size=4)
    d = rng.normal(size=3).astype(np.float32)
    d /= np.linalg.norm(d)
    x = oracle.mlp_input(cd, v, d)
    dd = d.astype(np.float64)
    ref = [cd, v, dd]
    for l in range(4):
        ref += [np.sin(2.0 ** l * dd), np.cos(2.0 ** l * dd)]
    np.testing.assert_allclose(x, np.concatenate(ref), rtol=0, atol=1e-15)


def _brute_force_ray(scene, dense, mlp, cam, px, py, unpremultiply=False, alpha_atlas=False, no_mlp=False):
    """Definition of the march evaluated by library routines on a dense grid:
    trilinear by scipy.ndimage.map_coordinates (order 1, clamp-to-edge), transmittance
    by a running product, MLP by torch float64 linear layers. With alpha_atlas, channel 0
    is alpha: a = trilinear / 255, T <- T (1 - a), stop once T < 1e-3."""
    from scipy.ndimage import map_coordinates
    N, B = scene.N, scene.B
    hit, o, d, ts, te = oracle.ray(scene, cam, px, py)
    dens = dense[..., 0].astype(np.float64)
    chans = [dense[..., c].astype(np.float64) / 255.0 for c in range(1, 8)]
    occ = scene.ind >= 0
    delta = float(np.float32(scene.extent)) / N
    sigma_max = float(np.float32(scene.sigma_max))     # the scene description is binary32
    T, feat, steps, visited, tau = 1.0, np.zeros(7), 0, [], 0.0
    k = 0
    while hit:
        tk = np.float32(ts) + (np.float32(k) + np.float32(0.5))
        k += 1
        if not tk < np.float32(te):
            break
        u = np.asarray(o, np.float32) + np.float32(tk) * np.asarray(d, np.float32)
        j = np.clip(np.floor(u).astype(np.int64), 0, N - 1)
        if not occ[j[2] // B, j[1] // B, j[0] // B]:
            continue
        steps += 1
        if dense[j[2], j[1], j[0], 0] == 0:
            continue
        visited.append(int((j[2] * N + j[1]) * N + j[0]))
        coord = (np.asarray(u[::-1], np.float64) - 0.5).reshape(3, 1)
        s = map_coordinates(dens, coord, order=1, mode="nearest")[0]
        sd = s / 255.0 * sigma_max * delta
        a = s / 255.0 if alpha_atlas else 1 - math.exp(-sd)
        w = T * a
        for c in range(7):
            feat[c] += w * map_coordinates(chans[c], coord, order=1, mode="nearest")[0]
        T *= 1 - a if alpha_atlas else math.exp(-sd)
        tau += sd
        if (T < 1e-3) if alpha_atlas else (tau > math.log(1000.0)):
            break
    raw = feat.copy()
    if unpremultiply and 1 - T > 0:
        a = 1 - T
        sc = min(1.0, 1.5 * a) / a
        feat = feat * sc
        T = 1 - min(1.0, 1.5 * a)
    rgb = np.asarray(scene.bg) * T
    if visited and no_mlp:
        rgb = rgb + feat[:3]
    elif visited:
        dd = np.asarray(d, np.float64)
        pe = [feat[:3], feat[3:], dd]
        for l in range(4):
            pe += [np.sin(2.0 ** l * dd), np.cos(2.0 ** l * dd)]
        rgb = rgb + feat[:3] + _torch_mlp(mlp, np.concatenate(pe)[None])[0]
    return rgb, raw, steps, visited


@pytest.mark.parametrize("name,unpremultiply,alpha", [("tiny", False, False), ("gauss64", False, False),
                                                       ("gauss64", True, False), ("tiny", False, True),
                                                       ("gauss64", False, True), ("gauss64", True, True)])
def test_brute_force_dense_grid(name, unpremultiply, alpha):
    sc = synth.make_scene(name)
    sc.flags = (1 if unpremultiply else 0) | (4 if alpha else 0)
    dense = helpers.blocks_to_dense(sc)
    rng = np.random.default_rng(5)
    W, H = int(sc.cameras[0]["W"]), int(sc.cameras[0]["H"])
    pix = np.stack([np.zeros(60, int), rng.integers(0, W, 60), rng.integers(0, H, 60)], 1)
    out = oracle.render_rays(sc, pix, trace_cap=256)
    n_active_rays = 0
    for i, (c, x, y) in enumerate(pix):
        rgb, feat, steps, visited = _brute_force_ray(sc, dense, sc.mlp, sc.cameras[c], x, y, unpremultiply, alpha)
        np.testing.assert_allclose(out["rgb"][i], rgb, rtol=0, atol=1e-10)
        np.testing.assert_allclose(out["aux"][i, :7], feat, rtol=0, atol=1e-10)
        assert out["counts"][i, 0] == steps
        assert out["counts"][i, 1] == len(visited)
        assert out["trace"][i, :len(visited)].tolist() == visited
        n_active_rays += bool(visited)
    assert n_active_rays >= 10


# --------------------------------------------------------------------------------------
# ray geometry (pinhole, Sec. 4.1 r(t) = o + t d)
# --------------------------------------------------------------------------------------

def test_ray_geometry_pinhole():
    sc = synth.make_scene("gauss64")
    rng = np.random.default_rng(9)
    cams = synth.orbit_cameras(rng, [(65, 47)] * 6, synth.CAM_RADIUS)
    s = sc.N / sc.extent
    for cam in cams:
        c2w = np.asarray(cam["c2w"], np.float64).reshape(3, 4)
        for _ in range(20):
            px, py = int(rng.integers(0, 65)), int(rng.integers(0, 47))
            hit, o, d, ts, te = oracle.ray(sc, cam, px, py)
            xs = (px + 0.5 - cam["cx"]) / cam["fx"]
            ys = (py + 0.5 - cam["cy"]) / cam["fy"]
            assert abs(np.linalg.norm(d.astype(np.float64)) - 1) < 1e-6
            ang = math.acos(float(np.clip(-(d.astype(np.float64) @ c2w[:, 2]), -1, 1)))
            assert abs(ang - math.atan(math.hypot(xs, ys))) < 1e-5
            np.testing.assert_allclose(o, (c2w[:, 3] - np.asarray(sc.bmin)) * s, atol=1e-4)
            if hit:
                for t, name in ((ts, "start"), (te, "end")):
                    p = o.astype(np.float64) + t * d.astype(np.float64)
                    assert (p > -1e-3).all() and (p < sc.N + 1e-3).all(), name
                pe = o.astype(np.float64) + te * d.astype(np.float64)
                on_face = np.minimum(np.abs(pe), np.abs(pe - sc.N)).min()
                assert on_face < 1e-3


def test_principal_ray_hits_look_at_target():
    """Odd image width/height: the centre pixel looks straight at the target (origin)."""
    sc = synth.make_scene("gauss64")
    cam = synth.look_at_camera((1.3, -1.1, 0.9), (0.0, 0.0, 0.0), 65, 33, 39.0)
    hit, o, d, ts, te = oracle.ray(sc, cam, 32, 16)
    centre = (np.zeros(3) - np.asarray(sc.bmin)) * sc.N / sc.extent
    rel = centre - o.astype(np.float64)
    dist = np.linalg.norm(rel - (rel @ d) * d.astype(np.float64))
    assert dist < 1e-3
    # image y grows downwards: the top row looks further up (+z) than the bottom row
    _, _, d_top, _, _ = oracle.ray(sc, cam, 32, 0)
    _, _, d_bot, _, _ = oracle.ray(sc, cam, 32, 32)
    assert d_top[2] > d[2] > d_bot[2]


# --------------------------------------------------------------------------------------
# gradient (adjoint of the render w.r.t. colour/feature values and MLP weights)
# --------------------------------------------------------------------------------------

def _loss(sc, pix, target, val=None, mlp=None):
    out = oracle.render_rays(sc, pix, val=val, mlp=mlp)
    return 0.5 * ((out["rgb"] - target) ** 2).sum(), out


def test_gradient_matches_central_differences():
    sc = synth.make_scene("tiny")
    rng = np.random.default_rng(21)
    pix = _pix(sc)
    target = rng.uniform(size=(pix.shape[0], 3))
    val = sc.atlas.astype(np.float64) / 255.0
    mlp = sc.mlp.astype(np.float64)
    L0, out = _loss(sc, pix, target, val, mlp)
    gval, gmlp = oracle.backward_rays(sc, pix, out["rgb"] - target, val=val, mlp=mlp)
    assert (gval[..., 0] == 0).all()
    h = 1e-6
    flat = gval.reshape(-1)
    nz = np.nonzero(np.abs(flat) > 1e-6)[0]
    nz = nz[nz % 8 != 0]
    picks = list(rng.choice(nz, 24, replace=False)) + list(rng.choice(flat.size, 8, replace=False))
    for idx in picks:
        vp, vm = val.copy().reshape(-1), val.copy().reshape(-1)
        vp[idx] += h
        vm[idx] -= h
        fd = (_loss(sc, pix, target, vp.reshape(val.shape), mlp)[0] -
              _loss(sc, pix, target, vm.reshape(val.shape), mlp)[0]) / (2 * h)
        if idx % 8 == 0:
            continue      # density is frozen: the oracle reports no gradient for it
        assert abs(fd - flat[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, flat[idx])
    for p in rng.choice(synth.MLP_NPARAM, 32, replace=False):
        mp, mm = mlp.copy(), mlp.copy()
        mp[p] += h
        mm[p] -= h
        fd = (_loss(sc, pix, target, val, mp)[0] - _loss(sc, pix, target, val, mm)[0]) / (2 * h)
        assert abs(fd - gmlp[p]) <= 1e-6 * max(1.0, abs(fd)), (p, fd, gmlp[p])


def test_gradient_sum_equals_opacity_when_linear():
    """Silent MLP and every block stored: C = C_d + T bg is linear in the colours, and the
    red-channel gradient summed over all voxels equals the summed opacity (the trilinear
    weights of each sample sum to one, and the composite weights to 1 - T)."""
    sc = synth.make_scene("tiny")
    dense = helpers.blocks_to_dense(sc)
    ind, atlas = helpers.dense_to_blocks(dense, sc.B, keep_empty=True)
    sc2 = synth.custom_scene(sc.N, sc.B, ind, atlas, sc.sigma_max, helpers.silent_mlp(), sc.cameras)
    pix = _pix(sc2)
    out = oracle.render_rays(sc2, pix)
    g = np.zeros((pix.shape[0], 3))
    g[:, 0] = 1.0
    gval, gmlp = oracle.backward_rays(sc2, pix, g)
    np.testing.assert_allclose(gval[..., 1].sum(), out["aux"][:, 7].sum(), rtol=1e-12)
    assert np.abs(gval[..., 2:]).max() == 0.0
    assert np.abs(gmlp).max() == 0.0      # sigmoid'(-1e4) underflows to exactly 0


# --------------------------------------------------------------------------------------
# constants the paper prints
# --------------------------------------------------------------------------------------

def test_paper_constants():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        g = json.load(f)
    assert synth.TAU_ALPHA == g["tau_alpha"]["value"]
    assert synth.MLP_HID == g["view_mlp_width"]["value"]
    assert len([s for s in synth.MLP_SIZES if len(s) == 2]) - 1 == g["view_mlp_hidden_layers"]["value"]
    # 8 channels of 8 bits at 8 trilinear corners = the 64 bytes per sample of App. A
    assert 8 * 8 == g["bytes_per_trilinear_sample"]["value"]
    assert synth.make_scene("shell1024").B == g["macroblock_edge"]["value"]
    assert synth.MLP_IN - 7 == 3 + 3 * 2 * 4    # direction + 4 octaves of sin/cos



# --------------------------------------------------------------------------------------
# partial un-premultiply (App. C): (C_d, alpha, V) *= min(1, 1.5 alpha) / alpha
# --------------------------------------------------------------------------------------

def test_unpremultiply_slab_closed_form():
    col = np.array([100, 150, 200, 10, 20, 30, 40])
    sc = helpers.slab_scene(z_range=(4, 6), q=60, color=col, sigma_max_vox=1.0)
    sc.flags = 1
    out = oracle.render_rays(sc, np.array([[0, 0, 0]]))
    T = math.exp(-2 * 60 / 255.0)
    a = 1 - T
    a2 = min(1.0, 1.5 * a)
    assert a2 < 1.0                                   # the soft-edge branch
    cd = col[:3] / 255.0 * a * (a2 / a)
    np.testing.assert_allclose(out["rgb"][0], cd + (1 - a2) * np.asarray(sc.bg), rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["aux"][0, 7], a, rtol=0, atol=1e-14)     # aux keeps the raw opacity


def test_unpremultiply_saturates_to_the_surface_colour():
    """Opacity above 2/3 is fully saturated: a uniform slab then shows exactly its own
    colour and no background."""
    col = np.array([100, 150, 200, 10, 20, 30, 40])
    sc = helpers.slab_scene(z_range=(4, 6), q=255, color=col, sigma_max_vox=1.0)
    sc.flags = 1
    out = oracle.render_rays(sc, np.array([[0, 0, 0]]))
    assert 1 - math.exp(-2.0) > 2.0 / 3.0
    np.testing.assert_allclose(out["rgb"][0], col[:3] / 255.0, rtol=0, atol=1e-14)


def test_unpremultiply_gradient_matches_central_differences():
    sc = synth.make_scene("tiny")
    sc.flags = 1
    rng = np.random.default_rng(22)
    pix = _pix(sc)
    target = rng.uniform(size=(pix.shape[0], 3))
    val = sc.atlas.astype(np.float64) / 255.0
    mlp = sc.mlp.astype(np.float64)
    L0, out = _loss(sc, pix, target, val, mlp)
    gval, gmlp = oracle.backward_rays(sc, pix, out["rgb"] - target, val=val, mlp=mlp)
    h = 1e-6
    flat = gval.reshape(-1)
    nz = np.nonzero(np.abs(flat) > 1e-6)[0]
    nz = nz[nz % 8 != 0]
    for idx in rng.choice(nz, 16, replace=False):
        vp, vm = val.copy().reshape(-1), val.copy().reshape(-1)
        vp[idx] += h
        vm[idx] -= h
        fd = (_loss(sc, pix, target, vp.reshape(val.shape), mlp)[0] -
              _loss(sc, pix, target, vm.reshape(val.shape), mlp)[0]) / (2 * h)
        assert abs(fd - flat[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, flat[idx])
    for p in rng.choice(synth.MLP_NPARAM, 16, replace=False):
        mp, mm = mlp.copy(), mlp.copy()
        mp[p] += h
        mm[p] -= h
        fd = (_loss(sc, pix, target, val, mp)[0] - _loss(sc, pix, target, val, mm)[0]) / (2 * h)
        assert abs(fd - gmlp[p]) <= 1e-6 * max(1.0, abs(fd)), (p, fd, gmlp[p])


def test_reference_adam_matches_torch():
    """The FP64 reference Adam against torch.optim.Adam (library routine)."""
    rng = np.random.default_rng(31)
    p0 = rng.normal(size=50)
    grads = rng.normal(size=(6, 50)) * np.logspace(-4, 1, 50)
    w = p0.copy()
    m = np.zeros(50)
    v = np.zeros(50)
    t = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=3e-4, betas=(0.9, 0.999), eps=1e-8)
    for k in range(6):
        oracle.adam_step(w, m, v, grads[k], k + 1)
        opt.zero_grad()
        t.grad = torch.tensor(grads[k])
        opt.step()
    np.testing.assert_allclose(w, t.detach().numpy(), rtol=0, atol=1e-12)



# --------------------------------------------------------------------------------------
# non-deferred comparison model (the per-sample ablation): the MLP at every composited
# sample on that sample's own (c_d, v)
# --------------------------------------------------------------------------------------

PER_SAMPLE = 2


def test_per_sample_zero_weights_give_half_the_opacity():
    """W = 0, b = 0: every composited sample adds 1/2 * w_k, so C = C_d + acc/2 + T bg
    (the deferred model adds 1/2 once: C_d + 1/2 + T bg)."""
    sc = synth.make_scene("tiny")
    sc.flags = PER_SAMPLE
    out = oracle.render_rays(sc, _pix(sc), mlp=np.zeros(synth.MLP_NPARAM, np.float32))
    acc = out["aux"][:, 7]
    np.testing.assert_allclose(out["rgb"], out["aux"][:, :3] + 0.5 * acc[:, None] + (1 - acc)[:, None],
                               rtol=0, atol=1e-14)
    assert (acc > 0.05).any()


def test_per_sample_silent_mlp_equals_deferred():
    sc = synth.make_scene("tiny")
    a = oracle.render_rays(sc, _pix(sc), mlp=helpers.silent_mlp())
    sc.flags = PER_SAMPLE
    b = oracle.render_rays(sc, _pix(sc), mlp=helpers.silent_mlp())
    np.testing.assert_allclose(b["rgb"], a["rgb"], rtol=0, atol=1e-14)


def test_per_sample_uniform_slab_closed_form():
    """A uniform slab: every sample has the same input, so C = (c + r)(1 - T) + T bg with
    r = sigmoid(MLP(c, v, PE(d))) from torch float64 linear layers."""
    col = np.array([100, 150, 200, 10, 20, 30, 40])
    rng = np.random.default_rng(41)
    w = synth.init_mlp(rng)
    sc = helpers.slab_scene(z_range=(4, 6), q=200, color=col, sigma_max_vox=1.0, mlp=w)
    sc.flags = PER_SAMPLE
    out = oracle.render_rays(sc, np.array([[0, 0, 0]]))
    T = math.exp(-2 * 200 / 255.0)
    d = np.array([0.0, 0.0, -1.0])
    pe = [col[:3] / 255.0, col[3:] / 255.0, d]
    for l in range(4):
        pe += [np.sin(2.0 ** l * d), np.cos(2.0 ** l * d)]
    res = _torch_mlp(w, np.concatenate(pe)[None])[0]
    np.testing.assert_allclose(out["rgb"][0], (col[:3] / 255.0 + res) * (1 - T) + T, rtol=0, atol=1e-13)


def test_per_sample_brute_force():
    sc = synth.make_scene("tiny")
    sc.flags = PER_SAMPLE
    dense = helpers.blocks_to_dense(sc)
    from scipy.ndimage import map_coordinates
    rng = np.random.default_rng(6)
    pix = np.stack([np.zeros(40, int), rng.integers(0, 24, 40), rng.integers(0, 20, 40)], 1)
    out = oracle.render_rays(sc, pix)
    N, B = sc.N, sc.B
    chans = [dense[..., c].astype(np.float64) / 255.0 for c in range(8)]
    sigma_max = float(np.float32(sc.sigma_max))
    delta = float(np.float32(sc.extent)) / N
    for i, (c, x, y) in enumerate(pix):
        hit, o, d, ts, te = oracle.ray(sc, sc.cameras[c], x, y)
        T, tau, rgb, k = 1.0, 0.0, np.zeros(3), 0
        while hit:
            tk = np.float32(ts) + (np.float32(k) + np.float32(0.5))
            k += 1
            if not tk < np.float32(te):
                break
            u = np.asarray(o, np.float32) + np.float32(tk) * np.asarray(d, np.float32)
            j = np.clip(np.floor(u).astype(np.int64), 0, N - 1)
            if sc.ind[j[2] // B, j[1] // B, j[0] // B] < 0 or dense[j[2], j[1], j[0], 0] == 0:
                continue
            coord = (np.asarray(u[::-1], np.float64) - 0.5).reshape(3, 1)
            v = [map_coordinates(ch, coord, order=1, mode="nearest")[0] for ch in chans]
            sd = v[0] * sigma_max * delta
            wk = T * (1 - math.exp(-sd))
            dd = np.asarray(d, np.float64)
            pe = [np.array(v[1:4]), np.array(v[4:8]), dd]
            for l in range(4):
                pe += [np.sin(2.0 ** l * dd), np.cos(2.0 ** l * dd)]
            rgb += wk * (np.array(v[1:4]) + _torch_mlp(sc.mlp, np.concatenate(pe)[None])[0])
            T *= math.exp(-sd)
            tau += sd
            if tau > math.log(1000.0):
                break
        np.testing.assert_allclose(out["rgb"][i], rgb + T * np.asarray(sc.bg), rtol=0, atol=1e-10)


# --------------------------------------------------------------------------------------
# alpha atlas (App. A keeps alpha in its own texture): channel 0 = alpha codes
# --------------------------------------------------------------------------------------

def test_alpha_atlas_slab_closed_form():
    """Uniform slab of alpha code q: every sample has alpha = q / 255, so after n samples
    T = (1 - alpha)^n and C_d = c (1 - T); the march stops after the first sample with
    T < 1e-3 (n = 10 for q = 128: 0.498^9 = 1.9e-3, 0.498^10 = 9.5e-4)."""
    col = np.array([100, 150, 200, 10, 20, 30, 40])
    sc = helpers.slab_scene(z_range=(2, 14), q=128, color=col, sigma_max_vox=1.0)
    sc.flags = 4
    out = oracle.render_rays(sc, np.array([[0, 0, 0]]), trace_cap=16)
    a = 128 / 255.0
    n = 10
    assert (1 - a) ** (n - 1) >= 1e-3 > (1 - a) ** n
    assert out["counts"][0, 1] == n
    assert out["counts"][0, 0] == 2 + n      # 2 samples of block row z 12..15 before the slab
    T = (1 - a) ** n
    np.testing.assert_allclose(out["aux"][0, :3], col[:3] / 255.0 * (1 - T), rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["aux"][0, 7], 1 - T, rtol=0, atol=1e-14)


def test_alpha_atlas_equals_density_atlas_at_matched_alpha():
    """A density code q_s with sigma_max chosen so that 1 - exp(-q_s/255 sigma_max delta)
    equals q_a / 255 composites like the alpha code q_a: same counts, and the same colours
    up to the binary32 rounding of sigma_max in the scene description (~1e-8)."""
    col = np.array([90, 30, 220, 40, 50, 60, 70])
    qa, qs = 77, 200
    a = qa / 255.0
    smax_vox = -math.log1p(-a) * 255.0 / qs
    dens = helpers.slab_scene(z_range=(3, 12), q=qs, color=col, sigma_max_vox=smax_vox)
    alph = helpers.slab_scene(z_range=(3, 12), q=qa, color=col, sigma_max_vox=smax_vox)
    alph.flags = 4
    pix = np.array([[0, 0, 0]])
    o1 = oracle.render_rays(dens, pix)
    o2 = oracle.render_rays(alph, pix)
    np.testing.assert_allclose(o2["rgb"], o1["rgb"], rtol=0, atol=1e-7)
    np.testing.assert_allclose(o2["aux"], o1["aux"], rtol=0, atol=1e-7)
    np.testing.assert_array_equal(o2["counts"], o1["counts"])
    assert o1["counts"][0, 1] == 9


def test_alpha_atlas_gradient_matches_central_differences():
    sc = synth.make_scene("tiny")
    sc.flags = 4
    pix = _pix(sc)[::2]
    rng = np.random.default_rng(12)
    target = rng.uniform(size=(pix.shape[0], 3))
    val = sc.atlas.astype(np.float64) / 255.0
    g_val, g_mlp = oracle.backward_rays(sc, pix, oracle.render_rays(sc, pix, val=val)["rgb"] - target, val=val)
    occupied = np.argwhere(np.abs(g_val[..., 1:]) > 1e-3)
    assert occupied.shape[0] > 10
    h = 1e-6
    for idx in occupied[rng.choice(occupied.shape[0], 8, replace=False)]:
        i = tuple(idx[:-1]) + (idx[-1] + 1,)
        vp, vm = val.copy(), val.copy()
        vp[i] += h
        vm[i] -= h
        fp = _loss(sc, pix, target, val=vp)[0]
        fm = _loss(sc, pix, target, val=vm)[0]
        np.testing.assert_allclose(g_val[i], (fp - fm) / (2 * h), rtol=1e-5, atol=1e-8)


# --------------------------------------------------------------------------------------
# the performance ablation without the view-dependence network (flag 8)
# --------------------------------------------------------------------------------------

def test_no_mlp_colour_is_diffuse_plus_background():
    """Without the network the pixel is its composited diffuse colour plus T * background,
    whatever the weights; the composites and counts are the deferred model's."""
    sc = synth.make_scene("gauss64")
    pix = _pix(sc)
    ref = oracle.render_rays(sc, pix)
    sc8 = synth.custom_scene(sc.N, sc.B, sc.ind, sc.atlas, sc.sigma_max, sc.mlp, sc.cameras, flags=8)
    out = oracle.render_rays(sc8, pix)
    T = 1.0 - out["aux"][:, 7]
    np.testing.assert_allclose(out["rgb"], out["aux"][:, :3] + T[:, None] * np.asarray(sc.bg), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(out["aux"], ref["aux"])
    np.testing.assert_array_equal(out["counts"], ref["counts"])
    other = oracle.render_rays(sc8, pix, mlp=np.zeros(synth.MLP_NPARAM, np.float32))
    np.testing.assert_array_equal(other["rgb"], out["rgb"])
    assert np.abs(out["rgb"] - ref["rgb"]).max() > 1e-2


def test_no_mlp_gradient_matches_central_differences():
    sc = synth.make_scene("tiny")
    sc = synth.custom_scene(sc.N, sc.B, sc.ind, sc.atlas, sc.sigma_max, sc.mlp, sc.cameras, flags=8)
    pix = _pix(sc)[::2]
    rng = np.random.default_rng(13)
    target = rng.uniform(size=(pix.shape[0], 3))
    val = sc.atlas.astype(np.float64) / 255.0
    g_val, g_mlp = oracle.backward_rays(sc, pix, oracle.render_rays(sc, pix, val=val)["rgb"] - target, val=val)
    assert (g_mlp == 0).all() and (g_val[..., 4:] == 0).all()      # features reach nothing
    idx = np.argwhere(np.abs(g_val[..., 1:4]) > 1e-4)
    assert idx.shape[0] > 10
    h = 1e-6
    for j in idx[rng.choice(idx.shape[0], 8, replace=False)]:
        i = tuple(j[:-1]) + (j[-1] + 1,)
        vp, vm = val.copy(), val.copy()
        vp[i] += h
        vm[i] -= h
        fd = (_loss(sc, pix, target, val=vp)[0] - _loss(sc, pix, target, val=vm)[0]) / (2 * h)
        np.testing.assert_allclose(g_val[i], fd, rtol=1e-5, atol=1e-9)



@pytest.mark.parametrize("seed", range(10))
def test_brute_force_random_tiny_scenes(seed):
    """Seeded random tiny grids (block edge 2 to 8, random occupancy, density scale, slot
    order, placement and scene flags) and random cameras, inside the grid too: the oracle
    equals the brute force on every ray (colours, composites, counts, visited voxels)."""
    rng = np.random.default_rng(500 + seed)
    B = int(rng.choice([2, 4, 8]))
    G = int(rng.integers(2, 5))
    N = B * G
    ind, atl = synth.gauss_grid(N, B, float(rng.uniform(0.2, 0.8)), float(rng.choice([0.3, 1.5, 6.0])),
                                int(rng.integers(0, 1 << 30)))
    if atl.shape[0] > 1:
        perm = rng.permutation(atl.shape[0])
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        ind = np.where(ind >= 0, inv[np.maximum(ind, 0)], -1).astype(np.int32)
        atl = atl[perm]
    flags = int(rng.choice([0, 1, 4, 5, 8]))
    extent = float(rng.uniform(1.0, 3.0))
    bmin = tuple(float(x) for x in rng.uniform(-2.0, 0.5, 3))
    centre = np.asarray(bmin) + extent / 2
    occ_blocks = np.argwhere(ind >= 0)                  # (z, y, x): look at an occupied block
    cams = np.zeros(2, synth.CAMERA_DTYPE)
    for i in range(2):
        bz, by, bx = occ_blocks[rng.integers(0, occ_blocks.shape[0])]
        tgt = np.asarray(bmin) + (np.array([bx, by, bz]) + 0.5) * B * extent / N
        if i == 1:
            pos = centre + rng.uniform(-0.3, 0.3, 3) * extent
        else:
            dvec = rng.normal(size=3)
            pos = centre + dvec / np.linalg.norm(dvec) * extent * rng.uniform(0.9, 2.0)
        cams[i] = synth.look_at_camera(pos, tgt, 9, 7, float(rng.uniform(30.0, 80.0)), i * 63)
    sc = synth.custom_scene(N, B, ind, atl, 1.5 / (extent / N), synth.init_mlp(rng), cams, bmin=bmin,
                            extent=extent, flags=flags)
    dense = helpers.blocks_to_dense(sc)
    pix = synth.all_pixels(cams)
    out = oracle.render_rays(sc, pix, trace_cap=4 * N + 16)
    assert (out["counts"][:, 1] > 0).any()
    for i, (c, x, y) in enumerate(pix):
        rgb, feat, steps, visited = _brute_force_ray(sc, dense, sc.mlp, cams[c], x, y, bool(flags & 1),
                                                     bool(flags & 4), bool(flags & 8))
        np.testing.assert_allclose(out["rgb"][i], rgb, rtol=0, atol=1e-10)
        np.testing.assert_allclose(out["aux"][i, :7], feat, rtol=0, atol=1e-10)
        assert out["counts"][i, 0] == steps
        assert out["counts"][i, 1] == len(visited)
        assert out["trace"][i, :len(visited)].tolist() == visited
