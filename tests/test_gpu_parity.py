"""GPU parity: the CUDA renderer (through the C ABI) against the FP64 oracle.

Bar: step counts, composited-sample counts and visited-voxel traces bit-exact; colours
and the auxiliary composites (C_d, V, opacity) within 1e-4 absolute; gradients within
1e-4 of the largest oracle gradient entry (FP32 accumulation of many terms vs FP64).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2103_14645_gb300 import renderer, synth
from tests import helpers

pytestmark = pytest.mark.gpu
TOL = 1e-4
DEV = torch.device("cuda:0")

_SCENES = {}


def scene(name):
    if name not in _SCENES:
        _SCENES[name] = synth.make_scene(name)
    return _SCENES[name]


def gpu_render(sc, cams=None, mlp=None, **kw):
    r = renderer.Renderer.from_scene(sc, DEV)
    w = torch.from_numpy(np.asarray(sc.mlp if mlp is None else mlp, np.float32)).to(DEV)
    out = r.render(sc.cameras if cams is None else cams, w, **kw)
    r.check_status()
    if isinstance(out, dict):
        return {k: v.cpu().numpy() for k, v in out.items()}, r
    return {"rgb": out.cpu().numpy()}, r


def oracle_all(sc, cams=None, mlp=None, trace_cap=0):
    cams = sc.cameras if cams is None else cams
    pix = synth.all_pixels(cams)
    return oracle.render_rays(sc, pix, mlp=mlp, cams=cams, trace_cap=trace_cap)


def assert_parity(g, o, trace=True):
    np.testing.assert_array_equal(g["counts"][:, :2], o["counts"])
    assert (g["counts"][:, 2] >= (g["counts"][:, 0] > 0)).all()
    if trace and "trace" in g:
        np.testing.assert_array_equal(g["trace"].astype(np.uint64), o["trace"])
    assert np.abs(g["rgb"] - o["rgb"]).max() <= TOL
    assert np.abs(g["aux"] - o["aux"]).max() <= TOL


@pytest.mark.parametrize("name", ["tiny", "gauss64"])
def test_forward_parity_full_image(name):
    sc = scene(name)
    g, _ = gpu_render(sc, aux=True, counts=True, trace_cap=64)
    o = oracle_all(sc, trace_cap=64)
    assert o["counts"][:, 1].max() <= 64
    assert_parity(g, o)
    assert (o["counts"][:, 1] > 0).mean() > 0.2


def test_forward_parity_ragged_and_multi_camera():
    """Image sizes that are not multiples of the 16x8 CTA tile, several cameras packed."""
    sc = scene("gauss64")
    cams = synth.orbit_cameras(np.random.default_rng(4), [(37, 23), (1, 1), (64, 9), (5, 70)], synth.CAM_RADIUS)
    g, _ = gpu_render(sc, cams=cams, aux=True, counts=True, trace_cap=64)
    o = oracle_all(sc, cams=cams, trace_cap=64)
    assert_parity(g, o)


def test_forward_parity_paper_scale_view():
    """1024^3 grid, 32^3 blocks, one 800x800 view: the benchmarked launch. Every pixel's
    colour and counts are compared; visited voxels on 4096 sampled rays."""
    sc = scene("shell1024")
    g, r = gpu_render(sc, counts=True, aux=True)
    o = oracle_all(sc)
    np.testing.assert_array_equal(g["counts"][:, :2], o["counts"])
    assert np.abs(g["rgb"] - o["rgb"]).max() <= TOL
    assert np.abs(g["aux"] - o["aux"]).max() <= TOL
    pix = synth.random_pixels(np.random.default_rng(7), sc.cameras, 4096)
    w = torch.from_numpy(sc.mlp).to(DEV)
    gt = r.render_rays(sc.cameras, torch.from_numpy(pix).to(DEV), w, counts=True, trace_cap=64)
    r.check_status()
    ot = oracle.render_rays(sc, pix, trace_cap=64)
    assert ot["counts"][:, 1].max() <= 64
    np.testing.assert_array_equal(gt["trace"].cpu().numpy().astype(np.uint64), ot["trace"])
    np.testing.assert_array_equal(gt["counts"].cpu().numpy()[:, :2], ot["counts"])


@pytest.mark.parametrize("name", ["gauss64", "shell1024"])
def test_rays_path_equals_image_path(name):
    """Every pixel of the views as one ray list renders what the image launch renders, bit
    for bit (colours, counts, composites, visited voxels): 4,096 rays (one wave: the
    ray-list build limited to 4 CTAs per SM) and the 640,000 of the 800x800 view (the 8-CTA
    build), with device weights and with weights as kernel parameters."""
    sc = scene(name)
    g, r = gpu_render(sc, aux=True, counts=True, trace_cap=8)
    pix = torch.from_numpy(synth.all_pixels(sc.cameras)).to(DEV)
    w = torch.from_numpy(sc.mlp).to(DEV)
    rr = r.render_rays(sc.cameras, pix, w).cpu().numpy()
    r.check_status()
    np.testing.assert_array_equal(rr, g["rgb"])
    # the debug build of each size (counts, composites, the first visited voxels), device
    # weights and weights as kernel parameters
    r.set_mlp(sc.mlp)
    for mlp in (w, None):
        d = r.render_rays(sc.cameras, pix, mlp, aux=True, counts=True, trace_cap=8)
        r.check_status()
        if mlp is None:      # the parameter-weight MLP rounds its sums in another order
            np.testing.assert_allclose(d["rgb"].cpu().numpy(), g["rgb"], rtol=0, atol=1e-6)
        else:
            np.testing.assert_array_equal(d["rgb"].cpu().numpy(), g["rgb"])
        np.testing.assert_array_equal(d["counts"].cpu().numpy(), g["counts"])
        np.testing.assert_array_equal(d["aux"].cpu().numpy(), g["aux"])
        np.testing.assert_array_equal(d["trace"].cpu().numpy(), g["trace"])


@pytest.mark.parametrize("tile", [None, (8, 4), (4, 8), (16, 2), (32, 1), (8, 16)])
def test_persistent_equals_plain(tile):
    """One persistent graph launch over several cameras of uneven sizes renders exactly
    what one launch per camera renders."""
    sc = scene("gauss64")
    cams = synth.orbit_cameras(np.random.default_rng(8), [(64, 64), (37, 23), (200, 120), (8, 8), (0, 5), (90, 31)],
                               synth.CAM_RADIUS)
    cams[4]["fx"] = cams[4]["fy"] = 1.0      # a zero-width image still needs valid focal lengths
    plain, _ = gpu_render(sc, cams=cams)
    r = renderer.Renderer.from_scene(sc, DEV)
    w = torch.from_numpy(sc.mlp).to(DEV)
    kw = {} if tile is None else {"tile": tile, "ctas_per_sm": 2}
    for _ in range(2):   # first call captures (and may autotune), second replays the graph
        out = r.render(cams, w, persistent=True, **kw).cpu().numpy()
        r.check_status()
        np.testing.assert_array_equal(out, plain["rgb"])
    tw, th, c = r.persistent_config()
    assert tw * th % 32 == 0 and c > 0


def test_persistent_replay_with_new_poses():
    sc = scene("gauss64")
    r = renderer.Renderer.from_scene(sc, DEV)
    w = torch.from_numpy(sc.mlp).to(DEV)
    for seed in range(3):
        cams = synth.orbit_cameras(np.random.default_rng(100 + seed), [(48, 40)] * 5, synth.CAM_RADIUS)
        out = r.render(cams, w, persistent=True, tile=(8, 4), ctas_per_sm=4).cpu().numpy()
        plain = r.render(cams, w).cpu().numpy()
        np.testing.assert_array_equal(out, plain)


def test_max_camera_count():
    sc = scene("tiny")
    cams = synth.orbit_cameras(np.random.default_rng(9), [(7, 5)] * renderer.MAX_CAMERAS, synth.CAM_RADIUS)
    g, _ = gpu_render(sc, cams=cams, counts=True)
    o = oracle_all(sc, cams=cams)
    np.testing.assert_array_equal(g["counts"][:, :2], o["counts"])
    assert np.abs(g["rgb"] - o["rgb"]).max() <= TOL
    p, _ = gpu_render(sc, cams=cams, persistent=True, tile=(8, 4), ctas_per_sm=2)
    np.testing.assert_array_equal(p["rgb"], g["rgb"])


def test_more_cameras_than_one_launch_holds():
    """snerg_render takes any number of cameras: 600 (more than two persistent launches'
    camera tables) render as one call, plain and persistent (consecutive launches of at
    most SNERG_MAX_CAMERAS), against the oracle; ray-list calls still reject more."""
    sc = scene("tiny")
    n = 2 * renderer.MAX_CAMERAS + 88
    cams = synth.orbit_cameras(np.random.default_rng(10), [(6, 5), (3, 7)] * (n // 2), synth.CAM_RADIUS)
    g, r = gpu_render(sc, cams=cams, counts=True)
    o = oracle_all(sc, cams=cams)
    np.testing.assert_array_equal(g["counts"][:, :2], o["counts"])
    assert np.abs(g["rgb"] - o["rgb"]).max() <= TOL
    w = torch.from_numpy(sc.mlp).to(DEV)
    p = r.render(cams, w, persistent=True).cpu().numpy()
    r.check_status()
    np.testing.assert_array_equal(p, g["rgb"])
    host = torch.empty((synth.all_pixels(cams).shape[0], 3), dtype=torch.float32, pin_memory=True)
    r.render_to_host(cams, host, w)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host.numpy(), g["rgb"])
    with pytest.raises(ValueError):
        r.render_rays(cams, torch.zeros((1, 3), dtype=torch.int32, device=DEV), w)


# --------------------------------------------------------------------------------------
# closed forms and degenerate cases on the GPU
# --------------------------------------------------------------------------------------

def test_gpu_uniform_slab_closed_form():
    import math
    col = np.array([100, 150, 200, 10, 20, 30, 40])
    sc = helpers.slab_scene(z_range=(4, 6), q=200, color=col, sigma_max_vox=1.0)
    g, _ = gpu_render(sc, aux=True, counts=True, trace_cap=4)
    T = math.exp(-2 * 200 / 255.0)
    assert g["counts"][0, :2].tolist() == [4, 2]
    np.testing.assert_allclose(g["aux"][0, 7], 1 - T, atol=1e-6)
    np.testing.assert_allclose(g["rgb"][0], col[:3] / 255.0 * (1 - T) + T, atol=1e-6)


def test_gpu_early_exit_count():
    sc = helpers.slab_scene(z_range=(2, 14), q=255, sigma_max_vox=1.0)
    g, _ = gpu_render(sc, counts=True)
    assert g["counts"][0, :2].tolist() == [9, 7]


def test_gpu_empty_grid_is_background():
    sc0 = scene("tiny")
    sc = synth.custom_scene(sc0.N, sc0.B, np.full_like(sc0.ind, -1), np.zeros((0, sc0.B, sc0.B, sc0.B, 8), np.uint8),
                            sc0.sigma_max, sc0.mlp, sc0.cameras)
    g, _ = gpu_render(sc, counts=True)
    assert (g["rgb"] == np.asarray(sc.bg, np.float32)).all()
    assert (g["counts"][:, :2] == 0).all()


def test_gpu_camera_inside_grid_and_axis_rays():
    """Camera inside the grid (t_start = 0), principal rays parallel to the axes (zero
    direction components), origins on voxel faces."""
    sc = scene("gauss64")
    cams = np.concatenate([
        helpers.axis_camera((0.0, 0.0, 0.0), W=9, H=7, f=4.0),
        helpers.axis_camera((0.25, -0.5, 1.5), W=1, H=1),
        helpers.axis_camera((0.03125, 0.0625, 1.2), W=3, H=3, f=1e6),
    ])
    cams["out_offset"] = [0, 63, 64]
    g, _ = gpu_render(sc, cams=cams, aux=True, counts=True, trace_cap=64)
    o = oracle_all(sc, cams=cams, trace_cap=64)
    assert_parity(g, o)
    assert o["counts"][:, 1].sum() > 0


def test_gpu_zero_weight_mlp():
    sc = scene("tiny")
    w0 = np.zeros(synth.MLP_NPARAM, np.float32)
    g, _ = gpu_render(sc, mlp=w0, aux=True, counts=True)
    act = g["counts"][:, 1] > 0
    T = 1 - g["aux"][:, 7]
    np.testing.assert_allclose(g["rgb"][act], g["aux"][act, :3] + 0.5 + T[act, None], atol=1e-6)
    assert (g["rgb"][~act] == 1.0).all()


def test_gpu_invalid_inputs_raise():
    sc = scene("tiny")
    ind = torch.from_numpy(sc.ind).to(DEV)
    atl = torch.from_numpy(sc.atlas).to(DEV)
    args = (sc.N, sc.B, sc.bmin, sc.extent, sc.sigma_max, sc.bg)
    bad = sc.ind.copy()
    bad.flat[np.nonzero(sc.ind.ravel() >= 0)[0][0]] = sc.nb
    with pytest.raises(renderer.SnergError) as e:
        renderer.Renderer(*args, torch.from_numpy(bad).to(DEV), atl)
    assert e.value.code == 1
    dup = sc.ind.copy()
    occ = np.nonzero(dup.ravel() >= 0)[0]
    dup.flat[occ[1]] = dup.flat[occ[0]]
    with pytest.raises(renderer.SnergError):
        renderer.Renderer(*args, torch.from_numpy(dup).to(DEV), atl)
    with pytest.raises((ValueError, renderer.SnergError)):
        renderer.Renderer(sc.N, 3, sc.bmin, sc.extent, sc.sigma_max, sc.bg, ind, atl)
    r = renderer.Renderer(*args, ind, atl)
    w = torch.from_numpy(sc.mlp).to(DEV)
    cams = sc.cameras.copy()
    cams[0]["fx"] = np.nan
    with pytest.raises(renderer.SnergError):
        r.render(cams, w)
    pix = torch.tensor([[0, 0, 0], [1, 0, 0], [0, 10 ** 6, 0]], dtype=torch.int32, device=DEV)
    r.render_rays(sc.cameras, pix, w)
    with pytest.raises(renderer.SnergError) as e:
        r.check_status()
    assert e.value.code == 1
    r.check_status()       # the status word was cleared by the previous read
    out = r.render_rays(sc.cameras, torch.zeros((0, 3), dtype=torch.int32, device=DEV), w)
    assert out.shape == (0, 3)


# --------------------------------------------------------------------------------------
# backward
# --------------------------------------------------------------------------------------

def _bwd_case(sc, n, seed):
    rng = np.random.default_rng(seed)
    pix = synth.random_pixels(rng, sc.cameras, n)
    g = rng.normal(size=(n, 3)).astype(np.float32)
    return pix, g


def gpu_backward(sc, pix, g, mlp=None):
    r = renderer.Renderer.from_scene(sc, DEV)
    w = torch.from_numpy(np.asarray(sc.mlp if mlp is None else mlp, np.float32)).to(DEV)
    ga = torch.zeros(sc.atlas.shape, dtype=torch.float32, device=DEV)
    gm = torch.zeros(883, dtype=torch.float32, device=DEV)
    r.backward(sc.cameras, torch.from_numpy(pix).to(DEV), w, torch.from_numpy(g).to(DEV), ga, gm)
    r.check_status()
    return ga.cpu().numpy(), gm.cpu().numpy(), r


@pytest.mark.parametrize("name,n", [("tiny", 480), ("gauss64", 4096), ("bwd512", 65536)])
def test_backward_matches_oracle_gradient(name, n):
    sc = scene(name)
    pix, g = _bwd_case(sc, n, 31)
    ga, gm, _ = gpu_backward(sc, pix, g)
    ra, rm = oracle.backward_rays(sc, pix, g)
    assert (ga[..., 0] == 0).all()
    sa = np.abs(ra).max()
    sm = np.abs(rm).max()
    assert sa > 0 and sm > 0
    assert np.abs(ga - ra).max() <= 1e-4 * sa
    assert np.abs(gm - rm).max() <= 1e-4 * sm


@pytest.mark.parametrize("sigma_vox,flags", [(0.05, 0), (0.3, 0), (0.3, renderer.FLAG_ALPHA_ATLAS)])
def test_backward_rays_longer_than_the_recording(sigma_vox, flags):
    """The adjoint's first march records its first 32 composited samples; the scatter
    walks those and marches on from the last of them. Here most rays composite more (up to
    ~100 samples of a thin medium): the backward and the fused training step against the
    FP64 oracle, and both against the backward that takes the forward's per-ray state
    (one march from the first composited sample)."""
    sc0 = _gauss_scene(128, 16, 0.5, sigma_vox, 3, [(40, 33), (17, 29), (30, 30)])
    atl = sc0.atlas.copy()
    if flags & renderer.FLAG_ALPHA_ATLAS:
        atl[..., 0] = (atl[..., 0] + 7) // 8          # a thin medium of alpha codes
    sc = synth.custom_scene(sc0.N, sc0.B, sc0.ind, atl, sc0.sigma_max, sc0.mlp, sc0.cameras, flags=flags)
    pix_np, g_np = _bwd_case(sc, 2048, 9)
    o = oracle.render_rays(sc, pix_np)
    assert (o["counts"][:, 1] > 32).sum() > 500 and (o["counts"][:, 1] > 64).any()
    ga, gm, r = gpu_backward(sc, pix_np, g_np)
    ra, rm = oracle.backward_rays(sc, pix_np, g_np)
    assert np.abs(ga - ra).max() <= 1e-4 * np.abs(ra).max()
    assert np.abs(gm - rm).max() <= 1e-4 * np.abs(rm).max()
    w = torch.from_numpy(sc.mlp).to(DEV)
    pix = torch.from_numpy(pix_np).to(DEV)
    fwd = r.render_rays(sc.cameras, pix, w, aux=True, counts=True)
    ga2 = torch.zeros(sc.atlas.shape, dtype=torch.float32, device=DEV)
    gm2 = torch.zeros(883, dtype=torch.float32, device=DEV)
    r.backward(sc.cameras, pix, w, torch.from_numpy(g_np).to(DEV), ga2, gm2, fwd_aux=fwd["aux"],
               fwd_counts=fwd["counts"])
    r.check_status()
    np.testing.assert_allclose(ga, ga2.cpu().numpy(), rtol=0, atol=1e-6 * np.abs(ga).max())
    # the fused step for dL/dC = 2 (C - C*): its gradients against the backward's for that dL/dC
    target = np.random.default_rng(10).uniform(size=(pix_np.shape[0], 3)).astype(np.float32)
    ga3 = torch.zeros_like(ga2)
    gm3 = torch.zeros_like(gm2)
    rgb = torch.empty((pix_np.shape[0], 3), dtype=torch.float32, device=DEV)
    r.train_rays(sc.cameras, pix, w, torch.from_numpy(target).to(DEV), ga3, gm3, out=rgb)
    r.check_status()
    gd = 2.0 * (rgb - torch.from_numpy(target).to(DEV))
    ga4, _, _ = gpu_backward(sc, pix_np, gd.cpu().numpy())
    np.testing.assert_allclose(ga3.cpu().numpy(), ga4, rtol=0, atol=1e-5 * np.abs(ga4).max())
    ra3, _ = oracle.backward_rays(sc, pix_np, 2.0 * (o["rgb"] - target))
    assert np.abs(ga3.cpu().numpy() - ra3).max() <= 1e-4 * np.abs(ra3).max()


def test_backward_mlp_central_differences():
    """GPU gradient w.r.t. 64 sampled MLP weights vs central differences (h = 1e-3) of
    the GPU forward, L = 1/2 sum |C - target|^2 over 4096 rays of the 512^3 scene."""
    sc = scene("bwd512")
    n = 4096
    pix = sc.extra["pix"][:n]
    target = sc.extra["target"][:n]
    r = renderer.Renderer.from_scene(sc, DEV)
    pt = torch.from_numpy(pix).to(DEV)
    w0 = torch.from_numpy(sc.mlp).to(DEV)

    def loss(w):
        c = r.render_rays(sc.cameras, pt, w).double().cpu().numpy()
        return 0.5 * ((c - target) ** 2).sum(), c

    L0, c0 = loss(w0)
    gm = torch.zeros(883, dtype=torch.float32, device=DEV)
    r.backward(sc.cameras, pt, w0, torch.from_numpy((c0 - target).astype(np.float32)).to(DEV), None, gm)
    r.check_status()
    gm = gm.cpu().numpy()
    h = 1e-3
    picks = np.random.default_rng(5).choice(883, 64, replace=False)
    scale = np.abs(gm).max()
    for p in picks:
        wp, wm = w0.clone(), w0.clone()
        wp[p] += h
        wm[p] -= h
        fd = (loss(wp)[0] - loss(wm)[0]) / (2 * h)
        assert abs(fd - gm[p]) <= 2e-2 * abs(fd) + 1e-3 * scale, (p, fd, gm[p])


def test_backward_atlas_code_differences():
    """GPU gradient w.r.t. 64 sampled colour/feature values vs central differences of
    the GPU forward with the uint8 code moved by +-1 (h = 1/255)."""
    sc = scene("gauss64")
    n = 4096
    pix, _ = _bwd_case(sc, n, 3)
    target = np.random.default_rng(4).uniform(size=(n, 3))
    w = torch.from_numpy(sc.mlp).to(DEV)
    pt = torch.from_numpy(pix).to(DEV)

    def loss(atlas):
        s2 = synth.custom_scene(sc.N, sc.B, sc.ind, atlas, sc.sigma_max, sc.mlp, sc.cameras)
        r = renderer.Renderer.from_scene(s2, DEV)
        c = r.render_rays(sc.cameras, pt, w).double().cpu().numpy()
        return 0.5 * ((c - target) ** 2).sum(), c

    L0, c0 = loss(sc.atlas)
    ga, _, _ = gpu_backward(sc, pix, (c0 - target).astype(np.float32))
    flat = ga.reshape(-1)
    atl = sc.atlas.reshape(-1)
    cand = np.nonzero((np.abs(flat) > 1e-3 * np.abs(flat).max()) & (np.arange(flat.size) % 8 != 0)
                      & (atl > 0) & (atl < 255))[0]
    picks = np.random.default_rng(6).choice(cand, 64, replace=False)
    h = 1.0 / 255.0
    for idx in picks:
        ap, am = sc.atlas.copy().reshape(-1), sc.atlas.copy().reshape(-1)
        ap[idx] += 1
        am[idx] -= 1
        fd = (loss(ap.reshape(sc.atlas.shape))[0] - loss(am.reshape(sc.atlas.shape))[0]) / (2 * h)
        assert abs(fd - flat[idx]) <= 2e-2 * abs(fd) + 1e-3 * np.abs(flat).max(), (idx, fd, flat[idx])


def test_autograd_function():
    sc = scene("gauss64")
    pix, _ = _bwd_case(sc, 2048, 8)
    r = renderer.Renderer.from_scene(sc, DEV)
    pt = torch.from_numpy(pix).to(DEV)
    w = torch.from_numpy(sc.mlp).to(DEV).requires_grad_(True)
    vals = (torch.from_numpy(sc.atlas).to(DEV).float() / 255.0).requires_grad_(True)
    target = torch.rand((2048, 3), device=DEV, generator=torch.Generator(DEV).manual_seed(0))
    c = renderer.render_rays_autograd(r, sc.cameras, pt, w, vals)
    loss = 0.5 * ((c - target) ** 2).sum()
    loss.backward()
    ga, gm, _ = gpu_backward(sc, pix, (c.detach() - target).cpu().numpy())
    np.testing.assert_allclose(w.grad.cpu().numpy(), gm, rtol=0, atol=1e-5 * np.abs(gm).max())
    np.testing.assert_allclose(vals.grad.cpu().numpy(), ga, rtol=0, atol=1e-5 * np.abs(ga).max())


# --------------------------------------------------------------------------------------
# the 2048^3 grid (8 views at 1920x1080, 262,144 backward rays)
# --------------------------------------------------------------------------------------

def test_paper_scale_2048_batched_forward_and_backward():
    """Batched persistent render of the 8 1080p views, compared with the oracle on 8192
    sampled pixels (colours and counts); backward on 16,384 of the listed rays against
    the oracle's FP64 MLP gradient (the atlas gradient of this grid would need a 13 GB
    FP64 array on the host; it is compared in full on the 512^3 grid)."""
    sc = scene("shell2048")
    r = renderer.Renderer.from_scene(sc, DEV)
    w = torch.from_numpy(sc.mlp).to(DEV)
    img = r.render(sc.cameras, w, persistent=True).cpu().numpy()
    r.check_status()
    pix = synth.random_pixels(np.random.default_rng(23), sc.cameras, 8192)
    o = oracle.render_rays(sc, pix)
    idx = sc.cameras["out_offset"][pix[:, 0]] + pix[:, 2].astype(np.int64) * sc.cameras["W"][pix[:, 0]] + pix[:, 1]
    assert np.abs(img[idx] - o["rgb"]).max() <= TOL
    g = r.render_rays(sc.cameras, torch.from_numpy(pix).to(DEV), w, counts=True)
    np.testing.assert_array_equal(g["counts"].cpu().numpy()[:, :2], o["counts"])
    assert (o["counts"][:, 1] > 0).mean() > 0.1
    bp = sc.extra["pix"][:16384]
    gr = np.random.default_rng(24).normal(size=(bp.shape[0], 3)).astype(np.float32)
    gm = torch.zeros(883, dtype=torch.float32, device=DEV)
    r.backward(sc.cameras, torch.from_numpy(bp).to(DEV), w, torch.from_numpy(gr).to(DEV), None, gm)
    r.check_status()
    _, rm = oracle.backward_rays(sc, bp, gr, atlas_grad=False)
    assert np.abs(rm).max() > 0
    assert np.abs(gm.cpu().numpy() - rm).max() <= 1e-4 * np.abs(rm).max()


def _subscene_for_rays(sc, pix, trace_cap=256):
    """The blocks that decide the listed rays: every occupied block holding a trilinear
    corner of one of their composited samples (the nearest voxels of those samples, from
    the oracle's trace, moved by -1, 0 or +1 voxel per axis). A block outside this set only
    ever holds samples of these rays whose nearest density code is 0, so emptying it
    changes nothing they composite. Returns (sub-scene, its blocks' raster indices)."""
    o = oracle.render_rays(sc, pix, trace_cap=trace_cap)
    act = o["counts"][:, 1]
    assert act.max() <= trace_cap
    N, B = sc.N, sc.B
    G = N // B
    vox = np.concatenate([o["trace"][i, :act[i]] for i in range(pix.shape[0])]).astype(np.int64)
    z, y, x = vox // (N * N), (vox // N) % N, vox % N
    blocks = np.unique(np.concatenate([
        (np.clip(z + dz, 0, N - 1) // B * G + np.clip(y + dy, 0, N - 1) // B) * G + np.clip(x + dx, 0, N - 1) // B
        for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]))
    ind = np.asarray(sc.ind).reshape(-1)
    keep = blocks[ind[blocks] >= 0]
    sub_ind = np.full(G ** 3, -1, np.int32)
    sub_ind[keep] = np.arange(keep.size, dtype=np.int32)
    sub = synth.custom_scene(N, B, sub_ind.reshape(np.asarray(sc.ind).shape), sc.atlas[ind[keep]], sc.sigma_max,
                             sc.mlp, sc.cameras)
    # the sub-scene renders these rays exactly as the full scene does
    np.testing.assert_array_equal(oracle.render_rays(sub, pix)["rgb"], o["rgb"])
    return sub, keep


def test_paper_scale_2048_atlas_gradient_subscene():
    """The atlas gradient of the 2048^3 grid (262,144-ray backward workload; Sec. 5.5),
    element by element against the FP64 oracle for 8192 of the listed rays. The oracle runs
    on a sub-scene holding only the blocks those rays composite from (see
    _subscene_for_rays), so its FP64 gradient array is a few GB instead of 13 GB; the GPU
    runs on the full grid, and every gradient entry outside those blocks must be 0."""
    sc = scene("shell2048")
    bp = sc.extra["pix"][:8192]
    sub, keep = _subscene_for_rays(sc, bp)
    gr = np.random.default_rng(25).normal(size=(bp.shape[0], 3)).astype(np.float32)
    r = renderer.Renderer.from_scene(sc, DEV)
    w = torch.from_numpy(sc.mlp).to(DEV)
    ga = torch.zeros(sc.atlas.shape, dtype=torch.float32, device=DEV)
    gm = torch.zeros(883, dtype=torch.float32, device=DEV)
    r.backward(sc.cameras, torch.from_numpy(bp).to(DEV), w, torch.from_numpy(gr).to(DEV), ga, gm)
    r.check_status()
    slots = torch.from_numpy(np.asarray(sc.ind).reshape(-1)[keep].astype(np.int64)).to(DEV)
    outside = torch.ones(sc.nb, dtype=torch.bool, device=DEV)
    outside[slots] = False
    flat = ga.view(sc.nb, -1)
    assert float(flat.amax(1)[outside].max()) == 0.0 and float(flat.amin(1)[outside].min()) == 0.0
    got = ga[slots].cpu().numpy()
    del ga
    ra, rm = oracle.backward_rays(sub, bp, gr)
    sa = np.abs(ra).max()
    assert sa > 0 and (got[..., 0] == 0).all()
    assert np.abs(got - ra).max() <= 1e-4 * sa
    assert np.abs(gm.cpu().numpy() - rm).max() <= 1e-4 * np.abs(rm).max()
    assert keep.size > 500                       # the rays reach many blocks of the grid


def test_tile_schedule_reproduces_raster_renders():
    """schedule=True launches each frame's tiles in the cost order recorded on the previous
    scheduled frame of the same size (a viewer's consecutive frames); the pixels must be
    those of a raster-order launch, bit for bit: consecutive orbit frames, a frame of
    another size in between (its own order), back to the first size, both weight paths,
    and the 800x800 view of the 1024^3 grid."""
    import math
    for name, size, frames in (("gauss64", (150, 110), 5), ("shell1024", (800, 800), 3)):
        sc = scene(name)
        r = renderer.Renderer.from_scene(sc, DEV)
        r.set_mlp(sc.mlp)
        w = torch.from_numpy(sc.mlp).to(DEV)
        cams = []
        for i in range(frames):
            az = 0.3 + 0.04 * i
            pos = synth.CAM_RADIUS * np.array([math.cos(0.35) * math.cos(az), math.cos(0.35) * math.sin(az),
                                               math.sin(0.35)])
            cams.append(np.asarray([synth.look_at_camera(pos, (0.0, 0.0, 0.0), size[0], size[1], 39.0)]))
        other = np.asarray([synth.look_at_camera(synth.CAM_RADIUS * np.array([0.0, 1.0, 0.2]), (0.0, 0.0, 0.0),
                                                 61, 37, 39.0)])
        seq = cams[:2] + [other] + cams[2:] + [other]
        assert r.schedule_stats() == (0, 0)
        sparse = []
        prev = None
        for k, cam in enumerate(seq):
            mlp = w if k % 2 else None
            want = r.render(cam, mlp).cpu().numpy()
            got = r.render(cam, mlp, schedule=True).cpu().numpy()
            np.testing.assert_array_equal(got, want)
            sp, ordered = r.schedule_stats()
            # a frame follows the recorded order when the scheduled frame before had its size
            size = (int(cam[0]["W"]), int(cam[0]["H"]))
            assert ordered == (1 if size == prev else 0), (k, ordered)
            assert sp == 0 or ordered == 1
            sparse.append(sp)
            prev = size
        r.check_status()
        if name == "shell1024":
            assert max(sparse) > 0      # the slowest tiles of the 800x800 view were rendered sparsely


def test_parameter_weights_match_device_weights():
    """snerg_set_mlp + d_mlp = NULL (weights as kernel parameters) renders what the
    device-weight path renders, for the plain, ray-list and persistent launches."""
    sc = scene("gauss64")
    cams = synth.orbit_cameras(np.random.default_rng(12), [(64, 64), (37, 23), (50, 70)], synth.CAM_RADIUS)
    r = renderer.Renderer.from_scene(sc, DEV)
    w = torch.from_numpy(sc.mlp).to(DEV)
    with pytest.raises(renderer.SnergError):
        r.render(cams, None)               # no weights stored yet
    r.set_mlp(sc.mlp)
    ref = r.render(cams, w).cpu().numpy()
    o = oracle_all(sc, cams=cams)
    for kw in ({}, {"persistent": True, "tile": (8, 4), "ctas_per_sm": 2}):
        got = r.render(cams, None, **kw).cpu().numpy()
        r.check_status()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-6)
        assert np.abs(got - o["rgb"]).max() <= TOL
    pix = torch.from_numpy(synth.all_pixels(cams)).to(DEV)
    got = r.render_rays(cams, pix, None).cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-6)
    with pytest.raises(renderer.SnergError):
        r.set_mlp(np.full(883, np.nan, np.float32))


# --------------------------------------------------------------------------------------
# grid shapes and media at the edges of the method
# --------------------------------------------------------------------------------------

def _gauss_scene(N, B, occ, sigma_vox, seed, sizes, radius=synth.CAM_RADIUS):
    ind, atl = synth.gauss_grid(N, B, occ, sigma_vox, seed)
    rng = np.random.default_rng(seed + 50)
    cams = synth.orbit_cameras(rng, sizes, radius)
    return synth.custom_scene(N, B, ind, atl, sigma_vox / (synth.WORLD_EXTENT / N), synth.init_mlp(rng), cams)


@pytest.mark.parametrize("N,B", [(48, 16), (96, 32), (32, 2), (128, 64)])
def test_grid_shapes(N, B):
    """G = N/B not a power of two, the smallest and the largest macroblock edge."""
    sc = _gauss_scene(N, B, 0.4, 0.8, 3, [(40, 33), (17, 29)])
    g, _ = gpu_render(sc, aux=True, counts=True, trace_cap=128)
    o = oracle_all(sc, trace_cap=128)
    assert o["counts"][:, 1].max() <= 128
    assert_parity(g, o)
    assert (o["counts"][:, 1] > 0).any()


def test_dense_grid_every_block_stored():
    """No empty block at all: every block visit is an occupied one."""
    sc0 = scene("gauss64")
    ind, atl = helpers.dense_to_blocks(helpers.blocks_to_dense(sc0), sc0.B, keep_empty=True)
    sc = synth.custom_scene(sc0.N, sc0.B, ind, atl, sc0.sigma_max, sc0.mlp, sc0.cameras)
    g, _ = gpu_render(sc, aux=True, counts=True, trace_cap=64)
    assert_parity(g, oracle_all(sc, trace_cap=64))


def _max_resolution_scene():
    """N = 16384, the largest grid snerg_create accepts, in 64^3 blocks (G = 256): a 3 x 3 x 3
    cluster of occupied blocks near the centre (5 % of their voxels with density, random
    codes), and two views: a narrow one filled by the cluster, and a 39-degree one whose
    rays cross the whole grid, nearly all of it empty."""
    import math
    N, B = 16384, 64
    G = N // B
    rng = np.random.default_rng(77)
    ind = np.full((G, G, G), -1, np.int32)
    c0 = G // 2 - 1
    cells = [(z, y, x) for z in range(c0, c0 + 3) for y in range(c0, c0 + 3) for x in range(c0, c0 + 3)]
    for i, (z, y, x) in enumerate(cells):
        ind[z, y, x] = i
    atl = rng.integers(0, 256, size=(len(cells), B, B, B, 8), dtype=np.uint8)
    atl[..., 0] = np.where(rng.random((len(cells), B, B, B)) < 0.05, atl[..., 0], 0)
    delta = synth.WORLD_EXTENT / N
    centre = np.array(synth.WORLD_BMIN) + (c0 + 1.5) * B * delta
    half = 1.5 * B * delta
    pos = centre + synth.CAM_RADIUS * np.array([math.cos(0.4) * math.cos(0.7), math.cos(0.4) * math.sin(0.7),
                                                math.sin(0.4)])
    fov = 2.0 * math.degrees(math.atan(1.2 * half / synth.CAM_RADIUS))
    narrow = synth.look_at_camera(pos, centre, 64, 64, fov)
    wide = synth.orbit_cameras(rng, [(48, 40)], synth.CAM_RADIUS)[0]
    cams = np.asarray([narrow, wide])
    cams[1]["out_offset"] = 64 * 64
    return synth.custom_scene(N, B, ind, atl, 2.0 / delta, synth.init_mlp(rng), cams)


def test_maximum_grid_resolution():
    """The largest grid (N = 16384: up to 28,000 lattice samples along a ray, block skips of
    up to 32 blocks of 64 voxels): counts and visited voxels bit-exact, colours and
    composites within 1e-4, against the oracle, for every pixel of both views."""
    sc = _max_resolution_scene()
    g, _ = gpu_render(sc, aux=True, counts=True, trace_cap=256)
    o = oracle_all(sc, trace_cap=256)
    assert o["counts"][:, 1].max() <= 256
    assert (o["counts"][:4096, 1] > 0).sum() > 3000          # the narrow view sees the cluster
    assert (o["aux"][:4096, 7] > 0.999).sum() > 100            # and some of its rays saturate
    assert_parity(g, o)
    assert g["counts"][4096:, 2].max() >= 8                    # wide-view rays cross the empty grid


@pytest.mark.parametrize("sigma_vox", [1e-3, 200.0])
def test_transparent_and_opaque_media(sigma_vox):
    """Nearly transparent (no ray saturates: every occupied sample is visited) and
    opaque (the first composited sample ends the ray)."""
    sc0 = scene("gauss64")
    sc = synth.custom_scene(sc0.N, sc0.B, sc0.ind, sc0.atlas, sigma_vox / (sc0.extent / sc0.N), sc0.mlp,
                            sc0.cameras)
    g, _ = gpu_render(sc, aux=True, counts=True, trace_cap=256)
    o = oracle_all(sc, trace_cap=256)
    assert_parity(g, o)
    if sigma_vox > 1:
        assert np.median(o["counts"][o["counts"][:, 1] > 0, 1]) <= 2


def test_distant_camera_and_boundary_origins():
    """A camera 60 grid widths away (large t_start: coarse binary32 lattice, so the exact
    exit search must correct the distance estimate) and cameras whose centres sit on the
    grid's faces and edges."""
    sc = scene("gauss64")
    far = synth.orbit_cameras(np.random.default_rng(31), [(48, 48)], 60.0, fov_deg=2.0)
    edge = np.concatenate([helpers.axis_camera((-1.0, 0.1, 0.3), W=7, H=5, f=3.0),
                           helpers.axis_camera((1.0, 1.0, 1.0), W=6, H=6, f=2.0),
                           helpers.axis_camera((0.3, -0.2, -1.0), W=5, H=5, f=2.0)])
    cams = np.concatenate([far, edge])
    off = 0
    for c in cams:
        c["out_offset"] = off
        off += int(c["W"]) * int(c["H"])
    g, _ = gpu_render(sc, cams=cams, aux=True, counts=True, trace_cap=64)
    o = oracle_all(sc, cams=cams, trace_cap=64)
    assert_parity(g, o)
    n_far = 48 * 48
    assert (o["counts"][:n_far, 1] > 0).mean() > 0.1


def test_step_limit_is_reported_and_cleared():
    """A lattice cap far below the ray length: rays stop at the cap, the device records
    SNERG_E_STEP_LIMIT, the host reads it once and the word is cleared. No wait, no fault."""
    sc = scene("gauss64")
    r = renderer.Renderer.from_scene(sc, DEV, max_steps=5)
    w = torch.from_numpy(sc.mlp).to(DEV)
    out = r.render(sc.cameras, w, counts=True)
    with pytest.raises(renderer.SnergError) as e:
        r.check_status()
    assert e.value.code == 4
    r.check_status()
    assert int(out["counts"][:, 0].max()) <= 5
    assert torch.isfinite(out["rgb"]).all()
    full = renderer.Renderer.from_scene(sc, DEV)
    full.render(sc.cameras, w)
    full.check_status()


def test_backward_with_forward_state_matches_recompute():
    """Given the forward's per-ray outputs (C_d, V, first composited index) the backward
    marches each ray once; its gradients equal those of the fully recomputing backward."""
    sc = scene("bwd512")
    pix_np, g_np = _bwd_case(sc, 16384, 41)
    r = renderer.Renderer.from_scene(sc, DEV)
    w = torch.from_numpy(sc.mlp).to(DEV)
    pix = torch.from_numpy(pix_np).to(DEV)
    g = torch.from_numpy(g_np).to(DEV)
    fwd = r.render_rays(sc.cameras, pix, w, aux=True, counts=True)
    outs = []
    for state in (False, True):
        ga = torch.zeros(sc.atlas.shape, dtype=torch.float32, device=DEV)
        gm = torch.zeros(883, dtype=torch.float32, device=DEV)
        kw = {"fwd_aux": fwd["aux"], "fwd_counts": fwd["counts"]} if state else {}
        r.backward(sc.cameras, pix, w, g, ga, gm, **kw)
        r.check_status()
        outs.append((ga.cpu().numpy(), gm.cpu().numpy()))
    (a0, m0), (a1, m1) = outs
    assert np.abs(a0).max() > 0
    np.testing.assert_allclose(a1, a0, rtol=0, atol=1e-6 * np.abs(a0).max())
    np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-6 * np.abs(m0).max())
    c = fwd["counts"].cpu().numpy()
    assert ((c[:, 3] >= 0) == (c[:, 1] > 0)).all()


# --------------------------------------------------------------------------------------
# partial un-premultiply (App. C)
# --------------------------------------------------------------------------------------

def _unpremultiplied(name):
    sc0 = scene(name)
    return synth.custom_scene(sc0.N, sc0.B, sc0.ind, sc0.atlas, sc0.sigma_max, sc0.mlp, sc0.cameras,
                              flags=renderer.FLAG_UNPREMULTIPLY)


def test_unpremultiply_forward_parity():
    sc = _unpremultiplied("gauss64")
    g, r = gpu_render(sc, aux=True, counts=True, trace_cap=64)
    o = oracle_all(sc, trace_cap=64)
    assert_parity(g, o)
    plain = oracle_all(scene("gauss64"))
    assert np.abs(o["rgb"] - plain["rgb"]).max() > 1e-2          # the option changes the image
    w = torch.from_numpy(sc.mlp).to(DEV)
    r.set_mlp(sc.mlp)
    for kw in ({}, {"persistent": True, "tile": (8, 4), "ctas_per_sm": 2}):
        got = r.render(sc.cameras, None, **kw).cpu().numpy()
        assert np.abs(got - o["rgb"]).max() <= TOL


def test_unpremultiply_backward_parity():
    sc = _unpremultiplied("gauss64")
    pix, g = _bwd_case(sc, 4096, 51)
    ga, gm, r = gpu_backward(sc, pix, g)
    ra, rm = oracle.backward_rays(sc, pix, g)
    assert np.abs(ga - ra).max() <= 1e-4 * np.abs(ra).max()
    assert np.abs(gm - rm).max() <= 1e-4 * np.abs(rm).max()
    # the same through the forward's per-ray state
    w = torch.from_numpy(sc.mlp).to(DEV)
    pt = torch.from_numpy(pix).to(DEV)
    fwd = r.render_rays(sc.cameras, pt, w, aux=True, counts=True)
    ga2 = torch.zeros(sc.atlas.shape, dtype=torch.float32, device=DEV)
    gm2 = torch.zeros(883, dtype=torch.float32, device=DEV)
    r.backward(sc.cameras, pt, w, torch.from_numpy(g).to(DEV), ga2, gm2, fwd_aux=fwd["aux"], fwd_counts=fwd["counts"])
    r.check_status()
    assert np.abs(ga2.cpu().numpy() - ra).max() <= 1e-4 * np.abs(ra).max()
    assert np.abs(gm2.cpu().numpy() - rm).max() <= 1e-4 * np.abs(rm).max()


# --------------------------------------------------------------------------------------
# non-deferred comparison model (per-sample view-dependence MLP)
# --------------------------------------------------------------------------------------

def _per_sample(name):
    sc0 = scene(name)
    return synth.custom_scene(sc0.N, sc0.B, sc0.ind, sc0.atlas, sc0.sigma_max, sc0.mlp, sc0.cameras,
                              flags=renderer.FLAG_PER_SAMPLE_MLP)


@pytest.mark.parametrize("param_weights", [False, True])
def test_per_sample_model_parity(param_weights):
    sc = _per_sample("gauss64")
    r = renderer.Renderer.from_scene(sc, DEV)
    w = torch.from_numpy(sc.mlp).to(DEV)
    if param_weights:
        r.set_mlp(sc.mlp)
    out = r.render(sc.cameras, None if param_weights else w, counts=True, aux=True)
    r.check_status()
    o = oracle_all(sc)
    np.testing.assert_array_equal(out["counts"].cpu().numpy()[:, :2], o["counts"])
    assert np.abs(out["rgb"].cpu().numpy() - o["rgb"]).max() <= TOL
    deferred = oracle_all(scene("gauss64"))
    assert np.abs(o["rgb"] - deferred["rgb"]).max() > 1e-2


def test_per_sample_model_paper_scale_view_sampled():
    sc = _per_sample("shell1024")
    r = renderer.Renderer.from_scene(sc, DEV)
    r.set_mlp(sc.mlp)
    img = r.render(sc.cameras, None).cpu().numpy()
    r.check_status()
    pix = synth.random_pixels(np.random.default_rng(44), sc.cameras, 4096)
    o = oracle.render_rays(sc, pix)
    idx = pix[:, 2].astype(np.int64) * 800 + pix[:, 1]
    assert np.abs(img[idx] - o["rgb"]).max() <= TOL


def test_per_sample_model_unsupported_paths():
    sc = _per_sample("tiny")
    r = renderer.Renderer.from_scene(sc, DEV)
    w = torch.from_numpy(sc.mlp).to(DEV)
    pix = torch.zeros((4, 3), dtype=torch.int32, device=DEV)
    for call in (lambda: r.render(sc.cameras, w, persistent=True, tile=(8, 4), ctas_per_sm=2),
                 lambda: r.render_rays(sc.cameras, pix, w),
                 lambda: r.backward(sc.cameras, pix, w, torch.zeros((4, 3), device=DEV), None,
                                    torch.zeros(883, device=DEV))):
        with pytest.raises(renderer.SnergError) as e:
            call()
        assert e.value.code == 5
    sc0 = scene("tiny")
    with pytest.raises((ValueError, renderer.SnergError)):
        renderer.Renderer(sc0.N, sc0.B, sc0.bmin, sc0.extent, sc0.sigma_max, sc0.bg,
                          torch.from_numpy(sc0.ind).to(DEV), torch.from_numpy(sc0.atlas).to(DEV), flags=3)


# --------------------------------------------------------------------------------------
# alpha atlas (channel 0 holds alpha codes, App. A's alpha texture)
# --------------------------------------------------------------------------------------

def _alpha(name, extra=0):
    sc0 = scene(name)
    return synth.custom_scene(sc0.N, sc0.B, sc0.ind, sc0.atlas, sc0.sigma_max, sc0.mlp, sc0.cameras,
                              flags=renderer.FLAG_ALPHA_ATLAS | extra)


@pytest.mark.parametrize("name,extra", [("tiny", 0), ("gauss64", 0), ("gauss64", renderer.FLAG_UNPREMULTIPLY)])
def test_alpha_atlas_forward_parity(name, extra):
    """Counts and visited voxels bit-exact (the binary32 running product decides the exit),
    colours within 1e-4, through the image, persistent and ray-list paths."""
    sc = _alpha(name, extra)
    g, r = gpu_render(sc, aux=True, counts=True, trace_cap=64)
    o = oracle_all(sc, trace_cap=64)
    assert o["counts"][:, 1].max() <= 64
    assert_parity(g, o)
    dens = oracle_all(scene(name))
    assert np.abs(o["rgb"] - dens["rgb"]).max() > 1e-2              # the flag changes the image
    r.set_mlp(sc.mlp)
    got = r.render(sc.cameras, None, persistent=True, tile=(8, 4), ctas_per_sm=2).cpu().numpy()
    assert np.abs(got - o["rgb"]).max() <= TOL
    pix = synth.all_pixels(sc.cameras)
    rr = r.render_rays(sc.cameras, torch.from_numpy(pix).to(DEV), torch.from_numpy(sc.mlp).to(DEV)).cpu().numpy()
    r.check_status()
    assert np.abs(rr - o["rgb"]).max() <= TOL


def test_alpha_atlas_paper_scale_view():
    """The 1024^3 grid read as an alpha atlas, the full 800x800 view: every pixel's counts
    and colour."""
    sc = _alpha("shell1024")
    r = renderer.Renderer.from_scene(sc, DEV)
    r.set_mlp(sc.mlp)
    out = r.render(sc.cameras, None, counts=True)
    r.check_status()
    o = oracle_all(sc)
    np.testing.assert_array_equal(out["counts"].cpu().numpy()[:, :2], o["counts"])
    assert np.abs(out["rgb"].cpu().numpy() - o["rgb"]).max() <= TOL


def test_alpha_atlas_backward_parity():
    sc = _alpha("gauss64")
    pix, g = _bwd_case(sc, 4096, 61)
    ga, gm, r = gpu_backward(sc, pix, g)
    ra, rm = oracle.backward_rays(sc, pix, g)
    assert np.abs(ga - ra).max() <= 1e-4 * np.abs(ra).max()
    assert np.abs(gm - rm).max() <= 1e-4 * np.abs(rm).max()
    w = torch.from_numpy(sc.mlp).to(DEV)
    pt = torch.from_numpy(pix).to(DEV)
    fwd = r.render_rays(sc.cameras, pt, w, aux=True, counts=True)
    ga2 = torch.zeros(sc.atlas.shape, dtype=torch.float32, device=DEV)
    gm2 = torch.zeros(883, dtype=torch.float32, device=DEV)
    r.backward(sc.cameras, pt, w, torch.from_numpy(g).to(DEV), ga2, gm2, fwd_aux=fwd["aux"], fwd_counts=fwd["counts"])
    r.check_status()
    assert np.abs(ga2.cpu().numpy() - ra).max() <= 1e-4 * np.abs(ra).max()


def test_alpha_atlas_per_sample_model():
    sc = _alpha("gauss64", renderer.FLAG_PER_SAMPLE_MLP)
    g, _ = gpu_render(sc, aux=True, counts=True)
    o = oracle_all(sc)
    np.testing.assert_array_equal(g["counts"][:, :2], o["counts"])
    assert np.abs(g["rgb"] - o["rgb"]).max() <= TOL


# --------------------------------------------------------------------------------------
# row bands and the banded render into pinned host memory
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["gauss64", "shell1024"])
def test_row_bands_reproduce_the_full_render(name):
    """Bands of rows (ragged edges included) render exactly the pixels of the full launch,
    bit for bit, and leave the other rows untouched."""
    sc = scene(name)
    r = renderer.Renderer.from_scene(sc, DEV)
    r.set_mlp(sc.mlp)
    full = r.render(sc.cameras, None).clone()
    H = int(sc.cameras[0]["H"])
    W = int(sc.cameras[0]["W"])
    edges = [0, 1, 13, H // 2 + 3, H - 1, H]
    out = torch.full_like(full, float("nan"))
    for y0, y1 in zip(edges[:-1], edges[1:]):
        r.render(sc.cameras, None, out=out, rows=(y0, y1))
        torch.cuda.synchronize()
        img = out.view(H, W, 3)
        assert torch.equal(img[y0:y1], full.view(H, W, 3)[y0:y1])
        assert torch.isnan(img[y1:]).all()
    r.check_status()
    assert torch.equal(out, full)


def test_render_to_host_matches_the_device_render():
    """Into pinned memory the kernels write the pixels directly; into pageable memory the
    frame goes in row bands (1, 3, 8, 16) with a copy per band. Both return the device image
    exactly, for one camera and for a batch of ragged cameras."""
    sc = scene("gauss64")
    r = renderer.Renderer.from_scene(sc, DEV)
    r.set_mlp(sc.mlp)
    cams = synth.orbit_cameras(np.random.default_rng(12), [(37, 23), (64, 64), (5, 70)], synth.CAM_RADIUS)
    for cs in (sc.cameras, cams):
        ref = r.render(cs, None).cpu()
        host = torch.full((ref.shape[0], 3), float("nan"), dtype=torch.float32, pin_memory=True)
        r.render_to_host(cs, host)
        torch.cuda.current_stream(DEV).synchronize()
        assert torch.equal(host, ref)
        for bands in (1, 3, 8, 16):
            page = torch.full((ref.shape[0], 3), float("nan"), dtype=torch.float32)
            r.render_to_host(cs, page, bands=bands)
            torch.cuda.current_stream(DEV).synchronize()
            assert torch.equal(page, ref), bands
    r.check_status()


def test_row_option_errors():
    sc = scene("tiny")
    r = renderer.Renderer.from_scene(sc, DEV)
    r.set_mlp(sc.mlp)
    for rows, code in (((-1, 4), 1), ((5, 3), 1)):
        with pytest.raises(renderer.SnergError) as e:
            r.render(sc.cameras, None, rows=rows)
        assert e.value.code == code
    with pytest.raises(renderer.SnergError) as e:
        r.render(sc.cameras, None, persistent=True, rows=(0, 4))
    assert e.value.code == 5
    host = torch.empty((int(sc.cameras[0]["W"]) * int(sc.cameras[0]["H"]), 3), pin_memory=True)
    for bands in (0, 17):
        with pytest.raises(renderer.SnergError) as e:
            r.render_to_host(sc.cameras, host, bands=bands)
        assert e.value.code == 1
    out = torch.full((int(sc.cameras[0]["W"]) * int(sc.cameras[0]["H"]), 3), 7.0, device=DEV)
    r.render(sc.cameras, None, out=out, rows=(int(sc.cameras[0]["H"]) + 5, int(sc.cameras[0]["H"]) + 9))
    torch.cuda.synchronize()
    assert (out == 7.0).all()                     # rows beyond the image: nothing written


# --------------------------------------------------------------------------------------
# the performance ablation without the view-dependence network
# --------------------------------------------------------------------------------------

def test_no_mlp_forward_and_backward_parity():
    sc0 = scene("gauss64")
    sc = synth.custom_scene(sc0.N, sc0.B, sc0.ind, sc0.atlas, sc0.sigma_max, sc0.mlp, sc0.cameras,
                            flags=renderer.FLAG_NO_MLP)
    g, r = gpu_render(sc, aux=True, counts=True, trace_cap=64)
    o = oracle_all(sc, trace_cap=64)
    assert_parity(g, o)
    r.set_mlp(sc.mlp)
    got = r.render(sc.cameras, None, persistent=True, tile=(8, 4), ctas_per_sm=2).cpu().numpy()
    assert np.abs(got - o["rgb"]).max() <= TOL
    pix, gr = _bwd_case(sc, 4096, 71)
    ga, gm, _ = gpu_backward(sc, pix, gr)
    ra, rm = oracle.backward_rays(sc, pix, gr)
    assert (gm == 0).all() and (rm == 0).all()
    assert np.abs(ga - ra).max() <= 1e-4 * np.abs(ra).max()
    assert (ga[..., 4:] == 0).all()


def test_batched_64_cameras_paper_scale_sampled():
    """The bench's batched workload (the 1024^3 grid, 64 cameras of mixed sizes, 40.6 M rays)
    in one persistent graph launch: 8,192 rays sampled over every camera match the oracle,
    and the ray-list path gives their counts bit-exactly."""
    sc = scene("batch1024")
    r = renderer.Renderer.from_scene(sc, DEV)
    r.set_mlp(sc.mlp)
    img = r.render(sc.cameras, None, persistent=True).cpu().numpy()
    r.check_status()
    pix = synth.random_pixels(np.random.default_rng(81), sc.cameras, 8192)
    o = oracle.render_rays(sc, pix)
    off = sc.cameras["out_offset"][pix[:, 0]] + pix[:, 2].astype(np.int64) * sc.cameras["W"][pix[:, 0]] + pix[:, 1]
    assert np.abs(img[off] - o["rgb"]).max() <= TOL
    got = r.render_rays(sc.cameras, torch.from_numpy(pix).to(DEV), None, counts=True)
    r.check_status()
    np.testing.assert_array_equal(got["counts"].cpu().numpy()[:, :2], o["counts"])
    assert (o["counts"][:, 1] > 0).mean() > 0.05


def test_render_into_pinned_host_memory_all_paths():
    """The plain and the persistent launches store into a pinned host tensor through the
    device's mapping and give the device render exactly."""
    sc = scene("gauss64")
    r = renderer.Renderer.from_scene(sc, DEV)
    r.set_mlp(sc.mlp)
    cams = synth.orbit_cameras(np.random.default_rng(13), [(37, 23), (64, 64), (5, 70), (80, 3)], synth.CAM_RADIUS)
    ref = r.render(cams, None).cpu()
    for persistent in (False, True):
        host = torch.full(ref.shape, float("nan"), dtype=torch.float32, pin_memory=True)
        r.render(cams, None, out=host, persistent=persistent)
        torch.cuda.current_stream(DEV).synchronize()
        assert torch.equal(host, ref), persistent
    with pytest.raises(ValueError):
        r.render(cams, None, out=torch.empty(ref.shape))          # pageable host memory
    r.check_status()
