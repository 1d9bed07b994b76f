"""Seeded random small scenes through every render path and the adjoint, against the
FP64 oracle: grid and block sizes, occupancy and density scale, grid placement, scene
flags, cameras outside and inside the grid at random poses and image sizes, slot order of
the atlas. The bar is the parity bar of the other GPU tests: step counts, composited
counts and visited voxels bit-exact, colours and composites within 1e-4, gradients within
1e-4 of the largest oracle entry."""

import numpy as np
import pytest
import torch

import oracle
from paper_2103_14645_gb300 import renderer, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL = 1e-4
CASES = 48


def _random_scene(seed):
    rng = np.random.default_rng(1000 + seed)
    B = int(rng.choice([2, 4, 8, 16]))
    G = int(rng.integers(2, max(3, 96 // B) + 1))
    N = B * G
    occ = float(rng.uniform(0.1, 0.7))
    sigma_vox = float(rng.choice([0.05, 0.5, 2.0, 20.0]))
    ind, atl = synth.gauss_grid(N, B, occ, sigma_vox, int(rng.integers(0, 1 << 30)))
    if atl.shape[0] > 1:                                   # a random slot order
        perm = rng.permutation(atl.shape[0])
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        ind = np.where(ind >= 0, inv[np.maximum(ind, 0)], -1).astype(np.int32)
        atl = atl[perm]
    flags = int(rng.choice([0, 0, 1, 4, 5, 8]))
    extent = float(rng.uniform(1.0, 3.0))
    bmin = tuple(float(x) for x in rng.uniform(-2.0, 0.5, 3))
    centre = np.asarray(bmin) + extent / 2
    cams = np.zeros(3, synth.CAMERA_DTYPE)
    off = 0
    for i in range(3):
        W, H = int(rng.integers(1, 48)), int(rng.integers(1, 48))
        if i == 2:                                         # inside the grid
            pos = centre + rng.uniform(-0.3, 0.3, 3) * extent
        else:
            d = rng.normal(size=3)
            pos = centre + d / np.linalg.norm(d) * extent * rng.uniform(0.9, 2.5)
        tgt = centre + rng.uniform(-0.2, 0.2, 3) * extent
        cams[i] = synth.look_at_camera(pos, tgt, W, H, float(rng.uniform(20.0, 90.0)), off)
        off += W * H
    mlp = synth.init_mlp(rng)
    sc = synth.custom_scene(N, B, ind, atl, sigma_vox / (extent / N), mlp, cams, bmin=bmin, extent=extent,
                            flags=flags)
    return sc, rng


@pytest.mark.parametrize("seed", range(CASES))
def test_random_scene_parity(seed):
    sc, rng = _random_scene(seed)
    r = renderer.Renderer.from_scene(sc, DEV)
    w = torch.from_numpy(sc.mlp).to(DEV)
    pix = synth.all_pixels(sc.cameras)
    cap = 4 * sc.N + 16
    g = r.render(sc.cameras, w, aux=True, counts=True, trace_cap=min(cap, 512))
    r.check_status()
    o = oracle.render_rays(sc, pix, trace_cap=min(cap, 512))
    np.testing.assert_array_equal(g["counts"].cpu().numpy()[:, :2], o["counts"])
    if o["counts"][:, 1].max() <= 512:
        np.testing.assert_array_equal(g["trace"].cpu().numpy().astype(np.uint64), o["trace"])
    assert np.abs(g["rgb"].cpu().numpy() - o["rgb"]).max() <= TOL
    assert np.abs(g["aux"].cpu().numpy() - o["aux"]).max() <= TOL
    # the fast paths: plain without debug outputs, persistent graph, ray list
    r.set_mlp(sc.mlp)
    plain = r.render(sc.cameras, None).cpu().numpy()
    pers = r.render(sc.cameras, None, persistent=True, tile=(8, 4), ctas_per_sm=4).cpu().numpy()
    rays = r.render_rays(sc.cameras, torch.from_numpy(pix).to(DEV), None).cpu().numpy()
    r.check_status()
    for got in (plain, pers, rays):
        assert np.abs(got - o["rgb"]).max() <= TOL
    # the adjoint on a random subset of the rays
    n = min(pix.shape[0], 512)
    sel = rng.choice(pix.shape[0], n, replace=False)
    gr = rng.normal(size=(n, 3)).astype(np.float32)
    ga = torch.zeros(sc.atlas.shape, dtype=torch.float32, device=DEV)
    gm = torch.zeros(synth.MLP_NPARAM, dtype=torch.float32, device=DEV)
    pt = torch.from_numpy(np.ascontiguousarray(pix[sel])).to(DEV)
    r.backward(sc.cameras, pt, w, torch.from_numpy(gr).to(DEV), ga, gm)
    r.check_status()
    ra, rm = oracle.backward_rays(sc, pix[sel], gr)
    if np.abs(ra).max() > 0:
        assert np.abs(ga.cpu().numpy() - ra).max() <= 1e-4 * np.abs(ra).max()
    if np.abs(rm).max() > 0:
        assert np.abs(gm.cpu().numpy() - rm).max() <= 1e-4 * np.abs(rm).max()
    else:
        assert (gm.cpu().numpy() == 0).all()


@pytest.mark.parametrize("seed", range(0, CASES, 3))
def test_random_scene_fused_training_step(seed):
    """snerg_train_rays on the random scenes: C, the L2 loss and both gradients against the
    oracle's render and adjoint for dL/dC = 2 (C - C*)."""
    sc, rng = _random_scene(seed)
    r = renderer.Renderer.from_scene(sc, DEV)
    pix = synth.all_pixels(sc.cameras)
    n = min(pix.shape[0], 1024)
    sel = np.ascontiguousarray(pix[rng.choice(pix.shape[0], n, replace=False)])
    target = rng.uniform(size=(n, 3)).astype(np.float32)
    w = torch.from_numpy(sc.mlp).to(DEV)
    ga = torch.zeros(sc.atlas.shape, dtype=torch.float32, device=DEV)
    gm = torch.zeros(synth.MLP_NPARAM, dtype=torch.float32, device=DEV)
    loss = torch.zeros(1, dtype=torch.float32, device=DEV)
    rgb = torch.empty((n, 3), dtype=torch.float32, device=DEV)
    r.train_rays(sc.cameras, torch.from_numpy(sel).to(DEV), w, torch.from_numpy(target).to(DEV), ga, gm, loss=loss,
                 out=rgb)
    r.check_status()
    o = oracle.render_rays(sc, sel)
    d = o["rgb"] - target
    ra, rm = oracle.backward_rays(sc, sel, 2.0 * d)
    assert np.abs(rgb.cpu().numpy() - o["rgb"]).max() <= TOL
    np.testing.assert_allclose(float(loss.item()), float((d * d).sum()), rtol=1e-4)
    if np.abs(ra).max() > 0:
        assert np.abs(ga.cpu().numpy() - ra).max() <= 1e-4 * np.abs(ra).max()
    if np.abs(rm).max() > 0:
        assert np.abs(gm.cpu().numpy() - rm).max() <= 1e-4 * np.abs(rm).max()
