"""GPU bake (snerg_bake, Sec. 5.3-5.4) against the FP64 oracle bake.

The kernel evaluates the field in binary32 (the PTX base-2 exponential ex2.approx,
sincosf), the oracle in FP64, so a code can differ only where the exact value lies within
the kernel's error of a rounding boundary. Error budget of the kernel's value before
rounding, in code units (255 x):
  density: each blob term 2^(-k |x - c|^2) (k in base-2 units) carries the rounding of x
           (|x| <= 2, 2^-23 relative) amplified by the exponent's slope 2 |x - c| k
           (about 100 for s = 0.03), the rounding of the expanded exponent (a few ulp of
           |exponent| <= 40, i.e. <= 1e-5 absolute), about 2^-22 relative of ex2.approx and
           a few ulp of the sums: below 2e-5 relative; band 5e-5 * raw + 1e-3;
  colour:  sin of an argument |w . x + phi| <= 8 * 5 + 2 pi accurate to a few ulp of 47
           (4e-6 each), halved, times 255: below 2e-3; band 4e-3.
Blobs left out where their term is below 2^-30 min(sigma_max, sigma_tau) move the
density by less than 64 * 2^-30 * 255 = 1.5e-5 code units, inside the density band.
Outside the band the codes are equal; inside it they differ by at most 1. The tau_alpha
decision is exact outside |alpha_max - tau| <= 5e-5 tau."""
import numpy as np
import pytest
import torch

import oracle
from paper_2103_14645_gb300 import renderer, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TAU = 0.005
BMIN = (-1.0, -1.0, -1.0)
EXTENT = 2.0


def _band(raw):
    """True where the exact value 255 x is within the kernel's error of a rounding
    boundary (channel 0 density, 1..7 colour)."""
    frac = np.abs(raw - np.floor(raw) - 0.5)
    band = np.empty_like(raw)
    band[..., 0] = 5e-5 * np.abs(raw[..., 0]) + 1e-3
    band[..., 1:] = 4e-3
    return frac <= band


def _gpu_bake(N, B, sigma_max, f, max_blocks=None, bmin=BMIN):
    field = renderer.bake_field(f["blobs"], f["colors"], f["jitter"], TAU)
    ind, atl = renderer.bake(N, B, bmin, EXTENT, sigma_max, field, DEV, max_blocks=max_blocks)
    return ind.cpu().numpy(), atl.cpu().numpy()


def _compare_blocks(got, want, raw):
    """got / want uint8 [n,B,B,B,8], raw f64: equal outside the rounding band, within 1
    inside it. Returns the number of differing codes."""
    d = np.abs(got.astype(np.int64) - want.astype(np.int64))
    inside = _band(raw)
    assert (d[~inside] == 0).all(), np.argwhere((d > 0) & ~inside)[:5]
    assert d.max(initial=0) <= 1
    return int((d > 0).sum())


def _check_bake(N, B, sigma_max, f, bmin=BMIN):
    ind_g, atl_g = _gpu_bake(N, B, sigma_max, f, bmin=bmin)
    ind_o, atl_o, amax = oracle.bake(N, B, bmin, EXTENT, sigma_max, f["blobs"], f["colors"], f["jitter"])
    ambiguous = np.abs(amax - TAU) <= 5e-5 * TAU
    kg, ko = ind_g >= 0, ind_o >= 0
    assert ((kg == ko) | ambiguous).all()
    # raster numbering (x fastest) of whatever the kernel kept
    assert (ind_g[kg] == np.arange(kg.sum())).all() and atl_g.shape[0] == kg.sum()
    both = kg & ko
    assert both.sum() > 0
    blocks = np.flatnonzero(both.ravel())
    _, content, raw = oracle.bake_blocks(N, B, bmin, EXTENT, sigma_max, f["blobs"], f["colors"], f["jitter"], blocks)
    np.testing.assert_array_equal(content, atl_o[ind_o.ravel()[blocks]])
    ndiff = _compare_blocks(atl_g[ind_g.ravel()[blocks]], content, raw)
    return ind_g, atl_g, ind_o, atl_o, ndiff


@pytest.mark.parametrize("N,B,n_blob", [(16, 2, 6), (32, 4, 12), (64, 8, 24), (128, 16, 24), (256, 16, 40),
                                        (128, 32, 64), (128, 64, 10)])
def test_bake_matches_oracle(N, B, n_blob):
    f = synth.analytic_field(100 + N + B, n_blob=n_blob, std=(0.04, 0.12), peak=(10.0, 120.0))
    _, atl_g, _, _, ndiff = _check_bake(N, B, 120.0, f)
    assert ndiff <= 1e-4 * atl_g.size + 2


def test_bake_offset_grid_and_saturated_density():
    """A grid not centred on the field, density codes that clamp at 255 (sigma_max below
    the peaks), and blobs partly outside the grid."""
    f = synth.analytic_field(7, n_blob=32, radius=0.9, std=(0.05, 0.15), peak=(50.0, 400.0))
    _, atl_g, _, _, _ = _check_bake(64, 8, 100.0, f, bmin=(-0.7, -1.2, -0.9))
    assert (atl_g[..., 0] == 255).any()


def test_bake_empty_field_and_capacity():
    f = synth.analytic_field(3, n_blob=0)
    ind, atl = _gpu_bake(32, 8, 50.0, f)
    assert (ind == -1).all() and atl.shape[0] == 0
    f = synth.analytic_field(3, n_blob=16)
    full_ind, full_atl = _gpu_bake(64, 8, 50.0, f)
    nb = full_atl.shape[0]
    assert nb > 2
    with pytest.raises(renderer.SnergError) as e:
        _gpu_bake(64, 8, 50.0, f, max_blocks=nb - 1)
    assert e.value.code == 2
    ind, atl = _gpu_bake(64, 8, 50.0, f, max_blocks=nb)          # exact capacity
    np.testing.assert_array_equal(ind, full_ind)
    np.testing.assert_array_equal(atl, full_atl)


def test_bake_invalid_arguments():
    f = synth.analytic_field(3, n_blob=4)
    bad = dict(f)
    bad["jitter"] = f["jitter"].copy()
    bad["jitter"][3, 1] = 9.0                                   # |offset| > 8 voxels
    with pytest.raises(renderer.SnergError):
        _gpu_bake(32, 8, 50.0, bad)
    bad = dict(f)
    bad["blobs"] = f["blobs"].copy()
    bad["blobs"][0, 3] = 0.0                                    # zero std
    with pytest.raises(renderer.SnergError):
        _gpu_bake(32, 8, 50.0, bad)
    with pytest.raises(ValueError):                             # G = 512 > 256
        _gpu_bake(1024, 2, 50.0, f)
    with pytest.raises(renderer.SnergError):
        field = renderer.bake_field(f["blobs"], f["colors"], f["jitter"], 0.0)   # tau = 0
        renderer.bake(32, 8, BMIN, EXTENT, 50.0, field, DEV)


def test_baked_grid_renders_like_the_oracle_bake():
    """Bake -> snerg_create from the device buffers -> render, against the oracle's bake
    rendered by the oracle. Where the two bakes are byte-identical the render must match at
    the usual tolerance with identical step counts; otherwise a few codes differ by one and
    the colours may differ by a few 1/255."""
    N, B, sigma_max = 128, 16, 120.0
    f = synth.analytic_field(21, n_blob=24, std=(0.04, 0.12), peak=(10.0, 120.0))
    ind_g, atl_g, ind_o, atl_o, ndiff = _check_bake(N, B, sigma_max, f)
    rng = np.random.default_rng(4)
    cams = synth.orbit_cameras(rng, [(48, 40), (40, 48)], synth.CAM_RADIUS)
    mlp = synth.init_mlp(rng)
    r = renderer.Renderer(N, B, BMIN, EXTENT, sigma_max, synth.BG, torch.from_numpy(ind_g).to(DEV),
                          torch.from_numpy(atl_g).to(DEV))
    pix = torch.from_numpy(synth.all_pixels(cams)).to(DEV)
    out = r.render_rays(cams, pix, torch.from_numpy(mlp).to(DEV), counts=True)
    r.check_status()
    sc = synth.custom_scene(N, B, ind_o, atl_o, sigma_max, mlp, cams, bmin=BMIN, extent=EXTENT)
    ref = oracle.render_rays(sc, pix.cpu().numpy())
    rgb = out["rgb"].cpu().numpy()
    hit = ref["counts"][:, 1] > 0
    assert hit.mean() > 0.1
    if ndiff == 0 and np.array_equal(ind_g, ind_o):
        np.testing.assert_array_equal(out["counts"].cpu().numpy()[:, :2], ref["counts"][:, :2])
        assert np.abs(rgb - ref["rgb"]).max() <= 1e-4
    else:
        err = np.abs(rgb - ref["rgb"]).max(axis=1)
        assert (err <= 1e-4).mean() > 0.99 and err.max() <= 0.05


def test_bake_paper_scale_sampled():
    """The bench's bake: the 1024^3 grid of 32^3 macroblocks with 64 blobs on a sphere.
    128 macroblocks -- 64 kept, 32 culled ones with a kept face neighbour (where the
    tau_alpha decision is closest) and 32 random ones -- are recomputed one by one by the
    oracle; kept decisions agree outside the tau_alpha ambiguity band, the kept blocks'
    codes agree outside the rounding band (within one code inside it), and the slots are
    numbered in raster order."""
    N, B, sigma_max = 1024, 32, 200.0
    G = N // B
    f = synth.analytic_field(1)
    ind_g, atl_g = _gpu_bake(N, B, sigma_max, f)
    flat = ind_g.ravel()
    kept = np.flatnonzero(flat >= 0)
    assert (flat[kept] == np.arange(kept.size)).all() and atl_g.shape[0] == kept.size
    assert 0.02 < kept.size / G ** 3 < 0.5
    rng = np.random.default_rng(9)
    occ = ind_g >= 0
    pad = np.pad(occ, 1)
    nbr = np.zeros_like(occ)
    for ax in range(3):
        for sh in (-1, 1):
            nbr |= np.roll(pad, sh, axis=ax)[1:-1, 1:-1, 1:-1]
    near = np.flatnonzero((~occ & nbr).ravel())
    sample = np.unique(np.concatenate([rng.choice(kept, 64, replace=False), rng.choice(near, 32, replace=False),
                                       rng.choice(G ** 3, 32, replace=False)]))
    amax, content, raw = oracle.bake_blocks(N, B, BMIN, EXTENT, sigma_max, f["blobs"], f["colors"], f["jitter"],
                                            sample)
    ambiguous = np.abs(amax - TAU) <= 5e-5 * TAU
    assert (((flat[sample] >= 0) == (amax >= TAU)) | ambiguous).all()
    sel = flat[sample] >= 0
    assert sel.sum() >= 64
    ndiff = _compare_blocks(atl_g[flat[sample][sel]], content[sel], raw[sel])
    assert ndiff <= 1e-4 * content[sel].size + 2


def test_bake_alpha_codes_match_oracle_and_render():
    """With the alpha-atlas flag the bake stores alpha = 1 - exp(-sigma v) codes; they match
    the oracle (rounding band), and the baked grid renders in alpha mode like the oracle's."""
    N, B, sigma_max = 64, 8, 120.0
    f = synth.analytic_field(31, n_blob=24, std=(0.04, 0.12), peak=(10.0, 120.0))
    field = renderer.bake_field(f["blobs"], f["colors"], f["jitter"], TAU)
    ind, atl = renderer.bake(N, B, BMIN, EXTENT, sigma_max, field, DEV, flags=renderer.FLAG_ALPHA_ATLAS)
    ind_g, atl_g = ind.cpu().numpy(), atl.cpu().numpy()
    ind_o, atl_o, amax = oracle.bake(N, B, BMIN, EXTENT, sigma_max, f["blobs"], f["colors"], f["jitter"],
                                     alpha_codes=True)
    ambiguous = np.abs(amax - TAU) <= 5e-5 * TAU
    assert (((ind_g >= 0) == (ind_o >= 0)) | ambiguous).all()
    both = (ind_g >= 0) & (ind_o >= 0)
    blocks = np.flatnonzero(both.ravel())
    _, content, raw = oracle.bake_blocks(N, B, BMIN, EXTENT, sigma_max, f["blobs"], f["colors"], f["jitter"], blocks,
                                         alpha_codes=True)
    np.testing.assert_array_equal(content, atl_o[ind_o.ravel()[blocks]])
    _compare_blocks(atl_g[ind_g.ravel()[blocks]], content, raw)
    assert (atl_g[..., 0] > 0).mean() > 0.2
    if np.array_equal(ind_g, ind_o) and np.array_equal(atl_g, atl_o):
        rng = np.random.default_rng(6)
        cams = synth.orbit_cameras(rng, [(40, 40)], synth.CAM_RADIUS)
        mlp = synth.init_mlp(rng)
        sc = synth.custom_scene(N, B, ind_o, atl_o, sigma_max, mlp, cams, bmin=BMIN, extent=EXTENT,
                                flags=renderer.FLAG_ALPHA_ATLAS)
        r = renderer.Renderer.from_scene(sc, DEV)
        pix = synth.all_pixels(cams)
        got = r.render_rays(cams, torch.from_numpy(pix).to(DEV), torch.from_numpy(mlp).to(DEV), counts=True)
        r.check_status()
        ref = oracle.render_rays(sc, pix)
        np.testing.assert_array_equal(got["counts"].cpu().numpy()[:, :2], ref["counts"])
        assert np.abs(got["rgb"].cpu().numpy() - ref["rgb"]).max() <= 1e-4
