"""Pins of the oracle's 8-bit requantisation (Sec. 5.4) and of its fine-tuning reference
with an FP32 shadow atlas (Sec. 5.5 extended to the baked colours and features), on CPU."""
import numpy as np
import pytest

import oracle
from paper_2103_14645_gb300 import synth


def test_requantize_matches_exact_rounding_off_the_boundaries():
    """floor(255 x + 1/2) with the product and sum exact in FP64 (x is binary32, so 255 x
    has at most 32 significant bits) equals the binary32 decision except where the exact
    value lies within half a binary32 ulp at 256 (2^-16) of an integer; clamped to
    [0, 255]; NaN -> 0."""
    rng = np.random.default_rng(0)
    x = rng.uniform(-0.1, 1.1, 1_000_000).astype(np.float32)
    y = x.astype(np.float64) * 255.0 + 0.5
    want = np.clip(np.floor(y), 0, 255).astype(np.uint8)
    got = oracle.requantize(x)
    far = np.abs(y - np.round(y)) > 2.0 ** -16
    assert far.mean() > 0.999
    np.testing.assert_array_equal(got[far], want[far])
    assert (np.abs(got.astype(int) - want.astype(int)) <= 1).all()
    special = np.array([np.nan, -np.inf, np.inf, -1.0, 2.0, 0.0, 1.0], np.float32)
    np.testing.assert_array_equal(oracle.requantize(special), [0, 0, 255, 0, 255, 0, 255])


def test_requantize_round_trips_every_code():
    q = np.arange(256)
    np.testing.assert_array_equal(oracle.requantize(q.astype(np.float32) / np.float32(255.0)), q)


def _small_scene():
    sc = synth.make_scene("gauss64")
    pix = synth.all_pixels(sc.cameras)[::3]
    return sc, pix


def test_finetune_with_zero_atlas_rate_is_the_mlp_only_loop():
    sc, pix = _small_scene()
    target = np.random.default_rng(1).uniform(size=(pix.shape[0], 3))
    p0, l0 = oracle.finetune_steps(sc, pix, target, sc.mlp, 3)
    p1, l1, codes = oracle.finetune_steps(sc, pix, target, sc.mlp, 3, atlas_lr=0.0)
    np.testing.assert_array_equal(l0, l1)
    # the adjoint's MLP gradient sums in another order when atlas gradients are taken too
    np.testing.assert_allclose(p0[-1], p1[-1], rtol=0, atol=1e-12)
    for c in codes:
        np.testing.assert_array_equal(c, sc.atlas)


def test_first_atlas_step_moves_each_code_by_the_rate_against_the_gradient():
    """Adam's first step is -lr * g / (|g| + eps): with lr = 3/255 every colour/feature code
    whose gradient is not tiny moves by exactly 3 against the gradient's sign (clamped to
    [0, 255]); codes with zero gradient and all density codes stay."""
    sc, pix = _small_scene()
    target = np.random.default_rng(2).uniform(size=(pix.shape[0], 3))
    out = oracle.render_rays(sc, pix)
    ga, _ = oracle.backward_rays(sc, pix, 2.0 * (out["rgb"] - target))
    _, _, codes = oracle.finetune_steps(sc, pix, target, sc.mlp, 1, lr=0.0, atlas_lr=3.0 / 255.0)
    c1 = codes[0].astype(int)
    c0 = sc.atlas.astype(int)
    np.testing.assert_array_equal(c1[..., 0], c0[..., 0])
    big = np.abs(ga) > 1e-6
    big[..., 0] = False
    assert big.sum() > 1000
    want = np.clip(c0 - 3 * np.sign(ga).astype(int), 0, 255)
    np.testing.assert_array_equal(c1[big], want[big])
    zero = ga == 0
    np.testing.assert_array_equal(c1[zero], c0[zero])


def test_atlas_finetuning_recovers_shifted_colours():
    """Targets rendered from an atlas whose colour codes were shifted by +24: fine-tuning the
    shadow atlas (MLP frozen) lowers the loss by more than half in 8 steps."""
    sc, pix = _small_scene()
    shifted = sc.atlas.copy()
    shifted[..., 1:4] = np.clip(shifted[..., 1:4].astype(int) + 24, 0, 255).astype(np.uint8)
    tsc = synth.custom_scene(sc.N, sc.B, sc.ind, shifted, sc.sigma_max, sc.mlp, sc.cameras)
    target = oracle.render_rays(tsc, pix)["rgb"]
    _, losses, codes = oracle.finetune_steps(sc, pix, target, sc.mlp, 8, lr=0.0, atlas_lr=4.0 / 255.0)
    assert losses[-1] < 0.5 * losses[0]
    np.testing.assert_array_equal(codes[-1][..., 0], sc.atlas[..., 0])
