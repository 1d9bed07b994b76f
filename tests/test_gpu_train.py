"""The fine-tuning loop of Sec. 5.5 on the GPU: the L2 loss kernel (Eq. 3), the Adam
kernel, and whole steps (render -> loss -> adjoint -> Adam) against the oracle-driven
reference (FP64 render and adjoint, FP64 Adam)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2103_14645_gb300 import renderer, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def test_l2_loss_kernel():
    rng = np.random.default_rng(3)
    n = 100003
    a = rng.uniform(size=(n, 3)).astype(np.float32)
    b = rng.uniform(size=(n, 3)).astype(np.float32)
    ta, tb = torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)
    g = torch.empty_like(ta)
    loss = torch.zeros(1, dtype=torch.float32, device=DEV)
    renderer.l2_loss(ta, tb, g, loss)
    renderer.l2_loss(ta, tb, None, loss)            # accumulates
    d = a.astype(np.float64) - b
    np.testing.assert_array_equal(g.cpu().numpy(), 2.0 * (a - b))
    np.testing.assert_allclose(float(loss.item()), 2 * (d * d).sum(), rtol=1e-5)


def test_adam_kernel_matches_reference():
    rng = np.random.default_rng(4)
    n = 4099
    p0 = rng.normal(size=n)
    grads = rng.normal(size=(5, n)) * np.logspace(-3, 1, n)
    w, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    tp = torch.tensor(p0, dtype=torch.float32, device=DEV)
    tm, tv = torch.zeros_like(tp), torch.zeros_like(tp)
    for k in range(5):
        tg = torch.tensor(grads[k], dtype=torch.float32, device=DEV)
        renderer.adam_step(tp, tm, tv, tg, k + 1, lr=1e-2)
        oracle.adam_step(w, m, v, grads[k].astype(np.float32).astype(np.float64), k + 1, lr=1e-2)
    np.testing.assert_allclose(tp.cpu().numpy(), w, rtol=0, atol=2e-6)


def test_finetune_steps_match_oracle_reference():
    """Five GPU fine-tuning steps vs five oracle-driven steps on the 64^3 grid's 4096 rays:
    the losses agree, and so do the weights whose gradient is not vanishingly small (Adam
    normalises each coordinate, so a coordinate with g ~ 0 may take either sign)."""
    sc = synth.make_scene("gauss64")
    pix_np = synth.all_pixels(sc.cameras)
    target = np.random.default_rng(5).uniform(size=(pix_np.shape[0], 3)).astype(np.float32)
    params, losses = oracle.finetune_steps(sc, pix_np, target, sc.mlp, 5)
    out0 = oracle.render_rays(sc, pix_np)
    _, g0 = oracle.backward_rays(sc, pix_np, 2.0 * (out0["rgb"] - target), atlas_grad=False)
    r = renderer.Renderer.from_scene(sc, DEV)
    ft = renderer.FineTuner(r, sc.mlp)
    pix = torch.from_numpy(pix_np).to(DEV)
    tg = torch.from_numpy(target).to(DEV)
    got_losses = []
    for k in range(5):
        got_losses.append(float(ft.step(sc.cameras, pix, tg).item()))
        r.check_status()
    np.testing.assert_allclose(got_losses, losses, rtol=1e-4)
    significant = np.abs(g0) > 1e-3 * np.abs(g0).max()
    assert significant.sum() > 100
    w = ft.mlp.cpu().numpy()
    assert np.abs(w - params[-1])[significant].max() <= 1e-5
    assert np.abs(w - params[-1]).max() <= 10 * 3e-4
    assert losses[-1] < losses[0]


def test_finetune_recovers_view_dependence():
    """Targets rendered with one set of weights, fine-tuning started from another: the L2
    loss falls by well over half in 150 steps (lr 3e-3) on 65,536 rays of the 512^3 grid."""
    sc = synth.make_scene("bwd512")
    pix = torch.from_numpy(sc.extra["pix"]).to(DEV)
    r = renderer.Renderer.from_scene(sc, DEV)
    w_true = torch.from_numpy(sc.mlp).to(DEV)
    target = r.render_rays(sc.cameras, pix, w_true).clone()
    w0 = synth.init_mlp(np.random.default_rng(99))
    ft = renderer.FineTuner(r, w0, lr=3e-3)
    first = float(ft.step(sc.cameras, pix, target).item())
    for _ in range(149):
        last = ft.step(sc.cameras, pix, target)
    r.check_status()
    assert float(last.item()) < 0.4 * first


def test_requantize_round_trip_leaves_the_render_unchanged():
    """Values q / 255 requantise to the same codes (also in the padded copies), so the
    render after snerg_requantize_atlas is bit-identical, step counts included."""
    sc = synth.make_scene("gauss64")
    r = renderer.Renderer.from_scene(sc, DEV)
    pix = torch.from_numpy(synth.all_pixels(sc.cameras)).to(DEV)
    w = torch.from_numpy(sc.mlp).to(DEV)
    a = r.render_rays(sc.cameras, pix, w, counts=True)
    rgb0, cnt0 = a["rgb"].clone(), a["counts"].clone()
    vals = (torch.from_numpy(sc.atlas).to(DEV).float() / 255.0).contiguous()
    out = torch.empty(sc.atlas.shape, dtype=torch.uint8, device=DEV)
    r.requantize_atlas(vals, out)
    np.testing.assert_array_equal(out.cpu().numpy(), sc.atlas)
    b = r.render_rays(sc.cameras, pix, w, counts=True)
    r.check_status()
    assert torch.equal(b["rgb"], rgb0) and torch.equal(b["counts"], cnt0)


def test_requantize_matches_oracle_codes_and_render():
    """Random values (outside [0, 1] too, garbage in the density channel): the codes equal
    the oracle's binary32 requantisation exactly, density codes stay, and the render from
    the updated padded atlas matches the oracle's render of the new codes (colours to
    1e-4, step counts exactly: density did not move)."""
    sc = synth.make_scene("gauss64")
    r = renderer.Renderer.from_scene(sc, DEV)
    rng = np.random.default_rng(8)
    vals = rng.uniform(-0.1, 1.1, sc.atlas.shape).astype(np.float32)
    out = torch.empty(sc.atlas.shape, dtype=torch.uint8, device=DEV)
    r.requantize_atlas(torch.from_numpy(vals).to(DEV), out)
    want = sc.atlas.copy()
    want[..., 1:] = oracle.requantize(vals[..., 1:])
    got = out.cpu().numpy()
    np.testing.assert_array_equal(got, want)
    pix_np = synth.all_pixels(sc.cameras)
    res = r.render_rays(sc.cameras, torch.from_numpy(pix_np).to(DEV), torch.from_numpy(sc.mlp).to(DEV), counts=True)
    r.check_status()
    ref = oracle.render_rays(synth.custom_scene(sc.N, sc.B, sc.ind, want, sc.sigma_max, sc.mlp, sc.cameras), pix_np)
    np.testing.assert_array_equal(res["counts"].cpu().numpy()[:, :2], ref["counts"])
    assert np.abs(res["rgb"].cpu().numpy() - ref["rgb"]).max() <= 1e-4


def test_finetune_with_shadow_atlas_matches_oracle_reference():
    """Three steps fine-tuning the MLP and the colours/features together (atlas rate
    2/255) against the FP64 shadow-atlas reference: the losses agree; after the first step
    every code whose gradient is clearly non-zero moved exactly as the reference's (Adam's
    first step is a signed step of the rate); after three steps the codes agree to within
    one on those coordinates and within the possible travel elsewhere; density never moves."""
    sc = synth.make_scene("gauss64")
    pix_np = synth.all_pixels(sc.cameras)
    target = np.random.default_rng(5).uniform(size=(pix_np.shape[0], 3)).astype(np.float32)
    alr = 2.0 / 255.0
    _, losses, codes = oracle.finetune_steps(sc, pix_np, target, sc.mlp, 3, atlas_lr=alr)
    out0 = oracle.render_rays(sc, pix_np)
    ga0, _ = oracle.backward_rays(sc, pix_np, 2.0 * (out0["rgb"] - target))
    sig = np.abs(ga0) > 1e-3 * np.abs(ga0).max()
    assert sig.sum() > 1000
    r = renderer.Renderer.from_scene(sc, DEV)
    ft = renderer.FineTuner(r, sc.mlp, atlas=sc.atlas, atlas_lr=alr)
    pix = torch.from_numpy(pix_np).to(DEV)
    tg = torch.from_numpy(target).to(DEV)
    got_losses, got_codes = [], []
    for _ in range(3):
        got_losses.append(float(ft.step(sc.cameras, pix, tg).item()))
        got_codes.append(ft.codes.cpu().numpy().astype(int))
    r.check_status()
    np.testing.assert_allclose(got_losses, losses, rtol=1e-4)
    np.testing.assert_array_equal(got_codes[0][sig], codes[0].astype(int)[sig])
    d = np.abs(got_codes[-1] - codes[-1].astype(int))
    assert d[sig].max() <= 1 and (d[sig] == 0).mean() > 0.99
    assert d.max() <= 2 * 3
    for c in got_codes:
        np.testing.assert_array_equal(c[..., 0], sc.atlas[..., 0])
    assert losses[-1] < losses[0]


def test_gradient_block_exchange_kernels():
    """The touched-block mask, gather and scatter kernels of the data-parallel exchange
    against plain tensor indexing."""
    rng = np.random.default_rng(9)
    nb, B = 37, 8
    g = rng.normal(size=(nb, B, B, B, 8)).astype(np.float32)
    zero = rng.choice(nb, 15, replace=False)
    g[zero] = 0.0
    g[zero[0], 3, 2, 1, 5] = -1e-30                       # one non-zero value keeps a block
    tg = torch.from_numpy(g).to(DEV)
    mask = renderer.GpuBlockOps.touched(tg).cpu().numpy()
    np.testing.assert_array_equal(mask, (g.reshape(nb, -1) != 0).any(1).astype(np.int32))
    idx = torch.from_numpy(np.flatnonzero(mask).astype(np.int32)).to(DEV)
    packed = renderer.GpuBlockOps.gather(tg, idx)
    np.testing.assert_array_equal(packed.cpu().numpy(), g.reshape(nb, -1)[np.flatnonzero(mask)])
    out = torch.zeros_like(tg)
    renderer.GpuBlockOps.scatter(packed * 2.0, idx, out)
    want = np.zeros_like(g)
    want[np.flatnonzero(mask)] = 2.0 * g[np.flatnonzero(mask)]
    np.testing.assert_array_equal(out.cpu().numpy(), want)


@pytest.mark.parametrize("flags", [0, renderer.FLAG_UNPREMULTIPLY, renderer.FLAG_ALPHA_ATLAS, renderer.FLAG_NO_MLP])
def test_train_rays_matches_oracle_and_the_separate_launches(flags):
    """snerg_train_rays (render, L2 loss and adjoint per ray in one launch) against the
    oracle's render and adjoint for dL/dC = 2 (C - C*), and against render_rays +
    l2_loss + backward on the GPU."""
    sc0 = synth.make_scene("gauss64")
    sc = synth.custom_scene(sc0.N, sc0.B, sc0.ind, sc0.atlas, sc0.sigma_max, sc0.mlp, sc0.cameras, flags=flags)
    rng = np.random.default_rng(17)
    pix_np = synth.random_pixels(rng, sc.cameras, 3000)
    target = rng.uniform(size=(pix_np.shape[0], 3)).astype(np.float32)
    r = renderer.Renderer.from_scene(sc, DEV)
    pix = torch.from_numpy(pix_np).to(DEV)
    tg = torch.from_numpy(target).to(DEV)
    w = torch.from_numpy(sc.mlp).to(DEV)
    ga = torch.zeros(sc.atlas.shape, dtype=torch.float32, device=DEV)
    gm = torch.zeros(883, dtype=torch.float32, device=DEV)
    loss = torch.zeros(1, dtype=torch.float32, device=DEV)
    rgb = torch.empty((pix.shape[0], 3), dtype=torch.float32, device=DEV)
    r.train_rays(sc.cameras, pix, w, tg, ga, gm, loss=loss, out=rgb)
    r.check_status()
    o = oracle.render_rays(sc, pix_np)
    d = o["rgb"] - target
    ra, rm = oracle.backward_rays(sc, pix_np, 2.0 * d)
    assert np.abs(rgb.cpu().numpy() - o["rgb"]).max() <= 1e-4
    np.testing.assert_allclose(float(loss.item()), float((d * d).sum()), rtol=1e-4)
    assert np.abs(ga.cpu().numpy() - ra).max() <= 1e-4 * np.abs(ra).max()
    if np.abs(rm).max() > 0:
        assert np.abs(gm.cpu().numpy() - rm).max() <= 1e-4 * np.abs(rm).max()
    else:
        assert (gm.cpu().numpy() == 0).all()
    # the three separate launches
    fwd = r.render_rays(sc.cameras, pix, w, aux=True, counts=True)
    g = torch.empty_like(fwd["rgb"])
    loss2 = torch.zeros(1, dtype=torch.float32, device=DEV)
    renderer.l2_loss(fwd["rgb"], tg, g, loss2)
    ga2 = torch.zeros_like(ga)
    gm2 = torch.zeros_like(gm)
    r.backward(sc.cameras, pix, w, g, ga2, gm2, fwd_aux=fwd["aux"], fwd_counts=fwd["counts"])
    r.check_status()
    assert torch.allclose(rgb, fwd["rgb"], rtol=0, atol=1e-6)
    np.testing.assert_allclose(float(loss.item()), float(loss2.item()), rtol=1e-5)
    assert (ga - ga2).abs().max().item() <= 1e-5 * ga2.abs().max().item()
    assert (gm - gm2).abs().max().item() <= 1e-5 * max(gm2.abs().max().item(), 1e-30)


def test_train_rays_at_the_benchmarked_batch():
    """The one-launch training step in the launch configuration the bench times (the 512^3
    grid, its 65,536 listed rays over 8 views and their targets): colours, loss, atlas and
    MLP gradients against the FP64 oracle."""
    sc = synth.make_scene("bwd512")
    pix_np, target = sc.extra["pix"], sc.extra["target"]
    r = renderer.Renderer.from_scene(sc, DEV)
    pix = torch.from_numpy(pix_np).to(DEV)
    w = torch.from_numpy(sc.mlp).to(DEV)
    ga = torch.zeros(sc.atlas.shape, dtype=torch.float32, device=DEV)
    gm = torch.zeros(883, dtype=torch.float32, device=DEV)
    loss = torch.zeros(1, dtype=torch.float32, device=DEV)
    rgb = torch.empty((pix_np.shape[0], 3), dtype=torch.float32, device=DEV)
    r.train_rays(sc.cameras, pix, w, torch.from_numpy(target).to(DEV), ga, gm, loss=loss, out=rgb)
    r.check_status()
    o = oracle.render_rays(sc, pix_np)
    d = o["rgb"] - target
    ra, rm = oracle.backward_rays(sc, pix_np, 2.0 * d)
    assert np.abs(rgb.cpu().numpy() - o["rgb"]).max() <= 1e-4
    np.testing.assert_allclose(float(loss.item()), float((d * d).sum()), rtol=1e-4)
    assert np.abs(ga.cpu().numpy() - ra).max() <= 1e-4 * np.abs(ra).max()
    assert np.abs(gm.cpu().numpy() - rm).max() <= 1e-4 * np.abs(rm).max()


def test_finetuner_large_batch_takes_the_separate_launches():
    """A batch larger than the fused limit (8 waves of the adjoint kernel; forced here)
    goes through render_rays -> l2_loss -> backward; one step gives the same loss and
    weights as the fused launch."""
    sc = synth.make_scene("gauss64")
    rng = np.random.default_rng(19)
    pix_np = synth.random_pixels(rng, sc.cameras, 4096)
    target = torch.from_numpy(rng.uniform(size=(4096, 3)).astype(np.float32)).to(DEV)
    pix = torch.from_numpy(pix_np).to(DEV)
    r = renderer.Renderer.from_scene(sc, DEV)
    a = renderer.FineTuner(r, sc.mlp)
    b = renderer.FineTuner(r, sc.mlp)
    b.fused_rays = 0
    la = float(a.step(sc.cameras, pix, target).item())
    lb = float(b.step(sc.cameras, pix, target).item())
    np.testing.assert_allclose(la, lb, rtol=1e-5)
    significant = a.grad.abs() > 1e-3 * a.grad.abs().max()
    assert torch.allclose(a.mlp[significant], b.mlp[significant], rtol=0, atol=1e-6)


def test_adam_vector_path_matches_reference():
    """A large parameter array goes through the four-wide kernel (plus a scalar tail for a
    length not divisible by four); the result equals the FP64 reference Adam to FP32."""
    rng = np.random.default_rng(23)
    n = 100_003
    p0 = rng.normal(size=n)
    grads = rng.normal(size=(3, n)) * np.logspace(-3, 1, n)
    w, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    tp = torch.tensor(p0, dtype=torch.float32, device=DEV)
    tm, tv = torch.zeros_like(tp), torch.zeros_like(tp)
    for k in range(3):
        tg = torch.tensor(grads[k], dtype=torch.float32, device=DEV)
        renderer.adam_step(tp, tm, tv, tg, k + 1, lr=1e-2)
        oracle.adam_step(w, m, v, grads[k].astype(np.float32).astype(np.float64), k + 1, lr=1e-2)
    np.testing.assert_allclose(tp.cpu().numpy(), w, rtol=0, atol=2e-6)
