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
