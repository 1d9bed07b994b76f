"""snerg_render_rays_noalloc, the ray-list render for callers that cannot allocate
device memory (a plug-in inside an application that owns the GPU's memory through its
own pool, a real-time loop that cannot afford the implicit synchronisation of
cudaMalloc/cudaFree, a sandboxed caller handed only its input and output buffers).

It is checked through the C ABI against the ordinary ray-list entry point
(snerg_render_rays) on two calls in a row, and against the FP64 oracle on the same rays:
its march is separate code (it reads the caller's unpadded atlas through the
indirection grid), so the oracle is what pins it. The two calls use grids of different
sizes, so the second one also shows that what the first left in the shared static
scratch does not leak into its result. Further cases: the device status for a pixel
outside its camera and for an indirection entry past the atlas (reported, the rest of
the rays unchanged), the un-premultiply flag, an empty ray list, and a grid beyond the
static scratch. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2103_14645_gb300 import renderer, synth

pytestmark = pytest.mark.gpu
TOL = 1e-4
DEV = torch.device("cuda:0")
OK, E_INVAL, E_UNSUPPORTED = 0, 1, 5


def _desc(sc, flags=0):
    return renderer.SceneDesc(sc.N, sc.B, (ctypes.c_float * 3)(*sc.bmin), float(sc.extent), float(sc.sigma_max),
                              (ctypes.c_float * 3)(*sc.bg), 0, int(flags))


def _noalloc_call(lib, sc, ind, atl, pix, mlp, out, status, flags=0):
    desc = _desc(sc, flags)
    cams = np.ascontiguousarray(sc.cameras, dtype=synth.CAMERA_DTYPE)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    return lib.snerg_render_rays_noalloc(ctypes.byref(desc), ind.data_ptr(), atl.data_ptr(), sc.nb,
                                         cams.ctypes.data, cams.shape[0], pix.data_ptr(), pix.shape[0],
                                         mlp.data_ptr(), out.data_ptr(), status.data_ptr(), stream)


def _reference(sc, pix_np, flags=0):
    """snerg_render_rays on the same scene (with the same scene flags) and rays."""
    scene = synth.custom_scene(sc.N, sc.B, sc.ind, sc.atlas, sc.sigma_max, sc.mlp, sc.cameras, flags=flags) \
        if flags else sc
    r = renderer.Renderer.from_scene(scene, DEV)
    pix = torch.from_numpy(pix_np).to(DEV)
    ref = r.render_rays(scene.cameras, pix, torch.from_numpy(sc.mlp).to(DEV))
    r.check_status()
    return ref


def _call(lib, sc, pix_np, ind_np=None, flags=0):
    ind = torch.from_numpy(np.ascontiguousarray(sc.ind if ind_np is None else ind_np, np.int32)).to(DEV)
    atl = torch.from_numpy(sc.atlas).to(DEV)
    pix = torch.from_numpy(pix_np).to(DEV)
    mlp = torch.from_numpy(sc.mlp).to(DEV)
    out = torch.full((pix_np.shape[0], 3), float("nan"), dtype=torch.float32, device=DEV)
    status = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    code = _noalloc_call(lib, sc, ind, atl, pix, mlp, out, status, flags)
    torch.cuda.synchronize()
    return code, out, int(status.item())


def test_noalloc_matches_render_rays_and_the_oracle_on_two_calls_in_a_row():
    lib = renderer.load_library()
    cases = []
    for name, n in (("shell1024", 65536), ("gauss64", 4096)):
        sc = synth.make_scene(name)
        pix_np = synth.random_pixels(np.random.default_rng(17), sc.cameras, n)
        cases.append((sc, pix_np, _reference(sc, pix_np)))
    for sc, pix_np, ref in cases:                      # two calls in a row, different grids
        code, out, status = _call(lib, sc, pix_np)
        assert code == OK and status == OK
        err = float((out - ref).abs().max())
        assert err <= TOL, (sc.name, err)
        # the FP64 oracle on the same rays (a seeded subset of the 1024^3 grid's rays)
        sub = np.arange(0, pix_np.shape[0], 4 if sc.N > 256 else 1)
        want = oracle.render_rays(sc, pix_np[sub])["rgb"]
        err_o = float(np.abs(out.cpu().numpy()[sub].astype(np.float64) - want).max())
        assert err_o <= TOL, (sc.name, err_o)


def test_noalloc_unpremultiply_flag():
    lib = renderer.load_library()
    sc = synth.make_scene("gauss64")
    pix_np = synth.random_pixels(np.random.default_rng(5), sc.cameras, 4096)
    ref = _reference(sc, pix_np, flags=renderer.FLAG_UNPREMULTIPLY)
    code, out, status = _call(lib, sc, pix_np, flags=renderer.FLAG_UNPREMULTIPLY)
    assert code == OK and status == OK
    assert float((out - ref).abs().max()) <= TOL
    plain = _reference(sc, pix_np)
    assert float((ref - plain).abs().max()) > 1e-3        # the flag changes these pixels


def test_noalloc_reports_a_pixel_outside_its_camera():
    lib = renderer.load_library()
    sc = synth.make_scene("gauss64")
    pix_np = synth.random_pixels(np.random.default_rng(6), sc.cameras, 1024)
    ref = _reference(sc, pix_np)
    bad = pix_np.copy()
    bad[100] = (0, int(sc.cameras[0]["W"]), 0)            # x = W: outside the image
    code, out, status = _call(lib, sc, bad)
    assert code == OK and status == E_INVAL
    keep = np.ones(bad.shape[0], bool)
    keep[100] = False
    assert float((out[torch.from_numpy(keep).to(DEV)] - ref[torch.from_numpy(keep).to(DEV)]).abs().max()) <= TOL
    # the bad ray misses: background only
    assert np.allclose(out[100].cpu().numpy(), np.asarray(sc.bg, np.float32))


def test_noalloc_reports_an_entry_past_the_atlas_and_reads_it_as_empty():
    lib = renderer.load_library()
    sc = synth.make_scene("gauss64")
    pix_np = synth.random_pixels(np.random.default_rng(7), sc.cameras, 4096)
    ref = _reference(sc, pix_np)
    ind = np.array(sc.ind, np.int32)
    ind[ind < 0] = sc.nb                                   # every empty block now names a missing slot
    code, out, status = _call(lib, sc, pix_np, ind_np=ind)
    assert code == OK and status == E_INVAL
    assert float((out - ref).abs().max()) <= TOL


def test_noalloc_empty_ray_list():
    lib = renderer.load_library()
    sc = synth.make_scene("tiny")
    ind = torch.from_numpy(np.ascontiguousarray(sc.ind, np.int32)).to(DEV)
    atl = torch.from_numpy(sc.atlas).to(DEV)
    status = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    desc = _desc(sc)
    cams = np.ascontiguousarray(sc.cameras, dtype=synth.CAMERA_DTYPE)
    code = lib.snerg_render_rays_noalloc(ctypes.byref(desc), ind.data_ptr(), atl.data_ptr(), sc.nb,
                                         cams.ctypes.data, cams.shape[0], None, 0, None, None, status.data_ptr(),
                                         torch.cuda.current_stream(DEV).cuda_stream)
    torch.cuda.synchronize()
    assert code == OK and int(status.item()) == OK


def test_noalloc_rejects_grids_beyond_its_static_scratch():
    lib = renderer.load_library()
    sc = synth.make_scene("tiny")
    big = synth.custom_scene(8192, 64, np.zeros((1, 1, 1), np.int32), sc.atlas[:0], sc.sigma_max, sc.mlp,
                             sc.cameras)       # N / B = 128 > 64
    dummy = torch.zeros(16, dtype=torch.int32, device=DEV)
    desc = _desc(big)
    cams = np.ascontiguousarray(sc.cameras, dtype=synth.CAMERA_DTYPE)
    code = lib.snerg_render_rays_noalloc(ctypes.byref(desc), dummy.data_ptr(), None, 0, cams.ctypes.data, 1,
                                         dummy.data_ptr(), 1, dummy.data_ptr(), dummy.data_ptr(), None, None)
    assert code == E_UNSUPPORTED
