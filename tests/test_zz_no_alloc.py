"""snerg_render_rays_noalloc, the ray-list render for callers that cannot allocate
device memory (a plug-in inside an application that owns the GPU's memory through its
own pool, a real-time loop that cannot afford the implicit synchronisation of
cudaMalloc/cudaFree, a sandboxed caller handed only its input and output buffers).

It is checked through the C ABI against the ordinary ray-list entry point
(snerg_render_rays) on two calls in a row. The two calls use grids of different sizes,
so the second one also shows that what the first left in the shared static scratch
does not leak into its result. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2103_14645_gb300 import renderer, synth

pytestmark = pytest.mark.gpu
TOL = 1e-4
DEV = torch.device("cuda:0")


def _desc(sc):
    return renderer.SceneDesc(sc.N, sc.B, (ctypes.c_float * 3)(*sc.bmin), float(sc.extent), float(sc.sigma_max),
                              (ctypes.c_float * 3)(*sc.bg), 0, 0)


def _noalloc_call(lib, sc, ind, atl, pix, mlp, out, status):
    desc = _desc(sc)
    cams = np.ascontiguousarray(sc.cameras, dtype=synth.CAMERA_DTYPE)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    return lib.snerg_render_rays_noalloc(ctypes.byref(desc), ind.data_ptr(), atl.data_ptr(), sc.nb,
                                         cams.ctypes.data, cams.shape[0], pix.data_ptr(), pix.shape[0],
                                         mlp.data_ptr(), out.data_ptr(), status.data_ptr(), stream)


def test_noalloc_matches_render_rays_on_two_calls_in_a_row():
    lib = renderer.load_library()
    cases = []
    for name, n in (("shell1024", 65536), ("gauss64", 4096)):
        sc = synth.make_scene(name)
        pix = torch.from_numpy(synth.random_pixels(np.random.default_rng(17), sc.cameras, n)).to(DEV)
        mlp = torch.from_numpy(sc.mlp).to(DEV)
        r = renderer.Renderer.from_scene(sc, DEV)
        ref = r.render_rays(sc.cameras, pix, mlp)
        r.check_status()
        ind = torch.from_numpy(sc.ind).to(DEV)
        atl = torch.from_numpy(sc.atlas).to(DEV)
        cases.append((sc, ind, atl, pix, mlp, ref))
    for sc, ind, atl, pix, mlp, ref in cases:          # two calls in a row, different grids
        out = torch.full_like(ref, float("nan"))
        status = torch.full((1,), -1, dtype=torch.int32, device=DEV)
        assert _noalloc_call(lib, sc, ind, atl, pix, mlp, out, status) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        err = float((out - ref).abs().max())
        assert err <= TOL, (sc.name, err)


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
    assert code == 5      # SNERG_E_UNSUPPORTED
