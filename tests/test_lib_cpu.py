"""Host-side checks of the C ABI library that need no GPU: it builds, loads, exports
every entry point include/snerg.h declares, sizes workspaces, and rejects invalid
arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2103_14645_gb300 import build, renderer, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "snerg.h")


@pytest.fixture(scope="module")
def lib():
    if build.sources_newer_than_lib():
        build.build()
    return renderer.load_library()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(snerg_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["snerg_create", "snerg_render", "snerg_render_rays", "snerg_render_backward", "snerg_destroy",
              "snerg_workspace_bytes", "snerg_last_status", "snerg_status_str"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(renderer.EXPORTED) == names


def test_nm_shows_c_linkage(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", renderer.LIB_PATH], capture_output=True, text=True).stdout
    for n in declared_functions():
        assert re.search(rf"\bT {n}$", out, flags=re.M), n


def _desc(N=64, B=8, extent=2.0, sigma=10.0):
    return renderer.SceneDesc(N, B, (ctypes.c_float * 3)(-1, -1, -1), extent, sigma, (ctypes.c_float * 3)(1, 1, 1), 0, 0)


def test_workspace_bytes(lib):
    for N, B, nb in [(64, 8, 155), (1024, 32, 1900), (16, 4, 0), (2048, 32, 6281)]:
        d = _desc(N, B)
        got = lib.snerg_workspace_bytes(ctypes.byref(d), nb)
        G, P = N // B, B + 2
        sched = 2 * (4096 + 32 * 65536 * 4)       # the viewer's tile schedule: two sets of buckets
        need = 35 * G ** 3 + 4 * nb + 16 * nb * P ** 3 + sched
        assert need <= got <= need + 8 * 256
        assert got % 256 == 0
    neg = _desc()
    neg.max_steps = -1
    badflag = _desc()
    badflag.flags = 16               # undefined bit
    nomlp_ps = _desc()
    nomlp_ps.flags = 10              # no network and the per-sample network
    combo = _desc()
    combo.flags = 3                  # un-premultiply belongs to the deferred model
    for bad in [_desc(64, 6), _desc(60, 8), _desc(64, 8, extent=0.0), _desc(64, 8, sigma=float("nan")),
                _desc(0, 8), _desc(64 * 1024, 8), _desc(8192, 4), neg, badflag, combo, nomlp_ps]:
        assert lib.snerg_workspace_bytes(ctypes.byref(bad), 10) == 0
    assert lib.snerg_workspace_bytes(ctypes.byref(_desc()), -1) == 0
    assert lib.snerg_workspace_bytes(None, 1) == 0


def test_invalid_arguments_rejected_on_host(lib):
    h = ctypes.c_void_p(123)
    d = _desc()
    assert lib.snerg_create(ctypes.byref(d), None, None, 0, None, 0, None, ctypes.byref(h)) == 1
    assert h.value is None
    bad = _desc(64, 6)
    assert lib.snerg_create(ctypes.byref(bad), 1, 1, 0, 256, 1 << 20, None, ctypes.byref(h)) == 1
    # workspace too small / misaligned
    assert lib.snerg_create(ctypes.byref(d), 256, 256, 1, 256, 16, None, ctypes.byref(h)) == 2
    assert lib.snerg_create(ctypes.byref(d), 256, 256, 1, 257, 1 << 30, None, ctypes.byref(h)) == 1
    cams = np.zeros(1, synth.CAMERA_DTYPE)
    assert lib.snerg_render(None, cams.ctypes.data, 1, None, None, None, None) == 1
    assert lib.snerg_render_rays(None, cams.ctypes.data, 1, None, 0, None, None, None, None) == 1
    assert lib.snerg_render_backward(None, cams.ctypes.data, 1, None, 0, None, None, None, None, None, None, None) == 1
    assert lib.snerg_last_status(None, None) == 1
    assert lib.snerg_requantize_atlas(None, 256, None, None) == 1
    assert lib.snerg_grad_blocks_touched(256, 4, 6, 256, None) == 1          # block_floats not a multiple of 4
    assert lib.snerg_grad_blocks_touched(260, 4, 8, 256, None) == 1          # misaligned
    assert lib.snerg_grad_blocks_gather(256, None, 3, 8, 256, None) == 1     # no list
    assert lib.snerg_grad_blocks_scatter(256, 256, -1, 8, 256, None) == 1
    assert lib.snerg_grad_blocks_gather(None, None, 0, 8, None, None) == 0   # nothing to do
    alpha = _desc()
    alpha.flags = 4                  # the allocation-free entry point renders density atlases only
    assert lib.snerg_render_rays_noalloc(ctypes.byref(alpha), 256, 256, 1, cams.ctypes.data, 1, 256, 1, 256, 256,
                                         None, None) == 1
    assert lib.snerg_launch_count(None) == 0
    lib.snerg_destroy(None)


def test_status_strings(lib):
    for code, text in renderer.STATUS.items():
        assert lib.snerg_status_str(code).decode() == text
    assert lib.snerg_status_str(99).decode() == "unknown status"


def test_camera_record_layout():
    """The numpy camera dtype matches snerg_camera (80 bytes, out_offset at byte 72)."""
    assert synth.CAMERA_DTYPE.itemsize == 80
    assert synth.CAMERA_DTYPE.fields["out_offset"][1] == 72
    assert synth.CAMERA_DTYPE.fields["W"][1] == 64
    assert ctypes.sizeof(renderer.RenderOpts) == 56
    assert ctypes.sizeof(renderer.SceneDesc) == 48


def test_no_cpu_fallback_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(renderer, "_LIB", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        renderer.load_library(str(tmp_path / "missing.so"))


def test_bake_workspace_and_invalid_arguments(lib):
    """snerg_bake sizes its workspace as G^3 flags + G^3 slot list + a header line, refuses
    grids with G > 256, and rejects bad fields and pointers before any CUDA call."""
    for N, B in [(64, 8), (1024, 32), (16, 2), (2048, 8)]:
        G = N // B
        got = lib.snerg_bake_workspace_bytes(ctypes.byref(_desc(N, B)))
        assert 8 * G ** 3 + 256 <= got <= 8 * G ** 3 + 3 * 256 and got % 256 == 0
    for bad in [_desc(4096, 8), _desc(64, 6), _desc(64, 8, sigma=0.0), _desc(64, 8, extent=-1.0)]:
        assert lib.snerg_bake_workspace_bytes(ctypes.byref(bad)) == 0
    assert lib.snerg_bake_workspace_bytes(None) == 0
    f = synth.analytic_field(0, n_blob=8)
    field = renderer.bake_field(f["blobs"], f["colors"], f["jitter"])
    assert ctypes.sizeof(field) == 8 + 64 * 20 + 7 * 16 + 16 * 12
    d = _desc()
    nb = ctypes.c_int64(-1)
    ws = lib.snerg_bake_workspace_bytes(ctypes.byref(d))

    def call(fld, ind=256, atlas=256, maxb=10, wsp=256, wsb=ws, out=ctypes.byref(nb)):
        return lib.snerg_bake(ctypes.byref(d), ctypes.byref(fld) if fld is not None else None, ind, atlas, maxb,
                              wsp, wsb, out, None)

    assert call(None) == 1
    assert call(field, ind=None) == 1
    assert call(field, out=None) == 1
    assert call(field, maxb=-1) == 1
    assert call(field, atlas=None) == 1
    assert call(field, atlas=260) == 1          # atlas not 8-byte aligned
    assert call(field, wsp=None) == 1
    assert call(field, wsp=264) == 1            # workspace not 256-byte aligned
    assert call(field, wsb=ws - 1) == 2
    for mutate in [lambda g: setattr(g, "n_blob", 65), lambda g: setattr(g, "n_blob", -1),
                   lambda g: setattr(g, "tau_alpha", 0.0), lambda g: setattr(g, "tau_alpha", 1.0),
                   lambda g: g.blob[0].__setitem__(3, 0.0), lambda g: g.blob[1].__setitem__(4, -1.0),
                   lambda g: g.blob[2].__setitem__(0, float("inf")), lambda g: g.color[3].__setitem__(1, float("nan")),
                   lambda g: g.jitter[5].__setitem__(2, 8.5)]:
        g = renderer.bake_field(f["blobs"], f["colors"], f["jitter"])
        mutate(g)
        assert call(g) == 1


def test_new_entry_points_reject_bad_arguments_on_host(lib):
    """snerg_train_rays, snerg_render_to_host and the gradient-block helpers validate their
    arguments before touching the device."""
    cams = np.zeros(1, synth.CAMERA_DTYPE)
    cams["fx"] = cams["fy"] = 1.0
    cams["W"] = cams["H"] = 4
    assert lib.snerg_train_rays(None, cams.ctypes.data, 1, 256, 1, 256, 256, None, None, None, None, None) == 1
    assert lib.snerg_render_to_host(None, cams.ctypes.data, 1, None, None, 256, 4, None) == 1
    assert lib.snerg_grad_blocks_scatter(256, None, 2, 8, 256, None) == 1
    assert lib.snerg_grad_blocks_touched(None, 3, 8, 256, None) == 1


def test_binding_validates_host_outputs_without_a_gpu():
    """render_to_host wants a contiguous float32 CPU tensor; these checks run before the
    library is called."""
    import torch
    r = renderer.Renderer.__new__(renderer.Renderer)   # no device state needed for the checks
    r.nb, r.B = 0, 8
    cams = synth.orbit_cameras(np.random.default_rng(0), [(4, 4)], synth.CAM_RADIUS)
    with pytest.raises(ValueError):
        r.render_to_host(cams, torch.empty((16, 3), dtype=torch.float64))
    with pytest.raises(ValueError):
        r.render_to_host(cams, torch.empty((8, 3), dtype=torch.float32))
    with pytest.raises(ValueError):
        r.render_to_host(cams, torch.empty((3, 16), dtype=torch.float32).t())
