"""FP64 CPU oracle for the SNeRG deferred volume render.

TEST INFRASTRUCTURE ONLY: this package may be imported by `tests/`, by
`__graft_entry__.smoke()` and by the CPU-baseline leg of `bench.py`, and by nothing in
the product path. It shares no code with the CUDA renderer; the only thing both sides
consume is the seeded input generator (`paper_2103_14645_gb300.synth`), which holds none
of the method's arithmetic, and this wrapper reads scenes from it by attribute only.

The arithmetic lives in `snerg_oracle.c` (plain C, FP64 colour arithmetic, binary32
integer decisions in a fixed operation order, `-ffp-contract=off`); every function there
cites the paper passage it follows (Sec. 4.2 Eqs. 2, 5-7; Sec. 5.1-5.2; App. A; Sec. 5.5;
the bake of Sec. 5.3-5.4).

Parity pins (tests/test_oracle_pins.py) tie it to closed forms, invariants, library
routines and brute force on tiny grids. No function here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snerg_oracle.c")
_SO = os.path.join(_HERE, "libsnerg_oracle.so")
_LIB = None

NPARAM = 883
MLP_IN = 34


def build_oracle(verbose: bool = False) -> str:
    """Compile the oracle with gcc. -ffp-contract=off keeps every binary32 operation a
    single rounding (aarch64 GCC would otherwise contract a*b+c to fma)."""
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, capture_output=not verbose)
    os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            build_oracle()
        lib = ctypes.CDLL(_SO)
        P, i32, i64, f32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
        common = [i32, i32, P, f32, f64, P, P, P, P, i64, i32, P, P, i32, P, i64]
        lib.oracle_render_rays.argtypes = common + [P, P, P, P, i32]
        lib.oracle_render_rays.restype = ctypes.c_int
        lib.oracle_backward_rays.argtypes = common + [P, P, P]
        lib.oracle_backward_rays.restype = ctypes.c_int
        lib.oracle_mlp_eval.argtypes = [P, P, i64, P]
        lib.oracle_mlp_eval.restype = None
        lib.oracle_mlp_input.argtypes = [P, P, P, P]
        lib.oracle_mlp_input.restype = None
        lib.oracle_ray.argtypes = [i32, f32, P, P, i32, i32, P]
        lib.oracle_ray.restype = ctypes.c_int
        lib.oracle_bake.argtypes = [i32, i32, P, f32, f32, f32, i32, P, P, P, P, P, i64, P, i32]
        lib.oracle_bake.restype = ctypes.c_int64
        lib.oracle_bake_blocks.argtypes = [i32, i32, P, f32, f32, i32, P, P, P, i64, P, P, P, P, i32]
        lib.oracle_bake_blocks.restype = None
        lib.oracle_requantize.argtypes = [P, i64, P]
        lib.oracle_requantize.restype = None
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = None
        _LIB = lib
    return _LIB


class OracleError(RuntimeError):
    pass


def _p(a):
    return None if a is None else a.ctypes.data


def cameras_f32(cams) -> np.ndarray:
    """Camera records -> float32 [n][16] = c2w (12), fx, fy, cx, cy."""
    out = np.zeros((len(cams), 16), np.float32)
    for i, c in enumerate(cams):
        out[i, :12] = np.asarray(c["c2w"], np.float32).reshape(-1)
        out[i, 12:] = [c["fx"], c["fy"], c["cx"], c["cy"]]
    return out


def _scene_args(scene, val, mlp, cams):
    # the scene description carries binary32 fields; read them at that precision
    bmin = np.asarray(scene.bmin, np.float32)
    bg = np.asarray(scene.bg, np.float32).astype(np.float64)
    ind = np.ascontiguousarray(scene.ind, np.int32)
    atlas = np.ascontiguousarray(scene.atlas, np.uint8)
    if val is not None:
        val = np.ascontiguousarray(val, np.float64)
        assert val.size == atlas.size
    w = np.ascontiguousarray(scene.mlp if mlp is None else mlp, np.float64)
    assert w.size == NPARAM
    cf = cameras_f32(scene.cameras if cams is None else cams)
    keep = (bmin, bg, ind, atlas, val, w, cf)
    flags = int(getattr(scene, "flags", 0))
    args = [int(scene.N), int(scene.B), _p(bmin), float(np.float32(scene.extent)),
            float(np.float32(scene.sigma_max)), _p(bg),
            _p(ind), _p(atlas), _p(val), int(atlas.shape[0]), flags, _p(w), _p(cf), int(cf.shape[0])]
    return args, keep


def render_rays(scene, pix, mlp=None, val=None, cams=None, trace_cap: int = 0):
    """Render rays pix[n][3] = (camera, x, y). Returns a dict with
    rgb [n,3] f64, aux [n,8] f64 (C_d, V, acc before any un-premultiply), counts [n,2]
    int32 (steps, active) and,
    when trace_cap > 0, trace [n,trace_cap] uint64 (visited voxel indices, 0-padded)."""
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 3)
    n = pix.shape[0]
    args, keep = _scene_args(scene, val, mlp, cams)
    rgb = np.zeros((n, 3), np.float64)
    aux = np.zeros((n, 8), np.float64)
    counts = np.zeros((n, 2), np.int32)
    trace = np.zeros((n, trace_cap), np.uint64) if trace_cap > 0 else None
    st = _lib().oracle_render_rays(*args, _p(pix), n, _p(rgb), _p(aux), _p(counts), _p(trace), int(trace_cap))
    if st:
        raise OracleError(f"oracle_render_rays status {st}")
    out = {"rgb": rgb, "aux": aux, "counts": counts}
    if trace is not None:
        out["trace"] = trace
    return out


def render_image(scene, cam_index: int = 0, mlp=None, val=None):
    """Full image of one camera as [H, W, 3] f64 (plus aux/counts reshaped)."""
    c = scene.cameras[cam_index]
    W, H = int(c["W"]), int(c["H"])
    y, x = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    pix = np.stack([np.full(W * H, cam_index), x.ravel(), y.ravel()], 1).astype(np.int32)
    out = render_rays(scene, pix, mlp=mlp, val=val)
    return {k: v.reshape(H, W, -1) for k, v in out.items()}


def backward_rays(scene, pix, g_rgb, mlp=None, val=None, cams=None, atlas_grad=True):
    """Adjoint for upstream dL/dC g_rgb[n,3]. Returns (grad_val [nb,B,B,B,8] f64 with
    channel 0 zero, or None when atlas_grad is False; grad_mlp [883] f64)."""
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 3)
    g = np.ascontiguousarray(g_rgb, np.float64).reshape(-1, 3)
    assert g.shape[0] == pix.shape[0]
    args, keep = _scene_args(scene, val, mlp, cams)
    grad = np.zeros(scene.atlas.shape, np.float64) if atlas_grad else None
    gmlp = np.zeros(NPARAM, np.float64)
    st = _lib().oracle_backward_rays(*args, _p(pix), pix.shape[0], _p(g), _p(grad), _p(gmlp))
    if st:
        raise OracleError(f"oracle_backward_rays status {st}")
    return grad, gmlp


def mlp_eval(mlp, x):
    """sigmoid(MLP(x)) for x[n,34] (FP64)."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, MLP_IN)
    w = np.ascontiguousarray(mlp, np.float64)
    out = np.zeros((x.shape[0], 3), np.float64)
    _lib().oracle_mlp_eval(_p(w), _p(x), x.shape[0], _p(out))
    return out


def mlp_input(cd, v, d):
    cd = np.ascontiguousarray(cd, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    d = np.ascontiguousarray(d, np.float32)
    x = np.zeros(MLP_IN, np.float64)
    _lib().oracle_mlp_input(_p(cd), _p(v), _p(d), _p(x))
    return x


def ray(scene, cam, px: int, py: int):
    """(hit, o[3], d[3], t_start, t_end) of one pixel, in voxel units (binary32)."""
    cf = cameras_f32([cam])[0]
    bmin = np.asarray(scene.bmin, np.float32)
    out = np.zeros(8, np.float32)
    hit = _lib().oracle_ray(int(scene.N), float(scene.extent), _p(bmin), _p(cf), int(px), int(py), _p(out))
    return bool(hit), out[0:3].copy(), out[3:6].copy(), float(out[6]), float(out[7])


def adam_step(param, m, v, grad, step, lr=3e-4, betas=(0.9, 0.999), eps=1e-8):
    """Reference Adam update in FP64 (Kingma & Ba), in place on numpy arrays; the
    optimiser of the paper's fine-tuning (Sec. 5.5)."""
    b1, b2 = betas
    m *= b1
    m += (1 - b1) * grad
    v *= b2
    v += (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    param -= lr * mh / (np.sqrt(vh) + eps)
    return param


def requantize(x) -> np.ndarray:
    """8-bit codes of float32 values (Sec. 5.4): floor(255 x + 1/2) clamped, decided in
    binary32."""
    x = np.ascontiguousarray(x, np.float32)
    out = np.zeros(x.shape, np.uint8)
    _lib().oracle_requantize(_p(x), x.size, _p(out))
    return out


def finetune_steps(scene, pix, target, mlp, steps, lr=3e-4, atlas_lr=None):
    """`steps` fine-tuning steps of the MLP with the oracle's render and adjoint and the
    reference Adam; returns (the parameter after each step, the loss before each step).

    With atlas_lr, the colour and feature values are fine-tuned too: an FP64 shadow copy
    of the decoded atlas (initialised from binary32 q / 255) takes Adam steps on the
    adjoint's atlas gradient, and after each step channels 1..7 of the atlas are
    requantised from it (density codes stay frozen). The render of the next step reads
    the requantised codes. Then the third return value is the codes after each step."""
    w = np.asarray(mlp, np.float64).copy()
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    codes = np.ascontiguousarray(scene.atlas, np.uint8).copy()
    sc = scene
    if atlas_lr is not None:
        shadow = (codes.astype(np.float32) / np.float32(255.0)).astype(np.float64)
        ma = np.zeros_like(shadow)
        va = np.zeros_like(shadow)
    params, losses, history = [], [], []
    for t in range(1, steps + 1):
        out = render_rays(sc, pix, mlp=w)
        d = out["rgb"] - np.asarray(target, np.float64)
        losses.append(float((d * d).sum()))
        ga, g = backward_rays(sc, pix, 2.0 * d, mlp=w, atlas_grad=atlas_lr is not None)
        adam_step(w, m, v, g, t, lr)
        params.append(w.copy())
        if atlas_lr is not None:
            adam_step(shadow, ma, va, ga, t, atlas_lr)
            codes = codes.copy()
            codes[..., 1:] = requantize(shadow[..., 1:])
            sc = _with_atlas(scene, codes)
            history.append(codes)
    if atlas_lr is not None:
        return params, losses, history
    return params, losses


def _with_atlas(scene, codes):
    import copy
    sc = copy.copy(scene)
    sc.atlas = codes
    return sc


def bake(N, B, bmin, extent, sigma_max, blobs, colors, jitter, tau_alpha=0.005, max_blocks=None,
         alpha_codes=False):
    """FP64 bake of the analytic field (Sec. 5.3): returns (ind [G,G,G] int32,
    atlas [nb,B,B,B,8] uint8, block max alpha [G,G,G] f64). With alpha_codes, channel 0
    stores alpha = 1 - exp(-sigma v) of the averaged density instead of sigma / sigma_max."""
    G = N // B
    blobs = np.ascontiguousarray(blobs, np.float32).reshape(-1, 5)
    colors = np.ascontiguousarray(colors, np.float32).reshape(7, 4)
    jitter = np.ascontiguousarray(jitter, np.float32).reshape(16, 3)
    bmin = np.asarray(bmin, np.float32)
    max_blocks = G ** 3 if max_blocks is None else max_blocks
    ind = np.zeros((G, G, G), np.int32)
    atlas = np.zeros((max_blocks, B, B, B, 8), np.uint8)
    amax = np.zeros((G, G, G), np.float64)
    nb = _lib().oracle_bake(int(N), int(B), _p(bmin), float(np.float32(extent)), float(np.float32(sigma_max)),
                            float(np.float32(tau_alpha)), blobs.shape[0], _p(blobs), _p(colors), _p(jitter),
                            _p(ind), _p(atlas), int(max_blocks), _p(amax), int(bool(alpha_codes)))
    if nb < 0:
        raise OracleError("more kept blocks than max_blocks")
    return ind, atlas[:nb].copy(), amax


def bake_blocks(N, B, bmin, extent, sigma_max, blobs, colors, jitter, blocks, alpha_codes=False):
    """Maximum alpha and 8-bit content of the listed macroblocks (raster indices
    b = x + G (y + G z)), kept or not: (alpha [n] f64, content [n,B,B,B,8] uint8,
    raw [n,B,B,B,8] f64 = 255 x before rounding)."""
    blobs = np.ascontiguousarray(blobs, np.float32).reshape(-1, 5)
    colors = np.ascontiguousarray(colors, np.float32).reshape(7, 4)
    jitter = np.ascontiguousarray(jitter, np.float32).reshape(16, 3)
    blocks = np.ascontiguousarray(blocks, np.int64)
    bmin = np.asarray(bmin, np.float32)
    amax = np.zeros(blocks.shape[0], np.float64)
    content = np.zeros((blocks.shape[0], B, B, B, 8), np.uint8)
    raw = np.zeros((blocks.shape[0], B, B, B, 8), np.float64)
    _lib().oracle_bake_blocks(int(N), int(B), _p(bmin), float(np.float32(extent)), float(np.float32(sigma_max)),
                              blobs.shape[0], _p(blobs), _p(colors), _p(jitter), blocks.shape[0], _p(blocks),
                              _p(amax), _p(content), _p(raw), int(bool(alpha_codes)))
    return amax, content, raw


def threads() -> int:
    """Threads the oracle's parallel loops use."""
    return int(_lib().oracle_threads())


def set_threads(n: int) -> None:
    """Threads for the oracle's later parallel loops (calling thread)."""
    _lib().oracle_set_threads(int(n))
