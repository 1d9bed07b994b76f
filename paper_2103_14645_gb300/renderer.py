"""Python binding of libsnerg.so (include/snerg.h): argument marshalling only.

Every step of the render and its adjoint runs in the library's CUDA kernels; PyTorch
supplies device memory and the current stream. There is no fallback: if the library is
missing or the device is not a CUDA GPU, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsnerg.so")
MLP_PARAMS = 883
FLAG_UNPREMULTIPLY = 1
FLAG_PER_SAMPLE_MLP = 2
FLAG_ALPHA_ATLAS = 4
FLAG_NO_MLP = 8
MAX_CAMERAS = 256
AUX_CH = 8

STATUS = {0: "ok", 1: "invalid argument", 2: "buffer too small", 3: "CUDA error",
          4: "a ray exceeded its iteration cap", 5: "unsupported", 6: "device fault"}

EXPORTED = ["snerg_workspace_bytes", "snerg_create", "snerg_render", "snerg_render_rays",
            "snerg_render_backward", "snerg_last_status", "snerg_launch_count",
            "snerg_persistent_config", "snerg_destroy", "snerg_status_str", "snerg_render_rays_noalloc",
            "snerg_set_mlp", "snerg_l2_loss", "snerg_adam_step", "snerg_bake_workspace_bytes", "snerg_bake",
            "snerg_requantize_atlas", "snerg_grad_blocks_touched", "snerg_grad_blocks_gather",
            "snerg_grad_blocks_scatter", "snerg_render_to_host", "snerg_train_rays", "snerg_schedule_stats"]
MAX_BAKE_BLOBS = 64


class SnergError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} (status {code})")
        self.code = code


class SceneDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("B", ctypes.c_int32), ("bmin", ctypes.c_float * 3),
                ("extent", ctypes.c_float), ("sigma_max", ctypes.c_float), ("bg", ctypes.c_float * 3),
                ("max_steps", ctypes.c_int32), ("flags", ctypes.c_int32)]


class RenderOpts(ctypes.Structure):
    _fields_ = [("d_aux", ctypes.c_void_p), ("d_counts", ctypes.c_void_p), ("d_trace", ctypes.c_void_p),
                ("trace_cap", ctypes.c_int32), ("persistent", ctypes.c_int32), ("tile_w", ctypes.c_int32),
                ("tile_h", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("row_begin", ctypes.c_int32),
                ("row_end", ctypes.c_int32), ("schedule", ctypes.c_int32)]


class BakeField(ctypes.Structure):
    _fields_ = [("n_blob", ctypes.c_int32), ("tau_alpha", ctypes.c_float),
                ("blob", (ctypes.c_float * 5) * MAX_BAKE_BLOBS), ("color", (ctypes.c_float * 4) * 7),
                ("jitter", (ctypes.c_float * 3) * 16)]


_LIB = None


def load_library(path: str = LIB_PATH):
    """Load libsnerg.so (raises if it has not been built: there is no CPU path)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2103_14645_gb300.build.build() "
                           "(the renderer has no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.snerg_workspace_bytes.argtypes = [P, i64]
    lib.snerg_workspace_bytes.restype = ctypes.c_size_t
    lib.snerg_create.argtypes = [P, P, P, i64, P, ctypes.c_size_t, P, P]
    lib.snerg_create.restype = ctypes.c_int
    lib.snerg_render.argtypes = [P, P, i32, P, P, P, P]
    lib.snerg_render.restype = ctypes.c_int
    lib.snerg_render_rays.argtypes = [P, P, i32, P, i64, P, P, P, P]
    lib.snerg_render_rays.restype = ctypes.c_int
    lib.snerg_render_backward.argtypes = [P, P, i32, P, i64, P, P, P, P, P, P, P]
    lib.snerg_render_backward.restype = ctypes.c_int
    lib.snerg_last_status.argtypes = [P, P]
    lib.snerg_last_status.restype = ctypes.c_int
    lib.snerg_launch_count.argtypes = [P]
    lib.snerg_launch_count.restype = ctypes.c_int64
    lib.snerg_persistent_config.argtypes = [P, P, P, P]
    lib.snerg_persistent_config.restype = ctypes.c_int
    lib.snerg_destroy.argtypes = [P]
    lib.snerg_destroy.restype = None
    lib.snerg_status_str.argtypes = [ctypes.c_int]
    lib.snerg_status_str.restype = ctypes.c_char_p
    lib.snerg_l2_loss.argtypes = [P, P, i64, P, P, P]
    lib.snerg_l2_loss.restype = ctypes.c_int
    lib.snerg_adam_step.argtypes = [P, P, P, P, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, i32, P]
    lib.snerg_adam_step.restype = ctypes.c_int
    lib.snerg_set_mlp.argtypes = [P, P]
    lib.snerg_set_mlp.restype = ctypes.c_int
    lib.snerg_render_rays_noalloc.argtypes = [P, P, P, i64, P, i32, P, i64, P, P, P, P]
    lib.snerg_render_rays_noalloc.restype = ctypes.c_int
    lib.snerg_train_rays.argtypes = [P, P, i32, P, i64, P, P, P, P, P, P, P]
    lib.snerg_train_rays.restype = ctypes.c_int
    lib.snerg_schedule_stats.argtypes = [P, P, P, P]
    lib.snerg_schedule_stats.restype = ctypes.c_int
    lib.snerg_render_to_host.argtypes = [P, P, i32, P, P, P, i32, P]
    lib.snerg_render_to_host.restype = ctypes.c_int
    lib.snerg_grad_blocks_touched.argtypes = [P, i64, i32, P, P]
    lib.snerg_grad_blocks_touched.restype = ctypes.c_int
    lib.snerg_grad_blocks_gather.argtypes = [P, P, i64, i32, P, P]
    lib.snerg_grad_blocks_gather.restype = ctypes.c_int
    lib.snerg_grad_blocks_scatter.argtypes = [P, P, i64, i32, P, P]
    lib.snerg_grad_blocks_scatter.restype = ctypes.c_int
    lib.snerg_requantize_atlas.argtypes = [P, P, P, P]
    lib.snerg_requantize_atlas.restype = ctypes.c_int
    lib.snerg_bake_workspace_bytes.argtypes = [P]
    lib.snerg_bake_workspace_bytes.restype = ctypes.c_size_t
    lib.snerg_bake.argtypes = [P, P, P, P, i64, P, ctypes.c_size_t, P, P]
    lib.snerg_bake.restype = ctypes.c_int
    _LIB = lib
    return lib


def _check(code: int, where: str):
    if code != 0:
        raise SnergError(code, where)


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _cams(cams, limit: bool = True) -> np.ndarray:
    """Cameras as the ABI's records; ray-list calls take at most MAX_CAMERAS (limit)."""
    c = np.ascontiguousarray(cams, dtype=synth.CAMERA_DTYPE).reshape(-1)
    if c.shape[0] < 1 or (limit and c.shape[0] > MAX_CAMERAS):
        raise ValueError(f"1..{MAX_CAMERAS if limit else 'any'} cameras per call, got {c.shape[0]}")
    return c


def _require_cuda(t: torch.Tensor, name: str, dtype):
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor")


class Renderer:
    """A baked SNeRG scene resident on one GPU (snerg_create) and its render calls."""

    def __init__(self, N: int, B: int, bmin, extent: float, sigma_max: float, bg,
                 indirection: torch.Tensor, atlas: torch.Tensor, max_steps: int = 0, flags: int = 0):
        self.lib = load_library()
        _require_cuda(indirection, "indirection", torch.int32)
        _require_cuda(atlas, "atlas", torch.uint8)
        self.device = atlas.device if atlas.numel() else indirection.device
        self.N, self.B = int(N), int(B)
        self.nb = int(atlas.shape[0]) if atlas.dim() > 0 else 0
        self.desc = SceneDesc(self.N, self.B, (ctypes.c_float * 3)(*bmin), float(extent),
                              float(sigma_max), (ctypes.c_float * 3)(*bg), int(max_steps), int(flags))
        nbytes = self.lib.snerg_workspace_bytes(ctypes.byref(self.desc), self.nb)
        if nbytes == 0:
            raise ValueError("invalid scene description")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            code = self.lib.snerg_create(ctypes.byref(self.desc), _ptr(indirection), _ptr(atlas), self.nb,
                                         _ptr(self.workspace), nbytes, _stream(self.device), ctypes.byref(h))
        _check(code, "snerg_create")
        self.handle = h

    @classmethod
    def from_scene(cls, scene, device="cuda", max_steps: int = 0) -> "Renderer":
        ind = torch.from_numpy(np.ascontiguousarray(scene.ind, np.int32)).to(device)
        atl = torch.from_numpy(np.ascontiguousarray(scene.atlas, np.uint8)).to(device)
        return cls(scene.N, scene.B, scene.bmin, scene.extent, scene.sigma_max, scene.bg, ind, atl, max_steps,
                   int(getattr(scene, "flags", 0)))

    # ---------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None):
            self.lib.snerg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self) -> int:
        return int(self.lib.snerg_launch_count(self.handle))

    def schedule_stats(self):
        """(tiles rendered sparsely, 1 if the previous order was used) of the last render
        with schedule=True (snerg_schedule_stats; synchronises)."""
        sp, od = ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib.snerg_schedule_stats(self.handle, _stream(self.device), ctypes.byref(sp), ctypes.byref(od)),
               "snerg_schedule_stats")
        return sp.value, od.value

    def persistent_config(self):
        tw, th, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib.snerg_persistent_config(self.handle, ctypes.byref(tw), ctypes.byref(th), ctypes.byref(c)),
               "snerg_persistent_config")
        return tw.value, th.value, c.value

    def set_mlp(self, weights):
        """Store host MLP weights in the handle; renders called with mlp=None use them as
        kernel parameters (snerg_set_mlp)."""
        w = np.ascontiguousarray(np.asarray(weights, np.float32).reshape(-1))
        if w.size != MLP_PARAMS:
            raise ValueError(f"{MLP_PARAMS} weights expected")
        _check(self.lib.snerg_set_mlp(self.handle, w.ctypes.data), "snerg_set_mlp")

    def check_status(self):
        """Synchronise and raise if a kernel recorded a device-side error."""
        _check(self.lib.snerg_last_status(self.handle, _stream(self.device)), "device status")

    def requantize_atlas(self, values: torch.Tensor, atlas_out: torch.Tensor | None = None):
        """Write fine-tuned colour/feature values (float32 [nb,B,B,B,8], channel 0 ignored)
        into the scene as 8-bit codes (snerg_requantize_atlas); optionally also into
        atlas_out (uint8, same shape, density codes in channel 0)."""
        _require_cuda(values, "values", torch.float32)
        if tuple(values.shape) != (self.nb, self.B, self.B, self.B, 8):
            raise ValueError("values must have the atlas shape [nb, B, B, B, 8]")
        if atlas_out is not None:
            _require_cuda(atlas_out, "atlas_out", torch.uint8)
            if atlas_out.shape != values.shape:
                raise ValueError("atlas_out must have the atlas shape")
        _check(self.lib.snerg_requantize_atlas(self.handle, _ptr(values), _ptr(atlas_out), _stream(self.device)),
               "snerg_requantize_atlas")

    def _opts(self, n_pix, aux, counts, trace_cap, persistent, tile, ctas_per_sm):
        out = {}
        o = RenderOpts()
        if aux:
            out["aux"] = torch.empty((n_pix, AUX_CH), dtype=torch.float32, device=self.device)
            o.d_aux = out["aux"].data_ptr()
        if counts:
            out["counts"] = torch.empty((n_pix, 4), dtype=torch.int32, device=self.device)
            o.d_counts = out["counts"].data_ptr()
        if trace_cap > 0:
            out["trace"] = torch.zeros((n_pix, trace_cap), dtype=torch.int64, device=self.device)
            o.d_trace = out["trace"].data_ptr()
            o.trace_cap = trace_cap
        o.persistent = 1 if persistent else 0
        if tile is not None:
            o.tile_w, o.tile_h = int(tile[0]), int(tile[1])
        o.ctas_per_sm = int(ctas_per_sm)
        return o, out

    def render(self, cams, mlp: torch.Tensor | None, out: torch.Tensor | None = None, aux=False, counts=False,
               trace_cap: int = 0, persistent=False, tile=None, ctas_per_sm: int = 0, rows=None,
               schedule: bool = False):
        """Render every pixel of the cameras into out [pixels, 3] (packed by out_offset), a
        device tensor or a pinned host tensor (written by the kernels through the mapping).
        mlp: device weights, or None for the weights stored with set_mlp.
        rows: (begin, end) renders only those image rows of every camera.
        schedule: launch the tiles in the order of the costs this handle recorded on its last
        scheduled render of an image of the same size (a viewer's consecutive frames), and
        record this render's costs (snerg_render_opts.schedule; one camera only).
        Returns out, or a dict with 'rgb' and the requested debug outputs."""
        c = _cams(cams, limit=False)
        if mlp is not None:
            _require_cuda(mlp, "mlp", torch.float32)
        n_pix = int(max((int(x["out_offset"]) + int(x["W"]) * int(x["H"]) for x in c), default=0))
        if out is None:
            out = torch.empty((n_pix, 3), dtype=torch.float32, device=self.device)
        else:
            if out.device.type == "cpu":
                # pinned host memory is mapped for the device: the kernels store into it
                if not out.is_pinned() or out.dtype != torch.float32 or not out.is_contiguous():
                    raise ValueError("a host out must be a contiguous pinned float32 tensor")
            else:
                _require_cuda(out, "out", torch.float32)
            if out.numel() < 3 * n_pix:
                raise ValueError("out is too small")
        o, extra = self._opts(n_pix, aux, counts, trace_cap, persistent, tile, ctas_per_sm)
        if rows is not None:
            o.row_begin, o.row_end = int(rows[0]), int(rows[1])
        o.schedule = 1 if schedule else 0
        code = self.lib.snerg_render(self.handle, c.ctypes.data, c.shape[0], _ptr(mlp), _ptr(out),
                                     ctypes.byref(o), _stream(self.device))
        _check(code, "snerg_render")
        if extra:
            extra["rgb"] = out
            return extra
        return out

    def render_to_host(self, cams, host_out: torch.Tensor, mlp: torch.Tensor | None = None,
                       out: torch.Tensor | None = None, bands: int = 4):
        """Render the cameras into host memory host_out [pixels, 3] (float32, contiguous) with
        snerg_render_to_host. Pinned host_out: the kernels write the pixels straight into it
        (no copy after the render). Pageable host_out: `bands` row bands rendered into the
        device image `out` (allocated if None) on the library's side streams, each copied out
        as soon as it is done. Enqueued after the current stream's work; host_out is complete
        once the current stream is synchronised."""
        c = _cams(cams, limit=False)
        if host_out.device.type != "cpu" or host_out.dtype != torch.float32 or not host_out.is_contiguous():
            raise ValueError("host_out must be a contiguous float32 CPU tensor")
        if mlp is not None:
            _require_cuda(mlp, "mlp", torch.float32)
        n_pix = int(max((int(x["out_offset"]) + int(x["W"]) * int(x["H"]) for x in c), default=0))
        if host_out.numel() < 3 * n_pix:
            raise ValueError("host_out is too small")
        if out is None and not host_out.is_pinned():
            out = torch.empty((n_pix, 3), dtype=torch.float32, device=self.device)
        elif out is not None:
            _require_cuda(out, "out", torch.float32)
            if out.numel() < 3 * n_pix:
                raise ValueError("out is too small")
        with torch.cuda.device(self.device):
            code = self.lib.snerg_render_to_host(self.handle, c.ctypes.data, c.shape[0], _ptr(mlp), _ptr(out),
                                                 host_out.data_ptr(), int(bands), _stream(self.device))
        _check(code, "snerg_render_to_host")
        return host_out

    def render_rays(self, cams, pix: torch.Tensor, mlp: torch.Tensor | None, out=None, aux=False, counts=False,
                    trace_cap: int = 0):
        c = _cams(cams)
        _require_cuda(pix, "pix", torch.int32)
        if mlp is not None:
            _require_cuda(mlp, "mlp", torch.float32)
        n = int(pix.shape[0])
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32, device=self.device)
        o, extra = self._opts(n, aux, counts, trace_cap, False, None, 0)
        code = self.lib.snerg_render_rays(self.handle, c.ctypes.data, c.shape[0], _ptr(pix), n, _ptr(mlp),
                                          _ptr(out), ctypes.byref(o), _stream(self.device))
        _check(code, "snerg_render_rays")
        if extra:
            extra["rgb"] = out
            return extra
        return out

    def backward(self, cams, pix: torch.Tensor, mlp: torch.Tensor, grad_rgb: torch.Tensor,
                 grad_atlas: torch.Tensor | None = None, grad_mlp: torch.Tensor | None = None,
                 fwd_aux: torch.Tensor | None = None, fwd_counts: torch.Tensor | None = None):
        """Accumulate dL/d(atlas values) [nb,B,B,B,8] and dL/d(mlp) [883] for dL/dC.
        fwd_aux / fwd_counts: the aux and counts outputs of the render_rays call that
        produced C (then the rays are marched once instead of twice)."""
        c = _cams(cams)
        _require_cuda(pix, "pix", torch.int32)
        _require_cuda(mlp, "mlp", torch.float32)
        _require_cuda(grad_rgb, "grad_rgb", torch.float32)
        if grad_atlas is not None:
            _require_cuda(grad_atlas, "grad_atlas", torch.float32)
            if grad_atlas.numel() != self.nb * self.B ** 3 * 8:
                raise ValueError("grad_atlas must have nb*B^3*8 elements")
        if grad_mlp is not None:
            _require_cuda(grad_mlp, "grad_mlp", torch.float32)
        if (fwd_aux is None) != (fwd_counts is None):
            raise ValueError("fwd_aux and fwd_counts go together")
        if fwd_aux is not None:
            _require_cuda(fwd_aux, "fwd_aux", torch.float32)
            _require_cuda(fwd_counts, "fwd_counts", torch.int32)
        code = self.lib.snerg_render_backward(self.handle, c.ctypes.data, c.shape[0], _ptr(pix), int(pix.shape[0]),
                                              _ptr(mlp), _ptr(grad_rgb), _ptr(fwd_aux), _ptr(fwd_counts),
                                              _ptr(grad_atlas), _ptr(grad_mlp), _stream(self.device))
        _check(code, "snerg_render_backward")



def _train_rays(self, cams, pix: torch.Tensor, mlp: torch.Tensor, target: torch.Tensor,
                grad_atlas: torch.Tensor | None, grad_mlp: torch.Tensor | None,
                loss: torch.Tensor | None = None, out: torch.Tensor | None = None):
    """One fine-tuning step's render, L2 loss (added to `loss`) and adjoint (accumulated
    into grad_atlas / grad_mlp) for the rays pix [n,3] with observed colours target [n,3],
    in one launch (snerg_train_rays); C goes to `out` when given."""
    c = _cams(cams)
    _require_cuda(pix, "pix", torch.int32)
    _require_cuda(mlp, "mlp", torch.float32)
    _require_cuda(target, "target", torch.float32)
    n = int(pix.shape[0])
    if target.numel() != 3 * n:
        raise ValueError("target must be [n, 3]")
    for name, t in (("grad_atlas", grad_atlas), ("grad_mlp", grad_mlp), ("loss", loss), ("out", out)):
        if t is not None:
            _require_cuda(t, name, torch.float32)
    if grad_atlas is not None and grad_atlas.numel() != self.nb * self.B ** 3 * 8:
        raise ValueError("grad_atlas must have the atlas shape")
    code = self.lib.snerg_train_rays(self.handle, c.ctypes.data, c.shape[0], _ptr(pix), n, _ptr(mlp), _ptr(target),
                                     _ptr(out), _ptr(loss), _ptr(grad_atlas), _ptr(grad_mlp), _stream(self.device))
    _check(code, "snerg_train_rays")


Renderer.train_rays = _train_rays


class SnergRenderFn(torch.autograd.Function):
    """C(rays) with gradients to the MLP weights and to the decoded atlas values.

    `atlas_values` stands for the decoded colour/feature values q/255 (shape
    [nb, B, B, B, 8]) of the atlas the renderer was created with; the forward pass reads
    the uint8 atlas inside the renderer, and backward returns dL/d(atlas_values) with the
    density channel (0) frozen at zero."""

    @staticmethod
    def forward(ctx, mlp, atlas_values, renderer, cams, pix):
        ctx.renderer = renderer
        ctx.cams = cams
        ctx.atlas_shape = atlas_values.shape
        out = renderer.render_rays(cams, pix, mlp.detach().contiguous(), aux=True, counts=True)
        # per-ray state (C_d, V, first composited index) for the backward's single march
        ctx.save_for_backward(mlp, pix, out["aux"], out["counts"])
        return out["rgb"]

    @staticmethod
    def backward(ctx, grad_rgb):
        mlp, pix, aux, counts = ctx.saved_tensors
        r = ctx.renderer
        g_mlp = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=r.device) if ctx.needs_input_grad[0] else None
        g_atl = (torch.zeros(ctx.atlas_shape, dtype=torch.float32, device=r.device)
                 if ctx.needs_input_grad[1] else None)
        if g_mlp is not None or g_atl is not None:
            r.backward(ctx.cams, pix, mlp.detach().contiguous(), grad_rgb.contiguous().float(), g_atl, g_mlp,
                       fwd_aux=aux, fwd_counts=counts)
        return g_mlp, g_atl, None, None, None


def render_rays_autograd(renderer: Renderer, cams, pix: torch.Tensor, mlp: torch.Tensor,
                         atlas_values: torch.Tensor) -> torch.Tensor:
    return SnergRenderFn.apply(mlp, atlas_values, renderer, cams, pix)


def l2_loss(rgb: torch.Tensor, target: torch.Tensor, grad: torch.Tensor | None = None,
            loss: torch.Tensor | None = None):
    """Eq. 3 on the GPU (snerg_l2_loss): accumulates sum |C - C*|^2 into `loss` (float32
    [1]) and writes dL/dC = 2 (C - C*) into `grad`."""
    lib = load_library()
    _require_cuda(rgb, "rgb", torch.float32)
    _require_cuda(target, "target", torch.float32)
    n = rgb.numel() // 3
    _check(lib.snerg_l2_loss(_ptr(rgb), _ptr(target), n, _ptr(grad), _ptr(loss), _stream(rgb.device)),
           "snerg_l2_loss")


def adam_step(param: torch.Tensor, m: torch.Tensor, v: torch.Tensor, grad: torch.Tensor, step: int,
              lr: float = 3e-4, betas=(0.9, 0.999), eps: float = 1e-8):
    """One in-place Adam step on the GPU (snerg_adam_step)."""
    lib = load_library()
    for t, name in ((param, "param"), (m, "m"), (v, "v"), (grad, "grad")):
        _require_cuda(t, name, torch.float32)
    _check(lib.snerg_adam_step(_ptr(param), _ptr(m), _ptr(v), _ptr(grad), param.numel(), float(lr), float(betas[0]),
                               float(betas[1]), float(eps), int(step), _stream(param.device)), "snerg_adam_step")


class GpuBlockOps:
    """The library's kernels behind the touched-block exchange of atlas gradients."""

    @staticmethod
    def touched(grad_atlas: torch.Tensor) -> torch.Tensor:
        nb = int(grad_atlas.shape[0])
        bf = grad_atlas[0].numel() if nb else 0
        mask = torch.empty(nb, dtype=torch.int32, device=grad_atlas.device)
        _check(load_library().snerg_grad_blocks_touched(_ptr(grad_atlas), nb, bf, _ptr(mask),
                                                        _stream(grad_atlas.device)), "snerg_grad_blocks_touched")
        return mask

    @staticmethod
    def gather(grad_atlas: torch.Tensor, idx: torch.Tensor) -> torch.Tensor:
        bf = grad_atlas[0].numel()
        packed = torch.empty((idx.numel(), bf), dtype=torch.float32, device=grad_atlas.device)
        _check(load_library().snerg_grad_blocks_gather(_ptr(grad_atlas), _ptr(idx), idx.numel(), bf, _ptr(packed),
                                                       _stream(grad_atlas.device)), "snerg_grad_blocks_gather")
        return packed

    @staticmethod
    def scatter(packed: torch.Tensor, idx: torch.Tensor, grad_atlas: torch.Tensor):
        bf = grad_atlas[0].numel()
        _check(load_library().snerg_grad_blocks_scatter(_ptr(packed), _ptr(idx), idx.numel(), bf, _ptr(grad_atlas),
                                                        _stream(grad_atlas.device)), "snerg_grad_blocks_scatter")


def allreduce_gradients(grad_mlp: torch.Tensor, grad_atlas: torch.Tensor | None = None, group=None,
                        ops=GpuBlockOps) -> int:
    """The exchange step of data-parallel fine-tuning: sum dL/dPhi over the ranks, and the
    atlas gradient over the union of the macroblocks any rank touched (mask all-reduced
    with MAX, touched blocks packed, summed, scattered back; blocks no rank touched stay
    zero on every rank). Returns the number of blocks exchanged. `ops` supplies the
    touched-mask / gather / scatter steps (the library's kernels by default)."""
    import torch.distributed as dist
    dist.all_reduce(grad_mlp, group=group)
    if grad_atlas is None or grad_atlas.shape[0] == 0:
        return 0
    mask = ops.touched(grad_atlas)
    dist.all_reduce(mask, op=dist.ReduceOp.MAX, group=group)
    idx = torch.nonzero(mask).flatten().to(torch.int32).contiguous()
    if idx.numel() == 0:
        return 0
    packed = ops.gather(grad_atlas, idx)
    dist.all_reduce(packed, group=group)
    ops.scatter(packed, idx, grad_atlas)
    return int(idx.numel())


class FineTuner:
    """Fine-tunes the view-dependence MLP of a baked grid against observed pixels with
    Adam and the L2 loss, as the paper does after baking (Sec. 5.5: Adam, learning rate
    3e-4). One step = the rays' render, L2 loss and adjoint (one launch of snerg_train_rays
    up to 8 waves of the adjoint kernel; render_rays -> l2_loss -> backward for larger
    batches) -> Adam, all in the library's kernels.

    With `atlas` (the scene's uint8 atlas [nb,B,B,B,8]) and `atlas_lr`, the baked colours
    and features are fine-tuned too: an FP32 shadow copy (q / 255) takes Adam steps on the
    backward's atlas gradient (zero on the density channel, which stays frozen) and is
    requantised into the scene's 8-bit codes after every step.

    Data parallel: when torch.distributed is initialised with more than one rank (or
    `group` names such a group), each rank passes its own rays and the gradients are summed
    over the ranks (allreduce_gradients) before the identical optimiser step on every rank;
    the returned loss is the rank's own."""

    def __init__(self, renderer: Renderer, mlp, lr: float = 3e-4, betas=(0.9, 0.999), eps: float = 1e-8,
                 atlas=None, atlas_lr: float | None = None, group=None):
        self.r = renderer
        self.group = group
        self.mlp = torch.as_tensor(np.asarray(mlp, np.float32)).to(renderer.device).contiguous()
        self.m = torch.zeros_like(self.mlp)
        self.v = torch.zeros_like(self.mlp)
        self.grad = torch.zeros_like(self.mlp)
        self.loss = torch.zeros(1, dtype=torch.float32, device=renderer.device)
        self.lr, self.betas, self.eps = lr, betas, eps
        self.steps = 0
        # 8 waves of the adjoint kernel (4 CTAs of 128 rays per SM): up to there the one-launch
        # step is the faster (0.69 vs 0.74 ms for 262,144 rays at 2048^3); at 16 waves the two
        # forms are within 1 %
        self.fused_rays = 8 * 4 * 128 * torch.cuda.get_device_properties(renderer.device).multi_processor_count
        self.atlas_lr = atlas_lr
        self.shadow = None
        if atlas_lr is not None:
            if atlas is None:
                raise ValueError("atlas_lr needs the scene's atlas")
            codes = torch.as_tensor(np.asarray(atlas, np.uint8)).to(renderer.device)
            self.shadow = (codes.float() / 255.0).contiguous()
            self.ma = torch.zeros_like(self.shadow)
            self.va = torch.zeros_like(self.shadow)
            self.grad_atlas = torch.zeros_like(self.shadow)
            self.codes = torch.empty_like(codes)

    def step(self, cams, pix: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
        """One Adam step on rays pix [n,3] with observed colours target [n,3]; returns the
        loss before the step (a device tensor [1])."""
        self.loss.zero_()
        self.grad.zero_()
        ga = None
        if self.shadow is not None:
            self.grad_atlas.zero_()
            ga = self.grad_atlas
        if pix.shape[0] <= self.fused_rays:
            # render, loss and adjoint of every ray in one launch: one launch tail replaces
            # two, and no per-ray forward state goes through memory
            self.r.train_rays(cams, pix, self.mlp, target, ga, self.grad, loss=self.loss)
        else:
            # larger batches: the forward at its own (higher) occupancy, keeping per-ray state
            fwd = self.r.render_rays(cams, pix, self.mlp, aux=True, counts=True)
            g = torch.empty_like(fwd["rgb"])
            l2_loss(fwd["rgb"], target, g, self.loss)
            self.r.backward(cams, pix, self.mlp, g, ga, self.grad, fwd_aux=fwd["aux"], fwd_counts=fwd["counts"])
        if _data_parallel(self.group):
            allreduce_gradients(self.grad, ga, self.group)
        self.steps += 1
        adam_step(self.mlp, self.m, self.v, self.grad, self.steps, self.lr, self.betas, self.eps)
        if self.shadow is not None:
            adam_step(self.shadow, self.ma, self.va, self.grad_atlas, self.steps, self.atlas_lr, self.betas, self.eps)
            self.r.requantize_atlas(self.shadow, self.codes)
        return self.loss


def _data_parallel(group) -> bool:
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1


def bake_field(blobs, colors, jitter, tau_alpha: float = 0.005) -> BakeField:
    """Pack an analytic field (blobs [n,5] = centre xyz, std, peak; colors [7,4] = w xyz,
    phi; jitter [16,3] in voxel units) into the snerg_bake_field struct."""
    blobs = np.asarray(blobs, np.float32).reshape(-1, 5)
    if blobs.shape[0] > MAX_BAKE_BLOBS:
        raise ValueError(f"at most {MAX_BAKE_BLOBS} blobs")
    f = BakeField()
    f.n_blob = blobs.shape[0]
    f.tau_alpha = float(tau_alpha)
    ctypes.memmove(f.blob, np.ascontiguousarray(blobs).ctypes.data, blobs.nbytes)
    ctypes.memmove(f.color, np.ascontiguousarray(colors, np.float32).reshape(7, 4).ctypes.data, 7 * 4 * 4)
    ctypes.memmove(f.jitter, np.ascontiguousarray(jitter, np.float32).reshape(16, 3).ctypes.data, 16 * 3 * 4)
    return f


def bake(N: int, B: int, bmin, extent: float, sigma_max: float, field: BakeField, device="cuda",
         max_blocks: int | None = None, flags: int = 0):
    """Bake an analytic field into (indirection int32 [G,G,G], atlas uint8 [nb,B,B,B,8]) on
    the GPU with snerg_bake (Sec. 5.3-5.4). With max_blocks None the atlas is sized by a
    first call that only counts the kept blocks. flags = FLAG_ALPHA_ATLAS stores alpha
    codes in channel 0."""
    lib = load_library()
    device = torch.device(device)
    if device.type != "cuda":
        raise ValueError("bake needs a CUDA device")
    desc = SceneDesc(int(N), int(B), (ctypes.c_float * 3)(*bmin), float(extent), float(sigma_max),
                     (ctypes.c_float * 3)(0, 0, 0), 0, int(flags))
    nbytes = lib.snerg_bake_workspace_bytes(ctypes.byref(desc))
    if nbytes == 0:
        raise ValueError("invalid scene description for baking")
    G = N // B
    ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
    ind = torch.empty((G, G, G), dtype=torch.int32, device=device)
    nb = ctypes.c_int64(0)
    with torch.cuda.device(device):
        st = _stream(device)
        if max_blocks is None:
            code = lib.snerg_bake(ctypes.byref(desc), ctypes.byref(field), _ptr(ind), None, 0, _ptr(ws), nbytes,
                                  ctypes.byref(nb), st)
            if code not in (0, 2):
                _check(code, "snerg_bake")
            max_blocks = nb.value
        atlas = torch.empty((max_blocks, B, B, B, 8), dtype=torch.uint8, device=device)
        code = lib.snerg_bake(ctypes.byref(desc), ctypes.byref(field), _ptr(ind), _ptr(atlas) if max_blocks else None,
                              int(max_blocks), _ptr(ws), nbytes, ctypes.byref(nb), st)
    _check(code, "snerg_bake")
    return ind, atlas[:nb.value]
