"""Seeded synthetic SNeRG scenes (input generator shared by the renderer and the oracle).

This module draws every random input of the test and benchmark workloads: the baked
grid (indirection + uint8 atlas), the view-dependence MLP weights, camera poses and
ray lists. It holds none of the renderer's arithmetic. The paper's datasets (NeRF
Synthetic 360 degrees, Sec. 6) are not available, so these grids stand in for them,
with the sizes and structure of the paper's baked representation (Sec. 5.1: an N^3
virtual grid stored as an (N/B)^3 indirection grid into an atlas of B^3 macroblocks,
8 bits per value, Sec. 5.4).

Recipes (all seeded):
  * "gauss": density = sum of 16 isotropic Gaussians (centres U[0.15,0.85]^3 of the
    cube, std U[0.04,0.12], amplitude U[0.5,1]), cut to zero below the block-maximum
    quantile that leaves the target fraction of blocks occupied.
  * "shells": density = exp(-(d/1 voxel)^2) around the closed surfaces of random
    spheres and axis-aligned ellipsoids (hollow inside), added until the target block
    occupancy is reached.
  * colour/feature channels: 0.5 + 0.5 sin(w.p + phi) with seeded w, phi.
  * Blocks are culled when their maximum opacity 1 - exp(-sigma * v) is below
    tau_alpha = 0.005 (Sec. 5.3), then packed into the atlas in a seeded order.
"""
from __future__ import annotations

import ctypes
import hashlib
import math
import os
from dataclasses import dataclass, field

import numpy as np

MLP_IN = 34          # 3 diffuse + 4 feature + 27 positional encoding of the view direction
MLP_HID = 16
MLP_OUT = 3
MLP_SIZES = [(MLP_HID, MLP_IN), (MLP_HID,), (MLP_HID, MLP_HID), (MLP_HID,), (MLP_OUT, MLP_HID), (MLP_OUT,)]
MLP_NPARAM = sum(int(np.prod(s)) for s in MLP_SIZES)   # 883
TAU_ALPHA = 0.005    # block culling threshold on opacity, Sec. 5.3

# Camera record shared with the C ABI (snerg_camera in include/snerg.h): 80 bytes.
CAMERA_DTYPE = np.dtype([
    ("c2w", np.float32, (12,)),   # row-major 3x4 camera-to-world; camera looks along -z
    ("fx", np.float32), ("fy", np.float32), ("cx", np.float32), ("cy", np.float32),
    ("W", np.int32), ("H", np.int32),
    ("out_offset", np.int64),     # first output pixel of this camera in the packed image
], align=True)
assert CAMERA_DTYPE.itemsize == 80

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = os.path.join(_HERE, "libsnerg_synth.so")
        if not os.path.exists(path):
            build_synth()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.synth_density.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, P,
                                      ctypes.c_int32, ctypes.c_int32, P, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, P, P]
        lib.synth_density.restype = None
        lib.synth_colors.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, P, P, P]
        lib.synth_colors.restype = None
        _LIB = lib
    return _LIB


def build_synth(verbose: bool = False) -> str:
    """Compile the C volume filler in place (gcc, OpenMP)."""
    import subprocess
    src = os.path.join(_HERE, "synth_fill.c")
    out = os.path.join(_HERE, "libsnerg_synth.so")
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True, capture_output=not verbose)
    os.replace(tmp, out)
    return out


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Scene:
    """A baked grid plus the draws that go with it. Arrays are host numpy arrays."""
    name: str
    N: int
    B: int
    bmin: tuple
    extent: float
    sigma_max: float
    bg: tuple
    ind: np.ndarray            # int32 [G, G, G] (z, y, x); -1 = empty, else atlas slot
    atlas: np.ndarray          # uint8 [nb, B, B, B, 8] (z, y, x, channel)
    mlp: np.ndarray            # float32 [883]
    cameras: np.ndarray        # CAMERA_DTYPE [n_cams]
    extra: dict = field(default_factory=dict)
    flags: int = 0             # bit 0: partial un-premultiply after compositing (App. C)

    @property
    def G(self) -> int:
        return self.N // self.B

    @property
    def nb(self) -> int:
        return int(self.atlas.shape[0])

    @property
    def occupancy(self) -> float:
        return self.nb / float(self.G ** 3)

    @property
    def n_pixels(self) -> int:
        return int(sum(int(c["W"]) * int(c["H"]) for c in self.cameras))

    def checksum(self) -> str:
        """SHA-256 (first 16 hex digits) over the grid description, the indirection grid,
        the atlas codes, the MLP weights and the cameras: identifies the synthetic input."""
        h = hashlib.sha256()
        h.update(np.asarray([self.N, self.B], np.int64).tobytes())
        h.update(np.asarray([*self.bmin, self.extent, self.sigma_max, *self.bg], np.float64).tobytes())
        for a in (self.ind, self.atlas, self.mlp, self.cameras):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()[:16]


def init_mlp(rng: np.random.Generator) -> np.ndarray:
    """Seeded weights U(+-1/sqrt(fan_in)) in the flat layout W1[16][34], b1[16],
    W2[16][16], b2[16], W3[3][16], b3[3] (row-major, out x in)."""
    parts = []
    fan_ins = [MLP_IN, MLP_IN, MLP_HID, MLP_HID, MLP_HID, MLP_HID]
    for s, fan_in in zip(MLP_SIZES, fan_ins):
        bound = 1.0 / math.sqrt(fan_in)
        parts.append(rng.uniform(-bound, bound, size=int(np.prod(s))))
    return np.concatenate(parts).astype(np.float32)


def look_at_camera(pos, target, W: int, H: int, fov_deg: float, out_offset: int = 0) -> np.ndarray:
    """Pinhole camera at `pos` looking at `target`, world up +z, horizontal FOV fov_deg."""
    pos = np.asarray(pos, np.float64)
    fwd = np.asarray(target, np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    up_w = np.array([0.0, 0.0, 1.0])
    if abs(float(fwd @ up_w)) > 0.999:
        up_w = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up_w)
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    R = np.stack([right, up, -fwd], axis=1)      # columns: camera x, y, z in world
    c2w = np.concatenate([R, pos[:, None]], axis=1)
    cam = np.zeros((), CAMERA_DTYPE)
    cam["c2w"] = c2w.reshape(-1).astype(np.float32)
    f = 0.5 * W / math.tan(math.radians(fov_deg) * 0.5)
    cam["fx"] = f
    cam["fy"] = f
    cam["cx"] = 0.5 * W
    cam["cy"] = 0.5 * H
    cam["W"] = W
    cam["H"] = H
    cam["out_offset"] = out_offset
    return cam


def orbit_cameras(rng: np.random.Generator, sizes, radius: float, fov_deg: float = 39.0) -> np.ndarray:
    """Cameras on a sphere around the grid centre at seeded directions (elevation in
    [-50, 70] degrees), images packed one after another in the output."""
    cams = np.zeros(len(sizes), CAMERA_DTYPE)
    off = 0
    for i, (W, H) in enumerate(sizes):
        az = rng.uniform(0.0, 2.0 * math.pi)
        el = math.radians(rng.uniform(-50.0, 70.0))
        pos = radius * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        cams[i] = look_at_camera(pos, (0.0, 0.0, 0.0), W, H, fov_deg, off)
        off += W * H
    return cams


def _color_freqs(rng):
    fr = np.zeros((7, 4))
    fr[:, :3] = rng.uniform(-12.0, 12.0, size=(7, 3))
    fr[:, 3] = rng.uniform(0.0, 2.0 * math.pi, size=7)
    return fr


def _q_min_occupied(sigma_max_vox: float) -> int:
    """Smallest density code whose opacity 1 - exp(-sigma v) reaches tau_alpha."""
    for q in range(1, 256):
        if 1.0 - math.exp(-q / 255.0 * sigma_max_vox) >= TAU_ALPHA:
            return q
    return 256


def _blocks_xyz(G: int) -> np.ndarray:
    z, y, x = np.meshgrid(np.arange(G), np.arange(G), np.arange(G), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.int32)   # raster order z,y,x


def _fill(N, B, blocks, mode, params, width, cut, scale):
    nblk = blocks.shape[0]
    atlas = np.zeros((nblk, B, B, B, 8), np.uint8)
    bmax = np.zeros(nblk, np.uint8)
    if nblk:
        prm = np.ascontiguousarray(params, np.float64)
        _lib().synth_density(N, B, nblk, _ptr(blocks), mode, prm.shape[0], _ptr(prm), width, cut,
                             scale, _ptr(atlas), _ptr(bmax))
    return atlas, bmax


def _pack(N, B, blocks, atlas, bmax, qmin, rng, freqs):
    """Cull blocks below tau_alpha, colour the survivors, pack in a seeded order."""
    G = N // B
    keep = np.nonzero(bmax >= qmin)[0]
    order = rng.permutation(keep.shape[0])
    sel = keep[order]
    blocks_kept = np.ascontiguousarray(blocks[sel])
    atl = np.ascontiguousarray(atlas[sel])
    if sel.shape[0]:
        fr = np.ascontiguousarray(freqs, np.float64)
        _lib().synth_colors(N, B, sel.shape[0], _ptr(blocks_kept), _ptr(fr), _ptr(atl))
    ind = np.full((G, G, G), -1, np.int32)
    ind[blocks_kept[:, 2], blocks_kept[:, 1], blocks_kept[:, 0]] = np.arange(sel.shape[0], dtype=np.int32)
    return ind, atl


def gauss_grid(N: int, B: int, occupancy: float, sigma_max_vox: float, seed: int):
    """Sum-of-16-Gaussians density cut so that about `occupancy` of blocks survive."""
    rng = np.random.default_rng(seed)
    g = np.zeros((16, 5))
    g[:, 0:3] = rng.uniform(0.15, 0.85, size=(16, 3))
    g[:, 3] = rng.uniform(0.04, 0.12, size=16)
    g[:, 4] = rng.uniform(0.5, 1.0, size=16)
    freqs = _color_freqs(rng)
    G = N // B
    blocks = _blocks_xyz(G)
    # First pass without a cut on a linear scale to find the block maxima of the field.
    probe_scale = 1.0 / (g[:, 4].sum())
    _, bmax = _fill(N, B, blocks, 0, g, 0.0, 0.0, probe_scale)
    bm = np.sort(bmax.astype(np.float64))[::-1]
    k = max(1, int(round(occupancy * blocks.shape[0])))
    cut_code = bm[min(k, bm.shape[0]) - 1]
    peak = bm[0]
    cut = (cut_code - 0.5) / 255.0 / probe_scale
    scale = probe_scale * 255.0 / max(peak, 1.0)
    atlas, bmax = _fill(N, B, blocks, 0, g, 0.0, cut, scale)
    qmin = _q_min_occupied(sigma_max_vox)
    ind, atl = _pack(N, B, blocks, atlas, bmax, qmin, rng, freqs)
    return ind, atl


def shell_grid(N: int, B: int, occupancy: float, sigma_max_vox: float, seed: int, max_shells: int = 64):
    """Thin shells (1-voxel Gaussian profile) on random closed surfaces until the
    block occupancy reaches `occupancy` (hollow interiors, as after visibility culling)."""
    rng = np.random.default_rng(seed)
    freqs = _color_freqs(rng)
    G = N // B
    blocks = _blocks_xyz(G)
    centres = (blocks.astype(np.float64) + 0.5) * B
    half_diag = 0.5 * math.sqrt(3.0) * B
    qmin = _q_min_occupied(sigma_max_vox)
    shells = []
    occ_mask = np.zeros(blocks.shape[0], bool)
    target = occupancy * blocks.shape[0]
    while len(shells) < max_shells:
        kind = 0 if rng.uniform() < 0.5 else 1
        c = rng.uniform(0.35, 0.65, size=3) * N
        if kind == 0:
            r = np.full(3, rng.uniform(0.10, 0.28) * N)
        else:
            r = rng.uniform(0.08, 0.30, size=3) * N
        s = np.array([kind, *c, *r], np.float64)
        # candidate blocks: centre within half-diagonal (+ profile support) of the surface,
        # with the ellipsoid bound widened by its axis ratio
        rel = (centres - c) / r
        k0 = np.sqrt((rel ** 2).sum(1))
        slack = (half_diag + 4.0) * (r.max() / r.min())
        cand = np.nonzero(np.abs(k0 - 1.0) * r.min() <= slack)[0]
        atl, bmax = _fill(N, B, np.ascontiguousarray(blocks[cand]), 1, s[None, :], 1.0, 0.0, 1.0)
        new_occ = occ_mask.copy()
        new_occ[cand[bmax >= qmin]] = True
        if shells and new_occ.sum() > 1.25 * target:
            continue          # this shell overshoots by too much; draw another
        shells.append(s)
        occ_mask = new_occ
        if occ_mask.sum() >= 0.95 * target:
            break
    sh = np.stack(shells)
    sel = np.nonzero(occ_mask)[0]
    atlas, bmax = _fill(N, B, np.ascontiguousarray(blocks[sel]), 1, sh, 1.0, 0.0, 1.0)
    ind, atl = _pack(N, B, np.ascontiguousarray(blocks[sel]), atlas, bmax, qmin, rng, freqs)
    return ind, atl


# ---------------------------------------------------------------------------------
# Named workloads (sizes from the paper's baked grids, Sec. 5 and App. B: 800x800 views
# at 39 degrees FOV, macroblocks of 32^3, Sec. 5.4)
# ---------------------------------------------------------------------------------
WORLD_BMIN = (-1.0, -1.0, -1.0)
WORLD_EXTENT = 2.0
CAM_RADIUS = 2.2
BG = (1.0, 1.0, 1.0)

MIXED_SIZES = [(200, 200), (400, 400), (800, 800), (1280, 720), (1920, 1080)]


def _scene(name, N, B, ind, atl, sigma_max_vox, rng, sizes, extra=None):
    delta = WORLD_EXTENT / N
    return Scene(name=name, N=N, B=B, bmin=WORLD_BMIN, extent=WORLD_EXTENT,
                 sigma_max=float(sigma_max_vox / delta), bg=BG, ind=ind, atlas=atl,
                 mlp=init_mlp(rng), cameras=orbit_cameras(rng, sizes, CAM_RADIUS),
                 extra=extra or {})


def make_scene(name: str, seed: int | None = None) -> Scene:
    """Build one of the named workloads.

    gauss64   : 64^3 grid, 8^3 blocks, ~30% occupied, one 64x64 view
    shell1024 : 1024^3 grid, 32^3 blocks, ~5% occupied, one 800x800 view
    batch1024 : the shell1024 grid with 64 cameras of mixed resolutions
    bwd512    : 512^3 grid, 32^3 blocks, ~8% occupied, 8 800x800 views, 65,536 rays
    shell2048 : 2048^3 grid, 32^3 blocks, ~2% occupied, 8 1920x1080 views, 262,144 rays
    tiny      : 16^3 grid, 4^3 blocks, ~40% occupied, one 24x20 view (unit tests)
    """
    if name == "gauss64":
        s = 1 if seed is None else seed
        ind, atl = gauss_grid(64, 8, 0.30, 0.6, s)
        rng = np.random.default_rng(s + 1000)
        return _scene(name, 64, 8, ind, atl, 0.6, rng, [(64, 64)])
    if name == "tiny":
        s = 7 if seed is None else seed
        ind, atl = gauss_grid(16, 4, 0.40, 0.8, s)
        rng = np.random.default_rng(s + 1000)
        return _scene(name, 16, 4, ind, atl, 0.8, rng, [(24, 20)])
    if name in ("shell1024", "batch1024"):
        s = 2 if seed is None else seed
        ind, atl = shell_grid(1024, 32, 0.05, 5.0, s)
        rng = np.random.default_rng(s + 1000)
        if name == "shell1024":
            return _scene(name, 1024, 32, ind, atl, 5.0, rng, [(800, 800)])
        rng2 = np.random.default_rng(s + 3000)
        picks = rng2.integers(0, len(MIXED_SIZES), size=64)
        return _scene(name, 1024, 32, ind, atl, 5.0, rng, [MIXED_SIZES[i] for i in picks])
    if name == "bwd512":
        s = 4 if seed is None else seed
        ind, atl = shell_grid(512, 32, 0.08, 5.0, s)
        rng = np.random.default_rng(s + 1000)
        sc = _scene(name, 512, 32, ind, atl, 5.0, rng, [(800, 800)] * 8)
        sc.extra["pix"] = random_pixels(np.random.default_rng(s + 2000), sc.cameras, 65536)
        sc.extra["target"] = np.random.default_rng(s + 2500).uniform(0, 1, (65536, 3)).astype(np.float32)
        return sc
    if name == "shell2048":
        s = 5 if seed is None else seed
        ind, atl = shell_grid(2048, 32, 0.02, 5.0, s)
        rng = np.random.default_rng(s + 1000)
        sc = _scene(name, 2048, 32, ind, atl, 5.0, rng, [(1920, 1080)] * 8)
        sc.extra["pix"] = random_pixels(np.random.default_rng(s + 2000), sc.cameras, 262144)
        sc.extra["target"] = np.random.default_rng(s + 2500).uniform(0, 1, (262144, 3)).astype(np.float32)
        return sc
    raise KeyError(name)


def random_pixels(rng: np.random.Generator, cams: np.ndarray, n: int) -> np.ndarray:
    """n seeded (camera, x, y) triples, int32 [n, 3], uniform over cameras then pixels."""
    ci = rng.integers(0, cams.shape[0], size=n)
    W = cams["W"][ci]
    H = cams["H"][ci]
    x = (rng.uniform(size=n) * W).astype(np.int64)
    y = (rng.uniform(size=n) * H).astype(np.int64)
    return np.stack([ci, np.minimum(x, W - 1), np.minimum(y, H - 1)], 1).astype(np.int32)


def all_pixels(cams: np.ndarray) -> np.ndarray:
    """Every pixel of every camera as (camera, x, y), in output order."""
    out = []
    for i, c in enumerate(cams):
        W, H = int(c["W"]), int(c["H"])
        y, x = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        out.append(np.stack([np.full(W * H, i), x.ravel(), y.ravel()], 1))
    return np.concatenate(out).astype(np.int32)


def custom_scene(N: int, B: int, ind: np.ndarray, atlas: np.ndarray, sigma_max: float,
                 mlp: np.ndarray, cameras: np.ndarray, bmin=WORLD_BMIN, extent=WORLD_EXTENT,
                 bg=BG, name="custom", flags: int = 0) -> Scene:
    """Wrap hand-built arrays (tests) in a Scene."""
    return Scene(name=name, N=N, B=B, bmin=tuple(bmin), extent=float(extent),
                 sigma_max=float(sigma_max), bg=tuple(bg), ind=np.ascontiguousarray(ind, np.int32),
                 atlas=np.ascontiguousarray(atlas, np.uint8), mlp=np.ascontiguousarray(mlp, np.float32),
                 cameras=np.ascontiguousarray(cameras), flags=int(flags))


def analytic_field(seed: int, n_blob: int = 64, radius: float = 0.6, std=(0.03, 0.08), peak=(20.0, 200.0),
                   freq: float = 8.0) -> dict:
    """Seeded parameters of an analytic radiance field to bake (the stand-in for a trained
    network): n_blob Gaussian density blobs with centres on a sphere of `radius` around the
    origin (a surface-like, mostly empty scene), std and peak uniform in the given ranges
    (world units); 7 sinusoidal channels (diffuse RGB, 4 features) with direction vectors
    uniform in [-freq, freq]^3 and phases in [0, 2 pi); 16 jitter offsets drawn from a
    Gaussian of std 1/sqrt(12) voxels (the anti-aliasing samples of the bake)."""
    rng = np.random.default_rng(seed)
    u = rng.normal(size=(n_blob, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    blobs = np.zeros((n_blob, 5), np.float32)
    blobs[:, :3] = radius * u
    blobs[:, 3] = rng.uniform(*std, n_blob)
    blobs[:, 4] = rng.uniform(*peak, n_blob)
    colors = np.zeros((7, 4), np.float32)
    colors[:, :3] = rng.uniform(-freq, freq, (7, 3))
    colors[:, 3] = rng.uniform(0.0, 2.0 * np.pi, 7)
    jitter = (rng.normal(size=(16, 3)) / np.sqrt(12.0)).astype(np.float32)
    return {"blobs": blobs, "colors": colors, "jitter": jitter}
