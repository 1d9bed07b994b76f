"""The empty-space maps snerg_create builds in the workspace, read back and compared with a
brute-force cone distance on small grids.

Per octant o of the ray direction (bit i of o set: d_i < 0), the cone of a cell p is
{q : q_i >= p_i where d_i >= 0, q_i <= p_i where d_i < 0}; a ray's later samples have
their nearest voxels in the cone of the current one. The workspace holds

- ind [8][G^3] int32: the atlas slot of an occupied block; for an empty block -D with
  D = min(32, Chebyshev distance to the nearest occupied block of the cone), or -32 if
  the cone has none;
- vskip [8][nb][(B+2)^3] uint8: per interior voxel of a stored block, min(255, Chebyshev
  distance to the nearest voxel of the same block in the cone with a non-zero density
  code); apron cells outside the grid hold the value of the voxel they clamp to.

Workspace layout (each region 256-byte aligned): a 256-byte header, ind, a G^3 byte map,
2 G^3 bytes of scratch, the int32 block-of-slot table [nb], vskip, the padded atlas."""

import numpy as np
import pytest
import torch

from paper_2103_14645_gb300 import renderer, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
BLOCK_CAP, VOXEL_CAP = 32, 255


def _align(v):
    return (v + 255) & ~255


def _cone_distance(occ: np.ndarray, octant: int, cap: int) -> np.ndarray:
    """Brute force over all pairs of cells of the cube occ [n, n, n] (z, y, x)."""
    n = occ.shape[0]
    cells = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    q = cells[occ.reshape(-1)]                       # occupied cells (z, y, x)
    out = np.full(n ** 3, cap, np.int64)
    if len(q) == 0:
        return out.reshape(occ.shape)
    diff = q[None, :, :] - cells[:, None, :]         # [cells, occupied, (z, y, x)]
    sign = np.array([-1 if (octant >> 2) & 1 else 1, -1 if (octant >> 1) & 1 else 1,
                     -1 if octant & 1 else 1])       # axis order z, y, x
    in_cone = ((diff * sign) >= 0).all(-1)
    dist = np.abs(diff).max(-1)
    dist = np.where(in_cone, dist, cap)
    return np.minimum(dist.min(1), cap).reshape(occ.shape)


def _scene(N, B, occupancy, seed):
    ind, atl = synth.gauss_grid(N, B, occupancy, 2.0, seed)
    rng = np.random.default_rng(seed)
    cams = np.zeros(1, synth.CAMERA_DTYPE)
    cams[0] = synth.look_at_camera((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), 8, 8, 40.0, 0)
    return synth.custom_scene(N, B, ind, atl, 5.0, synth.init_mlp(rng), cams)


def _maps(sc):
    r = renderer.Renderer.from_scene(sc, DEV)
    torch.cuda.synchronize()
    ws = r.workspace.cpu().numpy()
    G, B, nb = sc.G, sc.B, sc.nb
    P = B + 2
    G3, P3 = G ** 3, P ** 3
    o_ind = 256
    o_bdist = _align(o_ind + 8 * G3 * 4)
    o_btmp = _align(o_bdist + G3)
    o_blk = _align(o_btmp + 2 * G3)
    o_vskip = _align(o_blk + nb * 4)
    ind8 = ws[o_ind:o_ind + 8 * G3 * 4].view(np.int32).reshape(8, G, G, G)
    vskip = ws[o_vskip:o_vskip + 8 * nb * P3].reshape(8, nb, P, P, P)
    r.close()
    return ind8, vskip


@pytest.mark.parametrize("N,B,occ,seed", [(16, 4, 0.4, 3), (24, 4, 0.15, 5), (32, 8, 0.3, 7), (16, 2, 0.25, 9)])
def test_block_and_voxel_cone_distances(N, B, occ, seed):
    sc = _scene(N, B, occ, seed)
    ind8, vskip = _maps(sc)
    occupied = sc.ind >= 0
    for o in range(8):
        want = _cone_distance(occupied, o, BLOCK_CAP)
        want_word = np.where(occupied, sc.ind, -np.maximum(want, 1))
        np.testing.assert_array_equal(ind8[o], want_word, err_msg=f"block map, octant {o}")
    for s in range(sc.nb):
        dens = sc.atlas[s, ..., 0] != 0
        for o in range(8):
            want = _cone_distance(dens, o, VOXEL_CAP)
            got = vskip[o, s, 1:B + 1, 1:B + 1, 1:B + 1]
            np.testing.assert_array_equal(got, want, err_msg=f"voxel plane, slot {s}, octant {o}")


def test_cone_distance_is_at_least_the_two_sided_distance():
    """The one-sided maps never give less room than the two-sided Chebyshev distance
    (brute force on the same cube)."""
    rng = np.random.default_rng(1)
    occ = rng.uniform(size=(6, 6, 6)) < 0.08
    cells = np.stack(np.meshgrid(*[np.arange(6)] * 3, indexing="ij"), -1).reshape(-1, 3)
    q = cells[occ.reshape(-1)]
    two_sided = np.abs(q[None] - cells[:, None]).max(-1).min(1).reshape(occ.shape)
    for o in range(8):
        assert (_cone_distance(occ, o, 255) >= two_sided).all()


def test_grid_border_apron_holds_the_clamped_voxel():
    sc = _scene(16, 4, 0.5, 11)
    ind8, vskip = _maps(sc)
    G, B = sc.G, sc.B
    for z, y, x in zip(*np.nonzero(sc.ind >= 0)):
        s = sc.ind[z, y, x]
        for o in range(8):
            plane = vskip[o, s]
            # an apron face outside the grid repeats the adjacent interior face
            if x == 0:
                np.testing.assert_array_equal(plane[1:B + 1, 1:B + 1, 0], plane[1:B + 1, 1:B + 1, 1])
            if x == G - 1:
                np.testing.assert_array_equal(plane[1:B + 1, 1:B + 1, B + 1], plane[1:B + 1, 1:B + 1, B])
            if y == 0:
                np.testing.assert_array_equal(plane[1:B + 1, 0, 1:B + 1], plane[1:B + 1, 1, 1:B + 1])
            if z == G - 1:
                np.testing.assert_array_equal(plane[B + 1, 1:B + 1, 1:B + 1], plane[B, 1:B + 1, 1:B + 1])
