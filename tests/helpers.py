"""Hand-built scenes for tests (closed-form cases). Input construction only."""
import numpy as np

from paper_2103_14645_gb300 import synth


def axis_camera(o_world, W=1, H=1, f=1.0):
    """Camera with identity rotation (looks along world -z) whose principal point sits
    on the centre of pixel (0, 0), so that pixel's ray direction is exactly (0, 0, -1)."""
    cam = np.zeros(1, synth.CAMERA_DTYPE)
    c2w = np.eye(3, 4, dtype=np.float32)
    c2w[:, 3] = np.asarray(o_world, np.float32)
    cam[0]["c2w"] = c2w.reshape(-1)
    cam[0]["fx"] = f
    cam[0]["fy"] = f
    cam[0]["cx"] = 0.5
    cam[0]["cy"] = 0.5
    cam[0]["W"] = W
    cam[0]["H"] = H
    return cam


def dense_to_blocks(dense, B, keep_empty=False):
    """dense uint8 [N,N,N,8] (z,y,x,c) -> (ind [G,G,G], atlas [nb,B,B,B,8]); blocks whose
    density channel is all zero are left out unless keep_empty."""
    N = dense.shape[0]
    G = N // B
    ind = np.full((G, G, G), -1, np.int32)
    blocks = []
    for bz in range(G):
        for by in range(G):
            for bx in range(G):
                blk = dense[bz * B:(bz + 1) * B, by * B:(by + 1) * B, bx * B:(bx + 1) * B]
                if keep_empty or blk[..., 0].any():
                    ind[bz, by, bx] = len(blocks)
                    blocks.append(blk)
    atlas = np.stack(blocks) if blocks else np.zeros((0, B, B, B, 8), np.uint8)
    return ind, np.ascontiguousarray(atlas)


def silent_mlp(rng=None):
    """All weights zero and output bias -1e4: the residual sigmoid is exactly 0."""
    w = np.zeros(synth.MLP_NPARAM, np.float32)
    w[-3:] = -1e4
    return w


def blocks_to_dense(scene):
    """Decode a scene to dense uint8 [N,N,N,8] with empty blocks zero."""
    N, B = scene.N, scene.B
    G = N // B
    dense = np.zeros((N, N, N, 8), np.uint8)
    for bz in range(G):
        for by in range(G):
            for bx in range(G):
                s = scene.ind[bz, by, bx]
                if s >= 0:
                    dense[bz * B:(bz + 1) * B, by * B:(by + 1) * B, bx * B:(bx + 1) * B] = scene.atlas[s]
    return dense


def slab_scene(N=16, B=4, z_range=(4, 6), q=200, color=(100, 150, 200, 10, 20, 30, 40),
               sigma_max_vox=1.0, xy=(5, 5), o_z_vox=None, per_voxel_q=None, mlp=None):
    """A z-slab of uniform density/colour at voxel column (x, y) and one axis camera
    above the grid looking down -z through voxel centres."""
    dense = np.zeros((N, N, N, 8), np.uint8)
    z0, z1 = z_range
    dense[z0:z1, :, :, 0] = q
    if per_voxel_q is not None:
        for k, qq in enumerate(per_voxel_q):
            dense[z0 + k, :, :, 0] = qq
    dense[z0:z1, :, :, 1:] = np.asarray(color, np.uint8)
    ind, atlas = dense_to_blocks(dense, B)
    extent = 2.0
    s = N / extent
    ox = (xy[0] + 0.5) / s - 1.0
    oy = (xy[1] + 0.5) / s - 1.0
    oz = ((N + 2) if o_z_vox is None else o_z_vox) / s - 1.0
    cam = axis_camera((ox, oy, oz))
    delta = extent / N
    return synth.custom_scene(N, B, ind, atlas, sigma_max_vox / delta,
                              silent_mlp() if mlp is None else mlp, cam)
