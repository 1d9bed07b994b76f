"""The seeded synthetic inputs: checksums of the generated grids, weights and cameras
(SHA-256 of their bytes, first 16 hex digits), and the occupancy each workload asks for.
A change to a generator shows up here before it silently changes a parity case or a
benchmark workload."""

import numpy as np
import pytest

from paper_2103_14645_gb300 import synth

# generated on x86-64 with the C generator in paper_2103_14645_gb300/synth
CHECKSUMS = {
    "tiny": "b629fc87e17e9e47",
    "gauss64": "7d1b4a64895bb9c8",
    "bwd512": "700d15cdb2b2e714",
    "shell1024": "51ae98075803b79a",
}


@pytest.mark.parametrize("name", sorted(CHECKSUMS))
def test_scene_checksum(name):
    sc = synth.make_scene(name)
    assert sc.checksum() == CHECKSUMS[name]


def test_checksum_sees_every_part():
    sc = synth.make_scene("tiny")
    base = sc.checksum()
    for attr in ("ind", "atlas", "mlp"):
        a = getattr(sc, attr).copy()
        flat = getattr(sc, attr).reshape(-1)
        flat[0] = flat[0] + 1 if flat.dtype != np.float32 else flat[0] + 1.0
        assert sc.checksum() != base, attr
        setattr(sc, attr, a)
        assert sc.checksum() == base
    sc.cameras = sc.cameras.copy()
    sc.cameras["fx"] += 1.0
    assert sc.checksum() != base


@pytest.mark.parametrize("name,target,tol", [("gauss64", 0.30, 0.05), ("shell1024", 0.05, 0.02),
                                             ("bwd512", 0.08, 0.03)])
def test_occupancy_near_the_workload_definition(name, target, tol):
    assert abs(synth.make_scene(name).occupancy - target) <= tol
