"""The seeded input generators: determinism and the stated properties of the dense bed.

The jittered, randomly rotated FCC packing stands in for the porosity-0.4 packed
bed: its spheres must not overlap (minimum image on the periodic axis), the
same seed must give the same voxels, and the 256^3 instance must have the
stated porosity and node count.
"""
import numpy as np
from scipy.spatial import cKDTree

import geometry


def _min_image_dmin(c, dims, periodic):
    box = np.where(np.array(periodic, bool), dims, 8 * dims).astype(np.float64)
    d, _ = cKDTree(np.mod(c, box), boxsize=box).query(np.mod(c, box), k=2)
    return d[:, 1].min()


def test_fcc_spheres_small_properties():
    dims = np.array([96, 80, 72])
    solid, c = geometry.fcc_spheres(96, 80, 72, 8.0, 0.6, 3, periodic=(1, 0, 0), jitter=0.3)
    assert solid.shape == (72, 80, 96)
    assert _min_image_dmin(c, dims, (1, 0, 0)) >= 16.0
    assert np.all((c >= 0) & (c < dims))
    # every solid voxel lies within r of some centre (minimum image in x)
    z, y, x = np.nonzero(solid)
    v = np.stack([x, y, z], axis=1).astype(np.float64)
    box = np.array([96, 8 * 80, 8 * 72], np.float64)
    d, _ = cKDTree(np.mod(c, box), boxsize=box).query(v, k=1)
    assert d.max() <= 8.0 + 1e-9
    again, c2 = geometry.fcc_spheres(96, 80, 72, 8.0, 0.6, 3, periodic=(1, 0, 0), jitter=0.3)
    assert np.array_equal(again, solid) and np.array_equal(c2, c)
    other, _ = geometry.fcc_spheres(96, 80, 72, 8.0, 0.6, 4, periodic=(1, 0, 0), jitter=0.3)
    assert not np.array_equal(other, solid)


def test_dense_bed_256():
    solid = geometry.packed_bed_fcc_256(1)
    assert int((solid == 0).sum()) == 6751202
    assert abs(geometry.porosity(solid) - 0.4024) < 1e-4
