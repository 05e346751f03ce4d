"""Seeded synthetic voxel geometries and per-node input fields.

This module only *generates inputs*: solid/fluid voxel masks of the porous
media the method is benchmarked on (the paper uses an empty channel and a
fixed-bed reactor, Sect. 5.1; the large-scale runs use a reactor of the same
kind, Sect. 6) and smooth random scalar fields for the Brinkman solid
fraction.  It contains none of the lattice Boltzmann arithmetic, no lattice
tables and no enumeration.  Both the CPU oracle and the CUDA library consume
what it produces, so it is the one module the two sides share.

Conventions
-----------
* A geometry is a ``uint8`` array ``solid[Z, Y, X]`` (x fastest), 1 = solid.
* Randomness comes from SplitMix64 (S. Vigna's published generator): state
  advances by the golden-ratio increment 0x9E3779B97F4A7C15 and every output
  is passed through the 64-bit finaliser with shifts 30/27/31 and multipliers
  0xBF58476D1CE4E5B9 / 0x94D049BB133111EB.  A double in [0, 1) is
  ``(x >> 11) * 2**-53``.
"""
from __future__ import annotations

import hashlib
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64 stream; ``uniform(n)`` draws n doubles in [0, 1)."""

    def __init__(self, seed: int):
        self.counter = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, n: int) -> np.ndarray:
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = self.counter + k * _GOLDEN
            self.counter = self.counter + np.uint64(n) * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def porosity(solid: np.ndarray) -> float:
    return 1.0 - float(solid.mean())


# ---------------------------------------------------------------------------
# Geometries
# ---------------------------------------------------------------------------

def empty_box(X: int, Y: int, Z: int) -> np.ndarray:
    return np.zeros((Z, Y, X), dtype=np.uint8)


def square_channel(X: int, Y: int, Z: int, wall: int = 1) -> np.ndarray:
    """Empty duct along z with ``wall``-voxel thick solid walls at the x and y faces.

    With X = Y = 100, Z = 500 this is the paper's channel benchmark geometry
    (Sect. 5.1) with its long axis placed along z: a 98 x 98 fluid cross
    section and 4,802,000 fluid nodes.
    """
    s = np.zeros((Z, Y, X), dtype=np.uint8)
    s[:, :wall, :] = 1
    s[:, Y - wall:, :] = 1
    s[:, :, :wall] = 1
    s[:, :, X - wall:] = 1
    return s


def random_voxels(X: int, Y: int, Z: int, solid_fraction: float, seed: int) -> np.ndarray:
    """Independent Bernoulli voxels (tiny exhaustive table tests)."""
    u = SplitMix64(seed).uniform(X * Y * Z).reshape(Z, Y, X)
    return (u < solid_fraction).astype(np.uint8)


def _stamp_sphere(solid, cz, cy, cx, r, periodic):
    """Mark voxels v with |v - c|^2 <= r^2 solid (integer centre c).

    Periodic axes use the minimum image; on other axes the sphere is clipped
    by the box.
    """
    Z, Y, X = solid.shape
    ri = int(math.floor(r))
    r2 = r * r
    dz = np.arange(-ri, ri + 1)
    d2 = dz[:, None, None] ** 2 + dz[None, :, None] ** 2 + dz[None, None, :] ** 2
    inside = d2 <= r2
    zz = cz + dz
    yy = cy + dz
    xx = cx + dz
    okz = np.ones_like(zz, bool) if periodic[2] else (zz >= 0) & (zz < Z)
    oky = np.ones_like(yy, bool) if periodic[1] else (yy >= 0) & (yy < Y)
    okx = np.ones_like(xx, bool) if periodic[0] else (xx >= 0) & (xx < X)
    zz = zz % Z
    yy = yy % Y
    xx = xx % X
    m = inside & okz[:, None, None] & oky[None, :, None] & okx[None, None, :]
    iz, iy, ix = np.nonzero(m)
    before = int(solid[zz[iz], yy[iy], xx[ix]].sum())
    solid[zz[iz], yy[iy], xx[ix]] = 1
    return len(iz) - before


def overlapping_spheres(X, Y, Z, radius, seed, target_porosity, periodic=(1, 0, 0)):
    """Overlapping spheres with uniform integer centres, added until porosity <= target.

    Centres are ``floor(u * dim)`` from three consecutive draws (x, y, z).
    """
    rng = SplitMix64(seed)
    solid = np.zeros((Z, Y, X), dtype=np.uint8)
    total = X * Y * Z
    n_solid = 0
    while 1.0 - n_solid / total > target_porosity:
        u = rng.uniform(3)
        cx, cy, cz = int(u[0] * X), int(u[1] * Y), int(u[2] * Z)
        n_solid += _stamp_sphere(solid, cz, cy, cx, radius, periodic)
    return solid


def rsa_spheres(X, Y, Z, radius, seed, periodic=(1, 0, 0), max_consecutive_rejections=20000,
                target_porosity=0.0, batch=16384):
    """Random sequential addition of non-overlapping spheres (integer centres).

    A candidate centre (``floor(u * dim)`` per axis, drawn x, y, z) is accepted
    when its distance to every accepted centre (minimum image on periodic
    axes) is at least 2*radius.  Stops when ``max_consecutive_rejections``
    candidates in a row were rejected or the porosity reaches
    ``target_porosity``.  Candidates are drawn in batches but decided strictly
    in draw order, so the result equals one-at-a-time RSA.
    Returns (solid, centres[n, 3] as (x, y, z)).
    """
    from scipy.spatial import cKDTree

    rng = SplitMix64(seed)
    dims = np.array([X, Y, Z], dtype=np.int64)
    # non-periodic axes get a box so large that wrapping never matters
    box = np.where(np.array(periodic, bool), dims, 8 * dims).astype(np.float64)
    d2min = int(round((2 * radius) ** 2))
    solid = np.zeros((Z, Y, X), dtype=np.uint8)
    total = X * Y * Z
    n_solid = 0
    centres = np.zeros((0, 3), dtype=np.int64)
    run = 0  # consecutive rejections so far

    def min_image_d2(a, b):
        d = np.abs(a - b)
        d = np.where(np.array(periodic, bool), np.minimum(d, dims - d), d)
        return int((d * d).sum())

    while True:
        cand = np.floor(rng.uniform(3 * batch).reshape(batch, 3) * dims).astype(np.int64)
        if len(centres):
            tree = cKDTree(centres.astype(np.float64), boxsize=box)
            dist, _ = tree.query(cand.astype(np.float64), k=1)
            free = np.rint(dist * dist) >= d2min
        else:
            free = np.ones(batch, bool)
        new = []
        stop = False
        last = -1
        for j in np.nonzero(free)[0]:
            if run + (j - last - 1) >= max_consecutive_rejections:
                stop = True
                break
            c = cand[j]
            if any(min_image_d2(c, q) < d2min for q in new):
                continue
            run = 0
            last = j
            new.append(c)
            n_solid += _stamp_sphere(solid, int(c[2]), int(c[1]), int(c[0]), radius,
                                     (periodic[0], periodic[1], periodic[2]))
            if 1.0 - n_solid / total <= target_porosity:
                stop = True
                break
        if not stop:
            run += batch - 1 - last
            if run >= max_consecutive_rejections:
                stop = True
        if new:
            centres = np.concatenate([centres, np.array(new, dtype=np.int64)])
        if stop:
            break
    return solid, centres


def voronoi_foam(X, Y, Z, n_seeds, strut_radius, seed, chunk=1 << 20, threads=None):
    """Open-cell foam: solid = voxels within ``strut_radius`` of a Voronoi edge.

    Seeds are uniform in the periodic box.  For voxel centre p with nearest
    seeds s1, s2, s3 (periodic images), the local Voronoi edge is the line
    where the bisector planes of (s1, s2) and (s1, s3) meet; p is solid when
    its distance to that line is <= strut_radius.  With unit normals n2, n3
    and signed plane distances e2, e3 the squared distance to the line is
    e^T G^-1 e with G = [[1, n2.n3], [n2.n3, 1]].  Chunks of voxels are
    processed by a thread pool (the KD-tree queries and numpy kernels release
    the interpreter lock).
    """
    import os
    from concurrent.futures import ThreadPoolExecutor

    from scipy.spatial import cKDTree

    rng = SplitMix64(seed)
    dims = np.array([X, Y, Z], dtype=np.float64)
    seeds = rng.uniform(3 * n_seeds).reshape(n_seeds, 3) * dims
    tree = cKDTree(seeds, boxsize=dims)
    total = X * Y * Z
    solid = np.zeros(total, dtype=np.uint8)
    r2 = strut_radius * strut_radius

    def work(start):
        idx = np.arange(start, min(start + chunk, total), dtype=np.int64)
        p = np.stack([idx % X, (idx // X) % Y, idx // (X * Y)], axis=1).astype(np.float64)
        _, nb = tree.query(p, k=3)
        s1 = seeds[nb[:, 0]]
        v1 = p - s1
        v1 -= dims * np.round(v1 / dims)
        e, nrm = [], []
        for k in (1, 2):
            d = seeds[nb[:, k]] - s1
            d -= dims * np.round(d / dims)
            L = np.sqrt((d * d).sum(1))
            n = d / L[:, None]
            # signed distance of p from the bisector plane (mid-point at d/2)
            e.append((v1 * n).sum(1) - 0.5 * L)
            nrm.append(n)
        c = (nrm[0] * nrm[1]).sum(1)
        det = np.maximum(1.0 - c * c, 1e-12)
        q = (e[0] ** 2 - 2 * c * e[0] * e[1] + e[1] ** 2) / det
        solid[idx] = (q <= r2).astype(np.uint8)

    n_threads = threads or len(os.sched_getaffinity(0))
    with ThreadPoolExecutor(max_workers=n_threads) as ex:
        list(ex.map(work, range(0, total, chunk)))
    return solid.reshape(Z, Y, X)


def smooth_noise(X, Y, Z, sigma, seed, dtype=np.float32):
    """Min-max normalised periodic Gaussian filter (truncated at 4 sigma) of uniform noise."""
    from scipy.ndimage import gaussian_filter

    u = SplitMix64(seed).uniform(X * Y * Z).reshape(Z, Y, X)
    g = gaussian_filter(u, sigma=sigma, mode="wrap", truncate=4.0)
    g = (g - g.min()) / (g.max() - g.min())
    return g.astype(dtype)


def node_field(field_zyx: np.ndarray, node_xyz: np.ndarray) -> np.ndarray:
    """Sample a voxel field at the fluid nodes (node_xyz[n] = (x, y, z))."""
    return np.ascontiguousarray(field_zyx[node_xyz[:, 2], node_xyz[:, 1], node_xyz[:, 0]])


def uniform_field(n: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    return lo + (hi - lo) * SplitMix64(seed).uniform(n)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def sphere_box_64x32x32(seed: int = 0):
    """64x32x32 box, overlapping radius-4 spheres to porosity <= 0.70 (periodic x)."""
    return overlapping_spheres(64, 32, 32, 4.0, seed, 0.70, periodic=(1, 0, 0))


def packed_bed_256(seed: int = 1, max_consecutive_rejections: int = 20000):
    """256^3 bed of radius-12 non-overlapping spheres by random sequential addition."""
    s, _ = rsa_spheres(256, 256, 256, 12.0, seed, periodic=(1, 0, 0),
                       max_consecutive_rejections=max_consecutive_rejections)
    return s
