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


def _stamp_sphere_at(solid, c, r, periodic):
    """Mark voxels v (integer centres) with |v - c|^2 <= r^2 solid, c = (x, y, z) real.

    Periodic axes use the minimum image; on other axes the sphere is clipped.
    """
    Z, Y, X = solid.shape
    lo = [int(math.floor(c[a] - r)) for a in range(3)]
    hi = [int(math.ceil(c[a] + r)) for a in range(3)]
    xs, ys, zs = (np.arange(lo[a], hi[a] + 1) for a in range(3))
    d2 = ((zs - c[2]) ** 2)[:, None, None] + ((ys - c[1]) ** 2)[None, :, None] + ((xs - c[0]) ** 2)[None, None, :]
    inside = d2 <= r * r
    dims = (X, Y, Z)
    idx = []
    ok = []
    for a, v in ((0, xs), (1, ys), (2, zs)):
        ok.append(np.ones_like(v, bool) if periodic[a] else (v >= 0) & (v < dims[a]))
        idx.append(v % dims[a])
    m = inside & ok[2][:, None, None] & ok[1][None, :, None] & ok[0][None, None, :]
    iz, iy, ix = np.nonzero(m)
    solid[idx[2][iz], idx[1][iy], idx[0][ix]] = 1


def fcc_spheres(X, Y, Z, radius, solid_fraction, seed, periodic=(1, 0, 0), jitter=0.4):
    """Monodisperse non-overlapping spheres on a jittered, randomly rotated FCC lattice.

    Stands in for a dense packed bed where random sequential addition cannot
    reach the density (RSA jams near a solid fraction of 0.38).  The cubic
    cell side a follows from the target solid fraction (4 spheres of volume
    4/3 pi r^3 per a^3).  The lattice is rotated by a uniformly random
    rotation (Shoemake's quaternion from three draws), shifted by one uniform
    draw per axis, and every lattice point moves by up to +-jitter per axis
    (three draws per point, in lattice order).  Centres outside the box are dropped,
    and so is any centre closer than 2 r to an earlier kept one (minimum
    image on periodic axes: the rotated lattice does not tile the box).
    Returns (solid, centres[n, 3] as real (x, y, z)).
    """
    from scipy.spatial import cKDTree

    rng = SplitMix64(seed)
    a = (16.0 * math.pi * radius ** 3 / (3.0 * solid_fraction)) ** (1.0 / 3.0)
    u1, u2, u3 = rng.uniform(3)
    qx = math.sqrt(1 - u1) * math.sin(2 * math.pi * u2)
    qy = math.sqrt(1 - u1) * math.cos(2 * math.pi * u2)
    qz = math.sqrt(u1) * math.sin(2 * math.pi * u3)
    qw = math.sqrt(u1) * math.cos(2 * math.pi * u3)
    rot = np.array([
        [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
        [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
        [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)]])
    shift = rng.uniform(3) * a
    dims = np.array([X, Y, Z], dtype=np.float64)
    k = int(math.ceil(np.linalg.norm(dims) / a)) + 1
    g = np.arange(-k, k + 1, dtype=np.float64)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    pts = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a + shift
    pts = pts @ rot.T + dims / 2
    pts = pts + (rng.uniform(3 * len(pts)).reshape(-1, 3) - 0.5) * 2 * jitter
    pts = pts[np.all((pts >= 0) & (pts < dims), axis=1)]
    box = np.where(np.array(periodic, bool), dims, 8 * dims)
    keep = []
    tree_pts = np.zeros((0, 3))
    tree = None
    for i, c in enumerate(pts):
        if tree is not None and len(tree.query_ball_point(c, 2 * radius - 1e-9)):
            continue
        pending = [q for q in keep[len(tree_pts):]]
        if any(np.sum(np.minimum(np.abs(pts[q] - c), np.where(np.array(periodic, bool), dims - np.abs(pts[q] - c),
                                                                np.inf)) ** 2) < (2 * radius) ** 2 for q in pending):
            continue
        keep.append(i)
        if len(keep) - len(tree_pts) >= 256:
            tree_pts = pts[keep]
            tree = cKDTree(np.mod(tree_pts, box), boxsize=box)
    centres = pts[keep]
    solid = np.zeros((Z, Y, X), dtype=np.uint8)
    for c in centres:
        _stamp_sphere_at(solid, c, radius, periodic)
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


def packed_bed_fcc_256(seed: int = 1):
    """256^3 dense bed: radius-12 spheres on a jittered, randomly rotated FCC lattice, periodic x,
    porosity 0.402 (6,751,202 fluid nodes), the porosity-0.4 bed that RSA cannot reach."""
    return fcc_spheres(256, 256, 256, 12.0, 0.67, seed, periodic=(1, 0, 0), jitter=0.2)[0]


def packed_bed_256(seed: int = 1, max_consecutive_rejections: int = 20000):
    """256^3 bed of radius-12 non-overlapping spheres by random sequential addition."""
    s, _ = rsa_spheres(256, 256, 256, 12.0, seed, periodic=(1, 0, 0),
                       max_consecutive_rejections=max_consecutive_rejections)
    return s
