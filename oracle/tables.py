"""Sparse-lattice tables: enumeration, adjacency list, RIA run table (oracle).

Test infrastructure only (see ``oracle/__init__``).

* Only fluid voxels become nodes, stored in one 1-D vector in the order an
  enumeration function gives (Sect. 1; Sect. 5.6).
* The adjacency list holds, for each node and each of the 18 moving
  directions, where the PDF pulled into that node comes from (Sect. 4,
  "Loop Balance": 18 x 4-byte indices per node, Fig. 2a).
* Reduced indirect addressing (Sect. 4.1, Fig. 2b): a node whose access
  pattern equals its predecessor's shifted by one needs no index load; the
  runs of such nodes are stored run-length coded.

Readings where the paper is silent (each also implemented independently by
the library): the index stored is a *node* index (not a PDF index), with
negative markers -1 (halfway bounce-back: solid voxel or wall face), -2
(inlet face x = -1) and -3 (outlet face x = X); the lexicographic key inside
and across blocks has x fastest; the Hilbert variant is Skilling's transpose
algorithm with bits interleaved (x, y, z), most significant first.
"""
from __future__ import annotations

import numpy as np

from .d3q19 import C, INV

MARK_WALL = -1
MARK_INLET = -2
MARK_OUTLET = -3


# ---------------------------------------------------------------------------
# Enumeration (Sect. 5.6)
# ---------------------------------------------------------------------------

def fluid_coords(solid: np.ndarray):
    """(x, y, z) of every fluid voxel, in raster order (x fastest)."""
    z, y, x = np.nonzero(solid == 0)
    return x.astype(np.int64), y.astype(np.int64), z.astype(np.int64)


def lexicographic_order(solid: np.ndarray, B: int) -> np.ndarray:
    """Node order of LS with blocking factor B.

    Blocks are B^3 cubes aligned at the origin (partial at the far faces).
    Nodes are sorted by (block z, block y, block x, z, y, x), most significant
    first, so x runs fastest both inside a block and across blocks.  B = 1 is
    plain lexicographic order.  Returns the fluid coordinates as [N, 3]
    (x, y, z) in enumeration order.
    """
    x, y, z = fluid_coords(solid)
    order = np.lexsort((x, y, z, x // B, y // B, z // B))
    return np.stack([x[order], y[order], z[order]], axis=1)


def hilbert_keys(x: np.ndarray, y: np.ndarray, z: np.ndarray, bits: int) -> np.ndarray:
    """Hilbert-curve index of 3-D points with ``bits`` bits per axis.

    Skilling's method (J. Skilling, "Programming the Hilbert curve", AIP
    Conf. Proc. 707, 2004): the coordinates are turned in place into the
    "transposed" Hilbert index -- walking the bit levels from the top, each
    axis either flips the lower bits of the first axis or swaps its lower
    bits with it; the result is then Gray-coded across axes and corrected by
    the parity of the last axis -- and the transposed bits are read out
    level by level, axis 0 first, into one integer.
    """
    X = [np.asarray(x, dtype=np.uint64).copy(), np.asarray(y, dtype=np.uint64).copy(),
         np.asarray(z, dtype=np.uint64).copy()]
    if bits == 0:
        return np.zeros_like(X[0])
    top = np.uint64(1) << np.uint64(bits - 1)
    q = top
    while q > 1:
        low = q - np.uint64(1)
        for a in range(3):
            hit = (X[a] & q) != 0
            # bit set: invert the lower bits of axis 0
            flipped = X[0] ^ low
            # bit clear: exchange the lower bits of axis 0 and axis a
            t = (X[0] ^ X[a]) & low
            new0 = np.where(hit, flipped, X[0] ^ t)
            newa = np.where(hit, X[a], X[a] ^ t)
            X[0] = new0
            if a != 0:
                X[a] = newa
        q >>= np.uint64(1)
    # Gray code across the axes
    for a in range(1, 3):
        X[a] = X[a] ^ X[a - 1]
    fix = np.zeros_like(X[0])
    q = top
    while q > 1:
        fix = np.where((X[2] & q) != 0, fix ^ (q - np.uint64(1)), fix)
        q >>= np.uint64(1)
    for a in range(3):
        X[a] = X[a] ^ fix
    key = np.zeros_like(X[0])
    for b in range(bits - 1, -1, -1):
        for a in range(3):
            key = (key << np.uint64(1)) | ((X[a] >> np.uint64(b)) & np.uint64(1))
    return key


def hilbert_bits(X: int, Y: int, Z: int) -> int:
    m = max(X, Y, Z)
    k = 0
    while (1 << k) < m:
        k += 1
    return k


def hilbert_order(solid: np.ndarray) -> np.ndarray:
    """Node order along the Hilbert curve of the smallest 2^k cube holding the box."""
    Z, Y, X = solid.shape
    x, y, z = fluid_coords(solid)
    key = hilbert_keys(x, y, z, hilbert_bits(X, Y, Z))
    order = np.argsort(key, kind="stable")
    return np.stack([x[order], y[order], z[order]], axis=1)


def voxel_to_node(solid: np.ndarray, node_xyz: np.ndarray) -> np.ndarray:
    v2n = np.full(solid.shape, -1, dtype=np.int64)
    v2n[node_xyz[:, 2], node_xyz[:, 1], node_xyz[:, 0]] = np.arange(len(node_xyz))
    return v2n


# ---------------------------------------------------------------------------
# Adjacency list (Sect. 4, "Loop Balance"; Fig. 2a)
# ---------------------------------------------------------------------------

def adjacency(solid: np.ndarray, node_xyz: np.ndarray, periodic=(0, 0, 0),
              x_pressure: bool = False) -> np.ndarray:
    """adj[i-1, n] for i = 1..18: the node the pulled PDF f_i of node n comes from.

    The source voxel is x_n - c_i.  Periodic axes wrap.  On a non-periodic
    axis a source outside the box is a wall (-1), except across the x faces
    when ``x_pressure`` is set: -2 behind x = 0 (inlet), -3 beyond x = X-1
    (outlet).  A wall crossing on y or z takes precedence over a pressure
    crossing.  A solid source voxel is -1.
    """
    Z, Y, X = solid.shape
    dims = (X, Y, Z)
    if x_pressure and periodic[0]:
        raise ValueError("x cannot be both periodic and a pressure axis")
    v2n = voxel_to_node(solid, node_xyz)
    N = len(node_xyz)
    adj = np.empty((18, N), dtype=np.int32)
    for i in range(1, 19):
        src = node_xyz - C[i][None, :]
        wall = np.zeros(N, bool)
        inlet = np.zeros(N, bool)
        outlet = np.zeros(N, bool)
        for a in range(3):
            lo = src[:, a] < 0
            hi = src[:, a] >= dims[a]
            if periodic[a]:
                src[:, a] %= dims[a]
            elif a == 0 and x_pressure:
                inlet |= lo
                outlet |= hi
            else:
                wall |= lo | hi
        inside = ~(wall | inlet | outlet)
        vals = np.full(N, MARK_WALL, dtype=np.int64)
        s = src[inside]
        vals[inside] = v2n[s[:, 2], s[:, 1], s[:, 0]]
        vals[~wall & inlet] = MARK_INLET
        vals[~wall & outlet] = MARK_OUTLET
        adj[i - 1] = vals
    return adj


# ---------------------------------------------------------------------------
# RIA run table (Sect. 4.1, Fig. 2b)
# ---------------------------------------------------------------------------

def ria_continues(adj: np.ndarray) -> np.ndarray:
    """cont[n] (n >= 1): node n has node n-1's access pattern shifted by one.

    For every direction either both nodes pull from fluid nodes and the
    source index advances by exactly one, or both carry the same marker (the
    bounce-back source is the node itself, which also advances by one).
    """
    a = adj.astype(np.int64)
    prev, cur = a[:, :-1], a[:, 1:]
    fluid_ok = (prev >= 0) & (cur >= 0) & (cur == prev + 1)
    mark_ok = (prev < 0) & (cur < 0) & (cur == prev)
    return np.all(fluid_ok | mark_ok, axis=0)


def ria_tables(adj: np.ndarray):
    """(run_start[R+1], run_adj[18, R]) of the run-length coded access pattern."""
    N = adj.shape[1]
    if N == 0:
        return np.zeros(1, np.int32), np.zeros((18, 0), np.int32)
    cont = ria_continues(adj)
    heads = np.concatenate([[0], np.nonzero(~cont)[0] + 1]).astype(np.int64)
    run_start = np.concatenate([heads, [N]]).astype(np.int32)
    run_adj = np.ascontiguousarray(adj[:, heads])
    return run_start, run_adj


def ria_decode(run_start: np.ndarray, run_adj: np.ndarray) -> np.ndarray:
    """Expand the run table back into the full adjacency list."""
    N = int(run_start[-1])
    lengths = np.diff(run_start.astype(np.int64))
    run_of = np.repeat(np.arange(len(lengths)), lengths)
    off = np.arange(N) - run_start[:-1].astype(np.int64)[run_of]
    base = run_adj[:, run_of].astype(np.int64)
    return np.where(base >= 0, base + off[None, :], base).astype(np.int32)


def run_histogram(run_start: np.ndarray) -> np.ndarray:
    """hist[b] = number of runs with length in [2^b, 2^(b+1)), b = 0..32."""
    lengths = np.diff(run_start.astype(np.int64))
    hist = np.zeros(33, dtype=np.int64)
    if len(lengths):
        b = np.floor(np.log2(lengths)).astype(np.int64)
        np.add.at(hist, b, 1)
    return hist


def fraction_in_runs_at_least(run_start: np.ndarray, V: int) -> float:
    """Share of nodes in runs of length >= V (the paper's "vectorizable" share, Sect. 4.2)."""
    lengths = np.diff(run_start.astype(np.int64))
    N = lengths.sum()
    return float(lengths[lengths >= V].sum()) / float(N) if N else 0.0


class Tables:
    """All tables of one lattice."""

    def __init__(self, solid, periodic=(0, 0, 0), x_pressure=False, enum="lex", B=1):
        self.solid = solid
        self.shape = solid.shape
        self.periodic = tuple(int(p) for p in periodic)
        self.x_pressure = bool(x_pressure)
        if enum == "lex":
            self.node_xyz = lexicographic_order(solid, B)
        elif enum == "hilbert":
            self.node_xyz = hilbert_order(solid)
        else:
            raise ValueError(enum)
        self.N = len(self.node_xyz)
        self.adj = adjacency(solid, self.node_xyz, self.periodic, self.x_pressure)
        self.run_start, self.run_adj = ria_tables(self.adj)
        self.R = len(self.run_start) - 1


# ---------------------------------------------------------------------------
# Partitioning and the two-stage renumbering (Sect. 1, Sect. 6.1)
# ---------------------------------------------------------------------------

def partition_bounds(N: int, P: int):
    """Chunk p of an equal P-way cut of the node list is [N p / P, N (p+1) / P)."""
    return [(N * p // P, N * (p + 1) // P) for p in range(P)]


def renumber_partitions(node_xyz: np.ndarray, P: int) -> np.ndarray:
    """Cut the node order into P chunks and sort each chunk lexicographically (x fastest)."""
    out = []
    for a, b in partition_bounds(len(node_xyz), P):
        c = node_xyz[a:b]
        out.append(c[np.lexsort((c[:, 0], c[:, 1], c[:, 2]))])
    return np.concatenate(out) if out else node_xyz.copy()


def partition_ghosts(adj: np.ndarray, P: int) -> np.ndarray:
    """PDFs each chunk pulls from fluid nodes of other chunks, per step."""
    N = adj.shape[1]
    g = np.zeros(P, dtype=np.int64)
    for p, (a, b) in enumerate(partition_bounds(N, P)):
        m = adj[:, a:b].astype(np.int64)
        g[p] = int(((m >= 0) & ((m < a) | (m >= b))).sum())
    return g


def partition_local_tables(adj: np.ndarray, P: int):
    """Chunk-local tables of the P-way split (Sect. 6, Sect. 6.1).

    Each process of the paper's distributed run owns chunk p of the node
    vector and receives, every step, the PDFs its nodes pull from other
    chunks.  Reading (the paper does not fix a local layout): chunk p's local
    index space is its own nodes 0 .. Np-1 in order, then ghost slots; a pull
    of direction i from a node of another chunk gets slot Np + k, where k
    numbers chunk p's pulls of direction i from other chunks in local node
    order.  Returns one dict per chunk: ``first``, ``N``, ``adj`` [18, Np]
    (local indices and markers), ``slots`` (largest per-direction ghost count)
    and the ghost map ``q`` (owner chunk), ``dir`` (1..18), ``slot``, ``node``
    (owner-local source node), ordered by owner, direction, slot.
    """
    N = adj.shape[1]
    bounds = partition_bounds(N, P)
    starts = np.array([a for a, _ in bounds], dtype=np.int64)
    out = []
    for a, b in bounds:
        Np = b - a
        A = adj[:, a:b].astype(np.int64)
        local = np.where(A >= 0, A - a, A)
        foreign = (A >= 0) & ((A < a) | (A >= b))
        q_l, d_l, s_l, m_l = [], [], [], []
        slots = 0
        for i in range(18):
            cols = np.nonzero(foreign[i])[0]           # local nodes, ascending
            slot = Np + np.arange(len(cols))
            local[i, cols] = slot
            src = A[i, cols]
            q = np.searchsorted(starts, src, side="right") - 1
            q_l.append(q)
            d_l.append(np.full(len(cols), i + 1))
            s_l.append(slot)
            m_l.append(src - starts[q])
            slots = max(slots, len(cols))
        q = np.concatenate(q_l) if q_l else np.zeros(0, np.int64)
        order = np.argsort(q, kind="stable")
        out.append({
            "first": a, "N": Np, "adj": local.astype(np.int32), "slots": slots,
            "q": q[order].astype(np.int32), "dir": np.concatenate(d_l)[order].astype(np.int32),
            "slot": np.concatenate(s_l)[order].astype(np.int32),
            "node": np.concatenate(m_l)[order].astype(np.int32),
        })
    return out
