"""Pins of the oracle's enumeration, adjacency and RIA tables.

Brute force on tiny boxes (plain Python loops over voxels), the Hilbert
curve's defining properties, adjacency reciprocity, lossless run-length
decoding, and the paper's printed channel figures (Sect. 5.1, Table 2,
Sect. 5.6).
"""
import json
import os

import numpy as np
import pytest

import geometry
from oracle import d3q19, tables

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def _brute_lex(solid, B):
    Z, Y, X = solid.shape
    keys = []
    for z in range(Z):
        for y in range(Y):
            for x in range(X):
                if solid[z, y, x] == 0:
                    keys.append(((z // B, y // B, x // B, z, y, x), (x, y, z)))
    keys.sort()
    return np.array([k[1] for k in keys], dtype=np.int64).reshape(-1, 3)


@pytest.mark.parametrize("B", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("seed", [0, 1])
def test_lexicographic_blocked_bruteforce(B, seed):
    solid = geometry.random_voxels(7, 5, 6, 0.3, seed)
    assert np.array_equal(tables.lexicographic_order(solid, B), _brute_lex(solid, B))


def test_lexicographic_large_block_equals_plain():
    solid = geometry.random_voxels(9, 7, 5, 0.25, 3)
    a = tables.lexicographic_order(solid, 1)
    for B in (9, 10, 64):
        assert np.array_equal(tables.lexicographic_order(solid, B), a)


@pytest.mark.parametrize("bits", [1, 2, 3, 4])
def test_hilbert_curve_properties(bits):
    n = 1 << bits
    g = np.arange(n ** 3)
    x, y, z = g % n, (g // n) % n, g // (n * n)
    key = tables.hilbert_keys(x, y, z, bits).astype(np.int64)
    # bijection onto 0 .. n^3 - 1
    assert np.array_equal(np.sort(key), np.arange(n ** 3))
    order = np.argsort(key)
    pts = np.stack([x[order], y[order], z[order]], 1)
    # consecutive points are lattice neighbours (unit Manhattan steps)
    assert np.all(np.abs(np.diff(pts, axis=0)).sum(1) == 1)
    # the curve starts at the origin
    assert np.all(pts[0] == 0)
    # each octant is visited as one contiguous block of n^3/8 indices (self-similarity)
    if bits > 1:
        h = n // 2
        octant = (pts[:, 0] >= h) * 1 + (pts[:, 1] >= h) * 2 + (pts[:, 2] >= h) * 4
        blocks = octant.reshape(8, -1)
        assert np.all(blocks == blocks[:, :1])
        assert len(set(blocks[:, 0])) == 8


def _brute_adjacency(solid, node_xyz, periodic, x_pressure):
    Z, Y, X = solid.shape
    dims = (X, Y, Z)
    v2n = {}
    for n, (x, y, z) in enumerate(node_xyz):
        v2n[(int(x), int(y), int(z))] = n
    adj = np.zeros((18, len(node_xyz)), dtype=np.int64)
    for n, xyz in enumerate(node_xyz):
        for i in range(1, 19):
            s = [int(xyz[a] - d3q19.C[i][a]) for a in range(3)]
            mark = None
            for a in range(3):
                if 0 <= s[a] < dims[a]:
                    continue
                if periodic[a]:
                    s[a] %= dims[a]
                elif a == 0 and x_pressure:
                    if mark is None:
                        mark = -2 if s[a] < 0 else -3
                else:
                    mark = -1
                    break
            if mark is None:
                mark = v2n.get(tuple(s), -1)
            adj[i - 1, n] = mark
    return adj


CASES = [
    dict(periodic=(0, 0, 0), x_pressure=False),
    dict(periodic=(1, 0, 0), x_pressure=False),
    dict(periodic=(1, 1, 1), x_pressure=False),
    dict(periodic=(0, 1, 0), x_pressure=True),
    dict(periodic=(0, 0, 0), x_pressure=True),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("enum", ["lex1", "lex2", "hilbert"])
def test_adjacency_bruteforce(case, enum):
    bc = CASES[case]
    solid = geometry.random_voxels(6, 5, 4, 0.3, 10 + case)
    e, B = ("hilbert", 1) if enum == "hilbert" else ("lex", int(enum[3:]))
    T = tables.Tables(solid, enum=e, B=B, **bc)
    assert np.array_equal(T.adj, _brute_adjacency(solid, T.node_xyz, bc["periodic"], bc["x_pressure"]))


@pytest.mark.parametrize("case", range(len(CASES)))
def test_adjacency_reciprocity_and_link_count(case):
    bc = CASES[case]
    solid = geometry.random_voxels(8, 7, 6, 0.35, 20 + case)
    T = tables.Tables(solid, enum="lex", B=1, **bc)
    adj = T.adj.astype(np.int64)
    inv = d3q19.INV
    for i in range(1, 19):
        m = adj[i - 1]
        f = m >= 0
        back = adj[inv[i] - 1][m[f]]
        assert np.array_equal(back, np.nonzero(f)[0])
    # every -1 entry is one fluid-solid (or fluid-wall) link counted on the dense grid
    Z, Y, X = solid.shape
    dims = (X, Y, Z)
    links = 0
    for (x, y, z) in T.node_xyz:
        for i in range(1, 19):
            s = [x - d3q19.C[i][0], y - d3q19.C[i][1], z - d3q19.C[i][2]]
            wall = False
            press = False
            for a in range(3):
                if not (0 <= s[a] < dims[a]):
                    if bc["periodic"][a]:
                        s[a] %= dims[a]
                    elif a == 0 and bc["x_pressure"]:
                        press = True
                    else:
                        wall = True
            if wall or (not press and solid[s[2], s[1], s[0]]):
                links += 1
    assert int((adj == -1).sum()) == links


def _brute_runs(adj):
    N = adj.shape[1]
    heads = [0]
    for n in range(1, N):
        same = True
        for i in range(18):
            a, b = int(adj[i, n - 1]), int(adj[i, n])
            if a >= 0 and b >= 0:
                ok = b == a + 1
            else:
                ok = (a < 0 and b < 0 and a == b)
            if not ok:
                same = False
                break
        if not same:
            heads.append(n)
    return np.array(heads + [N])


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("enum", ["lex1", "lex3", "hilbert"])
def test_ria_bruteforce_and_decode(case, enum):
    bc = CASES[case]
    solid = geometry.random_voxels(9, 6, 5, 0.2, 30 + case)
    e, B = ("hilbert", 1) if enum == "hilbert" else ("lex", int(enum[3:]))
    T = tables.Tables(solid, enum=e, B=B, **bc)
    assert np.array_equal(T.run_start, _brute_runs(T.adj))
    assert np.array_equal(T.run_adj, T.adj[:, T.run_start[:-1]])
    assert np.array_equal(tables.ria_decode(T.run_start, T.run_adj), T.adj)
    h = tables.run_histogram(T.run_start)
    assert h.sum() == T.R
    assert (np.diff(T.run_start) * 1).sum() == T.N


def test_empty_and_single_node_lattices():
    solid = np.ones((3, 3, 3), np.uint8)
    T = tables.Tables(solid)
    assert T.N == 0 and T.R == 0 and T.adj.shape == (18, 0)
    solid[1, 1, 1] = 0
    T = tables.Tables(solid)
    assert T.N == 1 and T.R == 1 and np.all(T.adj == -1)
    T = tables.Tables(solid, periodic=(1, 1, 1))
    assert np.all(T.adj == -1)   # all neighbours are solid voxels


@pytest.mark.slow
def test_paper_channel_run_table():
    """Channel of Sect. 5.1 (500 x 100 x 100, long axis along z here).

    Every 98-node row splits into runs {first}, {2..97}, {last}: r = R/N = 3/98,
    which reproduces Table 2's channel loop balances (306 and 305 B/FLUP) and
    the 98 % SIMD share of Sect. 5.1 (runs of at least V = 4 nodes, Sect. 4.2).
    LS with B = 1 and B = 100 give the same order (Sect. 5.6).
    """
    g = GOLD
    L, D = g["channel"]["dims_long_first"][0], g["channel"]["dims_long_first"][1]
    solid = geometry.square_channel(D, D, L)
    T = tables.Tables(solid, periodic=(0, 0, 1), enum="lex", B=1)
    assert abs(T.N - g["channel"]["fluid_nodes_approx"]) / T.N < 0.01
    r = T.R / T.N
    assert T.R * 98 == 3 * T.N
    Dpdf, Didx, Dblk = g["D_pdf_B"]["value"], g["D_idx_B"]["value"], g["D_block_B"]["value"]
    tab = g["loop_balance_table"]["channel"]
    assert round(Dpdf + Didx) == tab[0]
    assert round(Dpdf + (Didx + Dblk) * r) == tab[1]
    assert round(Dpdf + Didx / 2) == tab[2]
    assert round(Dpdf + (Didx + Dblk) / 2 * r) == tab[3]
    V = g["channel"]["simd_width_V"]
    assert round(100 * tables.fraction_in_runs_at_least(T.run_start, V)) == g["channel"]["vectorizable_percent"]
    # Sect. 5.6 enumeration identity
    assert np.array_equal(tables.lexicographic_order(solid, 100), T.node_xyz)


def test_loop_balance_bounds():
    """Sect. 4.1 bounds follow from D_pdf, D_idx and D_block at r = 0 and r = 1."""
    g = GOLD
    Dpdf, Didx, Dblk = g["D_pdf_B"]["value"], g["D_idx_B"]["value"], g["D_block_B"]["value"]
    assert [Dpdf, Dpdf + Didx + Dblk] == g["B_l_OSNT_R_bounds"]["value"]
    assert [Dpdf, Dpdf + (Didx + Dblk) / 2] == g["B_l_AA_R_bounds"]["value"]
    assert 2 * 19 * 8 == Dpdf and 18 * 4 == Didx
