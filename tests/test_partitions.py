"""Partitioning of the node list and the two-stage renumbering (Sect. 1, Sect. 6.1).

The oracle's versions are pinned by brute force and invariants; the library's
are bit-exact against them; and the paper's qualitative claims hold on a bed
crop: the Hilbert order cuts far fewer links than plain LS, and renumbering
each Hilbert chunk lexicographically restores long runs at the same ghost
count.
"""
import numpy as np
import pytest

import geometry
from oracle import tables
import paper_1410_0412_gb300 as lbm


def _brute_ghosts(adj, P):
    N = adj.shape[1]
    owner = np.zeros(N, dtype=np.int64)
    for p in range(P):
        owner[N * p // P:N * (p + 1) // P] = p
    g = np.zeros(P, dtype=np.int64)
    for n in range(N):
        for i in range(18):
            m = adj[i, n]
            if m >= 0 and owner[m] != owner[n]:
                g[owner[n]] += 1
    return g


def test_oracle_partition_pins():
    solid = geometry.random_voxels(9, 8, 7, 0.2, 4)
    T = tables.Tables(solid, periodic=(1, 0, 0))
    for P in (1, 2, 3, 7):
        g = tables.partition_ghosts(T.adj, P)
        assert np.array_equal(g, _brute_ghosts(T.adj, P))
        # each cross-chunk link is pulled once from each side
        assert g.sum() % 2 == 0
        order = tables.renumber_partitions(T.node_xyz, P)
        assert sorted(map(tuple, order)) == sorted(map(tuple, T.node_xyz))
        for a, b in tables.partition_bounds(T.N, P):
            assert sorted(map(tuple, order[a:b])) == sorted(map(tuple, T.node_xyz[a:b]))
            z, y, x = order[a:b, 2], order[a:b, 1], order[a:b, 0]
            key = (z * 8 + y) * 9 + x
            assert np.all(np.diff(key) > 0)
    assert tables.partition_ghosts(T.adj, 1)[0] == 0


@pytest.mark.parametrize("enum", ["lex", "hilbert"])
@pytest.mark.parametrize("P", [1, 4, 13])
def test_library_matches_oracle(enum, P):
    solid = geometry.sphere_box_64x32x32(0)
    lat = lbm.Lattice(solid, periodic=(1, 0, 0), enum=enum)
    T = tables.Tables(solid, periodic=(1, 0, 0), enum=enum)
    assert np.array_equal(lat.partition_ghosts(P), tables.partition_ghosts(T.adj, P))
    order = lat.renumber_partitions(P)
    assert np.array_equal(order, tables.renumber_partitions(T.node_xyz, P).astype(np.int32))
    re = lbm.Lattice.from_order(solid, order, periodic=(1, 0, 0))
    ref_adj = tables.adjacency(solid, order.astype(np.int64), (1, 0, 0))
    t = re.tables()
    assert np.array_equal(t["adj"], ref_adj)
    assert np.array_equal(t["run_start"], tables.ria_tables(ref_adj)[0])
    re.validate()


def test_from_order_rejects_bad_orders():
    solid = geometry.random_voxels(5, 4, 3, 0.3, 2)
    T = tables.Tables(solid)
    bad = T.node_xyz.copy()
    bad[1] = bad[0]
    with pytest.raises(lbm.LbmError):
        lbm.Lattice.from_order(solid, bad)
    with pytest.raises(lbm.LbmError):
        lbm.Lattice.from_order(solid, T.node_xyz[:-1])


def test_paper_claims_hilbert_renumbering():
    """Sect. 6 / 6.1 on a 96^3 bed crop, P = 16: Hilbert cuts fewer links than LS B = 1,
    and Hilbert + per-chunk LS renumbering keeps Hilbert's ghosts with far fewer runs."""
    solid, _ = geometry.rsa_spheres(96, 96, 96, 12.0, 1, periodic=(1, 0, 0), max_consecutive_rejections=2000)
    P = 16
    ls = lbm.Lattice(solid, periodic=(1, 0, 0), enum="lex", B=1)
    hb = lbm.Lattice(solid, periodic=(1, 0, 0), enum="hilbert")
    rn = lbm.Lattice.from_order(solid, hb.renumber_partitions(P), periodic=(1, 0, 0))
    g_ls, g_hb, g_rn = ls.partition_ghosts(P), hb.partition_ghosts(P), rn.partition_ghosts(P)
    assert g_hb.max() < g_ls.max()
    assert np.array_equal(g_rn, g_hb)          # the same node sets per chunk
    assert rn.R < 0.5 * hb.R                   # runs restored inside the chunks
