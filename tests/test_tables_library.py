"""Bit-exact agreement of the library's host lattice builder with the oracle.

Enumeration (LS with blocking factor B, Hilbert; Sect. 5.6), adjacency list
(Sect. 4, Fig. 2a) and RIA run table (Sect. 4.1) must be identical integer
for integer.  These run on the CPU: the builder is host C++.
"""
import numpy as np
import pytest

import geometry
from oracle import tables
import paper_1410_0412_gb300 as lbm


def _compare(solid, periodic, x_pressure, enum, B):
    lat = lbm.Lattice(solid, periodic=periodic, x_pressure=x_pressure, enum=enum, B=B)
    ref = tables.Tables(solid, periodic=periodic, x_pressure=x_pressure, enum=enum, B=B)
    t = lat.tables()
    assert lat.N == ref.N and lat.R == ref.R
    assert np.array_equal(t["node_xyz"], ref.node_xyz.astype(np.int32))
    assert np.array_equal(t["adj"], ref.adj)
    assert np.array_equal(t["run_start"], ref.run_start)
    assert np.array_equal(t["run_adj"], ref.run_adj)
    assert np.array_equal(lat.run_hist, tables.run_histogram(ref.run_start))
    lat.validate()
    return lat


BCS = [((0, 0, 0), False), ((1, 0, 0), False), ((1, 1, 1), False), ((0, 1, 0), True), ((0, 0, 1), True)]


@pytest.mark.parametrize("bc", range(len(BCS)))
@pytest.mark.parametrize("enum,B", [("lex", 1), ("lex", 2), ("lex", 3), ("lex", 5), ("hilbert", 1)])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_random_boxes_exhaustive(bc, enum, B, seed):
    periodic, xp = BCS[bc]
    dims = [(7, 5, 6), (9, 4, 3), (5, 8, 7)][seed]
    solid = geometry.random_voxels(*dims, 0.1 + 0.15 * seed, 100 * bc + seed)
    _compare(solid, periodic, xp, enum, B)


def test_degenerate_boxes():
    # all solid, a single fluid voxel, a 1-voxel-thick slab, a fully fluid periodic box
    for solid, per, xp in [
        (np.ones((3, 4, 5), np.uint8), (0, 0, 0), False),
        (np.pad(np.zeros((1, 1, 1), np.uint8), 1, constant_values=1), (1, 1, 1), False),
        (np.zeros((1, 6, 5), np.uint8), (0, 0, 1), False),
        (np.zeros((4, 4, 4), np.uint8), (1, 1, 1), False),
        (np.zeros((3, 3, 1), np.uint8), (0, 1, 1), True),
    ]:
        for enum, B in [("lex", 1), ("lex", 2), ("hilbert", 1)]:
            _compare(solid, per, xp, enum, B)


@pytest.mark.parametrize("enum,B", [("lex", 1), ("lex", 8), ("lex", 16), ("lex", 32), ("lex", 64), ("hilbert", 1)])
def test_sphere_box_64x32x32(enum, B):
    solid = geometry.sphere_box_64x32x32(0)
    _compare(solid, (1, 0, 0), False, enum, B)


@pytest.mark.parametrize("enum,B", [("lex", 1), ("lex", 16), ("hilbert", 1)])
def test_packed_bed_crop_96(enum, B):
    solid, _ = geometry.rsa_spheres(96, 96, 96, 12.0, 1, periodic=(1, 0, 0), max_consecutive_rejections=2000)
    _compare(solid, (1, 0, 0), False, enum, B)


@pytest.mark.slow
def test_paper_channel_tables():
    solid = geometry.square_channel(100, 100, 500)
    lat = _compare(solid, (0, 0, 1), False, "lex", 1)
    assert lat.R * 98 == 3 * lat.N


def test_from_adjacency_and_validate_catches_corruption():
    solid = geometry.random_voxels(6, 5, 4, 0.2, 7)
    ref = tables.Tables(solid, periodic=(1, 0, 0))
    lat = lbm.Lattice.from_adjacency(ref.adj, ref.node_xyz)
    t = lat.tables()
    assert np.array_equal(t["adj"], ref.adj) and np.array_equal(t["run_start"], ref.run_start)
    lat.validate()
    bad = ref.adj.copy()
    n = int(np.argmax(bad[0] >= 0))
    bad[0, n] = (bad[0, n] + 1) % ref.N          # breaks reciprocity
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice.from_adjacency(bad).validate()
    assert e.value.code == 4
    bad = ref.adj.copy()
    bad[3, 0] = ref.N + 5                         # out of range
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice.from_adjacency(bad).validate()
    assert e.value.code == 4
    bad = ref.adj.copy()
    bad[5, 1] = -7                                # unknown marker
    with pytest.raises(lbm.LbmError):
        lbm.Lattice.from_adjacency(bad).validate()


def test_argument_errors():
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(np.zeros((2, 2, 2), np.uint8), periodic=(1, 0, 0), x_pressure=True)
    assert e.value.code == 1
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(np.zeros((2, 2, 2), np.uint8), enum="lex", B=0)


def test_adjacency_rows_export():
    solid = geometry.random_voxels(9, 7, 6, 0.2, 12)
    lat = lbm.Lattice(solid, periodic=(0, 1, 0), x_pressure=True)
    full = lat.tables()["adj"]
    nodes = np.array([0, 5, lat.N - 1, 3, 3])
    assert np.array_equal(lat.adjacency_rows(nodes), full[:, nodes])
    with pytest.raises(lbm.LbmError):
        lat.adjacency_rows(np.array([lat.N]))


@pytest.mark.parametrize("dims", [(2048, 2, 2), (3, 1025, 2), (2, 3, 700), (130, 33, 65)])
def test_hilbert_deep_curves(dims):
    # long thin boxes reach the deepest curve levels the builder supports (2^11
    # per axis) at a few thousand voxels, so every level of the index is checked
    X, Y, Z = dims
    solid = geometry.random_voxels(X, Y, Z, 0.2, X + Y + Z)
    _compare(solid, (0, 0, 0), False, "hilbert", 1)


@pytest.mark.parametrize("enum,B", [("lex", 1), ("lex", 4), ("hilbert", 1)])
def test_tables_do_not_depend_on_host_threads(enum, B, monkeypatch):
    # the builders split nodes, slabs and runs into per-thread chunks; runs and
    # phantom locations that cross a chunk boundary must come out the same
    solid = geometry.random_voxels(37, 29, 23, 0.3, 11)
    out = []
    for threads in ("1", "3", "7"):
        monkeypatch.setenv("LBM_HOST_THREADS", threads)
        lat = lbm.Lattice(solid, periodic=(1, 0, 0), x_pressure=False, enum=enum, B=B)
        t = lat.tables()
        nb, mask = lat.et_tables()
        out.append((t["node_xyz"], t["adj"], t["run_start"], t["run_adj"], nb, mask, lat.et_runs()))
    for other in out[1:]:
        for a, b in zip(out[0][:6], other[:6]):
            assert np.array_equal(a, b)
        for a, b in zip(out[0][6], other[6]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("case", [((1, 0, 0), "lex", 1, 0), ((1, 1, 1), "lex", 4, 1), ((0, 0, 0), "hilbert", 1, 2)])
def test_run_slot_tables_match_the_oracle_tables(case):
    """The run slot tables the RIA steps read: with h the first node of run r
    and a its adjacency entry for direction i (oracle tables), the AA odd step's
    slot is inv(i) Npad + a for a fluid source and i Npad + h through a wall;
    the OS-NT step's is i Npad + a or inv(i) Npad + h.  Lattices with pressure
    faces have no such tables."""
    from oracle.d3q19 import INV
    periodic, enum, B, seed = case
    solid = geometry.random_voxels(11, 9, 7, 0.25, 40 + seed)
    lat = lbm.Lattice(solid, periodic=periodic, enum=enum, B=B)
    ref = tables.Tables(solid, periodic=periodic, enum=enum, B=B)
    heads = ref.run_start[:-1].astype(np.int64)
    Np = lat.Npad
    want_aa = np.empty((ref.R, 18), np.int64)
    want_osnt = np.empty((ref.R, 18), np.int64)
    for i in range(1, 19):
        a = ref.adj[i - 1, heads].astype(np.int64)
        fluid = a >= 0
        want_aa[:, i - 1] = np.where(fluid, int(INV[i]) * Np + a, i * Np + heads)
        want_osnt[:, i - 1] = np.where(fluid, i * Np + a, int(INV[i]) * Np + heads)
    assert np.array_equal(lat.run_slots(0), want_aa)
    assert np.array_equal(lat.run_slots(1), want_osnt)
    xp = lbm.Lattice(solid, periodic=(0, 1, 1), x_pressure=True)
    assert xp.run_slots(0) is None and xp.run_slots(1) is None
    with pytest.raises(lbm.LbmError):
        lat.run_slots(2)
