"""The library's Esoteric Twist tables against the oracle's, bit for bit (CPU).

Locations of the six neighbour slots, the phantom locations and their
coordinates, and the link mask must equal ``oracle.esotwist.tables`` for every
boundary kind and enumeration.
"""
import ctypes

import numpy as np
import pytest

import geometry
from oracle import esotwist as et
from oracle import tables
import paper_1410_0412_gb300 as lbm

CASES = [
    dict(periodic=(1, 0, 0), x_pressure=False),
    dict(periodic=(1, 1, 1), x_pressure=False),
    dict(periodic=(0, 0, 1), x_pressure=True),
    dict(periodic=(0, 0, 0), x_pressure=False),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("enum", [("lex", 1), ("lex", 3), ("hilbert", 1)])
def test_et_tables_match_oracle(case, enum):
    solid = geometry.random_voxels(13, 11, 9, 0.25, 120 + case)
    lat = lbm.Lattice(solid, enum=enum[0], B=enum[1], **CASES[case])
    T = tables.Tables(solid, enum=enum[0], B=enum[1], **CASES[case])
    nb, mask, ph = et.tables(solid, T.node_xyz, T.adj, CASES[case]["periodic"])
    S, Spad, lph = lat.et_info()
    lnb, lmask = lat.et_tables()
    assert S == T.N + len(ph) and Spad % 128 == 0 and Spad >= S
    assert np.array_equal(lnb, nb)
    assert np.array_equal(lmask, mask)
    assert np.array_equal(lph, ph)


def test_et_tables_sphere_box():
    solid = geometry.sphere_box_64x32x32(0)
    lat = lbm.Lattice(solid, periodic=(1, 0, 0))
    T = tables.Tables(solid, periodic=(1, 0, 0))
    nb, mask, ph = et.tables(solid, T.node_xyz, T.adj, (1, 0, 0))
    lnb, lmask = lat.et_tables()
    assert np.array_equal(lnb, nb) and np.array_equal(lmask, mask)
    assert np.array_equal(lat.et_info()[2], ph)


def test_et_refused_where_undefined():
    solid = geometry.random_voxels(9, 8, 7, 0.25, 130)
    lat = lbm.Lattice(solid, periodic=(1, 0, 0))
    # a lattice from a bare adjacency list has no coordinates for its phantom locations
    bare = lbm.Lattice.from_adjacency(lat.tables(node_xyz=False, runs=False)["adj"])
    with pytest.raises(lbm.LbmError) as e:
        bare.et_info()
    assert e.value.code == lbm._lib.LBM_ERR_UNSUPPORTED
    # a fully periodic box of fluid needs no phantoms, so coordinates are not needed
    full = lbm.Lattice(np.zeros((4, 5, 6), np.uint8), periodic=(1, 1, 1))
    bare_full = lbm.Lattice.from_adjacency(full.tables(node_xyz=False, runs=False)["adj"])
    assert bare_full.et_info()[0] == full.N
    # a partition's local lattice has ghost slots, not locations
    part = lbm.Partitioning(lat, 2)
    with pytest.raises(lbm.LbmError):
        part.parts[0].et_info()
    # stepping without the ET tables on the device is refused before any launch
    lib = lbm._lib.load()
    prm = lbm.Params().c()
    assert lib.lbm_step_et(lat.handle, 0, ctypes.byref(prm), ctypes.c_void_p(256), 0, None, 0, None) == \
        lbm._lib.LBM_ERR_ARG
    assert lib.lbm_step_et(lat.handle, 0, ctypes.byref(prm), ctypes.c_void_p(256), 2, None, 1, None) == \
        lbm._lib.LBM_ERR_ARG


def test_et_empty_lattice():
    lat = lbm.Lattice(np.ones((3, 3, 3), np.uint8))
    S, Spad, ph = lat.et_info()
    assert S == 0 and len(ph) == 0


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("enum", [("lex", 1), ("hilbert", 1)])
def test_et_runs_match_oracle(case, enum):
    solid = geometry.random_voxels(13, 11, 9, 0.25, 180 + case)
    lat = lbm.Lattice(solid, enum=enum[0], B=enum[1], **CASES[case])
    T = tables.Tables(solid, enum=enum[0], B=enum[1], **CASES[case])
    nb, mask, _ = et.tables(solid, T.node_xyz, T.adj, CASES[case]["periodic"])
    rs, rnb, rmask = et.run_tables(nb, mask)
    lrs, lrnb, lrmask = lat.et_runs()
    assert np.array_equal(lrs, rs) and np.array_equal(lrnb, rnb) and np.array_equal(lrmask, rmask)


def test_et_runs_paper_channel():
    """The paper's channel cross-section rows: three ET runs per 98-node row, as for RIA."""
    solid = geometry.square_channel(100, 100, 8)
    lat = lbm.Lattice(solid, periodic=(0, 0, 1))
    rs, _, _ = lat.et_runs()
    assert len(rs) - 1 == 3 * 98 * 8


@pytest.mark.parametrize("dims,periodic", [((1, 8, 1), (1, 0, 1)), ((3, 1, 4), (1, 1, 0)), ((2, 2, 2), (1, 1, 1)),
                                           ((5, 4, 1), (0, 0, 1))])
def test_et_tables_degenerate_boxes(dims, periodic):
    solid = geometry.empty_box(*dims)
    lat = lbm.Lattice(solid, periodic=periodic)
    T = tables.Tables(solid, periodic=periodic)
    nb, mask, ph = et.tables(solid, T.node_xyz, T.adj, periodic)
    lnb, lmask = lat.et_tables()
    assert np.array_equal(lnb, nb) and np.array_equal(lmask, mask)
    assert np.array_equal(lat.et_info()[2], ph)
    rs, rnb, rm = et.run_tables(nb, mask)
    lrs, lrnb, lrm = lat.et_runs()
    assert np.array_equal(lrs, rs) and np.array_equal(lrnb, rnb) and np.array_equal(lrm, rm)
