"""Chunk-local tables and the ghost-PDF exchange of a P-chunk split (Sect. 6).

Pins of the oracle: its local tables decode back to the whole lattice's
adjacency list, their ghost count is the brute-force count of cross-chunk
pulls, and the ghost slots follow the stated numbering; an OS-NT step done
chunk by chunk with an exchange equals the whole-lattice step to round-off.
The library's local tables, ghost maps and local RIA tables are bit-exact
against the oracle's.
"""
import ctypes

import numpy as np
import pytest
import torch

import geometry
from oracle import lbm as olbm
from oracle import tables
import paper_1410_0412_gb300 as lbm

CASES = [
    dict(periodic=(1, 0, 0), x_pressure=False),
    dict(periodic=(1, 1, 1), x_pressure=False),
    dict(periodic=(0, 0, 1), x_pressure=True),
]


def _decode(part, starts):
    """Whole-lattice adjacency rows of a chunk from its local table and ghost map."""
    A = part["adj"].astype(np.int64)
    out = np.where(A >= 0, A + part["first"], A)
    src = {}
    for q, d, s, m in zip(part["q"], part["dir"], part["slot"], part["node"]):
        assert (d, s) not in src
        src[(int(d), int(s))] = int(starts[q] + m)
    for i in range(18):
        for n in np.nonzero(A[i] >= part["N"])[0]:
            out[i, n] = src[(i + 1, int(A[i, n]))]
    return out


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("P", [1, 2, 3, 7])
def test_oracle_local_tables_pins(case, P):
    solid = geometry.random_voxels(9, 8, 7, 0.2, 30 + case)
    T = tables.Tables(solid, enum="hilbert", **CASES[case])
    parts = tables.partition_local_tables(T.adj, P)
    starts = np.array([p["first"] for p in parts])
    ghosts = tables.partition_ghosts(T.adj, P)
    for k, part in enumerate(parts):
        a, n = part["first"], part["N"]
        assert np.array_equal(_decode(part, starts), T.adj[:, a:a + n])
        assert len(part["dir"]) == ghosts[k]
        assert np.all(part["q"] != k)
        # slots of each direction: Np, Np+1, ... in local node order
        for i in range(18):
            cols = np.nonzero(part["adj"][i] >= n)[0]
            assert np.array_equal(part["adj"][i, cols], n + np.arange(len(cols)))
        assert part["slots"] == max([0] + [int((part["adj"][i] >= n).sum()) for i in range(18)])
        # exchange order: owner ascending, then direction, then slot
        key = part["q"].astype(np.int64) * 10**9 + part["dir"].astype(np.int64) * 10**7 + part["slot"]
        assert np.all(np.diff(key) > 0)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("P", [2, 5])
def test_oracle_partitioned_osnt_equals_whole(case, P):
    solid = geometry.random_voxels(8, 7, 6, 0.25, 40 + case)
    T = tables.Tables(solid, enum="hilbert", **CASES[case])
    p = olbm.Params(omega_plus=1.1, magic=3 / 16, g=(1e-4, 2e-5, -3e-5), rho_in=1.001, rho_out=0.999)
    s = torch.as_tensor(geometry.uniform_field(T.N, 5 + case), dtype=torch.float64) * 0.5
    gen = torch.Generator().manual_seed(case)
    F0 = olbm.uniform_state(T.N, p, 1.0, (0.01, -0.02, 0.005))
    F0 = F0 * (1 + 1e-2 * (torch.rand(F0.shape, generator=gen, dtype=torch.float64) - 0.5))
    G = olbm.from_canonical(F0, 0, T.adj, p)
    parts = tables.partition_local_tables(T.adj, P)
    grids = []
    for part in parts:
        g = torch.zeros((19, part["N"] + part["slots"]), dtype=torch.float64)
        g[:, :part["N"]] = G[:, part["first"]:part["first"] + part["N"]]
        grids.append(g)
    for _ in range(5):
        G = olbm.osnt_step(G, T.adj, p, s)
        grids = olbm.partitioned_osnt_step(grids, parts, p, s)
    joined = torch.cat([g[:, :part["N"]] for g, part in zip(grids, parts)], dim=1)
    # equal up to the summation order inside the oracle's matrix products,
    # which depends on the column count; a misrouted ghost PDF errs by ~1e-3
    assert torch.max(torch.abs(joined - G)) <= 4e-16


def test_oracle_partitioned_step_needs_the_exchange():
    """Planted mistake: skipping the ghost copy changes the result."""
    solid = geometry.random_voxels(8, 7, 6, 0.25, 41)
    T = tables.Tables(solid, periodic=(1, 1, 1))
    p = olbm.Params(omega_plus=1.1, g=(1e-4, 0, 0))
    F0 = olbm.uniform_state(T.N, p, 1.0, (0.02, 0.0, 0.0))
    G = olbm.from_canonical(F0, 0, T.adj, p)
    parts = tables.partition_local_tables(T.adj, 3)
    grids = [torch.zeros((19, q["N"] + q["slots"]), dtype=torch.float64) for q in parts]
    for g, q in zip(grids, parts):
        g[:, :q["N"]] = G[:, q["first"]:q["first"] + q["N"]]
    no_ghost = [olbm.collide(olbm.stream(g, q["adj"], p), p) for g, q in zip(grids, parts)]
    whole = olbm.osnt_step(G, T.adj, p)
    assert not torch.equal(torch.cat(no_ghost, dim=1), whole)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("enum", ["lex", "hilbert"])
@pytest.mark.parametrize("P", [1, 2, 7])
def test_library_local_tables_match_oracle(case, enum, P):
    solid = geometry.random_voxels(11, 9, 8, 0.2, 50 + case)
    lat = lbm.Lattice(solid, enum=enum, **CASES[case])
    T = tables.Tables(solid, enum=enum, **CASES[case])
    part = lbm.Partitioning(lat, P)
    part.validate(lat)
    ref = tables.partition_local_tables(T.adj, P)
    for k, r in enumerate(ref):
        loc = part.parts[k]
        assert (part.first[k], part.sizes[k], part.ghost_slots[k]) == (r["first"], r["N"], r["slots"])
        assert loc.N == r["N"] and loc.Npad >= r["N"] + r["slots"]
        t = loc.tables()
        assert np.array_equal(t["adj"], r["adj"])
        rs, ra = tables.ria_tables(r["adj"])
        assert np.array_equal(t["run_start"], rs) and np.array_equal(t["run_adj"], ra)
        g = part.ghosts(k)
        for key in ("q", "dir", "slot", "node"):
            lib_key = "src_part" if key == "q" else ("src_node" if key == "node" else key)
            assert np.array_equal(g[lib_key], r[key]), key
        loc.validate()
    assert np.array_equal(np.array(part.ghost_pdfs), lat.partition_ghosts(P))


def test_partition_bad_arguments():
    solid = geometry.random_voxels(6, 5, 4, 0.2, 60)
    lat = lbm.Lattice(solid, periodic=(1, 0, 0))
    for P in (0, -1, lat.N + 1):
        with pytest.raises(lbm.LbmError):
            lbm.Partitioning(lat, P)
    part = lbm.Partitioning(lat, 2)
    lib = lbm._lib.load()
    loc = part.parts[0]
    prm = lbm.Params().c()
    # whole-lattice operations are refused on a chunk before touching any pointer
    assert lib.lbm_adjoint_step(loc.handle, 0, ctypes.byref(prm), None, None, None, None, None, 0, None) == \
        lbm._lib.LBM_ERR_UNSUPPORTED
    assert lib.lbm_objective_flux(loc.handle, 0, ctypes.byref(prm), None, 0, None, None, None, None, None, 0,
                                  None) == lbm._lib.LBM_ERR_UNSUPPORTED
    assert lib.lbm_load_canonical(loc.handle, 0, ctypes.byref(prm), None, None, 0, None) == \
        lbm._lib.LBM_ERR_UNSUPPORTED
    # the exchange refuses to run before its table is on the device
    assert lib.lbm_halo_exchange(part.handle, 0, None, 0, None) == lbm._lib.LBM_ERR_ARG
    # a partitioning of another lattice does not validate
    other = lbm.Lattice(geometry.random_voxels(6, 5, 4, 0.2, 61), periodic=(1, 0, 0))
    with pytest.raises(lbm.LbmError):
        part.validate(other)
    # freeing the partitioning leaves the chunk wrappers inert
    part.close()
    assert not loc.handle


def test_empty_lattice_partition():
    lat = lbm.Lattice(np.ones((3, 3, 3), np.uint8))
    part = lbm.Partitioning(lat, 1)
    assert part.sizes == [0] and part.ghost_pdfs == [0]
    part.validate(lat)


def test_one_node_per_chunk():
    """P = N: every pull from a fluid neighbour is a ghost; tables still match the oracle."""
    solid = geometry.random_voxels(5, 4, 3, 0.2, 1)
    lat = lbm.Lattice(solid, periodic=(1, 1, 0))
    T = tables.Tables(solid, periodic=(1, 1, 0))
    part = lbm.Partitioning(lat, lat.N)
    part.validate(lat)
    ref = tables.partition_local_tables(T.adj, lat.N)
    for k, r in enumerate(ref):
        assert np.array_equal(part.parts[k].tables()["adj"], r["adj"])
    assert sum(part.ghost_pdfs) == int((T.adj >= 0).sum())
