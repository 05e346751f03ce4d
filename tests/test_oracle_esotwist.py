"""Pins of the oracle's Esoteric Twist form (Sect. 1, Sect. 4 name it; rules are a reading).

* the tables agree with a voxel-by-voxel brute force (locations, phantoms, mask);
* every step is a permutation of slots: each (array, location) slot read in a
  step is written exactly once in it, and no other -- the in-place property
  that makes one grid enough;
* a node only touches its own location and the six +x, +y, +z, +xy, +xz, +yz ones;
* ET holds the same canonical state as OS-NT after every step, under every
  boundary kind (the OS-NT oracle is itself pinned to the dense LBM);
* layout round trips are exact.
"""
import numpy as np
import pytest
import torch

import geometry
from oracle import esotwist as et
from oracle import lbm, tables
from oracle.d3q19 import C, INV, Q

CASES = [
    dict(periodic=(1, 0, 0), x_pressure=False),
    dict(periodic=(1, 1, 1), x_pressure=False),
    dict(periodic=(0, 0, 1), x_pressure=True),
    dict(periodic=(0, 0, 0), x_pressure=False),
]


def _brute(solid, xyz, adj, periodic):
    Z, Y, X = solid.shape
    N = len(xyz)
    where = {tuple(v): n for n, v in enumerate(map(tuple, xyz))}
    offs = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
    cells = {}
    nb = np.zeros((6, N), dtype=np.int64)
    for n in range(N):
        for k, o in enumerate(offs):
            p = [xyz[n][a] + o[a] for a in range(3)]
            for a, d in enumerate((X, Y, Z)):
                if periodic[a]:
                    p[a] %= d
            p = tuple(p)
            if p in where:
                nb[k, n] = where[p]
            else:
                cells.setdefault(p, []).append((k, n))
    ph = sorted(cells, key=lambda p: (p[2], p[1], p[0]))
    for r, p in enumerate(ph):
        for k, n in cells[p]:
            nb[k, n] = N + r
    mask = np.zeros(N, dtype=np.int64)
    xr = 0
    for i in range(1, Q):
        for n in range(N):
            if adj[i - 1, n] < 0:
                mask[n] |= 1 << (i - 1)
        if C[i][0] != 0:
            for n in range(N):
                if adj[i - 1, n] <= -2:
                    mask[n] |= 1 << (18 + xr)
            xr += 1
    return nb, mask, np.array(ph, dtype=np.int64).reshape(-1, 3)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_tables_brute_force(case):
    solid = geometry.random_voxels(7, 6, 5, 0.3, 80 + case)
    T = tables.Tables(solid, enum="hilbert", **CASES[case])
    nb, mask, ph = et.tables(solid, T.node_xyz, T.adj, CASES[case]["periodic"])
    bnb, bmask, bph = _brute(solid, T.node_xyz, T.adj, CASES[case]["periodic"])
    assert np.array_equal(nb, bnb)
    assert np.array_equal(mask.astype(np.int64), bmask)
    assert np.array_equal(ph, bph)


def test_location_rows():
    for i in range(1, Q):
        k = et.loc_row(i)
        cp = np.maximum(C[i], 0)
        assert (k == -1) == (not cp.any())
        if k >= 0:
            assert np.array_equal(et.OFFSETS[k], cp)
    # six directions keep their slots at the node: the all-non-positive ones
    assert sorted(i for i in range(1, Q) if et.loc_row(i) == -1) == [2, 4, 6, 8, 12, 16]


def _slots(parity, nb, adj):
    """(read, written) slot lists of one step, as (array, location) pairs."""
    N = nb.shape[1]
    L = np.concatenate([np.arange(N)[None], nb.astype(np.int64)])
    read, wrote = [], []
    for n in range(N):
        read.append((0, n))
        wrote.append((0, n))
        for i in range(1, Q):
            read.append((i if parity == 0 else int(INV[i]), int(L[et.loc_row(int(INV[i])) + 1, n])))
        for j in range(1, Q):
            jj = int(INV[j])
            fluid = adj[jj - 1, n] >= 0
            a = (jj if parity == 0 else j) if fluid else (j if parity == 0 else jj)
            wrote.append((a, int(L[et.loc_row(j) + 1, n])))
    return read, wrote


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("parity", [0, 1])
def test_step_is_a_slot_permutation(case, parity):
    solid = geometry.random_voxels(7, 6, 5, 0.3, 90 + case)
    T = tables.Tables(solid, **CASES[case])
    nb, mask, ph = et.tables(solid, T.node_xyz, T.adj, CASES[case]["periodic"])
    read, wrote = _slots(parity, nb, T.adj)
    assert len(set(read)) == len(read)            # no slot read twice
    assert len(set(wrote)) == len(wrote)          # no slot written twice (race-free)
    # the slots a step writes are the ones the next step reads
    nxt, _ = _slots(1 - parity, nb, T.adj)
    assert set(wrote) == set(nxt)


def test_only_seven_locations():
    solid = geometry.random_voxels(7, 6, 5, 0.3, 95)
    T = tables.Tables(solid, periodic=(1, 1, 1))
    nb, _, ph = et.tables(solid, T.node_xyz, T.adj, (1, 1, 1))
    Z, Y, X = solid.shape
    S = T.N + len(ph)
    coord = np.concatenate([T.node_xyz, ph]).astype(np.int64)
    for n in range(T.N):
        for k in range(6):
            d = (coord[nb[k, n]] - T.node_xyz[n]) % np.array([X, Y, Z])
            assert np.array_equal(d, et.OFFSETS[k])
    assert nb.max() < S


@pytest.mark.parametrize("case", range(len(CASES)))
def test_esotwist_equals_osnt(case):
    bc = CASES[case]
    solid = geometry.random_voxels(8, 7, 6, 0.25, 100 + case)
    T = tables.Tables(solid, enum="lex", B=2, **bc)
    nb, mask, ph = et.tables(solid, T.node_xyz, T.adj, bc["periodic"])
    S = T.N + len(ph)
    p = lbm.Params(omega_plus=1.1, magic=3 / 16, g=(1e-4, 2e-5, -3e-5), rho_in=1.002, rho_out=0.998)
    s = torch.as_tensor(geometry.uniform_field(T.N, 11 + case), dtype=torch.float64) * 0.5
    g = torch.Generator().manual_seed(case)
    F0 = lbm.uniform_state(T.N, p, 1.0, (0.01, -0.02, 0.005))
    F0 = F0 * (1 + 1e-2 * (torch.rand(F0.shape, generator=g, dtype=torch.float64) - 0.5))
    G = lbm.from_canonical(F0, 0, T.adj, p)
    A = et.from_canonical(F0, 0, nb, S)
    for k in range(1, 7):
        G = lbm.osnt_step(G, T.adj, p, s)
        A = et.step(A, (k - 1) % 2, nb, T.adj, p, s)
        FG = lbm.canonical(G, 0, T.adj, p)
        FE = et.canonical(A, k % 2, nb)
        assert torch.max(torch.abs(FG - FE)) <= 1e-15, k


@pytest.mark.parametrize("parity", [0, 1])
def test_layout_roundtrip(parity):
    solid = geometry.random_voxels(6, 6, 6, 0.3, 110)
    T = tables.Tables(solid, periodic=(0, 1, 0), x_pressure=True)
    nb, _, ph = et.tables(solid, T.node_xyz, T.adj, (0, 1, 0))
    F = torch.rand((Q, T.N), generator=torch.Generator().manual_seed(3), dtype=torch.float64)
    A = et.from_canonical(F, parity, nb, T.N + len(ph))
    assert torch.equal(et.canonical(A, parity, nb), F)


def test_planted_mistake_is_caught(monkeypatch):
    """Swapping the slot locations of directions 9 (kept at +x) and 10 (kept at +y) is
    caught by the comparison with OS-NT."""
    solid = geometry.random_voxels(8, 7, 6, 0.25, 101)
    T = tables.Tables(solid, periodic=(1, 1, 1))
    nb, _, ph = et.tables(solid, T.node_xyz, T.adj, (1, 1, 1))
    p = lbm.Params(omega_plus=1.1, g=(1e-4, 0, 0))
    F0 = lbm.uniform_state(T.N, p, 1.0, (0.02, 0.01, 0.0))
    good = et.loc_row
    monkeypatch.setattr(et, "loc_row", lambda i: good(10) if i == 9 else (good(9) if i == 10 else good(i)))
    A = et.run(et.from_canonical(F0, 0, nb, T.N + len(ph)), nb, T.adj, p, 2)
    G = lbm.run_osnt(lbm.from_canonical(F0, 0, T.adj, p), T.adj, p, 2)
    assert torch.max(torch.abs(et.canonical(A, 0, nb) - lbm.canonical(G, 0, T.adj, p))) > 1e-6


@pytest.mark.parametrize("case", range(len(CASES)))
def test_et_runs_decode_and_are_maximal(case):
    solid = geometry.random_voxels(11, 9, 8, 0.25, 170 + case)
    T = tables.Tables(solid, **CASES[case])
    nb, mask, _ = et.tables(solid, T.node_xyz, T.adj, CASES[case]["periodic"])
    rs, rnb, rmask = et.run_tables(nb, mask)
    dnb, dmask = et.decode_runs(rs, rnb, rmask)
    assert np.array_equal(dnb, nb) and np.array_equal(dmask, mask)
    # maximal: no run head continues its predecessor (brute force per head)
    for h in rs[1:-1]:
        same = all(nb[k, h] == nb[k, h - 1] + 1 for k in range(6)) and mask[h] == mask[h - 1]
        assert not same
    assert rs[0] == 0 and rs[-1] == T.N and np.all(np.diff(rs) > 0)


def test_et_runs_on_the_paper_channel_rows():
    """A duct with walls on y and z, periodic x: every interior stretch of a row is one run,
    as in the paper's channel example for RIA (Sect. 4.1)."""
    solid = geometry.square_channel(40, 7, 6)          # X = 40: rows of 38 fluid nodes along x
    T = tables.Tables(solid, periodic=(0, 0, 1))
    nb, mask, _ = et.tables(solid, T.node_xyz, T.adj, (0, 0, 1))
    rs, _, _ = et.run_tables(nb, mask)
    # each row: the first node, the 36 interior ones, the last node
    assert len(rs) - 1 == 3 * 5 * 6


def test_esotwist_one_voxel_periodic_axes():
    """Plane Poiseuille geometry (1 x 8 x 1, periodic x and z): links in x and z join a node to
    itself, and the ET form still equals OS-NT and reaches the exact parabolic profile."""
    H = 8
    solid = geometry.empty_box(1, H, 1)
    T = tables.Tables(solid, periodic=(1, 0, 1))
    nb, mask, ph = et.tables(solid, T.node_xyz, T.adj, (1, 0, 1))
    p = lbm.Params(omega_plus=1.0, magic=3 / 16, g=(1e-4, 0, 0))
    F0 = lbm.uniform_state(T.N, p)
    A = et.from_canonical(F0, 0, nb, T.N + len(ph))
    G = lbm.from_canonical(F0, 0, T.adj, p)
    for k in range(6):
        A = et.step(A, k % 2, nb, T.adj, p)
        G = lbm.osnt_step(G, T.adj, p)
        assert torch.max(torch.abs(et.canonical(A, (k + 1) % 2, nb) - lbm.canonical(G, 0, T.adj, p))) <= 1e-16
    A = et.run(A, nb, T.adj, p, 3000, start_parity=0)
    rho, u, _ = lbm.macroscopic(et.canonical(A, 0, nb), p)
    y = torch.as_tensor(T.node_xyz[:, 1], dtype=torch.float64) + 0.5
    exact = p.g[0] / (2 * p.nu) * y * (H - y)
    assert torch.max(torch.abs(u[0] - exact)) / exact.max() <= 1e-10
