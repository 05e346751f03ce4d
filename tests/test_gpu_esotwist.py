"""GPU parity of the Esoteric Twist step (the single-grid form Sect. 1 and Sect. 4 name),
with its plain tables and with their run-length coding (ET-R).

The ET kernel runs through the C ABI on seeded synthetic lattices under every
boundary kind and storage precision and is compared with the FP64 oracle's
canonical state (OS-NT and ET oracles agree, see test_oracle_esotwist.py):
FP64 and double-float at the 1e-12 relative bar, FP32 / FP16 within the
storage-format bounds of the other forms.  ET and AA runs of the GPU hold the
same canonical state bit for bit (same collision code, same bounced values),
except FP16 storage at pressure faces, where the two forms round the bounced
value at different points.
"""
import numpy as np
import pytest
import torch

import geometry
from oracle import esotwist as oet
from oracle import lbm as olbm
from oracle import tables as otables

pytestmark = pytest.mark.gpu

import paper_1410_0412_gb300 as lbm

ALL = lbm.LBM_TABLES_ADJ | lbm.LBM_TABLES_RIA | lbm.LBM_TABLES_ET

CASES = [
    # (geometry, periodic, x_pressure, enum, B, drag)
    ("random", (1, 0, 0), False, "lex", 1, False),
    ("random", (1, 1, 1), False, "lex", 2, True),
    ("random", (0, 0, 1), True, "hilbert", 1, False),
    ("random", (0, 0, 0), False, "lex", 3, True),
    ("spheres", (1, 0, 0), False, "lex", 1, False),
]


def _geometry(kind, seed):
    if kind == "random":
        return geometry.random_voxels(23, 19, 17, 0.25, seed)
    return geometry.sphere_box_64x32x32(0)


def _state(N, seed):
    g = torch.Generator().manual_seed(seed)
    F = olbm.uniform_state(N, olbm.Params(), 1.0, (0.01, -0.02, 0.005))
    return F * (1 + 1e-2 * (torch.rand(F.shape, generator=g, dtype=torch.float64) - 0.5))


def _params(xp, shifted):
    kw = dict(omega_plus=1.1, magic=3 / 16, g=(1e-4, 2e-5, -3e-5), rho_in=1.002 if xp else 1.0,
              rho_out=0.998 if xp else 1.0)
    return olbm.Params(**kw), lbm.Params(shifted=shifted, **kw)


def _relerr(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f64df", 1e-12), ("f32", 2e-6), ("f16s", 5e-4)])
@pytest.mark.parametrize("ria", [False, True])
def test_et_parity_with_oracle(case, prec, tol, ria):
    kind, periodic, xp, enum, B, drag = CASES[case]
    solid = _geometry(kind, 140 + case)
    lat = lbm.Lattice(solid, periodic=periodic, x_pressure=xp, enum=enum, B=B).upload(ALL)
    T = lat.tables(runs=False)
    op, lp = _params(xp, prec in ("f32", "f16s"))
    s = torch.as_tensor(geometry.uniform_field(lat.N, 9 + case), dtype=torch.float64) * 0.5 if drag else None
    F0 = _state(lat.N, case)
    sv = lbm.Solver(lat, prec, lp, form="et", ria=ria, s=None if s is None else s.to(torch.float32).cuda())
    sv.load(F0.cuda())
    G = olbm.from_canonical(F0, 0, T["adj"], op)
    sref = None if s is None else s.to(torch.float32).to(torch.float64)
    done = 0
    for n in (1, 4, 15):
        sv.step(n)
        G = olbm.run_osnt(G, T["adj"], op, n, sref)
        done += n
        ref = olbm.canonical(G, 0, T["adj"], op)
        assert _relerr(sv.canonical().cpu(), ref) <= tol, (done, prec)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("ria", [False, True])
def test_et_equals_aa_bitwise(case, prec, ria):
    kind, periodic, xp, enum, B, drag = CASES[case]
    solid = _geometry(kind, 150 + case)
    lat = lbm.Lattice(solid, periodic=periodic, x_pressure=xp, enum=enum, B=B).upload(ALL)
    _, lp = _params(xp, prec != "f64")
    s = (torch.as_tensor(geometry.uniform_field(lat.N, 2), dtype=torch.float32) * 0.5).cuda() if drag else None
    F0 = _state(lat.N, 7).cuda()
    a = lbm.Solver(lat, prec, lp, form="aa", ria=True, s=s)
    e = lbm.Solver(lat, prec, lp, form="et", ria=ria, s=s)
    a.load(F0)
    e.load(F0)
    for n in (1, 1, 3, 5):
        a.step(n)
        e.step(n)
        if prec == "f16s" and xp:
            # AA bounces a pressure-face PDF after its half rounding (at the
            # next read), ET before it (at the write): FP16-level differences
            assert _relerr(e.canonical(), a.canonical()) <= 1e-3
        else:
            assert torch.equal(a.canonical(), e.canonical())


def test_et_matches_oracle_grid():
    """The ET grid itself (every slot, phantoms included) equals the oracle's ET grid."""
    solid = geometry.random_voxels(17, 13, 11, 0.25, 160)
    periodic = (0, 1, 0)
    lat = lbm.Lattice(solid, periodic=periodic, x_pressure=True).upload(ALL)
    T = otables.Tables(solid, periodic=periodic, x_pressure=True)
    op, lp = _params(True, False)
    nb, mask, ph = oet.tables(solid, T.node_xyz, T.adj, periodic)
    S, Spad, _ = lat.et_info()
    F0 = _state(lat.N, 3)
    sv = lbm.Solver(lat, "f64", lp, form="et", ria=False)
    sv.load(F0.cuda())
    A = oet.from_canonical(F0, 0, nb, S)
    for k in range(5):
        sv.step(1)
        A = oet.step(A, k % 2, nb, T.adj, op)
    got = sv.pdf[:, :S].cpu()
    # only slots some node reads are defined; compare those
    L = np.concatenate([np.arange(lat.N)[None], nb.astype(np.int64)])
    par = 5 % 2
    from oracle.d3q19 import INV
    rows, cols = [np.zeros(lat.N, np.int64)], [np.arange(lat.N)]
    for i in range(1, 19):
        rows.append(np.full(lat.N, i if par == 0 else INV[i]))
        cols.append(L[oet.loc_row(int(INV[i])) + 1])
    r, c = np.concatenate(rows), np.concatenate(cols)
    assert _relerr(got[r, c], A[r, c]) <= 1e-12


def test_et_macroscopic_and_init():
    solid = geometry.sphere_box_64x32x32(0)
    lat = lbm.Lattice(solid, periodic=(1, 0, 0)).upload(ALL)
    lp = lbm.Params(omega_plus=1.0, magic=3 / 16, g=(1e-5, 0, 0))
    e = lbm.Solver(lat, "f64", lp, form="et", ria=True)
    a = lbm.Solver(lat, "f64", lp, form="aa", ria=True)
    for sv in (e, a):
        sv.init_equilibrium(1.0, (0.01, 0.0, 0.0))
    assert torch.equal(e.canonical(), a.canonical())
    for n in (1, 2):
        e.step(n)
        a.step(n)
        re_, ue, se = e.macroscopic()
        ra, ua, sa = a.macroscopic()
        assert torch.equal(re_, ra) and torch.equal(ue, ua) and torch.equal(se, sa)


def test_et_graph_replay():
    solid = geometry.sphere_box_64x32x32(0)
    lat = lbm.Lattice(solid, periodic=(1, 0, 0)).upload(ALL)
    lp = lbm.Params(omega_plus=1.0, magic=3 / 16, g=(1e-5, 0, 0), shifted=True)
    a = lbm.Solver(lat, "f32", lp, form="et", ria=True)
    b = lbm.Solver(lat, "f32", lp, form="et", ria=True)
    a.init_equilibrium(1.0)
    b.init_equilibrium(1.0)
    a.step(40)
    b.step_graph(2)
    b.step_graph(38)
    torch.cuda.synchronize()
    assert torch.equal(a.pdf, b.pdf)


def test_et_empty_and_errors():
    empty = lbm.Lattice(np.ones((3, 3, 3), np.uint8)).upload(ALL)
    for ria in (False, True):
        sv = lbm.Solver(empty, "f64", lbm.Params(), form="et", ria=ria)
        sv.init_equilibrium(1.0)
        sv.step(3)
    lat = lbm.Lattice(geometry.random_voxels(9, 8, 7, 0.25, 5), periodic=(1, 0, 0)).upload()
    with pytest.raises(ValueError):
        lbm.Solver(lat, "f64", lbm.Params(), form="et")
    grid = lat.new_grid("f64", et=True)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_step_et(lat, "f64", lbm.Params(), grid, 0)


@pytest.mark.parametrize("prec", ["f64", "f64df"])
@pytest.mark.parametrize("ria", [False, True])
def test_et_plane_poiseuille(prec, ria):
    """1 x 8 x 1, periodic x and z (links joining a node to itself): the ET kernels reach the
    exact TRT Poiseuille profile (magic 3/16) and match the oracle's OS-NT state."""
    H = 8
    solid = geometry.empty_box(1, H, 1)
    lat = lbm.Lattice(solid, periodic=(1, 0, 1)).upload(ALL)
    T = otables.Tables(solid, periodic=(1, 0, 1))
    op = olbm.Params(omega_plus=1.0, magic=3 / 16, g=(1e-4, 0, 0))
    lp = lbm.Params(omega_plus=1.0, magic=3 / 16, g=(1e-4, 0, 0))
    sv = lbm.Solver(lat, prec, lp, form="et", ria=ria)
    sv.init_equilibrium(1.0)
    sv.step(20)
    G = olbm.run_osnt(olbm.from_canonical(olbm.uniform_state(T.N, op), 0, T.adj, op), T.adj, op, 20)
    assert _relerr(sv.canonical().cpu(), olbm.canonical(G, 0, T.adj, op)) <= 1e-12
    sv.step(5000)
    _, u, _ = sv.macroscopic(sums=False)
    y = torch.as_tensor(T.node_xyz[:, 1], dtype=torch.float64) + 0.5
    exact = op.g[0] / (2 * op.nu) * y * (H - y)
    assert float((u[0].cpu() - exact).abs().max() / exact.max()) <= 1e-10
