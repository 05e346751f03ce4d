"""GPU parity of the partitioned step: P chunks with a ghost exchange (Sect. 6).

The chunks run the same step kernels as the whole lattice, and every ghost PDF
is copied bit for bit, so after any number of steps the chunks' node slots
must equal the whole-lattice run's grid exactly, for every step form,
addressing, storage precision and boundary kind.  One case per form is also
compared with the FP64 oracle at the 1e-12 bar.  The exchange kernel alone is
checked slot by slot against the ghost map.
"""
import numpy as np
import pytest
import torch

import geometry
from oracle import lbm as olbm
from oracle import tables as otables

pytestmark = pytest.mark.gpu

import paper_1410_0412_gb300 as lbm

CASES = [
    # (periodic, x_pressure, enum, drag)
    ((1, 0, 0), False, "lex", False),
    ((1, 1, 1), False, "hilbert", True),
    ((0, 0, 1), True, "renumbered", False),
]


def _lattice(case, seed=70):
    periodic, xp, enum, _ = CASES[case]
    solid = geometry.random_voxels(29, 23, 19, 0.25, seed + case)
    if enum == "renumbered":
        h = lbm.Lattice(solid, periodic=periodic, x_pressure=xp, enum="hilbert")
        order = h.renumber_partitions(5)
        return solid, lbm.Lattice.from_order(solid, order, periodic=periodic, x_pressure=xp)
    return solid, lbm.Lattice(solid, periodic=periodic, x_pressure=xp, enum=enum)


def _state(N, seed):
    g = torch.Generator().manual_seed(seed)
    F = olbm.uniform_state(N, olbm.Params(), 1.0, (0.01, -0.02, 0.005))
    return F * (1 + 1e-2 * (torch.rand(F.shape, generator=g, dtype=torch.float64) - 0.5))


def _params(prec, xp):
    return lbm.Params(omega_plus=1.1, magic=3 / 16, g=(1e-4, 2e-5, -3e-5),
                      rho_in=1.001 if xp else 1.0, rho_out=0.999 if xp else 1.0, shifted=prec in ("f32", "f16s"))


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("form", ["osnt", "aa"])
@pytest.mark.parametrize("ria", [False, True])
@pytest.mark.parametrize("prec", ["f64", "f64df", "f32", "f16s"])
@pytest.mark.parametrize("P", [2, 7])
def test_partitioned_equals_whole(case, form, ria, prec, P):
    periodic, xp, enum, drag = CASES[case]
    solid, lat = _lattice(case)
    lat.upload()
    part = lbm.Partitioning(lat, P).upload()
    lp = _params(prec, xp)
    s = torch.as_tensor(geometry.uniform_field(lat.N, 3 + case), dtype=torch.float32).cuda() * 0.5 if drag else None
    whole = lbm.Solver(lat, prec, lp, form=form, ria=ria, s=s)
    whole.load(_state(lat.N, case).cuda())
    chunks = lbm.PartitionedSolver(part, prec, lp, form=form, ria=ria, s=s)
    chunks.load_global(whole.pdf)
    for n in (1, 2, 3):                     # 6 steps, odd and even counts between checks
        whole.step(n)
        chunks.step(n)
        torch.cuda.synchronize()
        got = chunks.to_global()
        assert torch.equal(got.view(torch.int16 if prec == "f16s" else got.dtype),
                           whole.pdf[:, :lat.N].view(torch.int16 if prec == "f16s" else got.dtype)), (n, prec)


@pytest.mark.parametrize("form", ["osnt", "aa"])
def test_partitioned_matches_oracle(form):
    periodic, xp, enum, drag = CASES[2]
    solid, lat = _lattice(2)
    lat.upload()
    part = lbm.Partitioning(lat, 7).upload()
    lp = _params("f64", xp)
    op = olbm.Params(omega_plus=1.1, magic=3 / 16, g=(1e-4, 2e-5, -3e-5), rho_in=1.001, rho_out=0.999)
    T = lat.tables(runs=False)
    F0 = _state(lat.N, 9)
    steps = 8
    if form == "osnt":
        ref = olbm.canonical(olbm.run_osnt(olbm.from_canonical(F0, 0, T["adj"], op), T["adj"], op, steps), 0,
                             T["adj"], op)
    else:
        ref = olbm.canonical(olbm.run_aa(olbm.from_canonical(F0, 1, T["adj"], op), T["adj"], op, steps, 0), 1,
                             T["adj"], op)
    whole = lbm.Solver(lat, "f64", lp, form=form, ria=True)
    whole.load(F0.cuda())
    chunks = lbm.PartitionedSolver(part, "f64", lp, form=form, ria=True)
    chunks.load_global(whole.pdf)
    chunks.step(steps)
    grid = lat.new_grid("f64")
    chunks.to_global(out=grid[:, :lat.N])
    layout = lbm.LBM_LAYOUT_OSNT if form == "osnt" else lbm.LBM_LAYOUT_AA_EVEN
    F = lbm.lbm_canonical_pdfs(lat, "f64", lp, grid, layout).cpu()
    assert float((F - ref).abs().max() / ref.abs().max()) <= 1e-12


@pytest.mark.parametrize("prec", ["f64", "f32", "f16s"])
def test_exchange_moves_exactly_the_ghosts(prec):
    solid, lat = _lattice(1)
    part = lbm.Partitioning(lat, 5).upload()
    dt = {"f64": torch.float64, "f32": torch.float32, "f16s": torch.float16}[prec]
    it = {"f64": torch.int64, "f32": torch.int32, "f16s": torch.int16}[prec]
    # random finite bit patterns, so a misrouted copy shows up; compared as integers
    gen = torch.Generator().manual_seed(11)
    grids = []
    for loc in part.parts:
        bits = torch.randint(0, 0x7b00, (19, loc.Npad), generator=gen, dtype=torch.int64)
        if prec == "f16s":
            grids.append(bits.to(torch.int16).view(torch.float16).cuda())
        else:
            grids.append(torch.rand((19, loc.Npad), generator=gen, dtype=torch.float64).to(dt).cuda())
    before = [g.clone() for g in grids]
    same = lambda x, y: torch.equal(x.view(it), y.view(it))
    ptrs = lbm.Partitioning.pointers(grids)
    inv = lambda i: i + 1 if i % 2 else i - 1
    for mode in (lbm.LBM_HALO_OSNT, lbm.LBM_HALO_AA_GATHER):
        for g, b in zip(grids, before):
            g.copy_(b)
        lbm.lbm_halo_exchange(part, prec, ptrs, mode)
        torch.cuda.synchronize()
        for p in range(part.P):
            want = before[p].clone()
            gh = part.ghosts(p)
            for q, d, sl, m in zip(gh["src_part"], gh["dir"], gh["slot"], gh["src_node"]):
                a = d if mode == lbm.LBM_HALO_OSNT else inv(int(d))
                want[a, sl] = before[q][a, m]
            assert same(grids[p], want), (mode, p)
    # scatter returns ghost slots to their owners' node slots
    for g, b in zip(grids, before):
        g.copy_(b)
    lbm.lbm_halo_exchange(part, prec, ptrs, lbm.LBM_HALO_AA_SCATTER)
    torch.cuda.synchronize()
    want = [b.clone() for b in before]
    for p in range(part.P):
        gh = part.ghosts(p)
        for q, d, sl, m in zip(gh["src_part"], gh["dir"], gh["slot"], gh["src_node"]):
            a = inv(int(d))
            want[q][a, m] = before[p][a, sl]
    for g, w in zip(grids, want):
        assert same(g, w)


def test_packed_bed_crop_partitioned_hilbert_renumbered():
    """A 128^3 RSA bed (about 1.3 M nodes): Hilbert order renumbered in 16 chunks, AA-R FP32 and
    OS-NT-R FP64, 4 steps, chunk node slots identical to the whole-lattice run."""
    solid, _ = geometry.rsa_spheres(128, 128, 128, 12, 1, periodic=(1, 0, 0), max_consecutive_rejections=20000)
    h = lbm.Lattice(solid, periodic=(1, 0, 0), enum="hilbert")
    lat = lbm.Lattice.from_order(solid, h.renumber_partitions(16), periodic=(1, 0, 0)).upload()
    part = lbm.Partitioning(lat, 16).upload()
    part.validate(lat)
    for prec, form in (("f32", "aa"), ("f64", "osnt")):
        lp = lbm.Params(omega_plus=1.0, magic=3 / 16, g=(1e-5, 0, 0), shifted=prec == "f32")
        whole = lbm.Solver(lat, prec, lp, form=form, ria=True)
        whole.init_equilibrium(1.0, (0.01, 0.0, 0.0))
        chunks = lbm.PartitionedSolver(part, prec, lp, form=form, ria=True)
        chunks.load_global(whole.pdf)
        whole.step(4)
        chunks.step(4)
        torch.cuda.synchronize()
        assert torch.equal(chunks.to_global(), whole.pdf[:, :lat.N])


@pytest.mark.parametrize("form", ["osnt", "aa"])
def test_one_node_per_chunk(form):
    """P = N: every fluid pull crosses a chunk border; the result still equals the whole lattice."""
    solid = geometry.random_voxels(7, 6, 5, 0.25, 90)
    lat = lbm.Lattice(solid, periodic=(1, 0, 1)).upload()
    part = lbm.Partitioning(lat, lat.N).upload()
    lp = _params("f64", False)
    whole = lbm.Solver(lat, "f64", lp, form=form, ria=True)
    whole.load(_state(lat.N, 4).cuda())
    chunks = lbm.PartitionedSolver(part, "f64", lp, form=form, ria=True)
    chunks.load_global(whole.pdf)
    whole.step(6)
    chunks.step(6)
    torch.cuda.synchronize()
    assert torch.equal(chunks.to_global(), whole.pdf[:, :lat.N])
