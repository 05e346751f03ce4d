"""GPU parity of the stream-collide kernels against the FP64 oracle.

Every variant of the step (OS-NT and AA pattern, adjacency list or RIA runs,
body force, Brinkman drag, bounce-back walls and pressure faces) runs through
the C ABI on seeded synthetic inputs and is compared element by element with
the oracle's canonical state.  FP64 must agree to a relative max-norm of
1e-12 (max |F_gpu - F_oracle| / max |F_oracle|).  FP32 / FP16 storage is
compared with stated error bounds (their error is a property of the storage
format, not a parity bar).
"""
import numpy as np
import pytest
import torch

import geometry
from oracle import lbm as olbm
from oracle import tables as otables

pytestmark = pytest.mark.gpu

TOL64 = 1e-12

import paper_1410_0412_gb300 as lbm


def _params(g=(1e-4, 2e-5, -3e-5), omega=1.1, magic=3 / 16, rho_in=1.0, rho_out=1.0, shifted=False):
    return (olbm.Params(omega_plus=omega, magic=magic, g=g, rho_in=rho_in, rho_out=rho_out),
            lbm.Params(omega_plus=omega, magic=magic, g=g, rho_in=rho_in, rho_out=rho_out, shifted=shifted))


def _state(N, seed, amp=1e-2, u0=(0.01, -0.02, 0.005)):
    g = torch.Generator().manual_seed(seed)
    p = olbm.Params()
    F = olbm.uniform_state(N, p, 1.0, u0)
    return F * (1 + amp * (torch.rand(F.shape, generator=g, dtype=torch.float64) - 0.5))


def _relerr(a, b):
    return float((a - b).abs().max() / b.abs().max())


def _run_oracle(T, F0, op, steps, s, form):
    if form == "osnt":
        G = olbm.from_canonical(F0, 0, T.adj, op)
        G = olbm.run_osnt(G, T.adj, op, steps, s)
        return olbm.canonical(G, 0, T.adj, op)
    A = olbm.from_canonical(F0, 1, T.adj, op)
    A = olbm.run_aa(A, T.adj, op, steps, 0, s)
    return olbm.canonical(A, 1 if steps % 2 == 0 else 2, T.adj, op)


def _run_gpu(lat, prec, lp, F0, steps, s, form, ria):
    sv = None if s is None else s.to(torch.float32).cuda()
    solver = lbm.Solver(lat, prec, lp, form=form, ria=ria, s=sv)
    solver.load(F0.cuda())
    solver.step(steps)
    torch.cuda.synchronize()
    return solver.canonical().cpu()


CASES = [
    # (geometry, periodic, x_pressure, enum, B, drag)
    ("random", (1, 0, 0), False, "lex", 1, False),
    ("random", (1, 1, 1), False, "lex", 2, True),
    ("random", (0, 0, 1), True, "hilbert", 1, False),
    ("random", (0, 0, 0), False, "lex", 3, True),
    ("spheres", (1, 0, 0), False, "lex", 1, False),
    ("spheres", (1, 0, 0), False, "hilbert", 1, True),
]


def _geometry(kind, seed):
    if kind == "random":
        return geometry.random_voxels(23, 19, 17, 0.25, seed)   # ragged: N not a multiple of the CTA size
    return geometry.sphere_box_64x32x32(0)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("form", ["osnt", "aa"])
@pytest.mark.parametrize("ria", [False, True])
@pytest.mark.parametrize("prec", ["f64", "f64df"])
def test_f64_parity(case, form, ria, prec):
    """FP64 storage, with native FP64 or double-float (f32 pair) collision arithmetic."""
    kind, per, xp, enum, B, drag = CASES[case]
    solid = _geometry(kind, 200 + case)
    T = otables.Tables(solid, periodic=per, x_pressure=xp, enum=enum, B=B)
    lat = lbm.Lattice(solid, periodic=per, x_pressure=xp, enum=enum, B=B).upload()
    op, lp = _params(rho_in=1.002 if xp else 1.0, rho_out=0.998 if xp else 1.0)
    s = torch.as_tensor(geometry.uniform_field(T.N, 9 + case), dtype=torch.float64) * 0.4 if drag else None
    if s is not None:
        s = s.to(torch.float32).to(torch.float64)   # the library reads s as float32
    F0 = _state(T.N, case)
    steps = 6
    ref = _run_oracle(T, F0, op, steps, s, form)
    got = _run_gpu(lat, prec, lp, F0, steps, s, form, ria)
    assert _relerr(got, ref) <= TOL64


@pytest.mark.parametrize("layout", [0, 1, 2])
@pytest.mark.parametrize("ria", [False, True])
def test_layout_roundtrip_and_init(layout, ria):
    solid = geometry.random_voxels(11, 9, 7, 0.3, 5)
    T = otables.Tables(solid, periodic=(0, 1, 0), x_pressure=True)
    lat = lbm.Lattice(solid, periodic=(0, 1, 0), x_pressure=True)
    lat.upload(lbm.LBM_TABLES_RIA if ria else lbm.LBM_TABLES_ADJ)
    op, lp = _params(rho_in=1.01, rho_out=0.99)
    F = _state(T.N, 3)
    pdf = lat.new_grid("f64")
    lbm.lbm_load_canonical(lat, "f64", lp, F.cuda(), pdf, layout)
    ref_grid = olbm.from_canonical(F, layout, T.adj, op)
    # pure data movement, except anti-bounce-back slots 2 w rho_bc - F, which the
    # device may evaluate as one fused multiply-add (one rounding less)
    assert float((pdf[:, :T.N].cpu() - ref_grid).abs().max()) <= 2e-16
    back = lbm.lbm_canonical_pdfs(lat, "f64", lp, pdf, layout).cpu()
    assert float((back - F).abs().max()) <= 1e-16    # a - (a - b) may differ from b by one ulp
    lbm.lbm_init_equilibrium(lat, "f64", lp, pdf, layout, 1.0, (0.02, 0.0, -0.01))
    Feq = olbm.uniform_state(T.N, op, 1.0, (0.02, 0.0, -0.01))
    assert _relerr(pdf[:, :T.N].cpu(), olbm.from_canonical(Feq, layout, T.adj, op)) <= 1e-15


def test_macroscopic_and_sums():
    solid = geometry.sphere_box_64x32x32(0)
    T = otables.Tables(solid, periodic=(1, 0, 0))
    lat = lbm.Lattice(solid, periodic=(1, 0, 0)).upload()
    op, lp = _params(g=(1e-5, 0, 0))
    F = _state(T.N, 8)
    s = torch.as_tensor(geometry.uniform_field(T.N, 3), dtype=torch.float32)
    pdf = lat.new_grid("f64")
    lbm.lbm_load_canonical(lat, "f64", lp, F.cuda(), pdf, 1)
    rho, u, sums = lbm.lbm_macroscopic(lat, "f64", lp, pdf, 1, s=s.cuda())
    r_ref, u_ref, s_ref = olbm.macroscopic(F, op, s.to(torch.float64))
    assert _relerr(rho.cpu(), r_ref) <= 1e-14
    assert float((u.cpu() - u_ref).abs().max()) <= 1e-15
    assert float((sums.cpu() - s_ref).abs().max() / s_ref.abs().max()) <= 1e-13
    # determinism: the same call twice gives bit-identical sums
    _, _, sums2 = lbm.lbm_macroscopic(lat, "f64", lp, pdf, 1, s=s.cuda())
    assert torch.equal(sums, sums2)


def test_osnt_equals_aa_on_gpu_bitwise_free():
    """Both forms compute the same canonical state after an even number of steps."""
    solid = geometry.sphere_box_64x32x32(0)
    lat = lbm.Lattice(solid, periodic=(1, 0, 0)).upload()
    _, lp = _params()
    F0 = _state(lat.N, 4).cuda()
    a = lbm.Solver(lat, "f64", lp, form="osnt", ria=True)
    b = lbm.Solver(lat, "f64", lp, form="aa", ria=True)
    a.load(F0)
    b.load(F0)
    a.step(10)
    b.step(10)
    assert _relerr(a.canonical(), b.canonical()) <= 1e-14


def test_config1_200_steps_parity():
    """64x32x32 overlapping-sphere box, g = 1e-6, from rest, 200 OS-NT steps (plain adjacency)."""
    solid = geometry.sphere_box_64x32x32(0)
    T = otables.Tables(solid, periodic=(1, 0, 0))
    lat = lbm.Lattice(solid, periodic=(1, 0, 0)).upload()
    op, lp = _params(g=(1e-6, 0, 0), omega=1.0)
    G = olbm.from_canonical(olbm.uniform_state(T.N, op), 0, T.adj, op)
    G = olbm.run_osnt(G, T.adj, op, 200)
    ref = olbm.canonical(G, 0, T.adj, op)
    for prec in ("f64", "f64df"):
        for form, ria in [("osnt", False), ("osnt", True), ("aa", True)]:
            solver = lbm.Solver(lat, prec, lp, form=form, ria=ria)
            solver.init_equilibrium(1.0)
            solver.step(200)
            assert _relerr(solver.canonical().cpu(), ref) <= TOL64


@pytest.mark.parametrize("case", range(4))
@pytest.mark.parametrize("prec", ["f64", "f64df"])
@pytest.mark.parametrize("form,ria", [("osnt", True), ("aa", False), ("aa", True), ("et", False)])
@pytest.mark.parametrize("g", [(1e-4, 2e-5, -3e-5), (1e-4, 0.0, 0.0)])
def test_unit_omega_fast_path(case, prec, form, ria, g):
    """omega+ = 1 selects the l+ = 1 collision of the FP64-storage kernels (the even-part
    products with (1 - l+)/2 = 0 are skipped): parity 1e-12 with every boundary kind, with
    and without drag, and a perturbed (non-equilibrium) state.  A force along x alone takes
    the FP64 collision's shorter branch."""
    kind, periodic, xp, enum, B, drag = CASES[case]
    solid = _geometry(kind, 300 + case)
    T = otables.Tables(solid, periodic=periodic, x_pressure=xp, enum=enum, B=B)
    lat = lbm.Lattice(solid, periodic=periodic, x_pressure=xp, enum=enum, B=B).upload(
        lbm.LBM_TABLES_ADJ | lbm.LBM_TABLES_RIA | lbm.LBM_TABLES_ET)
    op, lp = _params(g=g, omega=1.0, rho_in=1.002 if xp else 1.0, rho_out=0.998 if xp else 1.0)
    s = torch.as_tensor(geometry.uniform_field(T.N, 40 + case), dtype=torch.float64) * 0.5 if drag else None
    F0 = _state(T.N, 50 + case)
    ref = _run_oracle(T, F0, op, 12, None if s is None else s.to(torch.float32).to(torch.float64), "osnt")
    got = _run_gpu(lat, prec, lp, F0, 12, s, form, ria)
    assert _relerr(got, ref) <= TOL64


@pytest.mark.parametrize("prec", ["f64", "f64df"])
def test_fast_flow_200_steps_parity(prec):
    """A fast, strongly perturbed flow (|u| ~ 0.05) for 200 steps: the double-float
    collision's 48-bit arithmetic must stay within the FP64 bar too."""
    solid = geometry.random_voxels(31, 17, 13, 0.2, 77)
    T = otables.Tables(solid, periodic=(1, 1, 1))
    lat = lbm.Lattice(solid, periodic=(1, 1, 1)).upload()
    op, lp = _params(g=(2e-5, -1e-5, 1e-5), omega=1.6)
    F0 = _state(T.N, 21, amp=2e-2, u0=(0.05, -0.03, 0.02))
    ref = _run_oracle(T, F0, op, 200, None, "aa")
    got = _run_gpu(lat, prec, lp, F0, 200, None, "aa", True)
    assert _relerr(got, ref) <= TOL64


@pytest.mark.parametrize("prec,tol", [("f32", 2e-6), ("f16s", 5e-4)])
@pytest.mark.parametrize("form", ["osnt", "aa"])
def test_reduced_precision_error(prec, tol, form):
    """FP32 / shifted FP16 storage against the FP64 oracle (stated error bound).

    Per step the storage rounds each deviation f - w rho0 (|d| <~ 0.01 here)
    to 2^-24 (FP32) or 2^-11 (FP16 with scale 2^10) relative; over 20 steps
    the max-norm error relative to max |F| stays below the bounds used here.
    """
    solid = geometry.sphere_box_64x32x32(0)
    T = otables.Tables(solid, periodic=(1, 0, 0))
    lat = lbm.Lattice(solid, periodic=(1, 0, 0)).upload()
    op, lp = _params(g=(1e-5, 0, 0), shifted=True)
    F0 = _state(T.N, 11, amp=1e-3, u0=(0.01, 0, 0))
    steps = 20
    ref = _run_oracle(T, F0, op, steps, None, form)
    got = _run_gpu(lat, prec, lp, F0, steps, None, form, True)
    assert _relerr(got, ref) <= tol


def test_empty_lattice_is_a_no_op():
    solid = np.ones((4, 4, 4), np.uint8)
    lat = lbm.Lattice(solid).upload()
    _, lp = _params()
    solver = lbm.Solver(lat, "f64", lp, form="aa")
    solver.init_equilibrium()
    solver.step(3)
    rho, u, sums = solver.macroscopic()
    torch.cuda.synchronize()
    assert rho.numel() == 0 and float(sums.abs().sum()) == 0.0


def test_missing_tables_and_bad_arguments():
    solid = geometry.random_voxels(8, 8, 8, 0.2, 1)
    lat = lbm.Lattice(solid)
    lat.upload(lbm.LBM_TABLES_ADJ)
    _, lp = _params()
    a, b = lat.new_grid("f64"), lat.new_grid("f64")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step_osnt(lat, "f64", lp, a, b, ria=True)
    assert e.value.code == 1
    with pytest.raises(lbm.LbmError):
        lbm.lbm_step_osnt(lat, "f64", lp, a, a)
    bad = lbm.Params(omega_plus=2.5)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_step_aa(lat, "f64", bad, a, 0)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_step_aa(lat, "f16s", lbm.Params(shifted=False), lat.new_grid("f16s"), 0)


@pytest.mark.parametrize("omega", [1.1, 1.0])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_state_is_reported(omega, bad):
    """A NaN or Inf planted in one PDF surfaces as LBM_ERR_NONFINITE from the FP64 sums guard,
    through the integer-pipe moments of the general and the l+ = 1 collision."""
    solid = geometry.random_voxels(12, 10, 8, 0.2, 3)
    lat = lbm.Lattice(solid, periodic=(1, 1, 1)).upload()
    _, lp = _params(omega=omega)
    solver = lbm.Solver(lat, "f64", lp, form="aa", ria=True)
    solver.init_equilibrium(1.0)
    solver.step(2)
    _, _, sums = solver.macroscopic(fields=False)
    lbm.lbm_check_finite(sums)
    solver.pdf[7, lat.N // 2] = bad
    solver.step(2)
    _, _, sums = solver.macroscopic(fields=False)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_check_finite(sums)
    assert e.value.code == 6


@pytest.mark.parametrize("form", ["osnt", "aa"])
def test_cuda_graph_replay_matches_direct_launches(form):
    """Steps replayed from a captured CUDA graph equal directly launched steps bit for bit."""
    solid = geometry.sphere_box_64x32x32(0)
    lat = lbm.Lattice(solid, periodic=(1, 0, 0)).upload()
    _, lp = _params(g=(1e-5, 0, 0))
    F0 = _state(lat.N, 31).cuda()
    a = lbm.Solver(lat, "f64", lp, form=form, ria=True)
    b = lbm.Solver(lat, "f64", lp, form=form, ria=True)
    a.load(F0)
    b.load(F0)
    a.step(40)
    b.step_graph(2)          # the first pair runs directly while the graph is captured ...
    b.step_graph(38)         # ... then 19 replays
    torch.cuda.synchronize()
    assert b.t == 40
    assert torch.equal(a.canonical(), b.canonical())


@pytest.mark.parametrize("form,ria", [("aa", True), ("aa", False), ("osnt", True), ("et", False)])
def test_f64_mixed_arithmetic_paths(form, ria):
    """The FP64 collision picks, per warp, between the fixed-point pair update with
    short conversions, the same update with the general conversions, and the FP64
    update.  A state that mixes nodes for all three in one launch (most near
    equilibrium; some with |u_x| = 0.3, beyond the fixed-point range; some with
    PDFs spread over more than 5 binades; some with a negative PDF) still
    matches the oracle to 1e-12 after every step."""
    solid = geometry.random_voxels(23, 19, 17, 0.25, 77)
    per = (1, 0, 0)
    T = otables.Tables(solid, periodic=per)
    lat = lbm.Lattice(solid, periodic=per).upload(lbm.LBM_TABLES_ADJ | lbm.LBM_TABLES_RIA | lbm.LBM_TABLES_ET)
    op, lp = _params(g=(1e-4, 0.0, 0.0), omega=1.0)
    F0 = _state(T.N, 31)
    fast = olbm.uniform_state(T.N, op, 1.0, (0.3, 0.0, 0.0))
    idx = torch.arange(T.N)
    F0[:, idx % 37 == 5] = fast[:, idx % 37 == 5]          # |u| beyond the fixed-point range
    F0[7, idx % 41 == 3] *= 1e-3                              # PDFs over more than 5 binades
    F0[12, idx % 53 == 8] = -1e-4                             # a negative PDF
    for steps in (1, 2, 3):
        ref = _run_oracle(T, F0, op, steps, None, "osnt" if form == "et" else form)
        got = _run_gpu(lat, "f64", lp, F0, steps, None, form, ria)
        assert _relerr(got, ref) <= TOL64, (steps, _relerr(got, ref))
