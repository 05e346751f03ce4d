"""lbm_macroscopic_noalloc: macroscopic sums for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc (a host application whose
pool allocator owns all device memory, or a loop that must not run a
possibly synchronising allocation), so they cannot hand lbm_macroscopic its
reduction workspace.  lbm_macroscopic_noalloc keeps those partial sums in a
fixed array inside the library instead.  These tests check it against
lbm_macroscopic through the C ABI, on two calls in a row (different lattice
sizes, so stale partials from the first call would show in the second), and
that oversized lattices are refused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import geometry
import paper_1410_0412_gb300 as lbm
from paper_1410_0412_gb300 import _lib


def _case(solid, seed, prec="f64", form="aa"):
    lat = lbm.Lattice(solid, periodic=(1, 0, 0)).upload(lbm.LBM_TABLES_ADJ | lbm.LBM_TABLES_RIA | lbm.LBM_TABLES_ET)
    p = lbm.Params(g=(1e-5, 0.0, 0.0), shifted=(prec != "f64"))
    solver = lbm.Solver(lat, prec, p, form=form, ria=True)
    solver.init_equilibrium(1.0, (0.01, 0.0, 0.0))
    solver.step(3 + seed)          # odd step count: AA_ODD / ET_ODD layout, gathers through the tables
    return lat, p, solver


def _compare(lat, p, prec, solver, stream=None):
    ref_rho, ref_u, ref_sums = lbm.lbm_macroscopic(lat, prec, p, solver.pdf, solver.layout)
    rho = torch.full((lat.N,), float("nan"), dtype=torch.float64, device="cuda")
    u = torch.full((3, lat.N), float("nan"), dtype=torch.float64, device="cuda")
    sums = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())
    lbm.lbm_macroscopic_noalloc(lat, prec, p, solver.pdf, solver.layout, rho=rho, u=u, sums=sums, stream=stream)
    torch.cuda.synchronize()
    assert float((sums - ref_sums).abs().max() / ref_sums.abs().max()) <= 1e-13
    assert float((rho - ref_rho).abs().max()) <= 1e-15
    assert float((u - ref_u).abs().max()) <= 1e-15


@pytest.mark.gpu
def test_noalloc_matches_macroscopic_two_calls_in_a_row():
    cases = [(geometry.sphere_box_64x32x32(0), 0, "f64"),
             (geometry.random_voxels(23, 19, 17, 0.25, 9), 1, "f32")]
    for solid, seed, prec in cases:
        lat, p, solver = _case(solid, seed, prec)
        _compare(lat, p, prec, solver)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f16s"])
def test_noalloc_esoteric_twist_layout_on_a_side_stream(prec):
    """The Esoteric Twist layouts are accepted (as by lbm_macroscopic), also on a non-default stream."""
    side = torch.cuda.Stream()
    for seed in (0, 1):            # ET_ODD, then ET_EVEN
        lat, p, solver = _case(geometry.random_voxels(23, 19, 17, 0.25, 9 + seed), seed, prec, form="et")
        _compare(lat, p, prec, solver, stream=side)


@pytest.mark.gpu
def test_noalloc_wrapper_rejects_bad_outputs():
    """The kernels write N, 3N and 4 doubles: wrong dtypes, sizes or devices are refused before any launch."""
    lat, p, solver = _case(geometry.random_voxels(11, 9, 7, 0.25, 3), 0)
    good = dict(rho=torch.empty(lat.N, dtype=torch.float64, device="cuda"),
                u=torch.empty((3, lat.N), dtype=torch.float64, device="cuda"),
                sums=torch.empty(4, dtype=torch.float64, device="cuda"))
    bad = [("rho", torch.empty(lat.N, dtype=torch.float32, device="cuda"), TypeError),
           ("rho", torch.empty(lat.N - 1, dtype=torch.float64, device="cuda"), ValueError),
           ("u", torch.empty((3, lat.N - 1), dtype=torch.float64, device="cuda"), ValueError),
           ("u", torch.empty((lat.N, 3), dtype=torch.float64, device="cuda").t(), ValueError),
           ("sums", torch.empty(3, dtype=torch.float64, device="cuda"), ValueError),
           ("sums", torch.empty(4, dtype=torch.float64), TypeError)]
    for name, t, err in bad:
        kw = dict(good)
        kw[name] = t
        with pytest.raises(err):
            lbm.lbm_macroscopic_noalloc(lat, "f64", p, solver.pdf, solver.layout, **kw)


@pytest.mark.gpu
def test_noalloc_sums_only_and_mass():
    lat, p, solver = _case(geometry.sphere_box_64x32x32(0), 2)
    sums = torch.empty(4, dtype=torch.float64, device="cuda")
    for _ in range(2):
        lbm.lbm_macroscopic_noalloc(lat, "f64", p, solver.pdf, solver.layout, sums=sums)
        torch.cuda.synchronize()
        # walls and a periodic axis conserve mass: total = N * rho0
        assert abs(float(sums[0]) - lat.N) <= 1e-10 * lat.N


@pytest.mark.slow
def test_noalloc_rejects_lattices_beyond_its_limit():
    """One node past the limit is refused (host only).  Memory: the lattice's
    18 x (2^24 + 1) int32 adjacency list is built on the host, about 1.2 GB
    held twice while the library copies it; deselect with -m "not slow" on
    small hosts."""
    N = (1 << 24) + 1
    adj = np.full((18, N), -1, dtype=np.int32)
    lat = lbm.Lattice.from_adjacency(adj)
    del adj
    p = lbm.Params()
    rc = _lib.load().lbm_macroscopic_noalloc(lat.handle, lbm.LBM_F64, ctypes.byref(p.c()), ctypes.c_void_p(256),
                                             lbm.LBM_LAYOUT_AA_EVEN, None, None, None, None, None)
    assert rc == _lib.LBM_ERR_ARG
    assert b"16777216" in _lib.load().lbm_last_error()
