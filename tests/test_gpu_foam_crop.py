"""The foam precision study against the oracle on a 64^3 crop.

The crop is the corner z, y, x < 64 of the 512^3 Voronoi-edge foam of the
precision study (400 seeds, strut radius 2.5, seed 3), with pressure faces in
x (rho = 1 +- 5e-4) and walls elsewhere.  After 200 AA-R (or OS-NT-R) steps
from rest the GPU's canonical state, velocity and pressure drop are compared
with the FP64 oracle's AA run (the two forms agree after an even number of
steps): FP64 and double-float at the 1e-12 bar, FP32 and FP16S storage within
their stated storage-format bounds.
"""
import numpy as np
import pytest
import torch

import geometry
from oracle import lbm as olbm
from oracle import tables as otables

pytestmark = pytest.mark.gpu

import paper_1410_0412_gb300 as lbm

STEPS = 200


@pytest.fixture(scope="module")
def crop():
    solid = geometry.voronoi_foam(512, 512, 512, 400, 2.5, 3)[:64, :64, :64].copy()
    T = otables.Tables(solid, periodic=(0, 0, 0), x_pressure=True)
    op = olbm.Params(omega_plus=1.0, magic=3 / 16, rho_in=1.0 + 5e-4, rho_out=1.0 - 5e-4)
    A = olbm.from_canonical(olbm.uniform_state(T.N, op), 1, T.adj, op)
    A = olbm.run_aa(A, T.adj, op, STEPS, 0)
    F = olbm.canonical(A, 1, T.adj, op)
    rho, u, _ = olbm.macroscopic(F, op)
    x = T.node_xyz[:, 0]
    dp = float((rho[torch.as_tensor(x < 4)].mean() - rho[torch.as_tensor(x >= 60)].mean()) / 3.0)
    return solid, T, F, u, dp


@pytest.mark.parametrize("prec,tol_f,tol_u,tol_dp", [("f64", 1e-12, 1e-9, 1e-10), ("f64df", 1e-12, 1e-9, 1e-10),
                                                     ("f32", 2e-6, 1e-3, 1e-5), ("f16s", 5e-4, 5e-2, 1e-3)])
@pytest.mark.parametrize("form", ["aa", "osnt"])
def test_foam_crop_against_oracle(crop, prec, tol_f, tol_u, tol_dp, form):
    solid, T, F_ref, u_ref, dp_ref = crop
    lat = lbm.Lattice(solid, periodic=(0, 0, 0), x_pressure=True).upload()
    lp = lbm.Params(omega_plus=1.0, magic=3 / 16, rho_in=1.0 + 5e-4, rho_out=1.0 - 5e-4,
                    shifted=prec in ("f32", "f16s"))
    sv = lbm.Solver(lat, prec, lp, form=form, ria=True)
    sv.init_equilibrium(1.0)
    sv.step(STEPS)
    F = sv.canonical().cpu()
    rho, u, _ = sv.macroscopic(sums=False)
    rho, u = rho.cpu(), u.cpu()
    x = T.node_xyz[:, 0]
    dp = float((rho[torch.as_tensor(x < 4)].mean() - rho[torch.as_tensor(x >= 60)].mean()) / 3.0)
    assert float((F - F_ref).abs().max() / F_ref.abs().max()) <= tol_f
    assert float((u - u_ref).abs().max() / u_ref.abs().max()) <= tol_u
    assert abs(dp - dp_ref) / abs(dp_ref) <= tol_dp
