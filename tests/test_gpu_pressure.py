"""The library's pressure faces against the closed-form Darcy-duct steady state.

The same pin as the oracle's (tests/test_oracle_pressure.py): a straight duct,
periodic in y and z, pressure faces in x at x = -1/2 and X - 1/2, uniform
Brinkman drag s.  At steady state rho(x) falls linearly from rho_in to
rho_out between the faces, the flux rho u_x equals (rho_in - rho_out)/(3 s X)
at every node, and u_y = u_z = 0.  The tolerances are the bounds set by the
anti-bounce-back rule's dropped O(u^2) terms (4 rho u^2 on the density profile)
and round-off.  Every storage form and addressing runs in FP64; the ragged
duct covers several CTAs and a partial last one.
"""
import numpy as np
import pytest
import torch

import geometry

pytestmark = pytest.mark.gpu

import paper_1410_0412_gb300 as lbm

EPS = float(np.finfo(np.float64).eps)


@pytest.mark.parametrize("form,ria", [("osnt", False), ("osnt", True), ("aa", False), ("aa", True),
                                      ("et", False), ("et", True)])
@pytest.mark.parametrize("X,Y,Z,delta,s32,steps", [(8, 2, 2, 1e-5, 0.5, 2000), (40, 9, 7, 1e-5, 0.1, 30000)])
def test_darcy_duct_closed_form(form, ria, X, Y, Z, delta, s32, steps):
    solid = geometry.empty_box(X, Y, Z)
    lat = lbm.Lattice(solid, periodic=(0, 1, 1), x_pressure=True).upload(
        lbm.LBM_TABLES_ADJ | lbm.LBM_TABLES_RIA | lbm.LBM_TABLES_ET)
    s_val = float(np.float32(s32))
    s = torch.full((lat.N,), s_val, dtype=torch.float32, device="cuda")
    params = lbm.Params(omega_plus=1.0, magic=3 / 16, rho_in=1 + delta, rho_out=1 - delta)
    sv = lbm.Solver(lat, "f64", params, form=form, ria=ria, s=s)
    sv.init_equilibrium(1.0)
    sv.step(steps)
    rho, u, _ = sv.macroscopic(sums=False)
    rho2 = rho.clone()
    sv.step(2)
    rho_next, _, _ = sv.macroscopic(sums=False)
    assert float((rho_next - rho2).abs().max()) <= 1e-15   # steady
    x = torch.as_tensor(lat.tables(adj=False, runs=False)["node_xyz"][:, 0].astype(np.float64), device="cuda")
    rho_in, rho_out = 1 + delta, 1 - delta
    q0 = (rho_in - rho_out) / (3 * s_val * X)
    tol_rho = 4 * q0 ** 2 + 300 * EPS
    tol_q = (8 * q0 ** 2 + 600 * EPS) / (3 * s_val * X)
    rho_lin = rho_in - (rho_in - rho_out) * (x + 0.5) / X
    assert float((rho - rho_lin).abs().max()) <= tol_rho
    assert float((rho * u[0] - q0).abs().max()) <= tol_q
    assert float(u[1:].abs().max()) <= 1e-20
