"""Quantitative pins of the oracle's pressure (anti-bounce-back) faces.

The paper has no pressure boundary; the oracle's reading (both storage forms)
is F_i = -P_inv(i) + 2 w_i rho_bc at a node whose pull source lies behind the
x = -1 face (inlet, rho_in) or the x = X face (outlet, rho_out), with the
O(u^2) wall term of the full anti-bounce-back rule dropped.  The rule puts the
face halfway between the last node and the missing one: at x = -1/2 and
x = X - 1/2.

Pin: a straight duct, periodic in y and z, pressure faces in x, with a
uniform Brinkman drag s (Darcy flow).  Its steady state has a closed form:
 * mass: the flux q = rho u_x is the same at every node;
 * momentum: d/dx (rho/3 + rho u_x^2 + Pi_neq) = -s q; the u^2 and
   non-equilibrium terms vary along x only at O(u^2 delta) and O(nu q delta / X),
   so p = rho/3 falls linearly between the faces:
       rho(x) = rho_in - (rho_in - rho_out) (x + 1/2) / X,
       q = (rho_in - rho_out) / (3 s X);
 * symmetry: u_y = u_z = 0.
What the dropped wall term changes: the rule imposes
sum over the five incoming links of (F_i + P_inv(i)) = 2 rho_bc sum w_i = rho_bc/3
where the full rule has 2 rho_bc sum w_i (1 + 9/2 (c_i.u)^2 - 3/2 u.u) =
(rho_bc/3)(1 + 3 u_x^2) (c_x = 1 on every incoming link).  So each face sits at
a density off by 3 rho u^2.  The rule also sets the face pressure to rho/3
where the momentum flux through the face is rho/3 + rho u^2, another rho u^2.
The profile is therefore off by at most 4 rho u^2, and the flux by at most
8 rho u^2 / (3 s X).  Round-off adds a few hundred ulps of rho (about 1).  The tolerances below are
these bounds, not fitted values; a planted face-density mistake (faces
swapped, or 2 w rho_bc taken as w rho_bc + w rho0) misses them by orders of
magnitude.
"""
import numpy as np
import pytest
import torch

import geometry
from oracle import lbm, tables

EPS = float(np.finfo(np.float64).eps)


def _duct_steady_state(X, delta, s_val, form, steps=800):
    solid = geometry.empty_box(X, 2, 2)
    T = tables.Tables(solid, periodic=(0, 1, 1), x_pressure=True)
    p = lbm.Params(omega_plus=1.0, magic=3 / 16, rho_in=1 + delta, rho_out=1 - delta)
    s = torch.full((T.N,), s_val, dtype=torch.float64)
    F0 = lbm.uniform_state(T.N, p)
    if form == "osnt":
        G = lbm.run_osnt(lbm.from_canonical(F0, 0, T.adj, p), T.adj, p, steps, s)
        F = lbm.canonical(G, 0, T.adj, p)
        F_prev = lbm.canonical(lbm.run_osnt(G, T.adj, p, 2, s), 0, T.adj, p)
    else:
        A = lbm.run_aa(lbm.from_canonical(F0, 1, T.adj, p), T.adj, p, steps, 0, s)
        F = lbm.canonical(A, 1, T.adj, p)
        F_prev = lbm.canonical(lbm.run_aa(A, T.adj, p, 2, 0, s), 1, T.adj, p)
    # steady: two more steps change nothing beyond round-off
    assert float((F_prev - F).abs().max()) <= 1e-15
    rho, u, _ = lbm.macroscopic(F, p, s)
    x = torch.as_tensor(T.node_xyz[:, 0], dtype=torch.float64)
    return rho, u, x, p


def _duct_errors(rho, u, x, X, delta, s_val):
    rho_in, rho_out = 1 + delta, 1 - delta
    rho_lin = rho_in - (rho_in - rho_out) * (x + 0.5) / X
    q0 = (rho_in - rho_out) / (3 * s_val * X)
    u0 = q0  # rho ~ 1
    tol_rho = 4 * u0 ** 2 + 300 * EPS
    tol_q = (8 * u0 ** 2 + 600 * EPS) / (3 * s_val * X)
    err_rho = float((rho - rho_lin).abs().max())
    err_q = float((rho * u[0] - q0).abs().max())
    return err_rho, tol_rho, err_q, tol_q


@pytest.mark.parametrize("form", ["osnt", "aa"])
@pytest.mark.parametrize("X,delta,s_val", [(8, 1e-5, 0.5), (8, 1e-6, 0.25), (12, 1e-5, 0.5)])
def test_darcy_duct_matches_closed_form(form, X, delta, s_val):
    rho, u, x, p = _duct_steady_state(X, delta, s_val, form)
    err_rho, tol_rho, err_q, tol_q = _duct_errors(rho, u, x, X, delta, s_val)
    assert err_rho <= tol_rho, (err_rho, tol_rho)
    assert err_q <= tol_q, (err_q, tol_q)
    # the bounds are far below the pressure drop and the flux themselves
    assert tol_rho <= 1e-5 * 2 * delta and tol_q <= 1e-5 * 2 * delta / (3 * s_val * X)
    assert float(u[1:].abs().max()) <= 1e-20


def _planted(monkeypatch, kind):
    real = lbm._rho_bc

    def swapped(mark, p, dtype):
        return torch.where(mark == -2, torch.tensor(p.rho_out, dtype=dtype), torch.tensor(p.rho_in, dtype=dtype))

    def half_weight(mark, p, dtype):
        # 2 w rho_bc applied as w rho_bc + w rho0
        return (real(mark, p, dtype) + p.rho0) / 2

    monkeypatch.setattr(lbm, "_rho_bc", {"swapped": swapped, "half_weight": half_weight}[kind])


@pytest.mark.parametrize("kind", ["swapped", "half_weight"])
@pytest.mark.parametrize("form", ["osnt", "aa"])
def test_darcy_duct_catches_planted_face_errors(monkeypatch, kind, form):
    X, delta, s_val = 8, 1e-5, 0.5
    _planted(monkeypatch, kind)
    rho, u, x, p = _duct_steady_state(X, delta, s_val, form)
    err_rho, tol_rho, err_q, tol_q = _duct_errors(rho, u, x, X, delta, s_val)
    assert err_rho > 1e3 * tol_rho and err_q > 1e3 * tol_q
