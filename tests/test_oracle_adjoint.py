"""Pins of the oracle's taped reverse sweep (the discrete adjoint's reference).

* the gradient of J w.r.t. the Brinkman field matches central finite
  differences of the plain forward;
* the objective's closed-form derivatives dJ/dF and dJ/ds hold;
* the dot-product identity <lambda, J v> = <J^T lambda, v> for one step,
  with J v from a finite difference in FP64.
"""
import numpy as np
import torch

import geometry
from oracle import adjoint, lbm, tables


def _setup(seed=0):
    solid = geometry.random_voxels(6, 5, 4, 0.15, 80 + seed)
    T = tables.Tables(solid, periodic=(1, 0, 1))
    p = lbm.Params(omega_plus=1.0, magic=3 / 16, g=(1e-3, 0, 0))
    s = torch.as_tensor(geometry.uniform_field(T.N, 5 + seed), dtype=torch.float64) * 0.3
    G0 = lbm.from_canonical(lbm.uniform_state(T.N, p), 0, T.adj, p)
    return T, p, s, G0


def test_gradient_vs_central_differences():
    T, p, s, G0 = _setup()
    steps = 12
    J, dJ = adjoint.flux_and_gradient(G0, T.adj, p, s, steps)
    h = 1e-5
    rng = np.random.default_rng(1)
    for n in rng.choice(T.N, 6, replace=False):
        sp, sm = s.clone(), s.clone()
        sp[n] += h
        sm[n] -= h
        fd = (adjoint.flux(G0, T.adj, p, sp, steps) - adjoint.flux(G0, T.adj, p, sm, steps)) / (2 * h)
        assert abs(float(fd - dJ[n])) <= 1e-6 * abs(float(dJ[n])) + 1e-14


def test_objective_closed_form_derivatives():
    T, p, s, G0 = _setup(1)
    F = lbm.canonical(G0, 0, T.adj, p) * (1 + 1e-3 * torch.rand(19, T.N, dtype=torch.float64))
    F = F.requires_grad_(True)
    ss = s.clone().requires_grad_(True)
    J = lbm.objective_flux(F, p, ss)
    dF, ds = torch.autograd.grad(J, [F, ss])
    cx = lbm.C[:, 0][:, None]
    ex_dF = (cx + p.g[0] / 2) / ((1 + s / 2) * T.N)
    rho, _, u = lbm.moments(F.detach(), p, s)
    ex_ds = -rho * u[0] / (2 * (1 + s / 2) * T.N)
    assert torch.allclose(dF, ex_dF.expand_as(dF), rtol=0, atol=1e-17)
    assert torch.allclose(ds, ex_ds, rtol=1e-13, atol=1e-19)


def test_one_step_dot_product():
    T, p, s, G0 = _setup(2)
    F = lbm.canonical(G0, 0, T.adj, p) * (1 + 1e-2 * torch.rand(19, T.N, dtype=torch.float64))
    G = lbm.from_canonical(F, 0, T.adj, p)
    lam = torch.rand(19, T.N, dtype=torch.float64)
    v = torch.rand(19, T.N, dtype=torch.float64)
    Gr = G.clone().requires_grad_(True)
    out = lbm.osnt_step(Gr, T.adj, p, s)
    (vjp,) = torch.autograd.grad(out, Gr, lam)
    h = 1e-6
    jv = (lbm.osnt_step(G + h * v, T.adj, p, s) - lbm.osnt_step(G - h * v, T.adj, p, s)) / (2 * h)
    lhs = float((lam * jv).sum())
    rhs = float((vjp * v).sum())
    assert abs(lhs - rhs) <= 1e-8 * abs(rhs)
