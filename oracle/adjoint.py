"""Taped reverse sweep of the objective through T OS-NT steps (oracle).

Test infrastructure only (see ``oracle/__init__``).

The CUDA library hand-derives the discrete adjoint of one stream-collide
step; here the same derivative comes from torch autograd recording the
plain oracle forward, so the two share nothing but the definition of the
forward map and of the objective J = (1/N) sum_n rho_n u_x,n after T steps.
"""
from __future__ import annotations

import torch

from . import lbm


def flux_and_gradient(G0, adj, p: lbm.Params, s, T: int, wrt_state: bool = False):
    """J(s) after T OS-NT steps from grid G0, and dJ/ds (and dJ/dG0 if asked).

    Returns (J, dJ/ds[N]) or (J, dJ/ds, dJ/dG0[19, N]).
    """
    s = s.detach().clone().to(torch.float64).requires_grad_(True)
    G = G0.detach().clone().to(torch.float64).requires_grad_(wrt_state)
    X = G
    for _ in range(T):
        X = lbm.osnt_step(X, adj, p, s)
    F = lbm.stream(X, adj, p)
    J = lbm.objective_flux(F, p, s)
    inputs = [s, G] if wrt_state else [s]
    grads = torch.autograd.grad(J, inputs)
    if wrt_state:
        return J.detach(), grads[0], grads[1]
    return J.detach(), grads[0]


def flux(G0, adj, p: lbm.Params, s, T: int):
    """J(s) only (finite-difference checks)."""
    with torch.no_grad():
        X = G0.to(torch.float64)
        for _ in range(T):
            X = lbm.osnt_step(X, adj, p, s)
        return lbm.objective_flux(lbm.stream(X, adj, p), p, s)
