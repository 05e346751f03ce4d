"""Pins of the oracle's D3Q19 constants and TRT collision (Sect. 2).

Each pin is a property the collision must have independent of how the
oracle writes it: lattice isotropy, conservation, the exact momentum change
under a force, the rest state as a fixed point, and the reduction to the
textbook single-relaxation-time (BGK) operator with Guo forcing when both
TRT rates are equal.
"""
import itertools

import numpy as np
import torch

from oracle import d3q19, lbm

torch.manual_seed(0)


def _random_state(N, seed, amp=0.02):
    g = torch.Generator().manual_seed(seed)
    rho = 1 + 0.05 * (torch.rand(N, generator=g, dtype=torch.float64) - 0.5)
    u = 0.05 * (torch.rand(3, N, generator=g, dtype=torch.float64) - 0.5)
    feq = lbm.equilibrium(rho, u)
    return feq * (1 + amp * (torch.rand(19, N, generator=g, dtype=torch.float64) - 0.5))


def test_lattice_isotropy():
    C, W = d3q19.C.astype(float), d3q19.W
    assert abs(W.sum() - 1) < 1e-15
    assert np.allclose(W @ C, 0, atol=1e-16)
    assert np.allclose((W[:, None, None] * C[:, :, None] * C[:, None, :]).sum(0), np.eye(3) / 3, atol=1e-16)
    # fourth moment: sum w c_a c_b c_c c_d = (d_ab d_cd + d_ac d_bd + d_ad d_bc)/9
    d = np.eye(3)
    for a, b, c, e in itertools.product(range(3), repeat=4):
        m4 = (W * C[:, a] * C[:, b] * C[:, c] * C[:, e]).sum()
        ex = (d[a, b] * d[c, e] + d[a, c] * d[b, e] + d[a, e] * d[b, c]) / 9
        assert abs(m4 - ex) < 1e-16
    for i in range(19):
        assert np.all(C[d3q19.INV[i]] == -C[i])
    # odd directions paired with the next one (2k-1 <-> 2k)
    for k in range(1, 10):
        assert d3q19.INV[2 * k - 1] == 2 * k


def test_equilibrium_moments():
    N = 64
    rho = 1 + 0.1 * torch.rand(N, dtype=torch.float64)
    u = 0.1 * (torch.rand(3, N, dtype=torch.float64) - 0.5)
    feq = lbm.equilibrium(rho, u)
    C = lbm.C
    assert torch.allclose(feq.sum(0), rho, rtol=0, atol=1e-15)
    assert torch.allclose(C.t() @ feq, rho * u, rtol=0, atol=1e-15)
    # second moment: sum c c feq = rho/3 I + rho u u
    M2 = torch.einsum("ia,ib,in->abn", C, C, feq)
    ex = rho / 3 * torch.eye(3, dtype=torch.float64)[:, :, None] + rho * u[:, None, :] * u[None, :, :]
    assert torch.allclose(M2, ex, rtol=0, atol=1e-15)


def test_conservation_and_momentum_change():
    N = 200
    F = _random_state(N, 1)
    s = torch.rand(N, dtype=torch.float64)
    p = lbm.Params(omega_plus=1.3, magic=3 / 16, g=(1e-3, -2e-4, 5e-4))
    P = lbm.collide(F, p, s)
    rho, j0, u = lbm.moments(F, p, s)
    assert torch.allclose(P.sum(0), rho, rtol=0, atol=2e-15)
    g = torch.tensor(p.g, dtype=torch.float64)[:, None]
    force = rho * g - s * rho * u
    # post-collision momentum is exactly j0 + F
    assert torch.allclose(lbm.C.t() @ P, j0 + force, rtol=0, atol=2e-15)
    # u solves u = (j0 + F/2)/rho with the implicit drag
    assert torch.allclose(u, (j0 + force / 2) / rho, rtol=0, atol=1e-15)


def test_rest_state_fixed_point():
    N = 10
    rho = torch.full((N,), 1.02, dtype=torch.float64)
    F = lbm.equilibrium(rho, torch.zeros(3, N, dtype=torch.float64))
    for om in (0.6, 1.0, 1.9):
        p = lbm.Params(omega_plus=om, magic=0.25)
        assert torch.allclose(lbm.collide(F, p, torch.rand(N, dtype=torch.float64)), F, rtol=0, atol=4e-16)


def test_bgk_special_case():
    """lambda+ = lambda- reduces TRT to BGK with the Guo force term.

    Textbook form: f* = f - w (f - feq) + (1 - w/2) w_i [(c_i - u)/cs^2 + (c_i.u) c_i / cs^4] . F
    """
    N = 100
    F = _random_state(N, 2)
    om = 1.25
    # choose magic so that lambda- = lambda+ = om: Lambda = (1/om - 1/2)^2
    p = lbm.Params(omega_plus=om, magic=(1 / om - 0.5) ** 2, g=(2e-4, 1e-4, -3e-4))
    assert abs(p.lam_minus - om) < 1e-14
    P = lbm.collide(F, p)
    rho, j0, u = lbm.moments(F, p)
    force = rho * torch.tensor(p.g, dtype=torch.float64)[:, None]
    feq = lbm.equilibrium(rho, u)
    cs2 = 1.0 / 3.0
    ex = torch.empty_like(F)
    for i in range(19):
        c = lbm.C[i][:, None]
        term = ((c - u) / cs2 + (c * u).sum(0) * c / cs2 ** 2)
        Si = float(lbm.W[i]) * (term * force).sum(0)
        ex[i] = F[i] - om * (F[i] - feq[i]) + (1 - om / 2) * Si
    assert torch.allclose(P, ex, rtol=0, atol=1e-16)


def test_trt_rates_from_magic():
    p = lbm.Params(omega_plus=1.0, magic=3 / 16)
    assert abs(p.lam_minus - 8 / 7) < 1e-15
    assert abs(p.nu - 1 / 6) < 1e-16


def test_trt_pair_relaxation():
    """Even/odd parts relax with their own rate when there is no force."""
    N = 50
    F = _random_state(N, 3)
    p = lbm.Params(omega_plus=0.8, magic=0.1)
    P = lbm.collide(F, p)
    rho, j0, u = lbm.moments(F, p)
    feq = lbm.equilibrium(rho, u)
    inv = lbm.INV
    ep, em = (F + F[inv]) / 2 - (feq + feq[inv]) / 2, (F - F[inv]) / 2 - (feq - feq[inv]) / 2
    Pp, Pm = (P + P[inv]) / 2 - (feq + feq[inv]) / 2, (P - P[inv]) / 2 - (feq - feq[inv]) / 2
    assert torch.allclose(Pp, (1 - p.lam_plus) * ep, rtol=0, atol=1e-16)
    assert torch.allclose(Pm, (1 - p.lam_minus) * em, rtol=0, atol=1e-16)
