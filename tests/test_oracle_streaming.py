"""Pins of the oracle's streaming, boundaries and storage forms (Sect. 4).

* the sparse pull step equals the dense full-array push LBM node for node;
* OS-NT and the AA pattern hold the same canonical state after every even
  number of steps (both compute Eq. 1; they only store it differently);
* mass is conserved to round-off with walls and periodic faces;
* plane Poiseuille flow under a body force with halfway bounce-back and
  the TRT magic parameter 3/16 is reproduced exactly (known TRT property);
* anti-bounce-back with rho_in = rho_out = rho0 keeps the rest state.
"""
import numpy as np
import pytest
import torch

import geometry
from oracle import dense, lbm, tables


def _perturbed_state(T, p, seed, amp=1e-2):
    g = torch.Generator().manual_seed(seed)
    F = lbm.uniform_state(T.N, p, 1.0, (0.01, -0.02, 0.005))
    return F * (1 + amp * (torch.rand(F.shape, generator=g, dtype=torch.float64) - 0.5))


CASES = [
    dict(periodic=(1, 0, 0), x_pressure=False),
    dict(periodic=(1, 1, 1), x_pressure=False),
    dict(periodic=(0, 0, 1), x_pressure=True),
    dict(periodic=(0, 0, 0), x_pressure=False),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("enum", [("lex", 1), ("lex", 2), ("hilbert", 1)])
def test_sparse_equals_dense(case, enum):
    bc = CASES[case]
    solid = geometry.random_voxels(7, 6, 5, 0.25, 40 + case)
    T = tables.Tables(solid, enum=enum[0], B=enum[1], **bc)
    p = lbm.Params(omega_plus=1.1, magic=3 / 16, g=(1e-4, 2e-5, -3e-5), rho_in=1.001, rho_out=0.999)
    s = torch.as_tensor(geometry.uniform_field(T.N, 7 + case), dtype=torch.float64) * 0.5
    F0 = _perturbed_state(T, p, case)
    G = lbm.from_canonical(F0, 0, T.adj, p)
    steps = 6
    G = lbm.run_osnt(G, T.adj, p, steps, s)
    F_sparse = lbm.canonical(G, 0, T.adj, p)
    # dense oracle works on voxels in raster order; map nodes to raster order
    vox = dense.fluid_voxels(solid)
    v2n = tables.voxel_to_node(solid, T.node_xyz)
    perm = torch.as_tensor(v2n[vox[:, 2], vox[:, 1], vox[:, 0]])
    F_dense = dense.run_dense(solid, F0[:, perm], p, steps, bc["periodic"], bc["x_pressure"], s[perm])
    assert torch.max(torch.abs(F_dense - F_sparse[:, perm])) <= 1e-15


@pytest.mark.parametrize("case", range(len(CASES)))
def test_osnt_equals_aa_after_even_steps(case):
    bc = CASES[case]
    solid = geometry.random_voxels(8, 6, 5, 0.2, 50 + case)
    T = tables.Tables(solid, enum="lex", B=1, **bc)
    p = lbm.Params(omega_plus=0.9, magic=0.25, g=(5e-5, 0, 1e-5), rho_in=1.002, rho_out=0.998)
    s = torch.as_tensor(geometry.uniform_field(T.N, 3), dtype=torch.float64)
    F0 = _perturbed_state(T, p, 10 + case)
    G = lbm.from_canonical(F0, 0, T.adj, p)
    A = lbm.from_canonical(F0, 1, T.adj, p)
    for n in range(1, 7):
        G = lbm.osnt_step(G, T.adj, p, s)
        A = lbm.aa_even(A, p, s) if n % 2 == 1 else lbm.aa_odd(A, T.adj, p, s)
        FG = lbm.canonical(G, 0, T.adj, p)
        FA = lbm.canonical(A, 1 if n % 2 == 0 else 2, T.adj, p)
        assert torch.max(torch.abs(FG - FA)) <= 1e-15


@pytest.mark.parametrize("layout", [0, 1, 2])
def test_layout_roundtrip(layout):
    solid = geometry.random_voxels(6, 6, 6, 0.3, 60)
    T = tables.Tables(solid, periodic=(0, 1, 0), x_pressure=True)
    p = lbm.Params(rho_in=1.01, rho_out=0.99)
    F = _perturbed_state(T, p, 5)
    G = lbm.from_canonical(F, layout, T.adj, p)
    assert torch.max(torch.abs(lbm.canonical(G, layout, T.adj, p) - F)) <= 1e-16


def test_mass_conservation_walls_periodic():
    solid = geometry.sphere_box_64x32x32(0)[:, :12, :16].copy()
    T = tables.Tables(solid, periodic=(1, 0, 0))
    p = lbm.Params(omega_plus=1.0, magic=3 / 16, g=(1e-4, 0, 0))
    F0 = _perturbed_state(T, p, 1)
    M0 = F0.sum()
    G = lbm.from_canonical(F0, 0, T.adj, p)
    G = lbm.run_osnt(G, T.adj, p, 60)
    M = lbm.canonical(G, 0, T.adj, p).sum()
    assert abs(float(M - M0)) / float(M0) <= 1e-13


def test_momentum_gain_fully_periodic():
    """With no walls the total momentum grows by exactly sum_n rho_n g per step."""
    solid = geometry.empty_box(5, 4, 3)
    T = tables.Tables(solid, periodic=(1, 1, 1))
    p = lbm.Params(omega_plus=1.2, magic=0.2, g=(3e-4, -1e-4, 2e-4))
    F = _perturbed_state(T, p, 2)
    G = lbm.from_canonical(F, 0, T.adj, p)
    for _ in range(5):
        F = lbm.canonical(G, 0, T.adj, p)
        j_before = lbm.C.t() @ F
        G = lbm.osnt_step(G, T.adj, p)
        F2 = lbm.canonical(G, 0, T.adj, p)
        gain = (lbm.C.t() @ F2).sum(1) - j_before.sum(1)
        ex = F.sum() * torch.tensor(p.g, dtype=torch.float64)
        assert torch.max(torch.abs(gain - ex)) <= 1e-15


def test_plane_poiseuille_exact():
    """u(y_j) = g/(2 nu) y_j (H - y_j), y_j = j + 1/2, for TRT with Lambda = 3/16."""
    H = 8
    solid = geometry.empty_box(1, H, 1)
    T = tables.Tables(solid, periodic=(1, 0, 1))
    p = lbm.Params(omega_plus=1.0, magic=3 / 16, g=(1e-4, 0, 0))
    G = lbm.from_canonical(lbm.uniform_state(T.N, p), 0, T.adj, p)
    G = lbm.run_osnt(G, T.adj, p, 5000)
    rho, u, _ = lbm.macroscopic(lbm.canonical(G, 0, T.adj, p), p)
    y = torch.as_tensor(T.node_xyz[:, 1], dtype=torch.float64) + 0.5
    exact = p.g[0] / (2 * p.nu) * y * (H - y)
    assert torch.max(torch.abs(u[0] - exact)) / exact.max() <= 1e-12
    assert torch.max(torch.abs(u[1:])) <= 1e-15
    assert torch.max(torch.abs(rho - 1)) <= 1e-12


def test_pressure_boundary_rest_state():
    solid = geometry.random_voxels(6, 5, 5, 0.2, 70)
    T = tables.Tables(solid, periodic=(0, 0, 0), x_pressure=True)
    p = lbm.Params(rho_in=1.0, rho_out=1.0)
    F = lbm.uniform_state(T.N, p, 1.0)
    G = lbm.from_canonical(F, 0, T.adj, p)
    G = lbm.run_osnt(G, T.adj, p, 10)
    assert torch.max(torch.abs(lbm.canonical(G, 0, T.adj, p) - F)) <= 1e-15


def test_pressure_driven_duct_flows_downhill():
    """An empty duct with rho_in > rho_out develops +x flow and a falling pressure."""
    solid = geometry.empty_box(12, 6, 6)
    T = tables.Tables(solid, periodic=(0, 0, 0), x_pressure=True)
    p = lbm.Params(omega_plus=1.0, magic=3 / 16, rho_in=1.003, rho_out=0.997)
    G = lbm.from_canonical(lbm.uniform_state(T.N, p), 0, T.adj, p)
    G = lbm.run_osnt(G, T.adj, p, 400)
    rho, u, _ = lbm.macroscopic(lbm.canonical(G, 0, T.adj, p), p)
    x = T.node_xyz[:, 0]
    prof = np.array([float(rho[torch.as_tensor(x == k)].mean()) for k in range(12)])
    assert float(u[0].mean()) > 0
    assert np.all(np.diff(prof) < 0)


def test_stream_at_equals_stream():
    """Pointwise evaluation of the pull at chosen nodes equals the full stream."""
    solid = geometry.random_voxels(9, 7, 6, 0.25, 90)
    T = tables.Tables(solid, periodic=(0, 1, 0), x_pressure=True)
    p = lbm.Params(rho_in=1.01, rho_out=0.99)
    P = _perturbed_state(T, p, 7)
    full = lbm.stream(P, T.adj, p)
    targets = torch.as_tensor(np.random.default_rng(0).choice(T.N, 40, replace=False))
    part = lbm.stream_at(lambda i, nodes: P[i, nodes], targets, T.adj, p)
    assert torch.equal(part, full[:, targets])
