"""The largest configuration: 768^3 Voronoi foam, Hilbert order, pressure faces, FP32 AA-R.

About 4.4e8 fluid nodes: the lattice is validated in full (ranges,
reciprocity, run table), and two AA-R steps from a uniform moving
equilibrium are checked against the FP64 oracle at sampled nodes, each from
its two-step dependency cone.  The cones' adjacency rows come from the
library (the oracle cannot build tables of this size in a test; the tables
themselves are pinned bit-exact against the oracle on smaller lattices).
"""
import numpy as np
import pytest
import torch

import geometry
from oracle import lbm as olbm
import paper_1410_0412_gb300 as lbm

pytestmark = pytest.mark.gpu

W = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12


def test_maxsize_foam_sampled_parity():
    n = 768
    solid = geometry.voronoi_foam(n, n, n, 1500, 3.0, 5)
    lat = lbm.Lattice(solid, periodic=(0, 0, 0), x_pressure=True, enum="hilbert")
    del solid
    assert lat.N > 4e8
    lat.validate()
    lat.upload(lbm.LBM_TABLES_RIA)
    u0 = (0.02, -0.01, 0.005)
    kw = dict(omega_plus=1.0, magic=3 / 16, rho_in=1.0005, rho_out=0.9995)
    op = olbm.Params(**kw)
    lp = lbm.Params(shifted=True, **kw)
    solver = lbm.Solver(lat, "f32", lp, form="aa", ria=True)
    solver.init_equilibrium(1.0, u0)
    solver.step(2)
    torch.cuda.synchronize()
    rng = np.random.default_rng(21)
    S = np.sort(rng.choice(lat.N, 500, replace=False))
    got = (solver.pdf[:, torch.as_tensor(S, device="cuda")].double().cpu()
           + torch.tensor(W, dtype=torch.float64)[:, None] * lp.rho0)

    def cone(nodes):
        rows = torch.as_tensor(lat.adjacency_rows(nodes).astype(np.int64))
        nb = rows.reshape(-1)
        return np.unique(np.concatenate([nodes, nb[nb >= 0].numpy()]))

    S1 = cone(S)
    S0 = cone(S1)
    # canonical state and adjacency on the cone, re-indexed to local rows
    loc = {int(g): k for k, g in enumerate(S0)}
    g = lat.adjacency_rows(S0).astype(np.int64)
    pos = np.searchsorted(S0, g)
    inside = (g >= 0) & (S0[np.minimum(pos, len(S0) - 1)] == g)
    # rows of the outer shell may point outside the cone; those rows are never streamed
    adj_loc = torch.as_tensor(np.where(g >= 0, np.where(inside, pos, -99), g))
    F0 = olbm.uniform_state(len(S0), op, 1.0, u0)
    P0 = olbm.collide(F0, op)
    idx1 = torch.as_tensor([loc[int(g)] for g in S1])
    F1 = olbm.stream_at(lambda i, nodes: P0[i, nodes], idx1, adj_loc, op)
    P1full = torch.zeros_like(P0)
    P1full[:, idx1] = olbm.collide(F1, op)
    idx = torch.as_tensor([loc[int(g)] for g in S])
    ref = olbm.stream_at(lambda i, nodes: P1full[i, nodes], idx, adj_loc, op)
    err = float((got - ref).abs().max() / ref.abs().max())
    assert err <= 1e-6
