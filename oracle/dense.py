"""Full-array LBM with push streaming (oracle brute force for tiny boxes).

Test infrastructure only (see ``oracle/__init__``).

This is the lattice Boltzmann equation (Eq. 1, Sect. 2) on the dense voxel
array, written without any enumeration or adjacency list: every fluid voxel
collides, then pushes P_i to x + c_i.  A push that would land in a solid
voxel or through a wall face bounces back into the opposite slot of the same
voxel; one through a pressure face (x = -1 or x = X when x is a pressure
axis) is anti-bounced back with 2 w_i rho_bc.  The sparse oracle and the
CUDA library must both reproduce it node for node.
"""
from __future__ import annotations

import numpy as np
import torch

from .d3q19 import C, INV, W, Q
from .lbm import Params, collide


def fluid_voxels(solid):
    z, y, x = np.nonzero(solid == 0)
    return np.stack([x, y, z], axis=1).astype(np.int64)


def push_stream(Pv, solid, vox, periodic, x_pressure, p: Params):
    """Push post-collision PDFs Pv[19, M] of the fluid voxels ``vox`` (x, y, z)."""
    Z, Y, X = solid.shape
    dims = (X, Y, Z)
    idx = np.full(solid.shape, -1, dtype=np.int64)
    idx[vox[:, 2], vox[:, 1], vox[:, 0]] = np.arange(len(vox))
    out = torch.full_like(Pv, float("nan"))
    out[0] = Pv[0]
    for i in range(1, Q):
        ii = int(INV[i])
        t = vox + C[i][None, :]
        wall = np.zeros(len(vox), bool)
        press = np.zeros(len(vox), bool)
        rho_bc = np.zeros(len(vox))
        for a in range(3):
            lo, hi = t[:, a] < 0, t[:, a] >= dims[a]
            if periodic[a]:
                t[:, a] %= dims[a]
            elif a == 0 and x_pressure:
                press |= lo | hi
                rho_bc = np.where(lo, p.rho_in, np.where(hi, p.rho_out, rho_bc))
            else:
                wall |= lo | hi
        press &= ~wall
        inside = ~(wall | press)
        tgt = np.full(len(vox), -1, dtype=np.int64)
        ti = t[inside]
        tgt[inside] = idx[ti[:, 2], ti[:, 1], ti[:, 0]]
        to_fluid = tgt >= 0
        bounce = ~to_fluid & ~press
        src = np.arange(len(vox))
        out[i, torch.as_tensor(tgt[to_fluid])] = Pv[i, torch.as_tensor(src[to_fluid])]
        out[ii, torch.as_tensor(src[bounce])] = Pv[i, torch.as_tensor(src[bounce])]
        pr = torch.as_tensor(src[press])
        out[ii, pr] = -Pv[i, pr] + 2 * float(W[i]) * torch.as_tensor(rho_bc[press])
    return out


def run_dense(solid, F0v, p: Params, steps, periodic=(0, 0, 0), x_pressure=False, s_vox=None):
    """Advance the canonical states F0v[19, M] of the fluid voxels (raster order) by ``steps``."""
    vox = fluid_voxels(solid)
    F = F0v.clone()
    for _ in range(steps):
        P = collide(F, p, s_vox)
        F = push_stream(P, solid, vox, periodic, x_pressure, p)
    return F
