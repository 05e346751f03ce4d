"""Esoteric Twist propagation on the sparse lattice (oracle, torch CPU).

Test infrastructure only (see ``oracle/__init__``).

The paper lists Geier's Esoteric Twist next to OS-NT and the AA pattern as
the propagation schemes with the lowest loop balance, one that works on a
single grid like the AA pattern (Sect. 1, Sect. 4), but it does not evaluate
it or print its rules.  Reading implemented here (and, independently, by the
library):

* Every link between node x and x + c_i owns two slots, one per travel
  direction, at the *location* x + c_i^+ (c^+ = componentwise max(c, 0));
  seen from the other end y = x + c_i that is y + c_inv(i)^+, the same place.
  So a node touches only its own location and the six locations +x, +y, +z,
  +x+y, +x+z, +y+z.
* Even step (after an even number of steps): node n reads its incoming f_i
  from slot i at n + c_inv(i)^+, collides, and writes each outgoing P_j into
  slot inv(j) at n + c_j^+ -- the slot it read f_inv(j) from.  Odd step: the
  slot roles swap (read slot inv(i), write slot j).  Both ends of a fluid link
  read and write their own slot of the pair, so the step is race-free in
  place.
* A link whose far end is a wall (adjacency marker -1) or a pressure face
  (-2 / -3) has no partner; the writer stores the value the node itself pulls
  next step -- P_j (bounce-back) or 2 w rho_bc - P_j (anti-bounce-back) --
  into the *other* slot of the pair, the one the next step reads.  The
  canonical state is then read the same way for every direction.
* Locations that are not fluid nodes (a solid corner between two fluid nodes,
  a wall voxel, a face outside the box) still hold the slots of their links:
  they are "phantom" storage locations numbered after the N nodes, in
  lexicographic order of their (wrapped) coordinates, x fastest.

Layouts: 3 = after an even number of ET steps, 4 = after an odd number.
"""
from __future__ import annotations

import numpy as np
import torch

from .d3q19 import C, INV, W, Q
from .lbm import Params, collide

# the six neighbour locations, in table-row order
OFFSETS = np.array([(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1)], dtype=np.int64)


def loc_row(i: int) -> int:
    """Location of direction i's link slots relative to the node: -1 the node itself, else a row of OFFSETS."""
    cp = np.maximum(C[i], 0)
    if not cp.any():
        return -1
    return int(np.nonzero((OFFSETS == cp).all(axis=1))[0][0])


def tables(solid: np.ndarray, node_xyz: np.ndarray, adj: np.ndarray, periodic=(0, 0, 0)):
    """(nb [6, N], mask [N] uint32, phantom_xyz [M, 3]) of the ET form.

    nb[k, n]: storage index of location node_xyz[n] + OFFSETS[k] (wrapped on
    periodic axes): the node there, or N + the phantom's rank.  mask bit i-1
    (i = 1..18): the pull of direction i at n meets a marker; bit 18 + x(i)
    for the ten directions with c_ix != 0 (x(i) their rank in direction
    order): that marker is a pressure face.
    """
    Z, Y, X = solid.shape
    dims = np.array([X, Y, Z], dtype=np.int64)
    N = len(node_xyz)
    v2n = np.full((Z, Y, X), -1, dtype=np.int64)
    v2n[node_xyz[:, 2], node_xyz[:, 1], node_xyz[:, 0]] = np.arange(N)
    loc = np.empty((6, N, 3), dtype=np.int64)
    inside = np.empty((6, N), dtype=bool)
    for k in range(6):
        p = node_xyz.astype(np.int64) + OFFSETS[k]
        for a in range(3):
            if periodic[a]:
                p[:, a] %= dims[a]
        loc[k] = p
        inside[k] = (p < dims).all(axis=1)
    idx = np.full((6, N), -1, dtype=np.int64)
    for k in range(6):
        ok = inside[k]
        p = loc[k][ok]
        idx[k, ok] = v2n[p[:, 2], p[:, 1], p[:, 0]]
    need = idx < 0
    keys = ((loc[..., 2] * (Y + 1) + loc[..., 1]) * (X + 1) + loc[..., 0])[need]
    uniq = np.unique(keys)
    idx[need] = N + np.searchsorted(uniq, keys)
    phantom = np.stack([uniq % (X + 1), (uniq // (X + 1)) % (Y + 1), uniq // ((X + 1) * (Y + 1))], axis=1)
    mask = np.zeros(N, dtype=np.uint64)
    xdirs = [i for i in range(1, Q) if C[i][0] != 0]
    for i in range(1, Q):
        mask |= (adj[i - 1] < 0).astype(np.uint64) << np.uint64(i - 1)
    for r, i in enumerate(xdirs):
        mask |= (adj[i - 1] <= -2).astype(np.uint64) << np.uint64(18 + r)
    return idx.astype(np.int32), mask.astype(np.uint32), phantom.astype(np.int32)


def _locations(nb, N):
    """[7, N]: row 0 the node itself, rows 1..6 the six neighbour locations."""
    return torch.cat([torch.arange(N).unsqueeze(0), torch.as_tensor(nb, dtype=torch.int64)], dim=0)


def _rho_bc(mark, p: Params):
    return torch.where(mark == -2, torch.tensor(p.rho_in, dtype=torch.float64),
                       torch.tensor(p.rho_out, dtype=torch.float64))


def canonical(A, parity: int, nb):
    """Pre-collision F[19, N] of an ET grid A[19, S] after a step count of the given parity."""
    N = nb.shape[1]
    L = _locations(nb, N)
    F = torch.empty((Q, N), dtype=A.dtype)
    F[0] = A[0, :N]
    for i in range(1, Q):
        slot = i if parity == 0 else int(INV[i])
        F[i] = A[slot, L[loc_row(int(INV[i])) + 1]]
    return F


def from_canonical(F, parity: int, nb, S: int):
    """The ET grid [19, S] whose canonical state is F (phantom-only slots zero)."""
    N = F.shape[1]
    L = _locations(nb, N)
    A = torch.zeros((Q, S), dtype=F.dtype)
    A[0, :N] = F[0]
    for i in range(1, Q):
        slot = i if parity == 0 else int(INV[i])
        A[slot, L[loc_row(int(INV[i])) + 1]] = F[i]
    return A


def step(A, parity: int, nb, adj, p: Params, s=None):
    """One ET step of the grid A[19, S] from a step count of the given parity."""
    N = nb.shape[1]
    L = _locations(nb, N)
    adj = torch.as_tensor(adj, dtype=torch.int64)
    P = collide(canonical(A, parity, nb), p, s)
    out = A.clone()
    out[0, :N] = P[0]
    for j in range(1, Q):
        jj = int(INV[j])
        where = L[loc_row(j) + 1]
        mark = adj[jj - 1]                 # what node n pulls in direction inv(j) next step
        fluid = mark >= 0
        # fluid link: into the pair's slot this node read from (inv j even, j odd)
        own = jj if parity == 0 else j
        out[own, where[fluid]] = P[j, fluid]
        # wall or pressure face: the bounced value into the slot read next step
        other = j if parity == 0 else jj
        m = mark[~fluid]
        v = P[j, ~fluid]
        v = torch.where(m == -1, v, 2 * float(W[j]) * _rho_bc(m, p) - v)
        out[other, where[~fluid]] = v
    return out


def run(A, nb, adj, p: Params, steps: int, start_parity: int = 0, s=None):
    for k in range(steps):
        A = step(A, (start_parity + k) % 2, nb, adj, p, s)
    return A


def run_tables(nb, mask):
    """Run-length coding of the ET tables, the RIA idea of Sect. 4.1 applied to them.

    Node n >= 1 continues the run of node n-1 when each of its six locations
    is n-1's plus one and the link masks are equal (so both nodes' slots sit
    at the same offsets).  Returns (run_start [R+1], run_nb [6, R], run_mask [R])
    with the head's entries; decoding adds the offset within the run.
    """
    N = nb.shape[1]
    if N == 0:
        return np.zeros(1, np.int32), np.zeros((6, 0), np.int32), np.zeros(0, np.uint32)
    a = nb.astype(np.int64)
    cont = np.all(a[:, 1:] == a[:, :-1] + 1, axis=0) & (mask[1:] == mask[:-1])
    heads = np.concatenate([[0], np.nonzero(~cont)[0] + 1])
    run_start = np.concatenate([heads, [N]]).astype(np.int32)
    return run_start, np.ascontiguousarray(nb[:, heads]), mask[heads].copy()


def decode_runs(run_start, run_nb, run_mask):
    """Expand the ET run table back into (nb [6, N], mask [N])."""
    N = int(run_start[-1])
    lengths = np.diff(run_start.astype(np.int64))
    run_of = np.repeat(np.arange(len(lengths)), lengths)
    off = np.arange(N) - run_start[:-1].astype(np.int64)[run_of]
    return (run_nb[:, run_of].astype(np.int64) + off[None, :]).astype(np.int32), run_mask[run_of]
