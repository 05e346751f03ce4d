"""FP64 lattice Boltzmann stepping on the sparse lattice (oracle, torch CPU).

Test infrastructure only (see ``oracle/__init__``).

The lattice Boltzmann equation (Eq. 1, Sect. 2) splits into a local collision
Omega and a propagation to the neighbours.  The paper uses the two-relaxation-
time (TRT) operator of Ginzburg et al. (2008) without printing it; the form
implemented here is:

    rho = sum_i f_i,  j0 = sum_i c_i f_i,  F = rho g - s rho u,
    u = (j0/rho + g/2) / (1 + s/2)          (u = (j0 + F/2)/rho, drag implicit)
    feq+_i = w_i rho (1 + 9/2 (c_i.u)^2 - 3/2 u.u),  feq-_i = 3 w_i rho (c_i.u)
    S+_i = w_i (9 (c_i.u)(c_i.F) - 3 u.F),           S-_i = 3 w_i (c_i.F)
    f+-_i = (f_i +- f_inv(i)) / 2
    f*_i = f_i - l+ (f+_i - feq+_i) - l- (f-_i - feq-_i)
               + (1 - l+/2) S+_i + (1 - l-/2) S-_i

with l+ = omega_plus and l- fixed by the "magic" parameter
Lambda = (1/l+ - 1/2)(1/l- - 1/2).  s is the per-node Brinkman solid
fraction (0 when absent).

Streaming is the pull scheme of Sect. 4 ("Loop Balance"): F'[i][n] =
P[i][adj(i, n)].  Markers: -1 halfway bounce-back F'[i][n] = P[inv i][n];
-2 / -3 pressure anti-bounce-back F'[i][n] = -P[inv i][n] + 2 w_i rho_bc
with rho_bc = rho_in / rho_out.

Storage forms (Sect. 4):
  * OS-NT: the grid holds post-collision PDFs; one step pulls them from the
    neighbours (indirect), collides, and stores locally (direct) into the
    other grid.  The canonical (pre-collision) state is stream(grid).
  * AA pattern, one grid: the even step reads the 19 local PDFs, collides and
    writes them back into the opposite slots of the same node; the odd step
    reads and writes the neighbours' slots through the adjacency list.  After
    an even number of steps the grid holds the canonical state; after an odd
    number it holds the post-collision PDFs in opposite slots.

Layouts: 0 = OS-NT grid, 1 = AA after an even number of steps, 2 = AA after
an odd number of steps.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from .d3q19 import C as _C, INV as _INV, W as _W, Q

C = torch.tensor(_C, dtype=torch.float64)          # [19, 3]
W = torch.tensor(_W, dtype=torch.float64)          # [19]
INV = torch.tensor(_INV, dtype=torch.int64)        # [19]


@dataclass
class Params:
    omega_plus: float = 1.0
    magic: float = 3.0 / 16.0
    g: tuple = (0.0, 0.0, 0.0)
    rho0: float = 1.0
    rho_in: float = 1.0
    rho_out: float = 1.0

    @property
    def lam_plus(self) -> float:
        return self.omega_plus

    @property
    def lam_minus(self) -> float:
        # Lambda = (1/l+ - 1/2)(1/l- - 1/2)
        return 1.0 / (self.magic / (1.0 / self.omega_plus - 0.5) + 0.5)

    @property
    def nu(self) -> float:
        return (1.0 / self.omega_plus - 0.5) / 3.0


def as_t(a, dtype=torch.float64):
    if isinstance(a, torch.Tensor):
        return a.to(dtype)
    return torch.as_tensor(np.asarray(a), dtype=dtype)


# ---------------------------------------------------------------------------
# Collision (Sect. 2: TRT)
# ---------------------------------------------------------------------------

def moments(F, p: Params, s=None):
    """rho, j0 and the force-corrected velocity u of pre-collision PDFs F[19, N]."""
    rho = F.sum(0)
    j0 = C.t() @ F                                    # [3, N]
    g = torch.tensor(p.g, dtype=F.dtype)[:, None]
    sn = torch.zeros_like(rho) if s is None else s
    u = (j0 / rho + g / 2) / (1 + sn / 2)
    return rho, j0, u


def equilibrium(rho, u):
    """f^eq_i = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)."""
    cu = C @ u
    uu = (u * u).sum(0)
    return W[:, None] * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * uu)


def collide(F, p: Params, s=None):
    """Post-collision PDFs P[19, N] of the TRT operator with Guo forcing and drag."""
    lp, lm = p.lam_plus, p.lam_minus
    rho, _, u = moments(F, p, s)
    g = torch.tensor(p.g, dtype=F.dtype)[:, None]
    sn = torch.zeros_like(rho) if s is None else s
    Fo = rho * g - sn * rho * u                        # [3, N]
    cu = C @ u                                        # [19, N]
    cF = C @ Fo
    uu = (u * u).sum(0)
    uF = (u * Fo).sum(0)
    w = W[:, None]
    feq_p = w * rho * (1 + 4.5 * cu ** 2 - 1.5 * uu)
    feq_m = 3 * w * rho * cu
    S_p = w * (9 * cu * cF - 3 * uF)
    S_m = 3 * w * cF
    f_p = (F + F[INV]) / 2
    f_m = (F - F[INV]) / 2
    return (F - lp * (f_p - feq_p) - lm * (f_m - feq_m)
            + (1 - lp / 2) * S_p + (1 - lm / 2) * S_m)


# ---------------------------------------------------------------------------
# Streaming (Sect. 4: pull scheme) and its inverse
# ---------------------------------------------------------------------------

def _rho_bc(mark, p: Params, dtype):
    return torch.where(mark == -2, torch.tensor(p.rho_in, dtype=dtype),
                       torch.tensor(p.rho_out, dtype=dtype))


def stream(P, adj, p: Params):
    """Canonical pull: F'[i][n] from P via adj (node indices and markers).

    P may hold more columns than adj has nodes (a chunk's ghost slots, Sect. 6):
    nodes are the first adj.shape[1] columns, pulls may read any column.
    """
    adj = as_t(adj, torch.int64)
    N = adj.shape[1]
    Fn = torch.empty((Q, N), dtype=P.dtype)
    Fn[0] = P[0, :N]
    for i in range(1, Q):
        m = adj[i - 1]
        fluid = m >= 0
        ii = int(_INV[i])
        from_nb = P[i][m.clamp(min=0)]
        bb = P[ii, :N]
        abb = -bb + 2 * float(_W[i]) * _rho_bc(m, p, P.dtype)
        Fn[i] = torch.where(fluid, from_nb, torch.where(m == -1, bb, abb))
    return Fn


def stream_at(P_of, targets, adj, p: Params):
    """The canonical pull of ``stream`` evaluated only at the nodes ``targets``.

    ``P_of(i, nodes)`` returns the post-collision PDFs P[i][nodes] (global node
    ids); it only has to know the targets and their pull sources.  Used to
    check single nodes of a large lattice one by one.
    """
    adj = as_t(adj, torch.int64)
    targets = as_t(targets, torch.int64)
    Fn = torch.empty((Q, len(targets)), dtype=torch.float64)
    Fn[0] = P_of(0, targets)
    for i in range(1, Q):
        m = adj[i - 1][targets]
        ii = int(_INV[i])
        fluid = m >= 0
        from_nb = P_of(i, torch.where(fluid, m, targets))
        own = P_of(ii, targets)
        abb = -own + 2 * float(_W[i]) * _rho_bc(m, p, own.dtype)
        Fn[i] = torch.where(fluid, from_nb, torch.where(m == -1, own, abb))
    return Fn


def unstream(F, adj, p: Params):
    """The grid G with stream(G) = F (streaming is a bijection of PDF slots)."""
    adj = as_t(adj, torch.int64)
    G = torch.empty_like(F)
    G[0] = F[0]
    for j in range(1, Q):
        jj = int(_INV[j])
        m = adj[jj - 1]                  # the slot (j, n) is pulled by node m = adj(inv j, n)
        fluid = m >= 0
        from_nb = F[j][m.clamp(min=0)]
        bb = F[jj]
        abb = 2 * float(_W[j]) * _rho_bc(m, p, F.dtype) - F[jj]
        G[j] = torch.where(fluid, from_nb, torch.where(m == -1, bb, abb))
    return G


# ---------------------------------------------------------------------------
# The two storage forms (Sect. 4)
# ---------------------------------------------------------------------------

def osnt_step(G, adj, p: Params, s=None):
    """OS-NT: pull from the neighbours, collide, store locally in the other grid."""
    return collide(stream(G, adj, p), p, s)


def aa_even(A, p: Params, s=None):
    """AA even step: local read, collide, write to the opposite local slots."""
    P = collide(A, p, s)
    out = torch.empty_like(A)
    out[_INV] = P
    return out


def aa_odd(A, adj, p: Params, s=None):
    """AA odd step: read the neighbours' opposite slots, collide, write them back."""
    adj = as_t(adj, torch.int64)
    N = A.shape[1]
    n = torch.arange(N)
    F = torch.empty_like(A)
    F[0] = A[0]
    for i in range(1, Q):
        m = adj[i - 1]
        ii = int(_INV[i])
        nb = A[ii][m.clamp(min=0)]
        own = A[i]
        abb = -A[i] + 2 * float(_W[i]) * _rho_bc(m, p, A.dtype)
        F[i] = torch.where(m >= 0, nb, torch.where(m == -1, own, abb))
    P = collide(F, p, s)
    out = A.clone()
    out[0] = P[0]
    for i in range(1, Q):
        ii = int(_INV[i])
        m = adj[ii - 1]                   # where P_i of this node is pulled next
        fluid = m >= 0
        # to a neighbour: slot (i, m)
        out[i, m[fluid]] = P[i, n[fluid]]
        # to itself: slot (inv i, n), bounce-back or anti-bounce-back
        bb = ~fluid & (m == -1)
        out[ii, n[bb]] = P[i, n[bb]]
        ab = ~fluid & (m != -1)
        rb = _rho_bc(m[ab], p, A.dtype)
        out[ii, n[ab]] = -P[i, n[ab]] + 2 * float(_W[i]) * rb
    return out


def canonical(pdf, layout: int, adj, p: Params):
    """Pre-collision PDFs F[19, N] stored in a grid of the given layout."""
    if layout == 0:
        return stream(pdf, adj, p)
    if layout == 1:
        return pdf.clone()
    if layout == 2:
        return stream(pdf[_INV], adj, p)
    raise ValueError(layout)


def from_canonical(F, layout: int, adj, p: Params):
    """The grid of a layout whose canonical state is F (inverse of ``canonical``)."""
    if layout == 0:
        return unstream(F, adj, p)
    if layout == 1:
        return F.clone()
    if layout == 2:
        G = unstream(F, adj, p)
        out = torch.empty_like(G)
        out[_INV] = G
        return out
    raise ValueError(layout)


def uniform_state(N, p: Params, rho0=1.0, u0=(0.0, 0.0, 0.0)):
    rho = torch.full((N,), float(rho0), dtype=torch.float64)
    u = torch.tensor(u0, dtype=torch.float64)[:, None].expand(3, N)
    return equilibrium(rho, u)


# ---------------------------------------------------------------------------
# Macroscopic quantities and the objective
# ---------------------------------------------------------------------------

def macroscopic(F, p: Params, s=None):
    """rho[N], u[3, N] and sums [sum rho, sum rho u_x, sum rho u_y, sum rho u_z]."""
    rho, _, u = moments(F, p, s)
    j = rho * u
    sums = torch.stack([rho.sum(), j[0].sum(), j[1].sum(), j[2].sum()])
    return rho, u, sums


def objective_flux(F, p: Params, s=None):
    """J = (1/N) sum_n rho_n u_x,n (mean x-momentum flux)."""
    rho, _, u = moments(F, p, s)
    return (rho * u[0]).sum() / F.shape[1]


def partitioned_osnt_step(grids, parts, p: Params, s=None):
    """One OS-NT step of a P-chunk split (Sect. 6): every chunk first receives
    its ghost PDFs (slot `slot` of array i <- the owner's P_i at `node`), then
    pulls and collides its own nodes.  grids[k]: chunk k's grid [19, Np + slots]
    (post-collision state in the node columns); parts from
    ``tables.partition_local_tables``.  Returns the new chunk grids."""
    for G, part in zip(grids, parts):
        for q in np.unique(part["q"]):
            e = part["q"] == q
            d = torch.as_tensor(part["dir"][e], dtype=torch.int64)
            G[d, torch.as_tensor(part["slot"][e], dtype=torch.int64)] = \
                grids[int(q)][d, torch.as_tensor(part["node"][e], dtype=torch.int64)]
    out = []
    for G, part in zip(grids, parts):
        a, n = part["first"], part["N"]
        sk = None if s is None else s[a:a + n]
        Gn = torch.zeros_like(G)
        Gn[:, :n] = collide(stream(G, part["adj"], p), p, sk)
        out.append(Gn)
    return out


def run_osnt(G, adj, p: Params, steps: int, s=None):
    for _ in range(steps):
        G = osnt_step(G, adj, p, s)
    return G


def run_aa(A, adj, p: Params, steps: int, start_parity: int = 0, s=None):
    t = start_parity
    for _ in range(steps):
        A = aa_even(A, p, s) if t % 2 == 0 else aa_odd(A, adj, p, s)
        t += 1
    return A
