"""GB300 sparse-lattice D3Q19 TRT stream-collide: Python binding of liblbm.

A thin layer over the C ABI in ``include/lbm.h``: it marshals numpy arrays,
torch CUDA tensors (device memory and streams only) and parameters into the
library's calls.  Every step of the method runs in the library: the host
lattice builder (C++) and the sm_103a CUDA kernels.  Importing this package
fails if ``liblbm.so`` has not been built; there is no fallback.

Functions named ``lbm_*`` mirror the C entry points one to one; ``Lattice``
and ``Solver`` bundle them for convenience.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import (LBM_ENUM_HILBERT, LBM_ENUM_LEX, LBM_F16S, LBM_F32, LBM_F64, LBM_F64_DF, LBM_HALO_AA_GATHER,
                   LBM_HALO_AA_SCATTER, LBM_HALO_OSNT, LBM_LAYOUT_AA_EVEN, LBM_LAYOUT_ET_EVEN, LBM_LAYOUT_ET_ODD,
                   LBM_TABLES_ET,
                   LBM_LAYOUT_AA_ODD, LBM_LAYOUT_OSNT, LBM_TABLES_ADJ, LBM_TABLES_RIA, LbmError, check)

_lib.load()

PRECISIONS = {"f64": LBM_F64, "f32": LBM_F32, "f16s": LBM_F16S, "f64df": LBM_F64_DF}
BYTES_PER_PDF = {LBM_F64: 8, LBM_F32: 4, LBM_F16S: 2, LBM_F64_DF: 8}


def _torch():
    import torch
    return torch


def _dtype(prec):
    torch = _torch()
    return {LBM_F64: torch.float64, LBM_F32: torch.float32, LBM_F16S: torch.float16, LBM_F64_DF: torch.float64}[prec]


def _prec(prec) -> int:
    if isinstance(prec, str):
        return PRECISIONS[prec]
    return int(prec)


@dataclass
class Params:
    """Step parameters (``lbm_params``): TRT rates, body force, densities, storage shift."""

    omega_plus: float = 1.0
    magic: float = 3.0 / 16.0
    g: tuple = (0.0, 0.0, 0.0)
    rho0: float = 1.0
    rho_in: float = 1.0
    rho_out: float = 1.0
    shifted: bool = False
    f16_scale: float = 1024.0

    def c(self) -> _lib.lbm_params:
        p = _lib.lbm_params()
        p.omega_plus = self.omega_plus
        p.magic = self.magic
        for a in range(3):
            p.g[a] = float(self.g[a])
        p.rho0 = self.rho0
        p.rho_in = self.rho_in
        p.rho_out = self.rho_out
        p.shifted = 1 if self.shifted else 0
        p.f16_scale = self.f16_scale
        return p


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_grid(lat, prec, t, name, layout=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != _dtype(prec):
        raise TypeError(f"{name} has dtype {t.dtype}, precision needs {_dtype(prec)}")
    et = layout is not None and layout >= LBM_LAYOUT_ET_EVEN
    stride = lat.et_info()[1] if et else lat.Npad
    if not t.is_contiguous() or t.numel() < 19 * stride:
        raise ValueError(f"{name} must be contiguous with at least 19 * {'Spad' if et else 'Npad'} elements")


def _check_s(lat, s):
    torch = _torch()
    if s is None:
        return None
    if not s.is_cuda or s.dtype != torch.float32 or not s.is_contiguous() or s.numel() < lat.N:
        raise TypeError("s must be a contiguous CUDA float32 tensor with N elements")
    return s


class Lattice:
    """A sparse lattice (``lbm_build_lattice``): enumeration, adjacency and RIA tables."""

    def __init__(self, solid=None, periodic=(0, 0, 0), x_pressure=False, enum="lex", B=1, _handle=None,
                 _owner=None):
        self._h = ctypes.c_void_p()
        self._dev = None
        self._owner = _owner  # a Partitioning that owns this handle (never freed here)
        self.uploaded = 0
        if _handle is not None:
            self._h = _handle
        else:
            solid = np.ascontiguousarray(solid, dtype=np.uint8)
            if solid.ndim != 3:
                raise ValueError("solid must be [Z, Y, X]")
            Z, Y, X = solid.shape
            bc = _lib.lbm_bc()
            for a in range(3):
                bc.periodic[a] = 1 if periodic[a] else 0
            bc.x_pressure = 1 if x_pressure else 0
            e = {"lex": LBM_ENUM_LEX, "hilbert": LBM_ENUM_HILBERT}[enum]
            check(_lib.load().lbm_build_lattice(solid.ctypes.data_as(ctypes.c_void_p), X, Y, Z,
                                                ctypes.byref(bc), e, int(B), ctypes.byref(self._h)),
                  "lbm_build_lattice")
        self._info()

    @classmethod
    def from_order(cls, solid, node_xyz, periodic=(0, 0, 0), x_pressure=False):
        """A lattice with the caller's node order (every fluid voxel once)."""
        solid = np.ascontiguousarray(solid, dtype=np.uint8)
        Z, Y, X = solid.shape
        xyz = np.ascontiguousarray(node_xyz, dtype=np.int32)
        bc = _lib.lbm_bc()
        for a in range(3):
            bc.periodic[a] = 1 if periodic[a] else 0
        bc.x_pressure = 1 if x_pressure else 0
        h = ctypes.c_void_p()
        check(_lib.load().lbm_build_lattice_ordered(solid.ctypes.data_as(ctypes.c_void_p), X, Y, Z, ctypes.byref(bc),
                                                    xyz.ctypes.data_as(ctypes.c_void_p), len(xyz), ctypes.byref(h)),
              "lbm_build_lattice_ordered")
        return cls(_handle=h)

    def renumber_partitions(self, P):
        """Node order after the two-stage renumbering: P chunks, each re-sorted lexicographically."""
        out = np.empty((self.N, 3), np.int32)
        check(_lib.load().lbm_renumber_partitions(self._h, int(P), out.ctypes.data_as(ctypes.c_void_p)),
              "lbm_renumber_partitions")
        return out

    def partition_ghosts(self, P):
        """Ghost PDFs per chunk of a P-way split of the node list."""
        out = np.empty(int(P), np.int64)
        check(_lib.load().lbm_partition_ghosts(self._h, int(P), out.ctypes.data_as(ctypes.c_void_p)),
              "lbm_partition_ghosts")
        return out

    @classmethod
    def from_adjacency(cls, adj, node_xyz=None):
        adj = np.ascontiguousarray(adj, dtype=np.int32)
        N = adj.shape[1]
        h = ctypes.c_void_p()
        xyz = None
        if node_xyz is not None:
            xyz = np.ascontiguousarray(node_xyz, dtype=np.int32)
        check(_lib.load().lbm_lattice_from_adjacency(
            N, adj.ctypes.data_as(ctypes.c_void_p),
            None if xyz is None else xyz.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)),
            "lbm_lattice_from_adjacency")
        return cls(_handle=h)

    def _info(self):
        N, Np, R = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        hist = (ctypes.c_int64 * 33)()
        check(_lib.load().lbm_lattice_info(self._h, ctypes.byref(N), ctypes.byref(Np), ctypes.byref(R), hist),
              "lbm_lattice_info")
        self.N, self.Npad, self.R = N.value, Np.value, R.value
        self.run_hist = np.array(list(hist), dtype=np.int64)

    @property
    def handle(self):
        return self._h

    def tables(self, node_xyz=True, adj=True, runs=True):
        """Host tables as numpy arrays (node_xyz [N,3], adj [18,N], run_start [R+1], run_adj [18,R]);
        tables not asked for are returned as None."""
        N, R = self.N, self.R
        xyz = np.empty((N, 3), np.int32) if node_xyz else None
        adj = np.empty((18, N), np.int32) if adj else None
        rs = np.empty(R + 1, np.int32) if runs else None
        ra = np.empty((18, R), np.int32) if runs else None
        p = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
        check(_lib.load().lbm_export_tables(self._h, p(xyz), p(adj), p(rs), p(ra)), "lbm_export_tables")
        return {"node_xyz": xyz, "adj": adj, "run_start": rs, "run_adj": ra}

    def run_slots(self, kind):
        """The RIA steps' run slot table [R, 18] (kind 0: AA odd step, 1: OS-NT step),
        or None where the lattice has none (``lbm_export_run_slots``)."""
        avail = ctypes.c_int()
        lib = _lib.load()
        check(lib.lbm_export_run_slots(self._h, int(kind), None, ctypes.byref(avail)), "lbm_export_run_slots")
        if not avail.value:
            return None
        out = np.empty((self.R, 18), np.int32)
        check(lib.lbm_export_run_slots(self._h, int(kind), out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(avail)),
              "lbm_export_run_slots")
        return out

    def validate(self):
        check(_lib.load().lbm_validate_tables(self._h), "lbm_validate_tables")

    def adjacency_rows(self, nodes):
        """Adjacency entries [18, len(nodes)] of the given nodes (large lattices)."""
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        out = np.empty((18, len(nodes)), np.int32)
        check(_lib.load().lbm_export_adjacency_rows(self._h, nodes.ctypes.data_as(ctypes.c_void_p), len(nodes),
                                                    out.ctypes.data_as(ctypes.c_void_p)),
              "lbm_export_adjacency_rows")
        return out

    def device_table_bytes(self, which=LBM_TABLES_ADJ | LBM_TABLES_RIA) -> int:
        b = ctypes.c_size_t()
        check(_lib.load().lbm_device_table_bytes(self._h, which, ctypes.byref(b)), "lbm_device_table_bytes")
        return b.value

    def upload(self, which=LBM_TABLES_ADJ | LBM_TABLES_RIA, device="cuda", stream=None):
        """Copy the tables to a torch-allocated device buffer owned by this object."""
        torch = _torch()
        nbytes = self.device_table_bytes(which)
        buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        st = _stream(stream)
        check(_lib.load().lbm_lattice_upload(self._h, which, _ptr(buf), nbytes, st), "lbm_lattice_upload")
        torch.cuda.synchronize(buf.device)
        self._dev = buf
        self.uploaded = which
        return self

    def pdf_bytes(self, prec) -> int:
        b = ctypes.c_size_t()
        check(_lib.load().lbm_pdf_bytes(self._h, _prec(prec), ctypes.byref(b)), "lbm_pdf_bytes")
        return b.value

    def new_grid(self, prec, device="cuda", et=False):
        """A zeroed grid [19, Npad] (or [19, Spad] for the Esoteric Twist form)."""
        torch = _torch()
        return torch.zeros((19, self.et_info()[1] if et else self.Npad), dtype=_dtype(_prec(prec)), device=device)

    def et_info(self):
        """(S, Spad, phantom_xyz [S-N, 3]) of the Esoteric Twist form (``lbm_et_info``)."""
        if getattr(self, "_et", None) is None:
            S, Sp = ctypes.c_int64(), ctypes.c_int64()
            check(_lib.load().lbm_et_info(self._h, ctypes.byref(S), ctypes.byref(Sp), None), "lbm_et_info")
            ph = np.empty((S.value - self.N, 3), np.int32)
            check(_lib.load().lbm_et_info(self._h, None, None, ph.ctypes.data_as(ctypes.c_void_p)), "lbm_et_info")
            self._et = (S.value, Sp.value, ph)
        return self._et

    def et_runs(self):
        """Run-length coding of the Esoteric Twist tables: run_start [R+1], run_nb [6, R], run_mask [R]."""
        R = ctypes.c_int64()
        lib = _lib.load()
        check(lib.lbm_export_et_runs(self._h, ctypes.byref(R), None, None, None), "lbm_export_et_runs")
        rs = np.empty(R.value + 1, np.int32)
        rnb = np.empty((6, R.value), np.int32)
        rm = np.empty(R.value, np.uint32)
        q = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        check(lib.lbm_export_et_runs(self._h, None, q(rs), q(rnb), q(rm)), "lbm_export_et_runs")
        return rs, rnb, rm

    def et_tables(self):
        """Esoteric Twist tables on the host: nb [6, N] int32 and mask [N] uint32."""
        nb = np.empty((6, self.N), np.int32)
        mask = np.empty(self.N, np.uint32)
        check(_lib.load().lbm_export_et_tables(self._h, nb.ctypes.data_as(ctypes.c_void_p),
                                               mask.ctypes.data_as(ctypes.c_void_p)), "lbm_export_et_tables")
        return nb, mask

    def reduce_workspace_bytes(self) -> int:
        b = ctypes.c_size_t()
        check(_lib.load().lbm_reduce_workspace_bytes(self._h, ctypes.byref(b)), "lbm_reduce_workspace_bytes")
        return b.value

    def close(self):
        if self._h and self._owner is None:
            _lib.load().lbm_free_lattice(self._h)
        self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Partitioning:
    """P chunks of a lattice's node vector, each a local lattice with ghost slots (``lbm_partition_build``).

    Chunk p holds nodes [N p / P, N (p+1) / P) of ``lat`` (Sect. 6.1); ``parts[p]``
    is its local lattice, usable with the step functions, and the exchange
    table moves the ghost PDFs between the chunks' grids each step (Sect. 6).
    """

    def __init__(self, lat: Lattice, P: int):
        self._h = ctypes.c_void_p()
        lib = _lib.load()
        check(lib.lbm_partition_build(lat.handle, int(P), ctypes.byref(self._h)), "lbm_partition_build")
        self.P = int(P)
        self.N = lat.N
        self.first, self.sizes, self.ghost_pdfs, self.ghost_slots, self.parts = [], [], [], [], []
        for p in range(self.P):
            f, n, g, gs = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
            check(lib.lbm_partition_info(self._h, p, ctypes.byref(f), ctypes.byref(n), ctypes.byref(g),
                                         ctypes.byref(gs)), "lbm_partition_info")
            self.first.append(f.value)
            self.sizes.append(n.value)
            self.ghost_pdfs.append(g.value)
            self.ghost_slots.append(gs.value)
            h = ctypes.c_void_p()
            check(lib.lbm_partition_local(self._h, p, ctypes.byref(h)), "lbm_partition_local")
            self.parts.append(Lattice(_handle=h, _owner=self))
        self._dev = None

    @property
    def handle(self):
        return self._h

    def ghosts(self, p):
        """Chunk p's ghost PDFs in exchange order: owner chunk, direction 1..18, local slot, owner-local node."""
        n = self.ghost_pdfs[p]
        out = {k: np.empty(n, np.int32) for k in ("src_part", "dir", "slot", "src_node")}
        q = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        check(_lib.load().lbm_partition_export_ghosts(self._h, int(p), q(out["src_part"]), q(out["dir"]),
                                                      q(out["slot"]), q(out["src_node"])),
              "lbm_partition_export_ghosts")
        return out

    def validate(self, lat: Lattice):
        check(_lib.load().lbm_partition_validate(self._h, lat.handle), "lbm_partition_validate")

    def upload(self, which=LBM_TABLES_ADJ | LBM_TABLES_RIA, device="cuda", stream=None):
        """Upload every local lattice's tables and the exchange table (torch-owned buffers)."""
        torch = _torch()
        for lat in self.parts:
            lat.upload(which, device, stream)
        nbytes = ctypes.c_size_t()
        check(_lib.load().lbm_halo_table_bytes(self._h, ctypes.byref(nbytes)), "lbm_halo_table_bytes")
        buf = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=device)
        check(_lib.load().lbm_halo_upload(self._h, _ptr(buf), nbytes.value, _stream(stream)), "lbm_halo_upload")
        torch.cuda.synchronize(buf.device)
        self._dev = buf
        return self

    def new_grids(self, prec, device="cuda"):
        """One zeroed grid [19, Npad_p] per chunk."""
        return [lat.new_grid(prec, device) for lat in self.parts]

    @staticmethod
    def pointers(grids, device=None):
        """The device array of grid addresses that ``lbm_halo_exchange`` takes."""
        torch = _torch()
        dev = device or grids[0].device
        return torch.tensor([g.data_ptr() for g in grids], dtype=torch.int64, device=dev)

    def scatter(self, grid, grids):
        """Copy a whole-lattice grid [19, >= N] into the chunks' node slots."""
        for p, g in enumerate(grids):
            a, n = self.first[p], self.sizes[p]
            g[:, :n].copy_(grid[:, a:a + n])

    def gather(self, grids, out=None):
        """The chunks' node slots as one whole-lattice grid [19, N]."""
        torch = _torch()
        if out is None:
            out = torch.empty((19, self.N), dtype=grids[0].dtype, device=grids[0].device)
        for p, g in enumerate(grids):
            a, n = self.first[p], self.sizes[p]
            out[:, a:a + n].copy_(g[:, :n])
        return out

    def close(self):
        for lat in self.parts:
            lat.close()
        if self._h:
            _lib.load().lbm_free_partitioning(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- entry points with the C names ---------------------------------------------------------

def lbm_init_equilibrium(lat, prec, params, pdf, layout, rho0=1.0, u0=(0.0, 0.0, 0.0), stream=None):
    prec = _prec(prec)
    _check_grid(lat, prec, pdf, "pdf", layout)
    u = (ctypes.c_double * 3)(*[float(v) for v in u0])
    check(_lib.load().lbm_init_equilibrium(lat.handle, prec, ctypes.byref(params.c()), _ptr(pdf), layout,
                                           float(rho0), u, _stream(stream)), "lbm_init_equilibrium")


def lbm_load_canonical(lat, prec, params, F, pdf, layout, stream=None):
    torch = _torch()
    prec = _prec(prec)
    _check_grid(lat, prec, pdf, "pdf", layout)
    if not F.is_cuda or F.dtype != torch.float64 or tuple(F.shape) != (19, lat.N) or not F.is_contiguous():
        raise TypeError("F must be a contiguous CUDA float64 tensor [19, N]")
    check(_lib.load().lbm_load_canonical(lat.handle, prec, ctypes.byref(params.c()), _ptr(F), _ptr(pdf), layout,
                                         _stream(stream)), "lbm_load_canonical")


def lbm_canonical_pdfs(lat, prec, params, pdf, layout, F=None, stream=None):
    torch = _torch()
    prec = _prec(prec)
    _check_grid(lat, prec, pdf, "pdf", layout)
    if F is None:
        F = torch.empty((19, lat.N), dtype=torch.float64, device=pdf.device)
    check(_lib.load().lbm_canonical_pdfs(lat.handle, prec, ctypes.byref(params.c()), _ptr(pdf), layout, _ptr(F),
                                         _stream(stream)), "lbm_canonical_pdfs")
    return F


def lbm_step_osnt(lat, prec, params, src, dst, s=None, ria=False, stream=None):
    prec = _prec(prec)
    _check_grid(lat, prec, src, "src")
    _check_grid(lat, prec, dst, "dst")
    check(_lib.load().lbm_step_osnt(lat.handle, prec, ctypes.byref(params.c()), _ptr(src), _ptr(dst),
                                    _ptr(_check_s(lat, s)), 1 if ria else 0, _stream(stream)), "lbm_step_osnt")


def lbm_step_aa(lat, prec, params, pdf, parity, s=None, ria=False, stream=None):
    prec = _prec(prec)
    _check_grid(lat, prec, pdf, "pdf")
    check(_lib.load().lbm_step_aa(lat.handle, prec, ctypes.byref(params.c()), _ptr(pdf), int(parity),
                                  _ptr(_check_s(lat, s)), 1 if ria else 0, _stream(stream)), "lbm_step_aa")


def lbm_run_aa(lat, prec, params, pdf, start_parity, steps, s=None, ria=False, stream=None):
    prec = _prec(prec)
    _check_grid(lat, prec, pdf, "pdf")
    check(_lib.load().lbm_run_aa(lat.handle, prec, ctypes.byref(params.c()), _ptr(pdf), int(start_parity),
                                 int(steps), _ptr(_check_s(lat, s)), 1 if ria else 0, _stream(stream)),
          "lbm_run_aa")


def lbm_step_et(lat, prec, params, pdf, parity, s=None, ria=False, stream=None):
    prec = _prec(prec)
    _check_grid(lat, prec, pdf, "pdf", LBM_LAYOUT_ET_EVEN)
    check(_lib.load().lbm_step_et(lat.handle, prec, ctypes.byref(params.c()), _ptr(pdf), int(parity),
                                  _ptr(_check_s(lat, s)), 1 if ria else 0, _stream(stream)), "lbm_step_et")


def lbm_run_et(lat, prec, params, pdf, start_parity, steps, s=None, ria=False, stream=None):
    prec = _prec(prec)
    _check_grid(lat, prec, pdf, "pdf", LBM_LAYOUT_ET_EVEN)
    check(_lib.load().lbm_run_et(lat.handle, prec, ctypes.byref(params.c()), _ptr(pdf), int(start_parity),
                                 int(steps), _ptr(_check_s(lat, s)), 1 if ria else 0, _stream(stream)),
          "lbm_run_et")


def lbm_macroscopic(lat, prec, params, pdf, layout, s=None, fields=True, sums=True, workspace=None, stream=None):
    """(rho [N], u [3, N], sums [4]) as FP64 CUDA tensors (None where not asked for)."""
    torch = _torch()
    prec = _prec(prec)
    _check_grid(lat, prec, pdf, "pdf", layout)
    dev = pdf.device
    rho = torch.empty(lat.N, dtype=torch.float64, device=dev) if fields else None
    u = torch.empty((3, lat.N), dtype=torch.float64, device=dev) if fields else None
    out = torch.empty(4, dtype=torch.float64, device=dev) if sums else None
    ws_bytes = lat.reduce_workspace_bytes()
    if sums and workspace is None:
        workspace = torch.empty(ws_bytes // 8, dtype=torch.float64, device=dev)
    check(_lib.load().lbm_macroscopic(lat.handle, prec, ctypes.byref(params.c()), _ptr(pdf), layout,
                                      _ptr(_check_s(lat, s)), _ptr(rho), _ptr(u), _ptr(out), _ptr(workspace),
                                      ws_bytes if sums else 0, _stream(stream)), "lbm_macroscopic")
    return rho, u, out


def lbm_macroscopic_noalloc(lat, prec, params, pdf, layout, s=None, rho=None, u=None, sums=None, stream=None):
    """lbm_macroscopic for callers that cannot allocate device memory.

    The library keeps the reduction's partial sums in its own fixed device
    array, so no workspace is passed; rho [N], u [3, N] and sums [4] are
    caller-provided float64 CUDA tensors (any may be None) and nothing is
    allocated here.  At most 16,777,216 fluid nodes; concurrent calls that
    overlap on the GPU share the array and race.
    """
    torch = _torch()
    prec = _prec(prec)
    _check_grid(lat, prec, pdf, "pdf", layout)
    # the kernels write N, 3N and 4 doubles through these pointers: check them here
    for name, t, n in (("rho", rho, lat.N), ("u", u, 3 * lat.N), ("sums", sums, 4)):
        if t is None:
            continue
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device != pdf.device:
            raise TypeError(f"{name} must be a CUDA tensor on the device of pdf")
        if t.dtype != torch.float64:
            raise TypeError(f"{name} has dtype {t.dtype}, needs torch.float64")
        if not t.is_contiguous() or t.numel() < n:
            raise ValueError(f"{name} must be contiguous with at least {n} elements")
    check(_lib.load().lbm_macroscopic_noalloc(lat.handle, prec, ctypes.byref(params.c()), _ptr(pdf), layout,
                                              _ptr(_check_s(lat, s)), _ptr(rho), _ptr(u), _ptr(sums),
                                              _stream(stream)), "lbm_macroscopic_noalloc")


def lbm_halo_exchange(part, prec, pointers, mode, stream=None):
    """One ghost exchange of all chunks; ``pointers`` from ``Partitioning.pointers``."""
    torch = _torch()
    if not pointers.is_cuda or pointers.dtype != torch.int64 or pointers.numel() != part.P:
        raise TypeError("pointers must be a CUDA int64 tensor with one address per chunk")
    check(_lib.load().lbm_halo_exchange(part.handle, _prec(prec), _ptr(pointers), int(mode), _stream(stream)),
          "lbm_halo_exchange")


def _host_ptrs(grids):
    arr = (ctypes.c_void_p * len(grids))(*[g.data_ptr() for g in grids])
    return arr


def lbm_partition_run_aa(part, prec, params, grids, pointers, start_parity, steps, s=None, ria=False, stream=None):
    prec = _prec(prec)
    for lat, g in zip(part.parts, grids):
        _check_grid(lat, prec, g, "grid")
    if s is not None:
        _check_s(_Sized(part.N), s)
    check(_lib.load().lbm_partition_run_aa(part.handle, prec, ctypes.byref(params.c()), _host_ptrs(grids),
                                           _ptr(pointers), _ptr(s), int(start_parity), int(steps), 1 if ria else 0,
                                           _stream(stream)), "lbm_partition_run_aa")


def lbm_partition_run_osnt(part, prec, params, grids, pointers, steps, s=None, ria=False, stream=None):
    """grids: 2P grids (set 0 then set 1); pointers: their 2P addresses on the device."""
    prec = _prec(prec)
    for k, g in enumerate(grids):
        _check_grid(part.parts[k % part.P], prec, g, "grid")
    if s is not None:
        _check_s(_Sized(part.N), s)
    check(_lib.load().lbm_partition_run_osnt(part.handle, prec, ctypes.byref(params.c()), _host_ptrs(grids),
                                             _ptr(pointers), _ptr(s), int(steps), 1 if ria else 0, _stream(stream)),
          "lbm_partition_run_osnt")


class _Sized:
    def __init__(self, N):
        self.N = N


def lbm_check_finite(values, stream=None):
    """Raise LbmError(LBM_ERR_NONFINITE) if a float64 CUDA tensor holds NaN or Inf."""
    torch = _torch()
    if not values.is_cuda or values.dtype != torch.float64 or not values.is_contiguous():
        raise TypeError("values must be a contiguous CUDA float64 tensor")
    check(_lib.load().lbm_check_finite(_ptr(values), values.numel(), _stream(stream)), "lbm_check_finite")


def lbm_exact_moments_host(d):
    """Moments of nodes by the FP64 step's integer arithmetic, run on the host.

    d: float64 array [n, 19] (numpy or CPU tensor), direction order of the
    lattice.  Returns a numpy float64 array [n, 22]: drho, jx, jy, jz,
    sa_1..sa_9, da_1..da_9 (pair k holds directions 2k-1 and 2k).
    """
    import numpy as np
    a = np.ascontiguousarray(np.asarray(d, dtype=np.float64))
    if a.ndim != 2 or a.shape[1] != 19:
        raise ValueError("d must have shape [n, 19]")
    out = np.empty((a.shape[0], 22), dtype=np.float64)
    check(_lib.load().lbm_exact_moments_host(a.ctypes.data, a.shape[0], out.ctypes.data), "lbm_exact_moments_host")
    return out


def lbm_fx_pairs_host(d, terms, qm, qp, lp1, general=False):
    """Host image of the FP64 step's fixed-point pair update (``lbm_fx_pairs_host``).

    d: [n, 19] PDFs; terms: [n, 10] (ux, uy, uz, K0, Tx, Ty, Tz, Ox, Oy, Oz).
    Returns (out [n, 19], ok [n]): out[:, 0] is the pair scale es and
    out[:, 1:] the post-collision pair values where ok.  ``general`` takes the
    general conversions everywhere (the same bits as the shorter ones).
    """
    import numpy as np
    a = np.ascontiguousarray(np.asarray(d, dtype=np.float64))
    t = np.ascontiguousarray(np.asarray(terms, dtype=np.float64))
    if a.ndim != 2 or a.shape[1] != 19 or t.shape != (a.shape[0], 10):
        raise ValueError("d must have shape [n, 19] and terms [n, 10]")
    out = np.empty((a.shape[0], 19), dtype=np.float64)
    ok = np.empty(a.shape[0], dtype=np.int32)
    check(_lib.load().lbm_fx_pairs_host(a.ctypes.data, t.ctypes.data, a.shape[0], float(qm), float(qp),
                                        (1 if lp1 else 0) | (2 if general else 0), out.ctypes.data,
                                        ok.ctypes.data), "lbm_fx_pairs_host")
    return out, ok.astype(bool)


def lbm_bandwidth_kernel(kind, dst, src=None, arrays=1, stream=None):
    """One launch of the CNT-kA (kind 0, copy src -> dst with streaming stores) or
    U-kA (kind 1, update dst in place) bandwidth kernel over ``arrays`` equal
    slices of the CUDA tensors (their byte size / arrays each)."""
    nbytes = dst.numel() * dst.element_size()
    per = nbytes // arrays
    check(_lib.load().lbm_bandwidth_kernel(int(kind), _ptr(src), _ptr(dst), per, int(arrays), _stream(stream)),
          "lbm_bandwidth_kernel")


def lbm_fp64_peak_kernel(out, iters, stream=None):
    """One launch of the FP64-pipe throughput kernel over ``out.numel()`` threads
    (8 DFMA chains of ``iters`` steps each); ``out`` a CUDA float64 tensor."""
    torch = _torch()
    if not isinstance(out, torch.Tensor) or not out.is_cuda or out.dtype != torch.float64 or not out.is_contiguous():
        raise TypeError("out must be a contiguous CUDA float64 tensor")
    check(_lib.load().lbm_fp64_peak_kernel(_ptr(out), out.numel(), int(iters), _stream(stream)),
          "lbm_fp64_peak_kernel")


def _adjoint_dtype(prec):
    torch = _torch()
    return torch.float64 if prec in (LBM_F64, LBM_F64_DF) else torch.float32


def new_adjoint(lat, prec, device="cuda"):
    """A zeroed adjoint array [19, Npad] (double for f64, float otherwise)."""
    return _torch().zeros((19, lat.Npad), dtype=_adjoint_dtype(_prec(prec)), device=device)


def _check_adj(lat, prec, t, name):
    if t is None:
        return
    if not t.is_cuda or t.dtype != _adjoint_dtype(prec) or not t.is_contiguous() or t.numel() < 19 * lat.Npad:
        raise TypeError(f"{name} must be a contiguous CUDA {_adjoint_dtype(prec)} tensor [19, Npad]")


def lbm_objective_flux(lat, prec, params, pdf, layout, s=None, lambda_T=None, grad_s=None, stream=None):
    """J (CUDA float64 [1]); optionally fills lambda_T = dJ/dF and grad_s = direct dJ/ds."""
    torch = _torch()
    prec = _prec(prec)
    _check_grid(lat, prec, pdf, "pdf", layout)
    _check_adj(lat, prec, lambda_T, "lambda_T")
    J = torch.empty(1, dtype=torch.float64, device=pdf.device)
    ws_bytes = lat.reduce_workspace_bytes()
    ws = torch.empty(ws_bytes // 8, dtype=torch.float64, device=pdf.device)
    check(_lib.load().lbm_objective_flux(lat.handle, prec, ctypes.byref(params.c()), _ptr(pdf), layout,
                                         _ptr(_check_s(lat, s)), _ptr(J), _ptr(lambda_T), _ptr(grad_s), _ptr(ws),
                                         ws_bytes, _stream(stream)), "lbm_objective_flux")
    return J


def lbm_adjoint_step(lat, prec, params, G_n, lambda_next, lambda_n, s=None, grad_s=None, ria=False, stream=None):
    prec = _prec(prec)
    _check_grid(lat, prec, G_n, "G_n")
    _check_adj(lat, prec, lambda_next, "lambda_next")
    _check_adj(lat, prec, lambda_n, "lambda_n")
    check(_lib.load().lbm_adjoint_step(lat.handle, prec, ctypes.byref(params.c()), _ptr(G_n), _ptr(lambda_next),
                                       _ptr(lambda_n), _ptr(_check_s(lat, s)), _ptr(grad_s), 1 if ria else 0,
                                       _stream(stream)), "lbm_adjoint_step")


def lbm_ckpt_workspace_bytes(lat, prec, T, K) -> int:
    b = ctypes.c_size_t()
    check(_lib.load().lbm_ckpt_workspace_bytes(lat.handle, _prec(prec), int(T), int(K), ctypes.byref(b)),
          "lbm_ckpt_workspace_bytes")
    return b.value


def lbm_flux_forward(lat, prec, params, G0, s, T, K, ws, ria=False, stream=None):
    torch = _torch()
    prec = _prec(prec)
    _check_grid(lat, prec, G0, "G0")
    J = torch.empty(1, dtype=torch.float64, device=G0.device)
    check(_lib.load().lbm_flux_forward(lat.handle, prec, ctypes.byref(params.c()), _ptr(G0), _ptr(_check_s(lat, s)),
                                       int(T), int(K), 1 if ria else 0, _ptr(ws), ws.numel() * ws.element_size(),
                                       _ptr(J), _stream(stream)), "lbm_flux_forward")
    return J


def lbm_flux_backward(lat, prec, params, s, T, K, ws, ria=False, lambda_0=None, stream=None):
    torch = _torch()
    prec = _prec(prec)
    _check_adj(lat, prec, lambda_0, "lambda_0")
    grad = torch.empty(lat.N, dtype=torch.float64, device=ws.device)
    check(_lib.load().lbm_flux_backward(lat.handle, prec, ctypes.byref(params.c()), _ptr(_check_s(lat, s)), int(T),
                                        int(K), 1 if ria else 0, _ptr(ws), ws.numel() * ws.element_size(),
                                        _ptr(grad), _ptr(lambda_0), _stream(stream)), "lbm_flux_backward")
    return grad


_FLUX = None


def _flux_function():
    global _FLUX
    if _FLUX is not None:
        return _FLUX
    torch = _torch()

    class FluxObjective(torch.autograd.Function):
        """J(s) = mean x-momentum after T OS-NT steps from the OS-NT grid G0.

        forward: T steps with a checkpoint every K steps (lbm_flux_forward);
        backward: recompute each K-step segment from its checkpoint and run the
        discrete adjoint back through it (lbm_flux_backward), gradient in FP64.
        """

        @staticmethod
        def forward(ctx, s, lat, prec, params, G0, T, K, ria):
            sf = s.detach().to(torch.float32).contiguous()
            ws = torch.empty((lbm_ckpt_workspace_bytes(lat, prec, T, K) + 7) // 8, dtype=torch.float64,
                             device=G0.device)
            J = lbm_flux_forward(lat, prec, params, G0, sf, T, K, ws, ria)
            ctx.state = (lat, prec, params, sf, T, K, ws, ria)
            ctx.s_dtype = s.dtype
            return J[0]

        @staticmethod
        def backward(ctx, gJ):
            lat, prec, params, sf, T, K, ws, ria = ctx.state
            grad = lbm_flux_backward(lat, prec, params, sf, T, K, ws, ria)
            return (grad * gJ).to(ctx.s_dtype), None, None, None, None, None, None, None

    _FLUX = FluxObjective
    return FluxObjective


def __getattr__(name):
    # torch is imported on first use only; FluxObjective is the autograd Function
    # class (FluxObjective.apply(s, lat, prec, params, G0, T, K, ria)).
    if name == "FluxObjective":
        return _flux_function()
    raise AttributeError(name)


def flux_objective(s, lat, prec, params, G0, T, K, ria=False):
    """Differentiable J(s) (torch autograd through the checkpointed adjoint)."""
    return _flux_function().apply(s, lat, _prec(prec), params, G0, int(T), int(K), bool(ria))


class Solver:
    """A running simulation in one storage form ("osnt", "aa" or "et" = Esoteric Twist) and precision."""

    def __init__(self, lat: Lattice, prec="f64", params: Params | None = None, form="aa", ria=True, s=None,
                 device="cuda"):
        self.lat = lat
        self.prec = _prec(prec)
        self.params = params or Params()
        self.form = form
        self.ria = bool(ria)
        self.s = s
        self.t = 0
        if form == "osnt":
            self.grids = [lat.new_grid(self.prec, device), lat.new_grid(self.prec, device)]
        elif form == "aa":
            self.grids = [lat.new_grid(self.prec, device)]
        elif form == "et":
            if not lat.uploaded & LBM_TABLES_ET:
                raise ValueError("the Esoteric Twist form needs lat.upload(which=... | LBM_TABLES_ET)")
            self.grids = [lat.new_grid(self.prec, device, et=True)]
        else:
            raise ValueError(form)

    @property
    def layout(self):
        if self.form == "osnt":
            return LBM_LAYOUT_OSNT
        if self.form == "et":
            return LBM_LAYOUT_ET_EVEN if self.t % 2 == 0 else LBM_LAYOUT_ET_ODD
        return LBM_LAYOUT_AA_EVEN if self.t % 2 == 0 else LBM_LAYOUT_AA_ODD

    @property
    def pdf(self):
        return self.grids[0]

    def init_equilibrium(self, rho0=1.0, u0=(0.0, 0.0, 0.0), stream=None):
        self.t = 0
        lbm_init_equilibrium(self.lat, self.prec, self.params, self.grids[0], self.layout, rho0, u0, stream)

    def load(self, F, stream=None):
        self.t = 0
        lbm_load_canonical(self.lat, self.prec, self.params, F, self.grids[0], self.layout, stream)

    def step(self, n=1, stream=None):
        if self.form == "osnt":
            for _ in range(n):
                lbm_step_osnt(self.lat, self.prec, self.params, self.grids[0], self.grids[1], self.s, self.ria, stream)
                self.grids.reverse()
                self.t += 1
        elif self.form == "et":
            lbm_run_et(self.lat, self.prec, self.params, self.grids[0], self.t % 2, n, self.s, self.ria, stream)
            self.t += n
        else:
            lbm_run_aa(self.lat, self.prec, self.params, self.grids[0], self.t % 2, n, self.s, self.ria, stream)
            self.t += n

    def step_graph(self, n):
        """Advance n steps (n even) by replaying a CUDA graph of one step pair.

        For small lattices, where a step takes a few microseconds, launch
        overhead dominates; the pair (even + odd AA step, or two OS-NT steps
        ping-ponging the grids) is captured once and replayed n / 2 times on
        the current stream.  The graph is rebuilt when the solver's grids or
        parameters change (call ``reset_graph``).
        """
        torch = _torch()
        if n % 2:
            raise ValueError("step_graph advances an even number of steps")
        if n == 0:
            return
        if self.t % 2:
            raise ValueError("step_graph starts from an even step count")
        if getattr(self, "_graph", None) is None:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):  # the first pair runs directly, outside the capture
                self.step(2)
            torch.cuda.current_stream().wait_stream(side)
            n -= 2
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                st = torch.cuda.current_stream()
                if self.form == "osnt":
                    lbm_step_osnt(self.lat, self.prec, self.params, self.grids[0], self.grids[1], self.s, self.ria, st)
                    lbm_step_osnt(self.lat, self.prec, self.params, self.grids[1], self.grids[0], self.s, self.ria, st)
                elif self.form == "et":
                    lbm_run_et(self.lat, self.prec, self.params, self.grids[0], 0, 2, self.s, self.ria, st)
                else:
                    lbm_step_aa(self.lat, self.prec, self.params, self.grids[0], 0, self.s, self.ria, st)
                    lbm_step_aa(self.lat, self.prec, self.params, self.grids[0], 1, self.s, self.ria, st)
            self._graph = g
        for _ in range(n // 2):
            self._graph.replay()
        self.t += n

    def reset_graph(self):
        self._graph = None

    def canonical(self, stream=None):
        return lbm_canonical_pdfs(self.lat, self.prec, self.params, self.grids[0], self.layout, stream=stream)

    def macroscopic(self, fields=True, sums=True, stream=None):
        return lbm_macroscopic(self.lat, self.prec, self.params, self.grids[0], self.layout, self.s, fields, sums,
                               stream=stream)


__all__ = [
    "Params", "Lattice", "Solver", "LbmError", "lbm_init_equilibrium", "lbm_load_canonical", "lbm_canonical_pdfs",
    "lbm_step_osnt", "lbm_step_aa", "lbm_run_aa", "lbm_macroscopic", "LBM_F64", "LBM_F32", "LBM_F16S", "LBM_F64_DF",
    "LBM_LAYOUT_OSNT", "LBM_LAYOUT_AA_EVEN", "LBM_LAYOUT_AA_ODD", "LBM_TABLES_ADJ", "LBM_TABLES_RIA",
    "LBM_LAYOUT_ET_EVEN", "LBM_LAYOUT_ET_ODD", "LBM_TABLES_ET", "lbm_step_et", "lbm_run_et", "Partitioning",
    "PartitionedSolver", "lbm_halo_exchange", "lbm_partition_run_aa", "lbm_partition_run_osnt",
    "lbm_objective_flux", "lbm_adjoint_step", "lbm_ckpt_workspace_bytes", "lbm_flux_forward", "lbm_flux_backward",
    "flux_objective", "new_adjoint", "lbm_macroscopic_noalloc", "lbm_check_finite", "lbm_bandwidth_kernel", "lbm_fp64_peak_kernel",
    "lbm_exact_moments_host", "lbm_fx_pairs_host",
    "State", "FluxObjective",
]


# The simulation state object (grids, parity, grid swap) under its other name.
State = Solver


class PartitionedSolver:
    """The step on the P chunks of a ``Partitioning``, with a ghost exchange per step (Sect. 6).

    Holds one grid per chunk (two for OS-NT) and their device address tables;
    ``step`` runs ``lbm_partition_run_aa`` / ``lbm_partition_run_osnt``.  The
    state moves between this and a whole-lattice ``Solver`` grid with
    ``load_global`` / ``to_global`` (node slots only; ghost slots are refilled
    by the next exchange).
    """

    def __init__(self, part: Partitioning, prec="f64", params: Params | None = None, form="aa", ria=True, s=None,
                 device="cuda"):
        self.part = part
        self.prec = _prec(prec)
        self.params = params or Params()
        self.form = form
        self.ria = bool(ria)
        self.s = s
        self.t = 0
        if form == "osnt":
            self.sets = [part.new_grids(self.prec, device), part.new_grids(self.prec, device)]
        elif form == "aa":
            self.sets = [part.new_grids(self.prec, device)]
        else:
            raise ValueError(form)
        self._refresh()

    def _refresh(self):
        flat = [g for grids in self.sets for g in grids]
        self._ptrs = Partitioning.pointers(flat)

    @property
    def grids(self):
        """The chunk grids holding the current state."""
        return self.sets[0]

    def init_equilibrium(self, rho0=1.0, u0=(0.0, 0.0, 0.0), stream=None):
        self.t = 0
        layout = LBM_LAYOUT_OSNT if self.form == "osnt" else LBM_LAYOUT_AA_EVEN
        for lat, g in zip(self.part.parts, self.sets[0]):
            lbm_init_equilibrium(lat, self.prec, self.params, g, layout, rho0, u0, stream)

    def load_global(self, grid, t=0):
        """Take the state of a whole-lattice grid (same form and layout) after t steps."""
        if self.form == "aa" and t % 2:
            raise ValueError("load an AA state after an even step count")
        self.t = t
        self.part.scatter(grid, self.sets[0])

    def to_global(self, out=None):
        return self.part.gather(self.sets[0], out)

    def step(self, n=1, stream=None):
        P = self.part.P
        if self.form == "osnt":
            lbm_partition_run_osnt(self.part, self.prec, self.params, self.sets[0] + self.sets[1], self._ptrs, n,
                                   self.s, self.ria, stream)
            if n % 2:
                self.sets.reverse()
                self._refresh()
        else:
            lbm_partition_run_aa(self.part, self.prec, self.params, self.sets[0], self._ptrs[:P], self.t % 2, n,
                                 self.s, self.ria, stream)
        self.t += n
