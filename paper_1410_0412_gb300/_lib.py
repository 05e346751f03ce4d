"""ctypes declarations of liblbm's C ABI (include/lbm.h).

Loading fails loudly when the library has not been built: there is no
fallback implementation of any entry point.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK = 0
LBM_ERR_ARG = 1
LBM_ERR_ALLOC = 2
LBM_ERR_CUDA = 3
LBM_ERR_TABLE = 4
LBM_ERR_UNSUPPORTED = 5
LBM_ERR_NONFINITE = 6

LBM_ENUM_LEX = 0
LBM_ENUM_HILBERT = 1
LBM_F64 = 0
LBM_F32 = 1
LBM_F16S = 2
LBM_F64_DF = 3
LBM_LAYOUT_OSNT = 0
LBM_LAYOUT_AA_EVEN = 1
LBM_LAYOUT_AA_ODD = 2
LBM_LAYOUT_ET_EVEN = 3
LBM_LAYOUT_ET_ODD = 4
LBM_TABLES_ADJ = 1
LBM_TABLES_RIA = 2
LBM_TABLES_ET = 4
LBM_HALO_OSNT = 0
LBM_HALO_AA_GATHER = 1
LBM_HALO_AA_SCATTER = 2

_ERRNAMES = {1: "LBM_ERR_ARG", 2: "LBM_ERR_ALLOC", 3: "LBM_ERR_CUDA", 4: "LBM_ERR_TABLE",
             5: "LBM_ERR_UNSUPPORTED", 6: "LBM_ERR_NONFINITE"}


class LbmError(RuntimeError):
    def __init__(self, code: int, fn: str, msg: str):
        super().__init__(f"{fn} failed with {_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class lbm_bc(ctypes.Structure):
    _fields_ = [("periodic", ctypes.c_int * 3), ("x_pressure", ctypes.c_int)]


class lbm_params(ctypes.Structure):
    _fields_ = [("omega_plus", ctypes.c_double), ("magic", ctypes.c_double), ("g", ctypes.c_double * 3),
                ("rho0", ctypes.c_double), ("rho_in", ctypes.c_double), ("rho_out", ctypes.c_double),
                ("shifted", ctypes.c_int), ("f16_scale", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PSZ = ctypes.POINTER(ctypes.c_size_t)
_PD = ctypes.POINTER(ctypes.c_double)

# name -> argument types (all return int unless listed in _RESTYPES)
SIGNATURES = {
    "lbm_last_error": [],
    "lbm_build_lattice": [_P, _I, _I, _I, ctypes.POINTER(lbm_bc), _I, _I, ctypes.POINTER(_P)],
    "lbm_lattice_from_adjacency": [_I64, _P, _P, ctypes.POINTER(_P)],
    "lbm_build_lattice_ordered": [_P, _I, _I, _I, ctypes.POINTER(lbm_bc), _P, _I64, ctypes.POINTER(_P)],
    "lbm_renumber_partitions": [_P, _I, _P],
    "lbm_partition_ghosts": [_P, _I, _P],
    "lbm_free_lattice": [_P],
    "lbm_partition_build": [_P, _I, ctypes.POINTER(_P)],
    "lbm_free_partitioning": [_P],
    "lbm_partition_info": [_P, _I, _PI64, _PI64, _PI64, _PI64],
    "lbm_partition_local": [_P, _I, ctypes.POINTER(_P)],
    "lbm_partition_export_ghosts": [_P, _I, _P, _P, _P, _P],
    "lbm_partition_validate": [_P, _P],
    "lbm_halo_table_bytes": [_P, _PSZ],
    "lbm_halo_upload": [_P, _P, _SZ, _P],
    "lbm_halo_exchange": [_P, _I, _P, _I, _P],
    "lbm_partition_run_aa": [_P, _I, ctypes.POINTER(lbm_params), _P, _P, _P, _I, _I, _I, _P],
    "lbm_partition_run_osnt": [_P, _I, ctypes.POINTER(lbm_params), _P, _P, _P, _I, _I, _P],
    "lbm_lattice_info": [_P, _PI64, _PI64, _PI64, _PI64],
    "lbm_export_tables": [_P, _P, _P, _P, _P],
    "lbm_validate_tables": [_P],
    "lbm_export_adjacency_rows": [_P, _P, _I64, _P],
    "lbm_check_finite": [_P, _I64, _P],
    "lbm_exact_moments_host": [_P, _I64, _P],
    "lbm_fx_pairs_host": [_P, _P, _I64, ctypes.c_double, ctypes.c_double, _I, _P, _P],
    "lbm_device_table_bytes": [_P, _I, _PSZ],
    "lbm_lattice_upload": [_P, _I, _P, _SZ, _P],
    "lbm_pdf_bytes": [_P, _I, _PSZ],
    "lbm_init_equilibrium": [_P, _I, ctypes.POINTER(lbm_params), _P, _I, ctypes.c_double, _PD, _P],
    "lbm_load_canonical": [_P, _I, ctypes.POINTER(lbm_params), _P, _P, _I, _P],
    "lbm_canonical_pdfs": [_P, _I, ctypes.POINTER(lbm_params), _P, _I, _P, _P],
    "lbm_step_osnt": [_P, _I, ctypes.POINTER(lbm_params), _P, _P, _P, _I, _P],
    "lbm_step_aa": [_P, _I, ctypes.POINTER(lbm_params), _P, _I, _P, _I, _P],
    "lbm_run_aa": [_P, _I, ctypes.POINTER(lbm_params), _P, _I, _I, _P, _I, _P],
    "lbm_et_info": [_P, _PI64, _PI64, _P],
    "lbm_export_et_tables": [_P, _P, _P],
    "lbm_step_et": [_P, _I, ctypes.POINTER(lbm_params), _P, _I, _P, _I, _P],
    "lbm_run_et": [_P, _I, ctypes.POINTER(lbm_params), _P, _I, _I, _P, _I, _P],
    "lbm_export_et_runs": [_P, _PI64, _P, _P, _P],
    "lbm_export_run_slots": [_P, _I, _P, ctypes.POINTER(ctypes.c_int)],
    "lbm_reduce_workspace_bytes": [_P, _PSZ],
    "lbm_macroscopic": [_P, _I, ctypes.POINTER(lbm_params), _P, _I, _P, _P, _P, _P, _P, _SZ, _P],
    "lbm_bandwidth_kernel": [_I, _P, _P, _I64, _I, _P],
    "lbm_fp64_peak_kernel": [_P, _I64, _I, _P],
    "lbm_macroscopic_noalloc": [_P, _I, ctypes.POINTER(lbm_params), _P, _I, _P, _P, _P, _P, _P],
    "lbm_objective_flux": [_P, _I, ctypes.POINTER(lbm_params), _P, _I, _P, _P, _P, _P, _P, _SZ, _P],
    "lbm_adjoint_step": [_P, _I, ctypes.POINTER(lbm_params), _P, _P, _P, _P, _P, _I, _P],
    "lbm_ckpt_workspace_bytes": [_P, _I, _I, _I, _PSZ],
    "lbm_flux_forward": [_P, _I, ctypes.POINTER(lbm_params), _P, _P, _I, _I, _I, _P, _SZ, _P, _P],
    "lbm_flux_backward": [_P, _I, ctypes.POINTER(lbm_params), _P, _I, _I, _I, _P, _SZ, _P, _P, _P],
}
_RESTYPES = {"lbm_last_error": ctypes.c_char_p, "lbm_free_lattice": None, "lbm_free_partitioning": None}

_lib = None


def load() -> ctypes.CDLL:
    """The loaded library; raises if liblbm.so is missing (never falls back)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"liblbm.so not found at {LIB_PATH}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()'). There is no non-CUDA fallback.")
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _RESTYPES.get(name, ctypes.c_int)
    _lib = lib
    return lib


def check(rc: int, fn: str):
    if rc != LBM_OK:
        msg = load().lbm_last_error()
        raise LbmError(rc, fn, msg.decode() if msg else "")
