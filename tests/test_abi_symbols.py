"""The C-ABI library loads without a GPU and exports every entry point of include/lbm.h."""
import ctypes
import os
import re

import paper_1410_0412_gb300 as lbm
from paper_1410_0412_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    return re.findall(r"LBM_API\s+(?:const\s+)?\w+\s*\*?\s*(lbm_\w+)\s*\(", src)


def test_header_declares_the_boundary():
    names = declared()
    for n in ["lbm_build_lattice", "lbm_step_osnt", "lbm_step_aa", "lbm_macroscopic", "lbm_adjoint_step",
              "lbm_export_tables", "lbm_lattice_upload", "lbm_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert sorted(declared()) == sorted(_lib.SIGNATURES)


def test_no_other_symbols_exported():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    funcs = [l.split()[-1] for l in out.splitlines() if " T " in l]
    assert sorted(funcs) == sorted(declared())


def test_host_only_calls_work_without_gpu():
    import numpy as np
    lat = lbm.Lattice(np.zeros((3, 3, 3), np.uint8), periodic=(1, 1, 1))
    assert lat.N == 27 and lat.R >= 1
    assert lat.pdf_bytes("f64") == 19 * lat.Npad * 8
    assert lat.device_table_bytes() > 0
    assert lbm.lbm_ckpt_workspace_bytes(lat, "f32", 100, 10) > 0
    msg = _lib.load().lbm_last_error()
    assert isinstance(msg, bytes)
