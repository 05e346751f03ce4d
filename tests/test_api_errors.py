"""Argument checks of the partition, exchange and Esoteric Twist entry points (CPU).

Every refusal below happens before any device work, so no GPU is needed: the
call must return the stated status code and leave a message in
lbm_last_error().
"""
import ctypes

import numpy as np
import pytest

import geometry
import paper_1410_0412_gb300 as lbm

L = lbm._lib
ARG, UNSUP = L.LBM_ERR_ARG, L.LBM_ERR_UNSUPPORTED


@pytest.fixture(scope="module")
def lat():
    return lbm.Lattice(geometry.random_voxels(9, 8, 7, 0.2, 7), periodic=(1, 0, 0))


def _msg():
    return L.load().lbm_last_error().decode()


def test_partition_entry_points(lat):
    lib = L.load()
    out = ctypes.c_void_p()
    assert lib.lbm_partition_build(None, 2, ctypes.byref(out)) == ARG
    assert lib.lbm_partition_build(lat.handle, 2, None) == ARG
    part = lbm.Partitioning(lat, 3)
    n = ctypes.c_int64()
    assert lib.lbm_partition_info(part.handle, 3, None, ctypes.byref(n), None, None) == ARG
    assert lib.lbm_partition_info(part.handle, -1, None, None, None, None) == ARG
    assert "out of range" in _msg()
    loc = ctypes.c_void_p()
    assert lib.lbm_partition_local(part.handle, 0, None) == ARG
    assert lib.lbm_partition_local(part.handle, 5, ctypes.byref(loc)) == ARG
    assert lib.lbm_partition_validate(part.handle, None) == ARG
    nb = ctypes.c_size_t()
    assert lib.lbm_halo_table_bytes(part.handle, None) == ARG
    assert lib.lbm_halo_table_bytes(part.handle, ctypes.byref(nb)) == L.LBM_OK and nb.value > 0
    # upload refuses a NULL or misaligned buffer before touching it
    assert lib.lbm_halo_upload(part.handle, None, nb.value, None) == ARG
    assert lib.lbm_halo_upload(part.handle, ctypes.c_void_p(4096 + 8), nb.value, None) == ARG
    assert lib.lbm_halo_upload(part.handle, ctypes.c_void_p(4096), 16, None) == ARG
    # exchange and runs refuse to start without the table on the device
    prm = lbm.Params().c()
    assert lib.lbm_halo_exchange(part.handle, 0, ctypes.c_void_p(4096), 0, None) == ARG
    assert "not uploaded" in _msg()
    ptrs = (ctypes.c_void_p * 6)(*([4096] * 6))
    assert lib.lbm_partition_run_aa(part.handle, 0, ctypes.byref(prm), ptrs, ctypes.c_void_p(4096), None, 0, 2,
                                    1, None) == ARG
    assert lib.lbm_partition_run_aa(part.handle, 0, ctypes.byref(prm), ptrs, ctypes.c_void_p(4096), None, 2, 2,
                                    1, None) == ARG
    assert lib.lbm_partition_run_osnt(part.handle, 0, ctypes.byref(prm), ptrs, None, None, 2, 1, None) == ARG
    assert lib.lbm_partition_run_osnt(part.handle, 0, ctypes.byref(prm), ptrs, ctypes.c_void_p(4096), None, -1,
                                      1, None) == ARG


def test_exchange_mode_and_precision_checks(lat):
    lib = L.load()
    part = lbm.Partitioning(lat, 2)
    # a fake "uploaded" state cannot be made from Python, so check the order of the checks:
    # a NULL handle and bad modes are reported as argument errors
    assert lib.lbm_halo_exchange(None, 0, ctypes.c_void_p(4096), 0, None) == ARG
    assert lib.lbm_halo_exchange(part.handle, 0, ctypes.c_void_p(4096), 7, None) == ARG


def test_et_entry_points(lat):
    lib = L.load()
    prm = lbm.Params().c()
    S = ctypes.c_int64()
    assert lib.lbm_et_info(None, ctypes.byref(S), None, None) == ARG
    assert lib.lbm_et_info(lat.handle, ctypes.byref(S), None, None) == L.LBM_OK and S.value >= lat.N
    assert lib.lbm_export_et_tables(None, None, None) == ARG
    R = ctypes.c_int64()
    assert lib.lbm_export_et_runs(lat.handle, ctypes.byref(R), None, None, None) == L.LBM_OK and R.value >= 1
    for parity, steps in ((2, 1), (0, -1)):
        assert lib.lbm_run_et(lat.handle, 0, ctypes.byref(prm), ctypes.c_void_p(4096), parity, steps, None, 0,
                              None) == ARG
    assert lib.lbm_run_et(lat.handle, 0, ctypes.byref(prm), None, 0, 1, None, 0, None) == ARG
    bad = lbm.Params(omega_plus=2.5).c()
    assert lib.lbm_step_et(lat.handle, 0, ctypes.byref(bad), ctypes.c_void_p(4096), 0, None, 0, None) == ARG
    assert "omega_plus" in _msg()
    # layouts beyond ET_ODD are unknown everywhere a layout is taken
    assert lib.lbm_init_equilibrium(lat.handle, 0, ctypes.byref(prm), ctypes.c_void_p(4096), 5, ctypes.c_double(1.0),
                                    (ctypes.c_double * 3)(0, 0, 0), None) == ARG
    # the ET table selection bit is accepted by the size query, unknown bits are not
    nb = ctypes.c_size_t()
    assert lib.lbm_device_table_bytes(lat.handle, L.LBM_TABLES_ET, ctypes.byref(nb)) == L.LBM_OK
    assert lib.lbm_device_table_bytes(lat.handle, 8, ctypes.byref(nb)) == ARG
