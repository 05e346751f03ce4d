"""What the pattern-specific bandwidth kernels write (Sect. 5.2, Table 3).

CNT-kA copies k arrays with streaming stores and U-kA updates k arrays in
place; their GB/s figures are the roofline denominators P = b / B_l.  The
FP64 throughput kernel (the compute roof of the native FP64 step) is checked
the same way: its chains count exactly.  A kernel
that skipped part of its work would only look faster, so these tests read back
every byte: after CNT-kA each of the k destination arrays equals its source
bit for bit; after U-kA every float of the k arrays has grown by exactly 1
(the update adds 1.0f per element, exact for the small integers used here);
and the bytes after the k arrays are untouched in both cases.  Sizes: ragged
arrays (not a multiple of the grid-stride step) and the FP64 grid of the
256^3 bed (19 arrays of Npad = 10,897,024 doubles).
"""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu

import paper_1410_0412_gb300 as lbm
from paper_1410_0412_gb300 import _lib

BED_NPAD = (10_896_954 + 127) // 128 * 128


def _launch(kind, src, dst, bytes_per_array, arrays):
    rc = _lib.load().lbm_bandwidth_kernel(kind, ctypes.c_void_p(src.data_ptr() if src is not None else 0),
                                          ctypes.c_void_p(dst.data_ptr()), ctypes.c_int64(bytes_per_array),
                                          arrays, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, _lib.load().lbm_last_error()


@pytest.mark.parametrize("arrays,bytes_per_array", [(1, 16), (1, 16 * 1001), (19, 16 * 12_345),
                                                    (19, 8 * BED_NPAD)])
def test_cnt_copies_every_array_and_nothing_else(arrays, bytes_per_array):
    n = arrays * bytes_per_array // 4
    guard = 4096
    g = torch.Generator(device="cuda").manual_seed(arrays)
    src = torch.randint(-2 ** 31, 2 ** 31 - 1, (n + guard,), dtype=torch.int32, device="cuda", generator=g)
    dst = torch.full((n + guard,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    _launch(0, src, dst, bytes_per_array, arrays)
    torch.cuda.synchronize()
    assert torch.equal(dst[:n], src[:n])
    assert bool((dst[n:] == 0x5A5A5A5A).all())


@pytest.mark.parametrize("arrays,bytes_per_array", [(1, 16), (1, 16 * 1001), (19, 16 * 12_345),
                                                    (19, 8 * BED_NPAD)])
def test_update_adds_one_to_every_element_of_every_array(arrays, bytes_per_array):
    n = arrays * bytes_per_array // 4
    guard = 4096
    g = torch.Generator(device="cuda").manual_seed(100 + arrays)
    base = torch.randint(-1000, 1000, (n + guard,), device="cuda", generator=g).to(torch.float32)
    buf = base.clone()
    for rep in (1, 2):  # two launches in a row: +1 each
        _launch(1, None, buf, bytes_per_array, arrays)
        torch.cuda.synchronize()
        assert torch.equal(buf[:n], base[:n] + rep)
        assert torch.equal(buf[n:], base[n:])


def test_bandwidth_kernel_rejects_bad_sizes():
    buf = torch.empty(64, dtype=torch.float32, device="cuda")
    for kind, per, arrays in ((2, 16, 1), (0, 8, 1), (1, 24, 1), (1, 16, 0)):
        rc = _lib.load().lbm_bandwidth_kernel(kind, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                                              ctypes.c_int64(per), arrays, ctypes.c_void_p(0))
        assert rc == _lib.LBM_ERR_ARG


def test_fp64_peak_kernel_counts_every_fma():
    """The FP64 throughput kernel: 8 chains of x <- fma(x, 1, 1) per thread, so
    each thread's output is 8 (t mod 1024) + 28 + 8 iters, exactly."""
    threads, iters = 152 * 256 * 2, 1000
    out = torch.full((threads,), float("nan"), dtype=torch.float64, device="cuda")
    lbm.lbm_fp64_peak_kernel(out, iters)
    torch.cuda.synchronize()
    t = torch.arange(threads, device="cuda", dtype=torch.float64)
    assert torch.equal(out, 8 * torch.remainder(t, 1024) + 28 + 8 * iters)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_fp64_peak_kernel(out[:100], iters)
