"""The allocation-free convolution entry point (static device scratch) against the handle path.

hicu_conv_null_noalloc serves callers that cannot allocate device memory when they
call it (their framework already holds the free memory, or they cannot accept the
synchronisation an allocation may cause).  It must give the same R and ||R||^2 as
hicu_conv_null, on consecutive calls that reuse its shared static scratch.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

CASES = [
    # dims, coils, kernel, region offset, region extent, p
    ((64, 64, 1), 4, (5, 5, 1), (0, 0, 0), (64, 64, 1), 4),
    ((70, 45, 1), 3, (5, 3, 1), (3, 2, 0), (61, 40, 1), 20),
]


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_conv_null_noalloc_matches_handle_path_twice():
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from paper_2004_08962_gb300 import build, hicu
    build.build()
    L = hicu.lib()
    h = hicu.Handle()
    stream = torch.cuda.current_stream()
    for i, (dims, C, ker, off, ext, p) in enumerate(CASES):
        rng = np.random.default_rng(100 + i)
        n = C * ker[0] * ker[1] * ker[2]
        x = (rng.standard_normal((C, dims[2], dims[1], dims[0]))
             + 1j * rng.standard_normal((C, dims[2], dims[1], dims[0]))).astype(np.complex64)
        f = (rng.standard_normal((p, n)) + 1j * rng.standard_normal((p, n))).astype(np.complex64)
        xt, ft = torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda()
        geom = hicu.make_geom(dims, C, ker)
        reg = hicu.make_region(off, ext)
        R_ref, obj_ref = hicu.hicu_conv_null(h, geom, reg, xt, ft, want_objective=True)
        R = torch.full(hicu.out_shape(geom, reg) + (p,), float("nan"), dtype=torch.complex64,
                       device="cuda")
        obj = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = L.hicu_conv_null_noalloc(ctypes.byref(geom), ctypes.byref(reg),
                                      ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(ft.data_ptr()),
                                      p, ctypes.c_void_p(R.data_ptr()),
                                      ctypes.c_void_p(obj.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        assert _rel(R.cpu().numpy(), R_ref.cpu().numpy()) < 5e-6
        assert abs(obj.item() - obj_ref.item()) <= 1e-5 * obj_ref.item()
    # a request beyond the static scratch is refused, not truncated
    geom = hicu.make_geom((64, 64, 1), 64, (9, 9, 1))
    reg = hicu.make_region((0, 0, 0), (64, 64, 1))
    big_p = 64
    xt = torch.zeros((64, 1, 64, 64), dtype=torch.complex64, device="cuda")
    ft = torch.zeros((big_p, 64 * 81), dtype=torch.complex64, device="cuda")
    with pytest.raises(hicu.HicuError) as e:
        hicu.hicu_conv_null_noalloc(geom, reg, xt, ft)
    assert e.value.status == 8
    h.close()
