"""The allocation-free convolution entry point (static device scratch) against the handle path.

hicu_conv_null_noalloc serves callers that cannot allocate device memory when they
call it (their framework already holds the free memory, or they cannot accept the
synchronisation an allocation may cause).  It must give the same R and ||R||^2 as
hicu_conv_null, on consecutive calls that reuse its shared static scratch: a small call
followed by a larger one and a larger one followed by a smaller one (the old contents
stay in the array beyond the new layout), the objective-only call (R = NULL), a halo tile
above 48 KB of shared memory, and refusals (not truncation) beyond each documented limit.
"""
import ctypes

import numpy as np
import pytest
import torch

from closeness import assert_close

pytestmark = pytest.mark.gpu

CASES = [
    # dims, coils, kernel, region offset, region extent, p
    ((64, 64, 1), 4, (5, 5, 1), (0, 0, 0), (64, 64, 1), 4),
    ((70, 45, 1), 3, (5, 3, 1), (3, 2, 0), (61, 40, 1), 20),
    ((40, 33, 1), 2, (3, 3, 1), (1, 0, 0), (37, 33, 1), 3),
    # 11 x 11 x 11 kernel: halo tile 8 * 11 * 14 * 42 = 51744 bytes (> 48 KB)
    ((16, 16, 14), 1, (11, 11, 11), (0, 0, 0), (16, 16, 14), 2),
]


def _noalloc(L, geom, reg, xt, ft, p, R, obj, stream):
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    return L.hicu_conv_null_noalloc(ctypes.byref(geom), ctypes.byref(reg), ptr(xt), ptr(ft), p, ptr(R), ptr(obj),
                                    ctypes.c_void_p(stream.cuda_stream))


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
        for _ in range(2):   # two calls in a row on the shared scratch
            R = torch.full(hicu.out_shape(geom, reg) + (p,), float("nan"), dtype=torch.complex64,
                           device="cuda")
            obj = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            assert _noalloc(L, geom, reg, xt, ft, p, R, obj, stream) == 0
            torch.cuda.synchronize()
            assert_close(R.cpu().numpy(), R_ref.cpu().numpy(), 5e-6, f"case {i} R")
            assert abs(obj.item() - obj_ref.item()) <= 1e-5 * obj_ref.item()
        # objective only (R = NULL)
        obj = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(L, geom, reg, xt, ft, p, None, obj, stream) == 0
        torch.cuda.synchronize()
        assert abs(obj.item() - obj_ref.item()) <= 1e-5 * obj_ref.item()

    # requests beyond the static scratch or the shared memory are refused, not truncated
    refused = [
        # filter re-layout: n * roundup(p, 16) = 5184 * 64 > HICU_NOALLOC_MAX_FILTER_WORDS
        ((64, 64, 1), 64, (9, 9, 1), 64),
        # convolution CTAs: ceil(64/32) * ceil(4096/4) * 40 = 81920 > HICU_NOALLOC_MAX_PARTIALS
        ((64, 4096, 40), 1, (1, 1, 1), 1),
        # halo tile: 8 * 14 * (64 + 3) * (1 + 31) = 240128 bytes > the 227 KB per-block maximum
        ((8, 64, 16), 1, (1, 64, 14), 1),
    ]
    for dims, C, ker, p in refused:
        geom = hicu.make_geom(dims, C, ker)
        reg = hicu.make_region((0, 0, 0), dims)
        n = C * ker[0] * ker[1] * ker[2]
        xt = torch.zeros((C, dims[2], dims[1], dims[0]), dtype=torch.complex64, device="cuda")
        ft = torch.zeros((p, n), dtype=torch.complex64, device="cuda")
        obj = torch.zeros((1,), dtype=torch.float64, device="cuda")
        assert _noalloc(L, geom, reg, xt, ft, p, None, obj, stream) == 8, (dims, ker)
    torch.cuda.synchronize()
    h.close()
