"""The Python binding refuses tensors the C ABI cannot check (host logic; no GPU needed).

The library receives only pointers and sizes, so a wrong dtype, a transposed or strided view,
a wrong shape or a tensor on another device would be read out of bounds by the kernels.  The
wrappers check every tensor and raise ValueError before anything is launched.
"""
import types

import pytest
import torch

from paper_2004_08962_gb300 import hicu


def _fake_handle():
    # the checks run before the handle is used; this stands in for one on cuda:0
    h = types.SimpleNamespace(ptr=None, device=torch.device("cuda", 0))
    h._dev = lambda *ts: hicu.Handle._dev(h, *ts)
    return h


GEOM = hicu.make_geom((16, 12, 1), 2, (3, 3, 1))
REG = hicu.make_region((0, 0, 0), (16, 12, 1))


def test_wrong_dtype_shape_layout_and_device_are_refused():
    h = _fake_handle()
    x_ok = torch.zeros((2, 1, 12, 16), dtype=torch.complex64)
    f_ok = torch.zeros((4, 18), dtype=torch.complex64)
    with pytest.raises(ValueError, match="complex64"):
        hicu.hicu_conv_null(h, GEOM, REG, x_ok.to(torch.complex128), f_ok)
    with pytest.raises(ValueError, match="shape"):
        hicu.hicu_conv_null(h, GEOM, REG, torch.zeros((2, 1, 16, 12), dtype=torch.complex64), f_ok)
    with pytest.raises(ValueError, match="contiguous"):
        hicu.hicu_conv_null(h, GEOM, REG, torch.zeros((2, 1, 16, 12), dtype=torch.complex64).transpose(2, 3),
                            f_ok)
    with pytest.raises(ValueError, match="shape"):
        hicu.hicu_conv_null(h, GEOM, REG, x_ok, torch.zeros((4, 17), dtype=torch.complex64))
    with pytest.raises(ValueError, match="CUDA"):
        hicu.hicu_conv_null(h, GEOM, REG, x_ok, f_ok)
    with pytest.raises(ValueError, match="uint8"):
        hicu.hicu_gd_step_filters(h, GEOM, REG, x_ok, torch.zeros((1, 12, 16), dtype=torch.bool), f_ok)
    with pytest.raises(ValueError, match="shape"):
        hicu.hicu_conv_null_adjoint(h, GEOM, REG, torch.zeros((1, 10, 14, 3), dtype=torch.complex64), f_ok)
    with pytest.raises(ValueError, match="complex128"):
        hicu.hicu_nullspace(h, torch.zeros((18, 18), dtype=torch.complex64), 4)
    with pytest.raises(ValueError, match="shape"):
        hicu.hicu_reconstruct(h, GEOM, torch.zeros((2, 1, 12, 15), dtype=torch.complex64),
                              torch.zeros((1, 12, 16), dtype=torch.uint8), None)
    with pytest.raises(ValueError, match="complex64"):
        hicu.hicu_conv_null_noalloc(GEOM, REG, x_ok.real.contiguous(), f_ok)
