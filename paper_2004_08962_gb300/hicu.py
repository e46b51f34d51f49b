"""Thin ctypes binding of libhicu (include/hicu.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are torch CUDA tensors (device memory and streams come from
PyTorch); complex64 k-space has shape (C, Nz, Ny, Nx).  Function names match
the C entry points.  If the shared library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int32, c_int64, c_uint8, c_uint64, c_void_p
from typing import Optional, Sequence

import torch

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhicu.so")

HICU_FP32, HICU_SPLIT_BF16 = 0, 1
HICU_JL_NULLSPACE, HICU_JL_PROJECTOR, HICU_JL_COMPLEMENT = 0, 1, 2

EXPORTED = (
    "hicu_create", "hicu_destroy", "hicu_last_error", "hicu_status_string", "hicu_check",
    "hicu_filter_length", "hicu_num_outputs", "hicu_gram", "hicu_nullspace", "hicu_nullspace_info",
    "hicu_principal_subspace",
    "hicu_jl_compress",
    "hicu_conv_null", "hicu_conv_null_adjoint", "hicu_gd_step_filters", "hicu_gd_step",
    "hicu_reconstruct", "hicu_profile_select", "hicu_profile_read", "hicu_conv_null_noalloc",
    "hicu_profile_eig_sweeps", "hicu_batch_order", "hicu_reconstruct_batched",
    "hicu_conv_null_filter_grad", "hicu_project_unobserved",
    "hicu_support_length", "hicu_gram_support", "hicu_expand_filters",
    "hicu_gd_step_soft", "hicu_soft_threshold", "hicu_principal_rsvd",
)

HICU_K_GRAM, HICU_K_EIG, HICU_K_CONV, HICU_K_ADJOINT, HICU_K_JL, HICU_K_MISC = 0, 1, 2, 3, 4, 5
HICU_K_CONV_TC, HICU_K_ADJOINT_TC, HICU_K_TRIDIAG = 6, 7, 8


class hicu_geom(ctypes.Structure):
    _fields_ = [("dim", c_int64 * 3), ("ncoil", c_int32), ("k", c_int32 * 3),
                ("circular", c_uint8 * 3), ("mask_per_coil", c_uint8)]


class hicu_region(ctypes.Structure):
    _fields_ = [("off", c_int64 * 3), ("ext", c_int64 * 3)]


class hicu_stage(ctypes.Structure):
    _fields_ = [("region", hicu_region), ("iters", c_int32), ("gd_steps", c_int32), ("p", c_int32)]


class hicu_params(ctypes.Structure):
    _fields_ = [("rank", c_int64), ("nstages", c_int32), ("stages", POINTER(hicu_stage)),
                ("seed", c_uint64), ("jl", c_int32), ("prec", c_int32),
                ("gram_on_current", c_int32), ("init", c_int32), ("eig_solver", c_int32),
                ("kernel_mask", c_void_p), ("dc_weight", c_double), ("l1_threshold", c_double),
                ("jl_exact", c_int32), ("qplus", c_void_p), ("qplus_cols", c_int32), ("qplus_blocks", c_int32),
                ("rsvd_cols", c_int32), ("rsvd_seed", c_uint64)]


class hicu_log(ctypes.Structure):
    _fields_ = [("J", POINTER(c_double)), ("objective", POINTER(c_double)), ("eta", POINTER(c_double))]


class hicu_problem(ctypes.Structure):
    _fields_ = [("geom", hicu_geom), ("x0", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("params", hicu_params), ("x_out", ctypes.c_void_p), ("log", POINTER(hicu_log))]


class hicu_slice_report(ctypes.Structure):
    _fields_ = [("start_ms", c_double), ("end_ms", c_double), ("lane", c_int32), ("status", c_int32),
                ("gd_steps", c_int64)]


class HicuError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


_LIB = None


def lib() -> ctypes.CDLL:
    """Load libhicu.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build it with "
                               "`python -m paper_2004_08962_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        P = c_void_p
        G, R = POINTER(hicu_geom), POINTER(hicu_region)
        sig = {
            "hicu_create": ([POINTER(P)], c_int32),
            "hicu_destroy": ([P], c_int32),
            "hicu_last_error": ([P], ctypes.c_char_p),
            "hicu_status_string": ([c_int32], ctypes.c_char_p),
            "hicu_check": ([P, P], c_int32),
            "hicu_filter_length": ([G], c_int64),
            "hicu_num_outputs": ([G, R], c_int64),
            "hicu_gram": ([P, G, R, P, P, P], c_int32),
            "hicu_nullspace": ([P, c_int64, c_int64, P, P, P, c_int32, P], c_int32),
            "hicu_nullspace_info": ([P, POINTER(c_int32), POINTER(c_int32)], c_int32),
            "hicu_principal_subspace": ([P, c_int64, c_int64, P, P, P, P, P, P], c_int32),
            "hicu_jl_compress": ([P, c_int64, c_int64, c_int32, P, c_int32, P, c_uint64, c_uint64, P, P],
                                 c_int32),
            "hicu_conv_null": ([P, G, R, P, P, c_int32, P, P, c_int32, P], c_int32),
            "hicu_conv_null_adjoint": ([P, G, R, P, P, c_int32, P, P, P, c_int32, P], c_int32),
            "hicu_gd_step_filters": ([P, G, R, P, P, P, c_int32, P, c_int32, P], c_int32),
            "hicu_gd_step": ([P, G, R, P, P, P, c_int64, c_int32, c_int32, c_uint64, c_uint64, P, P,
                              c_int32, P], c_int32),
            "hicu_reconstruct": ([P, G, P, P, POINTER(hicu_params), P, POINTER(hicu_log), P], c_int32),
            "hicu_profile_select": ([P, c_int32], c_int32),
            "hicu_conv_null_noalloc": ([G, R, P, P, c_int32, P, P, P], c_int32),
            "hicu_profile_eig_sweeps": ([P, POINTER(c_int64)], c_int32),
            "hicu_profile_read": ([P, POINTER(c_double), POINTER(c_int64), POINTER(c_int64)], c_int32),
            "hicu_batch_order": ([c_int32, P, POINTER(c_int32), POINTER(c_double)], c_int32),
            "hicu_conv_null_filter_grad": ([P, G, R, P, P, c_int32, P, P], c_int32),
            "hicu_project_unobserved": ([P, G, R, P, P, P, P], c_int32),
            "hicu_reconstruct_batched": ([P, c_int32, P, c_int32, P, P], c_int32),
            "hicu_support_length": ([G, P], c_int64),
            "hicu_gram_support": ([P, G, R, P, P, P, P], c_int32),
            "hicu_expand_filters": ([P, G, P, P, c_int32, P, P], c_int32),
            "hicu_gd_step_soft": ([P, G, R, P, P, P, c_double, P, c_int32, P, c_int32, P], c_int32),
            "hicu_soft_threshold": ([P, G, P, c_double, P], c_int32),
            "hicu_principal_rsvd": ([P, G, R, P, P, c_int64, c_int64, P, c_int64, c_uint64, c_uint64, P, P, P, P],
                                    c_int32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _LIB = L
    return _LIB


# ----------------------------------------------------------------- helpers

def make_geom(dims: Sequence[int], ncoil: int, kernel: Sequence[int], circular=(0, 0, 0),
              mask_per_coil: bool = False) -> hicu_geom:
    g = hicu_geom()
    for a in range(3):
        g.dim[a] = int(dims[a])
        g.k[a] = int(kernel[a])
        g.circular[a] = int(circular[a])
    g.ncoil = int(ncoil)
    g.mask_per_coil = 1 if mask_per_coil else 0
    return g


def make_region(off: Sequence[int], ext: Sequence[int]) -> hicu_region:
    r = hicu_region()
    for a in range(3):
        r.off[a] = int(off[a])
        r.ext[a] = int(ext[a])
    return r


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)



# ------------------------------------------------------------ argument checks
#
# The C ABI sees only pointers, so a tensor of the wrong dtype, shape, layout or device would be
# read out of bounds by the kernels.  Every wrapper checks its tensors here and raises ValueError
# before anything is launched; calls then run with the tensors' device current.

def _dev(*ts):
    devs = {t.device for t in ts if t is not None}
    if len(devs) != 1:
        raise ValueError(f"tensors must all live on one CUDA device, got {sorted(map(str, devs))}")
    d = devs.pop()
    if d.type != "cuda":
        raise ValueError(f"expected CUDA tensors, got {d}")
    return d


def _need(t, name, dtype, shape=None):
    """dtype, layout and shape of one tensor (its device is checked by _dev)."""
    if t is None:
        return
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(int(v) for v in shape):
        raise ValueError(f"{name} must have shape {tuple(int(v) for v in shape)}, got {tuple(t.shape)}")


def _kshape(geom):
    return (geom.ncoil, geom.dim[2], geom.dim[1], geom.dim[0])


def _mshape(geom):
    return _kshape(geom) if geom.mask_per_coil else _kshape(geom)[1:]


def _filter_len(geom):
    return geom.ncoil * geom.k[0] * geom.k[1] * geom.k[2]


def _bank(f, geom, name="filters"):
    if f is None or f.dim() != 2:
        raise ValueError(f"{name} must be a (p, n) complex64 tensor")
    _need(f, name, torch.complex64, (f.shape[0], _filter_len(geom)))
    return f.shape[0]


class Handle:
    """Owns a hicu_handle (workspace, warm-start state) on the current device."""

    def __init__(self):
        self.ptr = c_void_p()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._check(lib().hicu_create(ctypes.byref(self.ptr)))

    def _dev(self, *ts):
        """The one CUDA device of the tensors, which must be the handle's own."""
        d = _dev(*ts)
        if d != self.device:
            raise ValueError(f"tensors on {d}, but the handle belongs to {self.device}")
        return d

    def _check(self, status: int):
        if status != 0:
            name = lib().hicu_status_string(status).decode()
            msg = lib().hicu_last_error(self.ptr).decode() if self.ptr else ""
            raise HicuError(status, f"{name}: {msg}")

    def close(self):
        if self.ptr:
            lib().hicu_destroy(self.ptr)
            self.ptr = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hicu_filter_length(geom: hicu_geom) -> int:
    return int(lib().hicu_filter_length(ctypes.byref(geom)))


def hicu_num_outputs(geom: hicu_geom, region: hicu_region) -> int:
    return int(lib().hicu_num_outputs(ctypes.byref(geom), ctypes.byref(region)))


def out_shape(geom: hicu_geom, region: hicu_region):
    out = []
    for a in range(3):
        out.append(region.ext[a] if geom.circular[a] else region.ext[a] - geom.k[a] + 1)
    return (out[2], out[1], out[0])


def hicu_check(h: Handle, stream=None):
    h._check(lib().hicu_check(h.ptr, _stream(stream)))


def hicu_profile_select(h: Handle, kernel_class: int = -1):
    h._check(lib().hicu_profile_select(h.ptr, kernel_class))


def hicu_profile_read(h: Handle):
    """-> (ms of timed launches, timed launches, all launches) since the last select/read."""
    ms, nc, na = c_double(), c_int64(), c_int64()
    h._check(lib().hicu_profile_read(h.ptr, ctypes.byref(ms), ctypes.byref(nc), ctypes.byref(na)))
    return ms.value, nc.value, na.value


def hicu_profile_eig_sweeps(h: Handle) -> int:
    v = c_int64()
    h._check(lib().hicu_profile_eig_sweeps(h.ptr, ctypes.byref(v)))
    return v.value


def hicu_gram(h: Handle, geom, region, x: torch.Tensor, G: Optional[torch.Tensor] = None, stream=None):
    n = hicu_filter_length(geom)
    _need(x, "x", torch.complex64, _kshape(geom))
    if G is None:
        G = torch.empty((n, n), dtype=torch.complex128, device=x.device)
    _need(G, "G", torch.complex128, (n, n))
    with torch.cuda.device(h._dev(x, G)):
        h._check(lib().hicu_gram(h.ptr, ctypes.byref(geom), ctypes.byref(region), _ptr(x), _ptr(G),
                                 _stream(stream)))
    return G


def _kmask(geom, kmask):
    """A kernel mask as a contiguous HOST uint8 array [kz][ky][kx] over the box geom.k."""
    import numpy as np
    m = np.ascontiguousarray(np.asarray(kmask.cpu() if isinstance(kmask, torch.Tensor) else kmask),
                             dtype=np.uint8)
    if m.shape != (geom.k[2], geom.k[1], geom.k[0]):
        raise ValueError(f"kernel mask must have shape (kz, ky, kx) = {(geom.k[2], geom.k[1], geom.k[0])}, "
                         f"got {m.shape}")
    if not m.any():
        raise ValueError("kernel mask has an empty support")
    return m


def hicu_support_length(geom, kmask) -> int:
    """C |K| for a kernel mask (the length of a filter on the mask's support)."""
    m = _kmask(geom, kmask)
    return int(lib().hicu_support_length(ctypes.byref(geom), m.ctypes.data_as(c_void_p)))


def hicu_gram_support(h: Handle, geom, region, kmask, x: torch.Tensor, G: Optional[torch.Tensor] = None,
                      stream=None):
    """G = H_K(x)^H H_K(x) over the C |K| coefficients of the kernel mask's support."""
    m = _kmask(geom, kmask)
    n = hicu_support_length(geom, m)
    _need(x, "x", torch.complex64, _kshape(geom))
    if G is None:
        G = torch.empty((n, n), dtype=torch.complex128, device=x.device)
    _need(G, "G", torch.complex128, (n, n))
    with torch.cuda.device(h._dev(x, G)):
        h._check(lib().hicu_gram_support(h.ptr, ctypes.byref(geom), ctypes.byref(region),
                                         m.ctypes.data_as(c_void_p), _ptr(x), _ptr(G), _stream(stream)))
    return G


def hicu_expand_filters(h: Handle, geom, kmask, bank_sup: torch.Tensor, stream=None):
    """(p, C |K|) filters on the mask's support -> (p, C kz ky kx) box-layout filters, zero off it."""
    m = _kmask(geom, kmask)
    n = hicu_support_length(geom, m)
    if bank_sup.dim() != 2:
        raise ValueError("bank_sup must be a (p, C |K|) complex64 tensor")
    p = bank_sup.shape[0]
    _need(bank_sup, "bank_sup", torch.complex64, (p, n))
    out = torch.empty((p, _filter_len(geom)), dtype=torch.complex64, device=bank_sup.device)
    with torch.cuda.device(h._dev(bank_sup)):
        h._check(lib().hicu_expand_filters(h.ptr, ctypes.byref(geom), m.ctypes.data_as(c_void_p), _ptr(bank_sup),
                                           p, _ptr(out), _stream(stream)))
    return out


HICU_NULLSPACE_WARM, HICU_NULLSPACE_SPLIT, HICU_NULLSPACE_GRID, HICU_NULLSPACE_CLUSTER = 1, 2, 4, 8
HICU_NULLSPACE_TRIDIAG = 16
HICU_NULLSPACE_RSVD = 32


def hicu_principal_rsvd(h: Handle, geom, region, x: torch.Tensor, r: int, l: int, V_prev=None, seed: int = 0,
                        counter: int = 0, kmask=None, want_tail: bool = False, stream=None):
    """-> (V [r][n] complex128 rows, eig_top [r] ascending[, tail J]) by randomized SVD."""
    m = None if kmask is None else _kmask(geom, kmask)
    n = _filter_len(geom) if m is None else hicu_support_length(geom, m)
    _need(x, "x", torch.complex64, _kshape(geom))
    r0 = 0
    if V_prev is not None:
        if V_prev.dim() != 2:
            raise ValueError("V_prev must be a (r0, n) complex128 tensor")
        r0 = V_prev.shape[0]
        _need(V_prev, "V_prev", torch.complex128, (r0, n))
    V = torch.empty((max(r, 0), n), dtype=torch.complex128, device=x.device)
    top = torch.empty((max(r, 0),), dtype=torch.float64, device=x.device)
    tail = torch.zeros((1,), dtype=torch.float64, device=x.device) if want_tail else None
    with torch.cuda.device(h._dev(x, V_prev)):
        h._check(lib().hicu_principal_rsvd(h.ptr, ctypes.byref(geom), ctypes.byref(region),
                                           None if m is None else m.ctypes.data_as(c_void_p), _ptr(x), r, l,
                                           _ptr(V_prev), r0, seed, counter, _ptr(V), _ptr(top), _ptr(tail),
                                           _stream(stream)))
    return (V, top, tail) if want_tail else (V, top)


def hicu_nullspace(h: Handle, G: torch.Tensor, r: int, warm: bool = False, split: bool = False,
                   solver: Optional[str] = None, stream=None):
    """solver: None (by size), "grid" or "cluster"."""
    n = G.shape[0]
    _need(G, "G", torch.complex128, (n, n))
    Q = torch.empty((max(n - r, 0), n), dtype=torch.complex128, device=G.device)  # r is checked by the library
    eig = torch.empty((n,), dtype=torch.float64, device=G.device)
    if solver not in (None, "grid", "cluster"):
        raise ValueError(f"unknown solver {solver!r}")
    flags = ((HICU_NULLSPACE_WARM if warm else 0) | (HICU_NULLSPACE_SPLIT if split else 0)
             | (HICU_NULLSPACE_GRID if solver == "grid" else 0)
             | (HICU_NULLSPACE_CLUSTER if solver == "cluster" else 0))
    with torch.cuda.device(h._dev(G)):
        h._check(lib().hicu_nullspace(h.ptr, n, r, _ptr(G), _ptr(Q), _ptr(eig), flags, _stream(stream)))
    return Q, eig


def hicu_principal_subspace(h: Handle, G: torch.Tensor, r: int, want_all: bool = False,
                            want_tail: bool = False, stream=None):
    """-> (V [r][n] complex128 rows, eig_top [r] ascending[, eig_all [n]][, tail J])."""
    n = G.shape[0]
    _need(G, "G", torch.complex128, (n, n))
    V = torch.empty((max(r, 0), n), dtype=torch.complex128, device=G.device)  # r is checked by the library
    top = torch.empty((max(r, 0),), dtype=torch.float64, device=G.device)
    allv = torch.empty((n,), dtype=torch.float64, device=G.device) if want_all else None
    tail = torch.zeros((1,), dtype=torch.float64, device=G.device) if want_tail else None
    with torch.cuda.device(h._dev(G)):
        h._check(lib().hicu_principal_subspace(h.ptr, n, r, _ptr(G), _ptr(V), _ptr(top), _ptr(allv),
                                               _ptr(tail), _stream(stream)))
    out = (V, top)
    if want_all:
        out += (allv,)
    if want_tail:
        out += (tail,)
    return out


def hicu_nullspace_info(h: Handle):
    """-> (sweeps, how): how = 0 not converged, 1 full decomposition, 2 split criterion."""
    sweeps, conv = c_int32(), c_int32()
    h._check(lib().hicu_nullspace_info(h.ptr, ctypes.byref(sweeps), ctypes.byref(conv)))
    return sweeps.value, conv.value


def hicu_jl_compress(h: Handle, Q: torch.Tensor, p: int, mode: int = HICU_JL_NULLSPACE,
                     P: Optional[torch.Tensor] = None, seed: int = 0, counter: int = 0, stream=None):
    if Q.dim() != 2:
        raise ValueError("Q must be a (rows, n) complex128 tensor")
    nr, n = Q.shape
    _need(Q, "Q", torch.complex128, (nr, n))
    _need(P, "P", torch.float64, ((nr if mode == HICU_JL_NULLSPACE else n), p))
    bank = torch.empty((p, n), dtype=torch.complex64, device=Q.device)
    with torch.cuda.device(h._dev(Q, P)):
        h._check(lib().hicu_jl_compress(h.ptr, n, nr, p, _ptr(Q), mode, _ptr(P), seed, counter,
                                        _ptr(bank), _stream(stream)))
    return bank


def hicu_conv_null_filter_grad(h: Handle, geom, region, x: torch.Tensor, Rbar: torch.Tensor, stream=None):
    """F = H(x)^H Rbar as a (p, n) complex64 filter bank."""
    p = Rbar.shape[-1]
    n = _filter_len(geom)
    _need(x, "x", torch.complex64, _kshape(geom))
    _need(Rbar, "Rbar", torch.complex64, out_shape(geom, region) + (p,))
    F = torch.empty((p, n), dtype=torch.complex64, device=x.device)
    with torch.cuda.device(h._dev(x, Rbar)):
        h._check(lib().hicu_conv_null_filter_grad(h.ptr, ctypes.byref(geom), ctypes.byref(region), _ptr(x),
                                                  _ptr(Rbar), p, _ptr(F), _stream(stream)))
    return F


def hicu_project_unobserved(h: Handle, geom, region, x: torch.Tensor, mask: Optional[torch.Tensor],
                            out: Optional[torch.Tensor] = None, stream=None):
    """(1 - M) o x on the region, 0 elsewhere."""
    _need(x, "x", torch.complex64, _kshape(geom))
    _need(mask, "mask", torch.uint8, _mshape(geom))
    if out is None:
        out = torch.empty_like(x)
    _need(out, "out", torch.complex64, _kshape(geom))
    with torch.cuda.device(h._dev(x, mask, out)):
        h._check(lib().hicu_project_unobserved(h.ptr, ctypes.byref(geom), ctypes.byref(region), _ptr(mask),
                                               _ptr(x), _ptr(out), _stream(stream)))
    return out


def hicu_conv_null(h: Handle, geom, region, x: torch.Tensor, filters: torch.Tensor,
                   prec: int = HICU_FP32, want_objective: bool = False, stream=None, store_R: bool = True):
    """store_R=False (with want_objective) only reduces ||R||^2 and returns (None, objective)."""
    _need(x, "x", torch.complex64, _kshape(geom))
    p = _bank(filters, geom)
    if not store_R and not want_objective:
        raise ValueError("store_R=False needs want_objective=True")
    R = (torch.empty(out_shape(geom, region) + (p,), dtype=torch.complex64, device=x.device)
         if store_R else None)
    obj = torch.zeros((1,), dtype=torch.float64, device=x.device) if want_objective else None
    with torch.cuda.device(h._dev(x, filters)):
        h._check(lib().hicu_conv_null(h.ptr, ctypes.byref(geom), ctypes.byref(region), _ptr(x),
                                      _ptr(filters), p, _ptr(R), _ptr(obj), prec, _stream(stream)))
    return (R, obj) if want_objective else R


def hicu_conv_null_noalloc(geom, region, x: torch.Tensor, filters: torch.Tensor,
                           want_objective: bool = False, stream=None, store_R: bool = True):
    """hicu_conv_null without a handle or any device allocation (static scratch)."""
    _need(x, "x", torch.complex64, _kshape(geom))
    p = _bank(filters, geom)
    R = (torch.empty(out_shape(geom, region) + (p,), dtype=torch.complex64, device=x.device)
         if store_R else None)
    if R is None and not want_objective:
        raise ValueError("store_R=False needs want_objective=True")
    obj = torch.zeros((1,), dtype=torch.float64, device=x.device) if want_objective else None
    with torch.cuda.device(_dev(x, filters)):
        st = lib().hicu_conv_null_noalloc(ctypes.byref(geom), ctypes.byref(region), _ptr(x),
                                          _ptr(filters), p, _ptr(R), _ptr(obj), _stream(stream))
    if st != 0:
        raise HicuError(st, lib().hicu_status_string(st).decode())
    return (R, obj) if want_objective else R


def hicu_conv_null_adjoint(h: Handle, geom, region, R: torch.Tensor, filters: torch.Tensor,
                           mask: Optional[torch.Tensor] = None, g: Optional[torch.Tensor] = None,
                           prec: int = HICU_FP32, want_gnorm2: bool = False, stream=None):
    p = _bank(filters, geom)
    _need(R, "R", torch.complex64, out_shape(geom, region) + (p,))
    _need(mask, "mask", torch.uint8, _mshape(geom))
    if g is None:
        g = torch.zeros(_kshape(geom), dtype=torch.complex64, device=R.device)
    _need(g, "g", torch.complex64, _kshape(geom))
    gn = torch.zeros((1,), dtype=torch.float64, device=R.device) if want_gnorm2 else None
    with torch.cuda.device(h._dev(R, filters, mask, g)):
        h._check(lib().hicu_conv_null_adjoint(h.ptr, ctypes.byref(geom), ctypes.byref(region), _ptr(R),
                                              _ptr(filters), p, _ptr(mask), _ptr(g), _ptr(gn), prec,
                                              _stream(stream)))
    return (g, gn) if want_gnorm2 else g


def hicu_gd_step_filters(h: Handle, geom, region, y: torch.Tensor, mask: Optional[torch.Tensor],
                         filters: torch.Tensor, prec: int = HICU_FP32, stats=None, stream=None):
    _need(y, "y", torch.complex64, _kshape(geom))
    _need(mask, "mask", torch.uint8, _mshape(geom))
    p = _bank(filters, geom)
    if stats is None:
        stats = torch.zeros((4,), dtype=torch.float64, device=y.device)
    _need(stats, "stats", torch.float64, (4,))
    with torch.cuda.device(h._dev(y, mask, filters, stats)):
        h._check(lib().hicu_gd_step_filters(h.ptr, ctypes.byref(geom), ctypes.byref(region), _ptr(y),
                                            _ptr(mask), _ptr(filters), p, _ptr(stats), prec,
                                            _stream(stream)))
    return stats


def hicu_gd_step_soft(h: Handle, geom, region, y: torch.Tensor, mask: torch.Tensor, x0: torch.Tensor,
                      lam: float, filters: torch.Tensor, prec: int = HICU_FP32, stats=None, stream=None):
    """One descent step with soft data consistency lam ||M o y - X0||^2 (y updated in place)."""
    _need(y, "y", torch.complex64, _kshape(geom))
    _need(x0, "x0", torch.complex64, _kshape(geom))
    if mask is None:
        raise ValueError("the soft data-consistency step needs the sampling mask")
    _need(mask, "mask", torch.uint8, _mshape(geom))
    p = _bank(filters, geom)
    if stats is None:
        stats = torch.zeros((4,), dtype=torch.float64, device=y.device)
    _need(stats, "stats", torch.float64, (4,))
    with torch.cuda.device(h._dev(y, mask, x0, filters, stats)):
        h._check(lib().hicu_gd_step_soft(h.ptr, ctypes.byref(geom), ctypes.byref(region), _ptr(y), _ptr(mask),
                                         _ptr(x0), float(lam), _ptr(filters), p, _ptr(stats), prec,
                                         _stream(stream)))
    return stats


def hicu_soft_threshold(h: Handle, geom, x: torch.Tensor, tau: float, stream=None):
    """The l1 proximal step on the coil images, in place on x; returns x."""
    _need(x, "x", torch.complex64, _kshape(geom))
    with torch.cuda.device(h._dev(x)):
        h._check(lib().hicu_soft_threshold(h.ptr, ctypes.byref(geom), _ptr(x), float(tau), _stream(stream)))
    return x


def hicu_gd_step(h: Handle, geom, region, y: torch.Tensor, mask: Optional[torch.Tensor],
                 Q: torch.Tensor, p: int, jl_mode: int = HICU_JL_NULLSPACE, seed: int = 0,
                 counter: int = 0, P: Optional[torch.Tensor] = None, prec: int = HICU_FP32,
                 stats=None, stream=None):
    _need(y, "y", torch.complex64, _kshape(geom))
    _need(mask, "mask", torch.uint8, _mshape(geom))
    if Q.dim() != 2:
        raise ValueError("Q must be a (rows, n) complex128 tensor")
    nr = Q.shape[0]
    _need(Q, "Q", torch.complex128, (nr, _filter_len(geom)))
    _need(P, "P", torch.float64, ((nr if jl_mode == HICU_JL_NULLSPACE else _filter_len(geom)), p))
    if stats is None:
        stats = torch.zeros((4,), dtype=torch.float64, device=y.device)
    _need(stats, "stats", torch.float64, (4,))
    with torch.cuda.device(h._dev(y, mask, Q, P, stats)):
        h._check(lib().hicu_gd_step(h.ptr, ctypes.byref(geom), ctypes.byref(region), _ptr(y), _ptr(mask),
                                    _ptr(Q), nr, p, jl_mode, seed, counter, _ptr(P), _ptr(stats), prec,
                                    _stream(stream)))
    return stats


def make_params(rank: int, stages, seed: int = 0, jl: int = HICU_JL_PROJECTOR, prec: int = HICU_FP32,
                gram_on_current: bool = False, init: int = 0, eig_solver: Optional[str] = None,
                kernel_mask=None, dc_weight: float = 0.0, l1_threshold: float = 0.0, jl_exact: bool = False,
                qplus: Optional[torch.Tensor] = None, qplus_blocks: int = 0, rsvd_cols: int = 0,
                rsvd_seed: int = 0):
    """stages: sequence of (off, ext, iters, gd_steps, p).  eig_solver: None (the library's
    default: tridiagonal principal subspace in projector mode, else Jacobi by size), "grid",
    "cluster" (Jacobi), "tridiag" or "rsvd" (randomized SVD with rsvd_cols test vectors, 0 = the
    library's default, Gaussian draws from rsvd_seed).  kernel_mask: optional (kz, ky, kx) {0,1} array over the
    kernel's box (the shape is checked by hicu_reconstruct's binding).  dc_weight: lambda of soft
    data consistency (0 = hard); l1_threshold: tau of the l1 step (0 = off); jl_exact: no JL
    compression (every step uses the whole null space: the exact gradient).  qplus: Q0 as a
    complex128 CUDA tensor (m0, n / qplus_blocks) of null vectors (rows), augmenting the null space
    with blockdiag(Q0, ..., Q0) over qplus_blocks channel groups."""
    arr = (hicu_stage * len(stages))()
    for i, (off, ext, iters, gd, p) in enumerate(stages):
        arr[i].region = make_region(off, ext)
        arr[i].iters = int(iters)
        arr[i].gd_steps = int(gd)
        arr[i].p = int(p)
    prm = hicu_params()
    prm.rank = int(rank)
    prm.nstages = len(stages)
    prm.stages = ctypes.cast(arr, POINTER(hicu_stage))
    prm.seed = int(seed)
    prm.jl = int(jl)
    prm.prec = int(prec)
    prm.gram_on_current = 1 if gram_on_current else 0
    prm.init = int(init)
    prm.eig_solver = {None: 0, "grid": HICU_NULLSPACE_GRID, "cluster": HICU_NULLSPACE_CLUSTER,
                      "tridiag": HICU_NULLSPACE_TRIDIAG, "rsvd": HICU_NULLSPACE_RSVD}[eig_solver]
    prm.rsvd_cols = int(rsvd_cols)
    prm.rsvd_seed = int(rsvd_seed)
    prm.jl_exact = 1 if jl_exact else 0
    if qplus is not None:
        if not (isinstance(qplus, torch.Tensor) and qplus.dtype == torch.complex128 and qplus.dim() == 2
                and qplus.is_contiguous() and qplus.device.type == "cuda"):
            raise ValueError("qplus must be a contiguous complex128 CUDA tensor (m0, n0)")
        prm.qplus = qplus.data_ptr()
        prm.qplus_cols = int(qplus.shape[0])
        prm.qplus_blocks = int(qplus_blocks)
        prm._keep_qplus = qplus
    prm.dc_weight = float(dc_weight)
    prm.l1_threshold = float(l1_threshold)
    prm._keep = arr  # keep the stage array alive with the struct
    if kernel_mask is not None:
        import numpy as np
        km = np.ascontiguousarray(np.asarray(kernel_mask), dtype=np.uint8)
        prm.kernel_mask = km.ctypes.data_as(c_void_p)
        prm._keep_mask = km
    return prm


def hicu_reconstruct(h: Handle, geom, x0: torch.Tensor, mask: torch.Tensor, params: hicu_params,
                     x_out: Optional[torch.Tensor] = None, want_log: bool = False, stream=None):
    """x0 / mask / x_out may live on the GPU or (pinned) on the host."""
    if getattr(params, "_keep_mask", None) is not None:
        _kmask(geom, params._keep_mask)
    if getattr(params, "_keep_qplus", None) is not None:
        q = params._keep_qplus
        nb = params.qplus_blocks
        n = hicu_filter_length(geom) if getattr(params, "_keep_mask", None) is None else \
            hicu_support_length(geom, params._keep_mask)
        if nb < 1 or n % nb or q.shape[1] != n // nb:
            raise ValueError(f"qplus must have n / qplus_blocks = {n // max(nb, 1)} columns per row")
    _need(x0, "x0", torch.complex64, _kshape(geom))
    _need(mask, "mask", torch.uint8, _mshape(geom))
    if x_out is None:
        x_out = torch.empty_like(x0)
    _need(x_out, "x_out", torch.complex64, _kshape(geom))
    on_gpu = [t for t in (x0, mask, x_out) if t.device.type == "cuda"]
    if on_gpu:
        h._dev(*on_gpu)
    log_struct, logs = None, None
    if want_log:
        iters = sum(params.stages[i].iters for i in range(params.nstages))
        steps = sum(params.stages[i].iters * params.stages[i].gd_steps for i in range(params.nstages))
        logs = {"J": (c_double * max(iters, 1))(), "objective": (c_double * max(steps, 1))(),
                "eta": (c_double * max(steps, 1))()}
        log_struct = hicu_log(ctypes.cast(logs["J"], POINTER(c_double)),
                              ctypes.cast(logs["objective"], POINTER(c_double)),
                              ctypes.cast(logs["eta"], POINTER(c_double)))
        logs["_n"] = (iters, steps)
    h._check(lib().hicu_reconstruct(h.ptr, ctypes.byref(geom), _ptr(x0), _ptr(mask),
                                    ctypes.byref(params), _ptr(x_out),
                                    ctypes.byref(log_struct) if log_struct is not None else None,
                                    _stream(stream)))
    if want_log:
        it, st = logs["_n"]
        return x_out, {"J": list(logs["J"])[:it], "objective": list(logs["objective"])[:st],
                       "eta": list(logs["eta"])[:st]}
    return x_out


# ------------------------------------------------------------------ batches

def make_problem_struct(geom, x0: torch.Tensor, mask: torch.Tensor, params: hicu_params,
                        x_out: torch.Tensor) -> hicu_problem:
    _need(x0, "x0", torch.complex64, _kshape(geom))
    _need(mask, "mask", torch.uint8, _mshape(geom))
    _need(x_out, "x_out", torch.complex64, _kshape(geom))
    pr = hicu_problem()
    pr.geom = geom
    pr.x0 = x0.data_ptr()
    pr.mask = mask.data_ptr()
    pr.params = params
    pr.x_out = x_out.data_ptr()
    pr.log = None
    pr._keep = (params, x0, mask, x_out)
    return pr


def hicu_batch_order(problems: Sequence[hicu_problem]):
    """-> (order, cost): start order of hicu_reconstruct_batched and the cost estimates."""
    n = len(problems)
    arr = (hicu_problem * max(n, 1))(*problems)
    order = (c_int32 * max(n, 1))()
    cost = (c_double * max(n, 1))()
    st = lib().hicu_batch_order(n, ctypes.cast(arr, ctypes.c_void_p), order, cost)
    if st != 0:
        raise HicuError(st, lib().hicu_status_string(st).decode())
    return list(order)[:n], list(cost)[:n]


def hicu_reconstruct_batched(h: Handle, problems: Sequence[hicu_problem], lanes: int = 0, stream=None,
                             check: bool = True):
    """Runs every problem (hicu_reconstruct semantics); returns one report dict per problem.
    With check=False a failing problem does not raise; its report carries the status."""
    n = len(problems)
    arr = (hicu_problem * max(n, 1))(*problems)
    rep = (hicu_slice_report * max(n, 1))()
    st = lib().hicu_reconstruct_batched(h.ptr, n, ctypes.cast(arr, ctypes.c_void_p), int(lanes),
                                        ctypes.cast(rep, ctypes.c_void_p), _stream(stream))
    if check:
        h._check(st)
    return [{"start_ms": r.start_ms, "end_ms": r.end_ms, "lane": r.lane, "status": r.status,
             "gd_steps": r.gd_steps} for r in list(rep)[:n]], st
