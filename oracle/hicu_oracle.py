"""Plain FP64 CPU oracle for the HICU hot path (test infrastructure only).

This module is the correctness reference for the CUDA library.  It is slow on
purpose: every operation is the paper's definition written out with numpy
slicing, ``einsum``, ``matmul`` and LAPACK's ``eigh``, in float64/complex128,
with no blocking, fusion or reordering beyond what the definition states.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It imports nothing from the CUDA package and the
CUDA package imports nothing from here.

Citations name the paper ("HICU", Zhao, Potter & Ahmad, MRM 2021) by section,
equation and algorithm step.

Conventions (fixed by this library, see the readings listed in the design notes):
  * k-space array x has shape (C, Nz, Ny, Nx); 2D uses Nz = 1 and 2D+t puts
    time in the Nz slot.
  * Kernel support K is rectangular (kx, ky, kz) over all C coils, so
    n = C*kz*ky*kx.  A filter vector v of length n is ordered (c, dz, dy, dx)
    with dx fastest, i.e. ``v.reshape(C, kz, ky, kx)``.
  * H(x) is the multi-level Hankel matrix whose row for output position p is
    the patch [x_c[p + d]] over (c, d) in that order, so H(x) v is the valid
    (correlation-form) convolution of x with v (Theory section).  A kernel
    flip only relabels v and leaves every singular value unchanged.
  * A region S is (off, ext) per axis (x, y, z).  Valid outputs are the
    positions whose whole kernel footprint lies inside S; an axis flagged
    circular wraps modulo its extent instead (2D+t time axis, Methods,
    Study II).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np

# --------------------------------------------------------------- geometry


@dataclass(frozen=True)
class Geom:
    dims: Tuple[int, int, int]          # (Nx, Ny, Nz)
    ncoil: int
    kernel: Tuple[int, int, int]        # (kx, ky, kz): the box that holds the kernel mask
    circular: Tuple[int, int, int] = (0, 0, 0)
    # kernel mask K (Algorithm 1 input; Theory: v lists the kernel values on the support of K):
    # the offsets (dz, dy, dx) of the support in scan order, or None for the whole box
    support: Optional[Tuple[Tuple[int, int, int], ...]] = None

    @property
    def nk(self) -> int:
        """|K|, the number of kernel offsets per coil."""
        kx, ky, kz = self.kernel
        return len(self.support) if self.support is not None else kx * ky * kz

    @property
    def n(self) -> int:
        return self.ncoil * self.nk


def ellipsoid_support(kernel: Tuple[int, int, int], radius: float) -> Tuple[Tuple[int, int, int], ...]:
    """Circular (2D) or spherical (3D) kernel mask inside the box `kernel` (Discussion: circumscribing
    circular or spherical kernel masks): the offsets d with sum_a (d_a - c_a)^2 <= radius^2 over the
    axes with k_a > 1, c_a = (k_a - 1) / 2 the box centre.  Offsets in (dz, dy, dx) scan order."""
    kx, ky, kz = kernel
    cx, cy, cz = (kx - 1) / 2.0, (ky - 1) / 2.0, (kz - 1) / 2.0
    out = []
    for dz in range(kz):
        for dy in range(ky):
            for dx in range(kx):
                r2 = (dx - cx) ** 2 + (dy - cy) ** 2 + (dz - cz) ** 2
                if r2 <= radius * radius + 1e-9:
                    out.append((dz, dy, dx))
    return tuple(out)


def support_mask(geom: Geom) -> np.ndarray:
    """The kernel mask K as a {0,1} array [kz][ky][kx]."""
    kx, ky, kz = geom.kernel
    m = np.zeros((kz, ky, kx), dtype=np.uint8)
    for dz, dy, dx in _offsets(geom):
        m[dz, dy, dx] = 1
    return m


@dataclass(frozen=True)
class Region:
    off: Tuple[int, int, int]
    ext: Tuple[int, int, int]


def full_region(geom: Geom) -> Region:
    return Region((0, 0, 0), tuple(geom.dims))


def out_shape(geom: Geom, reg: Region) -> Tuple[int, int, int]:
    """Valid-output grid (sz, sy, sx) inside region S (Theory: valid convolution)."""
    out = []
    for a in range(3):
        if geom.circular[a]:
            out.append(reg.ext[a])
        else:
            out.append(reg.ext[a] - geom.kernel[a] + 1)
    sx, sy, sz = out
    return (sz, sy, sx)


def num_outputs(geom: Geom, reg: Region) -> int:
    """s = |valid outputs in S| (Theory, complexity paragraph)."""
    sz, sy, sx = out_shape(geom, reg)
    return sz * sy * sx


def _axis_index(geom: Geom, reg: Region, axis: int, d: int) -> np.ndarray:
    """Absolute input index along ``axis`` (0=x,1=y,2=z) read by every output at kernel offset d."""
    sz, sy, sx = out_shape(geom, reg)
    nout = (sx, sy, sz)[axis]
    o = np.arange(nout)
    if geom.circular[axis]:
        rel = (o + d) % reg.ext[axis]
    else:
        rel = o + d
    return reg.off[axis] + rel


def _shifted_block(x: np.ndarray, geom: Geom, reg: Region, dz: int, dy: int, dx: int) -> np.ndarray:
    """x_c[p + d] for every coil c and every valid output p: shape (C, sz, sy, sx)."""
    iz = _axis_index(geom, reg, 2, dz)
    iy = _axis_index(geom, reg, 1, dy)
    ix = _axis_index(geom, reg, 0, dx)
    return x[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]]


def _offsets(geom: Geom):
    """The kernel offsets (dz, dy, dx) on the support of K, in scan order (dx fastest)."""
    if geom.support is not None:
        yield from geom.support
        return
    kx, ky, kz = geom.kernel
    for dz in range(kz):
        for dy in range(ky):
            for dx in range(kx):
                yield dz, dy, dx


def _check(x: np.ndarray, geom: Geom, reg: Region):
    C, nz, ny, nx = x.shape
    assert (nx, ny, nz) == tuple(geom.dims) and C == geom.ncoil, "array does not match geometry"
    for a in range(3):
        assert 0 <= reg.off[a] and reg.off[a] + reg.ext[a] <= geom.dims[a], "region outside array"
        if not geom.circular[a]:
            assert reg.ext[a] >= geom.kernel[a], "region smaller than kernel"


# ----------------------------------------------- Hankel operator H(x) and adjoints


def hankel_matrix(x: np.ndarray, geom: Geom, reg: Region) -> np.ndarray:
    """Explicit m-by-n multi-level Hankel matrix H(x) on region S (Theory section).

    Row order: valid outputs (z, y, x) with x fastest.  Column order: (c, kernel offset) with the
    offsets of the support of K in scan order (dz, dy, dx).  Only for small inputs (it is the object
    HICU never forms).
    """
    _check(x, geom, reg)
    s = num_outputs(geom, reg)
    cols = np.empty((geom.ncoil, geom.nk, s), dtype=np.complex128)
    for j, (dz, dy, dx) in enumerate(_offsets(geom)):
        cols[:, j, :] = _shifted_block(x, geom, reg, dz, dy, dx).reshape(geom.ncoil, s)
    return cols.reshape(geom.n, s).T.copy()


def conv_null(x: np.ndarray, geom: Geom, reg: Region, filters: np.ndarray) -> np.ndarray:
    """R[:, k] = H(x) q_k for each filter q_k (Theory: H(x)v is the valid convolution of x with v).

    filters: (p, C, kz, ky, kx) complex.  Returns R with shape (sz, sy, sx, p),
    i.e. R[p_out, k] = sum_{c,d} x_c[p_out + d] q_k[c, d].
    """
    _check(x, geom, reg)
    x = np.asarray(x, dtype=np.complex128)
    f = np.asarray(filters, dtype=np.complex128)
    R = np.zeros(out_shape(geom, reg) + (f.shape[0],), dtype=np.complex128)
    for dz, dy, dx in _offsets(geom):
        blk = _shifted_block(x, geom, reg, dz, dy, dx)            # (C, sz, sy, sx)
        R += np.einsum("czyx,kc->zyxk", blk, f[:, :, dz, dy, dx], optimize=True)
    return R


def conv_null_adjoint(R: np.ndarray, geom: Geom, reg: Region, filters: np.ndarray,
                      mask: Optional[np.ndarray] = None) -> np.ndarray:
    """Adjoint of x -> [H(x) q_k]_k, optionally projected onto unsampled entries.

    g_c[u] = sum_k sum_d conj(q_k[c, d]) R[u - d, k]  (the conjugate transpose of a valid
    convolution is itself a convolution, Theory section).  With ``mask`` the result is
    multiplied by (1 - M): the gradient is zero at observed locations (hard data
    consistency, end of the Theory section).  Output shape (C, Nz, Ny, Nx), zero outside S.
    """
    f = np.asarray(filters, dtype=np.complex128)
    R = np.asarray(R, dtype=np.complex128)
    nx, ny, nz = geom.dims
    g = np.zeros((geom.ncoil, nz, ny, nx), dtype=np.complex128)
    for dz, dy, dx in _offsets(geom):
        iz = _axis_index(geom, reg, 2, dz)
        iy = _axis_index(geom, reg, 1, dy)
        ix = _axis_index(geom, reg, 0, dx)
        contrib = np.einsum("zyxk,kc->czyx", R, np.conj(f[:, :, dz, dy, dx]), optimize=True)
        # for a fixed offset d the map p -> p + d is injective, so plain fancy-index add is exact
        g[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]] += contrib
    if mask is not None:
        g *= (1 - _mask4(mask, g.shape))
    return g


def filter_gradient(x: np.ndarray, geom: Geom, reg: Region, Rbar: np.ndarray) -> np.ndarray:
    """Adjoint of v -> H(x) v: F[k] = H(x)^H Rbar[:, k], returned as filters (p, C, kz, ky, kx).

    F_k[c, d] = sum_{p_out} conj(x_c[p_out + d]) Rbar[p_out, k].  The filters are the
    unknowns of the annihilation relation H(x) v = 0 (Theory section), so this is the
    gradient of Re<Rbar, H(x) v> with respect to v; with Rbar = H(x) v it equals the Gram
    product (H^H H) v.  Rbar has the shape of conv_null's output, (sz, sy, sx, p).
    """
    _check(x, geom, reg)
    x = np.asarray(x, dtype=np.complex128)
    Rb = np.asarray(Rbar, dtype=np.complex128)
    kx, ky, kz = geom.kernel
    F = np.zeros((Rb.shape[-1], geom.ncoil, kz, ky, kx), dtype=np.complex128)
    for dz, dy, dx in _offsets(geom):
        blk = _shifted_block(x, geom, reg, dz, dy, dx)            # (C, sz, sy, sx)
        F[:, :, dz, dy, dx] = np.einsum("czyx,zyxk->kc", np.conj(blk), Rb, optimize=True)
    return F


def conv_null_at(x: np.ndarray, geom: Geom, reg: Region, filters: np.ndarray, outs: np.ndarray) -> np.ndarray:
    """R[o, k] = H(x) q_k at chosen valid outputs only (Theory: row o of H(x) is the patch
    [x_c[o + d]] over (c, d)); for sampled checks of volumes too large to convolve here.

    outs: int array (m, 3) of (oz, oy, ox) indices into the valid-output grid out_shape(geom, reg).
    Returns (m, p).
    """
    _check(x, geom, reg)
    x = np.asarray(x, dtype=np.complex128)
    f = np.asarray(filters, dtype=np.complex128)
    if geom.support is not None:
        f = f * support_mask(geom)[None, None]   # the kernel lives on the support of K
    outs = np.asarray(outs, dtype=np.int64).reshape(-1, 3)
    kx, ky, kz = geom.kernel
    idx = []
    for a, (col, k) in enumerate(((2, kx), (1, ky), (0, kz))):   # axis a = x, y, z
        rel = outs[:, col][:, None] + np.arange(k)[None, :]
        if geom.circular[a]:
            rel = rel % reg.ext[a]
        idx.append(reg.off[a] + rel)                               # (m, k_a)
    ix, iy, iz = idx
    patch = x[:, iz[:, :, None, None], iy[:, None, :, None], ix[:, None, None, :]]   # (C, m, kz, ky, kx)
    return np.einsum("cmzyx,kczyx->mk", patch, f, optimize=True)


def gradient_at(x: np.ndarray, geom: Geom, reg: Region, filters: np.ndarray, us: np.ndarray,
                mask: Optional[np.ndarray] = None) -> np.ndarray:
    """The descent direction g = (1 - M) o sum_k H^H(H(x) q_k) at chosen positions u of region S.

    g_c[u] = sum_k sum_d conj(q_k[c, d]) R[u - d, k] over the offsets d for which u - d is a
    valid output (taken modulo the extent on a circular axis), R = H(x) q from conv_null_at;
    times (1 - M[u]) (hard data consistency, end of the Theory section).
    us: int array (m, 3) of (uz, uy, ux) in region coordinates.  Returns (C, m).
    """
    f = np.asarray(filters, dtype=np.complex128)
    us = np.asarray(us, dtype=np.int64).reshape(-1, 3)
    kx, ky, kz = geom.kernel
    sz, sy, sx = out_shape(geom, reg)
    lim = (sz, sy, sx)
    g = np.zeros((geom.ncoil, len(us)), dtype=np.complex128)
    for dz, dy, dx in _offsets(geom):
        o = us - np.array([dz, dy, dx])[None, :]
        ok = np.ones(len(us), dtype=bool)
        for col, a in ((0, 2), (1, 1), (2, 0)):
            if geom.circular[a]:
                o[:, col] %= reg.ext[a]
            else:
                ok &= (o[:, col] >= 0) & (o[:, col] < lim[col])
        if not ok.any():
            continue
        R = conv_null_at(x, geom, reg, f, o[ok])                   # (m_ok, p)
        g[:, ok] += np.einsum("mk,kc->cm", R, np.conj(f[:, :, dz, dy, dx]), optimize=True)
    if mask is not None:
        m = np.asarray(mask)
        m4 = m if m.ndim == 4 else m[None]
        mv = m4[:, reg.off[2] + us[:, 0], reg.off[1] + us[:, 1], reg.off[0] + us[:, 2]]
        g = g * (1 - mv.astype(np.float64))
    return g


def project_unobserved(x: np.ndarray, geom: Geom, reg: Region, mask: Optional[np.ndarray]) -> np.ndarray:
    """(1 - M) o x on the region S and 0 outside it (hard data consistency, Theory section)."""
    x = np.asarray(x, dtype=np.complex128)
    out = np.zeros_like(x)
    z0, y0, x0 = reg.off[2], reg.off[1], reg.off[0]
    z1, y1, x1 = z0 + reg.ext[2], y0 + reg.ext[1], x0 + reg.ext[0]
    out[:, z0:z1, y0:y1, x0:x1] = x[:, z0:z1, y0:y1, x0:x1]
    if mask is not None:
        out *= (1 - _mask4(mask, out.shape))
    return out


def _mask4(mask: np.ndarray, shape) -> np.ndarray:
    m = np.asarray(mask).astype(np.float64)
    if m.ndim == 3:
        m = m[None]
    return np.broadcast_to(m, shape)


# ------------------------------------------------------------ Gram and null space


def gram(x: np.ndarray, geom: Geom, reg: Region, chunk: int = 1 << 15) -> np.ndarray:
    """G = H(x)^H H(x), the n-by-n Gram matrix of the block-Hankel matrix on region S.

    Entry (a, b) is sum over valid outputs p of conj(h_p[a]) h_p[b]; its eigenvalues are
    the squared singular values of H(x) (Eq. 1), and the paper's Discussion names SVD of
    this Gram matrix as the alternative to rSVD.  Built in row chunks of H.
    """
    _check(x, geom, reg)
    x = np.asarray(x, dtype=np.complex128)
    sz, sy, sx = out_shape(geom, reg)
    G = np.zeros((geom.n, geom.n), dtype=np.complex128)
    plane = sy * sx
    zstep = max(1, chunk // max(plane, 1))
    for z0 in range(0, sz, zstep):
        z1 = min(sz, z0 + zstep)
        sub = Region(reg.off, reg.ext)
        Hc = _hankel_rows(x, geom, sub, z0, z1)
        G += Hc.conj().T @ Hc
    return G


def _hankel_rows(x, geom, reg, z0, z1):
    sz, sy, sx = out_shape(geom, reg)
    rows = (z1 - z0) * sy * sx
    cols = np.empty((geom.ncoil, geom.nk, rows), dtype=np.complex128)
    for j, (dz, dy, dx) in enumerate(_offsets(geom)):
        blk = _shifted_block(x, geom, reg, dz, dy, dx)[:, z0:z1]
        cols[:, j, :] = blk.reshape(geom.ncoil, rows)
    return cols.reshape(geom.n, rows).T


def nullspace(G: np.ndarray, r: int) -> Tuple[np.ndarray, np.ndarray]:
    """Null-space basis Q (n x (n-r)) and ascending eigenvalues of G (Algorithm 1 steps 2-3).

    The r principal right singular vectors V of H are the top-r eigenvectors of G = H^H H;
    Q spans their orthogonal complement, here taken directly as the eigenvectors of the
    n - r smallest eigenvalues.  J(x) = sum of those eigenvalues (Eq. 1).
    """
    n = G.shape[0]
    if not (0 < r < n):
        raise ValueError("rank must satisfy 0 < r < n")
    w, V = np.linalg.eigh(G)
    return V[:, : n - r].copy(), w


def tail_energy(eigvals: np.ndarray, r: int) -> float:
    """J(x) = sum_{k>r} sigma_k^2 {H(x)} (Eq. 1) from ascending eigenvalues of H^H H."""
    n = eigvals.shape[0]
    return float(np.sum(eigvals[: n - r]))


# ------------------------------------------------------- randomized SVD (Theory: rSVD)


def complex_gaussian(seed: int, counter: int, rows: int, cols: int) -> np.ndarray:
    """rows x cols complex Gaussian matrix of unit variance: entry (a, b) has real part
    gaussian(seed, counter, 2 e) / sqrt(2) and imaginary part gaussian(seed, counter, 2 e + 1) / sqrt(2),
    e = a cols + b (the same counter-based generator as the JL draws)."""
    out = np.empty((rows, cols), dtype=np.complex128)
    for a in range(rows):
        for b in range(cols):
            e = a * cols + b
            out[a, b] = complex(gaussian(seed, counter, 2 * e), gaussian(seed, counter, 2 * e + 1)) / math.sqrt(2.0)
    return out


# the stabilising shift nu of rsvd_principal, relative to ||Z||_F / sqrt(l): above the rounding level
# of an FP32 evaluation of Z = H^H H Omega (a smaller shift lets that rounding into Omega^H Y's
# smallest directions), 2^-17
RSVD_SHIFT = 2.0 ** -17


def rsvd_principal(x: np.ndarray, geom: Geom, reg: Region, r: int, l: int, seed: int, counter: int,
                   V_prev: Optional[np.ndarray] = None) -> Tuple[np.ndarray, np.ndarray]:
    """The r principal right singular vectors of H(x) on S by randomized SVD (Theory: rSVD, Algorithm
    1 step 2), with a warm start.

    Test matrix Omega (n x l): the previous outer iteration's principal vectors V_prev (when given),
    then complex Gaussian columns complex_gaussian(seed, counter, n, l - r0).  One application of the
    valid convolution and one of its conjugate transpose per column give Z = H^H (H Omega) =
    (H^H H) Omega.  The randomized SVD of H through its Gram H^H H (the single-pass form for a
    positive semidefinite matrix, with a small shift nu for stability):
        Y = Z + nu Omega,   T = Omega^H Y = R^H R (Cholesky),   K = Y R^{-1},
    so K K^H = (H^H H + nu I) Omega (Omega^H (H^H H + nu I) Omega)^{-1} Omega^H (H^H H + nu I) is the
    rank-l approximation of H^H H + nu I from range(H^H H Omega); the top r left singular vectors of
    K are V and their squared singular values minus nu the eigenvalue estimates.  Exact when
    rank(H) <= l.  nu = RSVD_SHIFT ||Z||_F / sqrt(l).  Returns (V n x r, estimates ascending)."""
    n = geom.n
    r0 = 0 if V_prev is None else V_prev.shape[1]
    gauss = complex_gaussian(seed, counter, n, l - r0)
    Omega = gauss if V_prev is None else np.concatenate([V_prev, gauss], axis=1)
    R = conv_null(x, geom, reg, as_filters(Omega.T.copy(), geom))          # H Omega, (sz, sy, sx, l)
    Z = _support_coeffs(filter_gradient(x, geom, reg, R).reshape(l, geom.ncoil, -1), geom).T   # n x l
    nu = RSVD_SHIFT * np.linalg.norm(Z) / math.sqrt(l)
    Y = Z + nu * Omega
    T = Omega.conj().T @ Y
    T = 0.5 * (T + T.conj().T)
    Rc = np.linalg.cholesky(T).conj().T                                   # T = Rc^H Rc, Rc upper
    K = np.linalg.solve(Rc.T, Y.T).T                                      # K Rc = Y
    W, sig, _ = np.linalg.svd(K, full_matrices=False)
    lam = np.maximum(sig[:r] ** 2 - nu, 0.0)
    return W[:, :r][:, ::-1].copy(), lam[::-1].copy()


def _support_coeffs(F: np.ndarray, geom: Geom) -> np.ndarray:
    """Box-layout coefficients (p, C, kz ky kx) -> the n coefficients on the support of K (p, n)."""
    p = F.shape[0]
    if geom.support is None:
        return F.reshape(p, -1)
    kx, ky, kz = geom.kernel
    idx = [(dz * ky + dy) * kx + dx for dz, dy, dx in geom.support]
    return F[:, :, idx].reshape(p, -1)


# --------------------------------------------------------------- JL compression

_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64_mix(z: int) -> int:
    """SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014)."""
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def splitmix64_output(seed: int, k: int) -> int:
    """k-th output (k >= 1) of the SplitMix64 sequence started at state ``seed``."""
    return splitmix64_mix((seed + k * _GAMMA) & _M64)


def gaussian(seed: int, counter: int, e: int) -> float:
    """Standard normal number e of draw ``counter``: Box-Muller on two SplitMix64 outputs.

    Outputs k0+1 and k0+2 with k0 = 2*(counter*2^32 + e) give u1 in (0, 1] and u2 in [0, 1);
    z = sqrt(-2 ln u1) cos(2 pi u2).
    """
    k0 = 2 * ((counter << 32) + e)
    o1 = splitmix64_output(seed, k0 + 1)
    o2 = splitmix64_output(seed, k0 + 2)
    u1 = ((o1 >> 11) + 1) * 2.0 ** -53
    u2 = (o2 >> 11) * 2.0 ** -53
    return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def jl_matrix(seed: int, counter: int, rows: int, p: int) -> np.ndarray:
    """P^(i,j): rows x p i.i.d. zero-mean Gaussian entries of variance 1/p (Theory, JL paragraph).

    Element (row, col) is gaussian(seed, counter, row * p + col) / sqrt(p).
    """
    out = np.empty((rows, p))
    for a in range(rows):
        for b in range(p):
            out[a, b] = gaussian(seed, counter, a * p + b)
    return out / math.sqrt(p)


def jl_compress(Q: np.ndarray, P: np.ndarray, mode: str = "nullspace") -> np.ndarray:
    """Q~ = Q P compressed to p filters (Algorithm 1 step 6).

    mode "nullspace": P is (n-r) x p and Q~ = Q P, the formula of step 6.
    mode "projector": P is n x p (the dimension the Theory text gives) and Q~ = Q (Q^H P),
    i.e. the n x p Gaussian projected onto span(Q); Q~ then depends only on the null
    subspace, not on the basis chosen for it.
    Returns filters of shape (p, n).
    """
    if mode == "nullspace":
        Qt = Q @ P
    elif mode == "projector":
        Qt = Q @ (Q.conj().T @ P)
    else:
        raise ValueError(mode)
    return Qt.T.copy()


def qplus_matrix(Q0: np.ndarray, blocks: int) -> np.ndarray:
    """Q+ = blockdiag(Q0, ..., Q0) with `blocks` repetitions (Methods, Study IV: the null space is
    augmented to [Q | Q+] with the null vectors Q0 of the non-diffusion (b0) data, one block per
    shot).  Q0 is n0 x m0 over one shot's channels (coil, then kernel offset); the shots' channels
    are consecutive in the filter order [channel][offset], so block s covers filter indices
    [s n0, (s + 1) n0)."""
    n0, m0 = Q0.shape
    out = np.zeros((blocks * n0, blocks * m0), dtype=np.complex128)
    for b in range(blocks):
        out[b * n0:(b + 1) * n0, b * m0:(b + 1) * m0] = Q0
    return out


def jl_compress_augmented(Q: np.ndarray, Qplus: np.ndarray, P: np.ndarray, mode: str = "projector") -> np.ndarray:
    """Q~ = [Q | Q+] P for the augmented null space (Algorithm 1 step 6 with step 3's basis
    [Q | Q+]): the first rows of P compress Q as jl_compress does, the last Q+.shape[1] rows
    multiply Q+.  E[Q~ Q~^H] = Q Q^H + Q+ Q+^H.  Returns (p, n)."""
    m = Qplus.shape[1]
    head, tail = P[:P.shape[0] - m], P[P.shape[0] - m:]
    return jl_compress(Q, head, mode) + (Qplus @ tail).T


def as_filters(Qt_pn: np.ndarray, geom: Geom) -> np.ndarray:
    """p filters of length n (coil, then the support offsets) as arrays (p, C, kz, ky, kx) over the
    kernel's box, zero outside the support of K."""
    kx, ky, kz = geom.kernel
    p = Qt_pn.shape[0]
    if geom.support is None:
        return Qt_pn.reshape(p, geom.ncoil, kz, ky, kx)
    out = np.zeros((p, geom.ncoil, kz, ky, kx), dtype=Qt_pn.dtype)
    v = Qt_pn.reshape(p, geom.ncoil, geom.nk)
    for j, (dz, dy, dx) in enumerate(geom.support):
        out[:, :, dz, dy, dx] = v[:, :, j]
    return out


# ------------------------------------------------------------ gradient step + ELS


@dataclass
class StepInfo:
    eta: float
    objective: float     # ||H(y) Q~||_F^2 before the step
    gnorm2: float        # ||g||^2
    denom: float         # ||H(g) Q~||_F^2


def gradient(y, geom, reg, filters, mask):
    """g = (1 - M) o sum_k H^H(H(y) q~_k)  (Algorithm 1 step 7 with hard data consistency).

    The exact Wirtinger gradient of sum_k ||H(y) q~_k||^2 is 2 g; the factor 2 is absorbed
    by the exact line search, which makes eta * g invariant to it.
    """
    R = conv_null(y, geom, reg, filters)
    return conv_null_adjoint(R, geom, reg, filters, mask), R


def gd_step(y: np.ndarray, mask: np.ndarray, geom: Geom, reg: Region, filters: np.ndarray
            ) -> Tuple[np.ndarray, StepInfo]:
    """One descent step with exact line search (Algorithm 1 steps 7-8).

    phi(eta) = ||H(y - eta g) Q~||^2 is quadratic in eta; its minimiser is
    eta = Re<H(y)Q~, H(g)Q~> / ||H(g)Q~||^2, obtained from one more convolution of g with
    each of the p filters (Theory, ELS paragraph).  Because g is the masked adjoint of
    H(y)Q~, the numerator equals ||g||^2.  A zero gradient or zero denominator gives eta = 0.
    """
    y = np.asarray(y, dtype=np.complex128)
    g, R = gradient(y, geom, reg, filters, mask)
    obj = float(np.vdot(R, R).real)
    gn2 = float(np.vdot(g, g).real)
    Rg = conv_null(g, geom, reg, filters)
    D = float(np.vdot(Rg, Rg).real)
    eta = gn2 / D if (D > 0.0 and gn2 > 0.0) else 0.0
    return y - eta * g, StepInfo(eta, obj, gn2, D)


def region_indicator(geom: Geom, reg: Region) -> np.ndarray:
    """1 on the entries of region S, 0 elsewhere, shape (1, Nz, Ny, Nx)."""
    nx, ny, nz = geom.dims
    ind = np.zeros((1, nz, ny, nx))
    ind[:, reg.off[2]:reg.off[2] + reg.ext[2], reg.off[1]:reg.off[1] + reg.ext[1],
        reg.off[0]:reg.off[0] + reg.ext[0]] = 1.0
    return ind


def gd_step_soft(y: np.ndarray, x0: np.ndarray, mask: np.ndarray, geom: Geom, reg: Region, filters: np.ndarray,
                 lam: float) -> Tuple[np.ndarray, StepInfo]:
    """One descent step on ||H(y) Q~||^2 + lam ||M o y - X0||^2 with exact line search: the soft
    data-consistency cost f_1 of the problem statement with multiplier lam (Theory, Eq. 3), in
    Algorithm 1 steps 7-8.

    Only the entries of region S move (the others are constants of this step), so the data term
    is taken over S.  With X0 zero off the samples, M o y - X0 = M o (y - X0) and
      g   = sum_k H^H(H(y) q~_k) + lam M o (y - X0)            (on S; the factor 2 dropped)
      phi(eta) = ||H(y - eta g) Q~||^2 + lam ||M o (y - eta g - X0)||^2,
    a quadratic in eta whose minimiser is Re<H(y)Q~, H(g)Q~> + lam Re<M(y - X0), M g> over
    ||H(g)Q~||^2 + lam ||M g||^2, and the numerator equals ||g||^2.  StepInfo.objective is
    phi(0), StepInfo.denom the denominator.
    """
    y = np.asarray(y, dtype=np.complex128)
    x0 = np.asarray(x0, dtype=np.complex128)
    ind = region_indicator(geom, reg)
    m = _mask4(mask, y.shape)
    R = conv_null(y, geom, reg, filters)
    dc = ind * m * (y - x0)
    g = conv_null_adjoint(R, geom, reg, filters) + lam * dc
    obj = float(np.vdot(R, R).real + lam * np.vdot(dc, dc).real)
    gn2 = float(np.vdot(g, g).real)
    Rg = conv_null(g, geom, reg, filters)
    mg = ind * m * g
    D = float(np.vdot(Rg, Rg).real + lam * np.vdot(mg, mg).real)
    eta = gn2 / D if (D > 0.0 and gn2 > 0.0) else 0.0
    return y - eta * g, StepInfo(eta, obj, gn2, D)


def image_axes(geom: Geom) -> Tuple[int, ...]:
    """Array axes of the sparsifying transform: x, y and z, except a circular z (the time axis of
    2D+t) and axes of length 1."""
    nx, ny, nz = geom.dims
    axes = []
    if nz > 1 and not geom.circular[2]:
        axes.append(1)
    if ny > 1:
        axes.append(2)
    if nx > 1:
        axes.append(3)
    return tuple(axes)


def soft_threshold(x: np.ndarray, geom: Geom, tau: float) -> np.ndarray:
    """The proximal step of tau ||T x||_1 for T the centred orthonormal inverse DFT of every coil
    over the image axes (the coil images): x <- T^H S_tau(T x), with the complex soft threshold
    S_tau(w) = w max(0, 1 - tau / |w|) (Discussion: an l1 norm of a linear sparsifying transform of
    X is a soft-thresholding after Algorithm 1 step 8)."""
    axes = image_axes(geom)
    x = np.asarray(x, dtype=np.complex128)
    w = np.fft.fftshift(np.fft.ifftn(np.fft.ifftshift(x, axes=axes), axes=axes, norm="ortho"), axes=axes)
    mag = np.abs(w)
    w = w * np.maximum(0.0, 1.0 - tau / np.maximum(mag, 1e-300))
    return np.fft.fftshift(np.fft.fftn(np.fft.ifftshift(w, axes=axes), axes=axes, norm="ortho"), axes=axes)


# ----------------------------------------------------------- the HICU iteration


@dataclass
class StageSpec:
    region: Region
    iters: int
    gd_steps: int
    p: int


@dataclass
class ReconLog:
    J: List[float]
    objective: List[float]
    eta: List[float]


def initial_estimate(x0: np.ndarray, mask: np.ndarray, mode: str = "zero_filled") -> np.ndarray:
    """x^(0) = vec{X0} (Algorithm 1); for 2D+t the time-averaged k-space (Methods, Study II):
    each unsampled (k_x, k_y, t) takes the mean of its sampled frames, or zero if none."""
    x = np.asarray(x0, dtype=np.complex128).copy()
    if mode == "zero_filled":
        return x
    if mode != "time_average":
        raise ValueError(mode)
    m = _mask4(mask, x.shape)
    cnt = m.sum(axis=1, keepdims=True)                       # frames sampled per (c, ky, kx)
    tot = (x * m).sum(axis=1, keepdims=True)
    avg = np.where(cnt > 0, tot / np.maximum(cnt, 1), 0.0)
    return np.where(m > 0, x, np.broadcast_to(avg, x.shape))


def reconstruct(x0: np.ndarray, mask: np.ndarray, geom: Geom, stages: Sequence[StageSpec], r: int,
                seed: int, jl_mode: str = "projector", gram_on: str = "previous",
                init: str = "zero_filled", log: Optional[ReconLog] = None, lam: float = 0.0,
                tau: float = 0.0, qplus: Optional[Tuple[np.ndarray, int]] = None,
                rsvd: Optional[Tuple[int, int]] = None) -> np.ndarray:
    """Algorithm 1 (HICU) with the Gram route for steps 2-3 and centre-out stages.

    For i = 1..I: null space of H^(i-1)(x^(i-1)) (step 2 names the previous region;
    ``gram_on="current"`` uses S^(i) instead), then G^(i) descent steps on S^(i), each with a
    fresh JL draw (counter = global step index, starting at 0).
    rsvd = (l, seed): the principal vectors by rsvd_principal with l test vectors, warm-started from
    the previous outer iteration's (counter = outer iteration index), then the projector-form filters
    (I - V V^H) P; J is logged as trace(G) - sum of the Ritz values.
    jl_mode "exact": no JL compression, every step uses the whole null basis Q as its filters.
    qplus = (Q0, blocks): the augmented null space [Q | Q+] of the multi-shot study (qplus_matrix);
    each step's JL matrix has Q+.shape[1] more rows (jl_compress_augmented), or without
    compression the filters are the columns of [Q | Q+].
    lam > 0: soft data consistency with that multiplier (gd_step_soft) instead of hard data
    consistency.  tau > 0: after every descent step of a stage whose region is the whole array,
    the l1 proximal step soft_threshold (Discussion), followed under hard data consistency by
    restoring the observed samples.
    """
    x = initial_estimate(x0, mask, init)
    counter = 0
    prev = stages[0].region
    V = None
    it = 0
    for st in stages:
        for _ in range(st.iters):
            greg = prev if gram_on == "previous" else st.region
            if rsvd is not None:
                V, lam_r = rsvd_principal(x, geom, greg, r, rsvd[0], rsvd[1], it, V)
                # the null space's projector I - V V^H through an orthonormal completion of V
                Q = np.linalg.svd(np.eye(geom.n) - V @ V.conj().T)[0][:, :geom.n - r]
                if log is not None:
                    tr = float(np.sum(np.abs(_hankel_rows(x, geom, greg, 0, out_shape(geom, greg)[0])) ** 2))
                    log.J.append(tr - float(np.sum(lam_r)))
            else:
                G = gram(x, geom, greg)
                Q, w = nullspace(G, r)
                if log is not None:
                    log.J.append(tail_energy(w, r))
            it += 1
            y = x
            rows = Q.shape[0] if jl_mode == "projector" else Q.shape[1]
            whole = tuple(st.region.off) == (0, 0, 0) and tuple(st.region.ext) == tuple(geom.dims)
            Qp = None if qplus is None else qplus_matrix(qplus[0], qplus[1])
            mplus = 0 if Qp is None else Qp.shape[1]
            for _ in range(st.gd_steps):
                if jl_mode == "exact":
                    # no JL compression: the n - r columns of Q (and of Q+) are the filters
                    basis = Q if Qp is None else np.concatenate([Q, Qp], axis=1)
                    f = as_filters(basis.T.copy(), geom)
                elif Qp is None:
                    P = jl_matrix(seed, counter, rows, st.p)
                    f = as_filters(jl_compress(Q, P, jl_mode), geom)
                else:
                    P = jl_matrix(seed, counter, rows + mplus, st.p)
                    f = as_filters(jl_compress_augmented(Q, Qp, P, jl_mode), geom)
                counter += 1
                if lam > 0.0:
                    y, info = gd_step_soft(y, x0, mask, geom, st.region, f, lam)
                else:
                    y, info = gd_step(y, mask, geom, st.region, f)
                if tau > 0.0 and whole:
                    y = soft_threshold(y, geom, tau)
                    if lam <= 0.0:
                        obs = _mask4(mask, y.shape) > 0
                        y = np.where(obs, np.asarray(x0, dtype=np.complex128), y)
                if log is not None:
                    log.objective.append(info.objective)
                    log.eta.append(info.eta)
            x = y
            prev = st.region
    return x


def ser_db(x_ref: np.ndarray, x_hat: np.ndarray) -> float:
    """SER = 20 log10(||X||_F / ||X_hat - X||_F) over all coils (Methods, Study I)."""
    num = np.linalg.norm(np.asarray(x_ref, dtype=np.complex128).ravel())
    den = np.linalg.norm((np.asarray(x_hat, dtype=np.complex128) - x_ref).ravel())
    return float(20.0 * np.log10(num / den))
