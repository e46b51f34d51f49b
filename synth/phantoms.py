"""Seeded phantoms, coil maps, sampling masks and noisy k-space.

Array conventions shared by every consumer:
  k-space x : complex64, shape (C, Nz, Ny, Nx)  (x fastest; 2D has Nz = 1,
              2D+t cine puts time in the Nz slot)
  mask      : uint8, shape (Nz, Ny, Nx) broadcast over coils, or
              (C, Nz, Ny, Nx) when the sampling differs per channel
              (multi-shot stacks)
  k-space is centred: DC sits at index N // 2 along every axis.

The recipes follow the workloads of the paper's Studies I-IV (2D brain,
2D+t cine, 3D knee, multi-shot diffusion), scaled to the sizes listed in
CONFIG_NAMES.  None of the paper's datasets is used; everything is drawn from
numpy's seeded PCG64 generator.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

CONFIG_NAMES = (
    "2d_small_64",      # 64x64, C=4, k=5x5, r=30
    "2d_brain_256",     # 256x256, C=8, k=5x5, r=75, centre-out from 64x64
    "cine_192x144x24",  # 192x144x24, C=8, k=5x5x5, r=300, circular in t
    "knee3d_256x256x160",  # 256x256x160, C=8, k=5x5x5, r=400
    "batched_uneven",   # 48 slices of mixed size/coils + 4 multi-shot slices
)


@dataclass
class Stage:
    """One centre-out stage: region (offset, extent), outer iterations, GD steps, JL dimension."""
    off: Tuple[int, int, int]
    ext: Tuple[int, int, int]
    iters: int
    gd_steps: int
    p: int


@dataclass
class Problem:
    name: str
    x_full: np.ndarray            # fully sampled noisy k-space (the SER reference)
    mask: np.ndarray              # sampling mask, uint8
    x0: np.ndarray                # zero-filled observed k-space
    kernel: Tuple[int, int, int]  # (kx, ky, kz)
    circular: Tuple[int, int, int]
    rank: int
    stages: List[Stage] = field(default_factory=list)
    seed: int = 0
    init: str = "zero_filled"     # or "time_average" (cine)

    @property
    def ncoil(self) -> int:
        return self.x_full.shape[0]

    @property
    def dims(self) -> Tuple[int, int, int]:
        c, nz, ny, nx = self.x_full.shape
        return (nx, ny, nz)


# ---------------------------------------------------------------- transforms
def centered_fft(img: np.ndarray, axes) -> np.ndarray:
    """Orthonormal DFT with DC moved to index N//2 (data generation only)."""
    return np.fft.fftshift(
        np.fft.fftn(np.fft.ifftshift(img, axes=axes), axes=axes, norm="ortho"),
        axes=axes)


# ------------------------------------------------------------------ images
def _grid(shape):
    """Normalised coordinates in [-1, 1) per axis, returned x-fastest order."""
    axes = [np.linspace(-1.0, 1.0, n, endpoint=False) for n in shape]
    return np.meshgrid(*axes, indexing="ij")


def _smooth_phase(rng, coords, order=2, amp=np.pi / 2):
    ph = np.zeros(coords[0].shape)
    for _ in range(4):
        w = rng.uniform(-order, order, size=len(coords)) * np.pi / 2
        ph += rng.uniform(0.2, 1.0) * np.cos(sum(wi * c for wi, c in zip(w, coords))
                                             + rng.uniform(0, 2 * np.pi))
    return amp * ph / 4


def ellipse_image_2d(rng, ny, nx, n_ellipses, texture=0.0, radius_scale=None):
    """Sum of random rotated ellipses with amplitudes U(0.2, 1) times a smooth phase."""
    yy, xx = _grid((ny, nx))
    img = np.zeros((ny, nx))
    for e in range(n_ellipses):
        cy, cx = rng.uniform(-0.55, 0.55, 2)
        ay, ax = rng.uniform(0.06, 0.4, 2)
        if radius_scale is not None:
            ay *= radius_scale[e]
            ax *= radius_scale[e]
        th = rng.uniform(0, np.pi)
        u = (xx - cx) * np.cos(th) + (yy - cy) * np.sin(th)
        v = -(xx - cx) * np.sin(th) + (yy - cy) * np.cos(th)
        img += rng.uniform(0.2, 1.0) * ((u / ax) ** 2 + (v / ay) ** 2 <= 1.0)
    if texture > 0:
        t = rng.standard_normal((ny, nx))
        # separable 5-tap box smoothing keeps the texture low-pass
        for ax_ in (0, 1):
            t = sum(np.roll(t, s, axis=ax_) for s in range(-2, 3)) / 5.0
        img += texture * t * (img > 0)
    return img * np.exp(1j * _smooth_phase(rng, (yy, xx)))


def ellipsoid_volume(rng, nz, ny, nx, n_ellipsoids):
    zz, yy, xx = _grid((nz, ny, nx))
    vol = np.zeros((nz, ny, nx))
    for _ in range(n_ellipsoids):
        c = rng.uniform(-0.5, 0.5, 3)
        a = rng.uniform(0.08, 0.45, 3)
        vol += rng.uniform(0.2, 1.0) * (((zz - c[0]) / a[0]) ** 2 + ((yy - c[1]) / a[1]) ** 2
                                        + ((xx - c[2]) / a[2]) ** 2 <= 1.0)
    return vol * np.exp(1j * _smooth_phase(rng, (zz, yy, xx)))


def coil_maps(rng, shape, ncoil):
    """Gaussian bumps on a circle (sphere band in 3D) times low-order complex exponentials."""
    coords = _grid(shape)
    maps = np.empty((ncoil,) + tuple(shape), dtype=np.complex128)
    for c in range(ncoil):
        ang = 2 * np.pi * c / ncoil + rng.uniform(-0.2, 0.2)
        centre = np.zeros(len(shape))
        centre[-1] = 0.8 * np.cos(ang)          # x
        centre[-2] = 0.8 * np.sin(ang)          # y
        if len(shape) == 3:
            centre[0] = rng.uniform(-0.5, 0.5)  # z
        r2 = sum((ci - cc) ** 2 for ci, cc in zip(coords, centre))
        mag = np.exp(-r2 / (2 * 0.55 ** 2))
        w = rng.uniform(-1.0, 1.0, len(shape)) * np.pi / 2
        phase = sum(wi * ci for wi, ci in zip(w, coords)) + rng.uniform(0, 2 * np.pi)
        maps[c] = mag * np.exp(1j * phase)
    return maps


# ------------------------------------------------------------------- masks
def vd_lines_mask(rng, ny, nx, R, n_center, power=2.0):
    """1D variable-density phase-encode mask: whole k_x lines at chosen k_y."""
    n_lines = max(n_center, int(round(ny / R)))
    ky = np.arange(ny)
    dist = np.abs(ky - ny // 2) / (ny / 2)
    w = (1.0 - dist) ** power + 0.02
    chosen = set(range(ny // 2 - n_center // 2, ny // 2 - n_center // 2 + n_center))
    rest = np.array([k for k in ky if k not in chosen])
    pr = w[rest] / w[rest].sum()
    extra = rng.choice(rest, size=n_lines - len(chosen), replace=False, p=pr)
    chosen.update(int(e) for e in extra)
    m = np.zeros((ny, nx), dtype=np.uint8)
    m[sorted(chosen), :] = 1
    return m


def poisson_disc_like_mask(rng, nz, ny, R, center):
    """Variable-density dart throwing over (k_z, k_y) with a fully sampled centre."""
    target = int(round(nz * ny / R))
    m = np.zeros((nz, ny), dtype=bool)
    z0, y0 = nz // 2 - center // 2, ny // 2 - center // 2
    m[z0:z0 + center, y0:y0 + center] = True
    zz, yy = np.meshgrid(np.arange(nz), np.arange(ny), indexing="ij")
    rad = np.sqrt(((zz - nz // 2) / (nz / 2)) ** 2 + ((yy - ny // 2) / (ny / 2)) ** 2)
    # exclusion radius grows with distance from the centre (variable density)
    excl = 0.6 + 1.2 * np.clip(rad, 0, 1.0)
    order = rng.permutation(nz * ny)
    count = int(m.sum())
    for idx in order:
        if count >= target:
            break
        z, y = divmod(int(idx), ny)
        if m[z, y]:
            continue
        r = excl[z, y]
        ri = int(np.ceil(r))
        zs, ze = max(0, z - ri), min(nz, z + ri + 1)
        ys, ye = max(0, y - ri), min(ny, y + ri + 1)
        sub = m[zs:ze, ys:ye]
        if sub.any():
            dz, dy = np.nonzero(sub)
            if np.min((dz + zs - z) ** 2 + (dy + ys - y) ** 2) < r * r:
                continue
        m[z, y] = True
        count += 1
    if count < target:  # top up at random if dart throwing saturated
        free = np.flatnonzero(~m.ravel())
        add = rng.choice(free, size=target - count, replace=False)
        m.ravel()[add] = True
    return m.astype(np.uint8)


# ---------------------------------------------------------------- problems
def _noisy(rng, k, sigma):
    n = (rng.standard_normal(k.shape) + 1j * rng.standard_normal(k.shape)) * (sigma / np.sqrt(2))
    return k + n


def _co_region(dims, full_axes):
    """Centred 1/4 region per spatial axis; axes listed in full_axes keep their whole extent."""
    off, ext = [], []
    for a, n in enumerate(dims):
        if a in full_axes or n == 1:
            off.append(0)
            ext.append(n)
        else:
            e = n // 4
            off.append(n // 2 - e // 2)
            ext.append(e)
    return tuple(off), tuple(ext)


def _slice_2d(rng, n, C, R, n_ellipses=10, texture=0.0, n_center=8, sigma=1e-3):
    img = ellipse_image_2d(rng, n, n, n_ellipses, texture=texture)
    maps = coil_maps(rng, (n, n), C)
    k = centered_fft(maps * img[None], axes=(-2, -1))
    k = _noisy(rng, k, sigma)[:, None]
    mask = vd_lines_mask(rng, n, n, R, n_center)[None]
    return k.astype(np.complex64), mask


def make_problem(name: str, seed: Optional[int] = None, scale: int = 1) -> Problem:
    """Build one seeded problem.  ``scale`` > 1 shrinks every spatial axis (tests)."""
    idx = CONFIG_NAMES.index(name)
    if seed is None:
        seed = idx * 1000
    rng = np.random.default_rng(seed)
    if name == "2d_small_64":
        n = 64 // scale
        k, mask = _slice_2d(rng, n, 4, 3.0, n_ellipses=6, n_center=8)
        full = ((0, 0, 0), (n, n, 1))
        stages = [Stage(full[0], full[1], iters=10, gd_steps=3, p=4)]
        return Problem(name, k, mask, (k * mask[None]).astype(np.complex64), (5, 5, 1), (0, 0, 0),
                       30, stages, seed)
    if name == "2d_brain_256":
        n = 256 // scale
        k, mask = _slice_2d(rng, n, 8, 4.0, n_ellipses=20, texture=0.02, n_center=8)
        co_off, co_ext = _co_region((n, n, 1), ())
        stages = [Stage(co_off, co_ext, iters=50, gd_steps=5, p=8),
                  Stage((0, 0, 0), (n, n, 1), iters=10, gd_steps=10, p=32)]
        return Problem(name, k, mask, (k * mask[None]).astype(np.complex64), (5, 5, 1), (0, 0, 0),
                       75, stages, seed)
    if name == "cine_192x144x24":
        nx, ny, nt = 192 // scale, 144 // scale, 24
        C = 8
        maps = coil_maps(rng, (ny, nx), C)
        n_e = 8
        base_rng_state = rng.integers(0, 2 ** 63)
        phases = rng.uniform(0, 2 * np.pi, n_e)
        amps = rng.uniform(0.05, 0.2, n_e)
        frames = []
        for t in range(nt):
            r = np.random.default_rng(int(base_rng_state))  # same ellipses every frame
            scale_t = 1.0 + amps * np.sin(2 * np.pi * t / nt + phases)
            frames.append(ellipse_image_2d(r, ny, nx, n_e, radius_scale=scale_t))
        img = np.stack(frames)                          # (Nt, Ny, Nx)
        k = centered_fft(maps[:, None] * img[None], axes=(-2, -1))
        k = _noisy(rng, k, 1e-3).astype(np.complex64)
        mask = np.stack([vd_lines_mask(rng, ny, nx, 6.0, 2) for _ in range(nt)])
        co_off, co_ext = _co_region((nx, ny, nt), (2,))
        stages = [Stage(co_off, co_ext, iters=20, gd_steps=5, p=8),
                  Stage((0, 0, 0), (nx, ny, nt), iters=1, gd_steps=100, p=8)]
        return Problem(name, k, mask, (k * mask[None]).astype(np.complex64), (5, 5, 5), (0, 0, 1),
                       300, stages, seed, init="time_average")
    if name == "knee3d_256x256x160":
        nx, ny, nz = 256 // scale, 256 // scale, 160 // scale
        C = 8
        vol = ellipsoid_volume(rng, nz, ny, nx, 12)
        maps = coil_maps(rng, (nz, ny, nx), C)
        k = np.empty((C, nz, ny, nx), dtype=np.complex64)
        for c in range(C):
            k[c] = _noisy(rng, centered_fft(maps[c] * vol, axes=(0, 1, 2)), 1e-3)
        m2 = poisson_disc_like_mask(rng, nz, ny, 5.0, max(2, 24 // scale))
        mask = np.repeat(m2[:, :, None], nx, axis=2)
        co_off, co_ext = _co_region((nx, ny, nz), ())
        stages = [Stage(co_off, co_ext, iters=10, gd_steps=5, p=8),
                  Stage((0, 0, 0), (nx, ny, nz), iters=1, gd_steps=20, p=8)]
        return Problem(name, k, mask, (k * mask[None]).astype(np.complex64), (5, 5, 5), (0, 0, 0),
                       400, stages, seed)
    raise ValueError(f"use make_batch() for {name}")


def make_batch(seed: int = 4000, n_plain: int = 48, n_dwi: int = 4, sizes=(128, 192, 256, 320),
               coils=(4, 8, 16), rates=(3.0, 4.0, 5.0)) -> List[Problem]:
    """Uneven batch: plain 2D slices of mixed size/coils/rate plus multi-shot stacks."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_plain):
        n = int(rng.choice(sizes))
        C = int(rng.choice(coils))
        R = float(rng.choice(rates))
        k, mask = _slice_2d(rng, n, C, R, n_ellipses=12)
        r = int(round(0.375 * 25 * C))
        co_off, co_ext = _co_region((n, n, 1), ())
        stages = [Stage(co_off, co_ext, iters=10, gd_steps=5, p=8),
                  Stage((0, 0, 0), (n, n, 1), iters=2, gd_steps=10, p=min(32, 25 * C - r))]
        out.append(Problem(f"slice{i}_{n}_c{C}_r{R:g}", k, mask,
                           (k * mask[None]).astype(np.complex64), (5, 5, 1), (0, 0, 0), r, stages,
                           seed + i))
    for i in range(n_dwi):
        n, C, S = 256, 8, 4
        img = ellipse_image_2d(rng, n, n, 12)
        maps = coil_maps(rng, (n, n), C)
        yy, xx = _grid((n, n))
        chans, masks = [], []
        for s in range(S):
            ph = np.exp(1j * _smooth_phase(rng, (yy, xx), order=1, amp=np.pi))
            k = centered_fft(maps * (img * ph)[None], axes=(-2, -1))
            chans.append(_noisy(rng, k, 1e-3))
            m = np.zeros((n, n), dtype=np.uint8)
            m[s::S, :] = 1                       # interleaved EPI shot s
            masks.append(np.repeat(m[None], C, axis=0))
        k = np.concatenate(chans)[:, None].astype(np.complex64)   # (S*C, 1, n, n)
        mask = np.concatenate(masks)[:, None]                     # per-channel mask
        co_off, co_ext = _co_region((n, n, 1), ())
        stages = [Stage(co_off, co_ext, iters=10, gd_steps=5, p=8),
                  Stage((0, 0, 0), (n, n, 1), iters=2, gd_steps=10, p=32)]
        out.append(Problem(f"dwi{i}_{n}_c{S * C}", k, mask, (k * mask).astype(np.complex64),
                           (5, 5, 1), (0, 0, 0), 150, stages, seed + 100 + i))
    return out


def make_msdwi(seed: int = 5000, n: int = 256, C: int = 8, S: int = 4, pf: float = 0.59,
               co_iters: int = 50, co_steps: int = 5, pf_steps: int = 100, rank: int = 45):
    """Multi-shot diffusion slice shaped like the paper's Study IV, and its non-diffusion (b0) data.

    Diffusion-weighted data: one image (ellipses), C coil maps, S interleaved EPI shots each with its
    own smooth random phase (the shot-to-shot motion phase), stacked as S*C channels [shot][coil].
    Shot s samples the phase-encode lines s, s + S, ... (uniform downsampling) inside the
    partial-Fourier extent: lines [round((1 - pf) n), n) (the first (1 - pf) n lines are never
    sampled).  The b0 data: a second image (the same ellipses, other intensities) with one smooth
    phase, fully sampled, C coils (the four shots of the non-diffusion scan summed).
    Schedule (Methods, Study IV): centre-out on the central n/4 x n/4 region for co_iters
    iterations of co_steps descent steps (p = C), then the partial-Fourier sampled region with
    pf_steps steps.  Returns (Problem, x_b0)."""
    rng = np.random.default_rng(seed)
    base = np.random.default_rng(int(rng.integers(0, 2 ** 63)))
    img = ellipse_image_2d(np.random.default_rng(int(base.integers(0, 2 ** 63))), n, n, 12)
    maps = coil_maps(rng, (n, n), C)
    yy, xx = _grid((n, n))
    y0 = int(round((1.0 - pf) * n))
    chans, masks = [], []
    for s in range(S):
        ph = np.exp(1j * _smooth_phase(rng, (yy, xx), order=1, amp=np.pi))
        k = centered_fft(maps * (img * ph)[None], axes=(-2, -1))
        chans.append(_noisy(rng, k, 1e-3))
        m = np.zeros((n, n), dtype=np.uint8)
        lines = np.arange(n)
        m[(lines % S == s) & (lines >= y0), :] = 1
        masks.append(np.repeat(m[None], C, axis=0))
    k = np.concatenate(chans)[:, None].astype(np.complex64)     # (S*C, 1, n, n)
    mask = np.concatenate(masks)[:, None]                       # per-channel mask
    # b0: same anatomy, different contrast, one phase, fully sampled
    rb = np.random.default_rng(int(rng.integers(0, 2 ** 63)))
    img0 = ellipse_image_2d(np.random.default_rng(int(base.integers(0, 2 ** 63))), n, n, 12) * 0.5 + img
    ph0 = np.exp(1j * _smooth_phase(rb, (yy, xx), order=1, amp=np.pi / 2))
    x_b0 = _noisy(rb, centered_fft(maps * (img0 * ph0)[None], axes=(-2, -1)), 1e-3)[:, None].astype(np.complex64)
    co_off, co_ext = _co_region((n, n, 1), ())
    stages = [Stage(co_off, co_ext, iters=co_iters, gd_steps=co_steps, p=C),
              Stage((0, y0, 0), (n, n - y0, 1), iters=1, gd_steps=pf_steps, p=C)]
    pb = Problem(f"msdwi_{n}_c{S * C}", k, mask, (k * mask).astype(np.complex64), (5, 5, 1), (0, 0, 0), rank,
                 stages, seed)
    return pb, x_b0


def lowrank_exponential_kspace(rng, shape, ncoil, n_terms):
    """Exactly low-rank multi-coil k-space: every coil is a sum of the same n_terms complex
    exponentials with coil-specific amplitudes, so any block-Hankel matrix built from it
    has rank <= n_terms."""
    nz, ny, nx = shape
    idx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x = np.zeros((ncoil, nz, ny, nx), dtype=np.complex128)
    for _ in range(n_terms):
        w = rng.uniform(-np.pi, np.pi, 3)
        if nz == 1:
            w[0] = 0.0
        wave = np.exp(1j * (w[0] * idx[0] + w[1] * idx[1] + w[2] * idx[2]))
        a = rng.standard_normal(ncoil) + 1j * rng.standard_normal(ncoil)
        x += a[:, None, None, None] * wave[None]
    return x


def random_complex(rng, shape, dtype=np.complex128):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype)
