"""The seeded synthetic inputs (synth/phantoms.py) against the recipe they claim: reproducible per
seed, the shared array layout, zero-filled observations, the DC convention of the centred FFT,
the sampling rates and fully sampled centres of the masks, and the stage schedules the benchmark
reports.  CPU only; the workloads are built at reduced scale where they are large."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from synth import phantoms as P  # noqa: E402

SCALED = (("2d_small_64", 1, 3.0), ("2d_brain_256", 4, 4.0), ("cine_192x144x24", 4, 6.0),
          ("knee3d_256x256x160", 4, 5.0))


@pytest.mark.parametrize("name,scale,R", SCALED)
def test_problem_layout_and_zero_filling(name, scale, R):
    pb = P.make_problem(name, scale=scale)
    C, nz, ny, nx = pb.x0.shape
    assert pb.x0.dtype == np.complex64 and pb.x_full.dtype == np.complex64
    assert pb.x_full.shape == pb.x0.shape
    assert pb.mask.dtype == np.uint8 and pb.mask.shape == (nz, ny, nx)
    assert set(np.unique(pb.mask)) <= {0, 1}
    assert pb.dims == (nx, ny, nz)
    # the observation is the fully sampled data on the mask, zero elsewhere
    np.testing.assert_array_equal(pb.x0, (pb.x_full * pb.mask[None]).astype(np.complex64))
    # sampling rate 1 / R (whole lines or columns: the rounding of one line count)
    assert abs(pb.mask.mean() - 1.0 / R) < 0.02
    assert 0 < pb.rank < C * np.prod(pb.kernel)


def test_same_seed_same_problem_other_seed_other_problem():
    a = P.make_problem("2d_small_64")
    b = P.make_problem("2d_small_64")
    c = P.make_problem("2d_small_64", seed=1)
    np.testing.assert_array_equal(a.x0, b.x0)
    np.testing.assert_array_equal(a.mask, b.mask)
    assert not np.array_equal(a.x_full, c.x_full)


def test_centred_fft_puts_dc_at_the_middle_index():
    # a constant image transforms to one sample at N // 2 on every axis (orthonormal: sqrt(N))
    img = np.ones((6, 10), dtype=np.complex128)
    k = P.centered_fft(img, axes=(0, 1))
    peak = np.unravel_index(np.argmax(np.abs(k)), k.shape)
    assert peak == (3, 5)
    assert abs(k[3, 5] - np.sqrt(60)) < 1e-12
    assert np.abs(k).sum() - abs(k[3, 5]) < 1e-9
    # orthonormal: energy kept
    rng = np.random.default_rng(0)
    x = P.random_complex(rng, (7, 9))
    assert abs(np.linalg.norm(P.centered_fft(x, axes=(0, 1))) - np.linalg.norm(x)) < 1e-9


def test_line_mask_keeps_the_centre_lines_and_the_line_count():
    rng = np.random.default_rng(3)
    m = P.vd_lines_mask(rng, 64, 40, 4.0, 8)
    rows = m.any(axis=1)
    assert (m[rows] == 1).all()                 # whole k_x lines
    assert rows.sum() == round(64 / 4.0)
    assert rows[32 - 4:32 + 4].all()            # the 8 centre lines


def test_dart_mask_hits_its_target_and_keeps_the_centre_block():
    rng = np.random.default_rng(4)
    m = P.poisson_disc_like_mask(rng, 40, 48, 5.0, 12)
    assert m.sum() == round(40 * 48 / 5.0)
    assert (m[20 - 6:20 + 6, 24 - 6:24 + 6] == 1).all()


@pytest.mark.parametrize("name,scale,text", [
    ("2d_brain_256", 1, "CO 64x64 50x5 p=8 + full 10x10 p=32"),
    ("cine_192x144x24", 4, "CO 12x9x24 20x5 p=8 + full 1x100 p=8"),
    ("knee3d_256x256x160", 4, "CO 16x16x10 10x5 p=8 + full 1x20 p=8"),
])
def test_schedules_are_centred_quarter_regions_then_the_whole_array(name, scale, text):
    pb = P.make_problem(name, scale=scale)
    assert bench.schedule_text(pb) == text
    co = pb.stages[0]
    for a, n in enumerate(pb.dims):
        if co.ext[a] != n:   # a centre-out axis: the centred quarter
            assert co.ext[a] == n // 4 and co.off[a] == n // 2 - co.ext[a] // 2
    assert tuple(pb.stages[-1].off) == (0, 0, 0) and tuple(pb.stages[-1].ext) == pb.dims


def test_multishot_stack_shots_interleave_inside_the_partial_fourier_extent():
    pb, x_b0 = P.make_msdwi(n=64)
    S, C = 4, 8
    assert pb.x0.shape == (S * C, 1, 64, 64) and pb.mask.shape == (S * C, 1, 64, 64)
    assert x_b0.shape == (C, 1, 64, 64)
    y0 = int(round((1 - 0.59) * 64))
    lines = [np.flatnonzero(pb.mask[s * C, 0].any(axis=1)) for s in range(S)]
    for s in range(S):
        assert (lines[s] >= y0).all() and (lines[s] % S == s).all()
        for c in range(C):   # every coil of a shot shares the shot's lines
            np.testing.assert_array_equal(pb.mask[s * C + c], pb.mask[s * C])
    # together the shots sample every line of the partial-Fourier extent once
    assert sorted(np.concatenate(lines).tolist()) == list(range(y0, 64))
    last = pb.stages[-1]
    assert tuple(last.off) == (0, y0, 0) and tuple(last.ext) == (64, 64 - y0, 1)


def test_uneven_batch_draws_its_sizes_coils_and_rates_from_the_recipe():
    b = P.make_batch(n_plain=6, n_dwi=1)
    assert len(b) == 7
    for pb in b[:6]:
        C, nz, ny, nx = pb.x0.shape
        assert nx == ny and nx in (128, 192, 256, 320) and nz == 1 and C in (4, 8, 16)
        assert pb.mask.shape == (1, ny, nx)
    dwi = b[6]
    assert dwi.x0.shape == (32, 1, 256, 256) and dwi.mask.shape == dwi.x0.shape
