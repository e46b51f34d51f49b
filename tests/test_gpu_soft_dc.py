"""Soft data consistency (Theory, Eq. 3: f_1 with multiplier lambda) and the l1 proximal step
(Discussion: soft-thresholding after Algorithm 1 step 8) on the GPU, against the FP64 oracle.

Step level, random data: the soft descent step's {eta, objective, ||g||^2, denominator} and update
(bounds as the hard steps: FP32 2e-5, split-BF16 1e-4 relative); entries outside the region
untouched bit for bit.  The l1 step on 2D, 3D and 2D+t arrays (the time axis not transformed) to
2e-5.  Reconstructions with either on the 64 x 64 problem against the oracle: NRMSE <= 1e-3,
SER within 0.05 dB; under hard consistency with the l1 step the observed samples bit-identical.
"""
import numpy as np
import pytest
import torch

from closeness import assert_close
from oracle import hicu_oracle as O
from synth.phantoms import make_problem, random_complex

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2004_08962_gb300 import build, hicu
    build.build()
    return hicu.Handle()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


STEP_CASES = {
    # dims, C, kernel, circular, region (off, ext), p, lambda
    "2d_region": ((48, 40, 1), 4, (5, 5, 1), (0, 0, 0), ((3, 2, 0), (41, 36, 1)), 6, 0.8),
    "3d_k5_c8": ((28, 26, 14), 8, (5, 5, 5), (0, 0, 0), ((1, 1, 1), (26, 24, 12)), 8, 3.0),
    "cine_circular_t": ((24, 20, 8), 2, (3, 3, 3), (0, 0, 1), ((0, 0, 0), (24, 20, 8)), 5, 0.3),
}


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
@pytest.mark.parametrize("name", list(STEP_CASES))
def test_soft_step_parity(H, name, prec):
    from paper_2004_08962_gb300 import hicu
    dims, C, ker, circ, (off, ext), p, lam = STEP_CASES[name]
    og, oreg = O.Geom(dims, C, ker, circ), O.Region(off, ext)
    rng = np.random.default_rng(9)
    shape = (C, dims[2], dims[1], dims[0])
    mask = (rng.random(shape[1:]) < 0.35).astype(np.uint8)
    x = random_complex(rng, shape).astype(np.complex64)
    x0 = (random_complex(rng, shape) * mask[None]).astype(np.complex64)
    f = random_complex(rng, (p, og.n)).astype(np.complex64)
    hg, hr = hicu.make_geom(dims, C, ker, circ), hicu.make_region(off, ext)
    y = cuda(x)
    pr = hicu.HICU_SPLIT_BF16 if prec == "split_bf16" else hicu.HICU_FP32
    stats = hicu.hicu_gd_step_soft(H, hg, hr, y, cuda(mask), cuda(x0), lam, cuda(f), prec=pr).cpu().numpy()
    y_ref, info = O.gd_step_soft(x, x0, mask, og, oreg, O.as_filters(f, og), lam)
    tol = 1e-4 if prec == "split_bf16" else 2e-5
    for got, want in zip(stats, (info.eta, info.objective, info.gnorm2, info.denom)):
        assert abs(got - want) <= tol * abs(want), (got, want)
    y1 = y.cpu().numpy()
    assert_close(y1 - x, y_ref - x, tol, f"soft step {name} ({prec})")
    inside = O.region_indicator(og, oreg)[0].astype(bool)
    np.testing.assert_array_equal(y1[:, ~inside], x[:, ~inside])
    hicu.hicu_check(H)


@pytest.mark.parametrize("dims,C,circ", [((64, 48, 1), 4, (0, 0, 0)), ((20, 18, 12), 3, (0, 0, 0)),
                                        ((24, 20, 8), 2, (0, 0, 1)), ((30, 1, 7), 2, (0, 0, 0))])
def test_soft_threshold_parity(H, dims, C, circ):
    from paper_2004_08962_gb300 import hicu
    og = O.Geom(dims, C, (1, 1, 1), circ)
    rng = np.random.default_rng(4)
    x = random_complex(rng, (C, dims[2], dims[1], dims[0])).astype(np.complex64)
    tau = 0.7
    ref = O.soft_threshold(x, og, tau)
    # the threshold sets a share of the coil-image samples to zero
    img = np.fft.ifftn(ref, axes=O.image_axes(og), norm="ortho")
    assert np.mean(np.abs(img) < 1e-9) > 0.05
    hg = hicu.make_geom(dims, C, (1, 1, 1), circ)
    y = cuda(x)
    hicu.hicu_soft_threshold(H, hg, y, tau)
    assert_close(y.cpu().numpy(), ref, 2e-5, f"l1 step {dims}")
    # tau = 0 leaves the array untouched
    y0 = cuda(x)
    hicu.hicu_soft_threshold(H, hg, y0, 0.0)
    np.testing.assert_array_equal(y0.cpu().numpy(), x)
    hicu.hicu_check(H)


def _coil_image_scale(pb):
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
    axes = O.image_axes(og)
    return float(np.median(np.abs(np.fft.ifftn(pb.x_full.astype(np.complex128), axes=axes, norm="ortho"))))


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
@pytest.mark.parametrize("mode", ["soft", "l1_hard", "soft_l1"])
def test_reconstruction_soft_dc_l1_matches_oracle(H, mode, prec):
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_small_64")
    lam = 0.5 if mode.startswith("soft") else 0.0
    tau = 0.5 * _coil_image_scale(pb) if mode.endswith("l1") or mode == "l1_hard" else 0.0
    stages = [(s.off, s.ext, 6, 3, s.p) for s in pb.stages]
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel)
    pr = hicu.HICU_SPLIT_BF16 if prec == "split_bf16" else hicu.HICU_FP32
    prm = hicu.make_params(pb.rank, stages, seed=11, jl=hicu.HICU_JL_PROJECTOR, prec=pr, dc_weight=lam,
                           l1_threshold=tau)
    x_gpu, log = hicu.hicu_reconstruct(H, hg, cuda(pb.x0), cuda(pb.mask), prm, want_log=True)
    x_gpu = x_gpu.cpu().numpy()
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    st = [O.StageSpec(O.Region(off, ext), it, gd, p) for off, ext, it, gd, p in stages]
    olog = O.ReconLog([], [], [])
    x_ref = O.reconstruct(pb.x0, pb.mask, og, st, pb.rank, seed=11, jl_mode="projector", lam=lam, tau=tau,
                          log=olog)
    assert_close(x_gpu, x_ref, 1e-3, f"reconstruction {mode} ({prec})")
    assert abs(O.ser_db(pb.x_full, x_gpu) - O.ser_db(pb.x_full, x_ref)) <= 0.05
    np.testing.assert_allclose(log["objective"], olog.objective, rtol=1e-3)
    m4 = np.broadcast_to(pb.mask[None], pb.x0.shape).astype(bool)
    if lam == 0.0:
        np.testing.assert_array_equal(x_gpu[m4], pb.x0[m4])
    else:
        assert not np.array_equal(x_gpu[m4], pb.x0[m4])   # soft consistency moves observed samples
    hicu.hicu_check(H)
