"""The 2D+t cine (192 x 144 x 24 frames, 8 coils, 5 x 5 x 5 kernel, circular time, n = 1000) and
3D knee (256 x 256 x 160, 8 coils, 5 x 5 x 5 kernel, n = 1000) workloads on the GPU.

Full size, one descent step as the reconstruction runs it (split-BF16 tensor cores, and the
plain FP32 form): the convolution R = H(y) q~ at 400 sampled outputs and the masked gradient
g = (1 - M) o H^H H(y) q~ at 48 sampled positions against the FP64 oracle's sampled forms
(conv_null_at, gradient_at); the exact line search against its closed form, the objective
decrease phi(0) - phi(eta) = ||g||^4 / D (Theory, ELS paragraph), which holds at any size.
Bounds: R and g to 2e-5 / 1e-4 relative (FP32 accumulation over n = 1000 terms; the north-star
bound for the split-BF16 gradient is 1e-3), the decrease to 1e-3.

Scaled down (cine 96 x 72 x 24, knee 64 x 64 x 40), a short centre-out reconstruction against the
oracle's: NRMSE <= 1e-3 and SER within 0.05 dB.
"""
import numpy as np
from closeness import assert_close
import pytest
import torch

from oracle import hicu_oracle as O
from synth.phantoms import make_problem, random_complex

pytestmark = pytest.mark.gpu

WORKLOADS = ["cine_192x144x24", "knee3d_256x256x160"]


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2004_08962_gb300 import build, hicu
    build.build()
    return hicu.Handle()


@pytest.fixture(scope="module")
def problems():
    return {name: make_problem(name) for name in WORKLOADS}




def _setup(pb, seed, p=8):
    from paper_2004_08962_gb300 import hicu
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
    reg = O.full_region(og)
    rng = np.random.default_rng(seed)
    f = (random_complex(rng, (p, og.n)) / np.sqrt(og.n)).astype(np.complex64)
    y = O.initial_estimate(pb.x0.astype(np.complex128), pb.mask,
                           "time_average" if pb.init == "time_average" else "zero_filled").astype(np.complex64)
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
    hr = hicu.make_region((0, 0, 0), pb.dims)
    return og, reg, rng, f, y, hg, hr


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
@pytest.mark.parametrize("name", WORKLOADS)
def test_full_size_step_sampled(H, problems, name, prec):
    from paper_2004_08962_gb300 import hicu
    pb = problems[name]
    og, reg, rng, f, y, hg, hr = _setup(pb, seed=21)
    pr = hicu.HICU_SPLIT_BF16 if prec == "split_bf16" else hicu.HICU_FP32
    fb = torch.from_numpy(f).cuda()
    yd = torch.from_numpy(y).cuda()
    md = torch.from_numpy(pb.mask).cuda()
    # convolution at sampled outputs
    R = hicu.hicu_conv_null(H, hg, hr, yd, fb, prec=pr)
    sz, sy, sx = O.out_shape(og, reg)
    outs = np.stack([rng.integers(0, sz, 400), rng.integers(0, sy, 400), rng.integers(0, sx, 400)], -1)
    Rg = R[torch.from_numpy(outs[:, 0]).cuda(), torch.from_numpy(outs[:, 1]).cuda(),
           torch.from_numpy(outs[:, 2]).cuda()].cpu().numpy()
    fo = O.as_filters(f.astype(np.complex128), og)
    Ro = O.conv_null_at(y, og, reg, fo, outs)
    assert_close(Rg, Ro, 2e-5)
    # masked gradient at sampled positions (including the region's borders)
    g = hicu.hicu_conv_null_adjoint(H, hg, hr, R, fb, mask=md, prec=pr)
    nx, ny, nz = pb.dims
    us = np.stack([rng.integers(0, nz, 48), rng.integers(0, ny, 48), rng.integers(0, nx, 48)], -1)
    us[:4] = [[0, 0, 0], [nz - 1, ny - 1, nx - 1], [0, ny - 1, 0], [nz - 1, 0, nx - 1]]
    gg = g[:, torch.from_numpy(us[:, 0]).cuda(), torch.from_numpy(us[:, 1]).cuda(),
           torch.from_numpy(us[:, 2]).cuda()].cpu().numpy()
    go = O.gradient_at(y, og, reg, fo, us, pb.mask)
    assert_close(gg, go, 1e-4)
    # one descent step: eta = ||g||^2 / D and the closed-form decrease of the objective
    stats = hicu.hicu_gd_step_filters(H, hg, hr, yd, md, fb, prec=pr).cpu().numpy()
    eta, obj0, gn2, D = stats
    assert abs(eta - gn2 / D) <= 1e-12 * eta
    _, obj1 = hicu.hicu_conv_null(H, hg, hr, yd, fb, prec=pr, want_objective=True, store_R=False)
    decrease = obj0 - obj1.item()
    assert abs(decrease - gn2 * gn2 / D) < 1e-3 * gn2 * gn2 / D
    # observed entries untouched
    m4 = np.broadcast_to(pb.mask[None], y.shape).astype(bool)
    np.testing.assert_array_equal(yd.cpu().numpy()[m4], y[m4])
    hicu.hicu_check(H)


SHORT = {"cine_192x144x24": (2, [(2, 2, 8), (1, 2, 8)]),
         "knee3d_256x256x160": (4, [(2, 2, 8), (1, 2, 8)])}


@pytest.mark.parametrize("name", WORKLOADS)
def test_scaled_reconstruction_matches_oracle(H, name):
    """Centre-out schedule shortened to (iters, gd_steps, p) per stage on the workload scaled down;
    the null space by tridiagonalisation (n = 1000), split-BF16 convolutions, circular time and
    the time-averaged start for the cine."""
    from paper_2004_08962_gb300 import hicu
    scale, sched = SHORT[name]
    pb = make_problem(name, scale=scale)
    stages = [(st.off, st.ext, it, gd, p) for st, (it, gd, p) in zip(pb.stages, sched)]
    init = 1 if pb.init == "time_average" else 0
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
    prm = hicu.make_params(pb.rank, stages, seed=5, jl=hicu.HICU_JL_PROJECTOR, prec=hicu.HICU_SPLIT_BF16,
                           init=init)
    x_gpu = hicu.hicu_reconstruct(H, hg, torch.from_numpy(pb.x0).cuda(), torch.from_numpy(pb.mask).cuda(),
                                  prm).cpu().numpy()
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
    ost = [O.StageSpec(O.Region(off, ext), it, gd, p) for off, ext, it, gd, p in stages]
    x_ref = O.reconstruct(pb.x0, pb.mask, og, ost, pb.rank, seed=5, jl_mode="projector", init=pb.init)
    assert_close(x_gpu, x_ref, 1e-3)
    assert abs(O.ser_db(pb.x_full, x_gpu) - O.ser_db(pb.x_full, x_ref)) <= 0.05
