"""The augmented null space [Q | Q+] of the multi-shot diffusion study (Methods, Study IV) on the GPU.

A scaled multi-shot slice (64 x 64, 2 coils x 4 shots stacked as 8 channels, per-shot phases,
interleaved shots inside a partial-Fourier extent of 59 % of the phase-encode lines) with its b0
data.  Q0 = the 10 null vectors of the b0 Gram (kernel 5 x 5 over the 2 coils); Q+ =
blockdiag(Q0, Q0, Q0, Q0).  The schedule: centre-out on the central 16 x 16 region, then the
partial-Fourier sampled region.  Against the oracle's reconstruction with the same Q0: NRMSE <= 1e-3,
SER within 0.05 dB, in both precisions and without compression (FP32).  The b0 null space computed
on the GPU (hicu_gram + hicu_nullspace) spans the oracle's.
"""
import numpy as np
import pytest
import torch

from closeness import assert_close
from oracle import hicu_oracle as O
from synth.phantoms import make_msdwi

pytestmark = pytest.mark.gpu

C0, S, M0 = 2, 4, 10


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2004_08962_gb300 import build, hicu
    build.build()
    return hicu.Handle()


@pytest.fixture(scope="module")
def case():
    pb, xb0 = make_msdwi(n=64, C=C0, S=S, co_iters=6, co_steps=4, pf_steps=8, rank=20)
    g0 = O.Geom((64, 64, 1), C0, (5, 5, 1))
    reg0 = O.Region((16, 16, 0), (32, 32, 1))
    G0 = O.gram(xb0.astype(np.complex128), g0, reg0)
    Q0, w0 = O.nullspace(G0, g0.n - M0)
    return pb, xb0, g0, reg0, Q0, w0


@pytest.mark.parametrize("mode", ["split_bf16", "fp32", "exact_fp32"])
def test_augmented_reconstruction_matches_oracle(H, case, mode):
    from paper_2004_08962_gb300 import hicu
    pb, xb0, g0, reg0, Q0, w0 = case
    stages = [(s.off, s.ext, s.iters, s.gd_steps, s.p) for s in pb.stages]
    assert stages[1][0][1] == 26 and stages[1][1][1] == 38   # the partial-Fourier sampled rows
    q0 = torch.from_numpy(np.ascontiguousarray(Q0.T)).cuda()   # [m0][n0]
    pr = hicu.HICU_SPLIT_BF16 if mode == "split_bf16" else hicu.HICU_FP32
    exact = mode == "exact_fp32"
    prm = hicu.make_params(pb.rank, stages, seed=3, jl=hicu.HICU_JL_PROJECTOR, prec=pr, qplus=q0, qplus_blocks=S,
                           jl_exact=exact)
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel, mask_per_coil=True)
    x_gpu, log = hicu.hicu_reconstruct(H, hg, torch.from_numpy(pb.x0).cuda(), torch.from_numpy(pb.mask).cuda(),
                                       prm, want_log=True)
    x_gpu = x_gpu.cpu().numpy()
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    ost = [O.StageSpec(O.Region(off, ext), it, gd, p) for off, ext, it, gd, p in stages]
    olog = O.ReconLog([], [], [])
    x_ref = O.reconstruct(pb.x0, pb.mask, og, ost, pb.rank, seed=3, jl_mode="exact" if exact else "projector",
                          qplus=(Q0, S), log=olog)
    assert_close(x_gpu, x_ref, 1e-3, f"augmented reconstruction ({mode})")
    assert abs(O.ser_db(pb.x_full, x_gpu) - O.ser_db(pb.x_full, x_ref)) <= 0.05
    np.testing.assert_allclose(log["objective"], olog.objective, rtol=1e-3)
    obs = pb.mask.astype(bool)
    np.testing.assert_array_equal(x_gpu[obs], pb.x0[obs])
    # rows outside the partial-Fourier extent and the centre region stay as they were
    np.testing.assert_array_equal(x_gpu[:, :, :20, :], pb.x0[:, :, :20, :])
    hicu.hicu_check(H)


def test_b0_null_space_on_the_gpu(H, case):
    from paper_2004_08962_gb300 import hicu
    pb, xb0, g0, reg0, Q0, w0 = case
    hg0 = hicu.make_geom((64, 64, 1), C0, (5, 5, 1))
    G = hicu.hicu_gram(H, hg0, hicu.make_region(reg0.off, reg0.ext), torch.from_numpy(xb0).cuda())
    Qg, eig = hicu.hicu_nullspace(H, G, g0.n - M0)
    Qg = Qg.cpu().numpy().T              # (n0, m0) columns
    lmax = w0[-1]
    gap = w0[M0] - w0[M0 - 1]
    dist = np.linalg.norm(Qg @ Qg.conj().T - Q0 @ Q0.conj().T, 2)
    assert dist < 1e-10 * lmax / gap + 1e-12, (dist, gap / lmax)
    np.testing.assert_allclose(eig.cpu().numpy(), w0, atol=1e-10 * lmax)


def test_augmentation_argument_errors(H, case):
    from paper_2004_08962_gb300 import hicu
    pb, xb0, g0, reg0, Q0, w0 = case
    stages = [(s.off, s.ext, 1, 1, s.p) for s in pb.stages]
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel, mask_per_coil=True)
    q0 = torch.from_numpy(np.ascontiguousarray(Q0.T)).cuda()
    prm = hicu.make_params(pb.rank, stages, seed=3, qplus=q0, qplus_blocks=3)   # 3 does not divide 8 channels
    with pytest.raises(ValueError):
        hicu.hicu_reconstruct(H, hg, torch.from_numpy(pb.x0).cuda(), torch.from_numpy(pb.mask).cuda(), prm)
