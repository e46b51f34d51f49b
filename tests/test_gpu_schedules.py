"""The 2D brain slice's whole centre-out schedule, as the benchmark times it, against the oracle.

256 x 256 k-space, 8 coils, 5 x 5 kernel (n = 200), rank 75: centre-out stage on the central
64 x 64 region (50 outer iterations x 5 descent steps, p = 8), then full k-space (10 x 10, p = 32):
60 Gram + principal-subspace updates and 350 descent steps with exact line search (Algorithm 1),
JL draws in projector form from seed 11.  The GPU runs it once with split-BF16 tensor-core
convolutions and once in plain complex FP32; the FP64 oracle runs it once (a few minutes on the
host cores).  Bounds (the benchmark spec): NRMSE <= 1e-3 against the oracle's final iterate, entry by
entry as well as in norm, and SER within 0.05 dB of the oracle's; observed entries bit-identical.
"""
import numpy as np
import pytest
import torch

from closeness import assert_close
from oracle import hicu_oracle as O
from synth.phantoms import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2004_08962_gb300 import build, hicu
    build.build()
    return hicu.Handle()


@pytest.fixture(scope="module")
def brain():
    pb = make_problem("2d_brain_256")
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
    st = [O.StageSpec(O.Region(s.off, s.ext), s.iters, s.gd_steps, s.p) for s in pb.stages]
    log = O.ReconLog([], [], [])
    x_ref = O.reconstruct(pb.x0, pb.mask, og, st, pb.rank, seed=11, jl_mode="projector", log=log)
    return pb, x_ref, log


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
def test_brain_schedule_matches_oracle(H, brain, prec):
    from paper_2004_08962_gb300 import hicu
    pb, x_ref, olog = brain
    assert [(s.iters, s.gd_steps, s.p) for s in pb.stages] == [(50, 5, 8), (10, 10, 32)]
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
    pr = hicu.HICU_SPLIT_BF16 if prec == "split_bf16" else hicu.HICU_FP32
    prm = hicu.make_params(pb.rank, [(s.off, s.ext, s.iters, s.gd_steps, s.p) for s in pb.stages],
                           seed=11, jl=hicu.HICU_JL_PROJECTOR, prec=pr)
    x_gpu, log = hicu.hicu_reconstruct(H, hg, torch.from_numpy(pb.x0).cuda(), torch.from_numpy(pb.mask).cuda(),
                                       prm, want_log=True)
    x_gpu = x_gpu.cpu().numpy()
    assert_close(x_gpu, x_ref, 1e-3, f"brain schedule ({prec})")
    ser_g, ser_o = O.ser_db(pb.x_full, x_gpu), O.ser_db(pb.x_full, x_ref)
    assert abs(ser_g - ser_o) <= 0.05, (ser_g, ser_o)
    assert ser_o > O.ser_db(pb.x_full, pb.x0) + 1.0   # the synthetic slice gains about 1.3 dB
    # J of Eq. 1 per outer iteration follows the oracle's
    np.testing.assert_allclose(log["J"], olog.J, rtol=1e-3)
    m4 = np.broadcast_to(pb.mask[None], pb.x0.shape).astype(bool)
    np.testing.assert_array_equal(x_gpu[m4], pb.x0[m4])
    hicu.hicu_check(H)
