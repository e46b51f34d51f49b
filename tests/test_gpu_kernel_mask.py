"""Kernel masks K (Algorithm 1 input; Discussion: circular and spherical supports) on the GPU.

The Gram matrix of the masked Hankel matrix H_K(x) (hicu_gram_support) against the oracle's, the
scatter of support-layout filters into the box (hicu_expand_filters) bit for bit, a full-box mask
giving exactly the unmasked reconstruction, and masked reconstructions (disc and sphere masks,
split-BF16 and FP32 convolutions) against the oracle's at NRMSE <= 1e-3 and SER within 0.05 dB.
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


GRAM_CASES = {
    # dims, C, kernel, circular, region (off, ext), radius
    "disc13_2d": ((40, 36, 1), 4, (5, 5, 1), (0, 0, 0), ((2, 1, 0), (36, 33, 1)), 2.0),
    "disc21_2d_wide": ((200, 20, 1), 2, (5, 5, 1), (0, 0, 0), ((0, 0, 0), (200, 20, 1)), 2.5),
    "sphere33_3d": ((30, 28, 16), 3, (5, 5, 5), (0, 0, 0), ((1, 2, 0), (28, 24, 16)), 2.0),
    "cross7_circular_t": ((24, 20, 8), 2, (3, 3, 3), (0, 0, 1), ((0, 0, 0), (24, 20, 8)), 1.0),
}


@pytest.mark.parametrize("name", list(GRAM_CASES))
def test_gram_support_parity(H, name):
    from paper_2004_08962_gb300 import hicu
    dims, C, ker, circ, (off, ext), rad = GRAM_CASES[name]
    og = O.Geom(dims, C, ker, circ, O.ellipsoid_support(ker, rad))
    km = O.support_mask(og)
    rng = np.random.default_rng(5)
    x = random_complex(rng, (C, dims[2], dims[1], dims[0])).astype(np.complex64)
    hg = hicu.make_geom(dims, C, ker, circ)
    hr = hicu.make_region(off, ext)
    assert hicu.hicu_support_length(hg, km) == og.n
    G = hicu.hicu_gram_support(H, hg, hr, km, torch.from_numpy(x).cuda()).cpu().numpy()
    ref = O.gram(x.astype(np.complex128), og, O.Region(off, ext))
    assert_close(G, ref, 1e-12, f"masked Gram {name}")
    np.testing.assert_array_equal(G, G.conj().T)
    # a second mask on the same handle (the maps are uploaded again), then the first once more
    og2 = O.Geom(dims, C, ker, circ, O.ellipsoid_support(ker, rad + 0.75))
    G2 = hicu.hicu_gram_support(H, hg, hr, O.support_mask(og2), torch.from_numpy(x).cuda()).cpu().numpy()
    assert_close(G2, O.gram(x.astype(np.complex128), og2, O.Region(off, ext)), 1e-12, f"second mask {name}")
    G3 = hicu.hicu_gram_support(H, hg, hr, km, torch.from_numpy(x).cuda()).cpu().numpy()
    np.testing.assert_array_equal(G3, G)
    hicu.hicu_check(H)


def test_expand_filters_places_the_support_in_the_box(H):
    from paper_2004_08962_gb300 import hicu
    ker = (5, 5, 5)
    og = O.Geom((20, 20, 20), 3, ker, (0, 0, 0), O.ellipsoid_support(ker, 2.0))
    rng = np.random.default_rng(2)
    v = random_complex(rng, (7, og.n)).astype(np.complex64)
    hg = hicu.make_geom(og.dims, og.ncoil, ker)
    box = hicu.hicu_expand_filters(H, hg, O.support_mask(og), torch.from_numpy(v).cuda()).cpu().numpy()
    np.testing.assert_array_equal(box, O.as_filters(v, og).reshape(7, -1))


def test_argument_errors(H):
    from paper_2004_08962_gb300 import hicu
    hg = hicu.make_geom((16, 16, 1), 2, (3, 3, 1))
    hr = hicu.make_region((0, 0, 0), (16, 16, 1))
    x = torch.zeros((2, 1, 16, 16), dtype=torch.complex64, device="cuda")
    with pytest.raises(ValueError, match="empty"):
        hicu.hicu_gram_support(H, hg, hr, np.zeros((1, 3, 3), np.uint8), x)
    with pytest.raises(ValueError, match="shape"):
        hicu.hicu_gram_support(H, hg, hr, np.ones((3, 3), np.uint8), x)
    assert hicu.hicu_support_length(hg, np.ones((1, 3, 3), np.uint8)) == 18


def _recon(H, pb, stages, support, prec, seed=5):
    from paper_2004_08962_gb300 import hicu
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel, pb.circular, support)
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
    init = 1 if pb.init == "time_average" else 0
    km = None if support is None else O.support_mask(og)
    prm = hicu.make_params(pb.rank, stages, seed=seed, jl=hicu.HICU_JL_PROJECTOR, prec=prec, init=init,
                           kernel_mask=km)
    x, log = hicu.hicu_reconstruct(H, hg, torch.from_numpy(pb.x0).cuda(), torch.from_numpy(pb.mask).cuda(), prm,
                                   want_log=True)
    return og, x.cpu().numpy(), log


def test_full_box_mask_equals_rectangular_kernel(H):
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_small_64")
    stages = [(s.off, s.ext, 3, 3, s.p) for s in pb.stages]
    box = O.ellipsoid_support(pb.kernel, 10.0)
    _, x_box, _ = _recon(H, pb, stages, None, hicu.HICU_SPLIT_BF16)
    _, x_mask, _ = _recon(H, pb, stages, box, hicu.HICU_SPLIT_BF16)
    np.testing.assert_array_equal(x_mask, x_box)


RECON_CASES = {
    # problem, scale, radius, (iters, gd_steps, p) per stage, rank
    "brain_disc21": ("2d_brain_256", 4, 2.5, [(6, 3, 8), (2, 3, 16)], 60),
    # scaled by 4: the centre region has 864 valid outputs, more than r (a rank above s would leave
    # the top-r eigenvectors undetermined inside a repeated zero eigenvalue)
    "knee_sphere33": ("knee3d_256x256x160", 4, 2.0, [(2, 2, 8), (1, 2, 8)], 100),
}


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
@pytest.mark.parametrize("name", list(RECON_CASES))
def test_masked_reconstruction_matches_oracle(H, name, prec):
    from paper_2004_08962_gb300 import hicu
    prob, scale, rad, sched, rank = RECON_CASES[name]
    pb = make_problem(prob, scale=scale)
    pb.rank = rank
    sup = O.ellipsoid_support(pb.kernel, rad)
    stages = [(st.off, st.ext, it, gd, p) for st, (it, gd, p) in zip(pb.stages, sched)]
    pr = hicu.HICU_SPLIT_BF16 if prec == "split_bf16" else hicu.HICU_FP32
    og, x_gpu, log = _recon(H, pb, stages, sup, pr)
    assert og.n == pb.ncoil * len(sup)
    ost = [O.StageSpec(O.Region(off, ext), it, gd, p) for off, ext, it, gd, p in stages]
    olog = O.ReconLog([], [], [])
    x_ref = O.reconstruct(pb.x0, pb.mask, og, ost, pb.rank, seed=5, jl_mode="projector", init=pb.init, log=olog)
    assert_close(x_gpu, x_ref, 1e-3, f"masked reconstruction {name} ({prec})")
    assert abs(O.ser_db(pb.x_full, x_gpu) - O.ser_db(pb.x_full, x_ref)) <= 0.05
    np.testing.assert_allclose(log["J"], olog.J, rtol=1e-3)
    m4 = np.broadcast_to(pb.mask[None] if pb.mask.ndim == 3 else pb.mask, pb.x0.shape).astype(bool)
    np.testing.assert_array_equal(x_gpu[m4], pb.x0[m4])
    hicu.hicu_check(H)
