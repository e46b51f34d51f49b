"""The randomized SVD null-space route (Theory: rSVD; Algorithm 1 step 2) on the GPU.

hicu_principal_rsvd against the oracle's rsvd_principal with the same test vectors (the same
counter-based draws, the same warm start): the principal subspace to 1e-4 lambda_max / gap and the
eigenvalue estimates to 1e-4 lambda_max, on 2D, 3D and kernel-mask cases and with l = 130 (the
Cholesky factorisation outside shared memory); on exactly low-rank data the subspace of eigh.  Reconstructions with
eig_solver "rsvd" against the oracle's: NRMSE <= 1e-3, SER within 0.05 dB, J per outer iteration
to 1e-3.
"""
import numpy as np
import pytest
import torch

from closeness import assert_close
from oracle import hicu_oracle as O
from synth.phantoms import lowrank_exponential_kspace, make_problem, random_complex

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2004_08962_gb300 import build, hicu
    build.build()
    return hicu.Handle()


def _proj(A, B):
    return float(np.linalg.norm(A @ A.conj().T - B @ B.conj().T, 2))


CASES = {
    # dims, C, kernel, circular, region (off, ext), r, l, kernel-mask radius (None = box); the data
    # have 10 exponentials plus a small random part, so the principal subspace at r = 10 is separated
    "2d": ((40, 36, 1), 4, (5, 5, 1), (0, 0, 0), ((2, 1, 0), (36, 33, 1)), 10, 20, None),
    "3d": ((20, 18, 12), 3, (3, 3, 3), (0, 0, 0), ((1, 1, 1), (18, 16, 10)), 10, 24, None),
    "2d_disc": ((40, 36, 1), 4, (5, 5, 1), (0, 0, 0), ((0, 0, 0), (40, 36, 1)), 10, 20, 2.0),
    "cine_circular_t": ((24, 20, 8), 2, (3, 3, 3), (0, 0, 1), ((0, 0, 0), (24, 20, 8)), 10, 20, None),
    # l = 130: the Cholesky factorisation's working copy (l^2 double-float entries) exceeds shared
    # memory and lives in the workspace
    "2d_c8_l130": ((48, 44, 1), 8, (5, 5, 1), (0, 0, 0), ((0, 0, 0), (48, 44, 1)), 10, 130, None),
}


@pytest.mark.parametrize("name", list(CASES))
def test_rsvd_parity(H, name):
    from paper_2004_08962_gb300 import hicu
    dims, C, ker, circ, (off, ext), r, l, rad = CASES[name]
    sup = None if rad is None else O.ellipsoid_support(ker, rad)
    og, oreg = O.Geom(dims, C, ker, circ, sup), O.Region(off, ext)
    rng = np.random.default_rng(11)
    # k-space-like data: smooth low-rank part plus a small random part (a decaying spectrum)
    x = (lowrank_exponential_kspace(rng, (dims[2], dims[1], dims[0]), C, 10)
         + 0.01 * random_complex(rng, (C, dims[2], dims[1], dims[0]))).astype(np.complex64)
    hg, hr = hicu.make_geom(dims, C, ker, circ), hicu.make_region(off, ext)
    km = None if sup is None else O.support_mask(og)
    xt = torch.from_numpy(x).cuda()
    w = np.linalg.eigvalsh(O.gram(x.astype(np.complex128), og, oreg))
    lmax = w[-1]
    # cold start, then a warm start from the first result
    V1, e1, t1 = hicu.hicu_principal_rsvd(H, hg, hr, xt, r, l, seed=4, counter=0, kmask=km, want_tail=True)
    V1o, e1o = O.rsvd_principal(x.astype(np.complex128), og, oreg, r, l, seed=4, counter=0)
    V2, e2 = hicu.hicu_principal_rsvd(H, hg, hr, xt, r, l, V_prev=V1, seed=4, counter=1, kmask=km)
    V2o, e2o = O.rsvd_principal(x.astype(np.complex128), og, oreg, r, l, seed=4, counter=1, V_prev=V1o)
    hicu.hicu_check(H)
    for V, e, Vo, eo in ((V1, e1, V1o, e1o), (V2, e2, V2o, e2o)):
        V = V.cpu().numpy().T
        e = e.cpu().numpy()
        assert np.max(np.abs(e - eo)) <= 1e-4 * lmax, (np.max(np.abs(e - eo)) / lmax)
        gap = eo[0] - np.sort(w)[::-1][r]
        assert gap > 1e-3 * lmax
        assert _proj(V, Vo) <= 1e-4 * lmax / gap, (_proj(V, Vo), gap / lmax)
        np.testing.assert_allclose(V.conj().T @ V, np.eye(r), atol=1e-6)
    # J = trace(G) - sum of the estimates
    assert abs(t1.item() - (np.sum(w) - np.sum(e1o))) <= 1e-4 * np.sum(w)


def test_rsvd_exact_on_low_rank_data(H):
    from paper_2004_08962_gb300 import hicu
    rng = np.random.default_rng(2)
    L = 6
    x = lowrank_exponential_kspace(rng, (1, 30, 32), 3, L).astype(np.complex64)
    og = O.Geom((32, 30, 1), 3, (5, 5, 1))
    hg, hr = hicu.make_geom(og.dims, 3, og.kernel), hicu.make_region((0, 0, 0), og.dims)
    V, e = hicu.hicu_principal_rsvd(H, hg, hr, torch.from_numpy(x).cuda(), L, L + 4, seed=1)
    G = O.gram(x.astype(np.complex128), og, O.full_region(og))
    w, U = np.linalg.eigh(G)
    # exact but for the stabilising shift nu: a perturbation of relative size nu / lambda_L
    nu = O.RSVD_SHIFT * np.linalg.norm(G @ O.complex_gaussian(1, 0, og.n, L + 4)) / np.sqrt(L + 4)
    assert _proj(V.cpu().numpy().T, U[:, -L:]) < 5 * nu / w[-L]
    # the estimates carry the shifted approximation's own bias (tens of nu below the eigenvalues
    # at l < n): they follow the oracle's, and stay below the eigenvalues
    _, eo = O.rsvd_principal(x.astype(np.complex128), og, O.full_region(og), L, L + 4, seed=1, counter=0)
    np.testing.assert_allclose(e.cpu().numpy(), eo, rtol=1e-5)
    assert np.all(e.cpu().numpy() <= w[-L:] * (1 + 1e-6))


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
@pytest.mark.parametrize("name", ["2d_small_64", "2d_brain_256"])
def test_rsvd_reconstruction_matches_oracle(H, name, prec):
    from paper_2004_08962_gb300 import hicu
    pb = make_problem(name, scale=1 if name == "2d_small_64" else 2)
    sched = [(4, 3, pb.stages[0].p)] if len(pb.stages) == 1 else [(4, 3, 8), (2, 3, 16)]
    stages = [(st.off, st.ext, it, gd, p) for st, (it, gd, p) in zip(pb.stages, sched)]
    l = pb.rank + max(pb.rank // 2, 8)
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel)
    pr = hicu.HICU_SPLIT_BF16 if prec == "split_bf16" else hicu.HICU_FP32
    prm = hicu.make_params(pb.rank, stages, seed=11, jl=hicu.HICU_JL_PROJECTOR, prec=pr, eig_solver="rsvd",
                           rsvd_cols=l, rsvd_seed=23)
    x_gpu, log = hicu.hicu_reconstruct(H, hg, torch.from_numpy(pb.x0).cuda(), torch.from_numpy(pb.mask).cuda(),
                                       prm, want_log=True)
    x_gpu = x_gpu.cpu().numpy()
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    st = [O.StageSpec(O.Region(off, ext), it, gd, p) for off, ext, it, gd, p in stages]
    olog = O.ReconLog([], [], [])
    x_ref = O.reconstruct(pb.x0, pb.mask, og, st, pb.rank, seed=11, jl_mode="projector", rsvd=(l, 23), log=olog)
    assert_close(x_gpu, x_ref, 1e-3, f"rsvd reconstruction {name} ({prec})")
    assert abs(O.ser_db(pb.x_full, x_gpu) - O.ser_db(pb.x_full, x_ref)) <= 0.05
    np.testing.assert_allclose(log["J"], olog.J, rtol=1e-3)
    m4 = np.broadcast_to(pb.mask[None], pb.x0.shape).astype(bool)
    np.testing.assert_array_equal(x_gpu[m4], pb.x0[m4])
    hicu.hicu_check(H)
