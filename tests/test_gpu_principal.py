"""Principal subspace by Householder tridiagonalisation (hicu_principal_subspace) and the
complement form of the JL filters, against LAPACK's eigh in the FP64 oracle.

The solver computes in double-float (FP32 pairs, unit roundoff u = 2^-48 ~ 3.6e-15, a few u per
operation).  Bounds: eigenvalues to 2e-12 lambda_max (bisection to 2^-46 ||T|| on a
backward-stable tridiagonal form whose backward error grows like sqrt(n) u ||G||); span of the r
principal vectors to 2e-12 lambda_max / gap (Davis-Kahan with that backward error);
orthonormality 1e-11; J of Eq. 1 (tail energy) to 1e-11 lambda_max n.
"""
import numpy as np
import pytest
import torch

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


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(H, G, r, span_tol=2e-12):
    from paper_2004_08962_gb300 import hicu
    n = G.shape[0]
    V, top, allv, tail = hicu.hicu_principal_subspace(H, cuda(G), r, want_all=True, want_tail=True)
    hicu.hicu_check(H)
    V = V.cpu().numpy().T          # (n, r) columns
    top, allv, tail = top.cpu().numpy(), allv.cpu().numpy(), tail.item()
    w, U = np.linalg.eigh(G)
    lmax = max(abs(w[0]), abs(w[-1]))
    assert np.max(np.abs(allv - w)) < 2e-12 * lmax
    assert np.max(np.abs(top - w[n - r:])) < 2e-12 * lmax
    np.testing.assert_allclose(V.conj().T @ V, np.eye(r), atol=1e-11)
    gap = w[n - r] - w[n - r - 1]
    Uo = U[:, n - r:]
    dist = np.linalg.norm(V @ V.conj().T - Uo @ Uo.conj().T, 2)
    assert dist < span_tol * lmax / max(gap, 1e-300) + 1e-12, (dist, gap / lmax)
    J = w[: n - r].sum()
    assert abs(tail - max(J, 0.0)) < 1e-11 * lmax * n
    return V


def test_principal_phantom_64(H):
    pb = make_problem("2d_small_64")
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    G = O.gram(pb.x0.astype(np.complex128), og, O.full_region(og))
    _check(H, G, pb.rank)


def test_principal_brain_centre_region(H):
    pb = make_problem("2d_brain_256")
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    st = pb.stages[0]
    G = O.gram(pb.x0.astype(np.complex128), og, O.Region(st.off, st.ext))
    _check(H, G, pb.rank)


@pytest.mark.parametrize("n,r", [(2, 1), (3, 2), (17, 5), (129, 40), (257, 100), (416, 150), (417, 150),
                                 (1000, 300)])
def test_principal_sizes(H, n, r):
    """Decaying spectra like a Gram of a low-rank Hankel matrix, from the smallest size to the
    n = 1000 of the 5 x 5 x 5 x 8 kernels; 416 and 417 are the largest one-cluster and the
    smallest grid tridiagonalisation."""
    rng = np.random.default_rng(n)
    U, _ = np.linalg.qr(random_complex(rng, (n, n)))
    sv = np.exp(-np.arange(n) / (n / 12.0))
    G = (U * sv**2) @ U.conj().T * 1e3
    G = (G + G.conj().T) / 2
    _check(H, G, r)


def test_principal_repeated_and_zero_eigenvalues(H):
    """Exactly repeated top eigenvalues (solved one after the other and orthogonalised) and an
    exactly rank-deficient Gram (eigenvalue 0 of multiplicity n - 4)."""
    rng = np.random.default_rng(5)
    n = 40
    U, _ = np.linalg.qr(random_complex(rng, (n, n)))
    w = np.concatenate([np.linspace(0.0, 1e-3, 20), np.full(10, 1.0), np.full(10, 5.0)])
    _check(H, (U * w) @ U.conj().T, 15)
    x = lowrank_exponential_kspace(rng, (1, 14, 13), 1, 4)
    og = O.Geom((13, 14, 1), 1, (3, 3, 1))
    G = O.gram(x, og, O.full_region(og))
    _check(H, G, 4)


def test_principal_scale_invariance(H):
    """The power-of-two pre-scale makes results bit-identical under G -> 2^k G."""
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_small_64")
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    G = O.gram(pb.x0.astype(np.complex128), og, O.full_region(og))
    V1, t1 = hicu.hicu_principal_subspace(H, cuda(G), pb.rank)
    for k in (-700, 600):
        Vk, tk = hicu.hicu_principal_subspace(H, cuda(G * 2.0**k), pb.rank)
        assert torch.equal(V1, Vk)
        assert torch.equal(t1 * 2.0**k, tk)


def test_jl_complement_equals_projector(H):
    """Q~ = P - V (V^H P) from the principal vectors equals Q~ = Q (Q^H P) from the null basis
    (same draws of P), because I - V V^H = Q Q^H."""
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_small_64")
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    G = O.gram(pb.x0.astype(np.complex128), og, O.full_region(og))
    n, r = og.n, pb.rank
    w, U = np.linalg.eigh(G)
    Q = U[:, : n - r].T.copy()
    V = U[:, n - r:].T.copy()
    p = 6
    fq = hicu.hicu_jl_compress(H, cuda(Q), p, mode=hicu.HICU_JL_PROJECTOR, seed=3, counter=7).cpu().numpy()
    fv = hicu.hicu_jl_compress(H, cuda(V), p, mode=hicu.HICU_JL_COMPLEMENT, seed=3, counter=7).cpu().numpy()
    Pm = O.jl_matrix(3, 7, n, p)
    ref = O.jl_compress(Q.T, Pm, "projector")
    assert np.linalg.norm(fv - ref) < 2e-6 * np.linalg.norm(ref)
    assert np.linalg.norm(fv - fq) < 2e-6 * np.linalg.norm(ref)


def test_principal_argument_errors(H):
    from paper_2004_08962_gb300 import hicu
    G = cuda(np.eye(4, dtype=np.complex128))
    for r in (0, 4):
        with pytest.raises(hicu.HicuError) as e:
            hicu.hicu_principal_subspace(H, G, r)
        assert e.value.status == 3
    hicu.hicu_check(H)
