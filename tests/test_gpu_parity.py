"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Operator-level cases use random complex data and random filters (no cancellation), so the
complex-FP32 path must match to a few ulps of the accumulation length.  Step-level cases use
phantom k-space and null-space filters, where the benchmark spec's bound for the plain FP32 form is a
gradient relative error <= 1e-4.  Integer-like outcomes (untouched observed entries, untouched
entries outside the region) are compared bit for bit.
"""
import numpy as np
from closeness import assert_close
import pytest
import torch

from oracle import hicu_oracle as O
from synth.phantoms import lowrank_exponential_kspace, make_problem, random_complex

pytestmark = pytest.mark.gpu

# dims (Nx, Ny, Nz), C, kernel, circular, region (off, ext), p
CASES = {
    "2d_64_c4_p4": ((64, 64, 1), 4, (5, 5, 1), (0, 0, 0), ((0, 0, 0), (64, 64, 1)), 4),
    "2d_odd_region": ((70, 45, 1), 3, (5, 3, 1), (0, 0, 0), ((3, 2, 0), (61, 40, 1)), 5),
    "3d_region": ((20, 18, 12), 2, (3, 3, 3), (0, 0, 0), ((1, 2, 1), (17, 14, 10)), 3),
    "cine_circular_t": ((24, 20, 8), 2, (3, 3, 3), (0, 0, 1), ((0, 0, 0), (24, 20, 8)), 8),
    "2d_c16_p20": ((40, 38, 1), 16, (3, 3, 1), (0, 0, 0), ((2, 1, 0), (36, 35, 1)), 20),
    "2d_c32_permask": ((36, 33, 1), 32, (3, 3, 1), (0, 0, 0), ((0, 0, 0), (36, 33, 1)), 8),
    "tiny_one_output": ((9, 9, 1), 2, (5, 5, 1), (0, 0, 0), ((2, 3, 0), (5, 5, 1)), 1),
}




@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2004_08962_gb300 import build, hicu
    build.build()
    return hicu.Handle()


def setup(name, seed=0):
    from paper_2004_08962_gb300 import hicu
    dims, C, ker, circ, (off, ext), p = CASES[name]
    og = O.Geom(dims, C, ker, circ)
    oreg = O.Region(off, ext)
    per_coil = name.endswith("permask")
    hg = hicu.make_geom(dims, C, ker, circ, mask_per_coil=per_coil)
    hr = hicu.make_region(off, ext)
    rng = np.random.default_rng(seed)
    x = random_complex(rng, (C, dims[2], dims[1], dims[0])).astype(np.complex64)
    f = random_complex(rng, (p, og.n)).astype(np.complex64)
    mshape = (C, dims[2], dims[1], dims[0]) if per_coil else (dims[2], dims[1], dims[0])
    mask = (rng.random(mshape) < 0.35).astype(np.uint8)
    return og, oreg, hg, hr, x, f, mask, p, rng


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def ofilters(f, og):
    return O.as_filters(f.astype(np.complex128), og)


@pytest.mark.parametrize("name", list(CASES))
def test_conv_null_parity(H, name):
    from paper_2004_08962_gb300 import hicu
    og, oreg, hg, hr, x, f, mask, p, _ = setup(name)
    R, obj = hicu.hicu_conv_null(H, hg, hr, cuda(x), cuda(f), want_objective=True)
    ref = O.conv_null(x.astype(np.complex128), og, oreg, ofilters(f, og))
    assert R.shape == ref.shape
    assert_close(R.cpu().numpy(), ref, 5e-6)
    assert abs(obj.item() - np.vdot(ref, ref).real) < 1e-5 * np.vdot(ref, ref).real


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_parity(H, name):
    from paper_2004_08962_gb300 import hicu
    og, oreg, hg, hr, x, f, mask, p, rng = setup(name, seed=1)
    R = random_complex(rng, O.out_shape(og, oreg) + (p,)).astype(np.complex64)
    sentinel = np.full(x.shape, 7.0 + 3.0j, dtype=np.complex64)
    gt = cuda(sentinel)
    g, gn = hicu.hicu_conv_null_adjoint(H, hg, hr, cuda(R), cuda(f), mask=cuda(mask), g=gt,
                                        want_gnorm2=True)
    ref = O.conv_null_adjoint(R.astype(np.complex128), og, oreg, ofilters(f, og), mask)
    g = g.cpu().numpy()
    inside = np.zeros(x.shape[1:], dtype=bool)
    (ox, oy, oz), (ex, ey, ez) = CASES[name][4]
    inside[oz:oz + ez, oy:oy + ey, ox:ox + ex] = True
    assert_close(g[:, inside], ref[:, inside], 5e-6)
    np.testing.assert_array_equal(g[:, ~inside], sentinel[:, ~inside])  # outside S untouched
    m4 = np.broadcast_to(mask if mask.ndim == 4 else mask[None], x.shape).astype(bool)
    assert np.all(g[m4 & inside[None]] == 0)                            # observed -> exactly 0
    assert abs(gn.item() - np.vdot(ref, ref).real) < 1e-5 * np.vdot(ref, ref).real
    # unmasked adjoint too
    g2 = hicu.hicu_conv_null_adjoint(H, hg, hr, cuda(R), cuda(f)).cpu().numpy()
    ref2 = O.conv_null_adjoint(R.astype(np.complex128), og, oreg, ofilters(f, og))
    assert_close(g2, ref2, 5e-6)


@pytest.mark.parametrize("name", list(CASES))
def test_gd_step_filters_parity(H, name):
    from paper_2004_08962_gb300 import hicu
    og, oreg, hg, hr, x, f, mask, p, _ = setup(name, seed=2)
    y = cuda(x)
    stats = hicu.hicu_gd_step_filters(H, hg, hr, y, cuda(mask), cuda(f)).cpu().numpy()
    y1_ref, info = O.gd_step(x, mask, og, oreg, ofilters(f, og))
    for got, want in zip(stats, (info.eta, info.objective, info.gnorm2, info.denom)):
        assert abs(got - want) <= 2e-5 * abs(want) + 1e-300
    y1 = y.cpu().numpy()
    assert_close(y1 - x, y1_ref - x, 2e-5)
    m4 = np.broadcast_to(mask if mask.ndim == 4 else mask[None], x.shape).astype(bool)
    np.testing.assert_array_equal(y1[m4], x[m4])                         # data consistency
    inside = np.zeros(x.shape[1:], dtype=bool)
    (ox, oy, oz), (ex, ey, ez) = CASES[name][4]
    inside[oz:oz + ez, oy:oy + ey, ox:ox + ex] = True
    np.testing.assert_array_equal(y1[:, ~inside], x[:, ~inside])         # outside S untouched


# Gram cases for each form: lag-row (every x lag in one thread; kx, ky <= 5 and regions up to 128
# wide, x-lag counts 1, 5, 7, 9, a circular y axis with one y cell), row-streaming (129 .. 256
# wide) and cells (wider)
CASES["gram_w128_k5x3"] = ((128, 20, 1), 3, (5, 3, 1), (0, 0, 0), ((0, 2, 0), (128, 17, 1)), 2)
CASES["gram_w200_rows"] = ((200, 12, 1), 2, (3, 3, 1), (0, 0, 0), ((0, 0, 0), (200, 12, 1)), 2)
CASES["gram_k1x_3d"] = ((10, 12, 9), 2, (1, 3, 3), (0, 0, 0), ((1, 1, 1), (8, 11, 8)), 2)
CASES["gram_k4x_2d"] = ((30, 20, 1), 3, (4, 2, 1), (0, 0, 0), ((1, 0, 0), (29, 20, 1)), 2)
CASES["gram_circ_y_3d"] = ((20, 16, 6), 2, (3, 3, 3), (0, 1, 0), ((0, 0, 0), (20, 16, 6)), 2)


@pytest.mark.parametrize("name", ["2d_64_c4_p4", "2d_odd_region", "3d_region", "cine_circular_t",
                                  "2d_c16_p20", "tiny_one_output", "2d_wide_two_x_tiles", "3d_c8_k5_region",
                                  "cine_c8_k5_circular_t", "gram_w128_k5x3", "gram_w200_rows", "gram_k1x_3d",
                                  "gram_k4x_2d", "gram_circ_y_3d"])
def test_gram_parity(H, name):
    """Regions up to 128 positions wide with kx, ky <= 5 run the lag-row kernel, up to 256 the
    row-streaming kernel, wider ones the cell kernel."""
    from paper_2004_08962_gb300 import hicu
    og, oreg, hg, hr, x, f, mask, p, _ = setup(name, seed=3)
    G = hicu.hicu_gram(H, hg, hr, cuda(x)).cpu().numpy()
    ref = O.gram(x.astype(np.complex128), og, oreg)
    assert_close(G, ref, 1e-12)
    np.testing.assert_array_equal(G, G.conj().T)                         # exactly Hermitian


def test_gram_phantom_config1(H):
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_small_64")
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    reg = O.full_region(og)
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel)
    G = hicu.hicu_gram(H, hg, hicu.make_region((0, 0, 0), pb.dims), cuda(pb.x0)).cpu().numpy()
    ref = O.gram(pb.x0.astype(np.complex128), og, reg)
    assert_close(G, ref, 1e-12)


DF_U = 2.0**-48   # unit roundoff of double-float (FP32 pair) arithmetic


def _uses_cluster(n, solver):
    return solver == "cluster" or (solver is None and n <= 128)


def _orth_tol(H, n, solver):
    """Orthonormality bound of the returned basis.  Grid solver (FP64): 1e-12.  Cluster solver
    (double-float, n <= 256): each rotation is unitary to a few u and each V update rounds to a
    few u, so the error is a random walk over the K = sweeps x (n_pad - 1) rotations a column
    goes through; 40 u sqrt(K) covers the largest of the n^2 entries of Q^H Q."""
    from paper_2004_08962_gb300 import hicu
    if not _uses_cluster(n, solver):
        return 1e-12
    sweeps, _ = hicu.hicu_nullspace_info(H)
    return max(1e-12, 40 * DF_U * np.sqrt(sweeps * (n + 32)))


def _nullspace_check(Q, eig, ref_G, r, orth_atol=1e-12):
    w, V = np.linalg.eigh(ref_G)
    n = ref_G.shape[0]
    lmax = abs(w).max()
    assert np.max(np.abs(eig - w)) < 1e-11 * lmax
    Qh = Q.T  # (n, n-r)
    np.testing.assert_allclose(Qh.conj().T @ Qh, np.eye(n - r), atol=orth_atol)
    res = ref_G @ Qh - Qh * eig[: n - r]
    assert np.linalg.norm(res) < 1e-11 * lmax * np.sqrt(n)
    Qo = V[:, : n - r]
    gap = w[n - r] - w[n - r - 1]
    dist = np.linalg.norm(Qh @ Qh.conj().T - Qo @ Qo.conj().T)
    assert dist < 1e-12 * lmax / gap * np.sqrt(n) + 1e-10


# both solvers (one-cluster double-float and grid-wide FP64) are held to the same bounds,
# except the orthonormality bound that each one's arithmetic sets
@pytest.mark.parametrize("solver", ["cluster", "grid"])
def test_nullspace_parity_phantom(H, solver):
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_small_64")
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    G = O.gram(pb.x0.astype(np.complex128), og, O.full_region(og))
    Q, eig = hicu.hicu_nullspace(H, cuda(G), pb.rank, solver=solver)
    tol = _orth_tol(H, G.shape[0], solver)
    _nullspace_check(Q.cpu().numpy(), eig.cpu().numpy(), G, pb.rank, tol)
    # warm start from the previous eigenvectors on a perturbed matrix
    rng = np.random.default_rng(9)
    E = random_complex(rng, G.shape) * 1e-3 * np.abs(G).max()
    G2 = G + (E + E.conj().T) / 2 * 1e-3
    Q2, eig2 = hicu.hicu_nullspace(H, cuda(G2), pb.rank, warm=True, solver=solver)
    # the warm start inherits the first basis' error
    tol += _orth_tol(H, G.shape[0], solver)
    _nullspace_check(Q2.cpu().numpy(), eig2.cpu().numpy(), G2, pb.rank, tol)


@pytest.mark.parametrize("solver", ["cluster", "grid"])
def test_nullspace_split_mode_matches_oracle_subspace(H, solver):
    """Warm split mode: same null space and the same J (Eq. 1) as LAPACK, not eigenvectors."""
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_small_64")
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    G = O.gram(pb.x0.astype(np.complex128), og, O.full_region(og))
    hicu.hicu_nullspace(H, cuda(G), pb.rank, solver=solver)          # cold: seeds the warm start
    rng = np.random.default_rng(12)
    E = random_complex(rng, G.shape)
    G2 = G + (E + E.conj().T) * 1e-4 * np.abs(G).max()
    tol = _orth_tol(H, G.shape[0], solver)
    Q, eig = hicu.hicu_nullspace(H, cuda(G2), pb.rank, warm=True, split=True, solver=solver)
    sweeps, how = hicu.hicu_nullspace_info(H)
    assert how == 2, (sweeps, how)
    tol += _orth_tol(H, G.shape[0], solver)
    Q = Q.cpu().numpy().T
    n, r = G.shape[0], pb.rank
    w, V = np.linalg.eigh(G2)
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(n - r), atol=tol)
    Qo = V[:, : n - r]
    gap = w[n - r] - w[n - r - 1]
    dist = np.linalg.norm(Q @ Q.conj().T - Qo @ Qo.conj().T)
    # the split stop guarantees a top-r / rest coupling block of Frobenius norm <= 1e-8 ||G||_F;
    # by the Davis-Kahan sin-theta theorem the projector distance is then <= sqrt(2) x that / gap
    assert dist < np.sqrt(2) * 1e-8 * np.linalg.norm(G2) / gap
    J = eig.cpu().numpy()[: n - r].sum()
    assert abs(J - w[: n - r].sum()) < 1e-11 * w[-1] * n


def test_nullspace_odd_n_lowrank(H):
    from paper_2004_08962_gb300 import hicu
    rng = np.random.default_rng(4)
    x = lowrank_exponential_kspace(rng, (1, 14, 13), 1, 3)   # C=1, k=3x3 -> n = 9 (odd)
    og = O.Geom((13, 14, 1), 1, (3, 3, 1))
    G = O.gram(x, og, O.full_region(og))
    Q, eig = hicu.hicu_nullspace(H, cuda(G), 3)
    _nullspace_check(Q.cpu().numpy(), eig.cpu().numpy(), G, 3, _orth_tol(H, 9, None))
    assert eig.cpu().numpy()[:6].max() < 1e-10 * eig.cpu().numpy().max()


@pytest.mark.parametrize("n,solver", [(256, "cluster"), (257, None), (200, "grid"), (200, "cluster"),
                                      (2, "cluster"), (2, "grid"), (128, None), (129, None)])
def test_nullspace_sizes(H, n, solver):
    """The cluster solver's largest size (n = 256), sizes above it (grid), the brain-slice size
    on both solvers, the smallest problem (n = 2, padded to 32) and both sides of the size at
    which the default switches from the cluster to the grid solver (128 / 129)."""
    from paper_2004_08962_gb300 import hicu
    rng = np.random.default_rng(n)
    r = max(1, n // 3)
    X = random_complex(rng, (n, n + 7))
    sv = np.exp(-np.arange(n) / 10.0)        # decaying spectrum, like a Gram of a low-rank Hankel
    U, _ = np.linalg.qr(X[:, :n])
    G = (U * sv**2) @ U.conj().T * 1e4
    G = (G + G.conj().T) / 2
    Q, eig = hicu.hicu_nullspace(H, cuda(G), r, solver=solver)
    _nullspace_check(Q.cpu().numpy(), eig.cpu().numpy(), G, r, _orth_tol(H, n, solver))


@pytest.mark.parametrize("solver", ["cluster", "grid"])
def test_nullspace_scale_invariance(H, solver):
    """Entries far outside the FP32 range (~1e270) or tiny (~1e-271): both solvers work on a
    power-of-two scaled copy, so eigenvalues scale exactly and the basis is bit-identical."""
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_small_64")
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    G = O.gram(pb.x0.astype(np.complex128), og, O.full_region(og))
    G = G / np.abs(G).max()
    Q1, e1 = hicu.hicu_nullspace(H, cuda(G), pb.rank, solver=solver)
    Q1, e1 = Q1.cpu().numpy(), e1.cpu().numpy()
    for s in (2.0**900, 2.0**-900):
        Qs, es = hicu.hicu_nullspace(H, cuda(G * s), pb.rank, solver=solver)
        Qs, es = Qs.cpu().numpy(), es.cpu().numpy()
        np.testing.assert_array_equal(es, e1 * s)
        np.testing.assert_array_equal(Qs, Q1)


@pytest.mark.parametrize("mode", [0, 1])
def test_jl_compress_parity(H, mode):
    from paper_2004_08962_gb300 import hicu
    rng = np.random.default_rng(5)
    n, r, p = 100, 30, 4
    Qo, _ = np.linalg.qr(random_complex(rng, (n, n - r)))
    Q = cuda(Qo.T.copy())
    bank = hicu.hicu_jl_compress(H, Q, p, mode=mode, seed=1234, counter=17).cpu().numpy()
    rows = n if mode == 1 else n - r
    P = O.jl_matrix(1234, 17, rows, p)
    ref = O.jl_compress(Qo, P, "projector" if mode == 1 else "nullspace")
    assert_close(bank, ref, 2e-6)
    # caller-supplied P
    Pc = rng.standard_normal((rows, p))
    bank2 = hicu.hicu_jl_compress(H, Q, p, mode=mode, P=cuda(Pc)).cpu().numpy()
    assert_close(bank2, O.jl_compress(Qo, Pc, "projector" if mode == 1 else "nullspace"), 2e-6)


def test_gd_step_with_jl_parity_phantom(H):
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_small_64")
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    reg = O.full_region(og)
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel)
    hr = hicu.make_region((0, 0, 0), pb.dims)
    G = O.gram(pb.x0.astype(np.complex128), og, reg)
    Qo, _ = O.nullspace(G, pb.rank)
    y = cuda(pb.x0)
    stats = hicu.hicu_gd_step(H, hg, hr, y, cuda(pb.mask), cuda(Qo.T.copy()), 4, jl_mode=1,
                              seed=7, counter=3).cpu().numpy()
    P = O.jl_matrix(7, 3, og.n, 4)
    f = O.as_filters(O.jl_compress(Qo, P, "projector"), og)
    y_ref, info = O.gd_step(pb.x0, pb.mask, og, reg, f)
    # null-space filters nearly annihilate the data: FP32 bound of the benchmark spec (1e-4)
    for got, want in zip(stats, (info.eta, info.objective, info.gnorm2, info.denom)):
        assert abs(got - want) <= 1e-4 * abs(want)
    assert_close(y.cpu().numpy() - pb.x0, y_ref - pb.x0, 1e-4)


def _oracle_recon(pb, jl="projector"):
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
    st = [O.StageSpec(O.Region(s.off, s.ext), s.iters, s.gd_steps, s.p) for s in pb.stages]
    log = O.ReconLog([], [], [])
    x = O.reconstruct(pb.x0, pb.mask, og, st, pb.rank, seed=11, jl_mode=jl,
                      init=pb.init, log=log)
    return x, log


def _gpu_params(pb, jl=1):
    from paper_2004_08962_gb300 import hicu
    return hicu.make_params(pb.rank, [(s.off, s.ext, s.iters, s.gd_steps, s.p) for s in pb.stages],
                            seed=11, jl=jl, init=1 if pb.init == "time_average" else 0)


def test_reconstruct_config1_matches_oracle(H):
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_small_64")
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel)
    x_gpu, log = hicu.hicu_reconstruct(H, hg, cuda(pb.x0), cuda(pb.mask), _gpu_params(pb),
                                       want_log=True)
    x_gpu = x_gpu.cpu().numpy()
    x_ref, olog = _oracle_recon(pb)
    assert_close(x_gpu, x_ref, 1e-3, "reconstruction")
    ser_g, ser_o = O.ser_db(pb.x_full, x_gpu), O.ser_db(pb.x_full, x_ref)
    assert abs(ser_g - ser_o) <= 0.05, (ser_g, ser_o)
    assert ser_o > O.ser_db(pb.x_full, pb.x0) + 1.0
    np.testing.assert_allclose(log["J"], olog.J, rtol=1e-3)
    np.testing.assert_allclose(log["eta"], olog.eta, rtol=1e-3)
    m4 = np.broadcast_to(pb.mask[None], pb.x0.shape).astype(bool)
    np.testing.assert_array_equal(x_gpu[m4], pb.x0[m4])
    # the same call with pinned HOST buffers gives bit-identical output
    x0h = torch.from_numpy(pb.x0).pin_memory()
    mh = torch.from_numpy(pb.mask).pin_memory()
    outh = torch.empty_like(x0h).pin_memory()
    hicu.hicu_reconstruct(H, hg, x0h, mh, _gpu_params(pb), x_out=outh)
    np.testing.assert_array_equal(outh.numpy(), x_gpu)


def test_reconstruct_host_input_staged_upload(H):
    """A 3D problem whose first stage covers a band of z planes: a host input is uploaded in two
    parts (the band first, the other planes while the first stage runs), and the result equals the
    device-buffer call bit for bit; the second stage reaches beyond the band and the third covers
    the whole array."""
    from paper_2004_08962_gb300 import hicu
    from synth.phantoms import Problem, Stage
    rng = np.random.default_rng(5)
    C, nx, ny, nz = 2, 20, 18, 16
    x_full = (lowrank_exponential_kspace(rng, (nz, ny, nx), C, 5)
              + 0.01 * random_complex(rng, (C, nz, ny, nx))).astype(np.complex64)
    mask = (rng.random((nz, ny, nx)) < 0.4).astype(np.uint8)
    x0 = (x_full * mask[None]).astype(np.complex64)
    stages = [Stage((4, 4, 5), (12, 10, 6), 2, 2, 3), Stage((2, 2, 4), (16, 14, 8), 1, 2, 3),
              Stage((0, 0, 0), (nx, ny, nz), 1, 2, 3)]
    pb = Problem("staged_3d", x_full, mask, x0, (3, 3, 3), (0, 0, 0), 8, stages)
    hg = hicu.make_geom(pb.dims, C, pb.kernel)
    prm = _gpu_params(pb)
    ref = hicu.hicu_reconstruct(H, hg, cuda(x0), cuda(mask), prm).cpu().numpy()
    assert not np.array_equal(ref, x0)
    x0h = torch.from_numpy(x0).pin_memory()
    mh = torch.from_numpy(mask).pin_memory()
    for _ in range(2):   # the second call reuses the handle's copy stream and workspace
        outh = torch.empty_like(x0h).pin_memory()
        hicu.hicu_reconstruct(H, hg, x0h, mh, prm, x_out=outh)
        np.testing.assert_array_equal(outh.numpy(), ref)
    outd = torch.empty(x0.shape, dtype=torch.complex64, device="cuda")
    hicu.hicu_reconstruct(H, hg, x0h, mh, prm, x_out=outd)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(outd.cpu().numpy(), ref)


def test_reconstruct_centre_out_and_time_average(H):
    """Small cine-shaped problem: circular time axis, time-averaged start, two CO stages."""
    from paper_2004_08962_gb300 import hicu
    from synth.phantoms import Problem, Stage
    rng = np.random.default_rng(21)
    C, nx, ny, nt = 2, 24, 20, 8
    x_full = (lowrank_exponential_kspace(rng, (nt, ny, nx), C, 5)
              + 0.01 * random_complex(rng, (C, nt, ny, nx))).astype(np.complex64)
    mask = (rng.random((nt, ny, nx)) < 0.5).astype(np.uint8)
    pb = Problem("cine_small", x_full, mask, (x_full * mask[None]).astype(np.complex64), (3, 3, 3),
                 (0, 0, 1), 10,
                 [Stage((6, 5, 0), (12, 10, 8), 3, 3, 4), Stage((0, 0, 0), (nx, ny, nt), 2, 4, 6)],
                 init="time_average")
    hg = hicu.make_geom(pb.dims, C, pb.kernel, pb.circular)
    x_gpu = hicu.hicu_reconstruct(H, hg, cuda(pb.x0), cuda(pb.mask), _gpu_params(pb)).cpu().numpy()
    x_ref, _ = _oracle_recon(pb)
    assert_close(x_gpu, x_ref, 1e-3)
    assert abs(O.ser_db(pb.x_full, x_gpu) - O.ser_db(pb.x_full, x_ref)) <= 0.05


def test_full_size_brain_slice_step(H):
    """256x256, C=8, 5x5 kernel, p=32: the full-k-space step of the 2D brain workload."""
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_brain_256")
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    reg = O.full_region(og)
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel)
    hr = hicu.make_region((0, 0, 0), pb.dims)
    rng = np.random.default_rng(6)
    f = random_complex(rng, (32, og.n)).astype(np.complex64) * 0.1
    R = hicu.hicu_conv_null(H, hg, hr, cuda(pb.x0), cuda(f)).cpu().numpy()
    Rref = O.conv_null(pb.x0.astype(np.complex128), og, reg, ofilters(f, og))
    assert_close(R, Rref, 5e-6)
    y = cuda(pb.x0)
    stats = hicu.hicu_gd_step_filters(H, hg, hr, y, cuda(pb.mask), cuda(f)).cpu().numpy()
    y_ref, info = O.gd_step(pb.x0, pb.mask, og, reg, ofilters(f, og))
    assert abs(stats[0] - info.eta) < 2e-5 * info.eta
    assert_close(y.cpu().numpy() - pb.x0, y_ref - pb.x0, 2e-5)
    G = hicu.hicu_gram(H, hg, hr, cuda(pb.x0)).cpu().numpy()
    assert_close(G, O.gram(pb.x0.astype(np.complex128), og, reg), 1e-12)


def test_deterministic(H):
    from paper_2004_08962_gb300 import hicu
    og, oreg, hg, hr, x, f, mask, p, _ = setup("2d_64_c4_p4", seed=8)
    outs = []
    for _ in range(2):
        y = cuda(x)
        s = hicu.hicu_gd_step_filters(H, hg, hr, y, cuda(mask), cuda(f))
        outs.append((y.cpu().numpy(), s.cpu().numpy(), hicu.hicu_gram(H, hg, hr, cuda(x)).cpu().numpy()))
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)


def test_argument_errors(H):
    from paper_2004_08962_gb300 import hicu
    og, oreg, hg, hr, x, f, mask, p, _ = setup("2d_64_c4_p4")
    big = hicu.make_region((10, 0, 0), (64, 64, 1))
    with pytest.raises(hicu.HicuError) as e:
        hicu.hicu_gram(H, hg, big, cuda(x))
    assert e.value.status == 2
    G = torch.zeros((100, 100), dtype=torch.complex128, device="cuda")
    with pytest.raises(hicu.HicuError) as e:
        hicu.hicu_nullspace(H, G, 0)
    assert e.value.status == 3
    G300 = torch.zeros((300, 300), dtype=torch.complex128, device="cuda")
    with pytest.raises(hicu.HicuError) as e:                 # cluster solver is for n <= 256
        hicu.hicu_nullspace(H, G300, 10, solver="cluster")
    assert e.value.status == 8
    with pytest.raises(hicu.HicuError) as e:
        hicu.hicu_conv_null(H, hg, hr, cuda(x), cuda(f), prec=7)
    assert e.value.status == 1
    hicu.hicu_check(H)


# ------------------------------------------------------------ split-bf16 tensor cores

CASES["tiny_one_output_c4"] = ((9, 9, 1), 4, (5, 5, 1), (0, 0, 0), ((2, 3, 0), (5, 5, 1)), 3)
CASES["2d_c8_p32_region"] = ((100, 90, 1), 8, (5, 5, 1), (0, 0, 0), ((7, 11, 0), (83, 70, 1)), 32)
# wider than one 256-position tile row, so the x axis splits into tiles
CASES["2d_wide_two_x_tiles"] = ((300, 24, 1), 4, (5, 5, 1), (0, 0, 0), ((0, 0, 0), (300, 24, 1)), 8)
# 2D with the row axis circular (streamed axis wraps)
CASES["2d_circular_rows"] = ((40, 30, 1), 8, (5, 5, 1), (0, 1, 0), ((0, 0, 0), (40, 30, 1)), 8)
# 3D shapes of the cine / knee workloads in miniature: 5x5x5 kernel, C = 8, p = 8
CASES["3d_c8_k5_region"] = ((44, 38, 18), 8, (5, 5, 5), (0, 0, 0), ((2, 1, 1), (40, 36, 16)), 8)
CASES["cine_c8_k5_circular_t"] = ((48, 36, 12), 8, (5, 5, 5), (0, 0, 1), ((0, 0, 0), (48, 36, 12)), 8)
TC_CASES = ["2d_64_c4_p4", "2d_c16_p20", "2d_c32_permask", "tiny_one_output_c4", "2d_c8_p32_region",
            "2d_odd_region", "tiny_one_output", "3d_region", "cine_circular_t", "2d_wide_two_x_tiles",
            "2d_circular_rows", "3d_c8_k5_region", "cine_c8_k5_circular_t"]


@pytest.mark.parametrize("name", TC_CASES)
def test_conv_null_split_bf16(H, name):
    from paper_2004_08962_gb300 import hicu
    og, oreg, hg, hr, x, f, mask, p, _ = setup(name)
    R, obj = hicu.hicu_conv_null(H, hg, hr, cuda(x), cuda(f), prec=hicu.HICU_SPLIT_BF16,
                                 want_objective=True)
    ref = O.conv_null(x.astype(np.complex128), og, oreg, ofilters(f, og))
    assert_close(R.cpu().numpy(), ref, 2e-5)
    assert abs(obj.item() - np.vdot(ref, ref).real) < 4e-5 * np.vdot(ref, ref).real


@pytest.mark.parametrize("name", TC_CASES)
def test_adjoint_split_bf16(H, name):
    from paper_2004_08962_gb300 import hicu
    og, oreg, hg, hr, x, f, mask, p, rng = setup(name, seed=1)
    R = random_complex(rng, O.out_shape(og, oreg) + (p,)).astype(np.complex64)
    sentinel = np.full(x.shape, 7.0 + 3.0j, dtype=np.complex64)
    g, gn = hicu.hicu_conv_null_adjoint(H, hg, hr, cuda(R), cuda(f), mask=cuda(mask), g=cuda(sentinel),
                                        prec=hicu.HICU_SPLIT_BF16, want_gnorm2=True)
    ref = O.conv_null_adjoint(R.astype(np.complex128), og, oreg, ofilters(f, og), mask)
    g = g.cpu().numpy()
    inside = np.zeros(x.shape[1:], dtype=bool)
    (ox, oy, oz), (ex, ey, ez) = CASES[name][4]
    inside[oz:oz + ez, oy:oy + ey, ox:ox + ex] = True
    assert_close(g[:, inside], ref[:, inside], 2e-5)
    np.testing.assert_array_equal(g[:, ~inside], sentinel[:, ~inside])
    m4 = np.broadcast_to(mask if mask.ndim == 4 else mask[None], x.shape).astype(bool)
    assert np.all(g[m4 & inside[None]] == 0)
    assert abs(gn.item() - np.vdot(ref, ref).real) < 4e-5 * np.vdot(ref, ref).real


@pytest.mark.parametrize("name", TC_CASES)
def test_gd_step_split_bf16(H, name):
    from paper_2004_08962_gb300 import hicu
    og, oreg, hg, hr, x, f, mask, p, _ = setup(name, seed=2)
    y = cuda(x)
    stats = hicu.hicu_gd_step_filters(H, hg, hr, y, cuda(mask), cuda(f),
                                      prec=hicu.HICU_SPLIT_BF16).cpu().numpy()
    y1_ref, info = O.gd_step(x, mask, og, oreg, ofilters(f, og))
    for got, want in zip(stats, (info.eta, info.objective, info.gnorm2, info.denom)):
        assert abs(got - want) <= 1e-4 * abs(want)
    y1 = y.cpu().numpy()
    assert_close(y1 - x, y1_ref - x, 1e-4)
    m4 = np.broadcast_to(mask if mask.ndim == 4 else mask[None], x.shape).astype(bool)
    np.testing.assert_array_equal(y1[m4], x[m4])


def test_split_bf16_full_size_brain_slice(H):
    """256x256, C=8, p=32 step of the 2D brain workload with null-space filters (spec bound
    for split-bf16: gradient error <= 1e-3)."""
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_brain_256")
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    reg = O.full_region(og)
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel)
    hr = hicu.make_region((0, 0, 0), pb.dims)
    G = O.gram(pb.x0.astype(np.complex128), og, reg)
    Qo, _ = O.nullspace(G, pb.rank)
    f = O.as_filters(O.jl_compress(Qo, O.jl_matrix(3, 1, og.n, 32), "projector"), og)
    fb = cuda(f.reshape(32, -1).astype(np.complex64))
    g_gpu = hicu.hicu_conv_null_adjoint(
        H, hg, hr, hicu.hicu_conv_null(H, hg, hr, cuda(pb.x0), fb, prec=hicu.HICU_SPLIT_BF16), fb,
        mask=cuda(pb.mask), prec=hicu.HICU_SPLIT_BF16).cpu().numpy()
    g_ref, _ = O.gradient(pb.x0.astype(np.complex128), og, reg, f, pb.mask)
    assert_close(g_gpu, g_ref, 1e-3)
    y = cuda(pb.x0)
    stats = hicu.hicu_gd_step_filters(H, hg, hr, y, cuda(pb.mask), fb, prec=hicu.HICU_SPLIT_BF16).cpu().numpy()
    y_ref, info = O.gd_step(pb.x0, pb.mask, og, reg, f)
    assert abs(stats[0] - info.eta) < 1e-3 * info.eta
    assert_close(y.cpu().numpy() - pb.x0, y_ref - pb.x0, 1e-3)


def test_reconstruct_config1_split_bf16(H):
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_small_64")
    hg = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel)
    prm = hicu.make_params(pb.rank, [(s.off, s.ext, s.iters, s.gd_steps, s.p) for s in pb.stages],
                           seed=11, jl=1, prec=hicu.HICU_SPLIT_BF16)
    x_gpu = hicu.hicu_reconstruct(H, hg, cuda(pb.x0), cuda(pb.mask), prm).cpu().numpy()
    x_ref, _ = _oracle_recon(pb)
    assert_close(x_gpu, x_ref, 1e-3)
    assert abs(O.ser_db(pb.x_full, x_gpu) - O.ser_db(pb.x_full, x_ref)) <= 0.05


@pytest.mark.parametrize("dims,ker,circ", [((24, 20, 1), (3, 3, 1), (1, 0, 0)),
                                           ((24, 20, 8), (3, 3, 3), (0, 1, 0)),
                                           ((24, 20, 8), (3, 3, 9), (0, 0, 1))])
def test_split_bf16_unsupported_geometry(H, dims, ker, circ):
    """The tensor-core tiling wraps only the streamed (outermost) axis and takes up to 8 offsets
    along it; anything else is refused with HICU_ERR_UNSUPPORTED before any launch."""
    from paper_2004_08962_gb300 import hicu
    rng = np.random.default_rng(3)
    hg = hicu.make_geom(dims, 4, ker, circ)
    hr = hicu.make_region((0, 0, 0), dims)
    n = 4 * ker[0] * ker[1] * ker[2]
    x = random_complex(rng, (4, dims[2], dims[1], dims[0])).astype(np.complex64)
    f = random_complex(rng, (2, n)).astype(np.complex64)
    with pytest.raises(hicu.HicuError) as e:
        hicu.hicu_conv_null(H, hg, hr, cuda(x), cuda(f), prec=hicu.HICU_SPLIT_BF16)
    assert e.value.status == 8
    hicu.hicu_check(H)
