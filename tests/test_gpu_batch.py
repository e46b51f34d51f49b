"""Batched uneven reconstructions (hicu_reconstruct_batched) against single-problem runs and the
oracle.  Every problem of a batch must give exactly the result of hicu_reconstruct with the same
parameters and eigen-solver: lanes share no mutable state and every kernel is deterministic."""
import numpy as np
from closeness import assert_close
import pytest
import torch

from oracle import hicu_oracle as O
from synth.phantoms import _slice_2d, make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2004_08962_gb300 import build, hicu
    build.build()
    return hicu.Handle()


def _case(rng, n, C, k, rank, stages, prec, per_coil=False, host=False, seed=0):
    from paper_2004_08962_gb300 import hicu
    x, mask = _slice_2d(rng, n, C, 3.0, n_ellipses=6)
    if per_coil:  # interleaved shots: coil c sees every C-th line starting at c
        mask = np.zeros((C, 1, n, n), dtype=np.uint8)
        for c in range(C):
            mask[c, 0, c % 4::4, :] = 1
            mask[c, 0, n // 2 - 4:n // 2 + 4, :] = 1
    x0 = (x * (mask if per_coil else mask[None])).astype(np.complex64)
    return dict(n=n, C=C, k=k, rank=rank, stages=stages, prec=prec, per_coil=per_coil, host=host,
                x0=x0, mask=mask, seed=seed)


def _cases():
    rng = np.random.default_rng(77)
    full = lambda n: ((0, 0, 0), (n, n, 1))
    from paper_2004_08962_gb300 import hicu
    bf16, fp32 = hicu.HICU_SPLIT_BF16, hicu.HICU_FP32
    return [
        _case(rng, 48, 8, 5, 60, [((12, 12, 0), (24, 24, 1), 2, 2, 8), (*full(48), 1, 3, 16)], bf16, seed=1),
        _case(rng, 40, 16, 5, 120, [(*full(40), 2, 2, 8)], bf16, seed=2),             # n = 400: grid solver
        _case(rng, 56, 4, 5, 30, [(*full(56), 2, 3, 4)], fp32, per_coil=True, seed=3),
        _case(rng, 72, 2, 3, 6, [(*full(72), 3, 2, 4)], fp32, host=True, seed=4),      # host buffers
        _case(rng, 36, 4, 3, 10, [(*full(36), 1, 1, 2)], bf16, seed=5),
    ]


def _tensors(c):
    x0 = torch.from_numpy(c["x0"])
    m = torch.from_numpy(c["mask"])
    if c["host"]:
        return x0.pin_memory(), m.pin_memory(), torch.empty_like(x0).pin_memory()
    x0, m = x0.cuda(), m.cuda()
    return x0, m, torch.empty_like(x0)


def _params(c, solver=None):
    from paper_2004_08962_gb300 import hicu
    return hicu.make_params(c["rank"], c["stages"], seed=c["seed"], jl=hicu.HICU_JL_PROJECTOR,
                            prec=c["prec"], eig_solver=solver)


def _geom(c):
    from paper_2004_08962_gb300 import hicu
    return hicu.make_geom((c["n"], c["n"], 1), c["C"], (c["k"], c["k"], 1), mask_per_coil=c["per_coil"])


def _jacobi_by_size(c):
    return "cluster" if c["C"] * c["k"] ** 2 <= 256 else "grid"


@pytest.mark.parametrize("solver", ["default", "jacobi"])
def test_batch_matches_single_problem_runs(H, solver):
    """default: the tridiagonal principal-subspace path (eig_solver 0, projector JL); jacobi: the
    one-cluster solver for n <= 256 and the grid solver above, requested explicitly."""
    from paper_2004_08962_gb300 import hicu
    cases = _cases()
    pick = (lambda c: None) if solver == "default" else _jacobi_by_size
    probs, outs = [], []
    for c in cases:
        x0, m, out = _tensors(c)
        probs.append(hicu.make_problem_struct(_geom(c), x0, m, _params(c, pick(c)), out))
        outs.append(out)
    reports, st = hicu.hicu_reconstruct_batched(H, probs, lanes=3)
    assert st == 0
    lanes_used = set()
    for c, rep in zip(cases, reports):
        assert rep["status"] == 0
        assert 0.0 <= rep["start_ms"] <= rep["end_ms"]
        assert rep["gd_steps"] == sum(it * gd for (_, _, it, gd, _) in c["stages"])
        lanes_used.add(rep["lane"])
    assert lanes_used <= {0, 1, 2} and len(lanes_used) >= 2
    torch.cuda.synchronize()
    for c, out in zip(cases, outs):
        x0, m, ref = _tensors(c)
        hicu.hicu_reconstruct(H, _geom(c), x0, m, _params(c, pick(c)), x_out=ref)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
        # observed entries untouched
        x0n = c["x0"]
        obs = (c["mask"] if c["per_coil"] else np.broadcast_to(c["mask"][None], x0n.shape)).astype(bool)
        np.testing.assert_array_equal(out.cpu().numpy()[obs], x0n[obs])


def test_batch_problem_matches_oracle(H):
    """The first configuration's problem run inside a batch (with a larger neighbour) stays within
    the reconstruction bound against the FP64 oracle."""
    from paper_2004_08962_gb300 import hicu
    pb = make_problem("2d_small_64")
    prm = hicu.make_params(pb.rank, [(s.off, s.ext, s.iters, s.gd_steps, s.p) for s in pb.stages], seed=11,
                           jl=hicu.HICU_JL_PROJECTOR)
    x0 = torch.from_numpy(pb.x0).cuda()
    m = torch.from_numpy(pb.mask).cuda()
    out = torch.empty_like(x0)
    c = _cases()[0]
    bx0, bm, bout = _tensors(c)
    probs = [hicu.make_problem_struct(hicu.make_geom(pb.dims, pb.ncoil, pb.kernel), x0, m, prm, out),
             hicu.make_problem_struct(_geom(c), bx0, bm, _params(c), bout)]
    hicu.hicu_reconstruct_batched(H, probs, lanes=2)
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
    st = [O.StageSpec(O.Region(s.off, s.ext), s.iters, s.gd_steps, s.p) for s in pb.stages]
    ref = O.reconstruct(pb.x0, pb.mask, og, st, pb.rank, seed=11, jl_mode="projector", init=pb.init)
    x = out.cpu().numpy()
    assert_close(x, ref, 1e-3, "batched slice")
    assert abs(O.ser_db(pb.x_full, x) - O.ser_db(pb.x_full, ref)) <= 0.05


def test_batch_failing_problem_does_not_stop_the_others(H):
    from paper_2004_08962_gb300 import hicu
    cases = _cases()[3:5]
    bad = dict(cases[1])
    bad["rank"] = bad["C"] * bad["k"] ** 2          # r = n: invalid
    probs, outs = [], []
    for c in (cases[0], bad, cases[1]):
        x0, m, out = _tensors(c)
        probs.append(hicu.make_problem_struct(_geom(c), x0, m, _params(c), out))
        outs.append(out)
    reports, st = hicu.hicu_reconstruct_batched(H, probs, lanes=2, check=False)
    assert st == 3 and [r["status"] for r in reports] == [0, 3, 0]
    for c, out in ((cases[0], outs[0]), (cases[1], outs[2])):
        x0, m, ref = _tensors(c)
        hicu.hicu_reconstruct(H, _geom(c), x0, m, _params(c), x_out=ref)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    assert "problem 1" in hicu.lib().hicu_last_error(H.ptr).decode()
