"""Differentiable convolutions (paper_2004_08962_gb300.autograd) against the FP64 oracle's
gradients and against central finite differences.

The checked losses are linear (Re<W, output>) or quadratic (||H(x) f||^2) in each input, so a
central difference equals the directional derivative exactly and the comparison only sees FP32
rounding."""
import numpy as np
from closeness import assert_close
import pytest
import torch

from oracle import hicu_oracle as O
from synth.phantoms import random_complex

pytestmark = pytest.mark.gpu

# dims (Nx, Ny, Nz), C, kernel, circular, region (off, ext), p
CASES = {
    "2d_region": ((40, 34, 1), 4, (5, 3, 1), (0, 0, 0), ((3, 2, 0), (33, 30, 1)), 6),
    "3d_region": ((18, 16, 10), 2, (3, 3, 3), (0, 0, 0), ((1, 2, 1), (15, 13, 8)), 3),
    "cine_circular_t": ((20, 18, 8), 2, (3, 3, 3), (0, 0, 1), ((0, 0, 0), (20, 18, 8)), 4),
    "2d_c8_p45": ((70, 38, 1), 8, (5, 5, 1), (0, 0, 0), ((0, 0, 0), (70, 38, 1)), 45),   # two filter chunks
}


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2004_08962_gb300 import build, hicu
    build.build()
    return hicu.Handle()




def setup(H, name, seed=0):
    from paper_2004_08962_gb300.autograd import HicuConv
    dims, C, ker, circ, (off, ext), p = CASES[name]
    og, oreg = O.Geom(dims, C, ker, circ), O.Region(off, ext)
    op = HicuConv(H, dims, C, ker, region=(off, ext), circular=circ)
    rng = np.random.default_rng(seed)
    x = random_complex(rng, (C, dims[2], dims[1], dims[0])).astype(np.complex64)
    f = random_complex(rng, (p, og.n)).astype(np.complex64)
    mask = (rng.random((dims[2], dims[1], dims[0])) < 0.35).astype(np.uint8)
    return og, oreg, op, x, f, mask, p, rng


def filt(f, og):
    return O.as_filters(f.astype(np.complex128), og)


@pytest.mark.parametrize("name", list(CASES))
def test_filter_gradient_parity(H, name):
    from paper_2004_08962_gb300 import hicu
    og, oreg, op, x, f, mask, p, rng = setup(H, name)
    Rb = random_complex(rng, O.out_shape(og, oreg) + (p,)).astype(np.complex64)
    F = hicu.hicu_conv_null_filter_grad(H, op.geom, op.region, torch.from_numpy(x).cuda(),
                                        torch.from_numpy(Rb).cuda()).cpu().numpy()
    ref = O.filter_gradient(x, og, oreg, Rb).reshape(p, -1)
    assert_close(F, ref, 5e-6)
    # deterministic: a second call is bit-identical
    F2 = hicu.hicu_conv_null_filter_grad(H, op.geom, op.region, torch.from_numpy(x).cuda(),
                                         torch.from_numpy(Rb).cuda()).cpu().numpy()
    np.testing.assert_array_equal(F, F2)


@pytest.mark.parametrize("name", ["2d_region", "3d_region"])
def test_project_unobserved_parity(H, name):
    from paper_2004_08962_gb300 import hicu
    og, oreg, op, x, f, mask, p, rng = setup(H, name)
    out = hicu.hicu_project_unobserved(H, op.geom, op.region, torch.from_numpy(x).cuda(),
                                       torch.from_numpy(mask).cuda()).cpu().numpy()
    np.testing.assert_array_equal(out, O.project_unobserved(x, og, oreg, mask).astype(np.complex64))
    inplace = torch.from_numpy(x).cuda()
    hicu.hicu_project_unobserved(H, op.geom, op.region, inplace, None, out=inplace)
    np.testing.assert_array_equal(inplace.cpu().numpy(), O.project_unobserved(x, og, oreg, None))


def _fd(loss, t, v):
    """Central difference of a real loss along v (exact for linear and quadratic losses)."""
    with torch.no_grad():
        return (loss(t + v).item() - loss(t - v).item()) / 2.0


def _dir(grad, v):
    return float(torch.real(torch.vdot(grad.reshape(-1), v.reshape(-1))).item())


@pytest.mark.parametrize("name", list(CASES))
def test_conv_null_autograd(H, name):
    og, oreg, op, x, f, mask, p, rng = setup(H, name)
    W = torch.from_numpy(random_complex(rng, O.out_shape(og, oreg) + (p,)).astype(np.complex64)).cuda()
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    loss = torch.real(torch.vdot(W.reshape(-1), op.conv_null(xt, ft).reshape(-1)))
    loss.backward()
    Wn = W.cpu().numpy().astype(np.complex128)
    # conjugate-Wirtinger convention: the gradient of Re<W, A z> is A^H W
    assert_close(xt.grad.cpu().numpy(), O.conv_null_adjoint(Wn, og, oreg, filt(f, og)), 5e-6)
    assert_close(ft.grad.cpu().numpy(), O.filter_gradient(x, og, oreg, Wn).reshape(p, -1), 5e-6)
    vx = torch.from_numpy(random_complex(rng, x.shape).astype(np.complex64)).cuda()
    vf = torch.from_numpy(random_complex(rng, f.shape).astype(np.complex64)).cuda()
    lx = lambda t: torch.real(torch.vdot(W.reshape(-1), op.conv_null(t, ft.detach()).reshape(-1)))
    lf = lambda t: torch.real(torch.vdot(W.reshape(-1), op.conv_null(xt.detach(), t).reshape(-1)))
    for l, t, v, g in ((lx, xt, vx, xt.grad), (lf, ft, vf, ft.grad)):
        fd, an = _fd(l, t.detach(), v), _dir(g, v)
        assert abs(fd - an) <= 1e-4 * (abs(an) + abs(loss.item())), (fd, an)


@pytest.mark.parametrize("name", ["2d_region", "3d_region", "cine_circular_t"])
def test_conv_null_adjoint_autograd(H, name):
    og, oreg, op, x, f, mask, p, rng = setup(H, name)
    R = random_complex(rng, O.out_shape(og, oreg) + (p,)).astype(np.complex64)
    W = torch.from_numpy(random_complex(rng, x.shape).astype(np.complex64)).cuda()
    mt = torch.from_numpy(mask).cuda()
    Rt = torch.from_numpy(R).cuda().requires_grad_(True)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    g = op.conv_null_adjoint(Rt, ft, mt)
    np.testing.assert_allclose(g.detach().cpu().numpy(),
                               O.conv_null_adjoint(R, og, oreg, filt(f, og), mask), rtol=0, atol=2e-4)
    loss = torch.real(torch.vdot(W.reshape(-1), g.reshape(-1)))
    loss.backward()
    PW = O.project_unobserved(W.cpu().numpy(), og, oreg, mask)
    assert_close(Rt.grad.cpu().numpy(), O.conv_null(PW, og, oreg, filt(f, og)), 5e-6)
    assert_close(ft.grad.cpu().numpy(), O.filter_gradient(PW, og, oreg, R).reshape(p, -1), 5e-6)
    vR = torch.from_numpy(random_complex(rng, R.shape).astype(np.complex64)).cuda()
    vf = torch.from_numpy(random_complex(rng, f.shape).astype(np.complex64)).cuda()
    lR = lambda t: torch.real(torch.vdot(W.reshape(-1), op.conv_null_adjoint(t, ft.detach(), mt).reshape(-1)))
    lf = lambda t: torch.real(torch.vdot(W.reshape(-1), op.conv_null_adjoint(Rt.detach(), t, mt).reshape(-1)))
    for l, t, v, gr in ((lR, Rt, vR, Rt.grad), (lf, ft, vf, ft.grad)):
        fd, an = _fd(l, t.detach(), v), _dir(gr, v)
        assert abs(fd - an) <= 1e-4 * (abs(an) + abs(loss.item())), (fd, an)


@pytest.mark.parametrize("name", list(CASES))
def test_null_objective_recomputes_and_matches(H, name):
    """F = ||H(x) f||^2 without a stored R; gradients 2 H^H(R f) and 2 H(x)^H R against the oracle,
    and finite differences of the quadratic along random directions."""
    og, oreg, op, x, f, mask, p, rng = setup(H, name)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    F = op.null_objective(xt, ft)
    Rref = O.conv_null(x, og, oreg, filt(f, og))
    assert abs(F.item() - np.sum(np.abs(Rref) ** 2)) < 1e-5 * F.item()
    (F * 0.75).backward()
    gx_ref = 1.5 * O.conv_null_adjoint(Rref, og, oreg, filt(f, og))
    gf_ref = 1.5 * O.filter_gradient(x, og, oreg, Rref).reshape(p, -1)
    assert_close(xt.grad.cpu().numpy(), gx_ref, 1e-5)
    assert_close(ft.grad.cpu().numpy(), gf_ref, 1e-5)
    scale = 0.05
    vx = torch.from_numpy(random_complex(rng, x.shape).astype(np.complex64) * scale).cuda()
    vf = torch.from_numpy(random_complex(rng, f.shape).astype(np.complex64) * scale).cuda()
    lx = lambda t: op.null_objective(t, ft.detach()) * 0.75
    lf = lambda t: op.null_objective(xt.detach(), t) * 0.75
    for l, t, v, g in ((lx, xt, vx, xt.grad), (lf, ft, vf, ft.grad)):
        fd, an = _fd(l, t.detach(), v), _dir(g, v)
        assert abs(fd - an) <= 1e-4 * abs(an) + 1e-6 * F.item(), (fd, an)


def test_gradient_step_on_filters_reduces_objective(H):
    """One autograd-driven descent step on the filters lowers ||H(x) f||^2 (used as a loss)."""
    og, oreg, op, x, f, mask, p, rng = setup(H, "2d_region")
    xt = torch.from_numpy(x).cuda()
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    F0 = op.null_objective(xt, ft)
    F0.backward()
    with torch.no_grad():
        g = ft.grad
        # exact minimiser along -g of the quadratic: t = ||g||^2 / (2 ||H(x) g||^2)
        t = (torch.vdot(g.reshape(-1), g.reshape(-1)).real / (2 * op.null_objective(xt, g))).item()
        F1 = op.null_objective(xt, ft - t * g)
    assert F1.item() < F0.item()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_autograd_full_size_brain_slice(H, prec):
    """The 256 x 256 x 8-coil slice (n = 200, p = 32): gradients of ||H(x) f||^2 with respect to
    x and the filters against the FP64 oracle and finite differences, in the plain FP32 form
    (bound 1e-5) and the split-BF16 tensor-core form (bound 1e-3)."""
    from paper_2004_08962_gb300 import hicu
    from paper_2004_08962_gb300.autograd import HicuConv
    from synth.phantoms import make_problem
    pb = make_problem("2d_brain_256")
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel)
    reg = O.full_region(og)
    op = HicuConv(H, pb.dims, pb.ncoil, pb.kernel,
                  prec=hicu.HICU_FP32 if prec == "fp32" else hicu.HICU_SPLIT_BF16)
    rng = np.random.default_rng(21)
    p = 32
    f = (random_complex(rng, (p, og.n)) * 0.05).astype(np.complex64)
    x = pb.x0
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    F = op.null_objective(xt, ft)
    F.backward()
    R = O.conv_null(x, og, reg, filt(f, og))
    tol = 1e-5 if prec == "fp32" else 1e-3
    assert abs(F.item() - np.sum(np.abs(R) ** 2)) < tol * F.item()
    assert_close(xt.grad.cpu().numpy(), 2 * O.conv_null_adjoint(R, og, reg, filt(f, og)), tol)
    assert_close(ft.grad.cpu().numpy(), 2 * O.filter_gradient(x, og, reg, R).reshape(p, -1), tol)
    vx = torch.from_numpy((random_complex(rng, x.shape) * 0.02 * np.abs(x).max()).astype(np.complex64)).cuda()
    vf = torch.from_numpy((random_complex(rng, f.shape) * 0.002).astype(np.complex64)).cuda()
    lx = lambda t: op.null_objective(t, ft.detach())
    lf = lambda t: op.null_objective(xt.detach(), t)
    for l, t, v, g in ((lx, xt, vx, xt.grad), (lf, ft, vf, ft.grad)):
        fd, an = _fd(l, t.detach(), v), _dir(g, v)
        assert abs(fd - an) <= 10 * tol * abs(an) + tol * F.item(), (fd, an)
