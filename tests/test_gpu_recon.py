"""GPU tests of the autograd wrappers and the iterative reconstructions (Section 8)."""

import math

import numpy as np
import pytest

from oracle import direct, geometry
from workloads import ellipse_image, ellipse_sinogram, gaussian_image, random_ellipses

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BLOBS = [(0.2, -0.1, 0.12, 1.0), (-0.3, 0.25, 0.08, -0.7), (0.05, 0.5, 0.1, 0.4)]
BLOBS2 = [(-0.1, -0.3, 0.15, 0.8), (0.3, 0.2, 0.1, 0.5)]


@pytest.fixture(scope="module")
def rl():
    from paper_1506_00014_gb300 import build

    if build.needs_build():
        build.build()
    import paper_1506_00014_gb300 as rl

    return rl


def _t(a):
    return torch.tensor(np.asarray(a, np.float32), device="cuda")


def test_autograd_gradients_pass_finite_differences_on_smooth_inputs(rl):
    from paper_1506_00014_gb300.autograd import backproject, radon

    N = 256
    plan = rl.radon_plan_create(N, N, 384, 3, 3)
    geo = geometry.make_geometry(N, N, 384, 3)
    th = np.arange(geo.n_angles) * geo.dtheta
    s = (np.arange(geo.n_det) - geo.n_det / 2) * geo.ds
    G = _t(direct.gaussian_radon(th[:, None], s[None, :], BLOBS2))
    f = _t(gaussian_image(N, BLOBS)).requires_grad_(True)
    loss = (radon(f, plan) * G).sum()
    (grad,) = torch.autograd.grad(loss, f)
    v = _t(gaussian_image(N, BLOBS2))
    eps = 1e-2
    with torch.no_grad():
        fd = ((radon(f + eps * v, plan) * G).sum() - (radon(f - eps * v, plan) * G).sum()) / (2 * eps)
    assert float((grad * v).sum()) == pytest.approx(float(fd), rel=2e-4)
    # and the other direction
    g = G.clone().requires_grad_(True)
    loss2 = (backproject(g, plan) * v).sum()
    (grad2,) = torch.autograd.grad(loss2, g)
    with torch.no_grad():
        fd2 = ((backproject(G + eps * G, plan) * v).sum() - (backproject(G - eps * G, plan) * v).sum()) / (2 * eps)
    assert float((grad2 * G).sum()) == pytest.approx(float(fd2), rel=2e-4)


def test_dot_product_identity_on_smooth_inputs(rl):
    """<R f, g> = c_R <f, R# g> (the adjoint relation the autograd backward relies on, c_R =
    dx^2 / (dtheta ds)) for smooth f and g; R# is the discretised continuous adjoint, so the
    identity holds to the method's accuracy, not to rounding."""
    from paper_1506_00014_gb300.autograd import adjoint_scales

    N, na, nd = 256, 384, 384
    plan = rl.radon_plan_create(N, na, nd, 3, 3)
    geo = geometry.make_geometry(N, na, nd, 3)
    th = np.arange(na) * geo.dtheta
    s = (np.arange(nd) - nd / 2) * geo.ds
    f = _t(gaussian_image(N, BLOBS))
    g = _t(direct.gaussian_radon(th[:, None], s[None, :], BLOBS2))
    rf = torch.empty((na, nd), device="cuda")
    bg = torch.empty((N, N), device="cuda")
    rl.radon_forward(plan, f, rf)
    rl.radon_backproject(plan, g, bg)
    c_r, _ = adjoint_scales(plan)
    lhs = float((rf.double() * g.double()).sum())
    rhs = c_r * float((f.double() * bg.double()).sum())
    assert lhs == pytest.approx(rhs, rel=1e-4)


def test_batched_autograd_equals_per_slice(rl):
    from paper_1506_00014_gb300.autograd import radon

    N = 64
    plan = rl.radon_plan_create(N, N, 96, 3, 3)
    fs = torch.stack([_t(ellipse_image(N, random_ellipses(5, s))) for s in range(3)])
    out = radon(fs, plan)
    for b in range(3):
        one = radon(fs[b], plan)
        assert torch.equal(out[b], one)


@pytest.mark.parametrize("use_graph", [False, True])
def test_least_squares_decreases_the_residual(rl, use_graph):
    from paper_1506_00014_gb300.recon import LeastSquares

    N, na, nd = 128, 96, 192
    plan = rl.radon_plan_create(N, na, nd, 3, 3)
    ell = random_ellipses(10, 200)
    g = ellipse_sinogram(ell, na, nd)
    rng = np.random.default_rng(200)
    g = g + rng.normal(0, 0.01 * np.abs(g).max(), g.shape)
    ls = LeastSquares(plan, _t(g), use_graph=use_graph)
    losses = [ls.loss()]
    for _ in range(5):
        ls.run(10)
        losses.append(ls.loss())
    assert all(b < a for a, b in zip(losses, losses[1:]))
    assert losses[-1] < 0.2 * losses[0]


def test_least_squares_graph_replay_equals_eager(rl):
    from paper_1506_00014_gb300.recon import LeastSquares

    N, na, nd = 64, 64, 96
    plan = rl.radon_plan_create(N, na, nd, 3, 3)
    g = _t(ellipse_sinogram(random_ellipses(6, 5), na, nd))
    a = LeastSquares(plan, g, step=0.3).run(20).clone()
    b = LeastSquares(plan, g, step=0.3, use_graph=True).run(20).clone()
    assert torch.equal(a, b)


def test_least_squares_config_64_slices_1024(rl):
    """64 slices, N = 1024, 720 angles, 1536 bins; data = analytic ellipse line integrals plus
    Gaussian noise at 1 % of the maximum; 50 gradient steps through the graph-captured step."""
    from paper_1506_00014_gb300.recon import LeastSquares

    N, na, nd = 1024, 720, 1536
    plan = rl.radon_plan_create(N, na, nd, 3, 3)
    step = None
    errs = []
    for sl in range(64):
        ell = random_ellipses(10, 200 + sl)
        g = ellipse_sinogram(ell, na, nd)
        g = g + np.random.default_rng(200 + sl).normal(0, 0.01 * np.abs(g).max(), g.shape)
        ls = LeastSquares(plan, _t(g), step=step, use_graph=True)
        step = ls.step
        l0 = ls.loss()
        ls.run(50)
        assert ls.loss() < 0.1 * l0
        if sl < 2:
            ref = ellipse_image(N, ell)
            errs.append(float(np.linalg.norm(ls.f.cpu().numpy() - ref) / np.linalg.norm(ref)))
    assert max(errs) < 0.5


def test_batched_least_squares_matches_per_slice(rl):
    """The batched autograd loop (batched C ABI, CUDA graph) follows the per-slice loop: both take
    x <- x - 2 c_R step R#(R x - g) for every slice."""
    from paper_1506_00014_gb300.recon import BatchedLeastSquares, LeastSquares, normal_operator_norm

    N, na, nd = 64, 96, 96
    plan = rl.radon_plan_create(N, na, nd, 3, 3)
    rl.radon_plan_reserve_batch(plan, 3)
    gs = torch.stack([_t(ellipse_sinogram(random_ellipses(5, 30 + b), na, nd)) for b in range(5)])
    step = 1.0 / (2.0 * normal_operator_norm(plan))
    ref = torch.stack([LeastSquares(plan, gs[b], step=step).run(15).clone() for b in range(5)])
    for use_graph in (False, True):  # the autograd gradient already carries the factor 2 c_R
        bl = BatchedLeastSquares(plan, gs, step=step, use_graph=use_graph)
        got = bl.run(15)
        assert float((got - ref).norm() / ref.norm()) < 1e-5
        l0 = (gs * gs).sum(dim=(1, 2))
        assert torch.all(bl.losses() < 0.5 * l0)


def test_em_keeps_positivity_and_fits_the_data(rl):
    from paper_1506_00014_gb300.recon import em

    N, na, nd = 128, 192, 128
    plan = rl.radon_plan_create(N, na, nd, 3, 3)
    ell = [e for e in random_ellipses(12, 9)]
    ell = [type(e)(e.cx, e.cy, e.a, e.b, e.psi, abs(e.density)) for e in ell]
    g = _t(ellipse_sinogram(ell, na, nd))
    f5 = em(plan, g, 5)
    f30 = em(plan, g, 30)
    assert float(f30.min()) >= 0.0

    def resid(f):
        s = torch.empty((na, nd), device="cuda")
        rl.radon_forward(plan, f.contiguous(), s)
        return float(torch.linalg.norm(s - g) / torch.linalg.norm(g))

    assert resid(f30) < resid(f5) < 1.0


def test_batched_em_on_a_slice_stack_equals_per_slice(rl):
    """em_batched (batched C ABI over a stack of slices) gives each slice the same bits as em()."""
    from paper_1506_00014_gb300.recon import em, em_batched

    N, na, nd = 64, 96, 64
    plan = rl.radon_plan_create(N, na, nd, 3, 3)
    rl.radon_plan_reserve_batch(plan, 2)
    stack = []
    for b in range(3):
        ell = [type(e)(e.cx, e.cy, e.a, e.b, e.psi, abs(e.density)) for e in random_ellipses(6, 50 + b)]
        stack.append(_t(ellipse_sinogram(ell, na, nd)))
    g = torch.stack(stack)
    got = em_batched(plan, g, 8)
    for b in range(3):
        assert torch.equal(got[b], em(plan, stack[b], 8))
