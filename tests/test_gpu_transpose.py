"""GPU parity of the exact transpose R^T (radon_transpose) against the oracle's transpose of
Algorithm 1, and the dot-product identity <R f, g> = <f, R^T g> of the CUDA path itself, at
small sizes with ragged tiles and at the full N = 2048, 2048 x 3072 size.  The scatters use FP32
atomics, so repeated calls agree to rounding rather than bit for bit."""

import numpy as np
import pytest

from oracle import geometry, kernels, logpolar
from workloads import ellipse_image, random_ellipses, random_sinogram, smooth_random_image

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative L2 against the FP64 oracle, as for R and R#


@pytest.fixture(scope="module")
def rl():
    from paper_1506_00014_gb300 import build

    if build.needs_build():
        build.build()
    import paper_1506_00014_gb300 as rl

    return rl


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def _gpu_transpose(rl, plan, g):
    out = torch.full(plan.image_shape, float("nan"), dtype=torch.float32, device="cuda")
    rl.radon_transpose(plan, _dev(g), out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _dot_gap(Rf, g, f, Rtg):
    """|<R f, g> - <f, R^T g>| over ||R f|| ||g|| (the Cauchy-Schwarz bound of either side):
    random f and g make the sums themselves cancel to far below that bound."""
    return abs(np.sum(Rf * g) - np.sum(f * Rtg)) / (np.linalg.norm(Rf) * np.linalg.norm(g))


def _gpu_forward(rl, plan, f):
    out = torch.full(plan.sino_shape, float("nan"), dtype=torch.float32, device="cuda")
    rl.radon_forward(plan, _dev(f), out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


CASES = [
    (128, 128, 192, 3, 3),   # the small CPU configuration
    (128, 128, 192, 1, 3),   # linear interpolation
    (96, 100, 150, 3, 4),    # M = 4, ragged angle / detector counts
    (200, 150, 310, 3, 3),   # image not a multiple of the tiles
    (64, 37, 90, 3, 5),      # M = 5, odd angle count
    (16, 5, 20, 1, 3),       # tiny, linear, n_theta_half = 2
    (64, 2048, 96, 3, 3),    # n_theta = 1372 (the specialised forward column kernel's length)
]


@pytest.mark.parametrize("N,na,nd,interp,M", CASES)
def test_transpose_matches_oracle_transpose(rl, N, na, nd, interp, M):
    geo = geometry.make_geometry(N, na, nd, M, interp)
    plan = rl.radon_plan_create(N, na, nd, interp, M)
    K = kernels.multiplier(geo, "R")
    dft = logpolar._Dft(geo)
    th = np.arange(na) * geo.dtheta
    s = (np.arange(nd) - nd / 2) * geo.ds
    smooth = np.exp(-((s[None, :] - 0.3 * np.cos(th[:, None])) ** 2) / 0.02)
    for g in (random_sinogram(na, nd, 31), smooth):
        ref = logpolar.transpose(_f32(g), geo, K=K, dft=dft)
        got = _gpu_transpose(rl, plan, g)
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) < TOL, _rel(got, ref)
        assert np.all(got[~geometry.disc_mask(N)] == 0.0)


@pytest.mark.parametrize("N,na,nd,interp,M", CASES[:5])
def test_cuda_path_satisfies_the_dot_product_identity(rl, N, na, nd, interp, M):
    plan = rl.radon_plan_create(N, na, nd, interp, M)
    rng = np.random.default_rng(N + na)
    f = rng.standard_normal((N, N))
    g = rng.standard_normal((na, nd))
    gap = _dot_gap(_gpu_forward(rl, plan, f), _f32(g), _f32(f), _gpu_transpose(rl, plan, g))
    assert gap < 1e-6, gap


def test_forward_is_unchanged_after_a_transpose_on_the_same_plan(rl):
    """The transpose shares the plan's scratch (it scatters into the coefficient image that the
    linear forward reads); the zero border must survive, so R f is bit-identical afterwards."""
    for interp in (1, 3):
        plan = rl.radon_plan_create(96, 80, 150, interp, 3)
        f = ellipse_image(96, random_ellipses(10, 7))
        before = _gpu_forward(rl, plan, f)
        _gpu_transpose(rl, plan, random_sinogram(80, 150, 8))
        assert np.array_equal(_gpu_forward(rl, plan, f), before)


def test_batched_transpose_equals_per_slice(rl):
    plan = rl.radon_plan_create(64, 48, 96, 3, 3)
    rl.radon_plan_reserve_batch(plan, 3)
    gs = [random_sinogram(48, 96, 40 + i) for i in range(3)]
    out = torch.empty((3, 64, 64), device="cuda")
    rl.radon_transpose_batch(plan, torch.stack([_dev(g) for g in gs]), out)
    torch.cuda.synchronize()
    for i, g in enumerate(gs):
        one = _gpu_transpose(rl, plan, g)
        assert _rel(out[i].cpu().numpy().astype(np.float64), one) < 1e-6


def test_transpose_launches_and_stages(rl):
    plan = rl.radon_plan_create(64, 64, 96, 3, 3)
    assert rl.radon_plan_kernel_launches(plan, "transpose") == 6
    rl.radon_profile_enable(plan, True)
    rl.radon_profile_read(plan)
    g = torch.zeros((64, 96), device="cuda")
    f = torch.empty((64, 64), device="cuda")
    rl.radon_transpose(plan, g, f)
    stages = rl.radon_profile_read(plan)
    rl.radon_profile_enable(plan, False)
    ran = {k for k, (ms, n) in stages.items() if n}
    assert ran == set(rl.binding.TRANSPOSE_STAGES)
    assert all(stages[k][1] == 1 for k in ran)
    assert torch.count_nonzero(f).item() == 0  # R^T 0 = 0 exactly


def test_exact_autograd_backward_is_the_transpose(rl):
    from paper_1506_00014_gb300 import autograd

    plan = rl.radon_plan_create(64, 48, 96, 3, 3)
    f = _dev(smooth_random_image(64, 3)).requires_grad_(True)
    w = _dev(random_sinogram(48, 96, 4))
    (autograd.radon(f, plan, exact=True) * w).sum().backward()
    ref = _gpu_transpose(rl, plan, w.cpu().numpy())
    assert _rel(f.grad.cpu().numpy().astype(np.float64), ref) < 1e-6
    # directional derivative of the (linear) loss along v equals <R v, w>
    v = np.random.default_rng(5).standard_normal((64, 64))
    gap = _dot_gap(_gpu_forward(rl, plan, v), w.cpu().numpy().astype(np.float64), _f32(v),
                   f.grad.cpu().numpy().astype(np.float64))
    assert gap < 1e-6, gap


def test_full_size_transpose(rl):
    """N = 2048, 2048 x 3072, cubic, M = 3: the dot-product identity of the CUDA path on the
    full workload, and R^T against the oracle's transpose on partition 0 (the oracle's
    transpose is linear in g, so a sinogram supported on partition 0's angles isolates it)."""
    N, na, nd = 2048, 2048, 3072
    plan = rl.radon_plan_create(N, na, nd, 3, 3)
    f = ellipse_image(N, random_ellipses(50, 2))
    g = random_sinogram(na, nd, 3)
    gap = _dot_gap(_gpu_forward(rl, plan, f), _f32(g), _f32(f), _gpu_transpose(rl, plan, g))
    assert gap < 1e-6, gap
    geo = geometry.make_geometry(N, na, nd, 3, 3)
    g0 = np.zeros_like(g)
    for a in range(na):
        if geometry.angle_partition(a, na, 3)[0] == 0:
            g0[a] = g[a]
    ref = logpolar.transpose(_f32(g0), geo, partitions=[0])
    got = _gpu_transpose(rl, plan, g0)
    assert _rel(got, ref) < TOL, _rel(got, ref)
