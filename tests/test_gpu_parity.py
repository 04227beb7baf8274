"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar (the stated target of this build): relative L2 error <= 1e-5 against the log-polar oracle
for both R and R#, cubic and linear, on the same seeded inputs.  Sizes span several tiles with
ragged tails; the full N = 2048 case runs the whole oracle (about a minute of CPU time).
"""

import math

import numpy as np
import pytest

from oracle import direct, fbp, geometry, kernels, logpolar
from workloads import ellipse_image, gaussian_image, random_ellipses, random_sinogram, smooth_random_image

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def rl():
    from paper_1506_00014_gb300 import build

    if build.needs_build():
        build.build()
    import paper_1506_00014_gb300 as rl

    return rl


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def _gpu_forward(rl, plan, f, stream=None):
    fd = torch.tensor(np.asarray(f, dtype=np.float32), device="cuda")
    out = torch.full(plan.sino_shape, float("nan"), dtype=torch.float32, device="cuda")
    rl.radon_forward(plan, fd, out, stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _gpu_back(rl, plan, g, stream=None):
    gd = torch.tensor(np.asarray(g, dtype=np.float32), device="cuda")
    out = torch.full(plan.image_shape, float("nan"), dtype=torch.float32, device="cuda")
    rl.radon_backproject(plan, gd, out, stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


CASES = [
    (128, 128, 192, 3, 3),   # the small CPU configuration
    (128, 128, 192, 1, 3),   # linear interpolation
    (96, 100, 150, 3, 4),    # M = 4, ragged angle / detector counts
    (200, 150, 310, 3, 3),   # image not a multiple of the 16 / 32 tiles
    (64, 37, 90, 3, 5),      # M = 5, odd angle count
    (16, 12, 24, 3, 3),      # tiny
    (16, 5, 20, 1, 3),       # tiny, linear, n_theta_half = 2
    (128, 384, 192, 3, 3),   # n_theta = 256: specialised in-place column kernel (16 x 16)
    (160, 1024, 240, 1, 4),  # n_theta = 512 (8 x 8 x 8), M = 4, linear
    (96, 1536, 150, 3, 3),   # n_theta = 1024 (16 x 8 x 8)
    (64, 2048, 96, 3, 3),    # n_theta = 1372 (14 x 14 x 7, 392 threads)
    (64, 4096, 96, 3, 3),    # n_theta = 2744 (14 x 14 x 14, 2 columns per work item)
    (120, 180, 170, 3, 3),   # r = 4 sub-angles (1.5 N angles), ragged image tiles
    (100, 100, 150, 3, 4),   # r = 6 sub-angles, n_theta_half = 28: a partial group of 8 rows
]


def _inputs(N, na, nd, seed):
    img_ell = ellipse_image(N, random_ellipses(10, seed))
    img_smooth = smooth_random_image(N, seed + 1)
    rng = np.random.default_rng(seed + 2)
    img_noise = rng.standard_normal((N, N))
    sino_noise = random_sinogram(na, nd, seed + 3)
    return img_ell, img_smooth, img_noise, sino_noise


@pytest.mark.parametrize("N,na,nd,interp,M", CASES)
def test_forward_matches_logpolar_oracle(rl, N, na, nd, interp, M):
    geo = geometry.make_geometry(N, na, nd, M, interp)
    plan = rl.radon_plan_create(N, na, nd, interp, M)
    K = kernels.multiplier(geo, "R")
    dft = logpolar._Dft(geo)
    for img in _inputs(N, na, nd, 11)[:3]:
        ref = logpolar.forward(_f32(img), geo, K=K, dft=dft)
        got = _gpu_forward(rl, plan, img)
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) < TOL, _rel(got, ref)


@pytest.mark.parametrize("N,na,nd,interp,M", CASES)
def test_backprojection_matches_logpolar_oracle(rl, N, na, nd, interp, M):
    geo = geometry.make_geometry(N, na, nd, M, interp)
    plan = rl.radon_plan_create(N, na, nd, interp, M)
    K = kernels.multiplier(geo, "B")
    dft = logpolar._Dft(geo)
    sino = _inputs(N, na, nd, 21)[3]
    th = np.arange(na) * geo.dtheta
    s = (np.arange(nd) - nd / 2) * geo.ds
    blobs = [(0.2, -0.1, 0.12, 1.0), (-0.3, 0.25, 0.08, -0.7)]
    smooth = direct.gaussian_radon(th[:, None], s[None, :], blobs)
    for g in (sino, smooth):
        ref = logpolar.backproject(_f32(g), geo, K=K, dft=dft)
        got = _gpu_back(rl, plan, g)
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) < TOL, _rel(got, ref)


def _gpu_fbp(rl, plan, g, kind):
    gd = torch.tensor(np.asarray(g, dtype=np.float32), device="cuda")
    out = torch.full(plan.image_shape, float("nan"), dtype=torch.float32, device="cuda")
    rl.radon_fbp(plan, gd, out, kind)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("N,na,nd,interp,M", CASES[:5])
def test_fbp_matches_oracle(rl, N, na, nd, interp, M):
    geo = geometry.make_geometry(N, na, nd, M, interp)
    plan = rl.radon_plan_create(N, na, nd, interp, M)
    K = kernels.multiplier(geo, "B")
    dft = logpolar._Dft(geo)
    g = random_sinogram(na, nd, 31)
    for kind, name in enumerate(fbp.FILTERS):
        ref = fbp.fbp(_f32(g), geo, name, K=K, dft=dft)
        got = _gpu_fbp(rl, plan, g, kind)
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) < TOL, (name, _rel(got, ref))


# One shape per sampling-kernel variant (r = 4, 5, 6 sub-angles and r = 7 on the one-warp-per-row
# form) and the two radix-7 theta lengths (1372, 2744).
INVARIANT_CASES = [
    (120, 180, 170, 3, 3),
    (128, 128, 192, 3, 3),
    (100, 100, 150, 3, 4),
    (200, 150, 310, 3, 3),
    (64, 2048, 96, 3, 3),
    (64, 4096, 96, 3, 3),
]


@pytest.mark.parametrize("N,na,nd,interp,M", INVARIANT_CASES)
def test_scaling_by_two_is_exact_and_runs_repeat_bit_for_bit(rl, N, na, nd, interp, M):
    """R and R# are linear and every step is a sum of products of the input with data-independent
    weights, so scaling the input by 2 (exact in FP32) scales each output exactly; no step depends
    on the run (no atomics in R or R#), so a repeated call gives the same bits."""
    plan = rl.radon_plan_create(N, na, nd, interp, M)
    f = ellipse_image(N, random_ellipses(10, 41)) + 0.3 * smooth_random_image(N, 42)
    g = random_sinogram(na, nd, 43)
    rf = _gpu_forward(rl, plan, f)
    assert np.array_equal(_gpu_forward(rl, plan, 2.0 * f), 2.0 * rf)
    assert np.array_equal(_gpu_forward(rl, plan, f), rf)
    bg = _gpu_back(rl, plan, g)
    assert np.array_equal(_gpu_back(rl, plan, 2.0 * g), 2.0 * bg)
    assert np.array_equal(_gpu_back(rl, plan, g), bg)
    assert np.count_nonzero(rf) > 0 and np.count_nonzero(bg) > 0


def test_zero_and_out_of_support_inputs_give_exact_zeros(rl):
    N, na, nd = 64, 64, 96
    plan = rl.radon_plan_create(N, na, nd, 3, 3)
    assert np.count_nonzero(_gpu_forward(rl, plan, np.zeros((N, N)))) == 0
    outside = np.where(geometry.disc_mask(N), 0.0, 1.0)  # only pixels with |x| >= 1
    assert np.count_nonzero(_gpu_forward(rl, plan, outside)) == 0
    dead = np.where(geometry.live_bins(nd)[None, :], 0.0, np.ones((na, nd)))  # only bins with |s| >= 1
    assert np.count_nonzero(_gpu_back(rl, plan, dead)) == 0
    # outputs outside the support are exactly zero
    rf = _gpu_forward(rl, plan, np.ones((N, N)))
    assert np.count_nonzero(rf[:, ~geometry.live_bins(nd)]) == 0
    bp = _gpu_back(rl, plan, np.ones((na, nd)))
    assert np.count_nonzero(bp[~geometry.disc_mask(N)]) == 0


def test_deterministic_and_stream_ordered(rl):
    N, na, nd = 256, 256, 384
    plan = rl.radon_plan_create(N, na, nd, 3, 3)
    f = ellipse_image(N, random_ellipses(20, 5))
    a = _gpu_forward(rl, plan, f)
    side = torch.cuda.Stream()
    b = _gpu_forward(rl, plan, f, stream=side)
    assert np.array_equal(a, b)
    g = random_sinogram(na, nd, 6)
    assert np.array_equal(_gpu_back(rl, plan, g), _gpu_back(rl, plan, g, stream=side))


def test_plans_of_different_sizes_coexist(rl):
    """A plan stays usable after a smaller (or larger) plan is created on the same device."""
    big = rl.radon_plan_create(256, 256, 384, 3, 3)
    small = rl.radon_plan_create(32, 32, 48, 3, 3)
    f_big = ellipse_image(256, random_ellipses(10, 4))
    geo = geometry.make_geometry(256, 256, 384, 3, 3)
    ref = logpolar.forward(_f32(f_big), geo)
    assert _rel(_gpu_forward(rl, big, f_big), ref) < TOL
    assert np.all(np.isfinite(_gpu_forward(rl, small, ellipse_image(32, random_ellipses(3, 4)))))
    assert _rel(_gpu_forward(rl, big, f_big), ref) < TOL


def test_host_buffer_entry_points_match_device_ones(rl):
    N, na, nd = 128, 128, 192
    plan = rl.radon_plan_create(N, na, nd, 3, 3)
    f = ellipse_image(N, random_ellipses(10, 1)).astype(np.float32)
    g = random_sinogram(na, nd, 3).astype(np.float32)
    hs = np.zeros((na, nd), np.float32)
    hi = np.zeros((N, N), np.float32)
    rl.radon_forward_host(plan, f, hs)
    rl.radon_backproject_host(plan, g, hi)
    assert np.array_equal(hs.astype(np.float64), _gpu_forward(rl, plan, f))
    assert np.array_equal(hi.astype(np.float64), _gpu_back(rl, plan, g))


def test_concurrent_plans_on_two_streams_match_serial(rl):
    """R with one plan and R# with another, on two streams at once (how the benchmark runs a step),
    give the same bits as running them one after the other."""
    N, na, nd = 256, 384, 384
    p1 = rl.radon_plan_create(N, na, nd, 3, 3)
    p2 = rl.radon_plan_create(N, na, nd, 3, 3)
    f = torch.tensor(ellipse_image(N, random_ellipses(20, 8)).astype(np.float32), device="cuda")
    g = torch.tensor(random_sinogram(na, nd, 9).astype(np.float32), device="cuda")
    s_ref = torch.empty((na, nd), device="cuda")
    i_ref = torch.empty((N, N), device="cuda")
    rl.radon_forward(p1, f, s_ref)
    rl.radon_backproject(p1, g, i_ref)
    main, side = torch.cuda.current_stream(), torch.cuda.Stream()
    s, i = torch.empty_like(s_ref), torch.empty_like(i_ref)
    for _ in range(3):
        side.wait_stream(main)
        rl.radon_forward(p1, f, s, main)
        rl.radon_backproject(p2, g, i, side)
        main.wait_stream(side)
    torch.cuda.synchronize()
    assert torch.equal(s, s_ref) and torch.equal(i, i_ref)


def test_kernel_launch_counts(rl):
    plan = rl.radon_plan_create(64, 64, 96, 3, 3)
    assert rl.radon_plan_kernel_launches(plan, "forward") == 6
    assert rl.radon_plan_kernel_launches(plan, "backproject") == 5
    assert rl.radon_plan_kernel_launches(plan, "fbp") == 6
    assert rl.load().radon_plan_kernel_launches(plan.handle, 7, None) == 1  # RADON_INVALID_ARG
    # the per-stage profile sees one launch per stage and call
    rl.radon_profile_enable(plan, True)
    rl.radon_profile_read(plan)
    f = torch.zeros((64, 64), device="cuda")
    s = torch.empty((64, 96), device="cuda")
    rl.radon_forward(plan, f, s)
    rl.radon_backproject(plan, s, f)
    stages = rl.radon_profile_read(plan)
    rl.radon_profile_enable(plan, False)
    ran = {k for k, (ms, n) in stages.items() if n}
    assert ran == {"prefilter_image", "sample_fwd", "rows_fwd", "columns_fwd", "rows_inv_fwd", "gather_sino",
                   "prefilter_sino", "rows_bp", "columns_bp", "rows_inv_bp", "gather_image"}
    assert all(n == 1 for k, (ms, n) in stages.items() if k in ran)


def test_invalid_arguments_raise(rl):
    plan = rl.radon_plan_create(32, 32, 48, 3, 3)
    with pytest.raises(TypeError):
        rl.radon_forward(plan, torch.zeros((32, 32)), torch.zeros((32, 48), device="cuda"))
    with pytest.raises(ValueError):
        rl.radon_forward(plan, torch.zeros((32, 33), device="cuda"), torch.zeros((32, 48), device="cuda"))
    lib = rl.load()
    assert lib.radon_forward(plan.handle, None, None, None) == 1  # RADON_INVALID_ARG
    assert lib.radon_backproject(None, None, None, None) == 1


# ------------------------------------------------------------------ full size (N = 2048)

@pytest.fixture(scope="module")
def full_geo():
    return {interp: geometry.make_geometry(2048, 2048, 3072, 3, interp) for interp in (3, 1)}


@pytest.mark.parametrize("interp", [3, 1])
def test_full_size_forward_matches_oracle(rl, full_geo, interp):
    geo = full_geo[interp]
    plan = rl.radon_plan_create(2048, 2048, 3072, interp, 3)
    f = ellipse_image(2048, random_ellipses(50, 2))
    got = _gpu_forward(rl, plan, f)
    ref = logpolar.forward(_f32(f), geo)
    assert _rel(got, ref) < TOL, _rel(got, ref)


@pytest.mark.parametrize("interp", [3, 1])
def test_full_size_backprojection_matches_oracle(rl, full_geo, interp):
    geo = full_geo[interp]
    plan = rl.radon_plan_create(2048, 2048, 3072, interp, 3)
    g = random_sinogram(2048, 3072, 3)
    got = _gpu_back(rl, plan, g)
    ref = logpolar.backproject(_f32(g), geo)
    assert _rel(got, ref) < TOL, _rel(got, ref)


def test_full_size_four_partitions_match_oracle(rl):
    """M = 4 at the full single-slice size (the lattice the batch tuner picks for N = 2048:
    n_theta = 1024, N_rho = 3500): R of the ellipse phantom and R# of the noise sinogram."""
    geo = geometry.make_geometry(2048, 2048, 3072, 4, 3)
    plan = rl.radon_plan_create(2048, 2048, 3072, 3, 4)
    assert (plan.info["n_theta"], plan.info["N_rho"]) == (geo.n_theta, geo.N_rho) == (1024, 3500)
    f = ellipse_image(2048, random_ellipses(50, 2))
    got = _gpu_forward(rl, plan, f)
    ref = logpolar.forward(_f32(f), geo)
    assert _rel(got, ref) < TOL, _rel(got, ref)
    g = random_sinogram(2048, 3072, 3)
    got = _gpu_back(rl, plan, g)
    ref = logpolar.backproject(_f32(g), geo)
    assert _rel(got, ref) < TOL, _rel(got, ref)


def test_full_size_fbp_matches_oracle(rl, full_geo):
    geo = full_geo[3]
    plan = rl.radon_plan_create(2048, 2048, 3072, 3, 3)
    g = random_sinogram(2048, 3072, 7)
    got = _gpu_fbp(rl, plan, g, 1)
    ref = fbp.fbp(_f32(g), geo, "shepp-logan")
    assert _rel(got, ref) < TOL, _rel(got, ref)


# ------------------------------------------------------------------ large sizes: closed forms

@pytest.mark.parametrize("N", [4096, 8192])
def test_large_sizes_against_closed_forms(rl, N):
    """At sizes the oracle cannot finish, R of sampled Gaussians must match their analytic
    Radon transform and R# of the analytic sinogram its closed-form back-projection."""
    na, nd = N, 3 * N // 2
    plan = rl.radon_plan_create(N, na, nd, 3, 3)
    geo = geometry.make_geometry(N, na, nd, 3, 3)
    blobs = [(0.2, -0.1, 0.12, 1.0), (-0.3, 0.25, 0.08, -0.7), (0.05, 0.5, 0.1, 0.4)]
    th = np.arange(na) * geo.dtheta
    s = (np.arange(nd) - nd / 2) * geo.ds
    sino = direct.gaussian_radon(th[:, None], s[None, :], blobs)
    sino[:, ~geometry.live_bins(nd)] = 0.0
    got = _gpu_forward(rl, plan, gaussian_image(N, blobs))
    assert _rel(got, sino) < 2e-5
    x = (np.arange(N) - N / 2) * (2.0 / N)
    bp = np.zeros((N, N))
    for cx, cy, sg, w in blobs:
        bp += w * math.sqrt(2 * math.pi) * sg * direct.gaussian_bp(np.hypot(x[None, :] - cx, x[:, None] - cy), sg)
    bp[~geometry.disc_mask(N)] = 0.0
    assert _rel(_gpu_back(rl, plan, sino), bp) < 2e-5
    # FBP with the Shepp-Logan window (Eq. FBP, Eq. SLfilt) of the analytic sinogram returns the
    # Gaussians themselves on the disc (at N = 8192 this is the 8192 x 12288 FBP workload)
    ref = np.where(geometry.disc_mask(N), gaussian_image(N, blobs), 0.0)
    err = _rel(_gpu_fbp(rl, plan, sino, 1), ref)
    assert err < 1e-3, err
