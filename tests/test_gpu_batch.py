"""Batched slices: same-size batches in one set of launches, uneven sizes grouped, CUDA graph."""

import numpy as np
import pytest

from workloads import ellipse_image, random_ellipses, random_sinogram

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl():
    from paper_1506_00014_gb300 import build

    if build.needs_build():
        build.build()
    import paper_1506_00014_gb300 as rl

    return rl


def _t(a):
    return torch.tensor(np.asarray(a, np.float32), device="cuda")


@pytest.mark.parametrize("N,na,nd,interp", [(128, 128, 192, 3), (96, 100, 150, 1)])
def test_same_size_batch_equals_single_calls(rl, N, na, nd, interp):
    plan = rl.radon_plan_create(N, na, nd, interp, 3)
    rl.radon_plan_reserve_batch(plan, 4)
    imgs = torch.stack([_t(ellipse_image(N, random_ellipses(8, s))) for s in range(3)]).contiguous()
    sins = torch.stack([_t(random_sinogram(na, nd, 10 + s)) for s in range(3)]).contiguous()
    out_s = torch.empty((3, na, nd), device="cuda")
    out_i = torch.empty((3, N, N), device="cuda")
    rl.radon_forward_batch(plan, imgs, out_s)
    rl.radon_backproject_batch(plan, sins, out_i)
    for b in range(3):
        one_s = torch.empty((na, nd), device="cuda")
        one_i = torch.empty((N, N), device="cuda")
        rl.radon_forward(plan, imgs[b].contiguous(), one_s)
        rl.radon_backproject(plan, sins[b].contiguous(), one_i)
        assert torch.equal(out_s[b], one_s)
        assert torch.equal(out_i[b], one_i)


def test_batch_capacity_limits(rl):
    plan = rl.radon_plan_create(64, 64, 96, 3, 3)
    x = torch.zeros((2, 64, 64), device="cuda")
    y = torch.zeros((2, 64, 96), device="cuda")
    with pytest.raises(rl.RadonError):  # capacity is 1 until reserved
        rl.radon_forward_batch(plan, x, y)
    big = rl.radon_plan_create(1024, 1024, 1536, 3, 3)
    with pytest.raises(rl.RadonError) as err:  # ~10^6 slices of scratch (about 200 TB) cannot be allocated
        rl.radon_plan_reserve_batch(big, 1 << 20)
    assert err.value.status == 2  # RADON_OUT_OF_MEMORY
    # the plan keeps its previous capacity and still runs
    f = torch.zeros((1024, 1024), device="cuda")
    s = torch.full((1024, 1536), float("nan"), device="cuda")
    rl.radon_forward(big, f, s)
    torch.cuda.synchronize()
    assert float(s.abs().max()) == 0.0
    few = rl.radon_plan_create(4096, 64, 96, 3, 3)  # few angles: many sub-angles per coarse angle
    assert few.info["r"] > 32  # more than one anchor per lane in the sampling warps


def test_column_group_does_not_change_results(rl):
    N = 128
    plan = rl.radon_plan_create(N, N, 192, 3, 3)
    f = _t(ellipse_image(N, random_ellipses(10, 1)))
    outs = []
    for g in (1, 2, 4):
        rl.radon_plan_set_column_group(plan, g)
        s = torch.empty((N, 192), device="cuda")
        rl.radon_forward(plan, f, s)
        outs.append(s)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_specialised_column_kernel_matches_generic(rl):
    """Group 0 (in-place power-of-two column FFT) equals the generic kernel up to FP32 rounding;
    it is the default where n_theta allows it and refused elsewhere."""
    N, na, nd = 128, 384, 192  # n_theta = 256
    plan = rl.radon_plan_create(N, na, nd, 3, 3)
    assert plan.info["n_theta"] == 256 and plan.info["column_group"] == 0
    f = _t(ellipse_image(N, random_ellipses(10, 2)))
    g = torch.randn((na, nd), device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    res = {}
    for grp in (0, 1, 4):
        rl.radon_plan_set_column_group(plan, grp)
        s = torch.empty((na, nd), device="cuda")
        b = torch.empty((N, N), device="cuda")
        rl.radon_forward(plan, f, s)
        rl.radon_backproject(plan, g, b)
        res[grp] = (s, b)
    for k in range(2):
        a, ref = res[0][k], res[1][k]
        assert float((a - ref).norm() / ref.norm()) < 2e-6
        assert torch.equal(res[1][k], res[4][k])
    other = rl.radon_plan_create(128, 128, 192, 3, 3)  # n_theta = 96: generic only
    assert other.info["column_group"] in (1, 2, 4)
    with pytest.raises(rl.RadonError) as err:
        rl.radon_plan_set_column_group(other, 0)
    assert err.value.status == 5  # RADON_NOT_SUPPORTED


def test_uneven_batch_with_graph_matches_per_slice(rl):
    from paper_1506_00014_gb300.batch import UnevenBatch

    sizes = [64, 128, 64, 96, 128, 64]
    ub = UnevenBatch(sizes, max_batch=2)
    choice = ub.tune()
    assert set(choice) == {64, 96, 128}
    assert all(1 <= c <= 2 and g in (0, 1, 2, 4) and M == 3 for c, g, M in choice.values())
    imgs = [_t(ellipse_image(n, random_ellipses(6, 40 + i))) for i, n in enumerate(sizes)]
    ub.set_images(imgs)
    ub.forward()
    eager = [ub.sinogram(i).clone() for i in range(len(sizes))]
    for i, n in enumerate(sizes):
        plan = ub.plans[n]
        one = torch.empty(plan.sino_shape, device="cuda")
        rl.radon_forward(plan, imgs[i], one)
        assert torch.equal(one, eager[i])
    ub.capture(lambda: ub.forward())
    ub.set_images(imgs)
    ub.replay()
    torch.cuda.synchronize()
    for i in range(len(sizes)):
        assert torch.equal(ub.sinogram(i), eager[i])


def test_uneven_batch_tunes_the_partition_count_and_matches_the_oracle(rl):
    """With candidate partition counts the tuner keeps the fastest M per size; every slice then
    matches the FP64 log-polar oracle at that M (Algorithms 1 and 2 with beta = pi / M)."""
    from oracle import geometry, logpolar
    from paper_1506_00014_gb300.batch import UnevenBatch

    sizes = [64, 96, 64, 128]
    ub = UnevenBatch(sizes, n_partitions=(3, 4), max_batch=2)
    choice = ub.tune()
    assert set(choice) == {64, 96, 128} and all(M in (3, 4) for _, _, M in choice.values())
    imgs = [_t(ellipse_image(n, random_ellipses(6, 50 + i))) for i, n in enumerate(sizes)]
    ub.capture()  # runs R then R# once before capturing: the inputs are set afterwards
    ub.set_images(imgs)
    ub.replay()
    torch.cuda.synchronize()
    for i, n in enumerate(sizes):
        M = choice[n][2]
        assert ub.plans[n].info["n_partitions"] == M
        geo = geometry.make_geometry(n, n, 3 * n // 2, M, 3)
        ref_s = logpolar.forward(imgs[i].cpu().numpy().astype(np.float64), geo)
        got_s = ub.sinogram(i).cpu().numpy()
        assert np.linalg.norm(got_s - ref_s) / np.linalg.norm(ref_s) < 1e-5
        ref_b = logpolar.backproject(got_s.astype(np.float64), geo)
        got_b = ub.image(i).cpu().numpy()
        assert np.linalg.norm(got_b - ref_b) / np.linalg.norm(ref_b) < 1e-5


def test_multi_plan_calls_equal_per_slice_calls(rl):
    """radon_forward_multi / radon_backproject_multi over plans of different sizes (one plan used
    twice) equal per-slice calls bit for bit, also when replayed from a CUDA graph."""
    sizes = [(64, 64, 96), (96, 100, 150), (64, 64, 96), (128, 128, 192)]
    plans = {}
    for n, na, nd in sizes:
        plans.setdefault((n, na, nd), rl.radon_plan_create(n, na, nd, 3, 3))
    pl = [plans[s] for s in sizes]
    imgs = [_t(ellipse_image(n, random_ellipses(6, 70 + i))) for i, (n, _, _) in enumerate(sizes)]
    sins = [_t(random_sinogram(na, nd, 80 + i)) for i, (_, na, nd) in enumerate(sizes)]
    out_s = [torch.empty((na, nd), device="cuda") for _, na, nd in sizes]
    out_i = [torch.empty((n, n), device="cuda") for n, _, _ in sizes]
    rl.radon_forward_multi(pl, imgs, out_s)
    rl.radon_backproject_multi(pl, sins, out_i)
    torch.cuda.synchronize()
    for k, (n, na, nd) in enumerate(sizes):
        one_s = torch.empty((na, nd), device="cuda")
        one_i = torch.empty((n, n), device="cuda")
        rl.radon_forward(pl[k], imgs[k], one_s)
        rl.radon_backproject(pl[k], sins[k], one_i)
        torch.cuda.synchronize()
        assert torch.equal(one_s, out_s[k]) and torch.equal(one_i, out_i[k])
    ref_s = [t.clone() for t in out_s]
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        rl.radon_forward_multi(pl, imgs, out_s)
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(graph):
        rl.radon_forward_multi(pl, imgs, out_s)
    for t in out_s:
        t.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(out_s, ref_s))
    with pytest.raises(ValueError):
        rl.radon_forward_multi(pl, imgs[:2], out_s)
