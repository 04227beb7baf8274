"""radon_forward_static_scratch: the forward transform for callers that must not allocate device
memory when they run it (for example code under a framework that owns every device allocation,
or a real-time loop with a fixed memory budget).  Its intermediates live in the library's static
device array; the result must equal radon_forward's on the same plan and input.

Collected last on purpose (file name), so a run that stops at the first failure has already run
every other test."""

import ctypes

import numpy as np
import pytest

from workloads import ellipse_image, random_ellipses, smooth_random_image

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5  # the relative L2 bar used by the other GPU tests
RADON_EXCEEDS_STATIC_SCRATCH = 6


@pytest.fixture(scope="module")
def lib():
    from paper_1506_00014_gb300 import binding, build

    if build.needs_build():
        build.build()
    c = binding.load()
    c.radon_forward_static_scratch.argtypes = [ctypes.c_void_p] * 4
    c.radon_forward_static_scratch.restype = ctypes.c_int
    return c


def _run_both(lib, plan, img):
    from paper_1506_00014_gb300 import binding

    f = torch.tensor(np.asarray(img, np.float32), device="cuda")
    ref = torch.full(plan.sino_shape, float("nan"), dtype=torch.float32, device="cuda")
    out = torch.full(plan.sino_shape, float("nan"), dtype=torch.float32, device="cuda")
    binding.radon_forward(plan, f, ref)
    stream = torch.cuda.current_stream().cuda_stream
    status = lib.radon_forward_static_scratch(plan.handle, f.data_ptr(), out.data_ptr(), stream)
    torch.cuda.synchronize()
    assert status == 0, binding.radon_status_string(status)
    ref, out = ref.cpu().numpy().astype(np.float64), out.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(out))
    return float(np.linalg.norm(out - ref) / np.linalg.norm(ref))


def test_static_scratch_forward_matches_radon_forward(lib):
    from paper_1506_00014_gb300 import binding

    plan_a = binding.radon_plan_create(128, 128, 192, 3, 3)
    plan_b = binding.radon_plan_create(96, 100, 150, 3, 4)
    # consecutive calls share the array: a smaller plan after a larger one, then the larger again
    assert _run_both(lib, plan_a, ellipse_image(128, random_ellipses(10, 1))) < TOL
    assert _run_both(lib, plan_b, smooth_random_image(96, 7)) < TOL
    assert _run_both(lib, plan_a, smooth_random_image(128, 8)) < TOL


def test_static_scratch_rejects_plans_that_do_not_fit(lib):
    from paper_1506_00014_gb300 import binding

    big = binding.radon_plan_create(1024, 1024, 1536, 3, 3)
    f = torch.zeros((1024, 1024), dtype=torch.float32, device="cuda")
    out = torch.zeros((1024, 1536), dtype=torch.float32, device="cuda")
    status = lib.radon_forward_static_scratch(big.handle, f.data_ptr(), out.data_ptr(),
                                              torch.cuda.current_stream().cuda_stream)
    assert status == RADON_EXCEEDS_STATIC_SCRATCH
    assert "static scratch" in binding.radon_status_string(status)
