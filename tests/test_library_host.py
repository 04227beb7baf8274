"""Host-side checks of libradon (no GPU): exported symbols, geometry rules and the kernel
transforms computed by the plan (trapezoid rule + end corrections, Eq. weightsa) against the
oracle's Gauss-Legendre values."""

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import geometry, kernels

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1506_00014_gb300 import binding, build

    build.build()
    return binding


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "radon.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(radon_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol(lib):
    declared = _declared_symbols()
    assert len(declared) >= 11
    cdll = ctypes.CDLL(lib.library_path())
    for name in declared:
        assert hasattr(cdll, name), name
    assert set(declared) == set(lib.EXPORTED)


def test_profiling_stage_table_matches_header(lib):
    src = open(os.path.join(ROOT, "include", "radon.h")).read()
    n = int(re.search(r"#define\s+RADON_NUM_STAGES\s+(\d+)", src).group(1))
    assert lib.RADON_NUM_STAGES == n == len(lib.STAGE_NAMES)
    assert len(set(lib.STAGE_NAMES)) == n


@pytest.mark.parametrize("args", [(128, 128, 192, 3, 3), (2048, 2048, 3072, 3, 3), (1024, 720, 1536, 3, 3),
                                  (96, 100, 150, 1, 4), (8192, 8192, 12288, 3, 3), (64, 37, 90, 3, 5)])
def test_geometry_matches_oracle_rules(lib, args):
    N, na, nd, interp, M = args
    g = lib.radon_geometry(N, na, nd, interp, M)
    o = geometry.make_geometry(N, na, nd, M, interp)
    assert (g["N_rho"], g["n_theta_half"], g["n_theta"], g["r"]) == (o.N_rho, o.n_th_h, o.n_theta, o.r)
    for a, b in (("beta", "beta"), ("a_R", "a_R"), ("a_r", "a_r"), ("L", "L"), ("d_phi", "dphi"),
                 ("d_rho", "drho"), ("d_s", "ds"), ("d_theta", "dtheta")):
        assert g[a] == pytest.approx(getattr(o, b), rel=1e-15)
    assert g["n_quad"] >= 8 * g["n_theta"]


def test_invalid_geometry_is_rejected(lib):
    for args in ((7, 8, 8, 3, 3), (6, 8, 8, 3, 3), (16, 8, 8, 2, 3), (16, 8, 8, 3, 2), (16, 1, 8, 3, 3)):
        with pytest.raises(lib.RadonError):
            lib.radon_geometry(*args)


@pytest.mark.parametrize("N,na,nd,M", [(64, 64, 96, 3), (128, 128, 192, 3), (256, 256, 384, 4),
                                       (16, 5, 20, 3), (16, 12, 24, 3), (64, 37, 90, 5)])
def test_plan_kernel_transforms_match_oracle(lib, N, na, nd, M):
    o = geometry.make_geometry(N, na, nd, M)
    for which, key in ((0, "R"), (1, "B")):
        plan_k = lib.radon_kernel_quadrant(N, na, nd, M, which)
        ref = kernels.kernel_quadrant(o, key)
        assert plan_k.shape == ref.shape
        assert np.max(np.abs(plan_k - ref)) < 1e-8 * np.max(np.abs(ref))


@pytest.mark.parametrize("N,na,nd,M", [(2048, 2048, 3072, 3), (1024, 720, 1536, 3), (4096, 4096, 6144, 3)])
def test_plan_kernel_transforms_match_oracle_at_full_size(lib, N, na, nd, M):
    """The plan's kernel tables at the full single-slice sizes (n_quad = 2^17 trapezoid nodes at
    N = 2048, pruned to the needed DFT bins over interleaved subsequences) against the oracle's
    Gauss-Legendre values on a seeded subset of k_rho columns: every k_theta, the first and last
    columns, and 40 random ones."""
    o = geometry.make_geometry(N, na, nd, M)
    rng = np.random.default_rng(2048)
    kmax = o.N_rho // 2
    cols = np.unique(np.concatenate([[0, 1, 2, kmax - 1, kmax], rng.integers(0, kmax + 1, 40)]))
    for which, key in ((0, "R"), (1, "B")):
        plan_k = lib.radon_kernel_quadrant(N, na, nd, M, which)
        assert plan_k.shape == (o.n_theta // 2 + 1, kmax + 1)
        ref = kernels.kernel_quadrant(o, key, kr_cols=cols)
        assert np.max(np.abs(plan_k[:, cols] - ref)) < 1e-8 * np.max(np.abs(ref)), key


def test_end_correction_weights_are_exact_to_degree_six():
    """Eq. weightsa: with f(a + j h) the moments sum_j c_j j^p / 120960 equal the
    Euler-Maclaurin end terms 0, 1/12, 0, -1/720 * 3!, 0, 1/30240 * 5!, 0."""
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "end_correction_weights.txt"))
            if l.strip() and not l.startswith("#")]
    c = np.array([float(v) for _, v in rows])
    j = np.arange(7.0)
    from math import factorial
    expect = [0.0, 1 / 12, 0.0, -factorial(3) / 720, 0.0, factorial(5) / 30240, 0.0]
    for p in range(7):
        assert np.sum(c * j**p) / 120960 == pytest.approx(expect[p], abs=1e-15)


def test_every_entry_point_rejects_null_arguments_without_a_gpu(lib):
    """The C ABI's argument checks run before any CUDA call: a NULL plan or pointer returns
    RADON_INVALID_ARG (1) from every entry point, with or without a device."""
    cdll = lib.load()
    for name in ("radon_forward", "radon_backproject", "radon_transpose", "radon_forward_host",
                 "radon_backproject_host", "radon_forward_static_scratch"):
        assert getattr(cdll, name)(None, None, None, None) == 1, name
    for name in ("radon_forward_batch", "radon_backproject_batch", "radon_transpose_batch"):
        assert getattr(cdll, name)(None, None, None, 1, None) == 1, name
    assert cdll.radon_fbp(None, None, None, 0, None) == 1
    for name in ("radon_forward_multi", "radon_backproject_multi"):
        assert getattr(cdll, name)(None, None, None, 1, None) == 1, name
        null = (ctypes.c_void_p * 2)(None, None)  # a list holding NULL plans is rejected before any launch
        assert getattr(cdll, name)(null, null, null, 2, None) == 1, name
    assert cdll.radon_plan_kernel_launches(None, 3, None) == 1
    assert cdll.radon_plan_reserve_batch(None, 2) == 1
    assert cdll.radon_plan_set_column_group(None, 1) == 1
    assert cdll.radon_profile_enable(None, 1) == 1
    assert cdll.radon_profile_read(None, None, None) == 1
    assert cdll.radon_plan_get_info(None, None) == 1
    assert cdll.radon_status_string(1) == b"invalid argument"
