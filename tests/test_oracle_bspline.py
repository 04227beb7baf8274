"""Pins of the oracle's B-spline pieces (Section 5) against definitions and printed values."""

import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import bspline

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_B_integer_samples_match_paper():
    """Eq. Bcoeff prints B(0) = 2/3, B(+-1) = 1/6, 0 elsewhere."""
    for j, frac in _golden_rows("bspline_integer_samples.txt"):
        assert bspline.B(float(j)) == pytest.approx(float(Fraction(frac)), abs=1e-15)


def test_B_partition_of_unity_and_c2():
    x = np.linspace(-0.5, 0.5, 101)
    total = sum(bspline.B(x - k) for k in range(-3, 4))
    assert np.max(np.abs(total - 1.0)) < 1e-14
    # C^2 at the knots: one-sided second differences agree
    h = 1e-4
    for k in (0.0, 1.0, 2.0):
        left = (bspline.B(k - 2 * h) - 2 * bspline.B(k - h) + bspline.B(k)) / h**2
        right = (bspline.B(k) - 2 * bspline.B(k + h) + bspline.B(k + 2 * h)) / h**2
        assert abs(left - right) < 2e-3


def test_Bhat_is_the_series_of_integer_samples():
    """Eq. Bhat: sum_j B(j) exp(-2 pi i j xi) = 2/3 + cos(2 pi xi) / 3."""
    xi = np.linspace(-0.5, 0.5, 41)
    series = sum(bspline.B(float(j)) * np.exp(-2j * np.pi * j * xi) for j in range(-3, 4))
    assert np.max(np.abs(series - bspline.Bhat(xi))) < 1e-15


def _banded(n, periodic):
    A = np.zeros((n, n))
    for k in range(n):
        A[k, k] = 4.0 / 6.0
        for d in (-1, 1):
            j = k + d
            if periodic:
                A[k, j % n] += 1.0 / 6.0
            elif 0 <= j < n:
                A[k, j] = 1.0 / 6.0
    return A


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 17, 64])
def test_prefilter_zero_solves_interpolation_condition(n):
    """Q f is the coefficient sequence (zero outside [0, n)) whose spline reproduces
    every sample (Eq. Bsplineinterp); checked against a dense solve of that system."""
    rng = np.random.default_rng(n)
    f = rng.standard_normal((n, 3))
    c = bspline.prefilter_zero(f, axis=0)
    ref = np.linalg.solve(_banded(n, periodic=False), f)
    assert np.max(np.abs(c - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [3, 4, 7, 16, 50])
def test_prefilter_periodic_solves_circulant_system(n):
    rng = np.random.default_rng(100 + n)
    f = rng.standard_normal((4, n))
    c = bspline.prefilter_periodic(f, axis=1)
    ref = np.linalg.solve(_banded(n, periodic=True), f.T).T
    assert np.max(np.abs(c - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_interpolant_reproduces_samples_2d():
    rng = np.random.default_rng(7)
    f = rng.standard_normal((9, 12))
    c = bspline.prefilter_zero(bspline.prefilter_zero(f, axis=0), axis=1)
    I, J = np.meshgrid(np.arange(9.0), np.arange(12.0), indexing="ij")
    assert np.max(np.abs(bspline.interp2d(c, I, J) - f)) < 1e-12
    assert np.max(np.abs(bspline.interp2d(f, I, J, order=1) - f)) < 1e-15


def test_interpolant_vanishes_beyond_array():
    c = np.ones((6, 6))
    assert bspline.interp2d(c, np.array([-2.0, 8.0]), np.array([3.0, 3.0])).tolist() == [0.0, 0.0]


@pytest.mark.parametrize("order,rate", [(3, 4.0), (1, 2.0)])
def test_interpolation_convergence_order(order, rate):
    """Cubic spline interpolation is O(h^4), linear O(h^2), on a smooth periodic function."""
    errs = []
    for n in (32, 64, 128):
        k = np.arange(n)
        fk = np.sin(2 * np.pi * k / n) + 0.3 * np.cos(6 * np.pi * k / n)
        c = bspline.prefilter_periodic(fk) if order == 3 else fk
        t = np.linspace(0, n, 997, endpoint=False) + 0.37
        v = bspline.interp1d(c, t, order=order, mode="periodic")
        ref = np.sin(2 * np.pi * t / n) + 0.3 * np.cos(6 * np.pi * t / n)
        errs.append(np.max(np.abs(v - ref)))
    for e0, e1 in zip(errs, errs[1:]):
        assert math.log2(e0 / e1) > rate - 0.3
