"""Pins of the oracle's exact transpose of Algorithm 1.

The transpose is defined by the identity sum(A x * y) = sum(x * A^T y) for all x and y; each
piece (the spreading that transposes interpolation, the transposed log-polar convolution,
the whole map) is checked against it on random inputs, and planted mistakes must break it.
Independently of the identity, the transpose of the discrete R approaches the continuous
adjoint R# (Section 2) scaled by dx^2 / (dtheta ds) on smooth sinograms, which pins its scale
against the closed-form back-projection of Gaussians.
"""

import math

import numpy as np
import pytest

from oracle import bspline, geometry, kernels, logpolar

from test_oracle_transforms import _analytic_gauss_sino, _gauss_bp_image, _rel


def _rel_gap(a, b):
    return abs(a - b) / max(abs(a), abs(b))


@pytest.mark.parametrize("order", [1, 3])
@pytest.mark.parametrize("modes", [("zero", "zero"), ("zero", "periodic"), ("periodic", "zero")])
def test_spread2d_is_the_transpose_of_interp2d(order, modes):
    rng = np.random.default_rng(11)
    shape = (13, 17)
    c = rng.standard_normal(shape)
    # points inside, on the border and beyond it, so dropped and wrapped taps are exercised
    t0 = rng.uniform(-3.0, shape[0] + 2.0, size=(7, 9))
    t1 = rng.uniform(-3.0, shape[1] + 2.0, size=(7, 9))
    v = rng.standard_normal(t0.shape)
    lhs = np.sum(bspline.interp2d(c, t0, t1, order=order, mode0=modes[0], mode1=modes[1]) * v)
    rhs = np.sum(c * bspline.spread2d(v, t0, t1, shape, order=order, mode0=modes[0], mode1=modes[1]))
    assert _rel_gap(lhs, rhs) < 1e-13


def test_spread2d_of_one_point_is_the_tap_weights():
    """A unit value at (2.25, 5.5) lands on rows 1..4 and columns 4..7 with weights
    B(alpha + 1), B(alpha), B(alpha - 1), B(alpha - 2) per axis (Eq. wsumn)."""
    out = bspline.spread2d(np.array([1.0]), np.array([2.25]), np.array([5.5]), (8, 10))
    wr = bspline.B(np.array([1.25, 0.25, -0.75, -1.75]))
    wc = bspline.B(np.array([1.5, 0.5, -0.5, -1.5]))
    expect = np.zeros((8, 10))
    expect[1:5, 4:8] = np.outer(wr, wc)
    assert np.max(np.abs(out - expect)) < 1e-15
    assert abs(out.sum() - 1.0) < 1e-14  # partition of unity


def test_convolution_transpose_identity():
    N = 48
    geo = geometry.make_geometry(N, 36, 72, 3)
    rng = np.random.default_rng(5)
    K = kernels.multiplier(geo, "R")
    h = rng.standard_normal((geo.n_th_h, geo.N_rho))
    yb = rng.standard_normal((geo.n_th_h + logpolar.HALO_LO + logpolar.HALO_HI, geo.N_rho))
    lhs = np.sum(logpolar.logpolar_convolution(h, K, geo) * yb)
    rhs = np.sum(h * logpolar.logpolar_convolution_transpose(yb, K, geo))
    assert _rel_gap(lhs, rhs) < 1e-12


@pytest.mark.parametrize("N,na,nd,M,interp", [(32, 24, 48, 3, 3), (32, 24, 48, 4, 3), (40, 30, 61, 3, 3),
                                               (32, 24, 48, 3, 1), (36, 40, 50, 5, 1)])
def test_transpose_dot_product_identity(N, na, nd, M, interp):
    geo = geometry.make_geometry(N, na, nd, M, interp=interp)
    rng = np.random.default_rng(N + na + nd + M + interp)
    f = rng.standard_normal((N, N))
    g = rng.standard_normal((na, nd))
    lhs = np.sum(logpolar.forward(f, geo) * g)
    rhs = np.sum(f * logpolar.transpose(g, geo))
    assert _rel_gap(lhs, rhs) < 1e-12


def test_transpose_is_zero_outside_the_disc_and_ignores_dead_bins():
    N = 32
    geo = geometry.make_geometry(N, 24, 48, 3)
    rng = np.random.default_rng(9)
    g = rng.standard_normal((geo.n_angles, geo.n_det))
    Rt = logpolar.transpose(g, geo)
    assert np.all(Rt[~geometry.disc_mask(N)] == 0.0)
    g2 = g.copy()
    g2[:, ~geometry.live_bins(geo.n_det)] = 123.0
    assert np.array_equal(logpolar.transpose(g2, geo), Rt)


def test_transpose_scale_matches_the_continuous_adjoint():
    """R^T g ~ dx^2 / (dtheta ds) R# g on the analytic sinogram of Gaussians (the sums of
    <R f, g> approximate the integrals of the adjoint relation).  The transpose carries the
    pixel-scale ripple of spreading from the log-polar samples, so it converges slowly; a
    wrong factor (a_R, r, e^rho, the Jacobian) would be off by O(1)."""
    errs = []
    for N in (64, 128):
        geo = geometry.make_geometry(N, N, 3 * N // 2, 3)
        c = (2.0 / N) ** 2 / (geo.dtheta * geo.ds)
        errs.append(_rel(logpolar.transpose(_analytic_gauss_sino(geo), geo) / c, _gauss_bp_image(geo)))
    assert errs[1] < 0.03
    assert errs[1] < 0.7 * errs[0]


@pytest.mark.parametrize("mistake", ["conj_kernel", "no_q_transpose", "no_erho", "no_inv_aR"])
def test_planted_mistakes_break_the_identity(monkeypatch, mistake):
    N = 32
    geo = geometry.make_geometry(N, 24, 48, 3)
    rng = np.random.default_rng(3)
    f = rng.standard_normal((N, N))
    g = rng.standard_normal((geo.n_angles, geo.n_det))
    lhs = np.sum(logpolar.forward(f, geo) * g)
    if mistake == "conj_kernel":
        orig = logpolar.logpolar_convolution_transpose
        monkeypatch.setattr(logpolar, "logpolar_convolution_transpose",
                            lambda yb, K, g_, d=None: orig(yb, np.conj(K), g_, d))
    elif mistake == "no_q_transpose":
        orig_pf = bspline.prefilter_zero
        monkeypatch.setattr(bspline, "prefilter_zero",
                            lambda x, axis=0: np.eye(x.shape[0]) if x.ndim == 2 and np.array_equal(x, np.eye(x.shape[0]))
                            else orig_pf(x, axis=axis))
    elif mistake == "no_erho":
        monkeypatch.setattr(type(geo), "rho", lambda self, i: np.zeros(np.shape(i)))  # e^rho -> 1
    elif mistake == "no_inv_aR":
        import dataclasses
        geo = dataclasses.replace(geo)
        orig_sp = bspline.spread2d
        monkeypatch.setattr(bspline, "spread2d",
                            lambda v, t0, t1, shape, **kw: orig_sp(v, t0, t1, shape, **kw)
                            * (geo.a_R if kw.get("mode1") == "periodic" else 1.0))
    rhs = np.sum(f * logpolar.transpose(g, geo))
    assert _rel_gap(lhs, rhs) > 1e-3
