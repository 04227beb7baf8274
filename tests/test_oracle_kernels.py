"""Pins of the oracle's kernel coefficients (Section 3, Eq. exprcoef1 / exprcoef2)."""

import math

import numpy as np
import pytest

from oracle import geometry, kernels


@pytest.fixture(scope="module")
def geo():
    return geometry.make_geometry(64, 64, 96, 3)


def test_zero_frequency_closed_forms(geo):
    """zeta_hat[0,0] = int sec = 2 log(sec beta + tan beta) (= 2.633916 for M = 3);
    zeta#_hat[0,0] = 2 beta; zeta#_hat[kt != 0, 0] = 0 (a full period of exp)."""
    ZR = kernels.kernel_quadrant(geo, "R")
    ZB = kernels.kernel_quadrant(geo, "B")
    b = geo.beta
    assert ZR[0, 0] == pytest.approx(2 * math.log(1 / math.cos(b) + math.tan(b)), abs=1e-13)
    assert round(ZR[0, 0].real, 6) == 2.633916
    assert ZB[0, 0] == pytest.approx(2 * b, abs=1e-13)
    assert np.max(np.abs(ZB[1:, 0])) < 1e-13


def test_quadrant_matches_unfolded_integral_and_symmetries(geo):
    ZR = kernels.kernel_quadrant(geo, "R")
    ZB = kernels.kernel_quadrant(geo, "B")
    for kt, kr in ((0, 3), (5, 0), (7, 11), (geo.n_theta // 2, geo.N_rho // 2), (20, 60)):
        for which, Z in (("R", ZR), ("B", ZB)):
            v = Z[kt, kr]
            assert kernels.kernel_direct(geo, which, kt, kr) == pytest.approx(v, abs=1e-11)
            assert kernels.kernel_direct(geo, which, -kt, kr) == pytest.approx(v, abs=1e-11)
            assert kernels.kernel_direct(geo, which, kt, -kr) == pytest.approx(np.conj(v), abs=1e-11)


def test_quadrature_converged():
    g = geometry.make_geometry(256, 256, 384, 3)
    for which in ("R", "B"):
        a = kernels.kernel_quadrant(g, which, phase_per_panel=10.0)
        b = kernels.kernel_quadrant(g, which, phase_per_panel=4.0)
        assert np.max(np.abs(a - b)) < 1e-12


@pytest.mark.parametrize("kt,kr", [(0, 1), (3, 2), (10, 7), (1, 25)])
def test_closed_form_P(geo, kt, kr):
    """Eq. P_closed_form (Gamma and 3F2 terms) against the quadrature, kr != 0
    (the closed form is singular at kr = 0 for zeta: Gamma(0))."""
    pytest.importorskip("mpmath")
    ZR = kernels.kernel_quadrant(geo, "R")
    ZB = kernels.kernel_quadrant(geo, "B")
    nu = 2 * math.pi / geo.L
    mu = -math.pi * kt / geo.beta
    pr = kernels.P_closed_form(mu, complex(-1.0, -nu * kr), geo.beta)
    pb = kernels.P_closed_form(mu, complex(0.0, nu * kr), geo.beta)
    assert abs(pr - ZR[kt, kr]) < 1e-9 * max(1.0, abs(pr))
    assert abs(pb - ZB[kt, kr]) < 1e-9 * max(1.0, abs(pb))


def test_closed_form_P_reduces_to_interval_length():
    """P(0, 0, beta) = 2 beta (the Gamma and 3F2 terms combine to pi - (pi - 2 beta))."""
    pytest.importorskip("mpmath")
    assert kernels.P_closed_form(0.0, 0.0, 0.7) == pytest.approx(1.4, abs=1e-14)


def test_full_grid_is_hermitian_except_rho_nyquist(geo):
    K = kernels.full_grid(kernels.kernel_quadrant(geo, "R"), geo.n_theta, geo.N_rho)
    nt, nr = K.shape
    p, q = np.meshgrid(np.arange(nt), np.arange(nr), indexing="ij")
    partner = K[(-p) % nt, (-q) % nr]
    off = q != nr // 2
    assert np.max(np.abs(K[off] - np.conj(partner[off]))) < 1e-14


def test_box_response(geo):
    D = kernels.box_response(geo.n_theta, geo.r)
    # mean of r samples of exp(i w phi) at offsets (q - (r-1)/2) dphi / r, w = 2 pi kt / (n_theta dphi)
    for kt in (1, 7, geo.n_theta // 2 - 1):
        offs = (np.arange(geo.r) - (geo.r - 1) / 2) / geo.r
        direct = np.mean(np.exp(2j * np.pi * kt * offs / geo.n_theta))
        assert D[kt] == pytest.approx(direct.real, abs=1e-15)
        assert abs(direct.imag) < 1e-15
