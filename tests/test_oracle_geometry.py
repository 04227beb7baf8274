"""Pins of the oracle's discretisation rules (Sections 2 and 4)."""

import math

import numpy as np
import pytest

from oracle import direct, geometry


def test_partition_constants_M3():
    """Eq. aconst with beta = pi/3: a_R = sin(pi/6)/(1 + sin(pi/6)) = 1/3,
    a_r = (cos(pi/6) - sin(pi/6))/(1 + sin(pi/6)) = 0.2440169..."""
    beta, a_R, a_r = geometry.partition_constants(3)
    assert beta == pytest.approx(math.pi / 3, abs=1e-16)
    assert a_R == pytest.approx(1.0 / 3.0, abs=1e-15)
    assert a_r == pytest.approx((math.sqrt(3.0) - 1.0) / 3.0, abs=1e-15)
    assert round(a_r, 7) == 0.2440169


@pytest.mark.parametrize("M", [3, 4, 5, 8])
def test_partition_geometry_of_the_disc_D(M):
    """Figure spans (a): the disc D of radius a_R centred at (1 - a_R, 0) touches the unit
    circle, subtends the half-angle beta/2, and its tangent line at normal angle beta/2 lies
    at distance a_r; the kernel's support curve rho = log cos(theta) stays inside
    [log a_r, 0] for |theta| <= beta."""
    beta, a_R, a_r = geometry.partition_constants(M)
    assert (1 - a_R) + a_R == pytest.approx(1.0)
    assert a_R / (1 - a_R) == pytest.approx(math.sin(beta / 2), rel=1e-14)
    assert (1 - a_R) * math.cos(beta / 2) - a_R == pytest.approx(a_r, rel=1e-14)
    assert 1 - 2 * a_R > a_r
    assert math.cos(beta) > a_r


def test_nrho_close_to_paper_estimate():
    """Section 6: for M = 3, N_rho ~ -N log(a_r) / (2 a_R) ~ 2.1 N."""
    for N in (512, 2048, 8192):
        g = geometry.make_geometry(N, N, 3 * N // 2, 3)
        assert 2.1 < g.N_rho / N < 2.2
        assert g.N_rho >= math.ceil(math.log(g.a_r) / math.log(1 - 2 * g.a_R / N))
        assert geometry.is_7smooth(g.N_rho) and g.N_rho % 2 == 0


def test_config_sizes():
    g1 = geometry.make_geometry(128, 128, 192, 3)
    assert (g1.N_rho, g1.n_th_h, g1.n_theta, g1.r) == (280, 48, 96, 5)
    g2 = geometry.make_geometry(2048, 2048, 3072, 3)
    assert (g2.N_rho, g2.n_th_h, g2.n_theta, g2.r) == (4374, 686, 1372, 5)
    # fine angular step of Omega_lp is at most the pixel size 2 a_R / N of T_m f (Section 4)
    for g in (g1, g2):
        assert g.dphi / g.r <= 2 * g.a_R / g.N + 1e-15


def test_every_angle_has_one_partition_within_half_beta():
    for na, M in ((128, 3), (2048, 3), (100, 4), (37, 5)):
        for a in range(na):
            m, num, flip = geometry.angle_partition(a, na, M)
            assert 0 <= m < M
            phi = num * math.pi / (M * na)
            assert abs(phi) <= math.pi / (2 * M) + 1e-15
            theta = a * math.pi / na
            expect = theta - math.pi if flip else theta - m * math.pi / M
            assert phi == pytest.approx(expect, abs=1e-13)


def test_T_m_maps_unit_disc_into_D_and_Radon_tm_identity():
    """Eq. Tdef and Eq. Radon_tm, checked on a Gaussian: T_m f is again a Gaussian
    (centre T_m c, width a_R sigma), and both sides use the analytic Radon transform."""
    M = 3
    beta, a_R, a_r = geometry.partition_constants(M)
    rng = np.random.default_rng(0)
    for m in range(M):
        rot = np.array([[math.cos(m * beta), math.sin(m * beta)], [-math.sin(m * beta), math.cos(m * beta)]])

        def T(x):
            return a_R * rot @ x + np.array([1 - a_R, 0.0]).reshape((2,) + (1,) * (x.ndim - 1))

        pts = rng.uniform(-1, 1, size=(2, 500))
        pts = pts[:, np.hypot(*pts) < 1]
        y = T(pts)
        assert np.all(np.hypot(y[0] - (1 - a_R), y[1]) < a_R + 1e-14)
        c = np.array([0.3, -0.2])
        sg = 0.1
        cT = T(c)
        theta = rng.uniform(0, math.pi, 50)
        s = rng.uniform(-1, 1, 50)
        lhs = direct.gaussian_radon(theta, s, [(c[0], c[1], sg, 1.0)])
        phi = theta - m * beta
        rhs = direct.gaussian_radon(phi, a_R * s + (1 - a_R) * np.cos(phi), [(cT[0], cT[1], a_R * sg, 1.0)]) / a_R
        assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_masks_are_exact_integer_tests():
    m = geometry.disc_mask(8)
    assert m[4, 0] == False  # noqa: E712  x = (-1, 0): |x| = 1 is outside
    assert m[4, 1] == True  # noqa: E712
    live = geometry.live_bins(192)
    s = (np.arange(192) - 96) * (2 * math.sqrt(2) / 192)
    assert np.array_equal(live, np.abs(s) < 1)
