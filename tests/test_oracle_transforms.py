"""Pins of the oracle's transforms against closed forms (Sections 1, 2 and 7).

The log-polar oracle (Algorithms 1 and 2) and the direct oracle are each
checked against analytic Radon transforms and back-projections; a few
deliberately planted mistakes in the oracle must make those pins fail.
"""

import math

import numpy as np
import pytest

from oracle import bspline, direct, geometry, kernels, logpolar
from workloads import ellipse_image, gaussian_image, random_ellipses

BLOBS = [(0.2, -0.1, 0.12, 1.0), (-0.3, 0.25, 0.08, -0.7), (0.05, 0.5, 0.1, 0.4)]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _analytic_gauss_sino(geo, blobs=BLOBS):
    th = np.arange(geo.n_angles) * geo.dtheta
    s = (np.arange(geo.n_det) - geo.n_det / 2) * geo.ds
    ref = direct.gaussian_radon(th[:, None], s[None, :], blobs)
    ref[:, ~geometry.live_bins(geo.n_det)] = 0.0
    return ref


def _gauss_bp_image(geo, blobs=BLOBS):
    N = geo.N
    x = (np.arange(N) - N / 2) * (2.0 / N)
    out = np.zeros((N, N))
    for cx, cy, sg, w in blobs:
        r = np.hypot(x[None, :] - cx, x[:, None] - cy)
        out += w * math.sqrt(2 * math.pi) * sg * direct.gaussian_bp(r, sg)
    return np.where(geometry.disc_mask(N), out, 0.0)


# ---------------------------------------------------------------- direct oracle

def test_direct_radon_of_one_basis_function():
    """Image samples B(i - l) B(j - k) have Q-coefficients delta_{lk}; at theta = 0 the
    line integral is (2/N) B(col - k) (the t-integral of B is 1 pixel = 2/N), at general
    theta it equals a brute-force Riemann sum of the closed-form basis function."""
    N = 32
    geo = geometry.make_geometry(N, 16, 40, 3)
    l, k = 15, 18
    i = np.arange(N)
    f = bspline.B(i[:, None] - l) * bspline.B(i[None, :] - k)
    R = direct.radon_direct(f, geo)
    s = (np.arange(geo.n_det) - geo.n_det / 2) * geo.ds
    live = geometry.live_bins(geo.n_det)
    expect0 = np.where(live, (2.0 / N) * bspline.B(s * N / 2 + N / 2 - k), 0.0)
    assert np.max(np.abs(R[0] - expect0)) < 1e-14
    a = 5
    th = a * geo.dtheta
    t = np.linspace(-1.5, 1.5, 600001)
    dt = t[1] - t[0]
    for kk in (10, 20, 25):
        x1 = s[kk] * math.cos(th) - t * math.sin(th)
        x2 = s[kk] * math.sin(th) + t * math.cos(th)
        ref = np.sum(bspline.B(x2 * N / 2 + N / 2 - l) * bspline.B(x1 * N / 2 + N / 2 - k)) * dt
        assert R[a, kk] == pytest.approx(ref, abs=1e-9)


def test_direct_radon_obeys_the_fourier_slice_theorem():
    """For the spline f~(x) = sum_ij c_ij B((x1 - x_j)/h) B((x2 - x_i)/h), h = 2/N, the 2-D Fourier
    transform is h^2 sinc^4(h xi1) sinc^4(h xi2) sum_ij c_ij exp(-2 pi i (xi1 x_j + xi2 x_i)), and
    int R f(theta, s) exp(-2 pi i sigma s) ds equals it at xi = sigma (cos theta, sin theta)
    (Fourier slice theorem).  The s integral is the sum over the detector grid: f~ is compactly
    supported, and the sum is accurate to ~2e-7 of F(0) at theta = 0 (where R f(0, .) is itself a
    spline with knots every pixel, whose aliased spectrum the sum picks up) and ~1e-10 elsewhere;
    a transposed or sign-flipped convention misses by more than 0.5.  Pins orientation, sign,
    scale and the interpolant model of the direct oracle, independently of its prefilter."""
    N = 32
    h = 2.0 / N
    geo = geometry.make_geometry(N, 12, 192, 3)
    x = (np.arange(N) - N / 2) * h
    X1, X2 = np.meshgrid(x, x)  # X1[i, j] = x_j (column), X2[i, j] = x_i (row)
    r2 = (X1 - 0.1) ** 2 + (X2 + 0.05) ** 2
    c = np.where(np.hypot(X1, X2) < 0.75, np.exp(-r2 / (2 * 0.12 ** 2)), 0.0)
    # image samples of the spline: [1, 4, 1] / 6 along both axes (zero outside the array)
    k3 = np.array([1.0, 4.0, 1.0]) / 6.0
    f = np.apply_along_axis(lambda v: np.convolve(v, k3, mode="same"), 0, c)
    f = np.apply_along_axis(lambda v: np.convolve(v, k3, mode="same"), 1, f)
    R = direct.radon_direct(f, geo)
    s = (np.arange(geo.n_det) - geo.n_det / 2) * geo.ds
    F0 = h * h * c.sum()
    for a in (0, 3, 7, 10):
        th = a * geo.dtheta
        for sigma in (0.7, 2.3, 5.1):
            num = geo.ds * np.sum(R[a] * np.exp(-2j * np.pi * sigma * s))
            xi1, xi2 = sigma * math.cos(th), sigma * math.sin(th)
            F = h * h * np.sinc(h * xi1) ** 4 * np.sinc(h * xi2) ** 4 * np.sum(
                c * np.exp(-2j * np.pi * (xi1 * X1 + xi2 * X2)))
            assert abs(num - F) < 1e-6 * abs(F0), (a, sigma, num, F)


def test_direct_radon_converges_to_analytic_gaussian():
    errs = []
    for N in (32, 64):
        geo = geometry.make_geometry(N, 24, 3 * N // 2, 3)
        f = gaussian_image(N, BLOBS)
        errs.append(_rel(direct.radon_direct(f, geo), _analytic_gauss_sino(geo)))
    assert errs[1] < 5e-5
    assert math.log2(errs[0] / errs[1]) > 3.5  # O(h^4)


def test_direct_radon_ellipses_close_to_analytic():
    N = 64
    geo = geometry.make_geometry(N, 32, 96, 3)
    ell = random_ellipses(10, 1)
    th = np.arange(geo.n_angles) * geo.dtheta
    s = (np.arange(geo.n_det) - geo.n_det / 2) * geo.ds
    ref = direct.ellipse_radon(th[:, None], s[None, :], ell)
    assert _rel(direct.radon_direct(ellipse_image(N, ell), geo), ref) < 0.1


def test_direct_backprojection_of_s_gaussian():
    errs = []
    for N in (32, 64):
        geo = geometry.make_geometry(N, N, 3 * N // 2, 3)
        g = _analytic_gauss_sino(geo)
        errs.append(_rel(direct.backproject_direct(g, geo), _gauss_bp_image(geo)))
    assert errs[1] < 1e-4
    assert errs[0] > errs[1]


# ---------------------------------------------------------------- log-polar oracle

@pytest.mark.parametrize("M", [3, 4])
def test_logpolar_forward_converges_to_analytic_gaussian(M):
    errs = []
    for N in (64, 128):
        geo = geometry.make_geometry(N, N, 3 * N // 2, M)
        errs.append(_rel(logpolar.forward(gaussian_image(N, BLOBS), geo), _analytic_gauss_sino(geo)))
    assert errs[1] < 3e-5
    assert math.log2(errs[0] / errs[1]) > 3.0


def test_logpolar_forward_linear_interpolation_second_order():
    errs = []
    for N in (64, 128):
        geo = geometry.make_geometry(N, N, 3 * N // 2, 3, interp=1)
        errs.append(_rel(logpolar.forward(gaussian_image(N, BLOBS), geo), _analytic_gauss_sino(geo)))
    assert errs[1] < 2e-2
    assert math.log2(errs[0] / errs[1]) > 1.5


@pytest.mark.parametrize("M", [3, 5])
def test_logpolar_backprojection_of_gaussian_sinogram(M):
    """R# of the analytic sinogram of Gaussians equals sum_k w sqrt(2 pi) s pi e^{-u} I_0(u)."""
    errs = []
    for N in (64, 128):
        geo = geometry.make_geometry(N, N, 3 * N // 2, M)
        errs.append(_rel(logpolar.backproject(_analytic_gauss_sino(geo), geo), _gauss_bp_image(geo)))
    assert errs[1] < 2e-5
    assert math.log2(errs[0] / errs[1]) > 3.0


@pytest.mark.parametrize("M", [3, 5])
def test_logpolar_backprojection_linear_variant_second_order(M):
    """Linear variant of Algorithm 2 (raw samples, bilinear weights, multiplier zeta#-hat without
    B-hat) on the analytic sinogram of Gaussians: R# converges to sum_k w sqrt(2 pi) s pi e^{-u}
    I_0(u) at second order, the order of linear interpolation."""
    errs = []
    for N in (64, 128):
        geo = geometry.make_geometry(N, N, 3 * N // 2, M, interp=1)
        errs.append(_rel(logpolar.backproject(_analytic_gauss_sino(geo), geo), _gauss_bp_image(geo)))
    assert errs[1] < 3e-3
    assert math.log2(errs[0] / errs[1]) > 1.8


ISOLATED = [[(0.0, 0.0, 0.2, 1.0)], [(0.2, -0.1, 0.15, 1.0)], [(-0.3, 0.3, 0.1, 1.0)]]


@pytest.mark.parametrize("blobs", ISOLATED)
def test_logpolar_backprojection_linear_variant_lowers_smooth_maxima(blobs):
    """Every resampling of the linear variant uses nonnegative weights that reproduce affine
    functions, so by Jensen's inequality it never exceeds a locally concave function; the
    convolution integrates along the curves rho = log cos theta with a positive weight.  At the
    maximum of an isolated Gaussian's back-projection the result therefore falls short of the
    closed form, by an amount that shrinks like h^2.  A sharpening step (such as dividing the
    linear multiplier by B-hat, which belongs to the cubic variant) overshoots instead."""
    defs = []
    for N in (64, 128):
        geo = geometry.make_geometry(N, N, 3 * N // 2, 3, interp=1)
        ref = _gauss_bp_image(geo, blobs)
        got = logpolar.backproject(_analytic_gauss_sino(geo, blobs), geo)
        i = np.unravel_index(np.argmax(ref), ref.shape)
        defs.append((got[i] - ref[i]) / ref[i])
    assert defs[0] < 0 and defs[1] < 0, defs
    assert 3.0 < defs[0] / defs[1] < 5.5, defs


@pytest.mark.parametrize("mistake", ["conj_kernel", "s_tap_shift", "theta_tap_shift", "bhat_in_linear"])
def test_planted_mistakes_fail_the_linear_backprojection_pins(monkeypatch, mistake):
    """Each planted mistake in the linear R# must break one of the two pins above: the error
    against the closed form grows by at least 5x, or the peak deficit changes sign."""
    N = 128
    geo = geometry.make_geometry(N, N, 3 * N // 2, 3, interp=1)
    g, ref = _analytic_gauss_sino(geo), _gauss_bp_image(geo)
    base = _rel(logpolar.backproject(g, geo), ref)
    orig_interp = bspline.interp2d

    def shifted(axis):
        def f(c, t0, t1, order=3, mode0="zero", mode1="zero"):
            if mode0 == "periodic" and mode1 == "zero":    # the sinogram gather of Algorithm 2
                t0, t1 = (t0 + 1, t1) if axis == 0 else (t0, t1 + 1)
            return orig_interp(c, t0, t1, order, mode0, mode1)
        return f

    if mistake == "conj_kernel":
        orig = kernels.kernel_quadrant
        monkeypatch.setattr(kernels, "kernel_quadrant", lambda gg, w, **kw: np.conj(orig(gg, w, **kw)))
    elif mistake == "s_tap_shift":
        monkeypatch.setattr(bspline, "interp2d", shifted(1))
    elif mistake == "theta_tap_shift":
        monkeypatch.setattr(bspline, "interp2d", shifted(0))
    elif mistake == "bhat_in_linear":
        orig_mult = kernels.multiplier
        monkeypatch.setattr(kernels, "multiplier", lambda gg, w: orig_mult(gg, w) / kernels.bhat2d(
            gg.n_theta, gg.N_rho))
    bad = _rel(logpolar.backproject(g, geo), ref)
    blobs = ISOLATED[0]
    gi, ri = _analytic_gauss_sino(geo, blobs), _gauss_bp_image(geo, blobs)
    i = np.unravel_index(np.argmax(ri), ri.shape)
    deficit = logpolar.backproject(gi, geo)[i] - ri[i]
    assert bad > 5 * base or deficit > 0, (bad, base, deficit)


def test_logpolar_forward_conserves_mass_and_centre_per_angle():
    """Fourier slice theorem at sigma = 0 and its first moment: int R f ds = int f and
    int s R f ds = theta . int x f, for every angle."""
    N = 128
    geo = geometry.make_geometry(N, N, 3 * N // 2, 3)
    f = gaussian_image(N, BLOBS)
    Rf = logpolar.forward(f, geo)
    s = (np.arange(geo.n_det) - geo.n_det / 2) * geo.ds
    mass = sum(w * 2 * math.pi * sg * sg for _, _, sg, w in BLOBS)
    mx = sum(w * 2 * math.pi * sg * sg * cx for cx, _, sg, w in BLOBS)
    my = sum(w * 2 * math.pi * sg * sg * cy for _, cy, sg, w in BLOBS)
    th = np.arange(geo.n_angles) * geo.dtheta
    assert np.max(np.abs(Rf.sum(axis=1) * geo.ds - mass)) < 2e-5
    assert np.max(np.abs((Rf * s).sum(axis=1) * geo.ds - (mx * np.cos(th) + my * np.sin(th)))) < 2e-5


def test_logpolar_agrees_with_direct_oracle_on_ellipse_phantom():
    """Config-1-style phantom at reduced size (the direct oracle is slow)."""
    N = 64
    geo = geometry.make_geometry(N, N, 96, 3)
    f = ellipse_image(N, random_ellipses(10, 1))
    sub = np.arange(0, geo.n_angles, 4)
    Rlp = logpolar.forward(f, geo)[sub]
    Rd = direct.radon_direct(f, geo, angle_idx=sub)
    assert _rel(Rlp, Rd) < 0.05


# ---------------------------------------------------------------- planted mistakes

def _forward_err(geo, monkeypatch=None):
    return _rel(logpolar.forward(gaussian_image(geo.N, BLOBS), geo), _analytic_gauss_sino(geo))


@pytest.mark.parametrize("mistake", ["conj_kernel", "no_bhat", "no_box_comp", "no_inv_aR", "kr_shift"])
def test_planted_mistakes_fail_the_forward_pin(monkeypatch, mistake):
    N = 128
    geo = geometry.make_geometry(N, N, 3 * N // 2, 3)
    base = _forward_err(geo)
    if mistake == "conj_kernel":
        orig = kernels.kernel_quadrant
        monkeypatch.setattr(kernels, "kernel_quadrant", lambda g, w, **kw: np.conj(orig(g, w, **kw)))
    elif mistake == "no_bhat":
        monkeypatch.setattr(kernels, "bhat2d", lambda a, b: np.ones((a, b)))
    elif mistake == "no_box_comp":
        monkeypatch.setattr(kernels, "box_response", lambda n, r: np.ones(n))
    elif mistake == "no_inv_aR":
        import dataclasses
        geo2 = dataclasses.replace(geo)
        orig_fwd = logpolar.forward
        monkeypatch.setattr(logpolar, "forward", lambda f, g, **kw: orig_fwd(f, g, **kw) * g.a_R)
        geo = geo2
    elif mistake == "kr_shift":
        orig = kernels.full_grid
        monkeypatch.setattr(kernels, "full_grid", lambda q, a, b: np.roll(orig(q, a, b), 1, axis=1))
    bad = _forward_err(geo)
    assert bad > 20 * base


# ---------------------------------------------------------------- symmetries and special cases

def test_logpolar_forward_of_the_constant_disc_is_the_chord_length():
    """f = 1 on the pixels inside the unit disc: R f(theta, s) -> 2 sqrt(1 - s^2) for every
    theta (Section 1), at first order in the pixel size (the disc's edge is a jump)."""
    errs = []
    for N in (64, 128):
        geo = geometry.make_geometry(N, N, 3 * N // 2, 3)
        Rf = logpolar.forward(np.ones((N, N)), geo)
        s = (np.arange(geo.n_det) - geo.n_det / 2) * geo.ds
        chord = np.where(np.abs(s) < 1, 2 * np.sqrt(np.clip(1 - s * s, 0, None)), 0.0)
        errs.append(_rel(Rf, np.broadcast_to(chord, Rf.shape)))
    assert errs[1] < 1e-2
    assert math.log2(errs[0] / errs[1]) > 0.8


def test_logpolar_forward_mirror_symmetry():
    """f(-x1, x2) has R f(pi - theta, s): angle a -> n_angles - a, and angle 0 -> angle 0 with
    s -> -s (bin k -> n_det - k); pixel column j -> N - j.  The partitions' half-open angle ranges
    are not mirror images, so the identity holds to the method's error, which falls like h^4; a
    sign or half-bin slip in theta, s or T_m would break it at O(1)."""
    errs = []
    for N in (64, 128):
        geo = geometry.make_geometry(N, N, 3 * N // 2, 3)
        f = gaussian_image(N, BLOBS)
        fm = np.zeros_like(f)
        fm[:, 1:] = f[:, :0:-1]
        R = logpolar.forward(f, geo)
        expect = np.zeros_like(R)
        expect[1:] = R[:0:-1]
        expect[0, 1:] = R[0, :0:-1]
        errs.append(_rel(logpolar.forward(fm, geo), expect))
    assert errs[1] < 2e-5
    assert math.log2(errs[0] / errs[1]) > 3.0


def test_logpolar_transforms_are_linear():
    N = 48
    geo = geometry.make_geometry(N, 40, 72, 3)
    rng = np.random.default_rng(12)
    f1, f2 = rng.standard_normal((2, N, N))
    g1, g2 = rng.standard_normal((2, 40, 72))
    a, b = 0.7, -1.9
    R = logpolar.forward
    assert _rel(R(a * f1 + b * f2, geo), a * R(f1, geo) + b * R(f2, geo)) < 1e-13
    B = logpolar.backproject
    assert _rel(B(a * g1 + b * g2, geo), a * B(g1, geo) + b * B(g2, geo)) < 1e-13
