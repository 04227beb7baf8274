"""Direct (non-log-polar) Radon transform and back-projection, and analytic references. FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``radon_direct``: R f(theta, s) = int f~(s theta + t theta_perp) dt (Eq. radon_def)
  for the interpolant f~ of the image (cubic spline of Q f, or bilinear),
  integrated exactly: between consecutive crossings of the line with the
  pixel grid lines f~ is a polynomial of degree <= 6 in t, so a 4-point
  Gauss-Legendre rule on each piece is exact.
* ``backproject_direct``: R# g(x) = int_0^pi g(theta, x . theta) dtheta
  (Section 1) by the rectangle rule over the measured angles, with g
  interpolated along s (cubic spline of Q g or linear).
* ``ellipse_radon``, ``gaussian_radon``, ``gaussian_bp``: closed forms used as
  pins (Section 7 uses the analytic Radon transform of ellipse indicators).
"""

from __future__ import annotations

import math

import numpy as np
from scipy import special

from . import bspline
from .geometry import live_bins
from .logpolar import image_coefficients


def _line_points(geo, theta, s_vals):
    """Gauss-Legendre nodes (in pixel-index coordinates) and weights along lines
    (theta, s) for s in s_vals; exact piecewise integration over the padded image."""
    N = geo.N
    half = N / 2
    c, sn = math.cos(theta), math.sin(theta)
    # pixel coordinates along the line: col = X0 + t dX, row = Y0 + t dY
    X0 = s_vals * c * half + half
    Y0 = s_vals * sn * half + half
    dX = -sn * half
    dY = c * half
    ks = np.arange(-3, N + 3, dtype=np.float64)
    pieces = []
    if abs(dX) > 1e-14:
        pieces.append((ks[None, :] - X0[:, None]) / dX)
    if abs(dY) > 1e-14:
        pieces.append((ks[None, :] - Y0[:, None]) / dY)
    brk = np.sort(np.concatenate(pieces, axis=1), axis=1)
    # the interpolant vanishes beyond the padded square, i.e. outside the breakpoint range
    a = brk[:, :-1]
    b = brk[:, 1:]
    xg, wg = np.polynomial.legendre.leggauss(4)
    t = 0.5 * (b - a)[..., None] * xg + 0.5 * (a + b)[..., None]
    w = 0.5 * (b - a)[..., None] * wg
    col = X0[:, None, None] + t * dX
    row = Y0[:, None, None] + t * dY
    return row, col, w


def radon_direct(f: np.ndarray, geo, angle_idx=None, det_idx=None) -> np.ndarray:
    """Exact line integrals of the interpolant of the disc-masked image.

    Returns [len(angle_idx), len(det_idx)] (all angles / bins by default);
    bins with |s| >= 1 are set to zero as in the log-polar operator.
    """
    c = image_coefficients(f, geo)
    angle_idx = np.arange(geo.n_angles) if angle_idx is None else np.asarray(angle_idx)
    det_idx = np.arange(geo.n_det) if det_idx is None else np.asarray(det_idx)
    live = live_bins(geo.n_det)[det_idx]
    s_vals = (det_idx - geo.n_det / 2) * geo.ds
    out = np.zeros((angle_idx.size, det_idx.size))
    for n_a, a in enumerate(angle_idx):
        theta = a * geo.dtheta
        row, col, w = _line_points(geo, theta, s_vals[live])
        vals = bspline.interp2d(c, row, col, order=geo.interp)
        out[n_a, live] = np.sum(vals * w, axis=(1, 2))
    return out


def sinogram_row_coefficients(g: np.ndarray, geo) -> np.ndarray:
    """Per-row coefficients along s (cubic: zero-boundary Q on k in [0, n_det]; linear: samples)."""
    gm = np.where(live_bins(geo.n_det)[None, :], np.asarray(g, dtype=np.float64), 0.0)
    E = np.zeros((gm.shape[0], geo.n_det + 1))
    E[:, :geo.n_det] = gm
    if geo.interp == 3:
        E = bspline.prefilter_zero(E, axis=1)
    return E


def backproject_direct(g: np.ndarray, geo, pixels=None) -> np.ndarray:
    """dtheta * sum_a g~(theta_a, x . theta_a) for pixels inside the unit disc.

    ``pixels``: optional (rows, cols) index arrays; returns the full image otherwise.
    """
    from .geometry import disc_mask

    N = geo.N
    E = sinogram_row_coefficients(g, geo)
    if pixels is None:
        ii, jj = np.nonzero(disc_mask(N))
    else:
        ii, jj = (np.asarray(p) for p in pixels)
    x1 = (jj - N / 2) * (2.0 / N)
    x2 = (ii - N / 2) * (2.0 / N)
    acc = np.zeros(ii.shape)
    for a in range(geo.n_angles):
        th = a * geo.dtheta
        s = x1 * math.cos(th) + x2 * math.sin(th)
        acc += bspline.interp1d(E[a], s / geo.ds + geo.n_det / 2, order=geo.interp)
    acc *= geo.dtheta
    if pixels is not None:
        return acc
    img = np.zeros((N, N))
    img[ii, jj] = acc
    return img


def ellipse_radon(theta, s, ellipses) -> np.ndarray:
    """Analytic Radon transform of sum_e density_e * 1_ellipse_e (textbook formula:
    2 rho a b sqrt(A^2 - t^2) / A^2 with A^2 = a^2 cos^2(theta - psi) + b^2 sin^2(theta - psi),
    t = s - c . theta)."""
    theta = np.asarray(theta, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    out = np.zeros(np.broadcast(theta, s).shape)
    for e in ellipses:
        A2 = (e.a * np.cos(theta - e.psi)) ** 2 + (e.b * np.sin(theta - e.psi)) ** 2
        t = s - (e.cx * np.cos(theta) + e.cy * np.sin(theta))
        inside = t * t < A2
        out += np.where(inside, 2.0 * e.density * e.a * e.b * np.sqrt(np.maximum(A2 - t * t, 0.0)) / A2, 0.0)
    return out


def gaussian_radon(theta, s, blobs) -> np.ndarray:
    """Analytic Radon transform of sum_k w_k exp(-|x - c_k|^2 / (2 s_k^2)):
    w sqrt(2 pi) s exp(-(s - c . theta)^2 / (2 s^2))."""
    theta = np.asarray(theta, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    out = np.zeros(np.broadcast(theta, s).shape)
    for cx, cy, sg, w in blobs:
        t = s - (cx * np.cos(theta) + cy * np.sin(theta))
        out += w * math.sqrt(2.0 * math.pi) * sg * np.exp(-t * t / (2.0 * sg * sg))
    return out


def gaussian_bp(r, sigma) -> np.ndarray:
    """int_0^pi exp(-(x . theta)^2 / (2 sigma^2)) dtheta = pi exp(-u) I_0(u), u = |x|^2 / (4 sigma^2)."""
    u = np.asarray(r, dtype=np.float64) ** 2 / (4.0 * sigma * sigma)
    return math.pi * special.i0e(u)
