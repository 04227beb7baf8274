"""Pins of the oracle's filtered back-projection (Eq. FBP, Eq. ramp, Eq. SLfilt, Eq. cosfilt)."""

import math

import numpy as np
import pytest

from oracle import direct, fbp, geometry
from workloads import gaussian_image

BLOBS = [(0.2, -0.1, 0.12, 1.0), (-0.3, 0.25, 0.08, -0.7), (0.05, 0.5, 0.1, 0.4)]


@pytest.mark.parametrize("nd", [96, 192, 500])
def test_ramp_transfer_is_abs_sigma_up_to_truncation(nd):
    """The band-limited ramp kernel is the sampled inverse transform of |sigma| on
    |sigma| <= 1/(2 ds); cut to |n| < P/2 its transfer function differs from |sigma| by at most
    the dropped tail, sum_{odd n > P/2} 2 / (pi^2 n^2 ds) < 2 / (pi^2 P ds)."""
    ds = 2 * math.sqrt(2) / nd
    P = fbp.filter_length(nd)
    H = fbp.transfer(P, ds, "ramp")
    k = np.arange(P)
    sigma = np.minimum(k, P - k) / (P * ds)
    assert np.max(np.abs(H - sigma)) <= 2.0 / (math.pi ** 2 * P * ds) * 1.01


def test_windows_vanish_or_shrink_at_the_band_edge():
    nd = 192
    ds = 2 * math.sqrt(2) / nd
    P = fbp.filter_length(nd)
    Hr = fbp.transfer(P, ds, "ramp")
    Hs = fbp.transfer(P, ds, "shepp-logan")
    Hc = fbp.transfer(P, ds, "cosine")
    nyq = P // 2
    assert abs(Hc[nyq]) < 1e-12 * abs(Hr[nyq])              # cos(pi/2) = 0 at sigma_max
    assert Hs[nyq] == pytest.approx(Hr[nyq] * 2 / math.pi, rel=1e-12)  # sinc(1/2) = 2/pi
    assert Hs[0] == pytest.approx(Hr[0]) and Hc[0] == pytest.approx(Hr[0])


def _gauss_sino(geo):
    th = np.arange(geo.n_angles) * geo.dtheta
    s = (np.arange(geo.n_det) - geo.n_det / 2) * geo.ds
    g = direct.gaussian_radon(th[:, None], s[None, :], BLOBS)
    g[:, ~geometry.live_bins(geo.n_det)] = 0.0
    return g


def test_fbp_inverts_the_radon_transform_of_gaussians():
    """f = R# W R f (Eq. FBP) with the R# of [0, pi): the reconstruction of smooth Gaussians
    converges to them."""
    errs = []
    for N in (64, 128):
        geo = geometry.make_geometry(N, 3 * N // 2, 3 * N // 2, 3)
        rec = fbp.fbp(_gauss_sino(geo), geo, "ramp")
        ref = np.where(geometry.disc_mask(N), gaussian_image(N, BLOBS), 0.0)
        errs.append(np.linalg.norm(rec - ref) / np.linalg.norm(ref))
    assert errs[1] < 1e-2
    assert errs[1] < errs[0]


def test_fbp_scale_on_a_centred_gaussian():
    """Peak value of the reconstruction of a centred unit Gaussian is 1 (scale check of W and R#)."""
    N = 128
    geo = geometry.make_geometry(N, 192, 192, 3)
    th = np.arange(geo.n_angles) * geo.dtheta
    s = (np.arange(geo.n_det) - geo.n_det / 2) * geo.ds
    sg = 0.15
    g = np.broadcast_to(direct.gaussian_radon(0.0, s, [(0, 0, sg, 1.0)]), (geo.n_angles, geo.n_det)).copy()
    rec = fbp.fbp(g, geo, "ramp")
    assert rec[N // 2, N // 2] == pytest.approx(1.0, abs=3e-3)
