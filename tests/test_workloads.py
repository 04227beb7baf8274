"""The synthetic inputs are what their recipe says (seeded, in the unit disc)."""

import numpy as np

from oracle import direct
from workloads import ellipse_image, ellipse_sinogram, random_ellipses, random_sinogram


def test_ellipses_are_seeded_and_inside_radius():
    a = random_ellipses(50, 2)
    assert a == random_ellipses(50, 2)
    for e in a:
        assert np.hypot(e.cx, e.cy) + max(e.a, e.b) <= 0.95 + 1e-12
        assert 0.05 <= e.a <= 0.4 and 0.05 <= e.b <= 0.4 and -1 <= e.density <= 1


def test_ellipse_image_vanishes_outside_095():
    N = 128
    img = ellipse_image(N, random_ellipses(10, 1))
    x = (np.arange(N) - N / 2) * (2.0 / N)
    r = np.hypot(x[None, :], x[:, None])
    assert np.all(img[r > 0.95 + 2.0 / N] == 0.0)


def test_ellipse_sinogram_matches_the_oracle_closed_form():
    ell = random_ellipses(7, 3)
    g = ellipse_sinogram(ell, 40, 60)
    th = np.arange(40) * np.pi / 40
    s = (np.arange(60) - 30) * (2 * np.sqrt(2) / 60)
    assert np.max(np.abs(g - direct.ellipse_radon(th[:, None], s[None, :], ell))) < 1e-12


def test_random_sinogram_is_standard_normal():
    g = random_sinogram(200, 300, 3)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01
