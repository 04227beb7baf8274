"""Seeded phantoms and sinograms.

Recipe (stated once, used by every test and by the benchmark):

* Ellipse phantom: ``n`` ellipses, semi-axes a, b ~ U(0.05, 0.4), orientation
  psi ~ U(0, pi), density ~ U(-1, 1); the centre is drawn uniformly in the unit
  disc and redrawn until |c| + max(a, b) <= 0.95, so the phantom vanishes
  outside radius 0.95.  The paper's test object is a linear combination of
  ellipse indicators inscribed in the unit circle (Section 7); these random
  ellipses stand in for the modified Shepp-Logan table, which is not used.
* Pixel value: the mean of the summed indicator functions over a 4 x 4 grid of
  sub-pixel points (area-coverage estimate).
* Random sinogram: i.i.d. N(0, 1) entries.
* All draws use ``numpy.random.default_rng(seed)`` (PCG64).
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Ellipse:
    cx: float
    cy: float
    a: float
    b: float
    psi: float
    density: float


def random_ellipses(n: int, seed: int, max_radius: float = 0.95) -> list[Ellipse]:
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        a, b = rng.uniform(0.05, 0.4, size=2)
        psi = rng.uniform(0.0, np.pi)
        dens = rng.uniform(-1.0, 1.0)
        reach = max(a, b)
        while True:
            cx, cy = rng.uniform(-1.0, 1.0, size=2)
            if np.hypot(cx, cy) + reach <= max_radius:
                break
        out.append(Ellipse(float(cx), float(cy), float(a), float(b), float(psi), float(dens)))
    return out


def _grid(N: int, sub: int):
    h = 2.0 / N
    base = (np.arange(N) - N / 2) * h
    off = ((np.arange(sub) + 0.5) / sub - 0.5) * h
    return base, off


def ellipse_image(N: int, ellipses: list[Ellipse], sub: int = 4) -> np.ndarray:
    """Area-coverage rasterisation of a sum of ellipse indicators, float64 [N, N]."""
    base, off = _grid(N, sub)
    img = np.zeros((N, N))
    for e in ellipses:
        c, s = np.cos(e.psi), np.sin(e.psi)
        reach = max(e.a, e.b) + 2.0 / N
        rows = np.nonzero(np.abs(base - e.cy) <= reach)[0]
        cols = np.nonzero(np.abs(base - e.cx) <= reach)[0]
        if rows.size == 0 or cols.size == 0:
            continue
        acc = np.zeros((rows.size, cols.size))
        for oy in off:
            y = (base[rows] + oy - e.cy)[:, None]
            for ox in off:
                x = (base[cols] + ox - e.cx)[None, :]
                u = x * c + y * s
                v = -x * s + y * c
                acc += ((u / e.a) ** 2 + (v / e.b) ** 2 <= 1.0)
        img[np.ix_(rows, cols)] += e.density * acc / (sub * sub)
    return img


def gaussian_image(N: int, blobs) -> np.ndarray:
    """Point samples of sum_k w_k exp(-|x - c_k|^2 / (2 s_k^2)); blobs = [(cx, cy, s, w), ...]."""
    h = 2.0 / N
    x = (np.arange(N) - N / 2) * h
    X1, X2 = np.meshgrid(x, x)
    img = np.zeros((N, N))
    for cx, cy, s, w in blobs:
        img += w * np.exp(-((X1 - cx) ** 2 + (X2 - cy) ** 2) / (2.0 * s * s))
    return img


def smooth_random_image(N: int, seed: int, n_blobs: int = 24) -> np.ndarray:
    """A seeded sum of Gaussian bumps (widths 0.03-0.2) inside radius 0.8."""
    rng = np.random.default_rng(seed)
    blobs = []
    for _ in range(n_blobs):
        s = rng.uniform(0.03, 0.2)
        while True:
            cx, cy = rng.uniform(-0.8, 0.8, size=2)
            if np.hypot(cx, cy) <= 0.8 - s:
                break
        blobs.append((cx, cy, s, rng.uniform(-1.0, 1.0)))
    return gaussian_image(N, blobs)


def random_sinogram(n_angles: int, n_det: int, seed: int) -> np.ndarray:
    """i.i.d. N(0, 1) sinogram, float64 [n_angles, n_det]."""
    return np.random.default_rng(seed).standard_normal((n_angles, n_det))


def ellipse_sinogram(ellipses: list[Ellipse], n_angles: int, n_det: int) -> np.ndarray:
    """Line integrals of the ellipse indicators on the sinogram grid theta_a = a pi / n_angles,
    s_k = (k - n_det/2) 2 sqrt(2) / n_det (chord length of each ellipse times its density)."""
    th = (np.arange(n_angles) * np.pi / n_angles)[:, None]
    s = ((np.arange(n_det) - n_det / 2) * (2.0 * np.sqrt(2.0) / n_det))[None, :]
    out = np.zeros((n_angles, n_det))
    for e in ellipses:
        c, sn = np.cos(th - e.psi), np.sin(th - e.psi)
        half2 = (e.a * c) ** 2 + (e.b * sn) ** 2  # squared support half-width along s
        t = s - (e.cx * np.cos(th) + e.cy * np.sin(th))
        chord = np.where(t * t < half2, 2.0 * e.a * e.b * np.sqrt(np.maximum(half2 - t * t, 0.0)) / half2, 0.0)
        out += e.density * chord
    return out


def ellipse_sinogram_torch(ellipses: list[Ellipse], n_angles: int, n_det: int, device="cuda"):
    """``ellipse_sinogram`` evaluated with torch in float64 on ``device`` (the same chord-length
    formula; for sinograms too large to build quickly on the host)."""
    import math

    import torch

    th = (torch.arange(n_angles, dtype=torch.float64, device=device) * (math.pi / n_angles))[:, None]
    s = ((torch.arange(n_det, dtype=torch.float64, device=device) - n_det / 2) * (2.0 * math.sqrt(2.0) / n_det))[None, :]
    out = torch.zeros((n_angles, n_det), dtype=torch.float64, device=device)
    cth, sth = torch.cos(th), torch.sin(th)
    for e in ellipses:
        c, sn = torch.cos(th - e.psi), torch.sin(th - e.psi)
        half2 = (e.a * c) ** 2 + (e.b * sn) ** 2
        t = s - (e.cx * cth + e.cy * sth)
        rem = torch.clamp(half2 - t * t, min=0.0)
        out += e.density * 2.0 * e.a * e.b * torch.sqrt(rem) / half2
    return out


def ellipse_values_at(ellipses: list[Ellipse], N: int, rows, cols, sub: int = 4) -> np.ndarray:
    """``ellipse_image`` at the listed pixels only (same 4 x 4 sub-pixel coverage)."""
    base, off = _grid(N, sub)
    y0 = base[np.asarray(rows)]
    x0 = base[np.asarray(cols)]
    out = np.zeros(y0.shape)
    for e in ellipses:
        c, s = np.cos(e.psi), np.sin(e.psi)
        acc = np.zeros(y0.shape)
        for oy in off:
            y = y0 + oy - e.cy
            for ox in off:
                x = x0 + ox - e.cx
                u = x * c + y * s
                v = -x * s + y * c
                acc += ((u / e.a) ** 2 + (v / e.b) ** 2 <= 1.0)
        out += e.density * acc / (sub * sub)
    return out


def slice_sizes(count: int, seed: int, choices=(256, 512, 1024, 2048, 4096)) -> list[int]:
    """Uneven slice sizes N drawn uniformly from ``choices``."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.choice(np.asarray(choices), size=count)]
