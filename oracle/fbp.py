"""Filtered back-projection f = R# W g (Eq. FBP), FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

W filters each sinogram row along s, with bins |s| >= 1 taken as zero.
- With R# over [0, pi), f = R# W R f for the transfer function |sigma|, sigma in cycles per unit
  of s. This follows from the Fourier slice theorem (Section 4) and the polar form of the inverse
  Fourier transform.
- The ramp is the band-limited kernel sampled at the detector spacing (the textbook
  Ramachandran-Lakshminarayanan form): h(0) = 1/(4 ds^2), h(n) = -1/(pi^2 n^2 ds^2) for odd n,
  and 0 for even n != 0.
- Its transfer function on the P-point DFT grid (P = n_filter, the smallest even 7-smooth
  integer >= 2 n_det) is ds * DFT(h).
- The Shepp-Logan and cosine filters multiply it by sinc(sigma / (2 sigma_max)) and
  cos(pi sigma / (2 sigma_max)), with sigma_k = k / (P ds) and sigma_max = 1 / (2 ds)
  (Eq. SLfilt, Eq. cosfilt, read with the cutoff at the sampling band edge).
- The filtered row is the first n_det values of the circular convolution of the zero-padded row
  with h, i.e. Re IDFT(DFT(row) * H).
"""

from __future__ import annotations

import functools
import math

import numpy as np

from . import logpolar
from .geometry import even_7smooth_at_least, live_bins

FILTERS = ("ramp", "shepp-logan", "cosine")


def filter_length(n_det: int) -> int:
    return even_7smooth_at_least(2 * n_det)


def ramp_kernel(P: int, ds: float) -> np.ndarray:
    """h(n) for n in DFT order (n and n - P identified), length P."""
    n = np.arange(P)
    n = np.where(n <= P // 2, n, n - P).astype(np.float64)
    h = np.zeros(P)
    odd = (np.abs(n) % 2) == 1
    h[odd] = -1.0 / (math.pi ** 2 * n[odd] ** 2 * ds * ds)
    h[n == 0] = 1.0 / (4.0 * ds * ds)
    return h


@functools.lru_cache(maxsize=8)
def transfer(P: int, ds: float, kind: str) -> np.ndarray:
    """Transfer function on the full P-point DFT grid (real and even).  Cached per (P, ds, kind);
    callers must not modify the returned array."""
    h = ramp_kernel(P, ds)
    k = np.arange(P)
    # the DFT of the even real kernel, written out as a cosine sum
    H = ds * np.array([np.sum(h * np.cos(2 * math.pi * kk * np.arange(P) / P)) for kk in k])
    kk = np.minimum(k, P - k).astype(np.float64)
    x = math.pi * kk / P  # pi sigma / (2 sigma_max)
    if kind == "shepp-logan":
        w = np.ones(P)
        w[kk > 0] = np.sin(x[kk > 0]) / x[kk > 0]
        H = H * w
    elif kind == "cosine":
        H = H * np.cos(x)
    elif kind != "ramp":
        raise ValueError(kind)
    H.flags.writeable = False  # shared by the cache
    return H


def filter_sinogram(g: np.ndarray, geo, kind: str = "ramp") -> np.ndarray:
    nd = geo.n_det
    P = filter_length(nd)
    gm = np.where(live_bins(nd)[None, :], np.asarray(g, dtype=np.float64), 0.0)
    pad = np.zeros((gm.shape[0], P))
    pad[:, :nd] = gm
    H = transfer(P, geo.ds, kind)
    out = np.fft.ifft(np.fft.fft(pad, axis=1) * H[None, :], axis=1).real
    return out[:, :nd]


def fbp(g: np.ndarray, geo, kind: str = "ramp", **kw) -> np.ndarray:
    """R# of the filtered sinogram (Algorithm 2 on W g)."""
    return logpolar.backproject(filter_sinogram(g, geo, kind), geo, **kw)
