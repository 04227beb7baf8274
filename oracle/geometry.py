"""Discretisation rules of the log-polar method (oracle side, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Conventions (readings of the paper where it is silent, ambiguous or garbled):

* Image grid X (Eq. Xgrid, rescaled to the unit disc): pixel (i, j) of an
  N x N array has centre x1 = (j - N/2) * 2/N, x2 = (i - N/2) * 2/N.
* Polar grid Sigma (Eq. Polargrid): theta_a = a * pi / n_angles for
  a in [0, n_angles); s_k = (k - n_det/2) * ds with ds = 2*sqrt(2)/n_det.
* Partitions (Section 2): beta = pi / M; a_R and a_r from Eq. aconst;
  L = -log(a_r) is the rho-period.
* N_rho: the bound of Eq. vrho, rounded up to an even 7-smooth integer.
* Angular FFT grid Omega_p (Eq. Lopolargrid_polar): n_theta = 2 * n_th_h
  points over the period [-beta, beta), where n_th_h is the smallest even
  7-smooth integer >= ceil(n_angles / M); phi_j = (j - n_th_h) * dphi with
  dphi = beta / n_th_h.  Data occupy the central half j in
  [n_th_h/2, 3 n_th_h/2), i.e. phi in [-beta/2, beta/2).
* rho grid: rho_i = (i - N_rho + 1) * drho, i in [0, N_rho), drho = L / N_rho
  (the paper's -N_rho < j_rho <= 0).
* Fine angular grid Omega_lp (Eq. Lopolargrid_f): r = ceil(dphi * N / (2 a_R))
  sub-samples per coarse angle at phi_j + (q - (r-1)/2) * dphi / r; their mean
  is the low-pass + downsample of Algorithm 1.
"""

from __future__ import annotations

import dataclasses
import math


def is_7smooth(n: int) -> bool:
    if n < 1:
        return False
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def even_7smooth_at_least(n: int) -> int:
    m = max(int(n), 2)
    while m % 2 or not is_7smooth(m):
        m += 1
    return m


@dataclasses.dataclass(frozen=True)
class Geometry:
    N: int
    n_angles: int
    n_det: int
    M: int
    interp: int
    beta: float
    a_R: float
    a_r: float
    L: float
    N_rho: int
    n_th_h: int
    n_theta: int
    r: int
    dphi: float
    drho: float
    ds: float
    dtheta: float

    def phi(self, j):
        return (j - self.n_th_h) * self.dphi

    def rho(self, i):
        return (i - self.N_rho + 1) * self.drho


def partition_constants(M: int):
    """beta, a_R, a_r of Eq. aconst for M partitions (Section 2)."""
    beta = math.pi / M
    sb = math.sin(beta / 2)
    cb = math.cos(beta / 2)
    a_R = sb / (1.0 + sb)
    a_r = (cb - sb) / (1.0 + sb)
    return beta, a_R, a_r


def make_geometry(N: int, n_angles: int, n_det: int, M: int = 3, interp: int = 3) -> Geometry:
    beta, a_R, a_r = partition_constants(M)
    L = -math.log(a_r)
    # Eq. vrho: N_rho >= ceil(log(a_r) / log(1 - 2 a_R / N))
    nrho_min = math.ceil(math.log(a_r) / math.log(1.0 - 2.0 * a_R / N))
    N_rho = even_7smooth_at_least(nrho_min)
    n_th_h = even_7smooth_at_least(-(-n_angles // M))
    dphi = beta / n_th_h
    r = math.ceil(dphi * N / (2.0 * a_R))
    return Geometry(
        N=N, n_angles=n_angles, n_det=n_det, M=M, interp=interp,
        beta=beta, a_R=a_R, a_r=a_r, L=L,
        N_rho=N_rho, n_th_h=n_th_h, n_theta=2 * n_th_h, r=r,
        dphi=dphi, drho=L / N_rho,
        ds=2.0 * math.sqrt(2.0) / n_det, dtheta=math.pi / n_angles,
    )


def disc_mask(N: int):
    """Pixels whose centre lies strictly inside the unit disc (exact integer test)."""
    import numpy as np

    v = 2 * np.arange(N) - N
    return (v[:, None] ** 2 + v[None, :] ** 2) < N * N


def live_bins(n_det: int):
    """Detector bins with |s_k| < 1, i.e. 2 (2k - n_det)^2 < n_det^2 (exact integer test)."""
    import numpy as np

    v = 2 * np.arange(n_det) - n_det
    return 2 * v * v < n_det * n_det


def angle_partition(a: int, n_angles: int, M: int):
    """Partition index m = round(theta / beta) (half up) for theta_a = a pi / n_angles.

    Returns (m, num, flip): phi = theta - m beta = num * pi / (M n_angles); when
    round() gives M the angle is mapped to m = 0 through Rf(theta, s) =
    Rf(theta - pi, -s) (flip = True).  Eq. Radon_all_pb.
    """
    m = (2 * a * M + n_angles) // (2 * n_angles)
    flip = False
    num = a * M - m * n_angles
    if m == M:
        m = 0
        flip = True
        num = a * M - M * n_angles
    return m, num, flip
