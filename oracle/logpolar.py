"""Algorithm 1 (fast Radon transform), Algorithm 2 (fast back-projection) and the exact
transpose of Algorithm 1, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Each step follows the paper's order and notation; the DFTs are dense matrix
products of the definition exp(-2 pi i j k / n).  Conventions are those of
``oracle.geometry``.  Additional readings:

* The image is taken to vanish outside the open unit disc (the method assumes
  supp f in the unit disc, Section 2): pixels with |x| >= 1 are zeroed before
  Q is applied.  Detector bins with |s| >= 1 are zero in R f and are ignored
  by R# (those lines miss the disc).
* R# g(x) = int_0^pi g(theta, x . theta) dtheta (no factor 2, no a_R); R f
  carries the factor 1 / a_R of Eq. Radon_all_pb.
* The output of each convolution is kept on the central half of the angular
  grid plus two rows on each side (the cubic taps of points with
  |phi| <= beta/2 reach one row below and two rows above the half).
* The multiplier on the rho-Nyquist column is applied through Re(.) of the
  complex inverse DFT, i.e. the Hermitian average of the +-N_rho/2 values.
* The sinogram is extended to theta in [0, 2 pi) by g(theta + pi, s) =
  g(theta, -s); with s_k = (k - n_det/2) ds the flip maps bin k to n_det - k,
  so each detector row is handled as the n_det + 1 samples k in [0, n_det]
  (the extra one, s = +sqrt(2), is zero).  Q acts on this (2 n_angles) x
  (n_det + 1) array: periodic in theta, zero boundary in s.
"""

from __future__ import annotations

import math

import numpy as np

from . import bspline, kernels
from .geometry import angle_partition, disc_mask, live_bins

HALO_LO = 2  # output rows kept below the central half
HALO_HI = 2  # and above it


def dft_matrix(n: int, inverse: bool = False) -> np.ndarray:
    p = np.outer(np.arange(n), np.arange(n)) % n
    sgn = 1.0 if inverse else -1.0
    return np.exp(sgn * 2j * np.pi * p / n)


class _Dft:
    """Cache of the DFT matrices of one geometry."""

    def __init__(self, geo):
        self.Frho = dft_matrix(geo.N_rho)
        self.Fth = dft_matrix(geo.n_theta)


def logpolar_convolution(h_central: np.ndarray, K: np.ndarray, geo, dft: _Dft | None = None) -> np.ndarray:
    """Periodic convolution on [-beta, beta) x [log a_r, 0) by the DFT (Section 3).

    ``h_central``: samples on the central half rows (n_th_h x N_rho); the other
    rows of the n_theta x N_rho lattice are zero.  Returns rows
    [n_th_h/2 - HALO_LO, 3 n_th_h/2 + HALO_HI) of Re(IDFT2(DFT2(h) * K)), with
    the inverse DFT normalised by 1 / (n_theta N_rho).
    """
    dft = dft or _Dft(geo)
    nh, nt, nr = geo.n_th_h, geo.n_theta, geo.N_rho
    rows_in = np.arange(nh // 2, nh // 2 + nh)
    rows_out = np.arange(nh // 2 - HALO_LO, nh // 2 + nh + HALO_HI) % nt  # output is nt-periodic
    A = h_central @ dft.Frho                  # DFT along rho (F is symmetric)
    H = dft.Fth[:, rows_in] @ A               # DFT along theta of the zero-padded columns
    H = H * K
    Yt = np.conj(dft.Fth[rows_out, :]) @ H    # inverse DFT along theta, kept rows only
    Fi = np.conj(dft.Frho)
    y = Yt.real @ Fi.real - Yt.imag @ Fi.imag  # real part of the inverse DFT along rho
    return y / (nt * nr)


def logpolar_convolution_transpose(ybar: np.ndarray, K: np.ndarray, geo, dft: _Dft | None = None) -> np.ndarray:
    """Transpose of ``logpolar_convolution`` (a real linear map h -> y).

    The forward map is y = Re(A h) with the complex-linear
    A h = conj(F_out) (K * (F_in h F_rho)) conj(F_rho) / (n_theta N_rho), where F_in are the
    DFT columns of the central rows and F_out the inverse-DFT rows kept.  For real h and y,
    sum(y * ybar) = sum(h * Re(A^T ybar)), and A^T applies the transposed factors in reverse
    order (K acts elementwise and is its own transpose; F_rho is symmetric).
    ``ybar``: (n_th_h + HALO_LO + HALO_HI) x N_rho; returns n_th_h x N_rho.
    """
    dft = dft or _Dft(geo)
    nh, nt, nr = geo.n_th_h, geo.n_theta, geo.N_rho
    rows_in = np.arange(nh // 2, nh // 2 + nh)
    rows_out = np.arange(nh // 2 - HALO_LO, nh // 2 + nh + HALO_HI) % nt
    Z = np.conj(dft.Fth[rows_out, :]).T @ np.asarray(ybar, dtype=np.float64) @ np.conj(dft.Frho).T
    Z = Z * K
    hb = dft.Fth[:, rows_in].T @ Z @ dft.Frho.T
    return hb.real / (nt * nr)


def image_coefficients(f: np.ndarray, geo) -> np.ndarray:
    """Mask to the disc, then Q (cubic) or the samples themselves (linear)."""
    fm = np.where(disc_mask(geo.N), np.asarray(f, dtype=np.float64), 0.0)
    if geo.interp == 3:
        fm = bspline.prefilter_zero(bspline.prefilter_zero(fm, axis=0), axis=1)
    return fm


def sinogram_coefficients(g: np.ndarray, geo) -> np.ndarray:
    """Extended (2 n_angles) x (n_det + 1) array of Q g (cubic) or samples (linear)."""
    na, nd = geo.n_angles, geo.n_det
    gm = np.where(live_bins(nd)[None, :], np.asarray(g, dtype=np.float64), 0.0)
    E = np.zeros((2 * na, nd + 1))
    E[:na, :nd] = gm
    E[na:, :] = E[:na, ::-1]        # row a + n_angles, column k  <-  row a, column n_det - k
    if geo.interp == 3:
        E = bspline.prefilter_zero(E, axis=1)
        E = bspline.prefilter_periodic(E, axis=0)
    return E


def _sample_rows(geo, jj):
    """phi of the central rows jj (array)."""
    return (jj + geo.n_th_h // 2 - geo.n_th_h) * geo.dphi


def forward(f: np.ndarray, geo, K: np.ndarray | None = None, dft: _Dft | None = None,
            partitions=None, row_chunk: int = 32) -> np.ndarray:
    """Algorithm 1.  Returns R f on Sigma, float64 [n_angles, n_det].

    ``partitions`` restricts the loop over m (the other angles stay zero).
    """
    N, M, r = geo.N, geo.M, geo.r
    nh, nr = geo.n_th_h, geo.N_rho
    c = image_coefficients(f, geo)                     # pre-filter Q
    K = kernels.multiplier(geo, "R") if K is None else K
    dft = dft or _Dft(geo)
    rho = geo.rho(np.arange(nr))
    erho = np.exp(rho)
    q = (np.arange(r) - (r - 1) / 2.0) * geo.dphi / r
    Rf = np.zeros((geo.n_angles, geo.n_det))
    live = live_bins(geo.n_det)
    sk = (np.arange(geo.n_det) - geo.n_det / 2) * geo.ds
    for m in (range(M) if partitions is None else partitions):
        cm, sm = math.cos(m * geo.beta), math.sin(m * geo.beta)
        h = np.zeros((nh, nr))
        for j0 in range(0, nh, row_chunk):
            jj = np.arange(j0, min(nh, j0 + row_chunk))
            phi = _sample_rows(geo, jj)[:, None, None] + q[None, :, None]   # Omega_lp angles
            y1 = erho[None, None, :] * np.cos(phi)
            y2 = erho[None, None, :] * np.sin(phi)
            u1 = (y1 - (1.0 - geo.a_R)) / geo.a_R                         # T_m^{-1}
            u2 = y2 / geo.a_R
            x1 = cm * u1 - sm * u2
            x2 = sm * u1 + cm * u2
            col = x1 * (N / 2) + N / 2
            row = x2 * (N / 2) + N / 2
            vals = bspline.interp2d(c, row, col, order=geo.interp)         # resample T_m f on Omega_lp
            h[jj - 0, :] = vals.mean(axis=1) * erho[None, :]               # downsample to Omega_p, times e^rho
        y = logpolar_convolution(h, K, geo, dft)                           # convolution with zeta / B-hat
        # resample from S_m^{-1} Omega_p to Sigma
        for a in range(geo.n_angles):
            am, num, flip = angle_partition(a, geo.n_angles, M)
            if am != m:
                continue
            phi_a = num * math.pi / (M * geo.n_angles)
            s = -sk if flip else sk
            t = geo.a_R * s[live] + (1.0 - geo.a_R) * math.cos(phi_a)
            crho = np.log(t) / geo.drho + nr - 1
            cth = np.full(crho.shape, phi_a / geo.dphi + nh // 2 + HALO_LO)
            Rf[a, live] = bspline.interp2d(y, cth, crho, order=geo.interp,
                                           mode0="zero", mode1="periodic") / geo.a_R
    return Rf


def backproject(g: np.ndarray, geo, K: np.ndarray | None = None, dft: _Dft | None = None,
                partitions=None, row_chunk: int = 64) -> np.ndarray:
    """Algorithm 2.  Returns R# g on X, float64 [N, N]."""
    N, M = geo.N, geo.M
    nh, nr = geo.n_th_h, geo.N_rho
    E = sinogram_coefficients(g, geo)                  # pre-filter Q
    K = kernels.multiplier(geo, "B") if K is None else K
    dft = dft or _Dft(geo)
    erho = np.exp(geo.rho(np.arange(nr)))
    img = np.zeros((N, N))
    mask = disc_mask(N)
    ii, jj_pix = np.nonzero(mask)
    x1 = (jj_pix - N / 2) * (2.0 / N)
    x2 = (ii - N / 2) * (2.0 / N)
    for m in (range(M) if partitions is None else partitions):
        G = np.zeros((nh, nr))
        for j0 in range(0, nh, row_chunk):
            jj = np.arange(j0, min(nh, j0 + row_chunk))
            phi = _sample_rows(geo, jj)[:, None]
            theta = phi + m * geo.beta
            s = (erho[None, :] - (1.0 - geo.a_R) * np.cos(phi)) / geo.a_R   # g(S_m) on Omega_p
            cth = np.broadcast_to(theta / geo.dtheta, s.shape)
            cs = s / geo.ds + geo.n_det / 2
            G[jj, :] = bspline.interp2d(E, cth, cs, order=geo.interp,
                                        mode0="periodic", mode1="zero")       # resample g(S_m)
        y = logpolar_convolution(G, K, geo, dft)                               # convolution with zeta# / B-hat
        cm, sm = math.cos(m * geo.beta), math.sin(m * geo.beta)
        y1 = geo.a_R * (cm * x1 + sm * x2) + 1.0 - geo.a_R                     # T_m x
        y2 = geo.a_R * (-sm * x1 + cm * x2)
        cth = np.arctan2(y2, y1) / geo.dphi + nh // 2 + HALO_LO
        crho = 0.5 * np.log(y1 * y1 + y2 * y2) / geo.drho + nr - 1
        img[ii, jj_pix] += bspline.interp2d(y, cth, crho, order=geo.interp,
                                            mode0="zero", mode1="periodic")    # to X, summed over m
    return img


def transpose(gbar: np.ndarray, geo, K: np.ndarray | None = None, dft: _Dft | None = None,
              partitions=None, row_chunk: int = 32) -> np.ndarray:
    """Exact transpose of the discrete map ``forward`` computes: sum(forward(f) * gbar) ==
    sum(f * transpose(gbar)) for every f and gbar.  Returns float64 [N, N].

    Algorithm 2 discretises the continuous adjoint R# instead, so R# is the transpose only up
    to the discretisation error and a scale; this map is the one whose gradients are exact for
    objectives built on ``forward``.  The steps of Algorithm 1 are transposed in reverse order:
    the resampling to Sigma becomes spreading onto the log-polar coefficient grid, the
    convolution becomes ``logpolar_convolution_transpose``, the resampling of T_m f on
    Omega_lp becomes spreading onto the image coefficient grid, and Q (applied along both
    axes) and the disc mask become Q^T and the mask.
    """
    N, M, r = geo.N, geo.M, geo.r
    nh, nr = geo.n_th_h, geo.N_rho
    K = kernels.multiplier(geo, "R") if K is None else K
    dft = dft or _Dft(geo)
    erho = np.exp(geo.rho(np.arange(nr)))
    q = (np.arange(r) - (r - 1) / 2.0) * geo.dphi / r
    live = live_bins(geo.n_det)
    sk = (np.arange(geo.n_det) - geo.n_det / 2) * geo.ds
    gbar = np.asarray(gbar, dtype=np.float64)
    cbar = np.zeros((N, N))
    for m in (range(M) if partitions is None else partitions):
        ybar = np.zeros((nh + HALO_LO + HALO_HI, nr))
        for a in range(geo.n_angles):                                    # transpose of S_m^{-1} Omega_p -> Sigma
            am, num, flip = angle_partition(a, geo.n_angles, M)
            if am != m:
                continue
            phi_a = num * math.pi / (M * geo.n_angles)
            s = -sk if flip else sk
            t = geo.a_R * s[live] + (1.0 - geo.a_R) * math.cos(phi_a)
            crho = np.log(t) / geo.drho + nr - 1
            cth = np.full(crho.shape, phi_a / geo.dphi + nh // 2 + HALO_LO)
            ybar += bspline.spread2d(gbar[a, live] / geo.a_R, cth, crho, ybar.shape, order=geo.interp,
                                     mode0="zero", mode1="periodic")
        hbar = logpolar_convolution_transpose(ybar, K, geo, dft)          # transpose of the convolution
        cm, sm = math.cos(m * geo.beta), math.sin(m * geo.beta)
        for j0 in range(0, nh, row_chunk):                               # transpose of the resampling on Omega_lp
            jj = np.arange(j0, min(nh, j0 + row_chunk))
            phi = _sample_rows(geo, jj)[:, None, None] + q[None, :, None]
            y1 = erho[None, None, :] * np.cos(phi)
            y2 = erho[None, None, :] * np.sin(phi)
            u1 = (y1 - (1.0 - geo.a_R)) / geo.a_R
            u2 = y2 / geo.a_R
            x1 = cm * u1 - sm * u2
            x2 = sm * u1 + cm * u2
            col = x1 * (N / 2) + N / 2
            row = x2 * (N / 2) + N / 2
            v = np.broadcast_to((hbar[jj, :] * erho[None, :] / r)[:, None, :], col.shape)
            cbar += bspline.spread2d(v, row, col, (N, N), order=geo.interp)
    if geo.interp == 3:
        Qn = bspline.prefilter_zero(np.eye(N), axis=0)                   # Q x = Qn @ x; c = Qn f Qn^T
        cbar = Qn.T @ cbar @ Qn
    return np.where(disc_mask(N), cbar, 0.0)
