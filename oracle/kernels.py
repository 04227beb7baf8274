"""Fourier coefficients of the log-polar kernels zeta and zeta# (Section 3), FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

With L = -log(a_r) and nu = 2 pi / L (Eq. exprcoef1, Eq. exprcoef2):

    zeta_hat [kt, kr] = int_{-beta}^{beta} exp(-i pi theta kt / beta) (cos theta)^(-1 - i nu kr) dtheta
    zeta#_hat[kt, kr] = int_{-beta}^{beta} exp(-i pi theta kt / beta) (cos theta)^(+i nu kr) dtheta

(the stray "rho" in the middle line of the paper's derivation of zeta# is
dropped; its final line is used).  Both integrands are even in theta apart
from the exponential, so each value equals
2 int_0^beta cos(pi theta kt / beta) (cos theta)^alpha dtheta; this is what is
evaluated, by composite Gauss-Legendre quadrature on panels of equal phase
(an independent method from the paper's trapezoid-plus-end-correction rule,
Eq. weightsa, which the GPU plan uses).

Index convention: kt in [-n_theta/2, n_theta/2), kr in [-N_rho/2, N_rho/2);
entry [p, q] of a full-grid array holds the frequency (p or p - n) in DFT
order.  Values for kr < 0 follow from zeta_hat[kt, -kr] = conj(zeta_hat[kt, kr]).
"""

from __future__ import annotations

import math

import numpy as np

GL_NODES = 20


def _panels(omega_lin: float, omega_log: float, beta: float, phase_per_panel: float, min_panels: int = 8):
    """Panel edges on [0, beta] with equal increments of the phase
    Phi(t) = omega_lin * t - omega_log * log(cos t)."""

    def phi(t):
        return omega_lin * t - omega_log * np.log(np.cos(t))

    total = phi(beta)
    P = max(min_panels, int(math.ceil(total / phase_per_panel)))
    targets = np.linspace(0.0, total, P + 1)
    lo = np.zeros(P + 1)
    hi = np.full(P + 1, beta)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        below = phi(mid) < targets
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    edges = 0.5 * (lo + hi)
    edges[0] = 0.0
    edges[-1] = beta
    return edges


def _nodes(edges):
    x, w = np.polynomial.legendre.leggauss(GL_NODES)
    a = edges[:-1, None]
    b = edges[1:, None]
    t = (0.5 * (b - a) * x[None, :] + 0.5 * (a + b)).ravel()
    wt = (0.5 * (b - a) * w[None, :]).ravel()
    return t, wt


def kernel_quadrant(geo, which: str, phase_per_panel: float = 10.0, chunk: int = 512, kr_cols=None):
    """zeta_hat (which='R') or zeta#_hat (which='B') for kt in [0, n_theta/2], kr in [0, N_rho/2].

    Returns a complex128 array of shape (n_theta/2 + 1, N_rho/2 + 1), or of shape
    (n_theta/2 + 1, len(kr_cols)) when only the columns ``kr_cols`` are asked for (the panels
    are the same in both cases: they resolve the fastest oscillation of the whole quadrant).
    """
    beta, L = geo.beta, geo.L
    nu = 2.0 * math.pi / L
    kt = np.arange(geo.n_theta // 2 + 1)
    kr_max = geo.N_rho // 2
    kr = np.arange(kr_max + 1) if kr_cols is None else np.asarray(kr_cols, dtype=np.int64)
    edges = _panels(math.pi * kt[-1] / beta, nu * kr_max, beta, phase_per_panel)
    t, w = _nodes(edges)
    lc = np.log(np.cos(t))
    # A[kt, q] = 2 w_q cos(pi t_q kt / beta) (cos t_q)^{-1 or 0}
    amp = 2.0 * w / np.cos(t) if which == "R" else 2.0 * w
    A = np.cos(np.outer(kt, t) * (math.pi / beta)) * amp[None, :]
    sign = -1.0 if which == "R" else 1.0
    out = np.empty((kt.size, kr.size), dtype=np.complex128)
    for c0 in range(0, kr.size, chunk):
        krc = kr[c0:c0 + chunk]
        ph = sign * nu * np.outer(lc, krc)  # (cos t)^{i sign nu kr} = exp(i sign nu kr log cos t)
        out[:, c0:c0 + chunk] = A @ np.cos(ph) + 1j * (A @ np.sin(ph))
    return out


def kernel_direct(geo, which: str, kt: int, kr: int, n_panels: int = 400):
    """One coefficient from the un-folded integral over [-beta, beta] (for symmetry pins)."""
    beta, L = geo.beta, geo.L
    nu = 2.0 * math.pi / L
    edges = np.linspace(-beta, beta, n_panels + 1)
    x, w = np.polynomial.legendre.leggauss(GL_NODES)
    a, b = edges[:-1, None], edges[1:, None]
    t = (0.5 * (b - a) * x + 0.5 * (a + b)).ravel()
    wt = (0.5 * (b - a) * w).ravel()
    alpha = (-1.0 - 1j * nu * kr) if which == "R" else (1j * nu * kr)
    f = np.exp(-1j * math.pi * t * kt / beta) * np.exp(alpha * np.log(np.cos(t)))
    return complex(np.sum(wt * f))


def full_grid(quadrant: np.ndarray, n_theta: int, N_rho: int) -> np.ndarray:
    """Expand the (kt >= 0, kr >= 0) quadrant to the DFT-ordered n_theta x N_rho grid
    with symmetric frequency indices, using evenness in kt and conjugate symmetry in kr."""
    p = np.arange(n_theta)
    q = np.arange(N_rho)
    kt = np.where(p < n_theta // 2, p, p - n_theta)
    kr = np.where(q < N_rho // 2, q, q - N_rho)
    vals = quadrant[np.abs(kt)[:, None], np.abs(kr)[None, :]]
    return np.where(kr[None, :] < 0, np.conj(vals), vals)


def bhat2d(n_theta: int, N_rho: int) -> np.ndarray:
    """Two-dimensional B-hat on the DFT grid (Eq. Bhat in each variable)."""
    p = np.arange(n_theta)
    q = np.arange(N_rho)
    bt = 2.0 / 3.0 + np.cos(2.0 * np.pi * p / n_theta) / 3.0
    br = 2.0 / 3.0 + np.cos(2.0 * np.pi * q / N_rho) / 3.0
    return bt[:, None] * br[None, :]


def box_response(n_theta: int, r: int) -> np.ndarray:
    """In-band response of the mean of r equally spaced sub-samples centred on each coarse
    angle (the theta low-pass of Algorithm 1, Omega_lp -> Omega_p), on the DFT grid:
    D(kt) = sin(pi kt / n_theta) / (r sin(pi kt / (r n_theta))), D(0) = 1."""
    p = np.arange(n_theta)
    kt = np.where(p < n_theta // 2, p, p - n_theta).astype(np.float64)
    x = np.pi * kt / n_theta
    D = np.ones(n_theta)
    nz = kt != 0
    D[nz] = np.sin(x[nz]) / (r * np.sin(x[nz] / r))
    return D


def multiplier(geo, which: str) -> np.ndarray:
    """Fourier multiplier of Algorithm 1 / 2 step "apply the log-polar transform with the
    pre-filter incorporated", DFT order: zeta_hat / B_hat (cubic) or zeta_hat (linear); for
    the forward transform also divided by the in-band response of the angular box
    low-pass (``box_response``), which the downsampling step applied to the data."""
    K = full_grid(kernel_quadrant(geo, which), geo.n_theta, geo.N_rho)
    if geo.interp == 3:
        K = K / bhat2d(geo.n_theta, geo.N_rho)
    if which == "R":
        K = K / box_response(geo.n_theta, geo.r)[:, None]
    return K


def P_closed_form(mu, alpha, beta, dps: int = 30):
    """Eq. P_closed_form: int_{-beta}^{beta} exp(i mu t) cos(t)^alpha dt via Gamma and 3F2 (mpmath)."""
    import mpmath as mp

    mp.mp.dps = dps
    mu = mp.mpc(mu)
    al = mp.mpc(alpha)
    be = mp.mpf(beta)
    cb = mp.cos(be)
    x = cb ** 2
    t0 = mp.gamma((al + 1) / 2) * mp.gamma(mp.mpf(1) / 2) * mp.gamma((al + 2) / 2) / (
        mp.gamma((al + mu) / 2 + 1) * mp.gamma((al - mu) / 2 + 1))
    a1, a2, a3 = 1, al / 2 + mu / 2 + 1, al / 2 - mu / 2 + 1
    t1 = 2 * mu * cb ** (al + 2) * mp.sin(mu * be) / ((al + 1) * (al + 2)) * mp.hyp3f2(
        a1, a2, a3, (al + 3) / 2, al / 2 + 2, x)
    t2 = 2 * cb ** (al + 1) * mp.cos(be * mu) * mp.sin(be) / (al + 1) * mp.hyp3f2(
        a1, a2, a3, (al + 3) / 2, al / 2 + 1, x)
    return complex(t0 + t1 - t2)
