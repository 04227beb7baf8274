"""Cubic B-spline pieces of the method (Section 5), FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``B`` is the cubic cardinal B-spline of Section 5.  Its second branch is
  read as (-|x|^3 + 6|x|^2 - 12|x| + 8)/6 = (2 - |x|)^3 / 6 (the printed
  "-12x" drops the absolute value).
* ``prefilter_*`` apply the pre-filter Q by the causal / anti-causal recursion
  of Eq. Qfrecursive with pole z = sqrt(3) - 2.  Two boundary rules are used:
  - "zero": samples outside [0, n) are zero and the coefficient sequence is
    zero outside [0, n) (c_{-1} = c_n = 0), so the spline interpolates every
    sample (the interpolation condition of Eq. Bsplineinterp) and vanishes
    beyond the array.  Exactly, this is the infinite recursion run on the
    extension of f that is odd about -1 and about n (period 2n + 2); the
    start values below are that extension's geometric sums.
  - "periodic": the sequence is periodic with period n.
* ``spread2d`` is the transpose of ``interp2d`` (used by the exact transpose of
  Algorithm 1).
* ``interp_*`` evaluate Eq. wsumn: with k = floor(t) and alpha = t - k the
  value is  B(alpha+1) c_{k-1} + B(alpha) c_k + B(alpha-1) c_{k+1} +
  B(alpha-2) c_{k+2}  (the printed w_0..w_3 are listed in reverse order of
  the taps; B is even so this is the same sum).
"""

from __future__ import annotations

import math

import numpy as np

Z1 = math.sqrt(3.0) - 2.0  # pole of the recursive pre-filter, Eq. Qfrecursive


def B(x):
    """Cubic cardinal B-spline (Section 5)."""
    ax = np.abs(np.asarray(x, dtype=np.float64))
    out = np.zeros_like(ax)
    m0 = ax < 1.0
    m1 = (ax >= 1.0) & (ax < 2.0)
    out[m0] = (3.0 * ax[m0] ** 3 - 6.0 * ax[m0] ** 2 + 4.0) / 6.0
    out[m1] = (-ax[m1] ** 3 + 6.0 * ax[m1] ** 2 - 12.0 * ax[m1] + 8.0) / 6.0
    return out


def Bhat(xi):
    """Fourier series of the integer samples of B, Eq. Bhat: 2/3 + cos(2 pi xi) / 3."""
    return 2.0 / 3.0 + np.cos(2.0 * np.pi * np.asarray(xi, dtype=np.float64)) / 3.0


def _move(f, axis):
    return np.moveaxis(np.asarray(f, dtype=np.float64), axis, 0)


def prefilter_zero(f, axis=0):
    """Q along ``axis`` with the zero boundary (c_{-1} = c_n = 0)."""
    x = _move(f, axis)
    n = x.shape[0]
    z = Z1
    P = 2 * n + 2
    # odd extension F of period P: F_j = f_j (j < n), 0 (j = n, 2n+1), -f_{2n-j} (n < j < 2n+1)
    S = np.zeros(x.shape[1:])
    zp = 1.0
    for j in range(P):
        if j < n:
            S = S + zp * x[j]
        elif n < j < 2 * n + 1:
            S = S - zp * x[2 * n - j]
        zp *= z
        if zp == 0.0:
            break
    S = S / (1.0 - z ** P)
    cplus = np.empty_like(x)
    prev = -6.0 * z * S  # (Q f^+)_{-1}
    for k in range(n):
        prev = 6.0 * x[k] + z * prev
        cplus[k] = prev
    c = np.empty_like(x)
    nxt = np.zeros(x.shape[1:])  # c_n = 0
    for k in range(n - 1, -1, -1):
        nxt = z * (nxt - cplus[k])
        c[k] = nxt
    return np.moveaxis(c, 0, axis)


def prefilter_periodic(f, axis=0):
    """Q along ``axis`` for an n-periodic sequence."""
    x = _move(f, axis)
    n = x.shape[0]
    z = Z1
    zn = z ** n
    S = np.zeros(x.shape[1:])
    zp = 1.0
    for j in range(n):
        S = S + zp * x[(-1 - j) % n]
        zp *= z
    cplus = np.empty_like(x)
    prev = 6.0 * S / (1.0 - zn)  # (Q f^+)_{-1}
    for k in range(n):
        prev = 6.0 * x[k] + z * prev
        cplus[k] = prev
    T = np.zeros(x.shape[1:])
    zp = 1.0
    for j in range(n):
        T = T + zp * cplus[(n - 1 + j) % n]
        zp *= z
    c = np.empty_like(x)
    nxt = -z * T / (1.0 - zn)  # c_{n-1}
    c[n - 1] = nxt
    for k in range(n - 2, -1, -1):
        nxt = z * (nxt - cplus[k])
        c[k] = nxt
    return np.moveaxis(c, 0, axis)


def cubic_weights(alpha):
    """Weights of taps k-1, k, k+1, k+2 (Eq. wsumn) as an array [..., 4]."""
    a = np.asarray(alpha, dtype=np.float64)
    return np.stack([B(a + 1.0), B(a), B(a - 1.0), B(a - 2.0)], axis=-1)


def linear_weights(alpha):
    """Weights of taps k, k+1 for linear interpolation."""
    a = np.asarray(alpha, dtype=np.float64)
    return np.stack([1.0 - a, a], axis=-1)


def _taps(t, order):
    t = np.asarray(t, dtype=np.float64)
    k = np.floor(t)
    alpha = t - k
    k = k.astype(np.int64)
    if order == 3:
        return k - 1, cubic_weights(alpha)
    return k, linear_weights(alpha)


def _index(idx, n, mode):
    """Map tap indices to the array; returns (index, valid)."""
    if mode == "periodic":
        return np.mod(idx, n), np.ones(idx.shape, dtype=bool)
    valid = (idx >= 0) & (idx < n)
    return np.where(valid, idx, 0), valid


def interp2d(c, t0, t1, order=3, mode0="zero", mode1="zero"):
    """Tensor-product spline (order 3) or bilinear (order 1) interpolation.

    ``c`` holds coefficients (order 3) or samples (order 1); ``t0`` / ``t1``
    are fractional indices along axis 0 / axis 1 (same shape).  Taps outside
    the array read zero ("zero") or wrap ("periodic").
    """
    c = np.asarray(c, dtype=np.float64)
    n0, n1 = c.shape
    k0, w0 = _taps(t0, order)
    k1, w1 = _taps(t1, order)
    ntap = w0.shape[-1]
    out = np.zeros(np.shape(t0))
    for d0 in range(ntap):
        i0, v0 = _index(k0 + d0, n0, mode0)
        for d1 in range(ntap):
            i1, v1 = _index(k1 + d1, n1, mode1)
            val = c[i0, i1]
            out += np.where(v0 & v1, val, 0.0) * w0[..., d0] * w1[..., d1]
    return out


def spread2d(v, t0, t1, shape, order=3, mode0="zero", mode1="zero"):
    """Transpose of ``interp2d`` with respect to ``c``: every value v (at fractional indices
    (t0, t1), arrays of one shape) is added, times the tap weight, to each tap ``interp2d``
    reads; taps that ``interp2d`` reads as zero are dropped, periodic taps wrap.  Returns an
    array of ``shape``, so that sum(interp2d(c, t0, t1) * v) == sum(c * spread2d(v, t0, t1))."""
    n0, n1 = shape
    t0 = np.asarray(t0, dtype=np.float64)
    t1 = np.asarray(t1, dtype=np.float64)
    v = np.broadcast_to(np.asarray(v, dtype=np.float64), t0.shape)
    k0, w0 = _taps(t0, order)
    k1, w1 = _taps(t1, order)
    ntap = w0.shape[-1]
    out = np.zeros(shape)
    for d0 in range(ntap):
        i0, v0 = _index(k0 + d0, n0, mode0)
        for d1 in range(ntap):
            i1, v1 = _index(k1 + d1, n1, mode1)
            ok = v0 & v1
            np.add.at(out, (i0[ok], i1[ok]), (v * w0[..., d0] * w1[..., d1])[ok])
    return out


def interp1d(c, t, order=3, mode="zero"):
    """One-dimensional version of ``interp2d`` along the last axis of ``c`` (1-D array)."""
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    k, w = _taps(t, order)
    out = np.zeros(np.shape(t))
    for d in range(w.shape[-1]):
        i, v = _index(k + d, n, mode)
        out += np.where(v, c[i], 0.0) * w[..., d]
    return out
