"""FP64 CPU oracle for the log-polar Radon transform and back-projection.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never imports it and
shares no code with it.

Contents
--------
geometry   discretisation rules (Sections 2 and 4: Eq. aconst, Eq. vrho, the
           grids X, Sigma, Omega_lp, Omega_p)
bspline    cubic B-spline, the recursive pre-filter Q (Eq. Qfrecursive) and
           tensor-product interpolation (Eq. Bsplineinterp, Eq. wsumn)
kernels    Fourier coefficients of zeta and zeta# (Eq. exprcoef1, exprcoef2)
           by composite Gauss-Legendre quadrature, and the closed form P
           (Eq. P_closed_form) for cross-checks
logpolar   Algorithm 1 (fast Radon transform) and Algorithm 2 (fast
           back-projection) written step by step, with DFTs as dense
           matrix products
direct     exact line integrals of the interpolated image and the direct
           back-projection, plus analytic Radon transforms of ellipses and
           Gaussians (Section 7)
"""
