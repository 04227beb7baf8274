"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

Nothing here computes any part of the Radon / back-projection method: these
functions only draw random numbers and rasterise simple shapes on the image
grid (pixel (i, j) has centre x1 = (j - N/2) * 2/N, x2 = (i - N/2) * 2/N).
"""

from .phantoms import (  # noqa: F401
    Ellipse,
    random_ellipses,
    ellipse_image,
    ellipse_sinogram,
    ellipse_sinogram_torch,
    ellipse_values_at,
    gaussian_image,
    random_sinogram,
    smooth_random_image,
    slice_sizes,
)
