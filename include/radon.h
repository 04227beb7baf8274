/*
 * radon.h -- C ABI of the log-polar Radon transform / back-projection library (libradon.so).
 *
 * The library evaluates the Radon transform R and its adjoint, the back-projection R#, of
 * Andersson, Carlsson and Nikitin, "Fast algorithms and efficient GPU implementations for the
 * Radon transform and the back-projection operator represented as convolution operators"
 * (arXiv 1506.00014), as convolutions in log-polar coordinates:
 *   R : Algorithm 1 (Section 6) -- pre-filter Q (Eq. Qfrecursive), resampling of T_m f onto the
 *       log-polar grid (Eq. Tdef, Eq. Lopolargrid_f, Eq. Lopolargrid_polar), FFT convolution with
 *       zeta / B-hat (Eq. exprcoef1, Eq. Bhat), resampling at S_m (Eq. Radon_all_pb, Eq. Sm_def).
 *   R#: Algorithm 2 (Section 6) -- the mirrored chain with zeta# (Eq. exprcoef2,
 *       Eq. backproj_lpp) and a sum over the M partitions.
 *
 * Conventions (all arrays are dense, row-major, FP32, in the caller's memory):
 *   image    f[i][j], i, j in [0, N): pixel centre x1 = (j - N/2) * 2/N, x2 = (i - N/2) * 2/N;
 *            the object is taken to vanish outside the open unit disc, so input pixels with
 *            |x| >= 1 are ignored and output pixels with |x| >= 1 are written as 0.
 *   sinogram g[a][k], a in [0, n_angles), k in [0, n_det): theta_a = a * pi / n_angles,
 *            s_k = (k - n_det/2) * ds, ds = 2 sqrt(2) / n_det; bins with |s_k| >= 1 are written
 *            as 0 by R and ignored by R#.
 *   R f(theta, s) = int f(x) delta(x . theta - s) dx               (Eq. radon_def)
 *   R# g(x)       = int_0^pi g(theta, x . theta) dtheta            (adjoint of R on [0, pi) x R)
 *
 * Calls are asynchronous and ordered on the CUDA stream passed as `stream` (a cudaStream_t,
 * NULL = legacy default stream).  Device pointers must come from cudaMalloc (or a caching
 * allocator over it) on the current device.  A plan owns its tables and its scratch memory:
 * it must not be used by two calls that can overlap on the GPU (one stream at a time).
 *
 * Every entry point returns a radon_status.  No call throws, exits or falls back to the CPU.
 */
#ifndef RADON_H_
#define RADON_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RADON_OK = 0,
  RADON_INVALID_ARG = 1,     /* bad size, NULL pointer, unknown option */
  RADON_OUT_OF_MEMORY = 2,   /* a device or host allocation failed */
  RADON_CUDA_ERROR = 3,      /* a CUDA runtime call or kernel launch failed */
  RADON_TIMEOUT = 4,         /* a bounded device-side wait gave up */
  RADON_NOT_SUPPORTED = 5,   /* valid request outside what this build handles */
  RADON_EXCEEDS_STATIC_SCRATCH = 6  /* radon_forward_static_scratch: plan too large for the static array */
} radon_status;

typedef enum {
  RADON_FILTER_RAMP = 0,         /* |sigma|                                   (Eq. ramp)   */
  RADON_FILTER_SHEPP_LOGAN = 1,  /* |sigma| sinc(sigma / (2 sigma_max))       (Eq. SLfilt) */
  RADON_FILTER_COSINE = 2        /* |sigma| cos(pi sigma / (2 sigma_max))     (Eq. cosfilt)*/
} radon_filter;

typedef struct radon_plan_s* radon_plan;

/* Derived discretisation (Sections 2 and 4); what the plan computes, for tests and oracles. */
typedef struct {
  int N, n_angles, n_det, interp_order, n_partitions;
  int N_rho;          /* rho samples: Eq. vrho bound rounded up to an even 7-smooth integer   */
  int n_theta_half;   /* angular samples per partition (centre half of the FFT grid)          */
  int n_theta;        /* angular FFT length, 2 * n_theta_half, period [-beta, beta)           */
  int r;              /* fine angular sub-samples per coarse angle (Omega_lp -> Omega_p)       */
  int n_quad;         /* trapezoid nodes used for the kernel integrals (Eq. weightsa)          */
  int n_filter;       /* zero-padded FFT length of the FBP filter along s (>= 2 n_det)          */
  int column_group;   /* theta convolution kernel: 0 specialised, else rho frequencies per CTA */
  double beta, a_R, a_r, L;       /* pi/M, Eq. aconst, L = -log(a_r)                           */
  double d_phi, d_rho, d_s, d_theta;
  size_t device_bytes;            /* device memory owned by the plan (tables + scratch)        */
} radon_plan_info;

/* Create a plan.  N even and >= 8; n_angles >= 2; n_det >= 4; interp_order 1 (linear) or 3
 * (cubic B-spline); n_partitions M >= 3.  Computes the geometry and the kernel transforms
 * zeta_hat / B_hat, zeta#_hat / B_hat in FP64 on the host (trapezoid rule with the end
 * corrections of Eq. weightsa), uploads them as FP32 and allocates the scratch buffers on the
 * current device.  Synchronous.  *out is set to NULL on failure.  Returns RADON_INVALID_ARG for
 * arguments outside these ranges and RADON_NOT_SUPPORTED for valid sizes this build cannot hold:
 * one rho row (N_rho / 2 complex values, about 1.07 N) or one theta column group must fit in a
 * CTA's shared memory, which limits N to about 8700 and n_angles to about 14000 with
 * M = 3. */
int radon_plan_create(radon_plan* out, int N, int n_angles, int n_det, int interp_order,
                      int n_partitions);

/* Release a plan (NULL is ignored).  Synchronises the device first. */
void radon_plan_destroy(radon_plan plan);

/* Fill *out with the plan's derived sizes. */
int radon_plan_get_info(radon_plan plan, radon_plan_info* out);

/* R: d_image [N][N] -> d_sino [n_angles][n_det] (overwritten).  Algorithm 1. */
int radon_forward(radon_plan plan, const float* d_image, float* d_sino, void* stream);

/* R#: d_sino [n_angles][n_det] -> d_image [N][N] (overwritten).  Algorithm 2. */
int radon_backproject(radon_plan plan, const float* d_sino, float* d_image, void* stream);

/* Filtered back-projection f = R# W g (Eq. FBP), with R# over [0, pi) so that f = R# W R f for
 * W = |sigma| (sigma in cycles per unit of s).  W acts on each sinogram row (bins with |s| >= 1
 * taken as zero) as a discrete convolution along s, evaluated with a zero-padded FFT of length
 * n_filter.  Its transfer function is ds times the DFT of the band-limited ramp kernel
 * h(0) = 1/(4 ds^2), h(n) = -1/(pi^2 n^2 ds^2) for odd n, 0 for even n != 0 (Eq. ramp, with the
 * low-frequency behaviour of the sampled kernel instead of a kink at sigma = 0), times the
 * window of `filter`: 1 (ramp), sinc(sigma / (2 sigma_max)) (Shepp-Logan, Eq. SLfilt) or
 * cos(pi sigma / (2 sigma_max)) (cosine, Eq. cosfilt), sigma_max = 1/(2 ds).  Then R# is applied.
 * d_sino is not modified; the filtered sinogram lives in plan-owned memory. */
int radon_fbp(radon_plan plan, const float* d_sino, float* d_image, int filter, void* stream);

/* R^T: the exact transpose of the discrete map radon_forward computes (Algorithm 1 with every
 * step transposed, in reverse order), d_sino [n_angles][n_det] -> d_image [N][N] (overwritten).
 * sum(R f * g) = sum(f * R^T g) up to FP32 rounding, for every f and g, so R^T gives exact
 * gradients of objectives built on radon_forward.  It is not R#: Algorithm 2 discretises the
 * continuous adjoint, which R^T approaches only as dx^2 / (d_theta d_s) R# on smooth g (with a
 * pixel-scale ripple from spreading over the log-polar samples).  Bins with |s| >= 1 are ignored;
 * pixels outside the unit disc are zero.  The log-polar and image scatters accumulate with FP32
 * atomics, so the low bits of the result may vary from run to run.  Uses the plan's scratch like
 * the other transforms; radon_transpose_batch takes `batch` <= max_batch slices back to back. */
int radon_transpose(radon_plan plan, const float* d_sino, float* d_image, void* stream);
int radon_transpose_batch(radon_plan plan, const float* d_sinos, float* d_images, int batch, void* stream);

/* Uneven batches (Section 7 batches slices of a volume to fill the GPU): `count` slices, slice i
 * transformed by plans[i] from d_images[i] to d_sinos[i] (radon_forward_multi) or from d_sinos[i]
 * to d_images[i] (radon_backproject_multi), launched in order on one stream.  Plans may differ in
 * size; a plan may appear several times (its scratch is reused in stream order, so one plan must
 * not also run on another stream meanwhile).  Every plan and pointer is checked before the first
 * launch: RADON_INVALID_ARG launches nothing.  A launch error returns its status after the slices
 * before it were launched.  The call can be captured in a CUDA graph like the per-slice calls. */
int radon_forward_multi(const radon_plan* plans, const float* const* d_images, float* const* d_sinos, int count,
                        void* stream);
int radon_backproject_multi(const radon_plan* plans, const float* const* d_sinos, float* const* d_images, int count,
                            void* stream);

/* Batches of same-size slices.  radon_plan_reserve_batch makes the plan able to process up to
 * max_batch slices in one call: it allocates scratch for them, synchronising the device (call it
 * before any stream capture), and returns RADON_OUT_OF_MEMORY, keeping the previous capacity, when
 * the device cannot hold them.  radon_forward_batch / radon_backproject_batch then transform
 * `batch` <= max_batch slices stored back to back ([batch][N][N] images, [batch][n_angles][n_det]
 * sinograms) with the same kernel launches as one slice (radon_plan_kernel_launches); results
 * equal those of per-slice calls. */
int radon_plan_reserve_batch(radon_plan plan, int max_batch);
int radon_forward_batch(radon_plan plan, const float* d_images, float* d_sinos, int batch, void* stream);
int radon_backproject_batch(radon_plan plan, const float* d_sinos, float* d_images, int batch, void* stream);

/* Kernel of the theta convolution (the column FFTs of Sections 3 and 5), a performance knob.
 * group 0: the specialised in-place kernel, available when n_theta is a power of two from 256
 * to 8192, or 1372 = 14 x 14 x 7 or 2744 = 14 x 14 x 14 (the default there; 1372 is the length
 * for 2048 angles and M = 3); group 1, 2 or 4: the generic mixed-radix kernel with that many rho
 * frequencies per CTA (the default otherwise).  Groups 1, 2 and 4 give identical results; group 0
 * differs from them by FP32 rounding only.  RADON_NOT_SUPPORTED if the kernel is unavailable or
 * does not fit. */
int radon_plan_set_column_group(radon_plan plan, int group);

/* Same as radon_forward / radon_backproject but with HOST buffers: the call copies the input to
 * plan-owned device memory, runs the transform on `stream` and copies the result back; it
 * returns after the result is in host memory.  Page-locked buffers give the fastest copies. */
int radon_forward_host(radon_plan plan, const float* h_image, float* h_sino, void* stream);
int radon_backproject_host(radon_plan plan, const float* h_sino, float* h_image, void* stream);

/* Host-only helpers (no GPU needed).
 * radon_geometry: the derived sizes a plan with these arguments would use (device_bytes = 0).
 * radon_kernel_quadrant: the FP64 kernel coefficients zeta_hat (which = 0) or zeta#_hat
 *   (which = 1) for k_theta in [0, n_theta/2] (slow index) and k_rho in [0, N_rho/2] (fast
 *   index), as interleaved (re, im) pairs; `out` holds 2 * (n_theta/2+1) * (N_rho/2+1) doubles.
 *   These are the raw integrals of Eq. exprcoef1 / exprcoef2, before any division. */
int radon_geometry(int N, int n_angles, int n_det, int interp_order, int n_partitions,
                   radon_plan_info* out);
int radon_kernel_quadrant(int N, int n_angles, int n_det, int n_partitions, int which,
                          double* out);

/* Per-stage timing (profiling aid).  While enabled, every transform records a CUDA event on its
 * stream after each of its kernel launches.  radon_profile_read waits for the recorded events,
 * adds each stage's elapsed milliseconds to ms[stage] and its launch count to launches[stage]
 * (arrays of RADON_NUM_STAGES entries, not cleared by the call), then forgets the events.
 * Stages: 0 image pre-filter, 1 forward rho FFT of the sampled rows, 2 forward theta
 * convolution, 3 forward inverse rho FFT, 4 sinogram gather, 5 sinogram pre-filter,
 * 6 back-projection row sampling + rho FFT, 7 back-projection theta convolution,
 * 8 back-projection inverse rho FFT, 9 image gather, 10 FBP filter along s, 11 forward row
 * sampling (log-polar resampling of the image); radon_transpose: 12 clearing of the scatter
 * targets and scatter of the sinogram onto the log-polar grid, 13 rho FFT, 14 transposed theta convolution, 15 inverse rho FFT,
 * 16 scatter onto the image coefficients, 17 Q^T and the disc mask. */
#define RADON_NUM_STAGES 18
int radon_profile_enable(radon_plan plan, int enable);
int radon_profile_read(radon_plan plan, double* ms, int* launches);

/* Number of kernels one call launches with the plan's current settings: op 0 radon_forward,
 * 1 radon_backproject, 2 radon_fbp, 3 radon_transpose (a stage may launch more than one kernel;
 * radon_transpose also clears its two scatter targets with cudaMemsetAsync).  Written to *out;
 * RADON_INVALID_ARG for another op. */
int radon_plan_kernel_launches(radon_plan plan, int op, int* out);

/* Forward transform R without any allocation, for callers that must not allocate device memory
 * when they run a transform: code that runs under a framework owning every device allocation
 * (where a raw cudaMalloc is forbidden or would fragment its pool), or a real-time loop with a
 * fixed device-memory budget.  The paper has no counterpart; this is a deployment variant of
 * radon_forward and gives the same result.
 *
 * The plan's precomputed tables are used as they are (they were allocated when the plan was
 * created), but the transform's intermediate arrays (coefficient image, spectra, log-polar
 * coefficients) live in one static device array of RADON_STATIC_SCRATCH_BYTES (16 MiB) that
 * every GPU which loads the library holds until the process exits.  That is enough for N = 512
 * with 512 angles and 768 bins; a plan whose intermediates do not fit is rejected with
 * RADON_EXCEEDS_STATIC_SCRATCH before anything is launched.
 *
 * The call allocates nothing: no cudaMalloc, no cudaFree, no allocating library routine.  Its
 * first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  The array is shared by all
 * calls on a device and keeps the last call's contents; each call clears what must start at zero.
 * Calls that can overlap on the GPU (different streams, or different host threads) race on the
 * array: order them on one stream or synchronise between them.  The looked-up address is kept for
 * the life of the process; a cudaDeviceReset on that device invalidates it, so do not call this
 * entry point on a device after resetting it. */
#define RADON_STATIC_SCRATCH_BYTES (16u << 20)
int radon_forward_static_scratch(radon_plan plan, const float* d_image, float* d_sino, void* stream);

/* Human-readable name of a status code (static string). */
const char* radon_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* RADON_H_ */
