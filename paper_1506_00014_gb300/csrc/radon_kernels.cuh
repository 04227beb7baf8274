// Device-side parameter blocks and launch entry points of the log-polar pipeline.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "radon_fft.cuh"

namespace radon {

// Pointers to the plan's FP32 tables and scratch (all device memory) plus the sizes the kernels
// need.  Filled once at plan creation; passed to kernels by value.
struct DevPlan {
  int N, n_angles, n_det, M, interp, N_rho, nh, n_theta, r, nc;
  int img_pitch;   // padded coefficient image: (N + 2 kPad) columns
  int sino_pitch;  // padded sinogram coefficients: n_det + 1 + 2 kPad columns
  int x_pitch;     // complex spectrum rows: >= N_rho/2 + 1
  int y_pitch;     // real log-polar rows with periodic wrap columns: >= N_rho + 2 kPad
  int n_eanc, n_ktiles, n_ptiles;
  int col_group;   // generic column kernel: rho frequencies per CTA (4, 2 or 1); 0: specialised kernel
  int col_fixed;   // kColumnRadices index of the specialised column kernel, -1 if none
  int col_blocks;  // persistent grid of the specialised column kernel (resident CTAs on the device)
  int col_blocks_t; // same for its transposed form (exact transpose); 0: generic theta pass
  int col_group_t; // rho frequencies per CTA of the transposed theta pass (0: does not fit)
  int live_lo, live_hi;  // detector bins with |s| < 1 are exactly [live_lo, live_hi]
  float inv_drho, inv_dphi, inv_aR, d_s;
  RadixList rad_rho, rad_th;
  // tables
  const float2* tw_rho;
  const float2* tw_r2c;
  const float2* tw_th;
  const float2* tw_col;  // per-pass twiddles of the specialised column transform
  const float2* k_fwd;
  const float2* k_bp;
  const float4* fwd_row;
  const float4* fwd_m;
  const float2* fwd_e;
  const float2* fwd_eanc;
  const int2* fwd_rng;
  const int4* fwd_ang;
  const int4* fwd_anc;
  const int2* bp_th;
  const int2* bp_c;
  const int2* bp_e;
  const int4* bp_anc;  // 2 int4 per (m, tile)
  const float2* bp_m;
  const float* filt;   // FBP transfer functions / n_filt: 3 tables of n_filt/2 + 1 real bins
  // scratch
  float* coef_img;     // (N + 2 kPad)^2, zero border
  float4* coef_q4;     // same grid; element (r, c) holds coefficients (r, c .. c+3) (zero past the edge)
  int img_quad;        // 1: forward sampling reads coef_q4 (one 16-byte load per tap row)
  int rows_tw_smem;    // 1: row kernels stage the rho twiddles in shared memory
  int rows_pipe_fwd;   // > 0: resident CTAs of the persistent forward rho transform (0: one CTA per row)
  int rows_pipe_inv;   // > 0: resident CTAs of the persistent inverse rho transform
  int rows_bp_blocks;  // > 0: resident CTAs of the persistent back-projection rows
  int row_fixed;       // kRowRadices index of the compiled row transform, -1: generic
  float* coef_sino;    // n_angles x sino_pitch, zero border
  float2* xspec;       // M x nh x x_pitch
  float2* yspec;       // M x (nh + 4) x x_pitch
  float* ylp;          // M x (nh + 4) x y_pitch
  float* sino_tmp;     // n_angles x n_det (filtered sinogram for FBP)
  // batches of same-size slices: slice b = blockIdx.z uses scratch at these strides (elements)
  size_t bs_img, bs_sino, bs_x, bs_ys, bs_y;
  int batch_cap;       // slices the scratch holds
  int n_filt;          // FBP: zero-padded real FFT length along s
  int filt_tw_smem;    // 1: the FBP row kernel stages its twiddles in shared memory
  RadixList rad_filt;
  const float2* tw_filt;
  const float2* tw_filt_r2c;
};

// Optional hook called after each kernel launch (stage ids as in radon.h) and once before the
// first one (stage -1); used for per-stage event timing.
struct StageHook {
  void (*mark)(void* ctx, int stage, cudaStream_t st);
  void* ctx;
  void operator()(int stage, cudaStream_t st) const {
    if (mark) mark(ctx, stage, st);
  }
};

// Each returns cudaGetLastError() after its launches.  `batch` same-size slices (contiguous
// [batch][...] inputs and outputs, batch <= p.batch_cap) are processed by the same launches.
cudaError_t launch_forward(const DevPlan& p, const float* image, float* sino, cudaStream_t st, StageHook hook,
                           int batch = 1);
cudaError_t launch_backproject(const DevPlan& p, const float* sino, float* image, cudaStream_t st, StageHook hook,
                               int batch = 1);
cudaError_t launch_fbp(const DevPlan& p, const float* sino, float* image, int filter, cudaStream_t st, StageHook hook);
// Exact transpose of launch_forward's map (stages 12-17).
cudaError_t launch_transpose(const DevPlan& p, const float* sino, float* image, cudaStream_t st, StageHook hook,
                             int batch = 1);

// Kernels launched by launch_forward (op 0), launch_backproject (1), launch_fbp (2) and
// launch_transpose (3).
int kernel_launches(const DevPlan& p, int op);

// Dynamic shared memory limits are raised once per device.
cudaError_t configure_kernels(DevPlan& p);

}  // namespace radon
