// CUDA kernels of the log-polar Radon transform (Algorithm 1) and back-projection (Algorithm 2).
//
// Pipeline of one transform (one launch each, all on the caller's stream):
//   prefilter  : B-spline coefficients Q f (Eq. Qfrecursive) as a truncated symmetric FIR
//                (the impulse response sqrt(3) z^|n| of the recursion), disc / |s| < 1 masks.
//   rows_fwd   : one CTA per angular row (m, j) of the log-polar grid: samples the row
//                (Algorithm 1: T_m f on Omega_lp, box-averaged to Omega_p, times e^rho;
//                 Algorithm 2: g(S_m) on Omega_p) into shared memory and applies the real FFT
//                along rho; writes the half spectrum.
//   columns    : one CTA per group of rho frequencies: FFT along theta (zero-padded centre
//                half), multiply by zeta_hat / B_hat (or zeta#_hat / B_hat), inverse FFT, keep
//                the centre half plus a 2-row halo.
//   rows_inv   : inverse real FFT along rho per kept row -> B-spline coefficients of the
//                partial transform on the log-polar grid (with periodic wrap columns).
//   gather     : forward -- resample at S_m(theta, s) onto the sinogram (Eq. Radon_all_pb);
//                back-projection -- resample at the log-polar coordinates of T_m x and sum m.
// Every gather clamps its tap indices into the buffer it reads.
#include <cuda_runtime.h>

#include <cstdint>

#include "plan_host.h"
#include "radon_kernels.cuh"

namespace radon {
namespace {

constexpr int kThreads = 256;
constexpr int kPfTile = 32;
constexpr int kPfWide = kPfTile + 2 * kFirHalf;

__device__ __forceinline__ int odd_ext(int p, int n, float* sgn) {
  // extension of [0, n) that is odd about -1 and about n (period 2n + 2)
  const int P = 2 * n + 2;
  int q = p % P;
  if (q < 0) q += P;
  if (q < n) {
    *sgn = 1.f;
    return q;
  }
  if (q == n || q == P - 1) {
    *sgn = 0.f;
    return 0;
  }
  *sgn = -1.f;
  return 2 * n - q;
}

__device__ __forceinline__ bool in_disc(int i, int j, int N) {
  const long long di = 2LL * i - N, dj = 2LL * j - N;
  return di * di + dj * dj < static_cast<long long>(N) * N;
}

__device__ __forceinline__ bool live_bin(int k, int nd) {
  const long long v = 2LL * k - nd;
  return 2 * v * v < static_cast<long long>(nd) * nd;
}

// Cubic B-spline weights of taps k-1, k, k+1, k+2 at fractional offset a (Eq. wsumn).
__device__ __forceinline__ void bspline_w(float a, float (&w)[4]) {
  const float om = 1.f - a;
  const float a2 = a * a;
  const float s6 = 1.f / 6.f;
  w[0] = om * om * om * s6;
  w[1] = fmaf(a2, fmaf(3.f, a, -6.f), 4.f) * s6;
  w[2] = fmaf(a, fmaf(a, fmaf(-3.f, a, 3.f), 3.f), 1.f) * s6;
  w[3] = a2 * a * s6;
}

// (ah + al) * (bh + bl) + (ch + cl) in double-float arithmetic.
__device__ __forceinline__ void df_mul_add(float ah, float al, float bh, float bl, float ch, float cl, float* rh,
                                           float* rl) {
  const float pr = ah * bh;
  float e = fmaf(ah, bh, -pr);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float s = pr + ch;
  const float bb = s - pr;
  const float err = (pr - (s - bb)) + (ch - bb);
  *rh = s;
  *rl = err + e + cl;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ------------------------------------------------------------------------------------------
// Pre-filter of the image: mask to the unit disc, separable truncated FIR with the odd
// (zero-boundary) extension.  interp == 1: masked copy.
__global__ void __launch_bounds__(kThreads) k_prefilter_image(DevPlan p, const float* __restrict__ f) {
  __shared__ float s_in[kPfWide][kPfWide + 1];
  __shared__ float s_mid[kPfWide][kPfTile + 1];
  const int N = p.N;
  const int tx0 = blockIdx.x * kPfTile, ty0 = blockIdx.y * kPfTile;
  const int tid = threadIdx.x;
  float q[kFirHalf + 1];
#pragma unroll
  for (int n = 0; n <= kFirHalf; ++n) q[n] = __ldg(p.fir + n);
  for (int idx = tid; idx < kPfWide * kPfWide; idx += kThreads) {
    const int ly = idx / kPfWide, lx = idx - (idx / kPfWide) * kPfWide;
    float sy, sx;
    const int gy = odd_ext(ty0 + ly - kFirHalf, N, &sy);
    const int gx = odd_ext(tx0 + lx - kFirHalf, N, &sx);
    float v = 0.f;
    const float sg = sy * sx;
    if (sg != 0.f && in_disc(gy, gx, N)) v = sg * __ldg(f + static_cast<size_t>(gy) * N + gx);
    s_in[ly][lx] = v;
  }
  __syncthreads();
  if (p.interp == 1) {
    for (int idx = tid; idx < kPfTile * kPfTile; idx += kThreads) {
      const int ly = idx / kPfTile, lx = idx % kPfTile;
      const int gy = ty0 + ly, gx = tx0 + lx;
      if (gy < N && gx < N)
        p.coef_img[static_cast<size_t>(gy + kPad) * p.img_pitch + gx + kPad] = s_in[ly + kFirHalf][lx + kFirHalf];
    }
    return;
  }
  for (int idx = tid; idx < kPfWide * kPfTile; idx += kThreads) {
    const int ly = idx / kPfTile, lx = idx % kPfTile;
    const float* row = &s_in[ly][lx + kFirHalf];
    float acc = q[0] * row[0];
#pragma unroll
    for (int n = 1; n <= kFirHalf; ++n) acc = fmaf(q[n], row[-n] + row[n], acc);
    s_mid[ly][lx] = acc;
  }
  __syncthreads();
  for (int idx = tid; idx < kPfTile * kPfTile; idx += kThreads) {
    const int ly = idx / kPfTile, lx = idx % kPfTile;
    const int gy = ty0 + ly, gx = tx0 + lx;
    if (gy >= N || gx >= N) continue;
    float acc = q[0] * s_mid[ly + kFirHalf][lx];
#pragma unroll
    for (int n = 1; n <= kFirHalf; ++n)
      acc = fmaf(q[n], s_mid[ly + kFirHalf - n][lx] + s_mid[ly + kFirHalf + n][lx], acc);
    p.coef_img[static_cast<size_t>(gy + kPad) * p.img_pitch + gx + kPad] = acc;
  }
}

// Pre-filter of the sinogram on the (2 n_angles) x (n_det + 1) extension: theta periodic with
// g(theta + pi, s) = g(theta, -s) (bin k <-> n_det - k), s with the zero boundary; bins with
// |s| >= 1 are zero.  Writes the first n_angles rows (the rest follow by the flip).
__global__ void __launch_bounds__(kThreads) k_prefilter_sino(DevPlan p, const float* __restrict__ g) {
  __shared__ float s_in[kPfWide][kPfWide + 1];
  __shared__ float s_mid[kPfWide][kPfTile + 1];
  const int na = p.n_angles, nd = p.n_det, ne = nd + 1;
  const int tx0 = blockIdx.x * kPfTile, ty0 = blockIdx.y * kPfTile;
  const int tid = threadIdx.x;
  float q[kFirHalf + 1];
#pragma unroll
  for (int n = 0; n <= kFirHalf; ++n) q[n] = __ldg(p.fir + n);
  for (int idx = tid; idx < kPfWide * kPfWide; idx += kThreads) {
    const int ly = idx / kPfWide, lx = idx - (idx / kPfWide) * kPfWide;
    int a2 = (ty0 + ly - kFirHalf) % (2 * na);
    if (a2 < 0) a2 += 2 * na;
    const bool flip = a2 >= na;
    const int arow = flip ? a2 - na : a2;
    float sc;
    const int qc = odd_ext(tx0 + lx - kFirHalf, ne, &sc);
    const int c = flip ? nd - qc : qc;
    float v = 0.f;
    if (sc != 0.f && c < nd && live_bin(c, nd)) v = sc * __ldg(g + static_cast<size_t>(arow) * nd + c);
    s_in[ly][lx] = v;
  }
  __syncthreads();
  if (p.interp == 1) {
    for (int idx = tid; idx < kPfTile * kPfTile; idx += kThreads) {
      const int ly = idx / kPfTile, lx = idx % kPfTile;
      const int a = ty0 + ly, c = tx0 + lx;
      if (a < na && c < ne)
        p.coef_sino[static_cast<size_t>(a) * p.sino_pitch + c + kPad] = s_in[ly + kFirHalf][lx + kFirHalf];
    }
    return;
  }
  for (int idx = tid; idx < kPfWide * kPfTile; idx += kThreads) {
    const int ly = idx / kPfTile, lx = idx % kPfTile;
    const float* row = &s_in[ly][lx + kFirHalf];
    float acc = q[0] * row[0];
#pragma unroll
    for (int n = 1; n <= kFirHalf; ++n) acc = fmaf(q[n], row[-n] + row[n], acc);
    s_mid[ly][lx] = acc;
  }
  __syncthreads();
  for (int idx = tid; idx < kPfTile * kPfTile; idx += kThreads) {
    const int ly = idx / kPfTile, lx = idx % kPfTile;
    const int a = ty0 + ly, c = tx0 + lx;
    if (a >= na || c >= ne) continue;
    float acc = q[0] * s_mid[ly + kFirHalf][lx];
#pragma unroll
    for (int n = 1; n <= kFirHalf; ++n)
      acc = fmaf(q[n], s_mid[ly + kFirHalf - n][lx] + s_mid[ly + kFirHalf + n][lx], acc);
    p.coef_sino[static_cast<size_t>(a) * p.sino_pitch + c + kPad] = acc;
  }
}

// ------------------------------------------------------------------------------------------
// Row sampling.

// Value of the image interpolant at padded index coordinates (ic + ac, ir + ar).
__device__ __forceinline__ float sample_image(const DevPlan& p, int ic, float ac, int ir, float ar) {
  const float* __restrict__ c = p.coef_img;
  const int pitch = p.img_pitch;
  if (p.interp == 3) {
    if (ic < 1 || ic > pitch - 3 || ir < 1 || ir > pitch - 3) return 0.f;
    float wc[4], wr[4];
    bspline_w(ac, wc);
    bspline_w(ar, wr);
    const float* base = c + static_cast<size_t>(ir - 1) * pitch + (ic - 1);
    float acc = 0.f;
#pragma unroll
    for (int dr = 0; dr < 4; ++dr) {
      const float* row = base + dr * pitch;
      const float v = fmaf(wc[0], __ldg(row), fmaf(wc[1], __ldg(row + 1), fmaf(wc[2], __ldg(row + 2), wc[3] * __ldg(row + 3))));
      acc = fmaf(wr[dr], v, acc);
    }
    return acc;
  }
  if (ic < 0 || ic > pitch - 2 || ir < 0 || ir > pitch - 2) return 0.f;
  const float* base = c + static_cast<size_t>(ir) * pitch + ic;
  const float v0 = fmaf(ac, __ldg(base + 1) - __ldg(base), __ldg(base));
  const float v1 = fmaf(ac, __ldg(base + pitch + 1) - __ldg(base + pitch), __ldg(base + pitch));
  return fmaf(ar, v1 - v0, v0);
}

// Forward: h(phi_j, rho_i) = e^rho_i / r * sum_q f~(T_m^{-1}(e^rho_i (cos phi_jq, sin phi_jq))).
// Coordinates: a double-float anchor per 32-sample rho tile plus an FP32 offset.
__device__ void sample_row_forward(const DevPlan& p, int m, int jj, float* __restrict__ h) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float4 um = p.fwd_m[m];
  const float4* rowc = p.fwd_row + (static_cast<size_t>(m) * p.nh + jj) * p.r;
  for (int tile = warp; tile < p.n_eanc; tile += nw) {
    const int i = tile * kETile + lane;
    const bool valid = i < p.N_rho;
    const float2 e = valid ? p.fwd_e[i] : make_float2(0.f, 0.f);
    const float2 ea = p.fwd_eanc[tile];
    float acc = 0.f;
    for (int q = 0; q < p.r; ++q) {
      const float4 cs = rowc[q];
      float ch, cl, rh, rl;
      df_mul_add(ea.x, ea.y, cs.x, cs.y, um.x, um.y, &ch, &cl);
      df_mul_add(ea.x, ea.y, cs.z, cs.w, um.z, um.w, &rh, &rl);
      const float Ic = floorf(ch), Ir = floorf(rh);
      const float Fc = fmaf(e.y, cs.x, (ch - Ic) + cl);
      const float Fr = fmaf(e.y, cs.z, (rh - Ir) + rl);
      const float fc = floorf(Fc), fr = floorf(Fr);
      acc += sample_image(p, static_cast<int>(Ic) + static_cast<int>(fc), Fc - fc, static_cast<int>(Ir) + static_cast<int>(fr),
                          Fr - fr);
    }
    if (valid) h[i] = acc * e.x;
  }
}

// Value of the sinogram interpolant at (theta index It + at, padded s index is + as).
__device__ __forceinline__ float sample_sino(const DevPlan& p, int It, float at, int is, float as) {
  const int na = p.n_angles, pitch = p.sino_pitch;
  const int ntap = p.interp == 3 ? 4 : 2;
  float wt[4], ws[4];
  if (p.interp == 3) {
    bspline_w(at, wt);
    bspline_w(as, ws);
    It -= 1;
    is -= 1;
  } else {
    wt[0] = 1.f - at;
    wt[1] = at;
    ws[0] = 1.f - as;
    ws[1] = as;
  }
  float acc = 0.f;
  for (int dt = 0; dt < ntap; ++dt) {
    int a2 = (It + dt) % (2 * na);
    if (a2 < 0) a2 += 2 * na;
    const bool flip = a2 >= na;
    const float* row = p.coef_sino + static_cast<size_t>(flip ? a2 - na : a2) * pitch;
    float v = 0.f;
    for (int ds = 0; ds < ntap; ++ds) {
      int c = is + ds;
      if (flip) c = p.n_det + 2 * kPad - c;
      c = clampi(c, 0, pitch - 1);
      v = fmaf(ws[ds], __ldg(row + c), v);
    }
    acc = fmaf(wt[dt], v, acc);
  }
  return acc;
}

// Back-projection: G(phi_j, rho_i) = g~(phi_j + m beta, (e^rho_i - (1 - a_R) cos phi_j) / a_R).
__device__ void sample_row_backproject(const DevPlan& p, int m, int jj, float* __restrict__ h) {
  const int2 th = p.bp_th[m * p.nh + jj];
  const int2 cj = p.bp_c[jj];
  const float Ft = __int_as_float(th.y), Fc = __int_as_float(cj.y);
  for (int i = threadIdx.x; i < p.N_rho; i += blockDim.x) {
    const int2 ei = p.bp_e[i];
    const float F = __int_as_float(ei.y) + Fc;
    const float fl = floorf(F);
    h[i] = sample_sino(p, th.x, Ft, ei.x + cj.x + static_cast<int>(fl), F - fl);
  }
}

// Sample one angular row, real FFT along rho, write the half spectrum (N_rho/2 + 1 bins).
template <bool BACK>
__global__ void __launch_bounds__(kThreads) k_rows_fwd(DevPlan p) {
  extern __shared__ float2 smem[];
  const int nc = p.nc;
  float2* bufA = smem;
  float2* bufB = smem + nc;
  const int jj = blockIdx.x, m = blockIdx.y;
  if (BACK)
    sample_row_backproject(p, m, jj, reinterpret_cast<float*>(bufA));
  else
    sample_row_forward(p, m, jj, reinterpret_cast<float*>(bufA));
  __syncthreads();
  const float2* Z = fft_block<false>(bufA, bufB, 1, nc, p.rad_rho, p.tw_rho, threadIdx.x, blockDim.x);
  float2* out = p.xspec + (static_cast<size_t>(m) * p.nh + jj) * p.x_pitch;
  for (int k = threadIdx.x; k <= nc; k += blockDim.x) {
    const float2 zk = Z[k == nc ? 0 : k];
    const float2 zc = cconj(Z[k == 0 ? 0 : nc - k]);
    const float2 ev = cscale(cadd(zk, zc), 0.5f);
    const float2 dv = cscale(csub(zk, zc), 0.5f);
    const float2 od = make_float2(dv.y, -dv.x);  // -i (Z_k - conj Z_{n-k}) / 2
    out[k] = cadd(ev, cmul(p.tw_r2c[k], od));
  }
}

// FFT along theta of col_group rho frequencies, multiply by the kernel, inverse FFT, keep the
// centre half plus the halo rows.
__global__ void __launch_bounds__(kThreads) k_columns(DevPlan p, const float2* __restrict__ kern) {
  extern __shared__ float2 smem[];
  const int nt = p.n_theta, nh = p.nh, nc = p.nc;
  const int G = p.col_group;
  float2* A = smem;
  float2* B = smem + G * nt;
  const int m = blockIdx.y, kr0 = blockIdx.x * G;
  const float2* xin = p.xspec + static_cast<size_t>(m) * nh * p.x_pitch;
  for (int idx = threadIdx.x; idx < G * nt; idx += blockDim.x) {
    const int g = idx % G, j = idx / G;
    const int jj = j - nh / 2;
    float2 v = make_float2(0.f, 0.f);
    if (jj >= 0 && jj < nh && kr0 + g <= nc) v = xin[static_cast<size_t>(jj) * p.x_pitch + kr0 + g];
    A[g * nt + j] = v;
  }
  __syncthreads();
  float2* S = fft_block<false>(A, B, G, nt, p.rad_th, p.tw_th, threadIdx.x, blockDim.x);
  float2* T = (S == A) ? B : A;
  const int nkt = nt / 2 + 1;
  for (int idx = threadIdx.x; idx < G * nt; idx += blockDim.x) {
    const int g = idx / nt, pp = idx - g * nt;
    const int kr = kr0 + g;
    if (kr <= nc) {
      const int kt = pp <= nt - pp ? pp : nt - pp;
      S[idx] = cmul(S[idx], kern[static_cast<size_t>(kr) * nkt + kt]);
    }
  }
  __syncthreads();
  const float2* Y = fft_block<true>(S, T, G, nt, p.rad_th, p.tw_th, threadIdx.x, blockDim.x);
  float2* yout = p.yspec + static_cast<size_t>(m) * (nh + kHaloLo + kHaloHi) * p.x_pitch;
  const int nrow = nh + kHaloLo + kHaloHi;
  for (int idx = threadIdx.x; idx < G * nrow; idx += blockDim.x) {
    const int g = idx % G, jr = idx / G;
    const int js = (jr + nh / 2 - kHaloLo + nt) % nt;  // the convolution output is nt-periodic
    if (kr0 + g <= nc) yout[static_cast<size_t>(jr) * p.x_pitch + kr0 + g] = Y[g * nt + js];
  }
}

// Inverse real FFT along rho of one kept row; writes N_rho values plus kPad wrap columns per side.
__global__ void __launch_bounds__(kThreads) k_rows_inv(DevPlan p) {
  extern __shared__ float2 smem[];
  const int nc = p.nc, nr = p.N_rho;
  float2* bufA = smem;
  float2* bufB = smem + nc;
  const int row = blockIdx.x, m = blockIdx.y;
  const int nrow = p.nh + kHaloLo + kHaloHi;
  const float2* X = p.yspec + (static_cast<size_t>(m) * nrow + row) * p.x_pitch;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const float2 xk = X[k];
    const float2 xc = cconj(X[nc - k]);
    const float2 sm = cadd(xk, xc);
    const float2 df = cmulc(csub(xk, xc), p.tw_r2c[k]);  // (X_k - conj X_{n-k}) exp(+2 pi i k / N_rho)
    bufA[k] = make_float2(sm.x - df.y, sm.y + df.x);      // + i * df
  }
  __syncthreads();
  const float2* Z = fft_block<true>(bufA, bufB, 1, nc, p.rad_rho, p.tw_rho, threadIdx.x, blockDim.x);
  const float* h = reinterpret_cast<const float*>(Z);
  float* y = p.ylp + (static_cast<size_t>(m) * nrow + row) * p.y_pitch;
  for (int c = static_cast<int>(threadIdx.x) - kPad; c < nr + kPad; c += blockDim.x) {
    int src = c < 0 ? c + nr : (c >= nr ? c - nr : c);
    y[c + kPad] = h[src];
  }
}

// ------------------------------------------------------------------------------------------
// Output gathers.

// Interpolant of partition m's log-polar coefficients at (halo row It + at, padded column
// Ir + ar); taps are clamped into the array.
__device__ __forceinline__ float sample_lp(const DevPlan& p, int m, int It, float at, int Ir, float ar) {
  const int nrow = p.nh + kHaloLo + kHaloHi;
  const float* __restrict__ y = p.ylp + static_cast<size_t>(m) * nrow * p.y_pitch;
  if (p.interp == 3) {
    float wt[4], wr[4];
    bspline_w(at, wt);
    bspline_w(ar, wr);
    const int r0 = clampi(It - 1, 0, nrow - 4);
    const int c0 = clampi(Ir - 1, 0, p.y_pitch - 4);
    const float* base = y + static_cast<size_t>(r0) * p.y_pitch + c0;
    float acc = 0.f;
#pragma unroll
    for (int dt = 0; dt < 4; ++dt) {
      const float* row = base + dt * p.y_pitch;
      const float v = fmaf(wr[0], __ldg(row), fmaf(wr[1], __ldg(row + 1), fmaf(wr[2], __ldg(row + 2), wr[3] * __ldg(row + 3))));
      acc = fmaf(wt[dt], v, acc);
    }
    return acc;
  }
  const int r0 = clampi(It, 0, nrow - 2);
  const int c0 = clampi(Ir, 0, p.y_pitch - 2);
  const float* base = y + static_cast<size_t>(r0) * p.y_pitch + c0;
  const float v0 = fmaf(ar, __ldg(base + 1) - __ldg(base), __ldg(base));
  const float v1 = fmaf(ar, __ldg(base + p.y_pitch + 1) - __ldg(base + p.y_pitch), __ldg(base + p.y_pitch));
  return fmaf(at, v1 - v0, v0);
}

// R f(theta_a, s_k) = a_R^{-1} * interpolant of partition m at S_m(theta_a, s_k).
__global__ void __launch_bounds__(128) k_gather_sino(DevPlan p, float* __restrict__ sino) {
  const int a = blockIdx.y;
  const int k = blockIdx.x * 128 + threadIdx.x;
  const int nd = p.n_det;
  if (k >= nd) return;
  float out = 0.f;
  if (live_bin(k, nd)) {
    const int4 ang = p.fwd_ang[a];
    const int4 anc = p.fwd_anc[static_cast<size_t>(a) * p.n_ktiles + k / kKTile];
    const int n = k - (k / kKTile) * kKTile;
    const float cr = fmaf(log1pf(static_cast<float>(n) * __int_as_float(anc.z)), p.inv_drho, __int_as_float(anc.y));
    const float fr = floorf(cr);
    out = sample_lp(p, ang.x, ang.z, __int_as_float(ang.w), anc.x + static_cast<int>(fr), cr - fr) * p.inv_aR;
  }
  sino[static_cast<size_t>(a) * nd + k] = out;
}

// R# g(x) = sum_m interpolant of partition m at the log-polar coordinates of T_m x.
__global__ void __launch_bounds__(kPTile * kPTile) k_gather_image(DevPlan p, float* __restrict__ img) {
  const int N = p.N;
  const int tj = blockIdx.x, ti = blockIdx.y;
  const int j = tj * kPTile + threadIdx.x, i = ti * kPTile + threadIdx.y;
  if (i >= N || j >= N) return;
  float acc = 0.f;
  if (in_disc(i, j, N)) {
    const float sc = 2.f / N;
    const float dx1 = static_cast<float>(static_cast<int>(threadIdx.x) - kPTile / 2) * sc;
    const float dx2 = static_cast<float>(static_cast<int>(threadIdx.y) - kPTile / 2) * sc;
    for (int m = 0; m < p.M; ++m) {
      const int4* anc = p.bp_anc + 2 * ((static_cast<size_t>(m) * p.n_ptiles + ti) * p.n_ptiles + tj);
      const int4 a0 = anc[0], a1 = anc[1];
      const float2 bm = p.bp_m[m];
      const float y0x = __int_as_float(a1.x), y0y = __int_as_float(a1.y);
      const float dy1 = fmaf(bm.x, dx1, bm.y * dx2);
      const float dy2 = fmaf(-bm.y, dx1, bm.x * dx2);
      const float cross = fmaf(y0x, dy2, -y0y * dy1);
      const float r2 = fmaf(y0x, y0x, y0y * y0y);
      const float ydot = fmaf(y0x, dy1, y0y * dy2);
      const float dth = atan2f(cross, r2 + ydot);
      const float drho = 0.5f * log1pf(fmaf(2.f, ydot, fmaf(dy1, dy1, dy2 * dy2)) / r2);
      const float ct = fmaf(dth, p.inv_dphi, __int_as_float(a0.y));
      const float cr = fmaf(drho, p.inv_drho, __int_as_float(a0.w));
      const float ft = floorf(ct), fr = floorf(cr);
      acc += sample_lp(p, m, a0.x + static_cast<int>(ft), ct - ft, a0.z + static_cast<int>(fr), cr - fr);
    }
  }
  img[static_cast<size_t>(i) * N + j] = acc;
}

size_t rows_smem(const DevPlan& p) { return 2 * static_cast<size_t>(p.nc) * sizeof(float2); }
size_t cols_smem(const DevPlan& p) { return 2 * static_cast<size_t>(p.col_group) * p.n_theta * sizeof(float2); }

void launch_columns_and_inverse(const DevPlan& p, const float2* kern, cudaStream_t st, const StageHook& hook,
                                int stage0) {
  const int ngroups = (p.nc + 1 + p.col_group - 1) / p.col_group;
  k_columns<<<dim3(ngroups, p.M), kThreads, cols_smem(p), st>>>(p, kern);
  hook(stage0, st);
  k_rows_inv<<<dim3(p.nh + kHaloLo + kHaloHi, p.M), kThreads, rows_smem(p), st>>>(p);
  hook(stage0 + 1, st);
}

}  // namespace

cudaError_t configure_kernels(const DevPlan& p) {
  // The limit is a per-function attribute shared by every plan on the device: raise it to the
  // device's opt-in maximum (never to one plan's need, which a later, smaller plan would lower).
  cudaError_t e;
  int dev = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  if (rows_smem(p) > static_cast<size_t>(optin) || cols_smem(p) > static_cast<size_t>(optin)) return cudaErrorInvalidValue;
  const int rs = optin, cs = optin;
  if ((e = cudaFuncSetAttribute(k_rows_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_rows_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_rows_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_columns, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_forward(const DevPlan& p, const float* image, float* sino, cudaStream_t st, StageHook hook) {
  const int tiles = (p.N + kPfTile - 1) / kPfTile;
  hook(-1, st);
  k_prefilter_image<<<dim3(tiles, tiles), kThreads, 0, st>>>(p, image);
  hook(0, st);
  k_rows_fwd<false><<<dim3(p.nh, p.M), kThreads, rows_smem(p), st>>>(p);
  hook(1, st);
  launch_columns_and_inverse(p, p.k_fwd, st, hook, 2);
  k_gather_sino<<<dim3((p.n_det + 127) / 128, p.n_angles), 128, 0, st>>>(p, sino);
  hook(4, st);
  return cudaGetLastError();
}

cudaError_t launch_backproject(const DevPlan& p, const float* sino, float* image, cudaStream_t st, StageHook hook) {
  hook(-1, st);
  k_prefilter_sino<<<dim3((p.n_det + 1 + kPfTile - 1) / kPfTile, (p.n_angles + kPfTile - 1) / kPfTile), kThreads, 0, st>>>(
      p, sino);
  hook(5, st);
  k_rows_fwd<true><<<dim3(p.nh, p.M), kThreads, rows_smem(p), st>>>(p);
  hook(6, st);
  launch_columns_and_inverse(p, p.k_bp, st, hook, 7);
  k_gather_image<<<dim3(p.n_ptiles, p.n_ptiles), dim3(kPTile, kPTile), 0, st>>>(p, image);
  hook(9, st);
  return cudaGetLastError();
}

cudaError_t launch_sino_filter(const DevPlan&, const float*, float*, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace radon
