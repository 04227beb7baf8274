// CUDA kernels of the log-polar Radon transform (Algorithm 1) and back-projection (Algorithm 2).
//
// Pipeline of one transform (one launch each, all on the caller's stream):
//   prefilter  : B-spline coefficients Q f (Eq. Qfrecursive): the recursion run inside each
//                thread's window of samples (response sqrt(3) z^|n| cut at |n| <= kFirHalf),
//                disc / |s| < 1 masks; for cubic images the quad-row layout.
//   sample_fwd : Algorithm 1's resampling of T_m f on Omega_lp, box-averaged to Omega_p, times
//                e^rho, into the spectrum scratch.
//   rows_fwd   : one CTA per angular row (m, j) of the log-polar grid: the sampled row (or, for
//                Algorithm 2, g(S_m) on Omega_p sampled in place) and its real FFT along rho;
//                writes the half spectrum.
//   columns    : one CTA per group of rho frequencies: FFT along theta (zero-padded centre
//                half), multiply by zeta_hat / B_hat (or zeta#_hat / B_hat), inverse FFT, keep
//                the centre half plus a 2-row halo.
//   rows_inv   : inverse real FFT along rho per kept row -> B-spline coefficients of the
//                partial transform on the log-polar grid (with periodic wrap columns).
//   gather     : forward -- resample at S_m(theta, s) onto the sinogram (Eq. Radon_all_pb);
//                back-projection -- resample at the log-polar coordinates of T_m x and sum m.
// Every gather clamps its tap indices into the buffer it reads.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "plan_host.h"
#include "radon_kernels.cuh"

namespace radon {
namespace {

constexpr int kThreads = 256;

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

// atan(y/x) for x > 0 and |y/x| < 0.1 by its Maclaurin series x - x^3/3 + x^5/5 (remainder
// below |y/x|^7 / 7 < 1.5e-8); other arguments use atan2f.
__device__ __forceinline__ float small_atan2(float y, float x) {
  const float t = __fdividef(y, x);  // |t| < 0.1 on the fast path: a few ulp of a small angle
  if (!(x > 0.f) || fabsf(t) >= 0.1f) return atan2f(y, x);
  const float t2 = t * t;
  return t * fmaf(t2, fmaf(t2, 0.2f, -1.f / 3.f), 1.f);
}

// log(1 + u) for |u| < 0.1 by its Maclaurin series up to u^7 (remainder below |u|^8 / 8 <
// 1.3e-9); other arguments use log1pf.
__device__ __forceinline__ float small_log1p(float u) {
  if (fabsf(u) >= 0.1f) return log1pf(u);
  const float p = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, 1.f / 7.f, -1.f / 6.f), 0.2f), -0.25f), 1.f / 3.f), -0.5f), 1.f);
  return u * p;
}

// ------------------------------------------------------------------------------------------
// Pre-filters.  One CTA computes a kPfRows x kPfCols tile of coefficients from the tile plus a
// kFirHalf halo, staged in shared memory; the filter runs along rows and then along columns,
// each thread producing kPfSeg consecutive outputs from a register window.  Tiles whose halo stays
// inside the array read it directly; border tiles map every index through the extension.

constexpr int kPfRows = 32, kPfCols = 64, kPfSeg = 8;
// the row pass (kPfRows + 2 kFirHalf rows) takes longer segments: fewer warm-up steps per output
constexpr int kPfSegRow = 16;
constexpr int kPfInR = kPfRows + 2 * kFirHalf, kPfInC = kPfCols + 2 * kFirHalf;

// Sources of the pre-filter.  Each gives the tile input (direct / extended reads), says when a
// window is all zero (dead), where its output columns start (kOutPad) and which outputs are kept
// (keep; the rest are written as zero).

// Masked image; extension odd about -1 and N in both axes (zero boundary, Eq. Qfrecursive).
struct ImageSource {
  static constexpr int kOutPad = kPad;  // output: padded coefficient image
  const float* __restrict__ f;
  int N;
  __device__ __forceinline__ bool keep(int, int) const { return true; }
  __device__ __forceinline__ void slice(int b) { f += static_cast<size_t>(b) * N * N; }
  __device__ __forceinline__ bool interior(int r0, int r1, int c0, int c1) const {
    return r0 >= 0 && r1 <= N && c0 >= 0 && c1 <= N;
  }
  __device__ __forceinline__ float direct(int r, int c) const {
    const int dr = 2 * r - N, dc = 2 * c - N;  // |x| < 1  <=>  dr^2 + dc^2 < N^2 (N <= 32768)
    const unsigned d2 = static_cast<unsigned>(dr * dr) + static_cast<unsigned>(dc * dc);
    return d2 < static_cast<unsigned>(N) * static_cast<unsigned>(N) ? __ldg(f + static_cast<size_t>(r) * N + c) : 0.f;
  }
  // True when every input of the window [r0, r1) x [c0, c1) is zero: the window lies inside the
  // array (no boundary extension) and its pixel nearest the centre is outside the disc (convex).
  __device__ __forceinline__ bool dead(int r0, int r1, int c0, int c1) const {
    if (!interior(r0, r1, c0, c1)) return false;
    const int r = min(max(N / 2, r0), r1 - 1), c = min(max(N / 2, c0), c1 - 1);
    const int dr = 2 * r - N, dc = 2 * c - N;
    return static_cast<unsigned>(dr * dr) + static_cast<unsigned>(dc * dc) >= static_cast<unsigned>(N) * static_cast<unsigned>(N);
  }
  __device__ __forceinline__ float extended(int r, int c) const {
    float sr, sc;
    const int rr = odd_ext(r, N, &sr);
    const int cc = odd_ext(c, N, &sc);
    const float sg = sr * sc;
    return sg != 0.f ? sg * direct(rr, cc) : 0.f;
  }
};

// Sinogram rows a (theta periodic over 2 n_angles, rows >= n_angles flipped k -> n_det - k) and
// columns k in [0, n_det] (the extra k = n_det is zero); zero boundary in k; dead bins zero.
struct SinoSource {
  static constexpr int kOutPad = kPad;  // output: padded sinogram coefficients
  const float* __restrict__ g;
  int na, nd, live_lo, live_hi;
  __device__ __forceinline__ bool keep(int, int) const { return true; }
  __device__ __forceinline__ void slice(int b) { g += static_cast<size_t>(b) * na * nd; }
  __device__ __forceinline__ bool interior(int r0, int r1, int c0, int c1) const {
    return r0 >= 0 && r1 <= na && c0 >= 0 && c1 <= nd + 1;
  }
  __device__ __forceinline__ float direct(int a, int k) const {
    return (k >= live_lo && k <= live_hi) ? __ldg(g + static_cast<size_t>(a) * nd + k) : 0.f;
  }
  // True when every input of the window is zero: its bins lie inside [0, n_det] (no s extension)
  // and miss the live range; theta rows (periodic, flipped k -> n_det - k) keep the live set.
  __device__ __forceinline__ bool dead(int, int, int c0, int c1) const {
    return c0 >= 0 && c1 <= nd + 1 && (c1 <= live_lo || c0 > live_hi);
  }
  __device__ __forceinline__ float extended(int r, int c) const {
    int a2 = r % (2 * na);
    if (a2 < 0) a2 += 2 * na;
    const bool flip = a2 >= na;
    float sc;
    const int q = odd_ext(c, nd + 1, &sc);
    if (sc == 0.f) return 0.f;
    const int k = flip ? nd - q : q;
    return sc * direct(flip ? a2 - na : a2, k);
  }
};

// Q^T for the exact transpose: the padded coefficient grid (N x N inside a kPad border), with
// the same odd extension as ImageSource.  The zero-boundary Q is a symmetric matrix (the
// filter's taps are even and the odd reflections about -1 and N enter as h(i + j + 2) and
// h(2N - i - j)), so Q^T is Q; the output is the unpadded image, zero outside the disc (the
// transpose of the input mask).
struct CoefSource {
  static constexpr int kOutPad = 0;
  const float* __restrict__ c;
  int N, pitch;
  size_t bstride;
  __device__ __forceinline__ void slice(int b) { c += b * bstride; }
  __device__ __forceinline__ bool interior(int r0, int r1, int c0, int c1) const {
    return r0 >= 0 && r1 <= N && c0 >= 0 && c1 <= N;
  }
  __device__ __forceinline__ float direct(int r, int col) const {
    return __ldg(c + static_cast<size_t>(r + kPad) * pitch + col + kPad);
  }
  __device__ __forceinline__ bool dead(int, int, int, int) const { return false; }
  __device__ __forceinline__ float extended(int r, int col) const {
    float sr, sc;
    const int rr = odd_ext(r, N, &sr);
    const int cc = odd_ext(col, N, &sc);
    const float sg = sr * sc;
    return sg != 0.f ? sg * direct(rr, cc) : 0.f;
  }
  __device__ __forceinline__ bool keep(int r, int col) const { return in_disc(r, col, N); }
};

// Pre-filter of one segment: the kPfSeg coefficients at the centre of a window of kPfSeg +
// 2 kFirHalf samples, by the recursion of Eq. Qfrecursive run inside the window: causal
// u[k] = w[k] + z u[k-1] from zero state at the window start, anticausal v[k] = u[k] + z v[k+1]
// from zero state at the window end, c = -6 z v (the pair's impulse response is
// -6 z / (1 - z^2) z^|n| = sqrt(3) z^|n|).  The zero states sit kFirHalf samples outside the
// segment, so the response is cut at z^15 ~ 2.7e-9, as a 29-tap truncated FIR would be, at 8
// operations per coefficient instead of 29.
template <int SEG>
__device__ __forceinline__ void segment_prefilter(float (&w)[SEG + 2 * kFirHalf], float (&c)[SEG]) {
  constexpr float z = -0.267949192431122706f;  // sqrt(3) - 2
  constexpr float g = -6.f * z;
  constexpr int W = SEG + 2 * kFirHalf;
#pragma unroll
  for (int k = 1; k < W; ++k) w[k] = fmaf(z, w[k - 1], w[k]);
  float v = w[W - 1];
#pragma unroll
  for (int k = W - 2; k >= kFirHalf; --k) {
    v = fmaf(z, v, w[k]);
    if (k < kFirHalf + SEG) c[k - kFirHalf] = g * v;
  }
}

// QUAD: the tile's output is the quad-row layout coef_q4 (element (r, c) = padded coefficients
// (r, c .. c+3), zero outside the image): kPfQuads quad origins per tile need the 64 coefficient
// columns starting 3 to their left, which the tile computes as usual and then regroups in shared
// memory.  Rows outside the image stay zero from allocation.
constexpr int kPfQuads = kPfCols - 3;

template <class Src, bool QUAD>
__global__ void __launch_bounds__(kThreads) k_prefilter(DevPlan p, Src src, int n_rows, int n_cols,
                                                        float* __restrict__ out, int out_pitch, int out_r0,
                                                        size_t out_bstride) {
  __shared__ float s_in[kPfInR][kPfInC + 1];
  __shared__ float s_mid[kPfInR][kPfCols + 1];
  const int b = blockIdx.z;  // slice of a batch
  src.slice(b);
  if (out) out += b * out_bstride;
  const int qcol = blockIdx.x * kPfQuads;                       // first quad origin (QUAD)
  const int ccol = QUAD ? qcol - 3 : blockIdx.x * kPfCols;      // first coefficient column computed
  const int r0 = blockIdx.y * kPfRows - kFirHalf, c0 = ccol - kFirHalf;
  const int tid = threadIdx.x;
  if (src.dead(r0, r0 + kPfInR, c0, c0 + kPfInC)) {  // all coefficients of the tile are zero
    const int orow = blockIdx.y * kPfRows;
    if constexpr (QUAD) {
      const int P = p.img_pitch;
      float4* q4 = p.coef_q4 + b * p.bs_img;
      for (int y = tid >> 5; y < kPfRows; y += kThreads / 32) {
        const int gr = orow + y;
        if (gr >= n_rows) break;
        float4* dst = q4 + static_cast<size_t>(gr + kPad) * P + qcol;
        for (int lx = tid & 31; lx < kPfQuads && qcol + lx < P; lx += 32) dst[lx] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    } else {
      for (int y = tid >> 5; y < kPfRows; y += kThreads / 32) {
        const int gr = orow + y;
        if (gr >= n_rows) break;
        float* dst = out + static_cast<size_t>(gr + out_r0) * out_pitch + ccol + Src::kOutPad;
        for (int lx = tid & 31; lx < kPfCols && ccol + lx < n_cols; lx += 32) dst[lx] = 0.f;
      }
    }
    return;
  }
  if (src.interior(r0, r0 + kPfInR, c0, c0 + kPfInC)) {
    // warp w reads rows w, w + 8, ... and lane l columns l, l + 32, l + 64 (no index division);
    // all loads of this thread are issued before the first shared-memory store
    constexpr int kWarpsPf = kThreads / 32;
    constexpr int kRowIt = (kPfInR + kWarpsPf - 1) / kWarpsPf, kColIt = (kPfInC + 31) / 32;
    const int lane = tid & 31, warp = tid >> 5;
    float v[kRowIt][kColIt];
#pragma unroll
    for (int i = 0; i < kRowIt; ++i) {
      const int ly = warp + i * kWarpsPf;
#pragma unroll
      for (int j = 0; j < kColIt; ++j) {
        const int lx = lane + 32 * j;
        v[i][j] = (ly < kPfInR && lx < kPfInC) ? src.direct(r0 + ly, c0 + lx) : 0.f;
      }
    }
#pragma unroll
    for (int i = 0; i < kRowIt; ++i) {
      const int ly = warp + i * kWarpsPf;
#pragma unroll
      for (int j = 0; j < kColIt; ++j) {
        const int lx = lane + 32 * j;
        if (ly < kPfInR && lx < kPfInC) s_in[ly][lx] = v[i][j];
      }
    }
  } else {
    for (int idx = tid; idx < kPfInR * kPfInC; idx += kThreads) {
      const int ly = idx / kPfInC, lx = idx - ly * kPfInC;
      s_in[ly][lx] = src.extended(r0 + ly, c0 + lx);
    }
  }
  __syncthreads();
  const int orow = blockIdx.y * kPfRows, ocol = ccol;
  if (!QUAD && p.interp == 1) {  // linear interpolation uses the masked samples themselves
    for (int idx = tid; idx < kPfRows * kPfCols; idx += kThreads) {
      const int ly = idx / kPfCols, lx = idx - ly * kPfCols;
      if (orow + ly < n_rows && ocol + lx < n_cols) {
        const float v = src.keep(orow + ly, ocol + lx) ? s_in[ly + kFirHalf][lx + kFirHalf] : 0.f;
        out[static_cast<size_t>(orow + ly + out_r0) * out_pitch + ocol + lx + Src::kOutPad] = v;
      }
    }
    return;
  }
  // along rows: kPfInR rows x (kPfCols / kPfSegRow) segments; consecutive threads take
  // consecutive rows of one segment, so their shared-memory accesses (row strides kPfInC + 1 and
  // kPfCols + 1, both odd) fall into distinct banks
  for (int task = tid; task < kPfInR * (kPfCols / kPfSegRow); task += kThreads) {
    const int seg = task / kPfInR, ly = task - seg * kPfInR, sx = seg * kPfSegRow;
    float w[kPfSegRow + 2 * kFirHalf];
#pragma unroll
    for (int t = 0; t < kPfSegRow + 2 * kFirHalf; ++t) w[t] = s_in[ly][sx + t];
    float c[kPfSegRow];
    segment_prefilter<kPfSegRow>(w, c);
#pragma unroll
    for (int t = 0; t < kPfSegRow; ++t) s_mid[ly][sx + t] = c[t];
  }
  __syncthreads();
  // along columns: kPfCols columns x (kPfRows / kPfSeg) segments
  for (int task = tid; task < kPfCols * (kPfRows / kPfSeg); task += kThreads) {
    const int lx = task % kPfCols, sy = (task / kPfCols) * kPfSeg;
    float w[kPfSeg + 2 * kFirHalf];
#pragma unroll
    for (int t = 0; t < kPfSeg + 2 * kFirHalf; ++t) w[t] = s_mid[sy + t][lx];
    const int gc = ocol + lx;
    float c[kPfSeg];
    segment_prefilter<kPfSeg>(w, c);
#pragma unroll
    for (int t = 0; t < kPfSeg; ++t) {
      const float acc = c[t];
      const int gr = orow + sy + t;
      if constexpr (QUAD) {
        s_in[sy + t][lx] = (gc >= 0 && gc < n_cols) ? acc : 0.f;  // s_in is free after the row pass
      } else if (gr < n_rows && gc < n_cols) {
        out[static_cast<size_t>(gr + out_r0) * out_pitch + gc + Src::kOutPad] = src.keep(gr, gc) ? acc : 0.f;
      }
    }
  }
  if constexpr (QUAD) {
    __syncthreads();
    const int P = p.img_pitch;
    float4* q4 = p.coef_q4 + b * p.bs_img;
    // warp w stores rows w, w + 8, ...; lane l quads l and l + 32
    for (int y = tid >> 5; y < kPfRows; y += kThreads / 32) {
      const int gr = orow + y;
      if (gr >= n_rows) break;  // rows only grow along the loop
      float4* dst = q4 + static_cast<size_t>(gr + kPad) * P + qcol;
      for (int lx = tid & 31; lx < kPfQuads && qcol + lx < P; lx += 32)
        dst[lx] = make_float4(s_in[y][lx], s_in[y][lx + 1], s_in[y][lx + 2], s_in[y][lx + 3]);
    }
  }
}

// ------------------------------------------------------------------------------------------
// Row sampling.

// Value of the image interpolant at padded index coordinates (ic + ac, ir + ar).
__device__ __forceinline__ float sample_image(const DevPlan& p, int b, int ic, float ac, int ir, float ar) {
  const float* __restrict__ c = p.coef_img + b * p.bs_img;
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
//
// Coordinates: for each sub-angle q and each 32-sample rho tile, a double-float anchor
// col/row = e^rho_anchor * (cos, sin)(psi_q) * N / (2 a_R) + offset, computed once per warp into
// shared memory as (integer, fraction); each sample adds the FP32 offset (e^rho_i - e^rho_anchor)
// times the direction.
//
// Taps: with img_quad each of the 4 tap rows is one aligned 16-byte load from the quad layout;
// otherwise 16 scalar loads from the padded coefficient image.  Samples whose tap block lies
// farther than kDiscMargin pixels outside the unit disc (or outside the padded array) are skipped
// through the host's per-sub-angle rho ranges: the pre-filtered disc-masked image decays like
// 0.27^d away from the disc, below 1e-8 of its maximum there.



// Forward sampling (Algorithm 1: resample T_m f on Omega_lp, average the r sub-angles onto
// Omega_p, multiply by e^rho).  One warp per tile of 32 rho samples of one angular row (m, jj);
// a CTA holds the same tile of kSampleWarps adjacent rows, so its taps overlap in L1.  The real row h is written to the
// spectrum scratch yspec (free until the theta convolution), 2 x_pitch floats per row.
constexpr int kSampleWarps = 8;
// Image sizes N whose forward sampling is compiled with a constant padded pitch N + 2 kPad.
#define RADON_SAMPLE_PITCHES(X) X(256) X(512) X(1024) X(2048) X(4096) X(8192)


// Cubic B-spline weights times 6 (the 1/36 of a 2-D tap block is applied once per output) for
// two fractions at once (.x and .y), with paired FP32 arithmetic.
__device__ __forceinline__ void bspline_w6_pair(float2 a, float2 (&w)[4]) {
  const float2 one = make_float2(1.f, 1.f);
  const float2 om = __ffma2_rn(a, make_float2(-1.f, -1.f), one);
  const float2 a2 = __fmul2_rn(a, a);
  w[0] = __fmul2_rn(__fmul2_rn(om, om), om);
  w[1] = __ffma2_rn(a2, __ffma2_rn(make_float2(3.f, 3.f), a, make_float2(-6.f, -6.f)), make_float2(4.f, 4.f));
  w[2] = __ffma2_rn(a, __ffma2_rn(a, __ffma2_rn(make_float2(-3.f, -3.f), a, make_float2(3.f, 3.f)), make_float2(3.f, 3.f)),
                    one);
  w[3] = __fmul2_rn(a2, a);
}

// Two rho samples per thread (i and i + 32, tiles 2 blockIdx.x and 2 blockIdx.x + 1) for each
// sub-angle q; a sample is read only when i lies in the sub-angle's range fwd_rng (its taps are
// then inside the padded array), so no per-sample bounds test is needed.  PITCH > 0 fixes the
// padded image width at compile time (the tabulated sizes N = PITCH - 2 kPad): a tap block's four
// quad rows are then one address plus constant offsets.
template <bool QUAD, int PITCH = 0>
__global__ void __launch_bounds__(kSampleWarps * 32) k_sample_fwd(DevPlan p) {
  extern __shared__ __align__(16) float4 sanc[];  // [warp][2][q] anchors, [warp][q] directions, [warp][q] ranges
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = p.r, ne = p.n_eanc;
  const int tile0 = 2 * blockIdx.x, m = blockIdx.z % p.M, b = blockIdx.z / p.M;
  const int jj = blockIdx.y * kSampleWarps + warp;
  if (jj >= p.nh) return;  // whole warp; only warp-level synchronisation below
  float4* anc = sanc + warp * 2 * r;
  float2* dir = reinterpret_cast<float2*>(sanc + kSampleWarps * 2 * r) + warp * r;
  int2* rng = reinterpret_cast<int2*>(reinterpret_cast<float2*>(sanc + kSampleWarps * 2 * r) + kSampleWarps * r) + warp * r;
  const float4 um = p.fwd_m[m];
  const size_t row0 = (static_cast<size_t>(m) * p.nh + jj) * r;
  const float4* rowc = p.fwd_row + row0;
  const float2 ea0 = p.fwd_eanc[tile0];
  const float2 ea1 = p.fwd_eanc[tile0 + 1 < ne ? tile0 + 1 : tile0];
  for (int q = lane; q < r; q += 32) {
    const float4 cs = rowc[q];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const float2 ea = u ? ea1 : ea0;
      float ch, cl, rh, rl;
      df_mul_add(ea.x, ea.y, cs.x, cs.y, um.x, um.y, &ch, &cl);
      df_mul_add(ea.x, ea.y, cs.z, cs.w, um.z, um.w, &rh, &rl);
      const float Ic = floorf(ch), Ir = floorf(rh);
      anc[u * r + q] = make_float4(Ic, (ch - Ic) + cl, Ir, (rh - Ir) + rl);
    }
    dir[q] = make_float2(cs.x, cs.z);
    rng[q] = p.fwd_rng[row0 + q];
  }
  __syncwarp();
  const int base = tile0 * kETile;
  const int i0 = base + lane, i1 = i0 + kETile;
  const float2 e0 = i0 < p.N_rho ? p.fwd_e[i0] : make_float2(0.f, 0.f);
  const float2 e1 = i1 < p.N_rho ? p.fwd_e[i1] : make_float2(0.f, 0.f);
  const int P = PITCH > 0 ? PITCH : p.img_pitch;
  float acc0 = 0.f, acc1 = 0.f;
  for (int q = 0; q < r; ++q) {
    const int2 rg = rng[q];
    if (rg.y < base || rg.x > base + 2 * kETile - 1) continue;  // warp-uniform: no sample in range
    const bool ok0 = i0 >= rg.x && i0 <= rg.y, ok1 = i1 >= rg.x && i1 <= rg.y;
    const float2 d = dir[q];
    const float4 a0 = anc[q], a1 = anc[r + q];
    const float Fc0 = fmaf(e0.y, d.x, a0.y), Fr0 = fmaf(e0.y, d.y, a0.w);
    const float Fc1 = fmaf(e1.y, d.x, a1.y), Fr1 = fmaf(e1.y, d.y, a1.w);
    const float fc0 = floorf(Fc0), fr0 = floorf(Fr0), fc1 = floorf(Fc1), fr1 = floorf(Fr1);
    // padded tap-block corners; samples out of range read element (1, 1) and are dropped
    const int ic0 = ok0 ? static_cast<int>(a0.x + fc0) : 1, ir0 = ok0 ? static_cast<int>(a0.z + fr0) : 1;
    const int ic1 = ok1 ? static_cast<int>(a1.x + fc1) : 1, ir1 = ok1 ? static_cast<int>(a1.z + fr1) : 1;
    if constexpr (QUAD) {
      const float4* __restrict__ img = p.coef_q4 + b * p.bs_img;
      float4 v0[4], v1[4];
      if constexpr (PITCH > 0) {
        // 32-bit element offsets (the padded image has fewer than 2^31 elements); the rows of a
        // tap block are constant offsets from its first element
        const float4* p0 = img + static_cast<unsigned>(ir0 * PITCH + ic0) - (PITCH + 1);
        const float4* p1 = img + static_cast<unsigned>(ir1 * PITCH + ic1) - (PITCH + 1);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          v0[k] = __ldg(p0 + k * PITCH);
          v1[k] = __ldg(p1 + k * PITCH);
        }
      } else {
        const float4* p0 = img + static_cast<size_t>(ir0 - 1) * P + (ic0 - 1);
        const float4* p1 = img + static_cast<size_t>(ir1 - 1) * P + (ic1 - 1);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          v0[k] = __ldg(p0 + k * P);
          v1[k] = __ldg(p1 + k * P);
        }
      }
      float2 wc[4], wr[4];  // .x: sample i0, .y: sample i1
      bspline_w6_pair(make_float2(Fc0 - fc0, Fc1 - fc1), wc);
      bspline_w6_pair(make_float2(Fr0 - fr0, Fr1 - fr1), wr);
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        s0 = fmaf(wr[k].x, fmaf(wc[0].x, v0[k].x, fmaf(wc[1].x, v0[k].y, fmaf(wc[2].x, v0[k].z, wc[3].x * v0[k].w))), s0);
        s1 = fmaf(wr[k].y, fmaf(wc[0].y, v1[k].x, fmaf(wc[1].y, v1[k].y, fmaf(wc[2].y, v1[k].z, wc[3].y * v1[k].w))), s1);
      }
      acc0 += ok0 ? s0 : 0.f;
      acc1 += ok1 ? s1 : 0.f;
    } else {
      const float s0 = sample_image(p, b, ic0, Fc0 - fc0, ir0, Fr0 - fr0);
      const float s1 = sample_image(p, b, ic1, Fc1 - fc1, ir1, Fr1 - fr1);
      acc0 += ok0 ? s0 : 0.f;
      acc1 += ok1 ? s1 : 0.f;
    }
  }
  const float scale = QUAD ? 1.f / 36.f : 1.f;
  float* h = reinterpret_cast<float*>(p.yspec + b * p.bs_ys + (static_cast<size_t>(m) * p.nh + jj) * p.x_pitch);
  if (i0 < p.N_rho) h[i0] = acc0 * e0.x * scale;
  if (i1 < p.N_rho) h[i1] = acc1 * e1.x * scale;
}

// Forward sampling, cubic, quad layout, with each load instruction spread over consecutive fine
// angles (the same outputs as k_sample_fwd<true>).  The r sub-angles of kSampleWarps adjacent
// rows are 8 r equally spaced fine angles; a CTA of R warps takes them all for 64 rho samples.
// Warp w owns fine angles 8 w .. 8 w + 7 and lane 4 a + o the fine angle 8 w + a at rho offsets
// o, o + 4, ..., so one load instruction reads a 4 (rho) x 8 (fine angle) block of samples: about
// as far apart across the rays as along them, which touches fewer L1 lines than 32 samples along
// one ray.  Each lane keeps its fine angle's anchors and rho range in registers.  The fine
// samples go to shared memory; a second phase sums each output's r sub-angles and applies
// e^rho / r and the 1/36 of the weights taken times 6.
constexpr int kArcStride = 68;  // floats per fine angle in shared memory: a store's 32 lanes hit distinct banks
template <int R, int PITCH>
__global__ void __launch_bounds__(R * 32, 36 / R) k_sample_fwd_arc(DevPlan p) {
  __shared__ float sval[kSampleWarps * R][kArcStride];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tile0 = 2 * blockIdx.x, m = blockIdx.z % p.M, b = blockIdx.z / p.M;
  const int jj0 = blockIdx.y * kSampleWarps;
  const int f = 8 * warp + (lane >> 2), o = lane & 3;  // fine angle within the CTA, rho offset
  const int jl = f / R, q = f - jl * R;
  const bool row_ok = jj0 + jl < p.nh;
  const int base = tile0 * kETile;
  const int P = PITCH > 0 ? PITCH : p.img_pitch;
  float4 a0 = make_float4(1.f, 0.f, 1.f, 0.f), a1 = a0;
  float2 d = make_float2(0.f, 0.f);
  int2 rg = make_int2(1, 0);  // empty range
  if (row_ok) {
    const size_t rq = (static_cast<size_t>(m) * p.nh + jj0 + jl) * R + q;
    const float4 cs = p.fwd_row[rq];
    const float4 um = p.fwd_m[m];
    const int ne = p.n_eanc;
    const float2 ea0 = p.fwd_eanc[tile0];
    const float2 ea1 = p.fwd_eanc[tile0 + 1 < ne ? tile0 + 1 : tile0];
    float ch, cl, rh, rl;
    df_mul_add(ea0.x, ea0.y, cs.x, cs.y, um.x, um.y, &ch, &cl);
    df_mul_add(ea0.x, ea0.y, cs.z, cs.w, um.z, um.w, &rh, &rl);
    float Ic = floorf(ch), Ir = floorf(rh);
    a0 = make_float4(Ic, (ch - Ic) + cl, Ir, (rh - Ir) + rl);
    df_mul_add(ea1.x, ea1.y, cs.x, cs.y, um.x, um.y, &ch, &cl);
    df_mul_add(ea1.x, ea1.y, cs.z, cs.w, um.z, um.w, &rh, &rl);
    Ic = floorf(ch);
    Ir = floorf(rh);
    a1 = make_float4(Ic, (ch - Ic) + cl, Ir, (rh - Ir) + rl);
    d = make_float2(cs.x, cs.z);
    rg = p.fwd_rng[rq];
  }
  const float4* __restrict__ img = p.coef_q4 + b * p.bs_img;
  float* sv = sval[f];
  // warp-uniform: does any lane of the warp have a sample in this CTA's 64 rho indices?
  const bool any = __any_sync(0xffffffffu, rg.y >= base && rg.x <= base + 2 * kETile - 1);
#pragma unroll 1
  for (int t = 0; t < 2 * kETile / 4; t += 2) {
    const int i0 = base + 4 * t + o, i1 = i0 + 4;  // same anchor tile: t and t + 1 lie on one side of 8
    const bool ok0 = any && i0 >= rg.x && i0 <= rg.y, ok1 = any && i1 >= rg.x && i1 <= rg.y;
    if (!__any_sync(0xffffffffu, ok0 || ok1)) {
      sv[4 * t + o] = 0.f;
      sv[4 * t + 4 + o] = 0.f;
      continue;
    }
    const float4 a = t < kETile / 4 ? a0 : a1;
    const float e0 = ok0 ? p.fwd_e[i0].y : 0.f, e1 = ok1 ? p.fwd_e[i1].y : 0.f;
    const float Fc0 = fmaf(e0, d.x, a.y), Fr0 = fmaf(e0, d.y, a.w);
    const float Fc1 = fmaf(e1, d.x, a.y), Fr1 = fmaf(e1, d.y, a.w);
    const float fc0 = floorf(Fc0), fr0 = floorf(Fr0), fc1 = floorf(Fc1), fr1 = floorf(Fr1);
    // padded tap-block corners; samples out of range read element (1, 1) and are dropped
    const int ic0 = ok0 ? static_cast<int>(a.x + fc0) : 1, ir0 = ok0 ? static_cast<int>(a.z + fr0) : 1;
    const int ic1 = ok1 ? static_cast<int>(a.x + fc1) : 1, ir1 = ok1 ? static_cast<int>(a.z + fr1) : 1;
    const float4* p0 = img + static_cast<unsigned>(ir0 * P + ic0) - (P + 1);
    const float4* p1 = img + static_cast<unsigned>(ir1 * P + ic1) - (P + 1);
    float4 v0[4], v1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v0[k] = __ldg(p0 + k * P);
      v1[k] = __ldg(p1 + k * P);
    }
    float2 wc[4], wr[4];  // .x: sample i0, .y: sample i1
    bspline_w6_pair(make_float2(Fc0 - fc0, Fc1 - fc1), wc);
    bspline_w6_pair(make_float2(Fr0 - fr0, Fr1 - fr1), wr);
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      s0 = fmaf(wr[k].x, fmaf(wc[0].x, v0[k].x, fmaf(wc[1].x, v0[k].y, fmaf(wc[2].x, v0[k].z, wc[3].x * v0[k].w))), s0);
      s1 = fmaf(wr[k].y, fmaf(wc[0].y, v1[k].x, fmaf(wc[1].y, v1[k].y, fmaf(wc[2].y, v1[k].z, wc[3].y * v1[k].w))), s1);
    }
    sv[4 * t + o] = ok0 ? s0 : 0.f;
    sv[4 * t + 4 + o] = ok1 ? s1 : 0.f;
  }
  __syncthreads();
  // outputs (row jl, rho base + il): the sum of the row's R fine samples
  for (int idx = threadIdx.x; idx < kSampleWarps * 2 * kETile; idx += R * 32) {
    const int rl = idx / (2 * kETile), il = idx - rl * (2 * kETile);
    const int jj = jj0 + rl, i = base + il;
    if (jj >= p.nh || i >= p.N_rho) continue;
    float acc = 0.f;
#pragma unroll
    for (int qq = 0; qq < R; ++qq) acc += sval[rl * R + qq][il];
    float* h = reinterpret_cast<float*>(p.yspec + b * p.bs_ys + (static_cast<size_t>(m) * p.nh + jj) * p.x_pitch);
    h[i] = acc * p.fwd_e[i].x * (1.f / 36.f);
  }
}

// Back-projection: G(phi_j, rho_i) = g~(phi_j + m beta, (e^rho_i - (1 - a_R) cos phi_j) / a_R).
// The theta taps (rows of the extended sinogram, flips, weights) are the same for the whole row;
// a flipped row (theta + pi) is read at k -> n_det - k, i.e. with reversed s weights.  FLIPS:
// 0 no tap row flipped, 1 all flipped, 2 mixed (the flags are uniform over the CTA, so the loop
// is chosen once per row).
template <int FLIPS>
__device__ __forceinline__ void backproject_row_cubic(const DevPlan& p, const float* const (&rows)[4],
                                                      const bool (&flip)[4], const float (&wt)[4], int cjx,
                                                      float Fc, float* __restrict__ h) {
  const int pitch = p.sino_pitch;
  const int K = p.n_det + 2 * kPad;  // padded index of a flipped tap: K - c
  for (int i = threadIdx.x; i < p.N_rho; i += blockDim.x) {
    const int2 ei = p.bp_e[i];
    const float F = __int_as_float(ei.y) + Fc;
    const float fl = floorf(F);
    const int is = ei.x + cjx + static_cast<int>(fl);
    float ws[4];
    bspline_w(F - fl, ws);
    const int bf = FLIPS == 1 ? 0 : clampi(is - 1, 0, pitch - 4);      // forward taps is-1 .. is+2
    const int bb = FLIPS == 0 ? 0 : clampi(K - is - 2, 0, pitch - 4);  // flipped taps K-is-2 .. K-is+1
    float acc = 0.f;
#pragma unroll
    for (int dt = 0; dt < 4; ++dt) {
      const bool fd = FLIPS == 2 ? flip[dt] : FLIPS == 1;
      const float* r = rows[dt] + (fd ? bb : bf);
      const float x0 = __ldg(r), x1 = __ldg(r + 1), x2 = __ldg(r + 2), x3 = __ldg(r + 3);
      const float v = fd ? fmaf(ws[3], x0, fmaf(ws[2], x1, fmaf(ws[1], x2, ws[0] * x3)))
                         : fmaf(ws[0], x0, fmaf(ws[1], x1, fmaf(ws[2], x2, ws[3] * x3)));
      acc = fmaf(wt[dt], v, acc);
    }
    h[i] = acc;
  }
}

constexpr int kCombGuard = 4;  // zero cells on each side of a theta-combined row in shared memory

// Cubic interpolation in s of a theta-combined detector row comb at rho sample i: taps c0 .. c0 + 3
// around the sample's padded bin, zero outside the row.
struct CombSample {
  const float* comb;
  const int2* __restrict__ bp_e;
  int cjx;
  float Fc;
  int pitch;
  __device__ __forceinline__ float operator()(int i) const {
    const int2 ei = bp_e[i];
    const float F = __int_as_float(ei.y) + Fc;
    const float fl = floorf(F);
    // taps c0 .. c0 + 3; comb has kCombGuard zero cells on each side, so a block that leaves the
    // row reads zeros, and one wholly outside it is moved into the guard band (still zeros)
    const int c0 = clampi(ei.x + cjx + static_cast<int>(fl) - 1, -kCombGuard, pitch);
    float ws[4];
    bspline_w(F - fl, ws);
    float acc = 0.f;
#pragma unroll
    for (int d = 0; d < 4; ++d) acc = fmaf(ws[d], comb[c0 + d], acc);
    return acc;
  }
};
// Complex input k of the row transform: real samples 2k and 2k + 1.
struct CombSamples {
  CombSample s;
  __device__ __forceinline__ float2 operator()(int k) const { return make_float2(s(2 * k), s(2 * k + 1)); }
};

// Cubic back-projection row with the theta interpolation done first: the four theta tap rows and
// their weights are the same for every rho sample of the row, so they are combined once into one
// detector row comb[c] = sum_t w_t row_t(c) (a flipped row read at K - c) in shared memory, and each
// rho sample then takes a 4-tap cubic interpolation in s of that row: 4 taps per sample instead of
// 16.  The sum runs in the other order than backproject_row_cubic's, so the two agree to FP32
// rounding.  Taps outside the padded row read zero.  All threads of the CTA call it.
__device__ __forceinline__ void backproject_row_cubic_comb(const DevPlan& p, const float* const (&rows)[4],
                                                           const bool (&flip)[4], const float (&wt)[4], int cjx,
                                                           float Fc, float* __restrict__ h, float* __restrict__ comb) {
  const int pitch = p.sino_pitch;
  const int K = p.n_det + 2 * kPad;  // padded index of a flipped tap: K - c
  // columns c <= K: both c and K - c lie inside the padded row, no test needed
  const int cin = K + 1 < pitch ? K + 1 : pitch;
  for (int c = threadIdx.x; c < cin; c += blockDim.x) {
    float acc = 0.f;
#pragma unroll
    for (int dt = 0; dt < 4; ++dt) acc = fmaf(wt[dt], __ldg(rows[dt] + (flip[dt] ? K - c : c)), acc);  // flip[] is uniform over the CTA
    comb[c] = acc;
  }
  // the alignment columns past K (at most 3): a flipped row has no tap there
  for (int c = cin + static_cast<int>(threadIdx.x); c < pitch; c += blockDim.x) {
    float acc = 0.f;
#pragma unroll
    for (int dt = 0; dt < 4; ++dt) acc = fmaf(wt[dt], flip[dt] ? 0.f : __ldg(rows[dt] + c), acc);
    comb[c] = acc;
  }
  if (threadIdx.x < kCombGuard) {
    comb[static_cast<int>(threadIdx.x) - kCombGuard] = 0.f;
    comb[pitch + threadIdx.x] = 0.f;
  }
  __syncthreads();
  if (h == nullptr) return;  // the caller's row transform samples comb itself (CombSamples)
  const CombSample smp{comb, p.bp_e, cjx, Fc, pitch};
  for (int i = threadIdx.x; i < p.N_rho; i += blockDim.x) h[i] = smp(i);
}

__device__ void sample_row_backproject(const DevPlan& p, int b, int m, int jj, float* __restrict__ h,
                                       float* __restrict__ comb) {
  const int2 th = p.bp_th[m * p.nh + jj];
  const int2 cj = p.bp_c[jj];
  const float Ft = __int_as_float(th.y), Fc = __int_as_float(cj.y);
  const int na = p.n_angles, pitch = p.sino_pitch;
  const int K = p.n_det + 2 * kPad;  // padded index of a flipped tap: K - c
  const bool cubic = p.interp == 3;
  const int ntap = cubic ? 4 : 2;
  float wt[4];
  const float* rows[4];
  bool flip[4];
  if (cubic) {
    bspline_w(Ft, wt);
  } else {
    wt[0] = 1.f - Ft;
    wt[1] = Ft;
    wt[2] = wt[3] = 0.f;
  }
  const int t0 = cubic ? th.x - 1 : th.x;
  int nflip = 0;
  for (int dt = 0; dt < 4; ++dt) {
    int a2 = (t0 + dt) % (2 * na);
    if (a2 < 0) a2 += 2 * na;
    flip[dt] = a2 >= na;
    nflip += (dt < ntap && flip[dt]) ? 1 : 0;
    rows[dt] = p.coef_sino + b * p.bs_sino + static_cast<size_t>(flip[dt] ? a2 - na : a2) * pitch;
  }
  if (cubic && comb) {
    backproject_row_cubic_comb(p, rows, flip, wt, cj.x, Fc, h, comb);
    return;
  }
  if (cubic) {
    if (nflip == 0)
      backproject_row_cubic<0>(p, rows, flip, wt, cj.x, Fc, h);
    else if (nflip == 4)
      backproject_row_cubic<1>(p, rows, flip, wt, cj.x, Fc, h);
    else
      backproject_row_cubic<2>(p, rows, flip, wt, cj.x, Fc, h);
    return;
  }
  for (int i = threadIdx.x; i < p.N_rho; i += blockDim.x) {
    const int2 ei = p.bp_e[i];
    const float F = __int_as_float(ei.y) + Fc;
    const float fl = floorf(F);
    const int is = ei.x + cj.x + static_cast<int>(fl);
    const float as = F - fl;
    const int bf = clampi(is, 0, pitch - 2);
    const int bb = clampi(K - is - 1, 0, pitch - 2);
    float acc = 0.f;
    for (int dt = 0; dt < ntap; ++dt) {
      const float* r = rows[dt] + (flip[dt] ? bb : bf);
      const float x0 = __ldg(r), x1 = __ldg(r + 1);
      const float v = flip[dt] ? fmaf(as, x0 - x1, x1) : fmaf(as, x1 - x0, x0);
      acc = fmaf(wt[dt], v, acc);
    }
    h[i] = acc;
  }
}

// Row transforms with a compile-time radix sequence, in kRowRadices order.
#define RADON_ROW_SEQUENCES(X) \
  X(0, 9, 9, 9, 3)             \
  X(1, 2, 9, 9, 9, 3)          \
  X(2, 8, 4, 5, 7)

template <int... Rs>
constexpr bool row_radices_match(const RowRadices& c) {
  int i = 0;
  bool ok = true;
  ((ok = ok && i < 5 && c.r[i] == Rs, ++i), ...);
  return ok && (i == 5 || c.r[i] == 0) && c.n == chain_length<Rs...>();
}

template <int SEQ, bool INV>
struct RowFft;
#define RADON_ROW_FFT(i, ...)                                                                              \
  template <bool INV>                                                                                      \
  struct RowFft<i, INV> {                                                                                  \
    __device__ __forceinline__ static float2* run(float2* a, float2* b, const float2* __restrict__ tw) {    \
      return FixedFft<chain_length<__VA_ARGS__>(), INV, kThreads, 1, __VA_ARGS__>::run(a, b, tw, threadIdx.x); \
    }                                                                                                      \
    template <class In>                                                                                    \
    __device__ __forceinline__ static float2* run_in(const In& in, float2* a, float2* b,                   \
                                                     const float2* __restrict__ tw) {                      \
      return FixedFftIn<chain_length<__VA_ARGS__>(), INV, kThreads, __VA_ARGS__>::run(in, a, b, tw, threadIdx.x); \
    }                                                                                                      \
    template <class In, class Out>                                                                         \
    __device__ __forceinline__ static void run_in_out(const In& in, float2* a, float2* b,                  \
                                                      const float2* __restrict__ tw, const Out& out) {     \
      FixedFftInOut<chain_length<__VA_ARGS__>(), INV, kThreads, __VA_ARGS__>::run(in, a, b, tw, out, threadIdx.x); \
    }                                                                                                      \
  };                                                                                                       \
  static_assert(row_radices_match<__VA_ARGS__>(kRowRadices[i]), "row radix table");
RADON_ROW_SEQUENCES(RADON_ROW_FFT)
#undef RADON_ROW_FFT
static_assert(kNumRowRadices == 3, "every kRowRadices entry has a compiled transform");

// Complex transform of length nc along a row (all threads of the CTA); SEQ < 0: generic.
template <bool INV, int SEQ>
__device__ __forceinline__ const float2* row_fft(float2* a, float2* b, const DevPlan& p, const float2* tw) {
  if constexpr (SEQ < 0)
    return fft_block<INV>(a, b, 1, p.nc, p.rad_rho, tw, threadIdx.x, blockDim.x);
  else
    return RowFft<SEQ, INV>::run(a, b, tw);
}

// Forward complex transform whose first pass reads in(k) (compiled transforms only; SEQ < 0 is
// never called).
template <int SEQ, class In>
__device__ __forceinline__ const float2* row_fft_in(const In& in, float2* a, float2* b, const DevPlan& p,
                                                   const float2* tw) {
  if constexpr (SEQ < 0)
    return nullptr;
  else
    return RowFft<SEQ, false>::run_in(in, a, b, tw);
}

// Sample one angular row, real FFT along rho, write the half spectrum (N_rho/2 + 1 bins).
template <bool BACK, int SEQ>
__global__ void __launch_bounds__(kThreads) k_rows_fwd(DevPlan p) {
  extern __shared__ __align__(16) float2 smem[];
  const int nc = p.nc;
  float2* bufA = smem;
  float2* bufB = smem + nc;
  const float2* tw;
  const int jj = blockIdx.x, m = blockIdx.y, b = blockIdx.z;
  if (BACK) {
    float2* tws = smem + 2 * nc;
    if (p.rows_tw_smem) stage_table(tws, p.tw_rho, nc, threadIdx.x, blockDim.x);
    tw = p.rows_tw_smem ? tws : p.tw_rho;
    // bufB (free until the FFT) holds the theta-combined detector row when it fits
    float* comb = p.sino_pitch + 2 * kCombGuard <= 2 * nc ? reinterpret_cast<float*>(bufB) + kCombGuard : nullptr;
    sample_row_backproject(p, b, m, jj, reinterpret_cast<float*>(bufA), comb);
  } else {  // the row sampled by k_sample_fwd, read as nc complex values
    float2* tws = smem + 2 * nc;
    if (p.rows_tw_smem) stage_table(tws, p.tw_rho, nc, threadIdx.x, blockDim.x);
    tw = p.rows_tw_smem ? tws : p.tw_rho;
    const float2* h = p.yspec + b * p.bs_ys + (static_cast<size_t>(m) * p.nh + jj) * p.x_pitch;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) bufA[k] = h[k];
  }
  __syncthreads();
  const float2* Z = row_fft<false, SEQ>(bufA, bufB, p, tw);
  float2* out = p.xspec + b * p.bs_x + (static_cast<size_t>(m) * p.nh + jj) * p.x_pitch;
  for (int k = threadIdx.x; k <= nc; k += blockDim.x) {
    const float2 zk = Z[k == nc ? 0 : k];
    const float2 zc = cconj(Z[k == 0 ? 0 : nc - k]);
    const float2 ev = cscale(cadd(zk, zc), 0.5f);
    const float2 dv = cscale(csub(zk, zc), 0.5f);
    const float2 od = make_float2(dv.y, -dv.x);  // -i (Z_k - conj Z_{n-k}) / 2
    out[k] = cadd(ev, cmul(p.tw_r2c[k], od));
  }
}

// Back-projection rows, persistent: one CTA per resident slot walks the rows (m, jj) of every
// slice; each row is sampled (theta-combined when the combined detector row fits in bufB),
// transformed and written as k_rows_fwd<true> does.  The rho twiddles are read through L1, so a
// CTA holds two row buffers and, at 48 registers, five CTAs share an SM.
template <int SEQ>
__global__ void __launch_bounds__(kThreads, 5) k_rows_bp_persistent(DevPlan p, int n_rows) {
  extern __shared__ __align__(16) float2 smem[];
  const int nc = p.nc;
  float2* bufA = smem;
  float2* bufB = smem + nc;
  const float2* tws = p.tw_rho;  // read through L1: two buffers per CTA leave room for a fifth CTA per SM
  float* comb = p.sino_pitch + 2 * kCombGuard <= 2 * nc ? reinterpret_cast<float*>(bufB) + kCombGuard : nullptr;
  const int per_slice = p.M * p.nh;
  for (int R = blockIdx.x; R < n_rows; R += gridDim.x) {
    const int b = R / per_slice, mj = R - b * per_slice, m = mj / p.nh, jj = mj - m * p.nh;
    __syncthreads();  // the previous row's buffers
    const float2* Z;
    if (SEQ >= 0 && comb && p.interp == 3) {
      // the compiled transform's first pass samples the combined row (in bufB) itself
      sample_row_backproject(p, b, m, jj, nullptr, comb);
      const int2 cj = p.bp_c[jj];
      Z = row_fft_in<SEQ>(CombSamples{CombSample{comb, p.bp_e, cj.x, __int_as_float(cj.y), p.sino_pitch}}, bufA,
                          bufB, p, tws);
    } else {
      sample_row_backproject(p, b, m, jj, reinterpret_cast<float*>(bufA), comb);
      __syncthreads();
      Z = row_fft<false, SEQ>(bufA, bufB, p, tws);
    }
    float2* out = p.xspec + b * p.bs_x + static_cast<size_t>(mj) * p.x_pitch;
    for (int k = threadIdx.x; k <= nc; k += blockDim.x) {
      const float2 zk = Z[k == nc ? 0 : k];
      const float2 zc = cconj(Z[k == 0 ? 0 : nc - k]);
      const float2 ev = cscale(cadd(zk, zc), 0.5f);
      const float2 dv = cscale(csub(zk, zc), 0.5f);
      const float2 od = make_float2(dv.y, -dv.x);  // -i (Z_k - conj Z_{n-k}) / 2
      out[k] = cadd(ev, cmul(p.tw_r2c[k], od));
    }
  }
}

// FFT along theta of col_group rho frequencies, multiply by the kernel, inverse FFT, keep the
// centre half plus the halo rows.
__global__ void __launch_bounds__(kThreads) k_columns(DevPlan p, const float2* __restrict__ kern) {
  extern __shared__ __align__(16) float2 smem[];
  const int nt = p.n_theta, nh = p.nh, nc = p.nc;
  const int G = p.col_group;
  float2* A = smem;
  float2* B = smem + G * nt;
  float2* tw = smem + 2 * G * nt;
  stage_table(tw, p.tw_th, nt, threadIdx.x, blockDim.x);
  const int m = blockIdx.y, kr0 = blockIdx.x * G, b = blockIdx.z;
  const float2* xin = p.xspec + b * p.bs_x + static_cast<size_t>(m) * nh * p.x_pitch;
  for (int idx = threadIdx.x; idx < G * nt; idx += blockDim.x) {
    const int g = idx % G, j = idx / G;
    const int jj = j - nh / 2;
    float2 v = make_float2(0.f, 0.f);
    if (jj >= 0 && jj < nh && kr0 + g <= nc) v = xin[static_cast<size_t>(jj) * p.x_pitch + kr0 + g];
    A[g * nt + j] = v;
  }
  __syncthreads();
  float2* S = fft_block<false>(A, B, G, nt, p.rad_th, tw, threadIdx.x, blockDim.x);
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
  const float2* Y = fft_block<true>(S, T, G, nt, p.rad_th, tw, threadIdx.x, blockDim.x);
  float2* yout = p.yspec + b * p.bs_ys + static_cast<size_t>(m) * (nh + kHaloLo + kHaloHi) * p.x_pitch;
  const int nrow = nh + kHaloLo + kHaloHi;
  for (int idx = threadIdx.x; idx < G * nrow; idx += blockDim.x) {
    const int g = idx % G, jr = idx / G;
    const int js = (jr + nh / 2 - kHaloLo + nt) % nt;  // the convolution output is nt-periodic
    if (kr0 + g <= nc) yout[static_cast<size_t>(jr) * p.x_pitch + kr0 + g] = Y[g * nt + js];
  }
}

// Specialised column kernel for n_theta = product of Rs: one work item is G rho frequencies of
// one partition, held interleaved ([row][g]) in shared
// memory and transformed in place.  The first forward pass reads the spectrum rows straight from
// global memory (rows outside the centre half are zero), the last forward pass multiplies by the
// kernel, and the last inverse pass writes only the kept rows (centre half plus halo).  The grid
// is persistent; the per-pass twiddles are staged once per CTA.
template <int G>
struct ColumnLoad {
  const float2* x;  // spectrum rows of this partition, x_pitch apart
  int x_pitch, nh, kr0, nc;
  __device__ __forceinline__ float2 operator()(int row, int g) const {
    const int jj = row - nh / 2;
    const bool live = jj >= 0 && jj < nh && kr0 + g <= nc;
    return live ? x[static_cast<size_t>(jj) * x_pitch + kr0 + g] : make_float2(0.f, 0.f);
  }
};
template <int G, int NN>
struct ColumnKernelStore {
  static constexpr bool kShared = true;
  float2* d;
  const float2* kern;  // [k_rho][k_theta], k_theta in [0, NN / 2]
  int kr0, nc;
  __device__ __forceinline__ void operator()(int row, int g, float2 v) const {
    const int kt = row <= NN - row ? row : NN - row;
    const int kr = kr0 + g <= nc ? kr0 + g : nc;  // columns past nc are computed but never stored
    d[row * G + g] = cmul(v, kern[static_cast<size_t>(kr) * (NN / 2 + 1) + kt]);
  }
};
template <int G, int NN>
struct ColumnStore {
  static constexpr bool kShared = false;
  float2* y;  // kept rows of this partition, x_pitch apart
  int x_pitch, nh, kr0, nc;
  __device__ __forceinline__ void operator()(int row, int g, float2 v) const {
    const int jr = (row - nh / 2 + kHaloLo + NN) % NN;  // the convolution output is NN-periodic
    if (jr < nh + kHaloLo + kHaloHi && kr0 + g <= nc) y[static_cast<size_t>(jr) * x_pitch + kr0 + g] = v;
  }
};

// The radix-7 lengths (1372, 2744) run their passes out of place between two buffers: their
// registers already hold them to 2 CTAs per SM, so the second buffer costs no occupancy, and each
// pass needs one barrier instead of two.
__host__ __device__ constexpr bool column_pingpong(int nn) { return nn % 7 == 0; }

template <int G, int TH, int MINB, int... Rs>
__global__ void __launch_bounds__(TH, MINB) k_columns_fixed(DevPlan p, const float2* __restrict__ kern, int n_items) {
  constexpr int NN = chain_length<Rs...>();
  constexpr int NTW = chain_twiddles<Rs...>();
  constexpr bool PP = column_pingpong(NN);
  extern __shared__ __align__(16) float2 smem[];
  float2* data = smem;
  float2* data2 = smem + NN * G;  // second buffer (PP)
  float2* tw = smem + (PP ? 2 : 1) * NN * G;
  stage_table(tw, p.tw_col, NTW, threadIdx.x, blockDim.x);
  // (the first pass's barrier orders these stores before any twiddle read)
  const int ngroups = (p.nc + G) / G;
  const int nrow = p.nh + kHaloLo + kHaloHi;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int gi = w % ngroups, mb = w / ngroups;
    const int m = mb % p.M, b = mb / p.M;
    const int kr0 = gi * G;
    const ColumnLoad<G> in{p.xspec + b * p.bs_x + static_cast<size_t>(m) * p.nh * p.x_pitch, p.x_pitch, p.nh, kr0,
                           p.nc};
    const ColumnStore<G, NN> out{p.yspec + b * p.bs_ys + static_cast<size_t>(m) * nrow * p.x_pitch, p.x_pitch, p.nh,
                                 kr0, p.nc};
    if constexpr (PP) {
      __syncthreads();  // the previous item's last pass has read both buffers
      // the last forward pass reads the buffer its predecessor wrote and writes the other one
      float2* fin = (sizeof...(Rs) % 2) ? data : data2;
      float2* oth = (sizeof...(Rs) % 2) ? data2 : data;
      const ColumnKernelStore<G, NN> mul{fin, kern, kr0, p.nc};
      PingPongChain<NN, G, TH, false, 1, 0, Rs...>::run(tw, in, data, data2, mul, threadIdx.x);
      PingPongChain<NN, G, TH, true, 1, 0, Rs...>::run(tw, SmemIn<G>{fin}, oth, fin, out, threadIdx.x);
    } else {
      const ColumnKernelStore<G, NN> mul{data, kern, kr0, p.nc};
      InplaceChain<NN, G, TH, false, 1, 0, Rs...>::run(tw, in, data, mul, threadIdx.x);
      InplaceChain<NN, G, TH, true, 1, 0, Rs...>::run(tw, SmemIn<G>{data}, data, out, threadIdx.x);
    }
  }
}

// Transposed theta pass of the exact transpose (k_columns_t's work with the specialised
// transform): the kept rows (centre half plus halo) are placed on their lattice rows (rows that
// alias when n_theta < n_theta_half + 4 are summed), transformed, multiplied by conj(K),
// transformed back, and the centre half is stored.
// The specialised lengths are at least 256, so n_theta >= n_theta_half + 4 rows: each lattice row
// holds at most one kept row (no aliasing to sum), and the load is one predicated read, which the
// pass issues together with its other loads.
template <int G, int NN>
struct ColumnLoadT {
  const float2* y;  // kept rows of this partition, x_pitch apart
  int x_pitch, nh, nrow, kr0, nc;
  __device__ __forceinline__ float2 operator()(int row, int g) const {
    const int jr = (row - nh / 2 + kHaloLo + NN) % NN;
    return (jr < nrow && kr0 + g <= nc) ? y[static_cast<size_t>(jr) * x_pitch + kr0 + g] : make_float2(0.f, 0.f);
  }
};
template <int G, int NN>
struct ColumnKernelStoreT {
  static constexpr bool kShared = true;
  float2* d;
  const float2* kern;  // [k_rho][k_theta], k_theta in [0, NN / 2]
  int kr0, nc;
  __device__ __forceinline__ void operator()(int row, int g, float2 v) const {
    const int kt = row <= NN - row ? row : NN - row;
    const int kr = kr0 + g <= nc ? kr0 + g : nc;
    d[row * G + g] = cmul(v, cconj(kern[static_cast<size_t>(kr) * (NN / 2 + 1) + kt]));
  }
};
template <int G, int NN>
struct ColumnStoreT {
  static constexpr bool kShared = false;
  float2* x;  // centre-half rows of this partition, x_pitch apart
  int x_pitch, nh, kr0, nc;
  __device__ __forceinline__ void operator()(int row, int g, float2 v) const {
    const int jj = row - nh / 2;
    if (jj >= 0 && jj < nh && kr0 + g <= nc) x[static_cast<size_t>(jj) * x_pitch + kr0 + g] = v;
  }
};

template <int G, int TH, int MINB, int... Rs>
__global__ void __launch_bounds__(TH, MINB) k_columns_fixed_t(DevPlan p, const float2* __restrict__ kern, int n_items) {
  constexpr int NN = chain_length<Rs...>();
  static_assert(NN >= 8, "n_theta = 2 n_theta_half >= n_theta_half + 4 kept rows (ColumnLoadT)");
  constexpr int NTW = chain_twiddles<Rs...>();
  extern __shared__ __align__(16) float2 smem[];
  float2* data = smem;
  float2* tw = smem + NN * G;
  stage_table(tw, p.tw_col, NTW, threadIdx.x, blockDim.x);
  const int ngroups = (p.nc + G) / G;
  const int nrow = p.nh + kHaloLo + kHaloHi;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int gi = w % ngroups, mb = w / ngroups;
    const int m = mb % p.M, b = mb / p.M;
    const int kr0 = gi * G;
    const ColumnLoadT<G, NN> in{p.yspec + b * p.bs_ys + static_cast<size_t>(m) * nrow * p.x_pitch, p.x_pitch, p.nh,
                                nrow, kr0, p.nc};
    const ColumnKernelStoreT<G, NN> mul{data, kern, kr0, p.nc};
    InplaceChain<NN, G, TH, false, 1, 0, Rs...>::run(tw, in, data, mul, threadIdx.x);
    const ColumnStoreT<G, NN> out{p.xspec + b * p.bs_x + static_cast<size_t>(m) * p.nh * p.x_pitch, p.x_pitch, p.nh,
                                  kr0, p.nc};
    InplaceChain<NN, G, TH, true, 1, 0, Rs...>::run(tw, SmemIn<G>{data}, data, out, threadIdx.x);
  }
}

template <int G, int TH, int MINB, int... Rs>
constexpr bool column_radices_match(const ColumnRadices& c) {
  int i = 0;
  bool ok = c.G == G && c.TH == TH && c.MINB == MINB;
  ((ok = ok && i < 4 && c.r[i] == Rs, ++i), ...);
  return ok && (i == 4 || c.r[i] == 0) && c.n == chain_length<Rs...>();
}

// The instantiations, in kColumnRadices order.
#define RADON_COLUMN_KERNELS(X)  \
  X(0, 32, 256, 2, 16, 16)       \
  X(1, 16, 256, 2, 8, 8, 8)      \
  X(2, 8, 256, 2, 16, 8, 8)      \
  X(3, 4, 256, 2, 16, 16, 8)     \
  X(4, 2, 256, 2, 16, 16, 16)    \
  X(5, 1, 256, 2, 16, 16, 16, 2) \
  X(6, 4, 392, 2, 14, 14, 7)    \
  X(7, 2, 392, 2, 14, 14, 14)

#define RADON_CHECK_COLUMN(i, ...) \
  static_assert(column_radices_match<__VA_ARGS__>(kColumnRadices[i]), "column radix table");
RADON_COLUMN_KERNELS(RADON_CHECK_COLUMN)
#undef RADON_CHECK_COLUMN
static_assert(kNumColumnRadices == 8, "every kColumnRadices entry has an instantiation");

template <int G, int TH, int MINB, int... Rs>
size_t columns_fixed_smem() {
  constexpr int NN = chain_length<Rs...>();
  return (static_cast<size_t>(NN) * G * (column_pingpong(NN) ? 2 : 1) + chain_twiddles<Rs...>()) * sizeof(float2);
}
// The transposed theta pass keeps its passes in place: one buffer.
template <int G, int TH, int MINB, int... Rs>
size_t columns_fixed_t_smem() {
  constexpr int NN = chain_length<Rs...>();
  return (static_cast<size_t>(NN) * G + chain_twiddles<Rs...>()) * sizeof(float2);
}

template <int G, int TH, int MINB, int... Rs>
cudaError_t launch_columns_fixed(const DevPlan& p, const float2* kern, cudaStream_t st, int batch) {
  const int n_items = (p.nc + G) / G * p.M * batch;
  const int grid = n_items < p.col_blocks ? n_items : p.col_blocks;
  k_columns_fixed<G, TH, MINB, Rs...><<<grid, TH, columns_fixed_smem<G, TH, MINB, Rs...>(), st>>>(p, kern, n_items);
  return cudaSuccess;
}

template <int G, int TH, int MINB, int... Rs>
cudaError_t launch_columns_fixed_t(const DevPlan& p, const float2* kern, cudaStream_t st, int batch) {
  const int n_items = (p.nc + G) / G * p.M * batch;
  const int grid = n_items < p.col_blocks_t ? n_items : p.col_blocks_t;
  k_columns_fixed_t<G, TH, MINB, Rs...><<<grid, TH, columns_fixed_t_smem<G, TH, MINB, Rs...>(), st>>>(p, kern, n_items);
  return cudaSuccess;
}

// Raises the kernel's shared memory limit and sizes its persistent grid (resident CTAs).
template <int G, int TH, int MINB, int... Rs>
cudaError_t configure_columns_fixed(DevPlan& p, int optin, int n_sm) {
  const size_t smem = columns_fixed_smem<G, TH, MINB, Rs...>();
  if (smem > static_cast<size_t>(optin)) return cudaErrorInvalidValue;
  auto* fn = k_columns_fixed<G, TH, MINB, Rs...>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TH, smem);
  if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidValue;
  p.col_blocks = per_sm * n_sm;
  auto* fn_t = k_columns_fixed_t<G, TH, MINB, Rs...>;
  int per_sm_t = 0;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn_t, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_t, fn_t, TH, columns_fixed_t_smem<G, TH, MINB, Rs...>());
  p.col_blocks_t = per_sm_t * n_sm;  // 0: the transpose keeps the generic theta pass
  return e;
}

// Inverse real FFT along rho of one kept row; writes N_rho values plus kPad wrap columns per side.
template <int SEQ>
__global__ void __launch_bounds__(kThreads) k_rows_inv(DevPlan p) {
  extern __shared__ __align__(16) float2 smem[];
  const int nc = p.nc, nr = p.N_rho;
  float2* bufA = smem;
  float2* bufB = smem + nc;
  float2* tws = smem + 2 * nc;
  if (p.rows_tw_smem) stage_table(tws, p.tw_rho, nc, threadIdx.x, blockDim.x);
  const float2* tw = p.rows_tw_smem ? tws : p.tw_rho;
  const int row = blockIdx.x, m = blockIdx.y, b = blockIdx.z;
  const int nrow = p.nh + kHaloLo + kHaloHi;
  const float2* X = p.yspec + b * p.bs_ys + (static_cast<size_t>(m) * nrow + row) * p.x_pitch;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const float2 xk = X[k];
    const float2 xc = cconj(X[nc - k]);
    const float2 sm = cadd(xk, xc);
    const float2 df = cmulc(csub(xk, xc), p.tw_r2c[k]);  // (X_k - conj X_{n-k}) exp(+2 pi i k / N_rho)
    bufA[k] = make_float2(sm.x - df.y, sm.y + df.x);      // + i * df
  }
  __syncthreads();
  const float2* Z = row_fft<true, SEQ>(bufA, bufB, p, tw);
  const float* h = reinterpret_cast<const float*>(Z);
  float* y = p.ylp + b * p.bs_y + (static_cast<size_t>(m) * nrow + row) * p.y_pitch;
  for (int c = static_cast<int>(threadIdx.x) - kPad; c < nr + kPad; c += blockDim.x) {
    const int src = c < 0 ? c + nr : (c >= nr ? c - nr : c);
    y[c + kPad] = h[src];
  }
}

// ------------------------------------------------------------------------------------------
// Persistent row transforms.  One CTA per resident slot walks the rows R = blockIdx.x,
// blockIdx.x + gridDim.x, ...; the twiddle table is staged once per CTA, and while row R is
// transformed the next row is already being copied into the other staging buffer with cp.async
// (16-byte asynchronous copies that bypass the registers), so the load latency that stalls the
// one-row-per-CTA kernels overlaps the FFT.  Results equal those of k_rows_fwd<false> /
// k_rows_inv bit for bit (same arithmetic in the same order).

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Shared-memory layout of the persistent row kernels (float2 entries): twiddles (nc, rounded up
// to even), two staging buffers of x_pitch entries, one work buffer of nc.
__host__ __device__ __forceinline__ int rows_pipe_stage0(const DevPlan& p) { return (p.nc + 1) & ~1; }

// Input k of the inverse real transform's half-length complex FFT, from the half spectrum X
// (k in [0, nc)): Z_k = (X_k + conj X_{nc-k}) + i (X_k - conj X_{nc-k}) exp(+2 pi i k / N_rho).
struct C2RInput {
  const float2* X;
  const float2* __restrict__ tw_r2c;
  int nc;
  __device__ __forceinline__ float2 operator()(int k) const {
    const float2 xk = X[k];
    const float2 xc = cconj(X[nc - k]);
    const float2 sm = cadd(xk, xc);
    const float2 df = cmulc(csub(xk, xc), tw_r2c[k]);
    return make_float2(sm.x - df.y, sm.y + df.x);
  }
};

// Output i of the inverse transform (real samples 2i, 2i + 1 of the row) to a log-polar row y
// of N_rho values plus kPad periodic wrap columns on each side (y[c + kPad] = h[c mod N_rho] for
// c in [-kPad, N_rho + kPad)).
struct RealRowOut {
  float* y;
  int nr;
  __device__ __forceinline__ void operator()(int i, float2 v) const {
    const int s = 2 * i;
    y[s + kPad] = v.x;
    y[s + 1 + kPad] = v.y;
    if (s < kPad) y[s + nr + kPad] = v.x;
    if (s + 1 < kPad) y[s + 1 + nr + kPad] = v.y;
    if (s >= nr - kPad) y[s - nr + kPad] = v.x;
    if (s + 1 >= nr - kPad) y[s + 1 - nr + kPad] = v.y;
  }
};

// Copy the first 16-byte chunks [0, chunks) of a spectrum-scratch row into shared memory.
__device__ __forceinline__ void prefetch_row(float2* dst, const float2* __restrict__ src, int chunks) {
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) cp_async16(dst + 2 * c, src + 2 * c);
}

// Forward: the rows k_sample_fwd wrote (n_rows = M nh per slice, batch slices), real FFT along
// rho, half spectrum to xspec.
template <int SEQ>
__global__ void __launch_bounds__(kThreads) k_rows_fwd_pipe(DevPlan p, int n_rows) {
  extern __shared__ __align__(16) float2 smem[];
  const int nc = p.nc, s0 = rows_pipe_stage0(p);
  float2* tws = smem;
  float2* stg0 = smem + s0;
  float2* stg1 = stg0 + p.x_pitch;
  float2* work = stg1 + p.x_pitch;
  stage_table(tws, p.tw_rho, nc, threadIdx.x, blockDim.x);
  const int per_slice = p.M * p.nh, chunks = (nc + 1) / 2;
  auto src_row = [&](int R) {
    const int b = R / per_slice;
    return p.yspec + b * p.bs_ys + static_cast<size_t>(R - b * per_slice) * p.x_pitch;
  };
  int R = blockIdx.x;
  if (R < n_rows) prefetch_row(stg0, src_row(R), chunks);
  cp_async_commit();
  for (int it = 0; R < n_rows; R += gridDim.x, ++it) {
    float2* cur = (it & 1) ? stg1 : stg0;
    if (R + static_cast<int>(gridDim.x) < n_rows) prefetch_row((it & 1) ? stg0 : stg1, src_row(R + gridDim.x), chunks);
    cp_async_commit();
    cp_async_wait_prev();  // this thread's copies of row R have landed
    __syncthreads();       // and everyone's
    const float2* Z = row_fft<false, SEQ>(cur, work, p, tws);
    const int b = R / per_slice;
    float2* out = p.xspec + b * p.bs_x + static_cast<size_t>(R - b * per_slice) * p.x_pitch;
    for (int k = threadIdx.x; k <= nc; k += blockDim.x) {
      const float2 zk = Z[k == nc ? 0 : k];
      const float2 zc = cconj(Z[k == 0 ? 0 : nc - k]);
      const float2 ev = cscale(cadd(zk, zc), 0.5f);
      const float2 dv = cscale(csub(zk, zc), 0.5f);
      const float2 od = make_float2(dv.y, -dv.x);  // -i (Z_k - conj Z_{n-k}) / 2
      out[k] = cadd(ev, cmul(p.tw_r2c[k], od));
    }
    __syncthreads();  // cur and work are overwritten by the next iteration
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Inverse: the kept rows after the theta convolution (n_rows = M (nh + halo) per slice), inverse
// real FFT along rho, N_rho values plus kPad wrap columns per side to the log-polar array.
template <int SEQ>
__global__ void __launch_bounds__(kThreads) k_rows_inv_pipe(DevPlan p, int n_rows) {
  extern __shared__ __align__(16) float2 smem[];
  const int nc = p.nc, nr = p.N_rho, s0 = rows_pipe_stage0(p);
  float2* tws = smem;
  float2* stg0 = smem + s0;
  float2* stg1 = stg0 + p.x_pitch;
  float2* work = stg1 + p.x_pitch;
  stage_table(tws, p.tw_rho, nc, threadIdx.x, blockDim.x);
  const int nrow = p.nh + kHaloLo + kHaloHi, per_slice = p.M * nrow, chunks = (nc + 2) / 2;
  auto src_row = [&](int R) {
    const int b = R / per_slice;
    return p.yspec + b * p.bs_ys + static_cast<size_t>(R - b * per_slice) * p.x_pitch;
  };
  int R = blockIdx.x;
  if (R < n_rows) prefetch_row(stg0, src_row(R), chunks);
  cp_async_commit();
  for (int it = 0; R < n_rows; R += gridDim.x, ++it) {
    const float2* X = (it & 1) ? stg1 : stg0;
    if (R + static_cast<int>(gridDim.x) < n_rows) prefetch_row((it & 1) ? stg0 : stg1, src_row(R + gridDim.x), chunks);
    cp_async_commit();
    cp_async_wait_prev();
    __syncthreads();
    const int b = R / per_slice, mr = R - b * per_slice;  // mr = m nrow + row
    float* y = p.ylp + b * p.bs_y + static_cast<size_t>(mr) * p.y_pitch;
    if constexpr (SEQ >= 0) {
      // the compiled transform's first pass forms its inputs from the staged row itself, and its
      // last pass writes the real row (with its wrap columns) straight to the log-polar array
      RowFft<SEQ, true>::run_in_out(C2RInput{X, p.tw_r2c, nc}, work, const_cast<float2*>(X), tws, RealRowOut{y, nr});
    } else {
      for (int k = threadIdx.x; k < nc; k += blockDim.x) work[k] = C2RInput{X, p.tw_r2c, nc}(k);
      __syncthreads();
      const float* h = reinterpret_cast<const float*>(row_fft<true, SEQ>(work, const_cast<float2*>(X), p, tws));
      for (int c = static_cast<int>(threadIdx.x) - kPad; c < nr + kPad; c += blockDim.x) {
        const int src = c < 0 ? c + nr : (c >= nr ? c - nr : c);
        y[c + kPad] = h[src];
      }
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ------------------------------------------------------------------------------------------
// Output gathers.

// Interpolant of partition m's log-polar coefficients at (halo row It + at, padded column
// Ir + ar), times lp_gain(p) (36 for cubic: the weights are taken times 6 per axis and the caller
// applies 1 / lp_gain once); taps are clamped into the array.  The coefficients are plain global
// rows (measured faster than gathers from a texture copy, which also needed a surface store per
// value in the inverse rho pass).
__device__ __forceinline__ float lp_gain_inv(const DevPlan& p) { return p.interp == 3 ? 1.f / 36.f : 1.f; }

__device__ __forceinline__ float sample_lp(const DevPlan& p, int b, int m, int It, float at, int Ir, float ar) {
  const int nrow = p.nh + kHaloLo + kHaloHi;
  const float* __restrict__ y = p.ylp + b * p.bs_y + static_cast<size_t>(m) * nrow * p.y_pitch;
  if (p.interp == 3) {
    float2 w[4];  // .x: theta weights, .y: rho weights
    bspline_w6_pair(make_float2(at, ar), w);
    const float wt[4] = {w[0].x, w[1].x, w[2].x, w[3].x}, wr[4] = {w[0].y, w[1].y, w[2].y, w[3].y};
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
  const int a = blockIdx.y, b = blockIdx.z;
  const int k = blockIdx.x * 128 + threadIdx.x;
  sino += static_cast<size_t>(b) * p.n_angles * p.n_det;
  const int nd = p.n_det;
  if (k >= nd) return;
  float out = 0.f;
  if (k >= p.live_lo && k <= p.live_hi) {
    const int4 ang = p.fwd_ang[a];
    const int4 anc = p.fwd_anc[static_cast<size_t>(a) * p.n_ktiles + k / kKTile];
    const int n = k - (k / kKTile) * kKTile;
    const float cr = fmaf(small_log1p(static_cast<float>(n) * __int_as_float(anc.z)), p.inv_drho, __int_as_float(anc.y));
    const float fr = floorf(cr);
    out = sample_lp(p, b, ang.x, ang.z, __int_as_float(ang.w), anc.x + static_cast<int>(fr), cr - fr) *
          (p.inv_aR * lp_gain_inv(p));
  }
  sino[static_cast<size_t>(a) * nd + k] = out;
}

constexpr int kCombMax = 1024;  // columns of the theta-combined row one scatter CTA may touch

// R# g(x) = sum_m interpolant of partition m at the log-polar coordinates of T_m x.
__global__ void __launch_bounds__(kPTile * kPTile, 6) k_gather_image(DevPlan p, float* __restrict__ img) {
  const int N = p.N;
  const int tj = blockIdx.x, ti = blockIdx.y, b = blockIdx.z;
  img += static_cast<size_t>(b) * N * N;
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
      const float dth = small_atan2(cross, r2 + ydot);
      const float drho = 0.5f * small_log1p(fmaf(2.f, ydot, fmaf(dy1, dy1, dy2 * dy2)) * __int_as_float(a1.z));
      const float ct = fmaf(dth, p.inv_dphi, __int_as_float(a0.y));
      const float cr = fmaf(drho, p.inv_drho, __int_as_float(a0.w));
      const float ft = floorf(ct), fr = floorf(cr);
      acc += sample_lp(p, b, m, a0.x + static_cast<int>(ft), ct - ft, a0.z + static_cast<int>(fr), cr - fr);
    }
  }
  img[static_cast<size_t>(i) * N + j] = acc * lp_gain_inv(p);
}

// ------------------------------------------------------------------------------------------
// Exact transpose R^T of the discrete forward map (the launches above, in reverse order, each
// replaced by its transpose).  Gathers become scatters (atomic adds at the same taps with the
// same weights and coordinates), the convolution with K becomes the convolution with conj(K)
// from the kept rows back to the centre half, and the pre-filter becomes Q^T = Q followed by the
// disc mask.  The log-polar scatter target is yspec read as real rows of 2 x_pitch floats.

// Padded index inside the image (not in the kPad zero border) of a P = N + 2 kPad wide array.
__device__ __forceinline__ bool interior_tap(int c, int P) { return c >= kPad && c < P - kPad; }

__device__ __forceinline__ float* lp_real_rows(const DevPlan& p, int b) {
  return reinterpret_cast<float*>(p.yspec + b * p.bs_ys);
}

// Transpose of k_gather_sino (cubic) with the theta weights applied last: a sinogram row reads
// the same four log-polar rows with the same theta weights for every bin, so the CTA's bins
// first add their rho-weighted values into one shared row over the columns they reach
// (shared-memory atomics), and that row is then spread onto the four log-polar rows with the theta
// weights: one global atomic per touched column and row instead of 16 per bin.  Equal to
// k_scatter_sino up to FP32 rounding.  CTAs whose bins span more than kCombMax columns take the
// per-bin path.
__global__ void __launch_bounds__(128) k_scatter_sino_comb(DevPlan p, const float* __restrict__ sino) {
  __shared__ float comb[kCombMax];
  __shared__ int red[2];
  const int a = blockIdx.y, b = blockIdx.z;
  const int k = blockIdx.x * 128 + threadIdx.x;
  const int nd = p.n_det;
  const bool live = k < nd && k >= p.live_lo && k <= p.live_hi;
  const int4 ang = p.fwd_ang[a];
  float v = 0.f, ar = 0.f;
  int c0 = INT_MAX;
  if (live) {
    v = __ldg(sino + (static_cast<size_t>(b) * p.n_angles + a) * nd + k) * (p.inv_aR * lp_gain_inv(p));
    const int4 anc = p.fwd_anc[static_cast<size_t>(a) * p.n_ktiles + k / kKTile];
    const int n = k - (k / kKTile) * kKTile;
    const float cr = fmaf(small_log1p(static_cast<float>(n) * __int_as_float(anc.z)), p.inv_drho, __int_as_float(anc.y));
    const float fr = floorf(cr);
    ar = cr - fr;
    c0 = clampi(anc.x + static_cast<int>(fr) - 1, 0, p.y_pitch - 4);
  }
  if (threadIdx.x == 0) {
    red[0] = INT_MAX;
    red[1] = INT_MAX;
  }
  __syncthreads();
  const int wmin = __reduce_min_sync(0xffffffffu, c0);
  const int wmaxn = __reduce_min_sync(0xffffffffu, live ? -c0 : INT_MAX);
  if ((threadIdx.x & 31) == 0 && wmin != INT_MAX) {
    atomicMin(red + 0, wmin);
    atomicMin(red + 1, wmaxn);
  }
  __syncthreads();
  if (red[0] == INT_MAX) return;  // uniform: no live bin
  const int lo = red[0], W = -red[1] + 3 - lo + 1;
  float2 w[4];  // .x: theta weights, .y: rho weights (times 6 each)
  bspline_w6_pair(make_float2(__int_as_float(ang.w), ar), w);
  const int nrow = p.nh + kHaloLo + kHaloHi, nr = p.N_rho, yp = 2 * p.x_pitch, wrap_end = nr + 2 * kPad;
  float* y = lp_real_rows(p, b) + static_cast<size_t>(ang.x) * nrow * yp;
  const int r0 = clampi(ang.z - 1, 0, nrow - 4);
  if (W > kCombMax) {  // uniform: per-bin taps
    if (!live || v == 0.f) return;
#pragma unroll
    for (int dt = 0; dt < 4; ++dt) {
      float* row = y + static_cast<size_t>(r0 + dt) * yp;
      const float vt = v * w[dt].x;
#pragma unroll
      for (int dc = 0; dc < 4; ++dc) {
        const int pc = c0 + dc;
        if (pc >= wrap_end) continue;
        int col = pc - kPad;
        col = col < 0 ? col + nr : (col >= nr ? col - nr : col);
        atomicAdd(row + col, vt * w[dc].y);
      }
    }
    return;
  }
  for (int j = threadIdx.x; j < W; j += blockDim.x) comb[j] = 0.f;
  __syncthreads();
  if (live && v != 0.f) {
#pragma unroll
    for (int dc = 0; dc < 4; ++dc) atomicAdd(comb + (c0 - lo + dc), v * w[dc].y);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < W; j += blockDim.x) {
    const float cv = comb[j];
    const int pc = lo + j;
    if (cv == 0.f || pc >= wrap_end) continue;
    int col = pc - kPad;
    col = col < 0 ? col + nr : (col >= nr ? col - nr : col);
#pragma unroll
    for (int dt = 0; dt < 4; ++dt) atomicAdd(y + static_cast<size_t>(r0 + dt) * yp + col, cv * w[dt].x);
  }
}

// Transpose of k_gather_sino: g(theta_a, s_k) / a_R is added to the 16 (cubic) or 4 (linear)
// log-polar coefficients the gather reads.  Padded column c holds rho index (c - kPad) mod
// N_rho (the wrap columns written by k_rows_inv), so the scatter wraps the same way.
__global__ void __launch_bounds__(128) k_scatter_sino(DevPlan p, const float* __restrict__ sino) {
  const int a = blockIdx.y, b = blockIdx.z;
  const int k = blockIdx.x * 128 + threadIdx.x;
  const int nd = p.n_det;
  if (k >= nd || k < p.live_lo || k > p.live_hi) return;
  const float v = __ldg(sino + (static_cast<size_t>(b) * p.n_angles + a) * nd + k) * (p.inv_aR * lp_gain_inv(p));
  if (v == 0.f) return;
  const int4 ang = p.fwd_ang[a];
  const int4 anc = p.fwd_anc[static_cast<size_t>(a) * p.n_ktiles + k / kKTile];
  const int n = k - (k / kKTile) * kKTile;
  const float cr = fmaf(small_log1p(static_cast<float>(n) * __int_as_float(anc.z)), p.inv_drho, __int_as_float(anc.y));
  const float fr = floorf(cr);
  const int It = ang.z, Ir = anc.x + static_cast<int>(fr);
  const float at = __int_as_float(ang.w), ar = cr - fr;
  const int nrow = p.nh + kHaloLo + kHaloHi, nr = p.N_rho, yp = 2 * p.x_pitch, wrap_end = nr + 2 * kPad;
  float* y = lp_real_rows(p, b) + static_cast<size_t>(ang.x) * nrow * yp;
  if (p.interp == 3) {
    float2 w[4];  // .x: theta weights, .y: rho weights (times 6 each)
    bspline_w6_pair(make_float2(at, ar), w);
    const int r0 = clampi(It - 1, 0, nrow - 4), c0 = clampi(Ir - 1, 0, p.y_pitch - 4);
#pragma unroll
    for (int dt = 0; dt < 4; ++dt) {
      float* row = y + static_cast<size_t>(r0 + dt) * yp;
      const float vt = v * w[dt].x;
#pragma unroll
      for (int dc = 0; dc < 4; ++dc) {
        const int pc = c0 + dc;
        if (pc >= wrap_end) continue;
        int col = pc - kPad;
        col = col < 0 ? col + nr : (col >= nr ? col - nr : col);
        atomicAdd(row + col, vt * w[dc].y);
      }
    }
  } else {
    const int r0 = clampi(It, 0, nrow - 2), c0 = clampi(Ir, 0, p.y_pitch - 2);
    const float wt[2] = {1.f - at, at}, wr[2] = {1.f - ar, ar};
#pragma unroll
    for (int dt = 0; dt < 2; ++dt) {
      float* row = y + static_cast<size_t>(r0 + dt) * yp;
#pragma unroll
      for (int dc = 0; dc < 2; ++dc) {
        const int pc = c0 + dc;
        if (pc >= wrap_end) continue;
        int col = pc - kPad;
        col = col < 0 ? col + nr : (col >= nr ? col - nr : col);
        atomicAdd(row + col, v * wt[dt] * wr[dc]);
      }
    }
  }
}

// Real FFT along rho of one kept row, in place: the row's N_rho reals become its half spectrum
// (N_rho/2 + 1 bins); same transform and post-processing as k_rows_fwd.
__global__ void __launch_bounds__(kThreads) k_rows_r2c_t(DevPlan p) {
  extern __shared__ __align__(16) float2 smem[];
  const int nc = p.nc;
  float2* bufA = smem;
  float2* bufB = smem + nc;
  float2* tws = smem + 2 * nc;
  if (p.rows_tw_smem) stage_table(tws, p.tw_rho, nc, threadIdx.x, blockDim.x);
  const float2* tw = p.rows_tw_smem ? tws : p.tw_rho;
  const int row = blockIdx.x, m = blockIdx.y, b = blockIdx.z;
  const int nrow = p.nh + kHaloLo + kHaloHi;
  float2* X = p.yspec + b * p.bs_ys + (static_cast<size_t>(m) * nrow + row) * p.x_pitch;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) bufA[k] = X[k];
  __syncthreads();  // the whole row is in shared memory before the first write below
  const float2* Z = fft_block<false>(bufA, bufB, 1, nc, p.rad_rho, tw, threadIdx.x, blockDim.x);
  for (int k = threadIdx.x; k <= nc; k += blockDim.x) {
    const float2 zk = Z[k == nc ? 0 : k];
    const float2 zc = cconj(Z[k == 0 ? 0 : nc - k]);
    const float2 ev = cscale(cadd(zk, zc), 0.5f);
    const float2 dv = cscale(csub(zk, zc), 0.5f);
    const float2 od = make_float2(dv.y, -dv.x);
    X[k] = cadd(ev, cmul(p.tw_r2c[k], od));
  }
}

// Transposed theta convolution of G rho frequencies: the kept rows (centre half plus halo) are
// placed at their lattice rows, transformed, multiplied by conj(K), transformed back, and the
// centre half is written to xspec.
__global__ void __launch_bounds__(kThreads) k_columns_t(DevPlan p, const float2* __restrict__ kern, int G) {
  extern __shared__ __align__(16) float2 smem[];
  const int nt = p.n_theta, nh = p.nh, nc = p.nc;
  const int nrow = nh + kHaloLo + kHaloHi;
  float2* A = smem;
  float2* B = smem + G * nt;
  float2* tw = smem + 2 * G * nt;
  stage_table(tw, p.tw_th, nt, threadIdx.x, blockDim.x);
  const int m = blockIdx.y, kr0 = blockIdx.x * G, b = blockIdx.z;
  const float2* yin = p.yspec + b * p.bs_ys + static_cast<size_t>(m) * nrow * p.x_pitch;
  for (int idx = threadIdx.x; idx < G * nt; idx += blockDim.x) {
    const int g = idx % G, j = idx / G;
    // kept rows jr = j - nh/2 + kHaloLo (mod nt) come from lattice row j; with nt < nrow (tiny
    // grids) two kept rows share a lattice row and the transpose sums them
    float2 v = make_float2(0.f, 0.f);
    if (kr0 + g <= nc)
      for (int jr = (j - nh / 2 + kHaloLo + nt) % nt; jr < nrow; jr += nt)
        v = cadd(v, yin[static_cast<size_t>(jr) * p.x_pitch + kr0 + g]);
    A[g * nt + j] = v;
  }
  __syncthreads();
  float2* S = fft_block<false>(A, B, G, nt, p.rad_th, tw, threadIdx.x, blockDim.x);
  float2* T = (S == A) ? B : A;
  const int nkt = nt / 2 + 1;
  for (int idx = threadIdx.x; idx < G * nt; idx += blockDim.x) {
    const int g = idx / nt, pp = idx - g * nt;
    const int kr = kr0 + g;
    if (kr <= nc) {
      const int kt = pp <= nt - pp ? pp : nt - pp;
      S[idx] = cmul(S[idx], cconj(kern[static_cast<size_t>(kr) * nkt + kt]));
    }
  }
  __syncthreads();
  const float2* Y = fft_block<true>(S, T, G, nt, p.rad_th, tw, threadIdx.x, blockDim.x);
  float2* xout = p.xspec + b * p.bs_x + static_cast<size_t>(m) * nh * p.x_pitch;
  for (int idx = threadIdx.x; idx < G * nh; idx += blockDim.x) {
    const int g = idx % G, jj = idx / G;
    if (kr0 + g <= nc) xout[static_cast<size_t>(jj) * p.x_pitch + kr0 + g] = Y[g * nt + jj + nh / 2];
  }
}

// Inverse real FFT along rho of one centre-half row of xspec (same pre-processing as
// k_rows_inv); the N_rho reals go to yspec row m nh + jj, where k_scatter_fwd reads them.
__global__ void __launch_bounds__(kThreads) k_rows_c2r_t(DevPlan p) {
  extern __shared__ __align__(16) float2 smem[];
  const int nc = p.nc, nr = p.N_rho;
  float2* bufA = smem;
  float2* bufB = smem + nc;
  float2* tws = smem + 2 * nc;
  if (p.rows_tw_smem) stage_table(tws, p.tw_rho, nc, threadIdx.x, blockDim.x);
  const float2* tw = p.rows_tw_smem ? tws : p.tw_rho;
  const int jj = blockIdx.x, m = blockIdx.y, b = blockIdx.z;
  const float2* X = p.xspec + b * p.bs_x + (static_cast<size_t>(m) * p.nh + jj) * p.x_pitch;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const float2 xk = X[k];
    const float2 xc = cconj(X[nc - k]);
    const float2 sm = cadd(xk, xc);
    const float2 df = cmulc(csub(xk, xc), p.tw_r2c[k]);
    bufA[k] = make_float2(sm.x - df.y, sm.y + df.x);
  }
  __syncthreads();
  const float2* Z = fft_block<true>(bufA, bufB, 1, nc, p.rad_rho, tw, threadIdx.x, blockDim.x);
  const float* h = reinterpret_cast<const float*>(Z);
  float* out = reinterpret_cast<float*>(p.yspec + b * p.bs_ys + (static_cast<size_t>(m) * p.nh + jj) * p.x_pitch);
  for (int c = threadIdx.x; c < nr; c += blockDim.x) out[c] = h[c];
}

// Transpose of k_sample_fwd: the same warps, anchors, ranges and FP32 coordinates; each fine
// sample adds h(phi_j, rho_i) e^rho_i / r times its tap weights to the padded coefficient image
// coef_img (zeroed beforehand).  Tap blocks are bounds-checked like sample_image, and taps in the
// zero border are dropped (the forward reads them as constants), so the border stays zero.
//
// The CTA's 8 rays x 64 rho samples x r sub-angles cover a thin wedge of the image (about
// 40 x 65 pixels at N = 2048).  Their taps are first summed in a shared-memory box over the
// wedge's bounding rectangle (found by a first pass over the same coordinates), and the box is
// then added to coef_img with one global atomic per touched pixel: about 30x fewer global atomics
// than one per tap.  A CTA whose rectangle exceeds kScatterBox floats adds its taps to coef_img
// directly.
constexpr int kScatterBox = 10240;  // floats of the per-CTA accumulation box (40 KB)

struct ScatterTap {
  int ic, ir;
  float ac, ar;
};

// Tap-block corner of one fine sample and its fractions; false if the block is out of range.
__device__ __forceinline__ bool scatter_corner(int interp, const float4& a, float ey, float2 d, int P, ScatterTap& t) {
  const float Fc = fmaf(ey, d.x, a.y), Fr = fmaf(ey, d.y, a.w);
  const float fc = floorf(Fc), fr = floorf(Fr);
  t.ic = static_cast<int>(a.x + fc);
  t.ir = static_cast<int>(a.z + fr);
  t.ac = Fc - fc;
  t.ar = Fr - fr;
  if (interp == 3) return !(t.ic < 1 || t.ic > P - 3 || t.ir < 1 || t.ir > P - 3);
  return !(t.ic < 0 || t.ic > P - 2 || t.ir < 0 || t.ir > P - 2);
}

// Adds the SPAN x SPAN tap block with top-left padded index (rt, ct) and weights wr x wc to the
// box (origin (r0, c0), W x H) or to coef_img.  Into the box every tap goes, border ones included:
// the flush drops the box cells that lie in the zero border, which is the same as dropping those
// taps here, without two tests per tap.  The block lies inside the box by construction (the box is
// the bounding rectangle of these corners); one test per block guards that.  Straight into coef_img
// the border taps are dropped one by one.
template <int SPAN>
__device__ __forceinline__ void scatter_block(const float (&wc)[SPAN], const float (&wr)[SPAN], int rt, int ct, int P,
                                              bool use_box, float* box, int W, int H, int r0, int c0,
                                              float* __restrict__ img) {
  if (use_box) {
    const int by = rt - r0, bx = ct - c0;
    if (by < 0 || by + SPAN > H || bx < 0 || bx + SPAN > W) return;
    float* b0 = box + by * W + bx;
#pragma unroll
    for (int dr = 0; dr < SPAN; ++dr) {
      float* row = b0 + dr * W;
#pragma unroll
      for (int dc = 0; dc < SPAN; ++dc) atomicAdd(row + dc, wr[dr] * wc[dc]);
    }
    return;
  }
#pragma unroll
  for (int dr = 0; dr < SPAN; ++dr) {
    if (!interior_tap(rt + dr, P)) continue;
#pragma unroll
    for (int dc = 0; dc < SPAN; ++dc)
      if (interior_tap(ct + dc, P)) atomicAdd(img + static_cast<size_t>(rt + dr) * P + (ct + dc), wr[dr] * wc[dc]);
  }
}

__global__ void __launch_bounds__(kSampleWarps * 32) k_scatter_fwd(DevPlan p) {
  extern __shared__ __align__(16) float4 sanc[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = p.r, ne = p.n_eanc;
  const int tile0 = 2 * blockIdx.x, m = blockIdx.z % p.M, b = blockIdx.z / p.M;
  const int jj = blockIdx.y * kSampleWarps + warp;
  const bool active = jj < p.nh;  // inactive warps still take part in the CTA barriers
  float4* anc = sanc + warp * 2 * r;
  float2* dir = reinterpret_cast<float2*>(sanc + kSampleWarps * 2 * r) + warp * r;
  int2* rng = reinterpret_cast<int2*>(reinterpret_cast<float2*>(sanc + kSampleWarps * 2 * r) + kSampleWarps * r) + warp * r;
  float* box = reinterpret_cast<float*>(sanc + kSampleWarps * 3 * r);  // after anchors, directions and ranges
  int* red = reinterpret_cast<int*>(box + kScatterBox);                 // min col, -max col, min row, -max row
  const float4 um = p.fwd_m[m];
  const size_t row0 = (static_cast<size_t>(m) * p.nh + (active ? jj : 0)) * r;
  if (active) {
    const float4* rowc = p.fwd_row + row0;
    const float2 ea0 = p.fwd_eanc[tile0];
    const float2 ea1 = p.fwd_eanc[tile0 + 1 < ne ? tile0 + 1 : tile0];
    for (int q = lane; q < r; q += 32) {
      const float4 cs = rowc[q];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float2 ea = u ? ea1 : ea0;
        float ch, cl, rh, rl;
        df_mul_add(ea.x, ea.y, cs.x, cs.y, um.x, um.y, &ch, &cl);
        df_mul_add(ea.x, ea.y, cs.z, cs.w, um.z, um.w, &rh, &rl);
        const float Ic = floorf(ch), Ir = floorf(rh);
        anc[u * r + q] = make_float4(Ic, (ch - Ic) + cl, Ir, (rh - Ir) + rl);
      }
      dir[q] = make_float2(cs.x, cs.z);
      rng[q] = p.fwd_rng[row0 + q];
    }
  }
  if (threadIdx.x == 0) {
    red[0] = INT_MAX;
    red[1] = INT_MAX;
    red[2] = INT_MAX;
    red[3] = INT_MAX;
  }
  __syncthreads();
  // lane L takes the adjacent samples base + 2L and base + 2L + 1 (both in tile L / 16), so the
  // 32 lanes of one atomic instruction are two samples apart: fewer of them hit the same pixel
  const int base = tile0 * kETile;
  const int i0 = base + 2 * lane, i1 = i0 + 1, tl = lane >> 4;
  float v0 = 0.f, v1 = 0.f, ey0 = 0.f, ey1 = 0.f;
  if (active) {
    const float* hrow = reinterpret_cast<const float*>(p.yspec + b * p.bs_ys + (static_cast<size_t>(m) * p.nh + jj) * p.x_pitch);
    const float scale = p.interp == 3 ? 1.f / 36.f : 1.f;
    if (i0 < p.N_rho) {
      const float2 e = p.fwd_e[i0];
      v0 = hrow[i0] * e.x * scale;
      ey0 = e.y;
    }
    if (i1 < p.N_rho) {
      const float2 e = p.fwd_e[i1];
      v1 = hrow[i1] * e.x * scale;
      ey1 = e.y;
    }
  }
  const int P = p.img_pitch;
  // pass 1: bounding rectangle of the tap-block corners this CTA scatters to
  int cmin = INT_MAX, cmax = INT_MIN, rmin = INT_MAX, rmax = INT_MIN;
  if (active) {
    for (int q = 0; q < r; ++q) {
      const int2 rg = rng[q];
      if (rg.y < base || rg.x > base + 2 * kETile - 1) continue;
      const float2 d = dir[q];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int i = u ? i1 : i0;
        const float v = u ? v1 : v0;
        if (i < rg.x || i > rg.y || v == 0.f) continue;
        ScatterTap t;
        if (!scatter_corner(p.interp, anc[tl * r + q], u ? ey1 : ey0, d, P, t)) continue;
        cmin = min(cmin, t.ic);
        cmax = max(cmax, t.ic);
        rmin = min(rmin, t.ir);
        rmax = max(rmax, t.ir);
      }
    }
  }
  cmin = __reduce_min_sync(0xffffffffu, cmin);
  rmin = __reduce_min_sync(0xffffffffu, rmin);
  cmax = __reduce_max_sync(0xffffffffu, cmax);
  rmax = __reduce_max_sync(0xffffffffu, rmax);
  if (lane == 0 && cmin <= cmax) {
    atomicMin(red + 0, cmin);
    atomicMin(red + 1, -cmax);
    atomicMin(red + 2, rmin);
    atomicMin(red + 3, -rmax);
  }
  __syncthreads();
  if (red[0] == INT_MAX) return;  // uniform over the CTA: nothing to scatter
  const int span = p.interp == 3 ? 4 : 2;  // taps per axis
  const int c0 = red[0] - (p.interp == 3 ? 1 : 0), r0 = red[2] - (p.interp == 3 ? 1 : 0);
  const int W = -red[1] - red[0] + span, H = -red[3] - red[2] + span;
  const bool use_box = W * H <= kScatterBox;  // uniform over the CTA
  float* __restrict__ img = p.coef_img + b * p.bs_img;
  if (use_box) {
    for (int idx = threadIdx.x; idx < W * H; idx += blockDim.x) box[idx] = 0.f;
    __syncthreads();
  }
  // pass 2: the taps, into the box or straight into coef_img
  if (active) {
    for (int q = 0; q < r; ++q) {
      const int2 rg = rng[q];
      if (rg.y < base || rg.x > base + 2 * kETile - 1) continue;
      const float2 d = dir[q];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int i = u ? i1 : i0;
        const float v = u ? v1 : v0;
        if (i < rg.x || i > rg.y || v == 0.f) continue;
        ScatterTap t;
        if (!scatter_corner(p.interp, anc[tl * r + q], u ? ey1 : ey0, d, P, t)) continue;
        if (p.interp == 3) {
          float2 w[4];  // .x: column weights, .y: row weights (times 6 each)
          bspline_w6_pair(make_float2(t.ac, t.ar), w);
          float wc[4], wr[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            wc[k] = w[k].x;
            wr[k] = v * w[k].y;
          }
          scatter_block<4>(wc, wr, t.ir - 1, t.ic - 1, P, use_box, box, W, H, r0, c0, img);
        } else {
          const float wc[2] = {1.f - t.ac, t.ac}, wr[2] = {v * (1.f - t.ar), v * t.ar};
          scatter_block<2>(wc, wr, t.ir, t.ic, P, use_box, box, W, H, r0, c0, img);
        }
      }
    }
  }
  if (!use_box) return;
  __syncthreads();
  for (int idx = threadIdx.x; idx < W * H; idx += blockDim.x) {
    const float v = box[idx];
    if (v != 0.f) {
      const int by = idx / W, bx = idx - by * W;
      if (interior_tap(r0 + by, P) && interior_tap(c0 + bx, P))  // the zero border stays zero
        atomicAdd(img + static_cast<size_t>(r0 + by) * P + (c0 + bx), v);
    }
  }
}

// FBP: filter one sinogram row along s (Eq. FBP, Eq. ramp / SLfilt / cosfilt).  The row (bins
// with |s| >= 1 zeroed) is zero-padded to n_filt, transformed with the real FFT, multiplied by
// the real transfer function H (divided by n_filt) and transformed back; the first n_det values
// are the filtered row.  Bins k and n - k of the half spectrum are handled by one thread, so the
// spectrum is processed in place.
__global__ void __launch_bounds__(kThreads) k_sino_filter(DevPlan p, const float* __restrict__ g,
                                                          const float* __restrict__ H, float* __restrict__ out) {
  extern __shared__ __align__(16) float2 smem[];
  const int nf = p.n_filt / 2, nd = p.n_det, a = blockIdx.x;
  float2* bufA = smem;
  float2* bufB = smem + nf;
  float2* tws = smem + 2 * nf;
  if (p.filt_tw_smem) stage_table(tws, p.tw_filt, nf, threadIdx.x, blockDim.x);
  const float2* tw = p.filt_tw_smem ? tws : p.tw_filt;
  float* row = reinterpret_cast<float*>(bufA);
  const float* gr = g + static_cast<size_t>(a) * nd;
  for (int k = threadIdx.x; k < 2 * nf; k += blockDim.x)
    row[k] = (k >= p.live_lo && k <= p.live_hi) ? __ldg(gr + k) : 0.f;
  __syncthreads();
  float2* Z = fft_block<false>(bufA, bufB, 1, nf, p.rad_filt, tw, threadIdx.x, blockDim.x);
  for (int k = threadIdx.x; k <= nf / 2; k += blockDim.x) {
    const int km = (nf - k) % nf;  // partner bin (0 pairs with itself, giving bins 0 and nf)
    const float2 zk = Z[k], zm = Z[km];
    if (k == 0) {
      const float x0 = zk.x + zk.y, xn = zk.x - zk.y;  // bins 0 and nf of the real transform
      const float y0 = x0 * __ldg(H), yn = xn * __ldg(H + nf);
      Z[0] = make_float2(y0 + yn, y0 - yn);
      continue;
    }
    const float2 wk = p.tw_filt_r2c[k], wm = p.tw_filt_r2c[nf - k];
    // forward real-FFT post-processing for bins k and nf - k
    const float2 ck = cconj(zm), cm = cconj(zk);
    const float2 ek = cscale(cadd(zk, ck), 0.5f), dk = cscale(csub(zk, ck), 0.5f);
    const float2 em = cscale(cadd(zm, cm), 0.5f), dm = cscale(csub(zm, cm), 0.5f);
    const float2 xk = cadd(ek, cmul(wk, make_float2(dk.y, -dk.x)));
    const float2 xm = cadd(em, cmul(wm, make_float2(dm.y, -dm.x)));
    const float2 yk = cscale(xk, __ldg(H + k)), ym = cscale(xm, __ldg(H + nf - k));
    // inverse real-FFT pre-processing
    const float2 sk = cadd(yk, cconj(ym)), fk = cmulc(csub(yk, cconj(ym)), wk);
    const float2 sm = cadd(ym, cconj(yk)), fm = cmulc(csub(ym, cconj(yk)), wm);
    Z[k] = make_float2(sk.x - fk.y, sk.y + fk.x);
    if (km != k) Z[km] = make_float2(sm.x - fm.y, sm.y + fm.x);
  }
  __syncthreads();
  float2* other = (Z == bufA) ? bufB : bufA;
  const float2* Y = fft_block<true>(Z, other, 1, nf, p.rad_filt, tw, threadIdx.x, blockDim.x);
  const float* y = reinterpret_cast<const float*>(Y);
  float* o = out + static_cast<size_t>(a) * nd;
  for (int k = threadIdx.x; k < nd; k += blockDim.x) o[k] = y[k];
}

size_t filt_smem(const DevPlan& p) {
  return (2 + (p.filt_tw_smem ? 1 : 0)) * static_cast<size_t>(p.n_filt / 2) * sizeof(float2);
}

size_t rows_smem(const DevPlan& p) {
  return (2 + (p.rows_tw_smem ? 1 : 0)) * static_cast<size_t>(p.nc) * sizeof(float2);
}
size_t rows_pipe_smem(const DevPlan& p) {
  return (static_cast<size_t>(rows_pipe_stage0(p)) + 2 * static_cast<size_t>(p.x_pitch) + p.nc) * sizeof(float2);
}
size_t sample_fwd_smem(const DevPlan& p) {
  return static_cast<size_t>(kSampleWarps) * p.r * (2 * sizeof(float4) + sizeof(float2) + sizeof(int2));
}
size_t scatter_fwd_smem(const DevPlan& p) {
  return sample_fwd_smem(p) + kScatterBox * sizeof(float) + 4 * sizeof(int);
}
size_t cols_smem(const DevPlan& p) { return (2 * static_cast<size_t>(p.col_group) + 1) * p.n_theta * sizeof(float2); }
size_t cols_t_smem(const DevPlan& p, int G) { return (2 * static_cast<size_t>(G) + 1) * p.n_theta * sizeof(float2); }

// Forward sampling with fine-angle blocks for r = R sub-angles (tabulated pitches compiled in).
template <int R>
void launch_sample_arc(const DevPlan& p, dim3 grid, cudaStream_t st) {
  switch (p.img_pitch) {
#define RADON_LAUNCH_ARC(n)                                          \
  case n + 2 * kPad:                                                 \
    k_sample_fwd_arc<R, n + 2 * kPad><<<grid, R * 32, 0, st>>>(p);  \
    return;
    RADON_SAMPLE_PITCHES(RADON_LAUNCH_ARC)
#undef RADON_LAUNCH_ARC
    default:
      k_sample_fwd_arc<R, 0><<<grid, R * 32, 0, st>>>(p);
  }
}

template <bool BACK>
void launch_rows_forward(const DevPlan& p, cudaStream_t st, int batch) {
  if (BACK && p.rows_bp_blocks > 0) {
    const int n_rows = p.M * p.nh * batch;
    const int blocks = n_rows < p.rows_bp_blocks ? n_rows : p.rows_bp_blocks;
    switch (p.row_fixed) {
#define RADON_LAUNCH_ROWS_BP(i, ...) \
  case i: k_rows_bp_persistent<i><<<blocks, kThreads, 2 * p.nc * sizeof(float2), st>>>(p, n_rows); break;
      RADON_ROW_SEQUENCES(RADON_LAUNCH_ROWS_BP)
#undef RADON_LAUNCH_ROWS_BP
      default: k_rows_bp_persistent<-1><<<blocks, kThreads, 2 * p.nc * sizeof(float2), st>>>(p, n_rows); break;
    }
    return;
  }
  if (!BACK && p.rows_pipe_fwd > 0) {
    const int n_rows = p.M * p.nh * batch;
    const int blocks = n_rows < p.rows_pipe_fwd ? n_rows : p.rows_pipe_fwd;
    switch (p.row_fixed) {
#define RADON_LAUNCH_ROWS_FWD_PIPE(i, ...) \
  case i: k_rows_fwd_pipe<i><<<blocks, kThreads, rows_pipe_smem(p), st>>>(p, n_rows); break;
      RADON_ROW_SEQUENCES(RADON_LAUNCH_ROWS_FWD_PIPE)
#undef RADON_LAUNCH_ROWS_FWD_PIPE
      default: k_rows_fwd_pipe<-1><<<blocks, kThreads, rows_pipe_smem(p), st>>>(p, n_rows); break;
    }
    return;
  }
  const dim3 grid(p.nh, p.M, batch);
  switch (p.row_fixed) {
#define RADON_LAUNCH_ROWS_FWD(i, ...) \
  case i: k_rows_fwd<BACK, i><<<grid, kThreads, rows_smem(p), st>>>(p); break;
    RADON_ROW_SEQUENCES(RADON_LAUNCH_ROWS_FWD)
#undef RADON_LAUNCH_ROWS_FWD
    default: k_rows_fwd<BACK, -1><<<grid, kThreads, rows_smem(p), st>>>(p); break;
  }
}

void launch_columns_and_inverse(const DevPlan& p, const float2* kern, cudaStream_t st, const StageHook& hook,
                                int stage0, int batch) {
  if (p.col_group == 0) {
#define RADON_LAUNCH_COLUMN(i, ...) \
  case i: launch_columns_fixed<__VA_ARGS__>(p, kern, st, batch); break;
    switch (p.col_fixed) {
      RADON_COLUMN_KERNELS(RADON_LAUNCH_COLUMN)
      default: break;
    }
#undef RADON_LAUNCH_COLUMN
  } else {
    const int ngroups = (p.nc + 1 + p.col_group - 1) / p.col_group;
    k_columns<<<dim3(ngroups, p.M, batch), kThreads, cols_smem(p), st>>>(p, kern);
  }
  hook(stage0, st);
  if (p.rows_pipe_inv > 0) {
    const int n_rows = p.M * (p.nh + kHaloLo + kHaloHi) * batch;
    const int blocks = n_rows < p.rows_pipe_inv ? n_rows : p.rows_pipe_inv;
    switch (p.row_fixed) {
#define RADON_LAUNCH_ROWS_INV_PIPE(i, ...) \
  case i: k_rows_inv_pipe<i><<<blocks, kThreads, rows_pipe_smem(p), st>>>(p, n_rows); break;
      RADON_ROW_SEQUENCES(RADON_LAUNCH_ROWS_INV_PIPE)
#undef RADON_LAUNCH_ROWS_INV_PIPE
      default: k_rows_inv_pipe<-1><<<blocks, kThreads, rows_pipe_smem(p), st>>>(p, n_rows); break;
    }
    hook(stage0 + 1, st);
    return;
  }
  const dim3 grid(p.nh + kHaloLo + kHaloHi, p.M, batch);
  switch (p.row_fixed) {
#define RADON_LAUNCH_ROWS_INV(i, ...) \
  case i: k_rows_inv<i><<<grid, kThreads, rows_smem(p), st>>>(p); break;
    RADON_ROW_SEQUENCES(RADON_LAUNCH_ROWS_INV)
#undef RADON_LAUNCH_ROWS_INV
    default: k_rows_inv<-1><<<grid, kThreads, rows_smem(p), st>>>(p); break;
  }
  hook(stage0 + 1, st);
}

}  // namespace

// Raise the dynamic shared memory limit of a persistent forward / inverse row kernel pair to the
// device maximum `optin` (the limit is per function, shared by every plan, so it is never set
// lower) and report how many CTAs of each fit on one SM with `smem` bytes.
template <class KF, class KI>
cudaError_t configure_rows_pipe(KF* kf, KI* ki, int optin, size_t smem, int* per_sm_fwd, int* per_sm_inv) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, optin)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(ki, cudaFuncAttributeMaxDynamicSharedMemorySize, optin)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm_fwd, kf, kThreads, smem)) != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm_inv, ki, kThreads, smem);
}

// Raise a persistent kernel's dynamic shared memory limit to the device maximum and report how
// many of its CTAs fit on one SM with `smem` bytes.
template <class K>
cudaError_t configure_persistent(K* k, int optin, size_t smem, int* per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, kThreads, smem);
}

cudaError_t configure_kernels(DevPlan& p) {
  // The limit is a per-function attribute shared by every plan on the device: raise it to the
  // device's opt-in maximum (never to one plan's need, which a later, smaller plan would lower).
  cudaError_t e;
  int dev = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  p.rows_tw_smem = 1;  // stage the rho twiddles in shared memory when everything fits
  if (rows_smem(p) > static_cast<size_t>(optin)) p.rows_tw_smem = 0;
  p.filt_tw_smem = 1;
  if (filt_smem(p) > static_cast<size_t>(optin)) p.filt_tw_smem = 0;
  if (scatter_fwd_smem(p) > static_cast<size_t>(optin) || rows_smem(p) > static_cast<size_t>(optin) ||
      cols_smem(p) > static_cast<size_t>(optin) || filt_smem(p) > static_cast<size_t>(optin))
    return cudaErrorInvalidValue;
  if ((e = cudaFuncSetAttribute(k_sino_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, optin)) != cudaSuccess) return e;
  const int rs = optin, cs = optin;
  if ((e = cudaFuncSetAttribute(k_rows_fwd<false, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_sample_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_sample_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess) return e;
#define RADON_CONFIGURE_SAMPLE(n)                                                                                 \
  if ((e = cudaFuncSetAttribute(k_sample_fwd<true, n + 2 * kPad>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != \
      cudaSuccess)                                                                                                \
    return e;
  RADON_SAMPLE_PITCHES(RADON_CONFIGURE_SAMPLE)
#undef RADON_CONFIGURE_SAMPLE
  if ((e = cudaFuncSetAttribute(k_rows_fwd<true, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_rows_inv<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess) return e;
#define RADON_CONFIGURE_ROWS(i, ...)                                                                                   \
  if ((e = cudaFuncSetAttribute(k_rows_fwd<false, i>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess) \
    return e;                                                                                                          \
  if ((e = cudaFuncSetAttribute(k_rows_fwd<true, i>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess)  \
    return e;                                                                                                          \
  if ((e = cudaFuncSetAttribute(k_rows_inv<i>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess) return e;
  RADON_ROW_SEQUENCES(RADON_CONFIGURE_ROWS)
#undef RADON_CONFIGURE_ROWS
  if ((e = cudaFuncSetAttribute(k_columns, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) != cudaSuccess) return e;
  // exact transpose: generic kernels; the theta pass takes the widest group that fits
  if ((e = cudaFuncSetAttribute(k_rows_r2c_t, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_rows_c2r_t, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_scatter_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_columns_t, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) != cudaSuccess) return e;
  p.col_group_t = 0;
  for (int G = 4; G >= 1 && !p.col_group_t; G /= 2)
    if (cols_t_smem(p, G) <= static_cast<size_t>(optin)) p.col_group_t = G;
  p.col_blocks = p.col_blocks_t = 0;
  if (p.col_fixed >= 0) {
    int n_sm = 0;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
#define RADON_CONFIGURE_COLUMN(i, ...) \
  case i: e = configure_columns_fixed<__VA_ARGS__>(p, optin, n_sm); break;
    switch (p.col_fixed) {
      RADON_COLUMN_KERNELS(RADON_CONFIGURE_COLUMN)
      default: e = cudaErrorInvalidValue;
    }
#undef RADON_CONFIGURE_COLUMN
    if (e != cudaSuccess) return e;
  }
  // persistent rho transforms: one CTA per resident slot, when their buffers fit
  p.rows_pipe_fwd = p.rows_pipe_inv = 0;
  const size_t ps = rows_pipe_smem(p);
  if (ps <= static_cast<size_t>(optin)) {
    int n_sm = 0, per_sm_fwd = 0, per_sm_inv = 0;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    switch (p.row_fixed) {
#define RADON_CONFIGURE_ROWS_PIPE(i, ...)                                                                   \
  case i:                                                                                                   \
    e = configure_rows_pipe(k_rows_fwd_pipe<i>, k_rows_inv_pipe<i>, optin, ps, &per_sm_fwd, &per_sm_inv);          \
    break;
      RADON_ROW_SEQUENCES(RADON_CONFIGURE_ROWS_PIPE)
#undef RADON_CONFIGURE_ROWS_PIPE
      default: e = configure_rows_pipe(k_rows_fwd_pipe<-1>, k_rows_inv_pipe<-1>, optin, ps, &per_sm_fwd, &per_sm_inv);
    }
    if (e != cudaSuccess) return e;
    p.rows_pipe_fwd = per_sm_fwd * n_sm;
    p.rows_pipe_inv = per_sm_inv * n_sm;
  }
  // persistent back-projection rows: for plans whose row kernels fit the twiddles in shared memory
  // (the persistent form itself reads them through L1)
  p.rows_bp_blocks = 0;
  if (p.rows_tw_smem) {
    int n_sm = 0, per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    switch (p.row_fixed) {
#define RADON_CONFIGURE_ROWS_BP(i, ...) \
  case i: e = configure_persistent(k_rows_bp_persistent<i>, optin, 2 * p.nc * sizeof(float2), &per_sm); break;
      RADON_ROW_SEQUENCES(RADON_CONFIGURE_ROWS_BP)
#undef RADON_CONFIGURE_ROWS_BP
      default: e = configure_persistent(k_rows_bp_persistent<-1>, optin, 2 * p.nc * sizeof(float2), &per_sm);
    }
    if (e != cudaSuccess) return e;
    p.rows_bp_blocks = per_sm * n_sm;
  }
  return cudaSuccess;
}

cudaError_t launch_forward(const DevPlan& p, const float* image, float* sino, cudaStream_t st, StageHook hook,
                           int batch) {
  if (batch < 1 || batch > p.batch_cap) return cudaErrorInvalidValue;
  hook(-1, st);
  ImageSource isrc{image, p.N};
  if (p.img_quad && p.interp == 3)
    k_prefilter<ImageSource, true><<<dim3((p.img_pitch + kPfQuads - 1) / kPfQuads, (p.N + kPfRows - 1) / kPfRows, batch),
                                     kThreads, 0, st>>>(p, isrc, p.N, p.N, nullptr, 0, 0, 0);
  else
    k_prefilter<ImageSource, false><<<dim3((p.N + kPfCols - 1) / kPfCols, (p.N + kPfRows - 1) / kPfRows, batch),
                                      kThreads, 0, st>>>(p, isrc, p.N, p.N, p.coef_img, p.img_pitch, kPad, p.bs_img);
  hook(0, st);
  const dim3 sgrid((p.n_eanc + 1) / 2, (p.nh + kSampleWarps - 1) / kSampleWarps, p.M * batch);
  if (p.img_quad && p.interp == 3 && p.r == 5) {
    launch_sample_arc<5>(p, sgrid, st);
  } else if (p.img_quad && p.interp == 3 && p.r == 4) {
    launch_sample_arc<4>(p, sgrid, st);
  } else if (p.img_quad && p.interp == 3 && p.r == 6) {
    launch_sample_arc<6>(p, sgrid, st);
  } else if (p.img_quad && p.interp == 3) {
    switch (p.img_pitch) {
#define RADON_LAUNCH_SAMPLE(n)                                                                    \
  case n + 2 * kPad:                                                                              \
    k_sample_fwd<true, n + 2 * kPad><<<sgrid, kSampleWarps * 32, sample_fwd_smem(p), st>>>(p);     \
    break;
      RADON_SAMPLE_PITCHES(RADON_LAUNCH_SAMPLE)
#undef RADON_LAUNCH_SAMPLE
      default:
        k_sample_fwd<true><<<sgrid, kSampleWarps * 32, sample_fwd_smem(p), st>>>(p);
    }
  } else {
    k_sample_fwd<false><<<sgrid, kSampleWarps * 32, sample_fwd_smem(p), st>>>(p);
  }
  hook(11, st);
  launch_rows_forward<false>(p, st, batch);
  hook(1, st);
  launch_columns_and_inverse(p, p.k_fwd, st, hook, 2, batch);
  k_gather_sino<<<dim3((p.n_det + 127) / 128, p.n_angles, batch), 128, 0, st>>>(p, sino);
  hook(4, st);
  return cudaGetLastError();
}

cudaError_t launch_backproject(const DevPlan& p, const float* sino, float* image, cudaStream_t st, StageHook hook,
                               int batch) {
  if (batch < 1 || batch > p.batch_cap) return cudaErrorInvalidValue;
  hook(-1, st);
  SinoSource ssrc{sino, p.n_angles, p.n_det, p.live_lo, p.live_hi};
  k_prefilter<SinoSource, false><<<dim3((p.n_det + 1 + kPfCols - 1) / kPfCols, (p.n_angles + kPfRows - 1) / kPfRows, batch),
                            kThreads, 0, st>>>(p, ssrc, p.n_angles, p.n_det + 1, p.coef_sino, p.sino_pitch, 0, p.bs_sino);
  hook(5, st);
  launch_rows_forward<true>(p, st, batch);
  hook(6, st);
  launch_columns_and_inverse(p, p.k_bp, st, hook, 7, batch);
  k_gather_image<<<dim3(p.n_ptiles, p.n_ptiles, batch), dim3(kPTile, kPTile), 0, st>>>(p, image);
  hook(9, st);
  return cudaGetLastError();
}

int kernel_launches(const DevPlan& p, int op) {
  const int fwd = 6;  // prefilter, sample, rows, columns, rows_inv, gather
  const int bp = 5;   // prefilter, rows, columns, rows_inv, gather
  const int tr = 6;   // scatter to log-polar, rows, columns, rows_inv, scatter to the image, Q^T
  return op == 0 ? fwd : op == 1 ? bp : op == 2 ? bp + 1 : op == 3 ? tr : -1;
}

cudaError_t launch_transpose(const DevPlan& p, const float* sino, float* image, cudaStream_t st, StageHook hook,
                             int batch) {
  if (batch < 1 || batch > p.batch_cap || p.col_group_t < 1) return cudaErrorInvalidValue;
  hook(-1, st);
  // scatter targets: the log-polar rows (yspec) and the padded coefficient image
  cudaError_t e = cudaMemsetAsync(p.yspec, 0, sizeof(float2) * p.bs_ys * batch, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.coef_img, 0, sizeof(float) * p.bs_img * batch, st);
  if (e != cudaSuccess) return e;
  const int nrow = p.nh + kHaloLo + kHaloHi;
  if (p.interp == 3)
    k_scatter_sino_comb<<<dim3((p.n_det + 127) / 128, p.n_angles, batch), 128, 0, st>>>(p, sino);
  else
    k_scatter_sino<<<dim3((p.n_det + 127) / 128, p.n_angles, batch), 128, 0, st>>>(p, sino);
  hook(12, st);
  k_rows_r2c_t<<<dim3(nrow, p.M, batch), kThreads, rows_smem(p), st>>>(p);
  hook(13, st);
  if (p.col_group == 0 && p.col_fixed >= 0 && p.col_blocks_t > 0) {
    switch (p.col_fixed) {
#define RADON_LAUNCH_COLUMN_T(i, ...) \
  case i: launch_columns_fixed_t<__VA_ARGS__>(p, p.k_fwd, st, batch); break;
      RADON_COLUMN_KERNELS(RADON_LAUNCH_COLUMN_T)
#undef RADON_LAUNCH_COLUMN_T
      default: break;
    }
  } else {
    const int G = p.col_group_t;
    k_columns_t<<<dim3((p.nc + 1 + G - 1) / G, p.M, batch), kThreads, cols_t_smem(p, G), st>>>(p, p.k_fwd, G);
  }
  hook(14, st);
  k_rows_c2r_t<<<dim3(p.nh, p.M, batch), kThreads, rows_smem(p), st>>>(p);
  hook(15, st);
  const dim3 sgrid((p.n_eanc + 1) / 2, (p.nh + kSampleWarps - 1) / kSampleWarps, p.M * batch);
  k_scatter_fwd<<<sgrid, kSampleWarps * 32, scatter_fwd_smem(p), st>>>(p);
  hook(16, st);
  const CoefSource csrc{p.coef_img, p.N, p.img_pitch, p.bs_img};
  k_prefilter<CoefSource, false><<<dim3((p.N + kPfCols - 1) / kPfCols, (p.N + kPfRows - 1) / kPfRows, batch),
                                   kThreads, 0, st>>>(p, csrc, p.N, p.N, image, p.N, 0, static_cast<size_t>(p.N) * p.N);
  hook(17, st);
  return cudaGetLastError();
}

cudaError_t launch_fbp(const DevPlan& p, const float* sino, float* image, int filter, cudaStream_t st, StageHook hook) {
  hook(-1, st);
  k_sino_filter<<<p.n_angles, kThreads, filt_smem(p), st>>>(p, sino, p.filt + static_cast<size_t>(filter) * (p.n_filt / 2 + 1),
                                                           p.sino_tmp);
  hook(10, st);
  return launch_backproject(p, p.sino_tmp, image, st, hook);
}

}  // namespace radon
