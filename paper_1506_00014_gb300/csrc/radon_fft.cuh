// Block-wide mixed-radix FFT in shared memory (Stockham, self-sorting), FP32 complex.
//
// Used for the log-polar convolution of Section 3: a length-N_rho/2 complex transform (the
// real rho transform of length N_rho) per angular row and a length-n_theta transform per rho
// frequency.  Twiddles come from FP64-computed tables.  Sizes are 7-smooth; radices are taken
// from {2, 3, 4, 5, 7, 8, 9}.
#pragma once

#include <cuda_runtime.h>

namespace radon {

// One Stockham pass: radix R after Ns points have been combined; nbf = n / R butterflies per
// transform, tstep = n / (Ns R).  m_nbf / m_ns are ceil(2^32 / d) for the divisions by nbf and
// Ns (exact for numerators and divisors below 2^15; 0 when the divisor is 1).
struct FftPass {
  int R, Ns, nbf, tstep;
  unsigned m_nbf, m_ns;
};

struct RadixList {
  int n;
  int count;
  FftPass p[16];
};

__device__ __forceinline__ int fast_div(int v, int d, unsigned m) {
  return d == 1 ? v : static_cast<int>(__umulhi(static_cast<unsigned>(v), m));
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft3(float2& a, float2& b, float2& c) {
  const float s3 = 0.866025403784438646763723170753f;  // sin(2 pi / 3)
  float2 t1 = cadd(b, c);
  float2 t2 = make_float2(fmaf(-0.5f, t1.x, a.x), fmaf(-0.5f, t1.y, a.y));
  float2 t3 = rot90<INV>(cscale(csub(b, c), s3));
  a = cadd(a, t1);
  b = cadd(t2, t3);
  c = csub(t2, t3);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d) {
  float2 s0 = cadd(a, c), d0 = csub(a, c);
  float2 s1 = cadd(b, d), d1 = rot90<INV>(csub(b, d));
  a = cadd(s0, s1);
  c = csub(s0, s1);
  b = cadd(d0, d1);
  d = csub(d0, d1);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&v)[R]);

template <>
__device__ __forceinline__ void dft<2, false>(float2 (&v)[2]) { dft2<false>(v[0], v[1]); }
template <>
__device__ __forceinline__ void dft<2, true>(float2 (&v)[2]) { dft2<true>(v[0], v[1]); }
template <>
__device__ __forceinline__ void dft<3, false>(float2 (&v)[3]) { dft3<false>(v[0], v[1], v[2]); }
template <>
__device__ __forceinline__ void dft<3, true>(float2 (&v)[3]) { dft3<true>(v[0], v[1], v[2]); }
template <>
__device__ __forceinline__ void dft<4, false>(float2 (&v)[4]) { dft4<false>(v[0], v[1], v[2], v[3]); }
template <>
__device__ __forceinline__ void dft<4, true>(float2 (&v)[4]) { dft4<true>(v[0], v[1], v[2], v[3]); }

template <bool INV>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
  const float h = 0.707106781186547524400844362105f;
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // W8^k, k = 1, 2, 3 (conjugated for the inverse)
  o1 = INV ? make_float2(h * (o1.x - o1.y), h * (o1.x + o1.y)) : make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));
  o2 = rot90<INV>(o2);
  o3 = INV ? make_float2(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : make_float2(h * (o3.y - o3.x), -h * (o3.x + o3.y));
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}
template <>
__device__ __forceinline__ void dft<8, false>(float2 (&v)[8]) { dft8<false>(v); }
template <>
__device__ __forceinline__ void dft<8, true>(float2 (&v)[8]) { dft8<true>(v); }

// Odd prime radix by pairing x_j with x_{R-j}: y_k = x_0 + sum_j (x_j + x_{R-j}) cos(2 pi jk/R)
//                                                 -/+ i (x_j - x_{R-j}) sin(2 pi jk/R).
template <int R, bool INV>
__device__ __forceinline__ void dft_odd(float2 (&v)[R], const float (&cs)[R], const float (&sn)[R]) {
  constexpr int H = (R - 1) / 2;
  float2 sp[H], sm[H];
#pragma unroll
  for (int j = 1; j <= H; ++j) {
    sp[j - 1] = cadd(v[j], v[R - j]);
    sm[j - 1] = csub(v[j], v[R - j]);
  }
  float2 y[R];
  y[0] = v[0];
#pragma unroll
  for (int j = 0; j < H; ++j) y[0] = cadd(y[0], sp[j]);
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    float2 re = v[0], im = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 1; j <= H; ++j) {
      const int q = (j * k) % R;
      re.x = fmaf(sp[j - 1].x, cs[q], re.x);
      re.y = fmaf(sp[j - 1].y, cs[q], re.y);
      im.x = fmaf(sm[j - 1].x, sn[q], im.x);
      im.y = fmaf(sm[j - 1].y, sn[q], im.y);
    }
    const float2 t = rot90<INV>(im);
    y[k] = cadd(re, t);
    y[R - k] = csub(re, t);
  }
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = y[k];
}

template <>
__device__ __forceinline__ void dft<5, false>(float2 (&v)[5]) {
  const float cs[5] = {1.f, 0.309016994374947424102293417183f, -0.809016994374947424102293417183f,
                       -0.809016994374947424102293417183f, 0.309016994374947424102293417183f};
  const float sn[5] = {0.f, 0.951056516295153572116439333379f, 0.587785252292473129168705954639f,
                       -0.587785252292473129168705954639f, -0.951056516295153572116439333379f};
  dft_odd<5, false>(v, cs, sn);
}
template <>
__device__ __forceinline__ void dft<5, true>(float2 (&v)[5]) {
  const float cs[5] = {1.f, 0.309016994374947424102293417183f, -0.809016994374947424102293417183f,
                       -0.809016994374947424102293417183f, 0.309016994374947424102293417183f};
  const float sn[5] = {0.f, 0.951056516295153572116439333379f, 0.587785252292473129168705954639f,
                       -0.587785252292473129168705954639f, -0.951056516295153572116439333379f};
  dft_odd<5, true>(v, cs, sn);
}

#define RADON_C7 {1.f, 0.623489801858733530525004884004f, -0.222520933956314404288902564497f, \
                  -0.900968867902419126236102319507f, -0.900968867902419126236102319507f,     \
                  -0.222520933956314404288902564497f, 0.623489801858733530525004884004f}
#define RADON_S7 {0.f, 0.781831482468029808708444526674f, 0.974927912181823607018131682994f,  \
                  0.433883739117558120475768332849f, -0.433883739117558120475768332849f,     \
                  -0.974927912181823607018131682994f, -0.781831482468029808708444526674f}
template <>
__device__ __forceinline__ void dft<7, false>(float2 (&v)[7]) {
  const float cs[7] = RADON_C7;
  const float sn[7] = RADON_S7;
  dft_odd<7, false>(v, cs, sn);
}
template <>
__device__ __forceinline__ void dft<7, true>(float2 (&v)[7]) {
  const float cs[7] = RADON_C7;
  const float sn[7] = RADON_S7;
  dft_odd<7, true>(v, cs, sn);
}

// Radix 9 = 3 x 3 with internal twiddles W9^(j k), j, k in {1, 2}.
template <bool INV>
__device__ __forceinline__ void dft9(float2 (&v)[9]) {
  // columns: (v0, v3, v6), (v1, v4, v7), (v2, v5, v8)
  dft3<INV>(v[0], v[3], v[6]);
  dft3<INV>(v[1], v[4], v[7]);
  dft3<INV>(v[2], v[5], v[8]);
  const float2 w1 = make_float2(0.766044443118978035202392650555f, -0.642787609686539326322643409907f);
  const float2 w2 = make_float2(0.173648177666930348851716626769f, -0.984807753012208059366743024590f);
  const float2 w4 = make_float2(-0.939692620785908384054109277324f, -0.342020143325668733044099614682f);
  if (INV) {
    v[4] = cmulc(v[4], w1);
    v[7] = cmulc(v[7], w2);
    v[5] = cmulc(v[5], w2);
    v[8] = cmulc(v[8], w4);
  } else {
    v[4] = cmul(v[4], w1);
    v[7] = cmul(v[7], w2);
    v[5] = cmul(v[5], w2);
    v[8] = cmul(v[8], w4);
  }
  dft3<INV>(v[0], v[1], v[2]);
  dft3<INV>(v[3], v[4], v[5]);
  dft3<INV>(v[6], v[7], v[8]);
  // output index 3 * k2 + k1 is stored at position 3 * k1 + k2: transpose
  float2 t;
  t = v[1]; v[1] = v[3]; v[3] = t;
  t = v[2]; v[2] = v[6]; v[6] = t;
  t = v[5]; v[5] = v[7]; v[7] = t;
}
template <>
__device__ __forceinline__ void dft<9, false>(float2 (&v)[9]) { dft9<false>(v); }
template <>
__device__ __forceinline__ void dft<9, true>(float2 (&v)[9]) { dft9<true>(v); }

// One Stockham pass of radix R over `nb` transforms of length n (transform b at src + b * fs).
// tw[p] = exp(-2 pi i p / n), normally staged in shared memory.
template <int R, bool INV>
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ src, float2* __restrict__ dst, int n,
                                              int nb, int fs, const FftPass& ps, const float2* __restrict__ tw,
                                              int tid, int nth) {
  const int nbf = ps.nbf, Ns = ps.Ns, tstep = ps.tstep;
  const int total = nbf * nb;
  for (int t = tid; t < total; t += nth) {
    const int b = fast_div(t, nbf, ps.m_nbf);
    const int j = t - b * nbf;
    const int q = fast_div(j, Ns, ps.m_ns);
    const int k = j - q * Ns;
    const float2* s = src + b * fs;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[j + r * nbf];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = tw[r * k * tstep];
        v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
      }
    }
    dft<R, INV>(v);
    float2* d = dst + b * fs + q * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[r * Ns] = v[r];
  }
}

// Full transform; ping-pongs between a and b, returns the buffer holding the result.
// All threads of the block must call it.
template <bool INV>
__device__ float2* fft_block(float2* a, float2* b, int nb, int fs, const RadixList& rl,
                             const float2* __restrict__ tw, int tid, int nth) {
  const int n = rl.n;
  for (int st = 0; st < rl.count; ++st) {
    const FftPass& ps = rl.p[st];
    switch (ps.R) {
      case 2: stockham_pass<2, INV>(a, b, n, nb, fs, ps, tw, tid, nth); break;
      case 3: stockham_pass<3, INV>(a, b, n, nb, fs, ps, tw, tid, nth); break;
      case 4: stockham_pass<4, INV>(a, b, n, nb, fs, ps, tw, tid, nth); break;
      case 5: stockham_pass<5, INV>(a, b, n, nb, fs, ps, tw, tid, nth); break;
      case 7: stockham_pass<7, INV>(a, b, n, nb, fs, ps, tw, tid, nth); break;
      case 8: stockham_pass<8, INV>(a, b, n, nb, fs, ps, tw, tid, nth); break;
      case 9: stockham_pass<9, INV>(a, b, n, nb, fs, ps, tw, tid, nth); break;
      default: break;
    }
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
  }
  return a;
}

// The same Stockham transform with a compile-time radix sequence (one transform, TH threads):
// index division by NS becomes a multiply-shift and the butterfly loop unrolls.  Same twiddle
// table as fft_block: tw[p] = exp(-2 pi i p / NN).
template <int NN, int R, int NS, bool INV, int TH>
__device__ __forceinline__ void stockham_pass_fixed(const float2* __restrict__ src, float2* __restrict__ dst,
                                                    const float2* __restrict__ tw, int tid) {
  constexpr int NBF = NN / R, TSTEP = NN / (NS * R);
#pragma unroll
  for (int t0 = 0; t0 < NBF; t0 += TH) {
    const int j = t0 + tid;
    if (NBF % TH != 0 && j >= NBF) break;
    const int q = j / NS, k = j - q * NS;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[j + r * NBF];
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = tw[r * k * TSTEP];
        v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
      }
    }
    dft<R, INV>(v);
    float2* d = dst + q * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[r * NS] = v[r];
  }
}

template <int NN, bool INV, int TH, int NS, int R, int... Rest>
struct FixedFft {
  // Ping-pongs between a and b; returns the buffer holding the result.
  __device__ __forceinline__ static float2* run(float2* a, float2* b, const float2* __restrict__ tw, int tid) {
    stockham_pass_fixed<NN, R, NS, INV, TH>(a, b, tw, tid);
    __syncthreads();
    if constexpr (sizeof...(Rest) == 0)
      return b;
    else
      return FixedFft<NN, INV, TH, NS * R, Rest...>::run(b, a, tw, tid);
  }
};

// The same transform with the first pass (NS = 1, no twiddles) reading its inputs through a
// functor in(i) instead of a buffer, so a caller that would first fill the buffer element by
// element (a pre-processing step) saves that pass and its barrier.  The first pass writes a; the
// others ping-pong between a and b.
template <int NN, bool INV, int TH, int R, int... Rest>
struct FixedFftIn {
  template <class In>
  __device__ __forceinline__ static float2* run(const In& in, float2* a, float2* b, const float2* __restrict__ tw,
                                                int tid) {
    constexpr int NBF = NN / R;
#pragma unroll
    for (int t0 = 0; t0 < NBF; t0 += TH) {
      const int j = t0 + tid;
      if (NBF % TH != 0 && j >= NBF) break;
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = in(j + r * NBF);
      dft<R, INV>(v);
      float2* d = a + j * R;
#pragma unroll
      for (int r = 0; r < R; ++r) d[r] = v[r];
    }
    __syncthreads();
    if constexpr (sizeof...(Rest) == 0)
      return a;
    else
      return FixedFft<NN, INV, TH, R, Rest...>::run(a, b, tw, tid);
  }
};

// The same pass with its outputs written through a functor out(i, value) (the last pass of a
// transform whose result goes straight to global memory); no barrier follows it.
template <int NN, int R, int NS, bool INV, int TH, class Out>
__device__ __forceinline__ void stockham_pass_fixed_out(const float2* __restrict__ src, const Out& out,
                                                        const float2* __restrict__ tw, int tid) {
  constexpr int NBF = NN / R, TSTEP = NN / (NS * R);
#pragma unroll
  for (int t0 = 0; t0 < NBF; t0 += TH) {
    const int j = t0 + tid;
    if (NBF % TH != 0 && j >= NBF) break;
    const int q = j / NS, k = j - q * NS;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[j + r * NBF];
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = tw[r * k * TSTEP];
        v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
      }
    }
    dft<R, INV>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) out(q * NS * R + k + r * NS, v[r]);
  }
}

// Passes after the first, ping-ponging between a and b, the last one writing through out.
template <int NN, bool INV, int TH, int NS, int R, int... Rest>
struct FixedFftOut {
  template <class Out>
  __device__ __forceinline__ static void run(float2* a, float2* b, const float2* __restrict__ tw, const Out& out,
                                             int tid) {
    if constexpr (sizeof...(Rest) == 0) {
      stockham_pass_fixed_out<NN, R, NS, INV, TH>(a, out, tw, tid);
    } else {
      stockham_pass_fixed<NN, R, NS, INV, TH>(a, b, tw, tid);
      __syncthreads();
      FixedFftOut<NN, INV, TH, NS * R, Rest...>::run(b, a, tw, out, tid);
    }
  }
};

// First pass through in (writes a), last pass through out: a transform from a computed input to a
// computed destination with no staging pass at either end.
template <int NN, bool INV, int TH, int R, int R2, int... Rest>
struct FixedFftInOut {
  template <class In, class Out>
  __device__ __forceinline__ static void run(const In& in, float2* a, float2* b, const float2* __restrict__ tw,
                                             const Out& out, int tid) {
    constexpr int NBF = NN / R;
#pragma unroll
    for (int t0 = 0; t0 < NBF; t0 += TH) {
      const int j = t0 + tid;
      if (NBF % TH != 0 && j >= NBF) break;
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = in(j + r * NBF);
      dft<R, INV>(v);
      float2* d = a + j * R;
#pragma unroll
      for (int r = 0; r < R; ++r) d[r] = v[r];
    }
    __syncthreads();
    FixedFftOut<NN, INV, TH, R, R2, Rest...>::run(a, b, tw, out, tid);
  }
};

// Copy an n-entry table into shared memory (all threads; caller synchronises).
__device__ __forceinline__ void stage_table(float2* dst, const float2* __restrict__ src, int n, int tid, int nth) {
  for (int i = tid; i < n; i += nth) dst[i] = __ldg(src + i);
}


// ------------------------------------------------------------------------------------------
// In-place passes of compile-time shape.  Dft<R> runs one radix-R
// butterfly in registers; idx(r) is the register that holds output r.

template <int R, bool INV>
struct Dft {
  __host__ __device__ static constexpr int idx(int r) { return r; }
  __device__ __forceinline__ static void run(float2 (&v)[R]) { dft<R, INV>(v); }
};

// Internal twiddles exp(-2 pi i q / R) of the composite radices below, as constants (q is known
// at compile time once the butterfly is unrolled).
template <int R>
struct Wconst;
template <>
struct Wconst<16> {  // q = n2 k1 in {0, 1, 2, 3, 4, 6, 9}
  __device__ __forceinline__ static float2 get(int q) {
    constexpr float c1 = 0.923879532511286756f;  // cos(pi / 8)
    constexpr float s1 = 0.382683432365089772f;  // sin(pi / 8)
    constexpr float h = 0.707106781186547524f;   // cos(pi / 4)
    switch (q) {
      case 1: return make_float2(c1, -s1);
      case 2: return make_float2(h, -h);
      case 3: return make_float2(s1, -c1);
      case 4: return make_float2(0.f, -1.f);
      case 6: return make_float2(-h, -h);
      case 9: return make_float2(-c1, s1);
      default: return make_float2(1.f, 0.f);
    }
  }
};
template <>
struct Wconst<14> {  // q = n2 k1 in {0, ..., 6}: cos(pi q / 7) - i sin(pi q / 7)
  __device__ __forceinline__ static float2 get(int q) {
    constexpr float c1 = 0.900968867902419126f, s1 = 0.433883739117558120f;
    constexpr float c2 = 0.623489801858733531f, s2 = 0.781831482468029809f;
    constexpr float c3 = 0.222520933956314404f, s3 = 0.974927912181823607f;
    switch (q) {
      case 1: return make_float2(c1, -s1);
      case 2: return make_float2(c2, -s2);
      case 3: return make_float2(c3, -s3);
      case 4: return make_float2(-c3, -s3);
      case 5: return make_float2(-c2, -s2);
      case 6: return make_float2(-c1, -s1);
      default: return make_float2(1.f, 0.f);
    }
  }
};

// R = R1 R2 Cooley-Tukey in registers: R1-point DFTs over n1 (input n = R2 n1 + n2), twiddles
// W_R^(n2 k1), R2-point DFTs over n2; X[k1 + R1 k2] is left at v[R2 k1 + k2].
template <int R1, int R2, bool INV>
struct DftComposite {
  static constexpr int R = R1 * R2;
  __host__ __device__ static constexpr int idx(int r) { return R2 * (r % R1) + r / R1; }
  __device__ __forceinline__ static void run(float2 (&v)[R]) {
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      float2 c[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) c[n1] = v[R2 * n1 + n2];
      dft<R1, INV>(c);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) {
        float2 t = c[k1];
        if (n2 * k1 != 0) {
          const float2 w = Wconst<R>::get(n2 * k1);
          t = INV ? cmulc(t, w) : cmul(t, w);
        }
        v[R2 * k1 + n2] = t;
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      float2 c[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) c[n2] = v[R2 * k1 + n2];
      dft<R2, INV>(c);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) v[R2 * k1 + k2] = c[k2];
    }
  }
};
template <bool INV>
struct Dft<16, INV> : DftComposite<4, 4, INV> {};
template <bool INV>
struct Dft<14, INV> : DftComposite<2, 7, INV> {};

// Twiddle entries a pass of radix R after NS combined points reads: NS (R - 1), laid out
// [k][r - 1] = exp(-2 pi i r k / (NS R)); none for the first pass (NS = 1).
__host__ __device__ constexpr int pass_twiddles(int R, int NS) { return NS > 1 ? NS * (R - 1) : 0; }

// One in-place Stockham pass over G interleaved transforms of length NN ([row][g] layout):
// butterfly t = tid + i TH (t < G NN / R) handles transform g = t % G, index j = t / G.  Each thread holds BM
// butterflies in registers from before the barrier (the whole array is read) until after it
// (the whole array is written).  `in(row, g)` loads, `out(row, g, value)` stores; Out::kShared
// says whether the stores go to shared memory and so need a barrier before the next pass.
template <int NN, int G, int TH, int R, int NS, bool INV, class In, class Out>
__device__ __forceinline__ void inplace_pass(const float2* __restrict__ tw, const In& in, const Out& out, int tid) {
  constexpr int NBF = NN / R;
  constexpr int NB = G * NBF;               // butterflies of the pass
  constexpr int BM = (NB + TH - 1) / TH;    // per thread (the last round may be partial)
  constexpr bool kExact = BM * TH == NB;
  float2 v[BM][R];
#pragma unroll
  for (int i = 0; i < BM; ++i) {
    const int t = tid + i * TH;
    if (!kExact && t >= NB) break;
    const int g = t % G, j = t / G;
    const int k = j % NS;
#pragma unroll
    for (int r = 0; r < R; ++r) v[i][r] = in(j + r * NBF, g);
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = tw[k * (R - 1) + r - 1];
        v[i][r] = INV ? cmulc(v[i][r], w) : cmul(v[i][r], w);
      }
    }
    Dft<R, INV>::run(v[i]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < BM; ++i) {
    const int t = tid + i * TH;
    if (!kExact && t >= NB) break;
    const int g = t % G, j = t / G;
    const int k = j % NS, q = j / NS;
#pragma unroll
    for (int r = 0; r < R; ++r) out(q * NS * R + k + r * NS, g, v[i][Dft<R, INV>::idx(r)]);
  }
  if constexpr (Out::kShared) __syncthreads();
}

// Interleaved shared-memory views used between passes.
template <int G>
struct SmemIn {
  const float2* d;
  __device__ __forceinline__ float2 operator()(int row, int g) const { return d[row * G + g]; }
};
template <int G>
struct SmemOut {
  static constexpr bool kShared = true;
  float2* d;
  __device__ __forceinline__ void operator()(int row, int g, float2 v) const { d[row * G + g] = v; }
};

// A whole transform as a chain of in-place passes Rs... (first radix first); the first pass reads
// through `in`, the last writes through `out`, the others use `data`.  TWO is the offset of the
// current pass in the concatenated per-pass twiddle table.
template <int NN, int G, int TH, bool INV, int NS, int TWO, int R, int... Rest>
struct InplaceChain {
  template <class In, class Out>
  __device__ __forceinline__ static void run(const float2* __restrict__ tw, const In& in, float2* data,
                                             const Out& out, int tid) {
    if constexpr (sizeof...(Rest) == 0) {
      inplace_pass<NN, G, TH, R, NS, INV>(tw + TWO, in, out, tid);
    } else {
      inplace_pass<NN, G, TH, R, NS, INV>(tw + TWO, in, SmemOut<G>{data}, tid);
      InplaceChain<NN, G, TH, INV, NS * R, TWO + pass_twiddles(R, NS), Rest...>::run(tw, SmemIn<G>{data}, data, out,
                                                                                      tid);
    }
  }
};

// One out-of-place Stockham pass (same butterflies and output order as inplace_pass): each
// butterfly reads its inputs through `in` and writes through `out` at once, so a pass needs one
// barrier (after its stores) instead of two, at the cost of a second buffer.
template <int NN, int G, int TH, int R, int NS, bool INV, class In, class Out>
__device__ __forceinline__ void pingpong_pass(const float2* __restrict__ tw, const In& in, const Out& out, int tid) {
  constexpr int NBF = NN / R;
  constexpr int NB = G * NBF;
  constexpr int BM = (NB + TH - 1) / TH;
  constexpr bool kExact = BM * TH == NB;
#pragma unroll
  for (int i = 0; i < BM; ++i) {
    const int t = tid + i * TH;
    if (!kExact && t >= NB) break;
    const int g = t % G, j = t / G;
    const int k = j % NS, q = j / NS;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in(j + r * NBF, g);
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = tw[k * (R - 1) + r - 1];
        v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
      }
    }
    Dft<R, INV>::run(v);
#pragma unroll
    for (int r = 0; r < R; ++r) out(q * NS * R + k + r * NS, g, v[Dft<R, INV>::idx(r)]);
  }
  if constexpr (Out::kShared) __syncthreads();
}

// A whole transform as a chain of out-of-place passes alternating between two buffers: the first
// pass reads `in` and writes `a`, the next reads `a` and writes `b`, and so on; the last writes
// through `out`.
template <int NN, int G, int TH, bool INV, int NS, int TWO, int R, int... Rest>
struct PingPongChain {
  template <class In, class Out>
  __device__ __forceinline__ static void run(const float2* __restrict__ tw, const In& in, float2* a, float2* b,
                                             const Out& out, int tid) {
    if constexpr (sizeof...(Rest) == 0) {
      pingpong_pass<NN, G, TH, R, NS, INV>(tw + TWO, in, out, tid);
    } else {
      pingpong_pass<NN, G, TH, R, NS, INV>(tw + TWO, in, SmemOut<G>{a}, tid);
      PingPongChain<NN, G, TH, INV, NS * R, TWO + pass_twiddles(R, NS), Rest...>::run(tw, SmemIn<G>{a}, b, a, out,
                                                                                       tid);
    }
  }
};

template <int... Rs>
__host__ __device__ constexpr int chain_length() {
  int n = 1;
  ((n *= Rs), ...);
  return n;
}
template <int... Rs>
__host__ __device__ constexpr int chain_twiddles() {
  int ns = 1, t = 0;
  ((t += pass_twiddles(Rs, ns), ns *= Rs), ...);
  return t;
}

}  // namespace radon
