// Host-side plan construction in FP64 (see plan_host.h).
#include "plan_host.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>
#include <thread>

namespace radon {
namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846264338327950288;

bool is_7smooth(long n) {
  if (n < 1) return false;
  for (long p : {2L, 3L, 5L, 7L})
    while (n % p == 0) n /= p;
  return n == 1;
}

long even_7smooth_at_least(long n) {
  long m = std::max(n, 2L);
  while ((m & 1) || !is_7smooth(m)) ++m;
  return m;
}

long floor_div(long a, long b) {  // b > 0
  long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

void split(double v, int32_t* i, float* f) {
  double fl = std::floor(v);
  *i = static_cast<int32_t>(fl);
  *f = static_cast<float>(v - fl);
}

int32_t fbits(float f) {
  int32_t b;
  std::memcpy(&b, &f, 4);
  return b;
}

void hilo(double v, float* hi, float* lo) {
  *hi = static_cast<float>(v);
  *lo = static_cast<float>(v - static_cast<double>(*hi));
}

cd cmul_plain(const cd& x, const cd& y) {  // plain complex product (no inf/NaN recovery path)
  return cd(x.real() * y.real() - x.imag() * y.imag(), x.real() * y.imag() + x.imag() * y.real());
}

// Out-of-place Stockham FFT, forward sign (exp(-2 pi i jk/n)), n a power of two, tw[k] =
// exp(-2 pi i k / n) for k < n: one radix-2 pass when log2 n is odd, then radix-4 passes.
// Ping-pongs between a and b; returns the buffer holding the result.
cd* fft_pow2(cd* a, cd* b, size_t n, const cd* tw) {
  size_t ns = 1;
  size_t lg = 0;
  while ((size_t(1) << lg) < n) ++lg;
  if (lg & 1) {
    for (size_t j = 0; j < n / 2; ++j) {
      const cd u = a[j], v = a[j + n / 2];
      b[2 * j] = u + v;
      b[2 * j + 1] = u - v;
    }
    std::swap(a, b);
    ns = 2;
  }
  const size_t q = n / 4;
  for (; ns < n; ns *= 4) {
    const size_t ts = n / (4 * ns);
    for (size_t j = 0; j < q; ++j) {
      const size_t k = j & (ns - 1);
      const cd x0 = a[j];
      const cd x1 = cmul_plain(a[j + q], tw[k * ts]);
      const cd x2 = cmul_plain(a[j + 2 * q], tw[2 * k * ts]);
      const cd x3 = cmul_plain(a[j + 3 * q], tw[3 * k * ts]);
      const cd t0 = x0 + x2, t1 = x0 - x2, t2 = x1 + x3, d = x1 - x3;
      const cd t3(d.imag(), -d.real());  // -i (x1 - x3)
      cd* o = b + 4 * (j - k) + k;
      o[0] = t0 + t2;
      o[ns] = t1 + t3;
      o[2 * ns] = t0 - t2;
      o[3 * ns] = t1 - t3;
    }
    std::swap(a, b);
  }
  return a;
}

// The first nk bins of the length-n DFT of a sequence with a[n - j] = a[j] (indices mod n),
// n = P Q with nk <= Q and P >= 2 powers of two.  Splitting j = m P + p into P interleaved
// subsequences s_p gives out[k] = sum_p w^(p k) DFT_Q(s_p)[k], w = exp(-2 pi i / n).  The
// symmetry maps s_(P-p)[m] to s_p[Q-1-m], so DFT_Q(s_(P-p))[k] = w^(-P k) DFT_Q(s_p)[Q-k] and
// only s_0 ... s_(P/2) are transformed:
//   out[k] = B_0[k] + sum_(0<p<P/2) (w^(p k) B_p[k] + w^(-p k) B_p[(Q-k) mod Q]) + w^(P k/2) B_(P/2)[k].
// at holds s_0 ... s_(P/2) back to back (at[p Q + m] = a[m P + p]) and is overwritten; scratch
// holds Q values.
void dft_first_bins_even(cd* at, cd* scratch, size_t n, size_t Q, size_t nk, const cd* tw_n, const cd* tw_q,
                         cd* out) {
  const size_t P = n / Q, half = P / 2;
  for (size_t k = 0; k < nk; ++k) out[k] = 0.0;
  for (size_t p = 0; p <= half; ++p) {
    const cd* B = fft_pow2(at + p * Q, scratch, Q, tw_q);
    size_t idx = 0;  // p k mod n
    for (size_t k = 0; k < nk; ++k) {
      const cd w = tw_n[idx];
      if (p == 0)
        out[k] += B[k];
      else if (p == half)
        out[k] += cmul_plain(w, B[k]);
      else
        out[k] += cmul_plain(w, B[k]) + cmul_plain(std::conj(w), B[(Q - k) & (Q - 1)]);
      idx += p;
      if (idx >= n) idx -= n;
    }
  }
}

void parallel_for(int n, const std::function<void(int, int)>& body) {
  int nt = static_cast<int>(std::thread::hardware_concurrency());
  nt = std::max(1, std::min(nt, 64));
  nt = std::min(nt, std::max(1, n));
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) {
    int b = static_cast<int>((static_cast<long>(n) * t) / nt);
    int e = static_cast<int>((static_cast<long>(n) * (t + 1)) / nt);
    th.emplace_back([&body, b, e]() { body(b, e); });
  }
  for (auto& x : th) x.join();
}

}  // namespace

bool factor_radices(int n, Radices* out) {
  out->n = n;
  out->count = 0;
  int m = n;
  auto push = [&](int r) {
    if (out->count >= kMaxRadices) return false;
    out->r[out->count++] = r;
    m /= r;
    return true;
  };
  while (m % 8 == 0) if (!push(8)) return false;
  while (m % 4 == 0) if (!push(4)) return false;
  while (m % 2 == 0) if (!push(2)) return false;
  while (m % 9 == 0) if (!push(9)) return false;
  while (m % 3 == 0) if (!push(3)) return false;
  while (m % 5 == 0) if (!push(5)) return false;
  while (m % 7 == 0) if (!push(7)) return false;
  return m == 1;
}

int compute_geometry(int N, int n_angles, int n_det, int interp, int M, radon_plan_info* g) {
  if (!g) return RADON_INVALID_ARG;
  if (N < 8 || (N & 1) || n_angles < 2 || n_det < 4 || (interp != 1 && interp != 3) || M < 3)
    return RADON_INVALID_ARG;
  if (N > 32768 || n_angles > 65535 || n_det > (1 << 20) || M > 64) return RADON_NOT_SUPPORTED;
  std::memset(g, 0, sizeof(*g));
  g->N = N;
  g->n_angles = n_angles;
  g->n_det = n_det;
  g->interp_order = interp;
  g->n_partitions = M;
  const double beta = kPi / M;
  const double sb = std::sin(beta / 2), cb = std::cos(beta / 2);
  g->beta = beta;
  g->a_R = sb / (1.0 + sb);                                   // Eq. aconst
  g->a_r = (cb - sb) / (1.0 + sb);
  g->L = -std::log(g->a_r);
  const long nrho_min = static_cast<long>(std::ceil(std::log(g->a_r) / std::log(1.0 - 2.0 * g->a_R / N)));  // Eq. vrho
  g->N_rho = static_cast<int>(even_7smooth_at_least(nrho_min));
  g->n_theta_half = static_cast<int>(even_7smooth_at_least((n_angles + M - 1) / M));
  g->n_theta = 2 * g->n_theta_half;
  g->d_phi = beta / g->n_theta_half;
  g->r = static_cast<int>(std::ceil(g->d_phi * N / (2.0 * g->a_R)));
  g->d_rho = g->L / g->N_rho;
  g->d_s = 2.0 * std::sqrt(2.0) / n_det;
  g->d_theta = kPi / n_angles;
  // trapezoid nodes for the kernel integrals: at least 8x the angular grid (Section 3) and
  // about 20 nodes per period of the fastest oscillation of exp(-i pi theta k_theta / beta)
  // cos(theta)^alpha (k_rho = N_rho/2 at theta = beta), where the corrected rule's error is
  // ~1e-9 of max |zeta_hat|, far below FP32 rounding.
  const double omega = 0.5 * g->N_rho * std::tan(beta) * 2.0 * beta / g->L;  // cycles per period
  const double need = std::max(8.0 * g->n_theta, 20.0 * (omega + 0.5 * g->n_theta));
  long nq = 64;
  while (nq < need) nq <<= 1;
  g->n_quad = static_cast<int>(nq);
  g->n_filter = static_cast<int>(even_7smooth_at_least(2L * n_det));
  return RADON_OK;
}

// zeta_hat / zeta#_hat by the trapezoidal rule over one period [-beta, beta) evaluated with an
// FFT, corrected at both ends by the weights of Eq. weightsa (Section 3).  The integrand is even
// in theta and continuous across the period boundary; the periodic sum counts the node at
// theta = -beta (= beta) once, so it receives the correction of both ends.
void kernel_quadrant(const radon_plan_info& g, int which, std::vector<double>* out) {
  static const double c[7] = {-23681, 55688, -66109, 57024, -31523, 9976, -1375};
  const int nq = g.n_quad;
  const int nkt = g.n_theta / 2 + 1;
  const int nkr = g.N_rho / 2 + 1;
  out->assign(2 * static_cast<size_t>(nkt) * nkr, 0.0);
  const double h = 2.0 * g.beta / nq;
  const double nu = 2.0 * kPi / g.L;
  // Only the first nkt DFT bins are needed (nkt << nq), and the integrand is even in theta, so the
  // node sequence is symmetric (node nq - n is -theta_n, same weight): dft_first_bins_even
  // transforms the interleaved subsequences p = 0 ... P/2 only.  The per-node arrays hold those
  // nodes regrouped for it (node n = m P + p at index p Q + m), so every pass below is sequential.
  size_t Q = 1;
  while (Q < static_cast<size_t>(nkt)) Q <<= 1;
  const size_t P = nq / Q;
  const int nh_nodes = static_cast<int>((P / 2 + 1) * Q);
  std::vector<double> w(nq, 1.0);
  w[0] += 2.0 * c[0] / 120960.0;
  for (int j = 1; j < 7; ++j) {
    w[j] += c[j] / 120960.0;
    w[nq - j] += c[j] / 120960.0;
  }
  const double sgn = which == 0 ? -1.0 : 1.0;
  std::vector<double> lc(nh_nodes), wq(nh_nodes);  // log cos(theta_n), corrected weights (regrouped)
  std::vector<cd> step(nh_nodes);                  // exp(-+ i nu log cos theta_n) (regrouped)
  for (size_t p = 0; p <= P / 2; ++p)
    for (size_t m = 0; m < Q; ++m) {
      const size_t n = m * P + p, i = p * Q + m;
      lc[i] = std::log(std::cos(-g.beta + static_cast<double>(n) * h));
      wq[i] = w[n];
      step[i] = std::polar(1.0, sgn * nu * lc[i]);
    }
  std::vector<cd> tw(nq), tw_q(Q);
  for (int k = 0; k < nq; ++k) tw[k] = std::polar(1.0, -2.0 * kPi * k / nq);
  for (size_t k = 0; k < Q; ++k) tw_q[k] = std::polar(1.0, -2.0 * kPi * static_cast<double>(k) / Q);
  // exp(alpha(k_rho) log cos theta_n) is stepped in k_rho by the factor step[n] and recomputed
  // directly every 64 steps.
  parallel_for(nkr, [&](int b, int e) {
    std::vector<cd> cur(nh_nodes), at(nh_nodes), scratch(Q), bins(nkt);
    for (int kr = b; kr < e; ++kr) {
      if ((kr - b) % 64 == 0) {
        const cd alpha = which == 0 ? cd(-1.0, -nu * kr) : cd(0.0, nu * kr);
        for (int n = 0; n < nh_nodes; ++n) cur[n] = std::exp(alpha * lc[n]);
      } else {
        for (int n = 0; n < nh_nodes; ++n) cur[n] = cmul_plain(cur[n], step[n]);
      }
      for (int n = 0; n < nh_nodes; ++n) at[n] = cur[n] * wq[n];
      dft_first_bins_even(at.data(), scratch.data(), nq, Q, nkt, tw.data(), tw_q.data(), bins.data());
      for (int kt = 0; kt < nkt; ++kt) {
        const cd v = bins[kt] * (h * ((kt & 1) ? -1.0 : 1.0));
        (*out)[2 * (static_cast<size_t>(kt) * nkr + kr)] = v.real();
        (*out)[2 * (static_cast<size_t>(kt) * nkr + kr) + 1] = v.imag();
      }
    }
  });
}

int column_radices_index(int n_theta) {
  for (int i = 0; i < kNumColumnRadices; ++i)
    if (kColumnRadices[i].n == n_theta) return i;
  return -1;
}

int row_radices_index(int nc) {
  for (int i = 0; i < kNumRowRadices; ++i)
    if (kRowRadices[i].n == nc) return i;
  return -1;
}

int build_tables(const radon_plan_info& g, HostTables* t) {
  const int N = g.N, na = g.n_angles, nd = g.n_det, M = g.n_partitions;
  const int nh = g.n_theta_half, nt = g.n_theta, nr = g.N_rho, nc = nr / 2, r = g.r;
  if (!factor_radices(nc, &t->rad_rho) || !factor_radices(nt, &t->rad_th)) return RADON_NOT_SUPPORTED;

  auto twiddles = [](int n, int count, std::vector<float>* v) {
    v->resize(2 * static_cast<size_t>(count));
    for (int p = 0; p < count; ++p) {
      const double a = -2.0 * kPi * p / n;
      (*v)[2 * p] = static_cast<float>(std::cos(a));
      (*v)[2 * p + 1] = static_cast<float>(std::sin(a));
    }
  };
  twiddles(nc, nc, &t->tw_rho);
  twiddles(nr, nc + 1, &t->tw_r2c);
  twiddles(nt, nt, &t->tw_th);
  // Specialised column transform: pass after NS combined points with radix R reads
  // exp(-2 pi i r k / (NS R)) at [k][r - 1]; the passes' tables are concatenated.
  t->col_fixed = column_radices_index(nt);
  t->tw_col.clear();
  if (t->col_fixed >= 0) {
    int ns = 1;
    for (int i = 0; i < 4 && kColumnRadices[t->col_fixed].r[i] > 0; ++i) {
      const int R = kColumnRadices[t->col_fixed].r[i];
      if (ns > 1)
        for (int k = 0; k < ns; ++k)
          for (int q = 1; q < R; ++q) {
            const double a = -2.0 * kPi * q * k / (static_cast<double>(ns) * R);
            t->tw_col.push_back(static_cast<float>(std::cos(a)));
            t->tw_col.push_back(static_cast<float>(std::sin(a)));
          }
      ns *= R;
    }
  }

  // Fourier multipliers (the convolution steps of Algorithms 1 and 2): zeta_hat / B_hat with the
  // inverse-DFT normalisation 1/(n_theta N_rho); the forward one also divided by the in-band
  // response of the angular box low-pass.  Stored [k_rho][k_theta], k_theta in [0, n_theta/2].
  std::vector<double> zr, zb;
  kernel_quadrant(g, 0, &zr);
  kernel_quadrant(g, 1, &zb);
  const int nkt = nt / 2 + 1, nkr = nc + 1;
  t->k_fwd.assign(2 * static_cast<size_t>(nkt) * nkr, 0.f);
  t->k_bp.assign(2 * static_cast<size_t>(nkt) * nkr, 0.f);
  for (int kr = 0; kr < nkr; ++kr) {
    const double br = 2.0 / 3.0 + std::cos(2.0 * kPi * kr / nr) / 3.0;
    for (int kt = 0; kt < nkt; ++kt) {
      const double bt = 2.0 / 3.0 + std::cos(2.0 * kPi * kt / nt) / 3.0;
      double scale = 1.0 / (static_cast<double>(nt) * nr);
      if (g.interp_order == 3) scale /= bt * br;
      double box = 1.0;
      if (kt != 0) {
        const double x = kPi * kt / nt;
        box = std::sin(x) / (r * std::sin(x / r));
      }
      const size_t src = 2 * (static_cast<size_t>(kt) * nkr + kr);
      const size_t dst = 2 * (static_cast<size_t>(kr) * nkt + kt);
      const bool nyq = (kr == nc);  // Hermitian average on the rho-Nyquist column: real part
      t->k_fwd[dst] = static_cast<float>(zr[src] * scale / box);
      t->k_fwd[dst + 1] = nyq ? 0.f : static_cast<float>(zr[src + 1] * scale / box);
      t->k_bp[dst] = static_cast<float>(zb[src] * scale);
      t->k_bp[dst + 1] = nyq ? 0.f : static_cast<float>(zb[src + 1] * scale);
    }
  }

  const double aR = g.a_R, beta = g.beta;
  const double S = N / (2.0 * aR);
  // Forward sampling: image index coordinates of T_m^{-1}(e^rho (cos phi, sin phi)) are
  // col = e^rho cos(phi + m beta) S + U0_m, row = e^rho sin(phi + m beta) S + V0_m (Eq. Tdef).
  t->fwd_row.resize(4 * static_cast<size_t>(M) * nh * r);
  for (int m = 0; m < M; ++m)
    for (int jj = 0; jj < nh; ++jj)
      for (int q = 0; q < r; ++q) {
        const double phi = (jj + nh / 2 - nh) * g.d_phi + (q - 0.5 * (r - 1)) * g.d_phi / r;
        const double psi = phi + m * beta;
        float* o = &t->fwd_row[4 * ((static_cast<size_t>(m) * nh + jj) * r + q)];
        hilo(std::cos(psi) * S, &o[0], &o[1]);
        hilo(std::sin(psi) * S, &o[2], &o[3]);
      }
  t->fwd_m.resize(4 * static_cast<size_t>(M));
  for (int m = 0; m < M; ++m) {
    const double u0 = N / 2.0 - (1.0 - aR) * std::cos(m * beta) * S + kPad;
    const double v0 = N / 2.0 - (1.0 - aR) * std::sin(m * beta) * S + kPad;
    hilo(u0, &t->fwd_m[4 * m], &t->fwd_m[4 * m + 1]);
    hilo(v0, &t->fwd_m[4 * m + 2], &t->fwd_m[4 * m + 3]);
  }
  // Fine samples worth reading: the position (col, row) = (C0 + t Cv, R0 + t Rv), t = e^rho, is a
  // line in t.  Keep t where the 4 x 4 tap block lies inside the padded array (col, row in
  // [1, P - 2), shrunk by 1e-3 of a pixel for the FP32 positions) and where the block is within
  // kDiscMargin (+ 1.5 for the integer block corner) pixels of the disc; map the t interval to
  // rho indices i (rho_i = (i - N_rho + 1) d_rho).
  t->fwd_rng.resize(2 * static_cast<size_t>(M) * nh * r);
  {
    const double P = N + 2.0 * kPad, lo_b = 1.0 + 1e-3, hi_b = P - 2.0 - 1e-3;
    const double cz = kPad + N / 2.0, Rd = N / 2.0 + kDiscMargin + 1.5;
    for (int m = 0; m < M; ++m) {
      const double C0 = N / 2.0 - (1.0 - aR) * std::cos(m * beta) * S + kPad;
      const double R0 = N / 2.0 - (1.0 - aR) * std::sin(m * beta) * S + kPad;
      for (int jj = 0; jj < nh; ++jj)
        for (int q = 0; q < r; ++q) {
          const double phi = (jj + nh / 2 - nh) * g.d_phi + (q - 0.5 * (r - 1)) * g.d_phi / r;
          const double Cv = std::cos(phi + m * beta) * S, Rv = std::sin(phi + m * beta) * S;
          double tl = 0.0, th = 1e300;
          auto clip_linear = [&](double x0, double v) {  // lo_b <= x0 + t v <= hi_b
            if (v == 0.0) {
              if (x0 < lo_b || x0 > hi_b) th = -1.0;
              return;
            }
            const double a = (lo_b - x0) / v, b = (hi_b - x0) / v;
            tl = std::max(tl, std::min(a, b));
            th = std::min(th, std::max(a, b));
          };
          clip_linear(C0, Cv);
          clip_linear(R0, Rv);
          // |(C0 - cz, R0 - cz) + t (Cv, Rv)|^2 <= Rd^2
          const double dx = C0 - cz, dy = R0 - cz;
          const double A = Cv * Cv + Rv * Rv, B = 2.0 * (dx * Cv + dy * Rv), Cq = dx * dx + dy * dy - Rd * Rd;
          const double disc = B * B - 4.0 * A * Cq;
          if (disc < 0.0) {
            th = -1.0;
          } else {
            const double sq = std::sqrt(disc);
            tl = std::max(tl, (-B - sq) / (2.0 * A));
            th = std::min(th, (-B + sq) / (2.0 * A));
          }
          int32_t ilo = 1, ihi = 0;
          if (th > tl && th > 0.0) {
            const double il = tl > 0.0 ? std::log(tl) / g.d_rho + nr - 1 : -1.0;
            const double ih = std::log(th) / g.d_rho + nr - 1;
            ilo = static_cast<int32_t>(std::max(0.0, std::ceil(il)));
            ihi = static_cast<int32_t>(std::min(static_cast<double>(nr - 1), std::floor(ih)));
            if (ilo > ihi) {
              ilo = 1;
              ihi = 0;
            }
          }
          const size_t o = 2 * ((static_cast<size_t>(m) * nh + jj) * r + q);
          t->fwd_rng[o] = ilo;
          t->fwd_rng[o + 1] = ihi;
        }
    }
  }
  const int n_eanc = (nr + kETile - 1) / kETile;
  t->fwd_e.resize(2 * static_cast<size_t>(nr));
  t->fwd_eanc.resize(2 * static_cast<size_t>(n_eanc));
  for (int i = 0; i < nr; ++i) {
    const double e = std::exp((i - nr + 1) * g.d_rho);
    const double ea = std::exp(((i / kETile) * kETile - nr + 1) * g.d_rho);
    t->fwd_e[2 * i] = static_cast<float>(e / r);
    t->fwd_e[2 * i + 1] = static_cast<float>(e - ea);
  }
  for (int a = 0; a < n_eanc; ++a)
    hilo(std::exp((a * kETile - nr + 1) * g.d_rho), &t->fwd_eanc[2 * a], &t->fwd_eanc[2 * a + 1]);

  // Forward output: partition, angular tap row and rho anchors per (angle, k tile)
  // (Eq. Radon_all_pb, Eq. Sm_def).  phi_a / dphi = num * n_th_h / n_angles is rational.
  const int nkt_tiles = (nd + kKTile - 1) / kKTile;
  t->fwd_ang.resize(4 * static_cast<size_t>(na));
  t->fwd_anc.resize(4 * static_cast<size_t>(na) * nkt_tiles);
  for (int a = 0; a < na; ++a) {
    long m = (2L * a * M + na) / (2L * na);
    int flip = 0;
    long num = static_cast<long>(a) * M - m * na;
    if (m == M) {
      m = 0;
      flip = 1;
      num = static_cast<long>(a) * M - static_cast<long>(M) * na;
    }
    const long numer = num * nh + static_cast<long>(nh / 2 + kHaloLo) * na;
    const long I = floor_div(numer, na);
    const float F = static_cast<float>(static_cast<double>(numer - I * na) / na);
    int32_t* o = &t->fwd_ang[4 * static_cast<size_t>(a)];
    o[0] = static_cast<int32_t>(m);
    o[1] = flip;
    o[2] = static_cast<int32_t>(I);
    o[3] = fbits(F);
    const double phi = static_cast<double>(num) * kPi / (static_cast<double>(M) * na);
    const double A = (1.0 - aR) * std::cos(phi);
    for (int kt = 0; kt < nkt_tiles; ++kt) {
      const int k0 = kt * kKTile;
      double s0 = (k0 - nd / 2.0) * g.d_s;
      double sgn = 1.0;
      if (flip) {
        s0 = -s0;
        sgn = -1.0;
      }
      const double t0 = aR * s0 + A;
      const double cr = std::log(t0) / g.d_rho + nr - 1 + kPad;
      int32_t Ii;
      float Ff;
      split(cr, &Ii, &Ff);
      int32_t* p = &t->fwd_anc[4 * (static_cast<size_t>(a) * nkt_tiles + kt)];
      p[0] = Ii;
      p[1] = fbits(Ff);
      p[2] = fbits(static_cast<float>(sgn * aR * g.d_s / t0));
      p[3] = 0;
    }
  }

  // Back-projection sampling (Algorithm 2, resampling of g(S_m)): theta = phi_j + m beta, and
  // s = (e^rho_i - (1 - a_R) cos phi_j) / a_R, both as (int, fraction) pairs.
  t->bp_th.resize(2 * static_cast<size_t>(M) * nh);
  for (int m = 0; m < M; ++m)
    for (int jj = 0; jj < nh; ++jj) {
      const long numer = static_cast<long>(jj - nh / 2) * na + static_cast<long>(m) * na * nh;
      const long den = static_cast<long>(M) * nh;
      long I = floor_div(numer, den);
      const float F = static_cast<float>(static_cast<double>(numer - I * den) / den);
      I = ((I % (2L * na)) + 2L * na) % (2L * na);
      t->bp_th[2 * (static_cast<size_t>(m) * nh + jj)] = static_cast<int32_t>(I);
      t->bp_th[2 * (static_cast<size_t>(m) * nh + jj) + 1] = fbits(F);
    }
  t->bp_c.resize(2 * static_cast<size_t>(nh));
  for (int jj = 0; jj < nh; ++jj) {
    const double phi = (jj + nh / 2 - nh) * g.d_phi;
    int32_t I;
    float F;
    split(-(1.0 - aR) * std::cos(phi) / (aR * g.d_s) + nd / 2.0 + kPad, &I, &F);
    t->bp_c[2 * jj] = I;
    t->bp_c[2 * jj + 1] = fbits(F);
  }
  t->bp_e.resize(2 * static_cast<size_t>(nr));
  for (int i = 0; i < nr; ++i) {
    int32_t I;
    float F;
    split(std::exp((i - nr + 1) * g.d_rho) / (aR * g.d_s), &I, &F);
    t->bp_e[2 * i] = I;
    t->bp_e[2 * i + 1] = fbits(F);
  }

  // Back-projection output (Algorithm 2, resampling to X): log-polar coordinates of T_m x at the centre
  // pixel of each kPTile x kPTile tile; pixels add small FP32 offsets to them.
  const int ntile = (N + kPTile - 1) / kPTile;
  t->bp_anc.resize(8 * static_cast<size_t>(M) * ntile * ntile);
  t->bp_m.resize(2 * static_cast<size_t>(M));
  for (int m = 0; m < M; ++m) {
    const double cm = std::cos(m * beta), sm = std::sin(m * beta);
    t->bp_m[2 * m] = static_cast<float>(aR * cm);
    t->bp_m[2 * m + 1] = static_cast<float>(aR * sm);
    for (int ti = 0; ti < ntile; ++ti)
      for (int tj = 0; tj < ntile; ++tj) {
        const int ia = ti * kPTile + kPTile / 2, ja = tj * kPTile + kPTile / 2;
        const double x1 = (ja - N / 2.0) * (2.0 / N), x2 = (ia - N / 2.0) * (2.0 / N);
        const double y1 = aR * (cm * x1 + sm * x2) + 1.0 - aR;
        const double y2 = aR * (-sm * x1 + cm * x2);
        int32_t It, Ir;
        float Ft, Fr;
        split(std::atan2(y2, y1) / g.d_phi + nh / 2 + kHaloLo, &It, &Ft);
        split(0.5 * std::log(y1 * y1 + y2 * y2) / g.d_rho + nr - 1 + kPad, &Ir, &Fr);
        int32_t* o = &t->bp_anc[8 * ((static_cast<size_t>(m) * ntile + ti) * ntile + tj)];
        o[0] = It;
        o[1] = fbits(Ft);
        o[2] = Ir;
        o[3] = fbits(Fr);
        o[4] = fbits(static_cast<float>(y1));
        o[5] = fbits(static_cast<float>(y2));
        o[6] = fbits(static_cast<float>(1.0 / (y1 * y1 + y2 * y2)));
        o[7] = 0;
      }
  }

  // FBP transfer functions on the n_filter-point DFT grid (sigma_k = k / (n_filter ds)):
  // ds * DFT of the band-limited ramp kernel, times the window, divided by n_filter (the inverse
  // real FFT on the device is unnormalised).
  {
    const int P = g.n_filter, nf = P / 2;
    if (!factor_radices(nf, &t->rad_filt)) return RADON_NOT_SUPPORTED;
    twiddles(nf, nf, &t->tw_filt);
    twiddles(P, nf + 1, &t->tw_filt_r2c);
    const double ds = g.d_s;
    std::vector<double> h(nf + 1, 0.0);  // h(n), n = 0..P/2 (even kernel, h(-P/2) = h(P/2))
    h[0] = 1.0 / (4.0 * ds * ds);
    for (int n = 1; n <= nf; n += 2) h[n] = -1.0 / (kPi * kPi * static_cast<double>(n) * n * ds * ds);
    t->filt.assign(3 * static_cast<size_t>(nf + 1), 0.f);
    std::vector<double> H(nf + 1);
    parallel_for(nf + 1, [&](int b, int e) {
      for (int k = b; k < e; ++k) {
        double acc = h[0] + h[nf] * ((k & 1) ? -1.0 : 1.0);
        for (int n = 1; n < nf; n += 2) acc += 2.0 * h[n] * std::cos(2.0 * kPi * static_cast<double>(k) * n / P);
        H[k] = ds * acc;
      }
    });
    for (int k = 0; k <= nf; ++k) {
      const double x = kPi * k / P;  // pi sigma_k / (2 sigma_max)
      const double sl = k == 0 ? 1.0 : std::sin(x) / x;
      t->filt[k] = static_cast<float>(H[k] / P);
      t->filt[(nf + 1) + k] = static_cast<float>(H[k] * sl / P);
      t->filt[2 * (nf + 1) + k] = static_cast<float>(H[k] * std::cos(x) / P);
    }
  }

  return RADON_OK;
}

}  // namespace radon
