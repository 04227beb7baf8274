// Host-side (FP64) plan construction: geometry, kernel transforms and coordinate tables.
//
// Everything here runs on the CPU in double precision.  The device kernels only ever see the
// FP32 tables produced by build_tables(); the split of each coordinate into an exact integer
// part and a small FP32 fraction is what keeps the FP32 interpolation on the GPU within a few
// 1e-6 of a grid cell at N = 2048.
#pragma once

#include <cstdint>
#include <vector>

#include "radon.h"

namespace radon {

constexpr int kMaxRadices = 24;
constexpr int kKTile = 32;   // detector bins per coordinate anchor (forward output gather)
constexpr int kPTile = 16;   // pixels per side of a coordinate-anchor tile (back-projection output)
constexpr int kETile = 32;   // rho samples per coordinate anchor (forward log-polar sampling)
constexpr int kHaloLo = 2;   // output rows kept below the centre half of the angular grid
constexpr int kHaloHi = 2;   // and above it (cubic taps of |phi| <= beta/2)
constexpr int kPad = 3;      // zero border around the coefficient arrays (cubic taps never leave it)
constexpr int kFirHalf = 14; // pre-filter halo: recursions start this far outside a segment (|z|^15 ~ 2.7e-9)
constexpr int kDiscMargin = 16;  // forward sampling skips fine samples farther than this many
                                 // pixels outside the disc (coefficients there are below 1e-9)

// Column (theta) transform lengths with a specialised in-place kernel: G columns per work item,
// TH threads per CTA, at least MINB resident CTAs per SM, and the radix sequence (0 ends it).
struct ColumnRadices {
  int n, G, TH, MINB;
  int r[4];
};
constexpr ColumnRadices kColumnRadices[] = {
    {256, 32, 256, 2, {16, 16, 0, 0}},  {512, 16, 256, 2, {8, 8, 8, 0}},     {1024, 8, 256, 2, {16, 8, 8, 0}},
    {2048, 4, 256, 2, {16, 16, 8, 0}},  {4096, 2, 256, 2, {16, 16, 16, 0}}, {8192, 1, 256, 2, {16, 16, 16, 2}},
    {1372, 4, 392, 2, {14, 14, 7, 0}},  {2744, 2, 392, 2, {14, 14, 14, 0}},
};
constexpr int kNumColumnRadices = sizeof(kColumnRadices) / sizeof(kColumnRadices[0]);

// Index into kColumnRadices, or -1 when n_theta has no specialised kernel.
int column_radices_index(int n_theta);

// Row (rho) complex transform lengths N_rho / 2 with a compile-time radix sequence (0 ends it).
// The compiled transform uses the same twiddle table as the generic one, not the plan's radix list.
struct RowRadices {
  int n;
  int r[5];
};
constexpr RowRadices kRowRadices[] = {
    {2187, {9, 9, 9, 3, 0}},  // N = 2048, M = 3
    {4374, {2, 9, 9, 9, 3}},  // N = 4096, M = 3
    {1120, {8, 4, 5, 7, 0}},  // N = 1024, M = 3
};
constexpr int kNumRowRadices = sizeof(kRowRadices) / sizeof(kRowRadices[0]);
int row_radices_index(int nc);  // index into kRowRadices, or -1

struct Radices {
  int n = 0;
  int count = 0;
  int r[kMaxRadices] = {0};
};

// Factor n (7-smooth) into Stockham radices from {8, 4, 2, 9, 3, 5, 7}.
bool factor_radices(int n, Radices* out);

int compute_geometry(int N, int n_angles, int n_det, int interp, int M, radon_plan_info* g);

// Raw FP64 zeta_hat (which = 0) / zeta#_hat (which = 1) on k_theta in [0, n_theta/2],
// k_rho in [0, N_rho/2]; interleaved (re, im), k_rho fastest.
void kernel_quadrant(const radon_plan_info& g, int which, std::vector<double>* out);

struct HostTables {
  Radices rad_rho;  // complex FFT of length N_rho / 2 (real transform of length N_rho)
  Radices rad_th;   // complex FFT of length n_theta
  std::vector<float> tw_rho;   // 2 * (N_rho/2): exp(-2 pi i p / (N_rho/2))
  std::vector<float> tw_r2c;   // 2 * (N_rho/2 + 1): exp(-2 pi i k / N_rho)
  std::vector<float> tw_th;    // 2 * n_theta: exp(-2 pi i p / n_theta)
  int col_fixed = -1;          // kColumnRadices index, -1: generic column kernel
  std::vector<float> tw_col;   // per-pass twiddles of the specialised column transform
  std::vector<float> k_fwd;    // 2 * (N_rho/2+1) * (n_theta/2+1), [k_rho][k_theta]
  std::vector<float> k_bp;     // same layout, back-projection kernel
  // forward sampling (Algorithm 1: resample T_m f on Omega_lp, downsample, multiply by e^rho)
  std::vector<float> fwd_row;  // 4 per (m, jj, q): cos(psi) S hi/lo, sin(psi) S hi/lo, S = N/(2 a_R)
  std::vector<float> fwd_m;    // 4 per m: column / row offset (hi, lo)
  std::vector<float> fwd_e;    // 2 per i: e^rho_i / r, e^rho_i - e^rho_anchor(i)
  std::vector<float> fwd_eanc; // 2 per anchor: e^rho_anchor hi/lo
  std::vector<int32_t> fwd_rng; // 2 per (m, jj, q): rho samples [lo, hi] whose taps lie in the
                                // padded array and within the disc margin (lo > hi: none)
  // forward output (Algorithm 1: resample from S_m^{-1} Omega_p to Sigma)
  std::vector<int32_t> fwd_ang;  // 4 per angle: m, flip, first tap row (halo index), frac (float bits)
  std::vector<int32_t> fwd_anc;  // 4 per (angle, k tile): I, F (float bits), g (float bits), 0
  // back-projection sampling (Algorithm 2: resample g(S_m) on Omega_p)
  std::vector<int32_t> bp_th;    // 2 per (m, jj): theta / dtheta as (int, frac bits)
  std::vector<int32_t> bp_c;     // 2 per jj: -(1-a_R) cos(phi_j) / (a_R ds) + n_det/2 as (int, frac bits)
  std::vector<int32_t> bp_e;     // 2 per i: e^rho_i / (a_R ds) as (int, frac bits)
  // back-projection output (Algorithm 2: resample to X and sum the partitions)
  std::vector<int32_t> bp_anc;   // 8 per (m, tile): I_theta, F_theta, I_rho, F_rho, y0x, y0y, 1/|y0|^2, 0
  std::vector<float> bp_m;       // 2 per m: a_R cos(m beta), a_R sin(m beta)
  // FBP filter along s: real FFT of length n_filter (complex length n_filter / 2)
  Radices rad_filt;
  std::vector<float> tw_filt;     // 2 * (n_filter/2): exp(-2 pi i p / (n_filter/2))
  std::vector<float> tw_filt_r2c; // 2 * (n_filter/2 + 1): exp(-2 pi i k / n_filter)
  std::vector<float> filt;        // 3 * (n_filter/2 + 1): transfer functions / n_filter (ramp, SL, cosine)
};

int build_tables(const radon_plan_info& g, HostTables* t);

}  // namespace radon
