// C ABI of libradon (declared in include/radon.h): plan lifecycle and transform entry points.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "plan_host.h"
#include "plan_internal.h"
#include "radon.h"
#include "radon_kernels.cuh"


namespace {

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return RADON_OK;
  if (e == cudaErrorMemoryAllocation) return RADON_OUT_OF_MEMORY;
  return RADON_CUDA_ERROR;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Packs host vectors into one device allocation.
class TablePacker {
 public:
  template <class T>
  size_t add(const std::vector<T>& v) {
    const size_t off = total_;
    parts_.push_back({off, v.data(), v.size() * sizeof(T)});
    total_ = align_up(total_ + v.size() * sizeof(T), 256);
    return off;
  }
  size_t total() const { return total_; }
  cudaError_t upload(void* dev) const {
    for (const auto& p : parts_) {
      if (!p.bytes) continue;
      cudaError_t e = cudaMemcpy(static_cast<char*>(dev) + p.off, p.src, p.bytes, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

 private:
  struct Part {
    size_t off;
    const void* src;
    size_t bytes;
  };
  std::vector<Part> parts_;
  size_t total_ = 0;
};

unsigned magic_of(int d) { return d == 1 ? 0u : static_cast<unsigned>((0x100000000ULL + d - 1) / d); }

bool copy_radices(const radon::Radices& r, int max_batch, radon::RadixList* out) {
  if (r.count > 16 || static_cast<long long>(r.n) * max_batch >= (1 << 15)) return false;
  std::memset(out, 0, sizeof(*out));
  out->n = r.n;
  out->count = r.count;
  int Ns = 1;
  for (int i = 0; i < r.count; ++i) {
    radon::FftPass& ps = out->p[i];
    ps.R = r.r[i];
    ps.Ns = Ns;
    ps.nbf = r.n / ps.R;
    ps.tstep = r.n / (Ns * ps.R);
    ps.m_nbf = magic_of(ps.nbf);
    ps.m_ns = magic_of(Ns);
    Ns *= ps.R;
  }
  return true;
}

void prof_mark(void* ctx, int stage, cudaStream_t st) {
  radon_plan_s* p = static_cast<radon_plan_s*>(ctx);
  if (p->prof_used == p->prof_pool.size()) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) {
      p->prof_err = e;
      return;
    }
    p->prof_pool.push_back(ev);
    p->prof_stage.push_back(0);
  }
  cudaError_t e = cudaEventRecord(p->prof_pool[p->prof_used], st);
  if (e != cudaSuccess) {
    p->prof_err = e;
    return;
  }
  p->prof_stage[p->prof_used++] = stage;
}

radon::StageHook hook_of(radon_plan_s* p) {
  radon::StageHook h;
  h.mark = p->prof_on ? prof_mark : nullptr;
  h.ctx = p;
  return h;
}

// Frees the scratch buffer (the device must be idle).
void release_scratch(radon_plan_s* p) {
  if (p->scratch_mem) cudaFree(p->scratch_mem);
  p->scratch_mem = nullptr;
}

// Scratch buffers for `cap` same-size slices; replaces the previous ones.  Slice b of a batch
// uses the buffers at offset b * (per-slice size).
cudaError_t allocate_scratch(radon_plan_s* p, int cap) {
  radon::DevPlan& d = p->dp;
  const int N = d.N, na = d.n_angles, nd = d.n_det;
  const size_t nrow = static_cast<size_t>(d.nh) + radon::kHaloLo + radon::kHaloHi;
  const size_t e_img = static_cast<size_t>(d.img_pitch) * d.img_pitch;
  const size_t e_sino = static_cast<size_t>(na) * d.sino_pitch;
  const size_t e_x = static_cast<size_t>(d.M) * d.nh * d.x_pitch;
  const size_t e_ys = static_cast<size_t>(d.M) * nrow * d.x_pitch;
  const size_t e_y = static_cast<size_t>(d.M) * nrow * d.y_pitch;
  if (cap < 1) return cudaErrorInvalidValue;
  size_t sc = 0;
  auto take = [&](size_t bytes) {
    const size_t off = sc;
    sc = align_up(sc + bytes, 256);
    return off;
  };
  const size_t s_img = take(sizeof(float) * e_img * cap);
  const size_t s_q4 = take(sizeof(float4) * e_img * cap);
  const size_t s_sino = take(sizeof(float) * e_sino * cap);
  const size_t s_x = take(sizeof(float2) * e_x * cap);
  const size_t s_ys = take(sizeof(float2) * e_ys * cap);
  const size_t s_y = take(sizeof(float) * e_y * cap);
  const size_t s_ftmp = take(sizeof(float) * static_cast<size_t>(na) * nd);
  const size_t s_io_img = take(sizeof(float) * static_cast<size_t>(N) * N);
  const size_t s_io_sino = take(sizeof(float) * static_cast<size_t>(na) * nd);
  void* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, sc);
  if (e == cudaSuccess) e = cudaMemset(mem, 0, sc);  // zero borders and pad columns stay zero
  if (e != cudaSuccess) {
    cudaFree(mem);
    return e;
  }
  release_scratch(p);
  char* sb = static_cast<char*>(mem);
  p->scratch_mem = mem;
  d.coef_img = reinterpret_cast<float*>(sb + s_img);
  d.coef_q4 = reinterpret_cast<float4*>(sb + s_q4);
  d.img_quad = 1;
  d.coef_sino = reinterpret_cast<float*>(sb + s_sino);
  d.xspec = reinterpret_cast<float2*>(sb + s_x);
  d.yspec = reinterpret_cast<float2*>(sb + s_ys);
  d.ylp = reinterpret_cast<float*>(sb + s_y);
  d.sino_tmp = reinterpret_cast<float*>(sb + s_ftmp);
  d.bs_img = e_img;
  d.bs_sino = e_sino;
  d.bs_x = e_x;
  d.bs_ys = e_ys;
  d.bs_y = e_y;
  d.batch_cap = cap;
  p->io_image = reinterpret_cast<float*>(sb + s_io_img);
  p->io_sino = reinterpret_cast<float*>(sb + s_io_sino);
  p->info.device_bytes = p->table_bytes + sc;
  return cudaSuccess;
}

bool on_plan_device(const radon_plan_s* p) {
  int dev = -1;
  return cudaGetDevice(&dev) == cudaSuccess && dev == p->device;
}

}  // namespace

extern "C" {

const char* radon_status_string(int status) {
  switch (status) {
    case RADON_OK: return "ok";
    case RADON_INVALID_ARG: return "invalid argument";
    case RADON_OUT_OF_MEMORY: return "out of memory";
    case RADON_CUDA_ERROR: return "CUDA error";
    case RADON_TIMEOUT: return "timeout";
    case RADON_NOT_SUPPORTED: return "not supported";
    case RADON_EXCEEDS_STATIC_SCRATCH:
      return "plan's intermediate arrays exceed the static scratch array (RADON_STATIC_SCRATCH_BYTES)";
    default: return "unknown status";
  }
}

int radon_geometry(int N, int n_angles, int n_det, int interp_order, int n_partitions, radon_plan_info* out) {
  return radon::compute_geometry(N, n_angles, n_det, interp_order, n_partitions, out);
}

int radon_kernel_quadrant(int N, int n_angles, int n_det, int n_partitions, int which, double* out) {
  if (!out || (which != 0 && which != 1)) return RADON_INVALID_ARG;
  radon_plan_info g;
  int s = radon::compute_geometry(N, n_angles, n_det, 3, n_partitions, &g);
  if (s != RADON_OK) return s;
  std::vector<double> v;
  radon::kernel_quadrant(g, which, &v);
  std::memcpy(out, v.data(), v.size() * sizeof(double));
  return RADON_OK;
}

void radon_plan_destroy(radon_plan plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  for (cudaEvent_t ev : plan->prof_pool) cudaEventDestroy(ev);
  release_scratch(plan);
  cudaFree(plan->table_mem);
  delete plan;
}

int radon_plan_create(radon_plan* out, int N, int n_angles, int n_det, int interp_order, int n_partitions) {
  if (!out) return RADON_INVALID_ARG;
  *out = nullptr;
  radon_plan_info g;
  int s = radon::compute_geometry(N, n_angles, n_det, interp_order, n_partitions, &g);
  if (s != RADON_OK) return s;
  radon::HostTables t;
  s = radon::build_tables(g, &t);
  if (s != RADON_OK) return s;

  radon_plan_s* p = new (std::nothrow) radon_plan_s();
  if (!p) return RADON_OUT_OF_MEMORY;
  p->info = g;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return RADON_CUDA_ERROR;
  }
  radon::DevPlan& d = p->dp;
  std::memset(&d, 0, sizeof(d));
  d.N = N;
  d.n_angles = n_angles;
  d.n_det = n_det;
  d.M = n_partitions;
  d.interp = interp_order;
  d.N_rho = g.N_rho;
  d.nh = g.n_theta_half;
  d.n_theta = g.n_theta;
  d.r = g.r;
  d.nc = g.N_rho / 2;
  d.img_pitch = N + 2 * radon::kPad;
  d.sino_pitch = static_cast<int>(align_up(n_det + 1 + 2 * radon::kPad, 4));
  d.x_pitch = static_cast<int>(align_up(d.nc + 1, 4));
  d.y_pitch = static_cast<int>(align_up(g.N_rho + 2 * radon::kPad, 4));
  d.n_eanc = (g.N_rho + radon::kETile - 1) / radon::kETile;
  d.n_ktiles = (n_det + radon::kKTile - 1) / radon::kKTile;
  d.n_ptiles = (N + radon::kPTile - 1) / radon::kPTile;
  d.live_lo = n_det;
  d.live_hi = -1;
  for (int k = 0; k < n_det; ++k) {  // |s_k| < 1  <=>  2 (2k - n_det)^2 < n_det^2
    const long long v = 2LL * k - n_det;
    if (2 * v * v < static_cast<long long>(n_det) * n_det) {
      if (k < d.live_lo) d.live_lo = k;
      d.live_hi = k;
    }
  }
  d.col_group = 4;  // shared memory of a column CTA: (2 G + 1) n_theta complex
  while (d.col_group > 1 && (2 * static_cast<size_t>(d.col_group) + 1) * g.n_theta * sizeof(float2) > (60u << 10))
    d.col_group /= 2;
  if ((2 * static_cast<size_t>(d.col_group) + 1) * g.n_theta * sizeof(float2) > (220u << 10) ||
      3 * static_cast<size_t>(g.N_rho / 2) * sizeof(float2) > (220u << 10)) {
    delete p;
    return RADON_NOT_SUPPORTED;
  }
  d.inv_drho = static_cast<float>(1.0 / g.d_rho);
  d.inv_dphi = static_cast<float>(1.0 / g.d_phi);
  d.inv_aR = static_cast<float>(1.0 / g.a_R);
  d.d_s = static_cast<float>(g.d_s);
  d.n_filt = g.n_filter;
  d.col_fixed = t.col_fixed;
  d.row_fixed = radon::row_radices_index(g.N_rho / 2);
  if (!copy_radices(t.rad_rho, 1, &d.rad_rho) || !copy_radices(t.rad_th, d.col_group, &d.rad_th) ||
      !copy_radices(t.rad_filt, 1, &d.rad_filt)) {
    delete p;
    return RADON_NOT_SUPPORTED;
  }

  TablePacker tp;
  const size_t o_tw_rho = tp.add(t.tw_rho), o_tw_r2c = tp.add(t.tw_r2c), o_tw_th = tp.add(t.tw_th);
  const size_t o_tw_col = tp.add(t.tw_col);
  const size_t o_kf = tp.add(t.k_fwd), o_kb = tp.add(t.k_bp);
  const size_t o_frow = tp.add(t.fwd_row), o_fm = tp.add(t.fwd_m), o_fe = tp.add(t.fwd_e), o_fea = tp.add(t.fwd_eanc);
  const size_t o_frng = tp.add(t.fwd_rng);
  const size_t o_fang = tp.add(t.fwd_ang), o_fanc = tp.add(t.fwd_anc);
  const size_t o_bth = tp.add(t.bp_th), o_bc = tp.add(t.bp_c), o_be = tp.add(t.bp_e);
  const size_t o_banc = tp.add(t.bp_anc), o_bm = tp.add(t.bp_m);
  const size_t o_twf = tp.add(t.tw_filt), o_twfr = tp.add(t.tw_filt_r2c), o_filt = tp.add(t.filt);

  cudaError_t e = cudaMalloc(&p->table_mem, tp.total());
  if (e == cudaSuccess) e = tp.upload(p->table_mem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    radon_plan_destroy(p);
    return status_of(e);
  }
  char* tb = static_cast<char*>(p->table_mem);
  d.tw_rho = reinterpret_cast<const float2*>(tb + o_tw_rho);
  d.tw_r2c = reinterpret_cast<const float2*>(tb + o_tw_r2c);
  d.tw_th = reinterpret_cast<const float2*>(tb + o_tw_th);
  d.tw_col = reinterpret_cast<const float2*>(tb + o_tw_col);
  d.k_fwd = reinterpret_cast<const float2*>(tb + o_kf);
  d.k_bp = reinterpret_cast<const float2*>(tb + o_kb);
  d.fwd_row = reinterpret_cast<const float4*>(tb + o_frow);
  d.fwd_m = reinterpret_cast<const float4*>(tb + o_fm);
  d.fwd_e = reinterpret_cast<const float2*>(tb + o_fe);
  d.fwd_eanc = reinterpret_cast<const float2*>(tb + o_fea);
  d.fwd_rng = reinterpret_cast<const int2*>(tb + o_frng);
  d.fwd_ang = reinterpret_cast<const int4*>(tb + o_fang);
  d.fwd_anc = reinterpret_cast<const int4*>(tb + o_fanc);
  d.bp_th = reinterpret_cast<const int2*>(tb + o_bth);
  d.bp_c = reinterpret_cast<const int2*>(tb + o_bc);
  d.bp_e = reinterpret_cast<const int2*>(tb + o_be);
  d.bp_anc = reinterpret_cast<const int4*>(tb + o_banc);
  d.bp_m = reinterpret_cast<const float2*>(tb + o_bm);
  d.tw_filt = reinterpret_cast<const float2*>(tb + o_twf);
  d.tw_filt_r2c = reinterpret_cast<const float2*>(tb + o_twfr);
  d.filt = reinterpret_cast<const float*>(tb + o_filt);
  p->table_bytes = tp.total();
  e = allocate_scratch(p, 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    radon_plan_destroy(p);
    return status_of(e);
  }
  e = radon::configure_kernels(d);
  if (e != cudaSuccess) {  // cudaErrorInvalidValue: a kernel's shared memory would exceed the device limit
    cudaGetLastError();
    radon_plan_destroy(p);
    return e == cudaErrorInvalidValue ? RADON_NOT_SUPPORTED : status_of(e);
  }
  if (d.col_fixed >= 0) {  // the specialised in-place column kernel is the default where it exists
    radon::DevPlan f = d;
    f.col_group = 0;
    if (radon::configure_kernels(f) == cudaSuccess) d = f;
    cudaGetLastError();
  }
  p->info.column_group = d.col_group;
  *out = p;
  return RADON_OK;
}

int radon_plan_get_info(radon_plan plan, radon_plan_info* out) {
  if (!plan || !out) return RADON_INVALID_ARG;
  *out = plan->info;
  return RADON_OK;
}

int radon_forward(radon_plan plan, const float* d_image, float* d_sino, void* stream) {
  if (!plan || !d_image || !d_sino) return RADON_INVALID_ARG;
  if (!on_plan_device(plan)) return RADON_INVALID_ARG;
  return status_of(radon::launch_forward(plan->dp, d_image, d_sino, static_cast<cudaStream_t>(stream), hook_of(plan)));
}

int radon_backproject(radon_plan plan, const float* d_sino, float* d_image, void* stream) {
  if (!plan || !d_sino || !d_image) return RADON_INVALID_ARG;
  if (!on_plan_device(plan)) return RADON_INVALID_ARG;
  return status_of(radon::launch_backproject(plan->dp, d_sino, d_image, static_cast<cudaStream_t>(stream), hook_of(plan)));
}

int radon_fbp(radon_plan plan, const float* d_sino, float* d_image, int filter, void* stream) {
  if (!plan || !d_sino || !d_image) return RADON_INVALID_ARG;
  if (filter < RADON_FILTER_RAMP || filter > RADON_FILTER_COSINE) return RADON_INVALID_ARG;
  if (!on_plan_device(plan)) return RADON_INVALID_ARG;
  return status_of(radon::launch_fbp(plan->dp, d_sino, d_image, filter, static_cast<cudaStream_t>(stream), hook_of(plan)));
}

int radon_forward_host(radon_plan plan, const float* h_image, float* h_sino, void* stream) {
  if (!plan || !h_image || !h_sino) return RADON_INVALID_ARG;
  if (!on_plan_device(plan)) return RADON_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const radon_plan_info& g = plan->info;
  cudaError_t e = cudaMemcpyAsync(plan->io_image, h_image, sizeof(float) * static_cast<size_t>(g.N) * g.N,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = radon::launch_forward(plan->dp, plan->io_image, plan->io_sino, st, hook_of(plan));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_sino, plan->io_sino, sizeof(float) * static_cast<size_t>(g.n_angles) * g.n_det,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return status_of(e);
}

int radon_backproject_host(radon_plan plan, const float* h_sino, float* h_image, void* stream) {
  if (!plan || !h_sino || !h_image) return RADON_INVALID_ARG;
  if (!on_plan_device(plan)) return RADON_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const radon_plan_info& g = plan->info;
  cudaError_t e = cudaMemcpyAsync(plan->io_sino, h_sino, sizeof(float) * static_cast<size_t>(g.n_angles) * g.n_det,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = radon::launch_backproject(plan->dp, plan->io_sino, plan->io_image, st, hook_of(plan));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_image, plan->io_image, sizeof(float) * static_cast<size_t>(g.N) * g.N,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return status_of(e);
}

int radon_transpose(radon_plan plan, const float* d_sino, float* d_image, void* stream) {
  if (!plan || !d_sino || !d_image) return RADON_INVALID_ARG;
  if (!on_plan_device(plan)) return RADON_INVALID_ARG;
  return status_of(radon::launch_transpose(plan->dp, d_sino, d_image, static_cast<cudaStream_t>(stream), hook_of(plan)));
}

int radon_transpose_batch(radon_plan plan, const float* d_sinos, float* d_images, int batch, void* stream) {
  if (!plan || !d_sinos || !d_images || batch < 1 || batch > plan->dp.batch_cap) return RADON_INVALID_ARG;
  if (!on_plan_device(plan)) return RADON_INVALID_ARG;
  return status_of(
      radon::launch_transpose(plan->dp, d_sinos, d_images, static_cast<cudaStream_t>(stream), hook_of(plan), batch));
}

int radon_plan_reserve_batch(radon_plan plan, int max_batch) {
  if (!plan || max_batch < 1) return RADON_INVALID_ARG;
  if (!on_plan_device(plan)) return RADON_INVALID_ARG;
  if (max_batch <= plan->dp.batch_cap) return RADON_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = allocate_scratch(plan, max_batch);
  if (e == cudaErrorMemoryAllocation) cudaGetLastError();  // not sticky: clear it for later launches
  if (e == cudaErrorInvalidValue) return RADON_NOT_SUPPORTED;
  return status_of(e);
}

int radon_forward_batch(radon_plan plan, const float* d_images, float* d_sinos, int batch, void* stream) {
  if (!plan || !d_images || !d_sinos || batch < 1 || batch > plan->dp.batch_cap) return RADON_INVALID_ARG;
  if (!on_plan_device(plan)) return RADON_INVALID_ARG;
  return status_of(
      radon::launch_forward(plan->dp, d_images, d_sinos, static_cast<cudaStream_t>(stream), hook_of(plan), batch));
}

int radon_backproject_batch(radon_plan plan, const float* d_sinos, float* d_images, int batch, void* stream) {
  if (!plan || !d_images || !d_sinos || batch < 1 || batch > plan->dp.batch_cap) return RADON_INVALID_ARG;
  if (!on_plan_device(plan)) return RADON_INVALID_ARG;
  return status_of(
      radon::launch_backproject(plan->dp, d_sinos, d_images, static_cast<cudaStream_t>(stream), hook_of(plan), batch));
}

namespace {

// Checks every slice of an uneven batch before anything is launched.
bool multi_args_ok(const radon_plan* plans, const void* const* in, const void* const* out, int count) {
  if (!plans || !in || !out || count < 0) return false;
  for (int i = 0; i < count; ++i)
    if (!plans[i] || !in[i] || !out[i] || !on_plan_device(plans[i])) return false;
  return true;
}

}  // namespace

int radon_forward_multi(const radon_plan* plans, const float* const* d_images, float* const* d_sinos, int count,
                        void* stream) {
  if (!multi_args_ok(plans, reinterpret_cast<const void* const*>(d_images),
                     reinterpret_cast<const void* const*>(d_sinos), count))
    return RADON_INVALID_ARG;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < count; ++i) {
    const cudaError_t e = radon::launch_forward(plans[i]->dp, d_images[i], d_sinos[i], st, hook_of(plans[i]));
    if (e != cudaSuccess) return status_of(e);
  }
  return RADON_OK;
}

int radon_backproject_multi(const radon_plan* plans, const float* const* d_sinos, float* const* d_images, int count,
                            void* stream) {
  if (!multi_args_ok(plans, reinterpret_cast<const void* const*>(d_sinos),
                     reinterpret_cast<const void* const*>(d_images), count))
    return RADON_INVALID_ARG;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < count; ++i) {
    const cudaError_t e = radon::launch_backproject(plans[i]->dp, d_sinos[i], d_images[i], st, hook_of(plans[i]));
    if (e != cudaSuccess) return status_of(e);
  }
  return RADON_OK;
}

int radon_plan_set_column_group(radon_plan plan, int group) {
  if (!plan || (group != 0 && group != 1 && group != 2 && group != 4)) return RADON_INVALID_ARG;
  radon::DevPlan d = plan->dp;
  d.col_group = group;
  if (group == 0) {
    if (d.col_fixed < 0) return RADON_NOT_SUPPORTED;
  } else {
    radon::Radices rad;
    if (!radon::factor_radices(d.n_theta, &rad) || !copy_radices(rad, group, &d.rad_th)) return RADON_NOT_SUPPORTED;
  }
  if (radon::configure_kernels(d) != cudaSuccess) return RADON_NOT_SUPPORTED;
  plan->dp = d;
  plan->info.column_group = group;
  return RADON_OK;
}

int radon_plan_kernel_launches(radon_plan plan, int op, int* out) {
  if (!plan || !out) return RADON_INVALID_ARG;
  const int n = radon::kernel_launches(plan->dp, op);
  if (n < 0) return RADON_INVALID_ARG;
  *out = n;
  return RADON_OK;
}

int radon_profile_enable(radon_plan plan, int enable) {
  if (!plan) return RADON_INVALID_ARG;
  plan->prof_on = enable != 0;
  return RADON_OK;
}

int radon_profile_read(radon_plan plan, double* ms, int* launches) {
  if (!plan || !ms || !launches) return RADON_INVALID_ARG;
  cudaError_t e = plan->prof_err;
  plan->prof_err = cudaSuccess;
  for (size_t i = 1; i < plan->prof_used && e == cudaSuccess; ++i) {
    const int st = plan->prof_stage[i];
    if (st < 0 || st >= RADON_NUM_STAGES) continue;
    float t = 0.f;
    e = cudaEventSynchronize(plan->prof_pool[i]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, plan->prof_pool[i - 1], plan->prof_pool[i]);
    if (e == cudaSuccess) {
      ms[st] += t;
      launches[st] += 1;
    }
  }
  plan->prof_used = 0;
  return status_of(e);
}

}  // extern "C"
