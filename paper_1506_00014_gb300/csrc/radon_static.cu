// radon_forward_static_scratch (include/radon.h): the forward transform with its intermediate
// arrays in a file-scope static device array instead of plan-owned memory, for callers that must
// not allocate device memory when they run a transform.  It launches the same kernels as
// radon_forward; only the scratch pointers differ.
#include <cuda_runtime.h>

#include <mutex>

#include "plan_host.h"
#include "plan_internal.h"
#include "radon.h"
#include "radon_kernels.cuh"

namespace {

constexpr size_t kStaticScratchBytes = RADON_STATIC_SCRATCH_BYTES;

// Held by every device that loads the library, until process exit.  In host code this name is a
// host-side stand-in: kernels get the device address obtained by cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_device_address[kMaxDevices] = {nullptr};

// Device address of g_static_scratch on the current device `dev`; looked up once per device.
cudaError_t static_scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_device_address[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_device_address[dev] = p;
  }
  *out = g_device_address[dev];
  return cudaSuccess;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return RADON_OK;
  if (e == cudaErrorMemoryAllocation) return RADON_OUT_OF_MEMORY;
  return RADON_CUDA_ERROR;
}

}  // namespace

extern "C" int radon_forward_static_scratch(radon_plan plan, const float* d_image, float* d_sino, void* stream) {
  if (!plan || !d_image || !d_sino) return RADON_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device) return RADON_INVALID_ARG;

  // Same intermediate arrays as the plan's own scratch, packed from offset 0.
  const radon::DevPlan& p0 = plan->dp;
  const size_t nrow = static_cast<size_t>(p0.nh) + radon::kHaloLo + radon::kHaloHi;
  const size_t b_img = sizeof(float) * static_cast<size_t>(p0.img_pitch) * p0.img_pitch;
  const size_t b_x = sizeof(float2) * static_cast<size_t>(p0.M) * p0.nh * p0.x_pitch;
  const size_t b_ys = sizeof(float2) * static_cast<size_t>(p0.M) * nrow * p0.x_pitch;
  const size_t b_y = sizeof(float) * static_cast<size_t>(p0.M) * nrow * p0.y_pitch;
  const size_t o_img = 0;
  const size_t o_x = align_up(o_img + b_img, 256);
  const size_t o_ys = align_up(o_x + b_x, 256);
  const size_t o_y = align_up(o_ys + b_ys, 256);
  if (o_y + b_y > kStaticScratchBytes) return RADON_EXCEEDS_STATIC_SCRATCH;

  void* base = nullptr;
  cudaError_t e = static_scratch_address(dev, &base);
  if (e != cudaSuccess) return status_of(e);
  char* b = static_cast<char*>(base);
  radon::DevPlan p = p0;
  p.coef_img = reinterpret_cast<float*>(b + o_img);
  p.img_quad = 0;  // no room for the quad layout: 16 scalar loads per sample
  p.batch_cap = 1;
  p.xspec = reinterpret_cast<float2*>(b + o_x);
  p.yspec = reinterpret_cast<float2*>(b + o_ys);
  p.ylp = reinterpret_cast<float*>(b + o_y);

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The coefficient image's zero border and the unused pad columns of the log-polar rows must
  // read zero; the array still holds whatever the previous call (of any plan) left there.
  e = cudaMemsetAsync(p.coef_img, 0, b_img, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.ylp, 0, b_y, st);
  if (e != cudaSuccess) return status_of(e);
  radon::StageHook no_hook;
  no_hook.mark = nullptr;
  no_hook.ctx = nullptr;
  return status_of(radon::launch_forward(p, d_image, d_sino, st, no_hook));
}
