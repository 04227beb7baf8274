// Definition of the opaque radon_plan handle (shared by the C ABI translation units).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "radon.h"
#include "radon_kernels.cuh"

struct radon_plan_s {
  radon_plan_info info;
  radon::DevPlan dp;
  int device = -1;
  void* table_mem = nullptr;
  void* scratch_mem = nullptr;
  size_t table_bytes = 0;
  float* io_image = nullptr;  // device staging for the host-buffer entry points
  float* io_sino = nullptr;
  // per-stage event timing (radon_profile_enable / radon_profile_read)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_pool;
  std::vector<int> prof_stage;  // stage id recorded with each used event (-1: start of a call)
  size_t prof_used = 0;
  cudaError_t prof_err = cudaSuccess;
};
