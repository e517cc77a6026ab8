// hist_internal.h -- host helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hist.h"

namespace histlib {

constexpr int kMaxDevices = 64;

// Record a CUDA error for hist_last_cuda_error() and return HIST_ECUDA.
int cuda_fail(cudaError_t e);
// SMs of the current device.
int sm_count();
// Opt a kernel into the library's dynamic shared-memory size on this device.
int ensure_smem_attr(const void* fn, int* done);
int ensure_smem_attr_bytes(const void* fn, int* done, size_t bytes);
// The one-shot histogram (hist_plain / hist_adaptive).
int oneshot(const uint8_t* d_in, size_t n, const hist_pattern* d_pat, uint32_t* d_out, cudaStream_t s);

}  // namespace histlib
