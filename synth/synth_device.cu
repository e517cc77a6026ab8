// synth_device.cu -- device side of the generator defined in synth.h (same
// bytes as synth_host.c).  Used to fill large inputs directly in HBM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "synth.h"

namespace {

struct Thr {
  unsigned long long v[256];
};

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t pick(const unsigned long long* thr, uint64_t r) {
  uint32_t lo = 0, hi = 255;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (r < thr[mid]) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

template <bool EARLY>
__global__ void fill_kernel(uint8_t* out, size_t n, Thr thr, uint64_t seed, uint64_t counter0) {
  // EARLY: let a kernel launched after this one with programmatic stream
  // serialisation start at once (as some library kernels do), so that it
  // runs while these bytes are still being written
  if (EARLY) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ unsigned long long t[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) t[i] = thr.v[i];
  __syncthreads();
  size_t stride = (size_t)gridDim.x * blockDim.x * 16;
  for (size_t a = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 16; a < n; a += stride) {
    uint8_t b[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) b[j] = (uint8_t)pick(t, splitmix64_at(seed, counter0 + a + j) >> 32);
    if (a + 16 <= n && (((uintptr_t)(out + a)) & 15) == 0) {
      uint4 w;
      w.x = b[0] | (b[1] << 8) | (b[2] << 16) | ((uint32_t)b[3] << 24);
      w.y = b[4] | (b[5] << 8) | (b[6] << 16) | ((uint32_t)b[7] << 24);
      w.z = b[8] | (b[9] << 8) | (b[10] << 16) | ((uint32_t)b[11] << 24);
      w.w = b[12] | (b[13] << 8) | (b[14] << 16) | ((uint32_t)b[15] << 24);
      *reinterpret_cast<uint4*>(out + a) = w;
    } else {
      for (int j = 0; j < 16 && a + j < n; ++j) out[a + j] = b[j];
    }
  }
}

__global__ void ramp_kernel(uint8_t* out, size_t n, uint64_t counter0) {
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = (uint8_t)(counter0 + i);
}

int grid_for(size_t work_items) {
  size_t g = (work_items + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

extern "C" int synth_fill_device(uint8_t* d_out, size_t n, const uint64_t thr[256], uint64_t seed,
                                 uint64_t counter0, void* stream) {
  if (n == 0) return 0;
  Thr t;
  for (int i = 0; i < 256; ++i) t.v[i] = thr[i];
  fill_kernel<false><<<grid_for((n + 15) / 16), 256, 0, (cudaStream_t)stream>>>(d_out, n, t, seed, counter0);
  return (int)cudaGetLastError();
}

extern "C" int synth_fill_device_early(uint8_t* d_out, size_t n, const uint64_t thr[256], uint64_t seed,
                                       uint64_t counter0, void* stream) {
  if (n == 0) return 0;
  Thr t;
  for (int i = 0; i < 256; ++i) t.v[i] = thr[i];
  fill_kernel<true><<<grid_for((n + 15) / 16), 256, 0, (cudaStream_t)stream>>>(d_out, n, t, seed, counter0);
  return (int)cudaGetLastError();
}

extern "C" int synth_ramp_device(uint8_t* d_out, size_t n, uint64_t counter0, void* stream) {
  if (n == 0) return 0;
  ramp_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(d_out, n, counter0);
  return (int)cudaGetLastError();
}
