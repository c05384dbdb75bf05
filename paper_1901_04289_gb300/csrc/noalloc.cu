// arbgpu_int_mat_mul_noalloc: the exact integer matrix product of arbgpu_int_mat_mul for callers
// that cannot allocate device memory.  Its scratch space is one file-scope __device__ array of
// ARBGPU_NOALLOC_SCRATCH_BYTES, which every GPU that loads this code keeps until the process exits.
#include <mutex>

#include "internal.h"

// The shared scratch.  Host code must not take its address directly (in host code the name is a
// stand-in, not a device address): the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) uint8_t g_noalloc_scratch[ARBGPU_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch per device, once set up

// Set-up, once per device, with that device current: look up the array's device address.
arbgpu_status scratch_on_device(int dev, void **out) {
  if (dev < 0 || dev >= kMaxDevices) return ARBGPU_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ARBGPU_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return ARBGPU_OK;
}

}  // namespace

extern "C" arbgpu_status arbgpu_int_mat_mul_noalloc(uint64_t *T, int32_t t_limbs,
                                                    const uint64_t *X, int32_t x_limbs,
                                                    const uint64_t *Y, int32_t y_limbs, int64_t M,
                                                    int64_t K, int64_t N, int *status,
                                                    void *stream) {
  if (x_limbs < 1 || y_limbs < 1 || x_limbs > 32 || y_limbs > 32 || t_limbs < 1 || M < 0 ||
      K < 0 || N < 0 || M > (1 << 30) || N > (1 << 30) || K > (1 << 30))
    return ARBGPU_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ARBGPU_ERR_CUDA;
  // A context on the stack: nothing is allocated; device-side errors go to the caller's word.
  arbgpu_ctx local;
  local.device = dev;
  local.sm_count = 0;
  local.status = status;
  local.launches = 0;
  local.trace = false;
  if (cudaDeviceGetAttribute(&local.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ARBGPU_ERR_CUDA;
  if (t_limbs > 2 * 32 + 4) return ARBGPU_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (M == 0 || N == 0 || K == 0) {
    // No scratch is needed: an empty product writes nothing, K = 0 writes zeros.
    if (status && cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return ARBGPU_ERR_CUDA;
    return arbgpu::int_mat_mul_run(&local, T, t_limbs, X, x_limbs, Y, y_limbs, M, K, N, nullptr,
                                   0, s);
  }
  // Every operand and output entry takes at least one byte of scratch, so these products bound
  // the layout's size before it is computed; all three are below 2^61 and cannot wrap.
  const uint64_t cap = ARBGPU_NOALLOC_SCRATCH_BYTES;
  if ((uint64_t)M * (uint64_t)K > cap || (uint64_t)K * (uint64_t)N > cap ||
      (uint64_t)M * (uint64_t)N > cap)
    return ARBGPU_ERR_LIMIT;
  const size_t need = arbgpu::int_mat_mul_workspace(&local, x_limbs, y_limbs, M, K, N);
  if (need > ARBGPU_NOALLOC_SCRATCH_BYTES) return ARBGPU_ERR_LIMIT;
  void *scratch = nullptr;
  const arbgpu_status st = scratch_on_device(dev, &scratch);
  if (st != ARBGPU_OK) return st;
  if (status && cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return ARBGPU_ERR_CUDA;
  return arbgpu::int_mat_mul_run(&local, T, t_limbs, X, x_limbs, Y, y_limbs, M, K, N, scratch,
                                 ARBGPU_NOALLOC_SCRATCH_BYTES, s);
}
