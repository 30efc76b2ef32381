// Shared helpers of the CUDA library: status codes, argument checks, the
// element-field loaders for each storage type, and launch bookkeeping.
#pragma once

#include <atomic>
#include <mutex>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/axhelm.h"

#define AX_HD __host__ __device__ __forceinline__
#define AX_D __device__ __forceinline__

namespace ax {

// Converts a CUDA launch status into an AX code (never aborts).
inline int launch_status() {
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  return AX_OK;
}

inline bool lx_ok(int lx) { return lx >= AX_LX_MIN && lx <= AX_LX_MAX; }

template <typename... P>
inline bool all_nonnull(P... p) {
  bool ok = true;
  ((ok = ok && (p != nullptr)), ...);
  return ok;
}

// Storage -> compute conversion of one element-field value.
template <typename T>
AX_D T ld_cvt(const double *p) { return (T)__ldg(p); }
template <typename T>
AX_D T ld_cvt(const float *p) { return (T)__ldg(p); }
template <typename T>
AX_D T ld_cvt(const __nv_bfloat16 *p) { return (T)__bfloat162float(__ldg(p)); }

// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device when that is above the 48 KB default and above what this kernel was
// granted on this device before (the attribute is per device, so a process
// driving several GPUs raises it on each).  `granted` is the caller's table
// for one kernel, zero-initialised; raises are serialised so the recorded
// size only grows.  False if the device refuses or its index is out of range.
constexpr int kMaxDevices = 64;
inline std::mutex &smem_grant_mutex() {
  static std::mutex m;
  return m;
}
// Static shared memory of the kernels (guard record, reduction buffers) stays
// below this; the 48 KB default covers static and dynamic bytes together.
constexpr size_t kStaticSmemMargin = 4 * 1024;
template <typename K>
inline bool grant_smem(K kernel, size_t bytes, std::atomic<size_t> (&granted)[kMaxDevices]) {
  if (bytes + kStaticSmemMargin <= 48 * 1024) return true;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return false;
  }
  if (bytes <= granted[dev].load(std::memory_order_acquire)) return true;
  std::lock_guard<std::mutex> lock(smem_grant_mutex());
  if (bytes <= granted[dev].load(std::memory_order_relaxed)) return true;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  granted[dev].store(bytes, std::memory_order_release);
  return true;
}

// Asks the memory system to bring [p, p + bytes) into L2 (bulk copy engine).
// No data is returned.  The bulk unit needs a 16-byte aligned address and
// size; anything else (a caller's offset view) is skipped, since a prefetch
// is only a hint.
AX_D void prefetch_l2(const void *p, unsigned bytes) {
  if (((reinterpret_cast<uintptr_t>(p) | bytes) & 15u) != 0) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Explicitly rounded arithmetic (never contracted by the compiler).
AX_D double mul_rn(double a, double b) { return __dmul_rn(a, b); }
AX_D float mul_rn(float a, float b) { return __fmul_rn(a, b); }
AX_D double add_rn(double a, double b) { return __dadd_rn(a, b); }
AX_D float add_rn(float a, float b) { return __fadd_rn(a, b); }
AX_D double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
AX_D float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

}  // namespace ax
