// Shared helpers of the CUDA library: status codes, argument checks, the
// element-field loaders for each storage type, and launch bookkeeping.
#pragma once

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

// Sets the dynamic shared-memory limit of a kernel once per process
// (per kernel and per size class); returns false if the device refuses.
template <typename K>
inline bool ensure_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return true;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
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
