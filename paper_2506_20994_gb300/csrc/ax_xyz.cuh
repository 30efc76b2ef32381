// Kernels of the element operator with one 1-D matrix per direction (the
// full argument list of Listings 1-2); instantiated per lx range in
// ax_xyz*.cu so that they compile in parallel.
#pragma once

#include "ax_df64.cuh"
#include "ax_kstep.cuh"
#include "dispatch.h"

namespace ax {
namespace xyz {

#define AX_XYZ_PARAMS                                                                          \
  double *__restrict__ w, const double *__restrict__ u, const double *__restrict__ dx,         \
      const double *__restrict__ dy, const double *__restrict__ dz,                            \
      const double *__restrict__ dxt, const double *__restrict__ dyt,                          \
      const double *__restrict__ dzt, const double *__restrict__ h1,                           \
      const double *__restrict__ g11, const double *__restrict__ g22,                          \
      const double *__restrict__ g33, const double *__restrict__ g12,                          \
      const double *__restrict__ g13, const double *__restrict__ g23, int nelv, int epb
#define AX_XYZ_ARGS w, u, dx, dy, dz, dxt, dyt, dzt, h1, g11, g22, g33, g12, g13, g23, nelv, epb

template <int LX>
__global__ void __launch_bounds__(256) ax_df64_xyz_kernel(AX_XYZ_PARAMS) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long e0 = (long long)blockIdx.x * epb;
  const long long left = nelv - e0;
  const int nel = left < epb ? (int)left : epb;
  df64_body<LX, true>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, e0, nel, epb, smem_raw,
                      dy, dz, dyt, dzt);
}

template <int LX>
__global__ void __launch_bounds__(256) ax_kstep_xyz_kernel(AX_XYZ_PARAMS) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long e0 = (long long)blockIdx.x * epb;
  const long long left = nelv - e0;
  const int nel = left < epb ? (int)left : epb;
  kstep_body<LX, double, double, double, double, false, true>(
      w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, e0, nel, epb, smem_raw, nullptr, dy, dz,
      dyt, dzt);
}

// about 256 threads per block, whole elements (lx*lx threads each)
// (double-float kernel for lx <= 12, fp64 units above: the six-matrix form
// is not a benchmark path, and this keeps its instantiations quick to build)
template <int LX>
int launch_xyz(AX_XYZ_PARAMS, cudaStream_t st) {
  constexpr bool DF = LX <= 12;
  epb = 256 / (LX * LX) < 1 ? 1 : 256 / (LX * LX);
  size_t smem;
  void (*kern)(AX_XYZ_PARAMS);
  if constexpr (DF) {
    smem = df64_smem<LX, true>(epb);
    kern = ax_df64_xyz_kernel<LX>;
  } else {
    smem = kstep_smem<LX, double, true>(epb);
    kern = ax_kstep_xyz_kernel<LX>;
  }
  static std::atomic<size_t> granted[kMaxDevices];
  if (!grant_smem(kern, smem, granted)) return AX_EINVAL;
  const unsigned grid = (unsigned)((nelv + epb - 1) / epb);
  kern<<<grid, epb * LX * LX, smem, st>>>(AX_XYZ_ARGS);
  return launch_status();
}

// per lx range (one translation unit each): a 2-7, b 8-10, c 11-12, d 13-16
int dispatch_a(int lx, AX_XYZ_PARAMS, cudaStream_t st);
int dispatch_b(int lx, AX_XYZ_PARAMS, cudaStream_t st);
int dispatch_c(int lx, AX_XYZ_PARAMS, cudaStream_t st);
int dispatch_d(int lx, AX_XYZ_PARAMS, cudaStream_t st);

}  // namespace xyz
}  // namespace ax

// switch over the lx of one range
#define AX_XYZ_DISPATCH(NAME, CASES)                               \
  int NAME(int lx, AX_XYZ_PARAMS, cudaStream_t st) {               \
    switch (lx) {                                                  \
      CASES(AX_XYZ_CASE)                                           \
      default:                                                     \
        return AX_EINVAL;                                          \
    }                                                              \
  }
#define AX_XYZ_CASE(L) \
  case L:              \
    return launch_xyz<L>(AX_XYZ_ARGS, st);
