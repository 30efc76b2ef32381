// Deterministic block reductions and the fixed launch shape of the solver's
// vector kernels.
//
// Every reduction runs in two passes with a fixed grid: pass one writes one
// partial per block (grid-stride loop in a fixed order, a fixed warp-shuffle
// tree inside the block), pass two sums the partials in index order in one
// block.  The result is therefore bitwise reproducible run to run, which the
// solvers' checkpoint/resume relies on.
#pragma once

#include "common.cuh"

namespace ax {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 152 * 4;  // 4 blocks per SM of the 152-SM part

// Sum of v over the block; valid in thread 0.  Deterministic order.
template <int NV>
AX_D void block_sum(double (&v)[NV], double *sh /* [NV][kRedThreads/32] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    if (lane == 0) sh[q * (kRedThreads / 32) + wid] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int k = 0; k < kRedThreads / 32; ++k) s += sh[q * (kRedThreads / 32) + k];
      v[q] = s;
    }
  }
}

// Sums partials[q * nblk + b] over b for q < NV: one warp per quantity,
// lane l adding b = l, l+32, ... in order, then a fixed shuffle tree.
template <int NV>
AX_D void warp_sum_partials(const double *__restrict__ partials, int nblk, double *out) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= NV) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += partials[(size_t)q * nblk + b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) out[q] = s;
}

// Sum of partials[0 .. nblk) by the whole block (blockDim.x a multiple of
// 32, at most 1024): thread t adds t, t + blockDim.x, ... in order, then a
// fixed shuffle tree and a fixed-order sum over the warps.  Valid in thread
// 0.  For the many partials (one per element block) of a fused reduction.
AX_D double block_sum_partials(const double *__restrict__ partials, int nblk, double *sh) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partials[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
  return t;
}

}  // namespace ax
