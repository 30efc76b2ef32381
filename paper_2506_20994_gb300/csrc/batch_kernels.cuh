// Persistent multi-mesh kernels of the batched operator (batch.cu): one
// kernel per (dtype, lx), each block walking its own statically assigned
// list of work items and running the single-mesh device body on each, so
// that every kernel keeps the register footprint and occupancy of its
// single-mesh counterpart.  fp64 meshes of the even-odd orders run on
// geometry the plan prepared once (as the operator handle does).
#pragma once

#include "ax_df64.cuh"
#include "ax_df64_eo.cuh"
#include "ax_kstep.cuh"

namespace ax {

struct BatchMeshDev {
  int lx, epb;
  void *w;
  const void *u, *dx, *dxt, *h1, *g[6];
  const df::dd2 *gp;  // geometry prepared for the even-odd kernel, or null
  const unsigned *gstat;  // its per-element exponent keys (guard.cuh)
};

struct BatchItem {
  int mesh, nel;
  long long e0;
};

constexpr int kBatchThreads = 256;

// Thread layout of a group's kernel: the k-loop body (lx^2 threads per
// element walking k) or the even-odd body on prepared geometry ((lx/2)^3
// threads per element, fp64 and even lx only).
enum BatchBody : int { kBodyKLoop = 0, kBodyEvenOdd = 1 };

// The default fp64 layout (ax_helm's built-in choice) for lx.
__host__ __device__ constexpr bool batch_uses_eo(int lx) {
  return lx == 8 || lx == 10 || lx == 12;
}
__host__ __device__ constexpr bool batch_eo_ok(int lx) { return lx >= 4 && lx <= 12 && lx % 2 == 0; }

template <bool F64, int LX, int BODY = kBodyKLoop>
__global__ void __launch_bounds__(kBatchThreads, 2)
batch_lx_kernel(const BatchMeshDev *__restrict__ meshes, const BatchItem *__restrict__ items,
                const int *__restrict__ block_start) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b0 = block_start[blockIdx.x], b1 = block_start[blockIdx.x + 1];
  for (int it = b0; it < b1; ++it) {
    const BatchItem itm = items[it];
    const BatchMeshDev m = meshes[itm.mesh];
    if constexpr (F64 && BODY == kBodyEvenOdd) {
      // every mesh of this group has prepared geometry (the plan made it)
      df64eo_body<LX, true>((double *)m.w, (const double *)m.u, (const double *)m.dx,
                            (const double *)m.dxt, (const double *)m.h1, (const double *)m.g[0],
                            (const double *)m.g[1], (const double *)m.g[2], (const double *)m.g[3],
                            (const double *)m.g[4], (const double *)m.g[5], m.gp, m.gstat,
                            itm.e0, itm.nel, m.epb, smem_raw);
    } else if constexpr (F64) {
      df64_body<LX>((double *)m.w, (const double *)m.u, (const double *)m.dx,
                    (const double *)m.dxt, (const double *)m.h1, (const double *)m.g[0],
                    (const double *)m.g[1], (const double *)m.g[2], (const double *)m.g[3],
                    (const double *)m.g[4], (const double *)m.g[5], itm.e0, itm.nel, m.epb,
                    smem_raw);
    } else {
      kstep_body<LX, float, float, float, float>(
          (float *)m.w, (const float *)m.u, (const float *)m.dx, (const float *)m.dxt,
          (const float *)m.h1, (const float *)m.g[0], (const float *)m.g[1],
          (const float *)m.g[2], (const float *)m.g[3], (const float *)m.g[4],
          (const float *)m.g[5], itm.e0, itm.nel, m.epb, smem_raw);
    }
    __syncthreads();  // the next item reuses shared memory
  }
}

// Per-(dtype, lx) host helpers, defined in batch_f64.cu / batch_f32.cu.
// launch: one persistent launch; setup: sets the shared-memory limit and
// returns the resident blocks per SM for smem bytes (0 if it does not fit).
int batch_lx_launch(bool f64, int lx, int nblocks, size_t smem, const BatchMeshDev *meshes,
                    const BatchItem *items, const int *block_start, cudaStream_t st);
int batch_lx_setup(bool f64, int lx, size_t smem, int *blocks_per_sm);

}  // namespace ax
