// The batched operator's persistent kernel for fp32 meshes
// (batch_kernels.cuh): the fp32 k-loop body for every lx in [2, 12].
#include "batch_kernels.cuh"

namespace ax {

#define AX_BATCH_LX(M) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12)

__global__ void __launch_bounds__(kBatchThreads, 4)
batch_f32_kernel(const BatchMeshDev *__restrict__ meshes, const BatchItem *__restrict__ items,
                 const BatchGroup *__restrict__ groups, const int *__restrict__ cta_start) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int g1 = cta_start[blockIdx.x + 1];
  for (int g = cta_start[blockIdx.x]; g < g1; ++g) {
    const BatchGroup G = groups[g];
    switch (G.key / 2) {
#define AX_CASE(L)                                   \
  case L:                                            \
    batch_run_kloop<false, L>(G, items, meshes, sm); \
    break;
      AX_BATCH_LX(AX_CASE)
#undef AX_CASE
      default:
        break;
    }
    __syncthreads();
  }
}

size_t batch_key_smem_f32(int key) {
  switch (key / 2) {
#define AX_CASE(L) \
  case L:          \
    return kstep_smem<L, float, false, kstep_vec<L, float>()>(batch_kloop_epb(L));
    AX_BATCH_LX(AX_CASE)
#undef AX_CASE
    default:
      return 0;
  }
}

int batch_launch_f32(int nblocks, size_t smem, const BatchMeshDev *meshes,
                     const BatchItem *items, const BatchGroup *groups, const int *cta_start,
                     cudaStream_t st) {
  batch_f32_kernel<<<nblocks, kBatchThreads, smem, st>>>(meshes, items, groups, cta_start);
  return launch_status();
}

int batch_setup_f32(size_t smem, int *bps) {
  static std::atomic<size_t> granted[kMaxDevices];
  if (!grant_smem(batch_f32_kernel, smem, granted)) return AX_EINVAL;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, batch_f32_kernel, kBatchThreads, smem) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  return AX_OK;
}

}  // namespace ax
