// The batched operator's persistent kernel for fp32 meshes
// (batch_kernels.cuh): the even-odd fp32 body for lx 6, 8, 10, the fp32
// k-loop body for every lx in [2, 12].
#include "batch_kernels.cuh"

namespace ax {

#define AX_BATCH_LX(M) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12)
#define AX_BATCH_E32(M) M(6) M(8) M(10)

__global__ void __launch_bounds__(kBatchThreads, 3)
batch_f32_kernel(const BatchMeshDev *__restrict__ meshes, const F32Mesh *__restrict__ fmesh,
                 const BatchItem *__restrict__ items, const BatchGroup *__restrict__ groups,
                 const int *__restrict__ cta_start, int *__restrict__ err) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int g1 = cta_start[blockIdx.x + 1];
  for (int g = cta_start[blockIdx.x]; g < g1; ++g) {
    const BatchGroup G = groups[g];
    switch (G.key) {
#define AX_CASE(L)                                   \
  case 2 * L + kBodyKLoop:                           \
    batch_run_kloop<false, L>(G, items, meshes, sm); \
    break;
      AX_BATCH_LX(AX_CASE)
#undef AX_CASE
#define AX_CASE(L)                                   \
  case 2 * L + kBodyEvenOdd:                         \
    batch_run_e32<L>(G, items, fmesh, sm, err);      \
    break;
      AX_BATCH_E32(AX_CASE)
#undef AX_CASE
      default:
        break;
    }
    __syncthreads();  // the next group gives the shared memory another layout
  }
}

size_t batch_key_smem_f32(int key) {
  if (key % 2 == kBodyEvenOdd) {
    switch (key / 2) {
#define AX_CASE(L) \
  case L:          \
    return (size_t)batch_e32_slots<L>() * batch_e32_slot_bytes<L>();
      AX_BATCH_E32(AX_CASE)
#undef AX_CASE
      default:
        return 0;
    }
  }
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
                     const F32Mesh *fmesh, const BatchItem *items, const BatchGroup *groups,
                     const int *cta_start, int *err, cudaStream_t st) {
  batch_f32_kernel<<<nblocks, kBatchThreads, smem, st>>>(meshes, fmesh, items, groups, cta_start,
                                                         err);
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
