// Persistent batched kernels for the f32 dtype, one per lx in [2, 12].
#include "batch_kernels.cuh"

namespace ax {

namespace {
template <int LX>
int launch_one(int nblocks, size_t smem, const BatchMeshDev *meshes, const BatchItem *items,
               const int *block_start, cudaStream_t st) {
  batch_lx_kernel<false, LX><<<nblocks, kBatchThreads, smem, st>>>(meshes, items, block_start);
  return launch_status();
}
template <int LX>
int setup_one(size_t smem, int *bps) {
  auto k = batch_lx_kernel<false, LX>;
  if (smem + kStaticSmemMargin > 48 * 1024 &&
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
    (void)cudaGetLastError();
    return AX_EINVAL;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, kBatchThreads, smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  return AX_OK;
}
}  // namespace

#define AX_BATCH_LX(M) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12)

int batch_lx_launch_f32(int lx, int nblocks, size_t smem, const BatchMeshDev *meshes,
                            const BatchItem *items, const int *block_start, cudaStream_t st) {
  switch (lx) {
#define AX_CASE(L) \
  case L:          \
    return launch_one<L>(nblocks, smem, meshes, items, block_start, st);
    AX_BATCH_LX(AX_CASE)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

int batch_lx_setup_f32(int lx, size_t smem, int *bps) {
  switch (lx) {
#define AX_CASE(L) \
  case L:          \
    return setup_one<L>(smem, bps);
    AX_BATCH_LX(AX_CASE)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

}  // namespace ax
