// Persistent batched kernels for the f64 dtype, one per lx in [2, 12].
#include "batch_kernels.cuh"

namespace ax {

namespace {
template <int LX, int BODY>
int launch_one(int nblocks, size_t smem, const BatchMeshDev *meshes, const BatchItem *items,
               const int *block_start, cudaStream_t st) {
  batch_lx_kernel<true, LX, BODY><<<nblocks, kBatchThreads, smem, st>>>(meshes, items,
                                                                        block_start);
  return launch_status();
}
template <int LX, int BODY>
int setup_one(size_t smem, int *bps) {
  auto k = batch_lx_kernel<true, LX, BODY>;
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
#define AX_BATCH_EO(M) M(4) M(6) M(8) M(10) M(12)

int batch_lx_launch_f64(int lx, int body, int nblocks, size_t smem, const BatchMeshDev *meshes,
                        const BatchItem *items, const int *block_start, cudaStream_t st) {
  switch (lx * 2 + (body == kBodyEvenOdd)) {
#define AX_CASE(L)                                                                   \
  case 2 * L:                                                                        \
    return launch_one<L, kBodyKLoop>(nblocks, smem, meshes, items, block_start, st);
    AX_BATCH_LX(AX_CASE)
#undef AX_CASE
#define AX_CASE(L)                                                                     \
  case 2 * L + 1:                                                                      \
    return launch_one<L, kBodyEvenOdd>(nblocks, smem, meshes, items, block_start, st);
    AX_BATCH_EO(AX_CASE)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

int batch_lx_setup_f64(int lx, int body, size_t smem, int *bps) {
  switch (lx * 2 + (body == kBodyEvenOdd)) {
#define AX_CASE(L) \
  case 2 * L:      \
    return setup_one<L, kBodyKLoop>(smem, bps);
    AX_BATCH_LX(AX_CASE)
#undef AX_CASE
#define AX_CASE(L) \
  case 2 * L + 1:  \
    return setup_one<L, kBodyEvenOdd>(smem, bps);
    AX_BATCH_EO(AX_CASE)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

}  // namespace ax
