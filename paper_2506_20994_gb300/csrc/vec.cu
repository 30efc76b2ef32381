// Vector kernels of the partitioned solve: weighted dot products and the
// pack / unpack of the values at nodes shared with another partition.
#include <algorithm>

#include "reduce.cuh"

namespace {

__global__ void wdot_kernel(const double *__restrict__ a, const double *__restrict__ b,
                            const double *__restrict__ wgt, double *__restrict__ partials,
                            int64_t n) {
  __shared__ double sh[ax::kRedThreads / 32];
  double s = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    s += wgt[q] * a[q] * b[q];
  double v[1] = {s};
  ax::block_sum<1>(v, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

__global__ void wdot_final_kernel(const double *__restrict__ partials, int nblk,
                                  double *__restrict__ out) {
  ax::warp_sum_partials<1>(partials, nblk, out);
}

__global__ void gather_kernel(double *__restrict__ out, const double *__restrict__ v,
                              const int64_t *__restrict__ idx, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = v[idx[q]];
}

__global__ void scatter_add_kernel(double *__restrict__ v, const double *__restrict__ vals,
                                   const int64_t *__restrict__ idx,
                                   const int64_t *__restrict__ pos, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    v[idx[q]] += vals[pos[q]];
}

unsigned grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, ax::kRedBlocks));
}

}  // namespace

extern "C" int ax_dot_weighted(const double *a, const double *b, const double *wgt, int64_t n,
                               double *work, double *out, void *stream) {
  if (n < 0 || !out || !work || (n > 0 && !ax::all_nonnull(a, b, wgt))) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  wdot_kernel<<<ax::kRedBlocks, ax::kRedThreads, 0, st>>>(a, b, wgt, work, n);
  wdot_final_kernel<<<1, 32, 0, st>>>(work, ax::kRedBlocks, out);
  return ax::launch_status();
}

extern "C" int ax_gather(double *out, const double *v, const int64_t *idx, int64_t n,
                         void *stream) {
  if (n < 0) return AX_EINVAL;
  if (n == 0) return AX_OK;
  if (!ax::all_nonnull(out, v, idx)) return AX_EINVAL;
  gather_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(out, v, idx, n);
  return ax::launch_status();
}

extern "C" int ax_scatter_add(double *v, const double *vals, const int64_t *idx,
                              const int64_t *pos, int64_t n, void *stream) {
  if (n < 0) return AX_EINVAL;
  if (n == 0) return AX_OK;
  if (!ax::all_nonnull(v, vals, idx, pos)) return AX_EINVAL;
  scatter_add_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(v, vals, idx, pos, n);
  return ax::launch_status();
}
