// Vector kernels of the partitioned solve: weighted dot products and the
// pack / unpack of the values at nodes shared with another partition.
#include <algorithm>

#include "op.h"
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

// w += hb .* u; partials (optional, kRedBlocks of them): sum u . hb . u
template <typename T>
__global__ void mass_add_kernel(T *__restrict__ w, const T *__restrict__ hb,
                                const T *__restrict__ u, int64_t n,
                                double *__restrict__ partials) {
  __shared__ double sh[ax::kRedThreads / 32];
  T acc = T(0);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const T m = hb[q] * u[q];
    w[q] += m;
    acc += m * u[q];
  }
  if (partials) {  // kernel-uniform
    double v[1] = {(double)acc};
    ax::block_sum<1>(v, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
  }
}

// w += (h2 .* B) .* u
__global__ void mass_add2_kernel(double *__restrict__ w, const double *__restrict__ h2,
                                 const double *__restrict__ B, const double *__restrict__ u,
                                 int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    w[q] += (h2[q] * B[q]) * u[q];
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

namespace ax {

template <typename T>
int mass_add(T *w, const T *hb, const T *u, int64_t n, double *partials, cudaStream_t st) {
  if (n < 0) return AX_EINVAL;
  if (n > 0 && !all_nonnull(w, hb, u)) return AX_EINVAL;
  mass_add_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>(w, hb, u, n, partials);
  return launch_status();
}
template int mass_add<double>(double *, const double *, const double *, int64_t, double *,
                              cudaStream_t);
template int mass_add<float>(float *, const float *, const float *, int64_t, double *,
                             cudaStream_t);

int mass_add2(double *w, const double *h2, const double *B, const double *u, int64_t n,
              cudaStream_t st) {
  if (n < 0) return AX_EINVAL;
  if (n > 0 && !all_nonnull(w, h2, B, u)) return AX_EINVAL;
  mass_add2_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(w, h2, B, u, n);
  return launch_status();
}

}  // namespace ax

extern "C" int ax_mass_add(double *w, const double *hb, const double *u, int64_t n,
                           void *stream) {
  return ax::mass_add<double>(w, hb, u, n, nullptr, (cudaStream_t)stream);
}

extern "C" int ax_mass_add_f32(float *w, const float *hb, const float *u, int64_t n,
                               void *stream) {
  return ax::mass_add<float>(w, hb, u, n, nullptr, (cudaStream_t)stream);
}
