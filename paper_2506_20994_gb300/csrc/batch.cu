// Batched element operator over many independent meshes of uneven size and
// mixed polynomial order in ONE persistent launch (optionally replayed as a
// CUDA graph), and the autotuner that picks elements per block for each lx.
//
// The paper's kernel (Listing 2) runs one mesh per launch, and Neko chooses
// its kernel variant by timing at run time (Sec. "Methodology"); here a
// host-built plan cuts every mesh into work items of `epb` elements (epb
// tuned per lx), and a static longest-processing-time-first assignment
// gives every persistent block a contiguous list of items of about equal
// cost (cost ~ elements * lx^4).  Blocks walk their own list; there are no
// atomics and no inter-block waits.  Each item runs the same device body
// as the single-mesh kernels (ax_df64.cuh / ax_kstep.cuh).
#include <algorithm>
#include <cstring>
#include <new>
#include <queue>
#include <vector>

#include "ax_df64.cuh"
#include "ax_kstep.cuh"
#include "dispatch.h"

namespace {

struct MeshDev {
  int lx, epb;
  void *w;
  const void *u, *dx, *dxt, *h1, *g[6];
};

struct Item {
  int mesh, nel;
  long long e0;
};

constexpr int kBatchThreads = 256;
constexpr int kBatchLxMin = 2, kBatchLxMax = 12;

#define AX_BATCH_LX(M) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12)

template <bool F64>
__global__ void __launch_bounds__(kBatchThreads)
batch_kernel(const MeshDev *__restrict__ meshes, const Item *__restrict__ items,
             const int *__restrict__ block_start) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b0 = block_start[blockIdx.x], b1 = block_start[blockIdx.x + 1];
  for (int it = b0; it < b1; ++it) {
    const Item itm = items[it];
    const MeshDev m = meshes[itm.mesh];
    switch (m.lx) {
#define AX_BODY(L)                                                                            \
  case L:                                                                                     \
    if (F64)                                                                                  \
      ax::df64_body<L>((double *)m.w, (const double *)m.u, (const double *)m.dx,              \
                       (const double *)m.dxt, (const double *)m.h1, (const double *)m.g[0],   \
                       (const double *)m.g[1], (const double *)m.g[2], (const double *)m.g[3],\
                       (const double *)m.g[4], (const double *)m.g[5], itm.e0, itm.nel,       \
                       m.epb, smem_raw);                                                      \
    else                                                                                      \
      ax::kstep_body<L, float, float, float, float>(                                          \
          (float *)m.w, (const float *)m.u, (const float *)m.dx, (const float *)m.dxt,        \
          (const float *)m.h1, (const float *)m.g[0], (const float *)m.g[1],                  \
          (const float *)m.g[2], (const float *)m.g[3], (const float *)m.g[4],                \
          (const float *)m.g[5], itm.e0, itm.nel, m.epb, smem_raw);                           \
    break;
      AX_BATCH_LX(AX_BODY)
#undef AX_BODY
      default:
        break;
    }
    __syncthreads();  // the next item reuses shared memory
  }
}

size_t body_smem(bool f64, int lx, int epb) {
  const size_t n2 = (size_t)lx * lx, n3 = n2 * lx;
  return (2 * n2 + (size_t)epb * 3 * n3) * (f64 ? 8 : 4);
}

}  // namespace

// process-wide tuned elements-per-block table, [dtype][lx]; 0 = default
static int g_tuned_epb[3][AX_LX_MAX + 1];

namespace ax {
int tuned_epb(int dtype, int lx) {
  if (dtype < 1 || dtype > 2 || lx < 0 || lx > AX_LX_MAX) return 0;
  return g_tuned_epb[dtype][lx];
}
}  // namespace ax

struct ax_batch {
  int dtype = 0;
  int nmesh = 0, nitems = 0, nblocks = 0;
  size_t smem = 0;
  MeshDev *d_mesh = nullptr;
  Item *d_items = nullptr;
  int *d_start = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double flops = 0, bytes = 0;
};

namespace {

int batch_launch_raw(ax_batch *B, cudaStream_t st) {
  if (B->nitems == 0) return AX_OK;
  if (B->dtype == AX_BATCH_F64)
    batch_kernel<true><<<B->nblocks, kBatchThreads, B->smem, st>>>(B->d_mesh, B->d_items,
                                                                   B->d_start);
  else
    batch_kernel<false><<<B->nblocks, kBatchThreads, B->smem, st>>>(B->d_mesh, B->d_items,
                                                                    B->d_start);
  return ax::launch_status();
}

int default_epb(int lx) { return std::max(1, kBatchThreads / (lx * lx)); }

}  // namespace

extern "C" {

int ax_batch_destroy(ax_batch *B) {
  if (!B) return AX_OK;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  cudaFree(B->d_mesh);
  cudaFree(B->d_items);
  cudaFree(B->d_start);
  delete B;
  return AX_OK;
}

int ax_batch_create(ax_batch **out, int dtype, int nmesh, const ax_batch_mesh *meshes,
                    int blocks_per_sm, void *stream) {
  if (!out || (dtype != AX_BATCH_F64 && dtype != AX_BATCH_F32) || nmesh < 0 ||
      (nmesh > 0 && !meshes))
    return AX_EINVAL;
  *out = nullptr;
  const bool f64 = dtype == AX_BATCH_F64;
  std::vector<MeshDev> mh(nmesh);
  std::vector<Item> items;
  std::vector<double> cost;
  size_t smem = 0;
  double flops = 0, bytes = 0;
  for (int m = 0; m < nmesh; ++m) {
    const ax_batch_mesh &s = meshes[m];
    if (s.lx < kBatchLxMin || s.lx > kBatchLxMax || s.nelv < 0) return AX_EINVAL;
    if (s.nelv > 0 && !ax::all_nonnull(s.w, s.u, s.dx, s.dxt, s.h1, s.g11, s.g22, s.g33, s.g12,
                                       s.g13, s.g23))
      return AX_EINVAL;
    int epb = ax::tuned_epb(dtype, s.lx);
    if (epb <= 0) epb = default_epb(s.lx);
    epb = std::min(epb, kBatchThreads / (s.lx * s.lx));
    mh[m] = MeshDev{s.lx, epb, s.w, s.u, s.dx, s.dxt, s.h1,
                    {s.g11, s.g22, s.g33, s.g12, s.g13, s.g23}};
    smem = std::max(smem, body_smem(f64, s.lx, epb));
    const double l = s.lx, l3 = l * l * l;
    for (long long e = 0; e < s.nelv; e += epb) {
      const int nel = (int)std::min<long long>(epb, s.nelv - e);
      items.push_back(Item{m, nel, e});
      cost.push_back(nel * (l3 * l + 2.0 * l3));
    }
    flops += (double)s.nelv * (12.0 * l3 * l + 18.0 * l3);
    bytes += (double)s.nelv * 9.0 * l3 * (f64 ? 8 : 4);
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (blocks_per_sm <= 0) blocks_per_sm = f64 ? 2 : 4;
  int nblocks = std::max(1, std::min<int>(nsm * blocks_per_sm, (int)items.size()));
  // longest processing time first onto the least-loaded block
  std::vector<int> order(items.size());
  for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  using Load = std::pair<double, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int b = 0; b < nblocks; ++b) heap.push({0.0, b});
  std::vector<std::vector<int>> per(nblocks);
  for (int q : order) {
    Load l = heap.top();
    heap.pop();
    per[l.second].push_back(q);
    heap.push({l.first + cost[q], l.second});
  }
  std::vector<Item> flat;
  flat.reserve(items.size());
  std::vector<int> start(nblocks + 1, 0);
  for (int b = 0; b < nblocks; ++b) {
    std::sort(per[b].begin(), per[b].end());  // memory order inside a block
    for (int q : per[b]) flat.push_back(items[q]);
    start[b + 1] = (int)flat.size();
  }
  ax_batch *B = new (std::nothrow) ax_batch();
  if (!B) return AX_ENOMEM;
  B->dtype = dtype;
  B->nmesh = nmesh;
  B->nitems = (int)flat.size();
  B->nblocks = nblocks;
  B->smem = smem;
  B->flops = flops;
  B->bytes = bytes;
  cudaStream_t st = (cudaStream_t)stream;
  bool ok = cudaMalloc(&B->d_mesh, std::max<size_t>(1, mh.size()) * sizeof(MeshDev)) ==
                cudaSuccess &&
            cudaMalloc(&B->d_items, std::max<size_t>(1, flat.size()) * sizeof(Item)) ==
                cudaSuccess &&
            cudaMalloc(&B->d_start, start.size() * sizeof(int)) == cudaSuccess;
  if (ok && !mh.empty())
    ok = cudaMemcpyAsync(B->d_mesh, mh.data(), mh.size() * sizeof(MeshDev),
                         cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (ok && !flat.empty())
    ok = cudaMemcpyAsync(B->d_items, flat.data(), flat.size() * sizeof(Item),
                         cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (ok)
    ok = cudaMemcpyAsync(B->d_start, start.data(), start.size() * sizeof(int),
                         cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaStreamSynchronize(st) == cudaSuccess;
  if (ok && smem > 48 * 1024) {
    ok = cudaFuncSetAttribute(f64 ? batch_kernel<true> : batch_kernel<false>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem) == cudaSuccess;
  }
  if (!ok) {
    (void)cudaGetLastError();
    ax_batch_destroy(B);
    return AX_ENOMEM;
  }
  *out = B;
  return AX_OK;
}

int ax_batch_launch(ax_batch *B, void *stream) {
  if (!B) return AX_EINVAL;
  return batch_launch_raw(B, (cudaStream_t)stream);
}

int ax_batch_graph_launch(ax_batch *B, void *stream) {
  if (!B) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!B->exec) {
    // capture on a private stream so the caller's stream may be the legacy one
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return AX_ELAUNCH;
    int rc = AX_OK;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = AX_ELAUNCH;
    if (rc == AX_OK) rc = batch_launch_raw(B, cap);
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(cap, &g) != cudaSuccess) rc = AX_ELAUNCH;
    cudaStreamDestroy(cap);
    if (rc == AX_OK && cudaGraphInstantiate(&B->exec, g, 0) != cudaSuccess) rc = AX_ELAUNCH;
    if (rc != AX_OK) {
      (void)cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      B->exec = nullptr;
      return rc;
    }
    B->graph = g;
  }
  if (cudaGraphLaunch(B->exec, st) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  return AX_OK;
}

int ax_batch_info(const ax_batch *B, int *nitems, int *nblocks, int64_t *smem_bytes,
                  double *flops, double *bytes) {
  if (!B) return AX_EINVAL;
  if (nitems) *nitems = B->nitems;
  if (nblocks) *nblocks = B->nblocks;
  if (smem_bytes) *smem_bytes = (int64_t)B->smem;
  if (flops) *flops = B->flops;
  if (bytes) *bytes = B->bytes;
  return AX_OK;
}

int ax_tune_set(int dtype, int lx, int elems_per_block) {
  if ((dtype != AX_BATCH_F64 && dtype != AX_BATCH_F32) || !ax::lx_ok(lx) ||
      elems_per_block < 0 || elems_per_block * lx * lx > 256)
    return AX_EINVAL;
  g_tuned_epb[dtype][lx] = elems_per_block;
  return AX_OK;
}

int ax_tune_get(int dtype, int lx, int *elems_per_block) {
  if ((dtype != AX_BATCH_F64 && dtype != AX_BATCH_F32) || !ax::lx_ok(lx) || !elems_per_block)
    return AX_EINVAL;
  *elems_per_block = g_tuned_epb[dtype][lx];
  return AX_OK;
}

// Times every admissible elements-per-block value for (dtype, lx) on the
// caller's buffers (nelv elements; w is overwritten) and records the best.
int ax_tune_run(int dtype, int lx, int nelv, void *w, const void *u, const void *dx,
                const void *dxt, const void *h1, const void *g11, const void *g22,
                const void *g33, const void *g12, const void *g13, const void *g23, int reps,
                int *best_epb, float *best_ms, void *stream) {
  if ((dtype != AX_BATCH_F64 && dtype != AX_BATCH_F32) || !ax::lx_ok(lx) || nelv <= 0 ||
      reps < 1 || !ax::all_nonnull(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23))
    return AX_EINVAL;
  if (dtype == AX_BATCH_F64 && lx > ax::AX_DF64_LX_MAX) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return AX_ELAUNCH;
  const int emax = std::max(1, 256 / (lx * lx));
  int best = 0;
  float best_t = 1e30f;
  for (int epb = 1; epb <= emax; ++epb) {
    auto run = [&]() {
      if (dtype == AX_BATCH_F64)
        return ax::dispatch_df64(lx, (double *)w, (const double *)u, (const double *)dx,
                                 (const double *)dxt, (const double *)h1, (const double *)g11,
                                 (const double *)g22, (const double *)g33, (const double *)g12,
                                 (const double *)g13, (const double *)g23, nelv, epb, st);
      return ax::dispatch_kstep_f32(lx, (float *)w, (const float *)u, (const float *)dx,
                                    (const float *)dxt, (const float *)h1, (const float *)g11,
                                    (const float *)g22, (const float *)g33, (const float *)g12,
                                    (const float *)g13, (const float *)g23, nelv, epb, st);
    };
    if (run() != AX_OK) continue;  // warm-up (also rejects inadmissible shapes)
    cudaEventRecord(e0, st);
    int rc = AX_OK;
    for (int r = 0; r < reps && rc == AX_OK; ++r) rc = run();
    cudaEventRecord(e1, st);
    if (rc != AX_OK || cudaEventSynchronize(e1) != cudaSuccess) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (ms < best_t) {
      best_t = ms;
      best = epb;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best == 0) return AX_ELAUNCH;
  g_tuned_epb[dtype][lx] = best;
  if (best_epb) *best_epb = best;
  if (best_ms) *best_ms = best_t;
  return AX_OK;
}

}  // extern "C"
