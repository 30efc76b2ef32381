// Batched element operator over many independent meshes of uneven size and
// mixed polynomial order, launched as one persistent kernel per polynomial
// order present (all recorded into one CUDA graph on first replay), and the
// autotuner that picks elements per block for each lx.
//
// The paper's kernel (Listing 2) runs one mesh per launch, and Neko chooses
// its kernel variant by timing at run time (Sec. "Methodology"); here a
// host-built plan cuts every mesh into work items of `epb` elements (epb
// tuned per lx), groups the items by lx, and assigns each group's items
// longest-processing-time-first (cost ~ elements * lx^4) to a fixed set of
// persistent blocks sized by the occupancy of that group's kernel.  Blocks
// walk their own contiguous item list; there are no atomics and no
// inter-block waits.  Each item runs the same device body as the
// single-mesh kernel (ax_df64.cuh / ax_df64_eo.cuh / ax_kstep.cuh), so the
// results are bit-identical to ax_helm / ax_helm_f32, or, for fp64 meshes
// with lx in {8, 10, 12}, to the operator handle (geometry prepared here).  One kernel per lx
// (rather than one kernel switching over lx) keeps each kernel's register
// footprint, and so its occupancy, that of its single-mesh counterpart.
#include <algorithm>
#include <cstring>
#include <new>
#include <queue>
#include <vector>

#include "batch_kernels.cuh"
#include "dispatch.h"

namespace ax {
int batch_lx_launch_f64(int, int, int, size_t, const BatchMeshDev *, const BatchItem *,
                        const int *, cudaStream_t);
int batch_lx_launch_f32(int, int, size_t, const BatchMeshDev *, const BatchItem *, const int *,
                        cudaStream_t);
int batch_lx_setup_f64(int, int, size_t, int *);
int batch_lx_setup_f32(int, size_t, int *);
int batch_lx_launch(bool f64, int lx, int body, int nblocks, size_t smem, const BatchMeshDev *m,
                    const BatchItem *it, const int *bs, cudaStream_t st) {
  return f64 ? batch_lx_launch_f64(lx, body, nblocks, smem, m, it, bs, st)
             : batch_lx_launch_f32(lx, nblocks, smem, m, it, bs, st);
}
int batch_lx_setup(bool f64, int lx, int body, size_t smem, int *bps) {
  return f64 ? batch_lx_setup_f64(lx, body, smem, bps) : batch_lx_setup_f32(lx, smem, bps);
}
}  // namespace ax

namespace {

using ax::BatchItem;
using ax::BatchMeshDev;
using ax::kBatchThreads;
constexpr int kBatchLxMin = 2, kBatchLxMax = 12;

size_t body_smem(bool f64, int lx, int body, int epb) {
  const size_t n2 = (size_t)lx * lx, n3 = n2 * lx;
  if (f64 && body == ax::kBodyEvenOdd) {
    const size_t h = lx / 2;
    return 2 * h * h * 24 + (size_t)epb * 3 * n2 * (h + 1) * 16;
  }
  return (2 * n2 + (size_t)epb * 3 * n3) * (f64 ? 8 : 4);
}

int default_epb(int lx) { return std::max(1, kBatchThreads / (lx * lx)); }

// Thread layout of the fp64 kernel for lx: the variant the tuner recorded
// (ax_tune_variant_run; either k-loop variant runs the double-float k-loop
// body here), else ax_helm's built-in choice.
int choose_body(int lx) {
  int v = 0;
  if (ax_tune_variant_get(lx, &v) != AX_OK) v = 0;
  if (v == AX_VARIANT_F64_DF_EO && ax::batch_eo_ok(lx)) return ax::kBodyEvenOdd;
  if (v == AX_VARIANT_F64_DF || v == AX_VARIANT_F64_NATIVE) return ax::kBodyKLoop;
  return ax::batch_uses_eo(lx) ? ax::kBodyEvenOdd : ax::kBodyKLoop;
}

struct Group {
  int lx = 0, body = 0, nblocks = 0;
  size_t smem = 0;
  int item_off = 0, start_off = 0;  // into d_items / d_start
};

}  // namespace

// process-wide tuned elements-per-block table, [dtype][lx]; 0 = default
static std::atomic<int> g_tuned_epb[3][AX_LX_MAX + 1];  // written by the tuner

namespace ax {
int tuned_epb(int dtype, int lx) {
  if (dtype < 1 || dtype > 2 || lx < 0 || lx > AX_LX_MAX) return 0;
  return g_tuned_epb[dtype][lx].load(std::memory_order_relaxed);
}
}  // namespace ax

struct ax_batch {
  int dtype = 0;
  int nmesh = 0, nitems = 0, nblocks = 0;
  size_t smem = 0;
  std::vector<Group> groups;
  BatchMeshDev *d_mesh = nullptr;
  std::vector<void *> prepared;  // owned prepared geometry of even-odd fp64 meshes
  BatchItem *d_items = nullptr;
  int *d_start = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double flops = 0, bytes = 0;
};

namespace {

int batch_launch_raw(ax_batch *B, cudaStream_t st) {
  const bool f64 = B->dtype == AX_BATCH_F64;
  for (const Group &g : B->groups) {
    int rc = ax::batch_lx_launch(f64, g.lx, g.body, g.nblocks, g.smem, B->d_mesh,
                                 B->d_items + g.item_off, B->d_start + g.start_off, st);
    if (rc) return rc;
  }
  return AX_OK;
}

}  // namespace

extern "C" {

int ax_batch_destroy(ax_batch *B) {
  if (!B) return AX_OK;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  cudaFree(B->d_mesh);
  cudaFree(B->d_items);
  cudaFree(B->d_start);
  for (void *q : B->prepared) cudaFree(q);
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
  std::vector<BatchMeshDev> mh(nmesh);
  std::vector<int> mbody(nmesh, ax::kBodyKLoop);
  // per (lx, layout): key = 2 lx + layout
  const int nkey = 2 * (kBatchLxMax + 1);
  std::vector<std::vector<BatchItem>> items(nkey);
  std::vector<std::vector<double>> cost(nkey);
  std::vector<size_t> smem(nkey, 0);
  double flops = 0, bytes = 0;
  for (int m = 0; m < nmesh; ++m) {
    const ax_batch_mesh &s = meshes[m];
    if (s.lx < kBatchLxMin || s.lx > kBatchLxMax || s.nelv < 0) return AX_EINVAL;
    if (s.nelv > 0 && !ax::all_nonnull(s.w, s.u, s.dx, s.dxt, s.h1, s.g11, s.g22, s.g33, s.g12,
                                       s.g13, s.g23))
      return AX_EINVAL;
    int epb;
    const int body = f64 ? choose_body(s.lx) : ax::kBodyKLoop;
    mbody[m] = body;
    const int key = 2 * s.lx + body;
    if (body == ax::kBodyEvenOdd) {
      // even-odd body: (lx/2)^3 threads per element
      const int h = s.lx / 2;
      epb = std::max(1, kBatchThreads / (h * h * h));
    } else {
      epb = ax::tuned_epb(dtype, s.lx);
      if (epb <= 0) epb = default_epb(s.lx);
      epb = std::min(epb, kBatchThreads / (s.lx * s.lx));
    }
    mh[m] = BatchMeshDev{s.lx, epb, s.w, s.u, s.dx, s.dxt, s.h1,
                         {s.g11, s.g22, s.g33, s.g12, s.g13, s.g23}, nullptr};
    smem[key] = std::max(smem[key], body_smem(f64, s.lx, body, epb));
    const double l = s.lx, l3 = l * l * l;
    for (long long e = 0; e < s.nelv; e += epb) {
      const int nel = (int)std::min<long long>(epb, s.nelv - e);
      items[key].push_back(BatchItem{m, nel, e});
      cost[key].push_back(nel * (l3 * l + 2.0 * l3));
    }
    flops += (double)s.nelv * (12.0 * l3 * l + 18.0 * l3);
    bytes += (double)s.nelv * 9.0 * l3 * (f64 ? 8 : 4);
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  std::vector<Group> groups;
  std::vector<BatchItem> flat;
  std::vector<int> start;
  size_t smem_max = 0;
  for (int key = 2 * kBatchLxMin; key < nkey; ++key) {
    if (items[key].empty()) continue;
    const int lx = key / 2, body = key % 2;
    int bps = 0;
    int rc = ax::batch_lx_setup(f64, lx, body, smem[key], &bps);
    if (rc) return rc;
    if (bps < 1) return AX_EINVAL;
    if (blocks_per_sm > 0) bps = std::min(bps, blocks_per_sm);
    const int nb = std::max(1, std::min<int>(nsm * bps, (int)items[key].size()));
    // longest processing time first onto the least-loaded block
    std::vector<int> order(items[key].size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return cost[key][a] > cost[key][b]; });
    using Load = std::pair<double, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int b = 0; b < nb; ++b) heap.push({0.0, b});
    std::vector<std::vector<int>> per(nb);
    for (int q : order) {
      Load ld = heap.top();
      heap.pop();
      per[ld.second].push_back(q);
      heap.push({ld.first + cost[key][q], ld.second});
    }
    Group g;
    g.lx = lx;
    g.body = body;
    g.nblocks = nb;
    g.smem = smem[key];
    g.item_off = (int)flat.size();
    g.start_off = (int)start.size();
    int cnt = 0;
    for (int b = 0; b < nb; ++b) {
      std::sort(per[b].begin(), per[b].end());  // memory order inside a block
      start.push_back(cnt);
      for (int q : per[b]) flat.push_back(items[key][q]), ++cnt;
    }
    start.push_back(cnt);
    groups.push_back(g);
    smem_max = std::max(smem_max, g.smem);
  }
  ax_batch *B = new (std::nothrow) ax_batch();
  if (!B) return AX_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  // fp64 meshes of the even-odd orders: prepare their geometry once
  for (int m = 0; f64 && m < nmesh; ++m) {
    const ax_batch_mesh &s = meshes[m];
    if (mbody[m] != ax::kBodyEvenOdd || s.nelv == 0) continue;
    void *gp = nullptr;
    if (cudaMalloc(&gp, ax::eo_prep_bytes(s.lx, s.nelv)) != cudaSuccess) {
      (void)cudaGetLastError();
      ax_batch_destroy(B);
      return AX_ENOMEM;
    }
    B->prepared.push_back(gp);
    auto d = [](const void *q) { return static_cast<const double *>(q); };
    int rc = ax::dispatch_eo_prepare(s.lx, static_cast<ax::df::dd2 *>(gp), d(s.h1), d(s.g11),
                                     d(s.g22), d(s.g33), d(s.g12), d(s.g13), d(s.g23), s.nelv,
                                     0x7F, st);
    if (rc) {
      ax_batch_destroy(B);
      return rc;
    }
    mh[m].gp = static_cast<const ax::df::dd2 *>(gp);
    mh[m].gstat = reinterpret_cast<const unsigned *>(static_cast<const char *>(gp) +
                                                     (size_t)s.nelv * 56 * s.lx * s.lx * s.lx);
  }
  B->dtype = dtype;
  B->nmesh = nmesh;
  B->nitems = (int)flat.size();
  B->groups = groups;
  for (const Group &g : groups) B->nblocks += g.nblocks;
  B->smem = smem_max;
  B->flops = flops;
  B->bytes = bytes;
  bool ok = cudaMalloc(&B->d_mesh, std::max<size_t>(1, mh.size()) * sizeof(BatchMeshDev)) ==
                cudaSuccess &&
            cudaMalloc(&B->d_items, std::max<size_t>(1, flat.size()) * sizeof(BatchItem)) ==
                cudaSuccess &&
            cudaMalloc(&B->d_start, std::max<size_t>(1, start.size()) * sizeof(int)) ==
                cudaSuccess;
  if (ok && !mh.empty())
    ok = cudaMemcpyAsync(B->d_mesh, mh.data(), mh.size() * sizeof(BatchMeshDev),
                         cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (ok && !flat.empty())
    ok = cudaMemcpyAsync(B->d_items, flat.data(), flat.size() * sizeof(BatchItem),
                         cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (ok && !start.empty())
    ok = cudaMemcpyAsync(B->d_start, start.data(), start.size() * sizeof(int),
                         cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (ok) ok = cudaStreamSynchronize(st) == cudaSuccess;
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
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      rc = AX_ELAUNCH;
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
  g_tuned_epb[dtype][lx].store(elems_per_block, std::memory_order_relaxed);
  return AX_OK;
}

int ax_tune_get(int dtype, int lx, int *elems_per_block) {
  if ((dtype != AX_BATCH_F64 && dtype != AX_BATCH_F32) || !ax::lx_ok(lx) || !elems_per_block)
    return AX_EINVAL;
  *elems_per_block = g_tuned_epb[dtype][lx].load(std::memory_order_relaxed);
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
  g_tuned_epb[dtype][lx].store(best, std::memory_order_relaxed);
  if (best_epb) *best_epb = best;
  if (best_ms) *best_ms = best_t;
  return AX_OK;
}

}  // extern "C"
