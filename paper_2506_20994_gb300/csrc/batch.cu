// Batched element operator over many independent meshes of uneven size and
// mixed polynomial order in one persistent launch (optionally replayed from a
// CUDA graph), and the autotuner tables the single-mesh kernels use.
//
// The paper's kernel (Listing 2) runs one mesh per launch, and Neko chooses
// its kernel variant by timing at run time (Sec. "Methodology").  Here a
// host-built plan cuts every mesh into work items, balances them over the
// persistent CTAs of one kernel per dtype (longest processing time first,
// cost ~ elements * lx^3 * measured time per point), and gives each CTA its
// items sorted into groups of
// one lx and thread layout (batch_kernels.cuh).  The layout of an fp64 mesh
// is the variant table's (ax_tune_variant_*): the persistent even-odd body
// for lx in {6, 8, 10} unless the table asks for the k-loop layout or the
// mesh's matrices are not centro-antisymmetric, the double-float k-loop body
// otherwise.  Each body is the single-mesh one, so results equal the
// operator handle's (even-odd meshes) or ax_helm's / ax_helm_f32's bit for
// bit.  No atomics and no waits between CTAs.
#include <algorithm>
#include <cstring>
#include <new>
#include <queue>
#include <vector>

#include "batch_kernels.cuh"
#include "dispatch.h"

namespace {

using ax::BatchGroup;
using ax::BatchItem;
using ax::BatchMeshDev;
using ax::kBatchThreads;
constexpr int kBatchLxMin = 2, kBatchLxMax = 12;

// Layout of an fp64 mesh of order lx from the variant table (before the
// symmetry check of its matrices).
int choose_body(int lx) {
  int v = 0;
  if (ax_tune_variant_get(lx, &v) != AX_OK) v = 0;
  if (v == AX_VARIANT_F64_DF || v == AX_VARIANT_F64_NATIVE) return ax::kBodyKLoop;
  return ax::batch_eo_ok(lx) ? ax::kBodyEvenOdd : ax::kBodyKLoop;
}

// Cost of one element in a batch CTA for balancing: lx^3 times the time per
// point of its body, in ns (measured on GB300 on the uneven benchmark batch,
// one order at a time; other orders take the nearest body's rate).  A model
// proportional to the flops (lx^4) balanced the mixed batch 14 % worse: the
// even-odd body is most efficient per point at lx = 8.
double elem_cost(int lx, bool f64, bool eo) {
  double ns;
  if (f64 && eo)
    ns = lx == 6 ? 7.4 : lx == 8 ? 7.2 : 8.6;
  else if (eo)  // fp32 even-odd body: single-mesh rates scaled to the batch CTA
    ns = lx <= 6 ? 3.9 : lx == 8 ? 3.0 : 4.2;
  else if (f64)
    ns = 13.0;
  else
    ns = lx <= 5 ? 5.5 : lx == 6 ? 4.7 : lx <= 9 ? 3.8 : 5.4;
  return (double)lx * lx * lx * ns;
}

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
  int nmesh = 0, nitems = 0, nblocks = 0, ngroups = 0;
  size_t smem = 0;
  BatchMeshDev *d_mesh = nullptr;
  ax::eop::EopMesh *d_emesh = nullptr;
  ax::F32Mesh *d_fmesh = nullptr;
  BatchItem *d_items = nullptr;
  BatchGroup *d_groups = nullptr;
  int *d_start = nullptr;
  int *d_err = nullptr;
  std::vector<void *> owned;  // prepared geometry and coefficients of even-odd meshes
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double flops = 0, bytes = 0;
};

namespace {

int batch_launch_raw(ax_batch *B, cudaStream_t st) {
  if (B->nblocks == 0) return AX_OK;
  if (B->dtype == AX_BATCH_F64)
    return ax::batch_launch_f64(B->nblocks, B->smem, B->d_mesh, B->d_emesh, B->d_items,
                                B->d_groups, B->d_start, B->d_err, st);
  return ax::batch_launch_f32(B->nblocks, B->smem, B->d_mesh, B->d_fmesh, B->d_items,
                              B->d_groups, B->d_start, B->d_err, st);
}

template <typename T>
bool upload(T **dst, const std::vector<T> &src, cudaStream_t st) {
  if (cudaMalloc((void **)dst, std::max<size_t>(1, src.size()) * sizeof(T)) != cudaSuccess)
    return false;
  return src.empty() || cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T),
                                        cudaMemcpyHostToDevice, st) == cudaSuccess;
}

}  // namespace

extern "C" {

int ax_batch_destroy(ax_batch *B) {
  if (!B) return AX_OK;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  cudaFree(B->d_mesh);
  cudaFree(B->d_emesh);
  cudaFree(B->d_fmesh);
  cudaFree(B->d_items);
  cudaFree(B->d_groups);
  cudaFree(B->d_start);
  cudaFree(B->d_err);
  for (void *q : B->owned) cudaFree(q);
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
  for (int m = 0; m < nmesh; ++m) {
    const ax_batch_mesh &s = meshes[m];
    if (s.lx < kBatchLxMin || s.lx > kBatchLxMax || s.nelv < 0) return AX_EINVAL;
    if (s.nelv > 0 && !ax::all_nonnull(s.w, s.u, s.dx, s.dxt, s.h1, s.g11, s.g22, s.g33, s.g12,
                                       s.g13, s.g23))
      return AX_EINVAL;
  }
  ax_batch *B = new (std::nothrow) ax_batch();
  if (!B) return AX_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  auto fail = [&](int rc) {
    (void)cudaGetLastError();
    ax_batch_destroy(B);
    return rc;
  };
  std::vector<BatchMeshDev> mh(nmesh);
  std::vector<ax::eop::EopMesh> em(nmesh);
  std::vector<ax::F32Mesh> fm(nmesh);
  std::vector<int> mbody(nmesh, ax::kBodyKLoop);
  double flops = 0, bytes = 0, total_cost = 0;
  for (int m = 0; m < nmesh; ++m) {
    const ax_batch_mesh &s = meshes[m];
    mh[m] = BatchMeshDev{s.lx, s.w, s.u, s.dx, s.dxt, s.h1,
                         {s.g11, s.g22, s.g33, s.g12, s.g13, s.g23}};
    em[m] = ax::eop::EopMesh{};
    const double l3 = (double)s.lx * s.lx * s.lx;
    flops += (double)s.nelv * (12.0 * l3 * s.lx + 18.0 * l3);
    bytes += (double)s.nelv * 9.0 * l3 * (f64 ? 8 : 4);
    if (!f64) {
      // fp32: the even-odd body exactly where ax_helm_f32 takes it
      auto fl = [](const void *q) { return static_cast<const float *>(q); };
      if (s.nelv > 0 && ax::batch_e32_ok(s.lx) &&
          ax::eo32_ok(s.lx, s.w, s.u, s.h1, s.g11, s.g22, s.g33, s.g12, s.g13, s.g23)) {
        ax::F32Mesh &f = fm[m];
        f.w = static_cast<float *>(s.w);
        f.u = fl(s.u);
        const void *g[7] = {s.h1, s.g11, s.g22, s.g33, s.g12, s.g13, s.g23};
        for (int q = 0; q < 7; ++q) f.g[q] = fl(g[q]);
        f.dx = fl(s.dx);
        f.dxt = fl(s.dxt);
        mbody[m] = ax::kBodyEvenOdd;
      }
      continue;
    }
    if (s.nelv == 0 || choose_body(s.lx) != ax::kBodyEvenOdd) continue;
    // even-odd layout: the matrices must be centro-antisymmetric; geometry and
    // coefficients are prepared here, once, as the operator handle does
    const int lx = s.lx;
    std::vector<double> dh((size_t)lx * lx), dth((size_t)lx * lx);
    std::vector<unsigned char> cb(ax::eop_coef_bytes(lx));
    if (cudaMemcpyAsync(dh.data(), s.dx, dh.size() * 8, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(dth.data(), s.dxt, dth.size() * 8, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(AX_ELAUNCH);
    int dfield = 0;
    if (!ax::eop_coefficients(lx, dh.data(), dth.data(), cb.data(), &dfield)) continue;
    void *gp = nullptr, *cf = nullptr;
    if (cudaMalloc(&gp, ax::eo_prep_bytes(lx, s.nelv)) != cudaSuccess) return fail(AX_ENOMEM);
    B->owned.push_back(gp);
    if (cudaMalloc(&cf, cb.size()) != cudaSuccess) return fail(AX_ENOMEM);
    B->owned.push_back(cf);
    if (cudaMemcpyAsync(cf, cb.data(), cb.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail(AX_ELAUNCH);
    auto d = [](const void *q) { return static_cast<const double *>(q); };
    const ax::guard::RawGeo raw{d(s.h1), d(s.g11), d(s.g22), d(s.g33), d(s.g12), d(s.g13),
                                d(s.g23)};
    int rc = ax::eop_prepare(lx, static_cast<ax::df::dd2 *>(gp), raw, s.nelv, 0x7F, dfield, st);
    if (rc) return fail(rc);
    ax::eop::EopMesh &e = em[m];
    e.w = static_cast<double *>(s.w);
    e.u = d(s.u);
    e.coef = static_cast<const ax::df::dd2 *>(cf);
    e.gp = static_cast<const ax::df::dd2 *>(gp);
    e.urange = reinterpret_cast<const uint2 *>(static_cast<const char *>(gp) +
                                               (size_t)s.nelv * 56 * lx * lx * lx);
    e.raw = raw;
    e.dx = d(s.dx);
    e.dxt = d(s.dxt);
    mbody[m] = ax::kBodyEvenOdd;
  }
  for (int m = 0; m < nmesh; ++m)
    total_cost += meshes[m].nelv * elem_cost(meshes[m].lx, f64, mbody[m] == ax::kBodyEvenOdd);
  // shared memory of the kernel: the largest group layout present
  size_t smem = 0;
  for (int m = 0; m < nmesh; ++m) {
    if (meshes[m].nelv == 0) continue;
    const int key = 2 * meshes[m].lx + mbody[m];
    smem = std::max(smem, f64 ? ax::batch_key_smem_f64(key) : ax::batch_key_smem_f32(key));
  }
  int dev = 0, nsm = 0, bps = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(AX_ELAUNCH);
  if (smem > 0) {
    int rc = f64 ? ax::batch_setup_f64(smem, &bps) : ax::batch_setup_f32(smem, &bps);
    if (rc) return fail(rc);
    if (bps < 1) return fail(AX_EINVAL);
    if (blocks_per_sm > 0) bps = std::min(bps, blocks_per_sm);
  }
  const int ncta = smem > 0 ? nsm * bps : 0;
  // work items: about 8 per CTA of equal cost, k-loop items whole chunks
  std::vector<BatchItem> items;
  std::vector<double> cost;
  const double target = ncta > 0 ? total_cost / (8.0 * ncta) : 1.0;
  for (int m = 0; m < nmesh; ++m) {
    const ax_batch_mesh &s = meshes[m];
    if (s.nelv == 0) continue;
    const double c = elem_cost(s.lx, f64, mbody[m] == ax::kBodyEvenOdd);
    long long chunk = std::max<long long>(1, (long long)(target / c));
    if (mbody[m] == ax::kBodyKLoop) {
      const int epb = ax::batch_kloop_epb(s.lx);
      chunk = (chunk + epb - 1) / epb * epb;
    }
    for (long long e = 0; e < s.nelv; e += chunk) {
      const int nel = (int)std::min<long long>(chunk, s.nelv - e);
      items.push_back(BatchItem{m, nel, e});
      cost.push_back(nel * c);
    }
  }
  // longest processing time first onto the least-loaded CTA
  std::vector<std::vector<int>> per(std::max(ncta, 1));
  {
    std::vector<int> order(items.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    using Load = std::pair<double, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int b = 0; b < ncta; ++b) heap.push({0.0, b});
    for (int q : order) {
      Load ld = heap.top();
      heap.pop();
      per[ld.second].push_back(q);
      heap.push({ld.first + cost[q], ld.second});
    }
  }
  // per CTA: items sorted by (layout key, mesh, first element), then groups
  std::vector<BatchItem> flat;
  std::vector<BatchGroup> groups;
  std::vector<int> start;
  auto key_of = [&](const BatchItem &it) { return 2 * meshes[it.mesh].lx + mbody[it.mesh]; };
  for (int b = 0; b < ncta; ++b) {
    std::vector<BatchItem> mine;
    for (int q : per[b]) mine.push_back(items[q]);
    std::sort(mine.begin(), mine.end(), [&](const BatchItem &x, const BatchItem &y) {
      const int kx = key_of(x), ky = key_of(y);
      if (kx != ky) return kx > ky;
      if (x.mesh != y.mesh) return x.mesh < y.mesh;
      return x.e0 < y.e0;
    });
    start.push_back((int)groups.size());
    for (const BatchItem &it : mine) {
      const int k = key_of(it);
      if (groups.empty() || (int)groups.size() == start.back() || groups.back().key != k)
        groups.push_back(BatchGroup{k, (int)flat.size(), (int)flat.size()});
      flat.push_back(it);
      groups.back().ie = (int)flat.size();
    }
  }
  start.push_back((int)groups.size());
  B->dtype = dtype;
  B->nmesh = nmesh;
  B->nitems = (int)flat.size();
  B->nblocks = ncta;
  B->ngroups = (int)groups.size();
  B->smem = smem;
  B->flops = flops;
  B->bytes = bytes;
  bool ok = upload(&B->d_mesh, mh, st) && upload(&B->d_emesh, em, st) &&
            upload(&B->d_fmesh, fm, st) &&
            upload(&B->d_items, flat, st) && upload(&B->d_groups, groups, st) &&
            upload(&B->d_start, start, st) &&
            cudaMalloc((void **)&B->d_err, sizeof(int)) == cudaSuccess &&
            cudaMemsetAsync(B->d_err, 0, sizeof(int), st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess;
  if (!ok) return fail(AX_ENOMEM);
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

int ax_batch_error(const ax_batch *B, int *flag) {
  if (!B || !flag) return AX_EINVAL;
  *flag = 0;
  if (!B->d_err) return AX_OK;
  if (cudaMemcpy(flag, B->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
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
