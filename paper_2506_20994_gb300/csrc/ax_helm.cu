// C-ABI entry points of the element operator (Listing 2): argument checks
// and dispatch over lx and storage type to the templated kernels.
#include "common.cuh"
#include "dispatch.h"
#include "op.h"

namespace {


template <typename W, typename S, typename T>
int check_args(W *w, const S *u, const T *dx, const T *dxt, const S *h1, const S *g11,
               const S *g22, const S *g33, const S *g12, const S *g13, const S *g23, int lx,
               int nelv) {
  if (!ax::lx_ok(lx) || nelv < 0) return AX_EINVAL;
  if (nelv == 0) return 1;  // no-op
  if (!ax::all_nonnull(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23)) return AX_EINVAL;
  return AX_OK;
}

// variant chosen for AX_VARIANT_AUTO per lx by the tuner; 0 = built-in
// (atomic: the tuner may run on one host thread while others launch)
std::atomic<int> g_variant[AX_LX_MAX + 1];

}  // namespace

extern "C" {

const char *ax_strerror(int code) {
  switch (code) {
    case AX_OK: return "ok";
    case AX_EINVAL: return "invalid argument";
    case AX_ELAUNCH: return "CUDA launch or call failed";
    case AX_ENOMEM: return "allocation failed";
    case AX_ENOTCONV: return "solver did not converge within maxit";
    case AX_EBREAKDOWN: return "solver breakdown (p.Ap <= 0 or non-finite value)";
    case AX_EIO: return "file could not be opened, read or written";
    default: return "unknown status";
  }
}

const char *ax_version(void) { return "axhelm 0.1 sm_103a"; }

int ax_helm_variant(int variant, double *w, const double *u, const double *dx,
                    const double *dxt, const double *h1, const double *g11, const double *g22,
                    const double *g33, const double *g12, const double *g13, const double *g23,
                    int lx, int nelv, int elems_per_block, void *stream) {
  int rc = check_args(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx, nelv);
  if (rc != AX_OK) return rc > 0 ? AX_OK : rc;
  cudaStream_t st = (cudaStream_t)stream;
  // measured on GB300 at E = 32768: the persistent even-odd kernel wins for
  // lx 6, 8, 10, 12 (197 / 416 / 989 / 2021 us against 218 / 564 / 2133 /
  // 4440 for the k-loop); the k-loop double-float kernel for the other lx
  // (13-16 included: the fp64 units run only on request)
  if (variant == AX_VARIANT_AUTO) {
    const int v = g_variant[lx].load(std::memory_order_relaxed);
    if (v != 0) variant = v;
  }
  if (variant == AX_VARIANT_AUTO)
    variant = (lx == 6 || lx == 8 || lx == 10 || lx == 12) ? AX_VARIANT_F64_DF_EO
              : lx <= ax::AX_DF64_LX_MAX        ? AX_VARIANT_F64_DF
                                                : AX_VARIANT_F64_NATIVE;
  switch (variant) {
    case AX_VARIANT_F64_NATIVE:
      return ax::dispatch_kstep_f64(lx, w, u, dx, dxt, h1, g11, g22, g33, g12,
                                                    g13, g23, nelv, elems_per_block, st);
    case AX_VARIANT_F64_DF_EO:
      if (elems_per_block <= 0) {  // the persistent form (lx 6-12, aligned arrays)
        const ax::guard::RawGeo raw{h1, g11, g22, g33, g12, g13, g23};
        const int rp = ax::eopr_launch(lx, w, u, dx, dxt, raw, nelv, st);
        if (rp != AX_EINVAL) return rp;
      }
      return ax::dispatch_df64eo(lx, w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nelv,
                                 elems_per_block, st);
    case AX_VARIANT_F64_DF:
      if (elems_per_block <= 0) elems_per_block = ax::tuned_epb(AX_BATCH_F64, lx);
      return ax::dispatch_df64(lx, w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nelv,
                           elems_per_block, st);
    default:
      return AX_EINVAL;
  }
}

int ax_helm_h2(double *w, const double *u, const double *dx, const double *dxt,
               const double *h1, const double *g11, const double *g22, const double *g33,
               const double *g12, const double *g13, const double *g23, const double *h2,
               const double *B, int lx, int nelv, void *stream) {
  if (nelv > 0 && !ax::all_nonnull(h2, B)) return AX_EINVAL;
  int rc = ax_helm(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx, nelv, stream);
  if (rc || nelv == 0) return rc;
  return ax::mass_add2(w, h2, B, u, (int64_t)nelv * lx * lx * lx, (cudaStream_t)stream);
}

int ax_helm(double *w, const double *u, const double *dx, const double *dxt, const double *h1,
            const double *g11, const double *g22, const double *g33, const double *g12,
            const double *g13, const double *g23, int lx, int nelv, void *stream) {
  return ax_helm_variant(AX_VARIANT_AUTO, w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx,
                         nelv, 0, stream);
}

int ax_helm_f32(float *w, const float *u, const float *dx, const float *dxt, const float *h1,
                const float *g11, const float *g22, const float *g33, const float *g12,
                const float *g13, const float *g23, int lx, int nelv, void *stream) {
  int rc = check_args(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx, nelv);
  if (rc != AX_OK) return rc > 0 ? AX_OK : rc;
  if (ax::eo32_ok(lx, w, u, h1, g11, g22, g33, g12, g13, g23)) {
    const float *g[7] = {h1, g11, g22, g33, g12, g13, g23};
    return ax::dispatch_eo32_f32(lx, w, u, dx, dxt, g, nelv, nullptr, nullptr,
                                 (cudaStream_t)stream);
  }
  return ax::dispatch_kstep_f32(lx, w, u, dx, dxt, h1, g11, g22, g33, g12, g13,
                                             g23, nelv, ax::tuned_epb(AX_BATCH_F32, lx),
                                             (cudaStream_t)stream);
}

int ax_helm_bf16(float *w, const ax_bf16 *u, const float *dx, const float *dxt,
                 const ax_bf16 *h1, const ax_bf16 *g11, const ax_bf16 *g22, const ax_bf16 *g33,
                 const ax_bf16 *g12, const ax_bf16 *g13, const ax_bf16 *g23, int lx, int nelv,
                 void *stream) {
  int rc = check_args(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx, nelv);
  if (rc != AX_OK) return rc > 0 ? AX_OK : rc;
  using B = __nv_bfloat16;
  auto c = [](const ax_bf16 *p) { return reinterpret_cast<const B *>(p); };
  if (ax::eo32_ok(lx, w, u, h1, g11, g22, g33, g12, g13, g23)) {
    const B *g[7] = {c(h1), c(g11), c(g22), c(g33), c(g12), c(g13), c(g23)};
    return ax::dispatch_eo32_bf16(lx, w, c(u), dx, dxt, g, nelv, nullptr, nullptr,
                                  (cudaStream_t)stream);
  }
  return ax::dispatch_kstep_bf16(lx, w, c(u), dx, dxt, c(h1), c(g11), c(g22), c(g33),
                                         c(g12), c(g13), c(g23), nelv, 0, (cudaStream_t)stream);
}

}  // extern "C"

extern "C" int ax_tune_variant_run(int lx, int nelv, double *w, const double *u,
                                   const double *dx, const double *dxt, const double *h1,
                                   const double *g11, const double *g22, const double *g33,
                                   const double *g12, const double *g13, const double *g23,
                                   int reps, int *best_variant, float *best_ms, void *stream) {
  if (!ax::lx_ok(lx) || nelv <= 0 || reps < 1 ||
      !ax::all_nonnull(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23))
    return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return AX_ELAUNCH;
  const int cands[3] = {AX_VARIANT_F64_NATIVE, AX_VARIANT_F64_DF, AX_VARIANT_F64_DF_EO};
  int best = 0;
  float best_t = 1e30f;
  for (int v : cands) {
    auto run = [&]() {
      return ax_helm_variant(v, w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx, nelv, 0,
                             stream);
    };
    if (run() != AX_OK) {  // inadmissible for this lx
      (void)cudaGetLastError();
      continue;
    }
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
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best == 0) return AX_ELAUNCH;
  g_variant[lx].store(best, std::memory_order_relaxed);
  if (best_variant) *best_variant = best;
  if (best_ms) *best_ms = best_t;
  return AX_OK;
}

extern "C" int ax_tune_variant_set(int lx, int variant) {
  if (!ax::lx_ok(lx) || variant < AX_VARIANT_AUTO || variant > AX_VARIANT_F64_DF_EO)
    return AX_EINVAL;
  g_variant[lx].store(variant, std::memory_order_relaxed);
  return AX_OK;
}

extern "C" int ax_tune_variant_get(int lx, int *variant) {
  if (!ax::lx_ok(lx) || !variant) return AX_EINVAL;
  *variant = g_variant[lx].load(std::memory_order_relaxed);
  return AX_OK;
}
