// The element operator on host buffers: the inputs stream to the device and
// the result back in chunks of elements, with the copies in and out and the
// apply of different chunks in flight at once (three streams, two device
// buffer sets), so the transfer over the host link, which bounds this path,
// hides the apply and most of the result copy.
#include <algorithm>
#include <mutex>
#include <new>

#include "../../include/axhelm.h"
#include "common.cuh"

namespace {

constexpr int kFields = 9;  // u, h1, g11, g22, g33, g12, g13, g23 in; w out
constexpr int kSlots = 2;   // device buffer sets

// Per-device staging: buffers grow to the largest chunk asked for and are
// kept (the path is meant to be called repeatedly); streams and events are
// created once.
struct Staging {
  bool ready = false;
  size_t per_field = 0;  // doubles per field and slot
  double *buf[kSlots][kFields] = {};
  double *dmat = nullptr;  // dx, dxt
  cudaStream_t s_in = nullptr, s_cmp = nullptr, s_out = nullptr;
  cudaEvent_t in_done[kSlots] = {}, cmp_done[kSlots] = {}, out_done[kSlots] = {};
};

constexpr int kMaxDevices = 64;
Staging g_staging[kMaxDevices];
std::mutex g_staging_mu;

int prepare(Staging &S, size_t per_field) {
  if (!S.ready) {
    if (cudaStreamCreateWithFlags(&S.s_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S.s_cmp, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S.s_out, cudaStreamNonBlocking) != cudaSuccess)
      return AX_ELAUNCH;
    for (int k = 0; k < kSlots; ++k)
      if (cudaEventCreateWithFlags(&S.in_done[k], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&S.cmp_done[k], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&S.out_done[k], cudaEventDisableTiming) != cudaSuccess)
        return AX_ELAUNCH;
    if (cudaMalloc((void **)&S.dmat, 2 * 16 * 16 * sizeof(double)) != cudaSuccess)
      return AX_ENOMEM;
    S.ready = true;
  }
  if (per_field > S.per_field) {
    // the streams are idle here (the previous call synchronised them)
    for (auto &slot : S.buf)
      for (double *&p : slot) {
        cudaFree(p);
        p = nullptr;
      }
    S.per_field = 0;
    for (auto &slot : S.buf)
      for (double *&p : slot)
        if (cudaMalloc((void **)&p, per_field * sizeof(double)) != cudaSuccess) {
          (void)cudaGetLastError();
          return AX_ENOMEM;
        }
    S.per_field = per_field;
  }
  return AX_OK;
}

}  // namespace

extern "C" int ax_helm_host(double *w, const double *u, const double *dx, const double *dxt,
                            const double *h1, const double *g11, const double *g22,
                            const double *g33, const double *g12, const double *g13,
                            const double *g23, int lx, int nelv, int chunk, void *stream) {
  if (!ax::lx_ok(lx) || nelv < 0 || chunk < 0) return AX_EINVAL;
  if (nelv == 0) return AX_OK;
  if (!ax::all_nonnull(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23)) return AX_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AX_ELAUNCH;
  const int64_t n3 = (int64_t)lx * lx * lx;
  if (chunk == 0) chunk = std::max(1, (int)std::min<int64_t>(nelv, (1 << 22) / n3));
  chunk = std::min(chunk, nelv);
  std::lock_guard<std::mutex> lock(g_staging_mu);  // one host-buffer call per process at a time
  Staging &S = g_staging[dev];
  int rc = prepare(S, (size_t)chunk * n3);
  if (rc) return rc;
  cudaStream_t caller = (cudaStream_t)stream;
  // start after the caller's prior work
  cudaEvent_t start;
  if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) return AX_ELAUNCH;
  cudaEventRecord(start, caller);
  cudaStreamWaitEvent(S.s_in, start, 0);
  cudaStreamWaitEvent(S.s_cmp, start, 0);
  cudaStreamWaitEvent(S.s_out, start, 0);
  cudaEventDestroy(start);
  const size_t dm = (size_t)lx * lx * sizeof(double);
  bool ok = cudaMemcpyAsync(S.dmat, dx, dm, cudaMemcpyHostToDevice, S.s_in) == cudaSuccess &&
            cudaMemcpyAsync(S.dmat + lx * lx, dxt, dm, cudaMemcpyHostToDevice, S.s_in) ==
                cudaSuccess;
  const double *in[8] = {u, h1, g11, g22, g33, g12, g13, g23};
  const int nchunk = (nelv + chunk - 1) / chunk;
  for (int c = 0; c < nchunk && ok && rc == AX_OK; ++c) {
    const int k = c % kSlots;
    const int64_t e0 = (int64_t)c * chunk;
    const int ne = (int)std::min<int64_t>(chunk, nelv - e0);
    const size_t off = (size_t)e0 * n3, bytes = (size_t)ne * n3 * sizeof(double);
    // slot k is free once the compute of chunk c - 2 (its inputs) is done
    if (c >= kSlots) cudaStreamWaitEvent(S.s_in, S.cmp_done[k], 0);
    for (int f = 0; f < 8 && ok; ++f)
      ok = cudaMemcpyAsync(S.buf[k][f], in[f] + off, bytes, cudaMemcpyHostToDevice, S.s_in) ==
           cudaSuccess;
    cudaEventRecord(S.in_done[k], S.s_in);
    // compute: after the inputs arrived and the previous result of slot k left
    cudaStreamWaitEvent(S.s_cmp, S.in_done[k], 0);
    if (c >= kSlots) cudaStreamWaitEvent(S.s_cmp, S.out_done[k], 0);
    double *const *b = S.buf[k];
    rc = ax_helm(b[8], b[0], S.dmat, S.dmat + lx * lx, b[1], b[2], b[3], b[4], b[5], b[6], b[7],
                 lx, ne, S.s_cmp);
    cudaEventRecord(S.cmp_done[k], S.s_cmp);
    cudaStreamWaitEvent(S.s_out, S.cmp_done[k], 0);
    ok = ok && cudaMemcpyAsync(w + off, b[8], bytes, cudaMemcpyDeviceToHost, S.s_out) ==
                   cudaSuccess;
    cudaEventRecord(S.out_done[k], S.s_out);
  }
  // the caller's stream continues after the last copy out; the staging
  // streams are drained before the next call may reuse the buffers
  cudaEvent_t end;
  if (cudaEventCreateWithFlags(&end, cudaEventDisableTiming) == cudaSuccess) {
    cudaEventRecord(end, S.s_out);
    cudaStreamWaitEvent(caller, end, 0);
    cudaEventDestroy(end);
  }
  if (cudaStreamSynchronize(S.s_out) != cudaSuccess || cudaStreamSynchronize(S.s_cmp) !=
                                                           cudaSuccess)
    ok = false;
  if (!ok) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  return rc;
}
