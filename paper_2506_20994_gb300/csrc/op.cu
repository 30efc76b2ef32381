// Operator handle: the element operator of one mesh for repeated applies
// (the opaque handle of the paper's C interface, Listing 1).  Where the
// even-odd kernel applies, the handle keeps the geometry in that kernel's
// prepared order (converted once here), so each apply reads the same bytes
// per point as from the fp64 arrays but spends no instruction on converting
// them.
#include <algorithm>
#include <new>
#include <vector>

#include "../../include/axhelm.h"
#include "common.cuh"
#include "dispatch.h"
#include "op.h"

struct ax_op {
  int lx = 0, nelv = 0;
  const double *dx = nullptr, *dxt = nullptr, *h1 = nullptr, *g[6] = {};
  ax::df::dd2 *gp = nullptr;    // prepared geometry (owned), or null
  ax::df::dd2 *coef = nullptr;  // staged half-size coefficients of D, D^T (owned)
  int *err = nullptr;           // device word: a staged copy never arrived (owned)
  int dfield = 0;               // exponent field of the matrices' largest entry
  double *hb = nullptr;         // h2 .* B of the Helmholtz form (owned), or null
  long long drop = -1;          // testing aid (ax_op_inject_copy_loss)
};

namespace {
__global__ void hb_kernel(double *__restrict__ hb, const double *__restrict__ h2,
                          const double *__restrict__ B, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    hb[q] = h2[q] * B[q];
}
}  // namespace

namespace {

// measured on GB300: the persistent even-odd kernel on prepared geometry is
// the fastest fp64 form for these orders
bool op_prepares(int lx) { return ax::eop_supported(lx); }

ax::EopArgs eop_args(const ax_op *op, double *w, const double *u) {
  ax::EopArgs a;
  a.w = w;
  a.u = u;
  a.coef = op->coef;
  a.gp = op->gp;
  a.raw = ax::guard::RawGeo{op->h1, op->g[0], op->g[1], op->g[2], op->g[3], op->g[4], op->g[5]};
  a.dx = op->dx;
  a.dxt = op->dxt;
  a.dfield = op->dfield;
  a.nelv = op->nelv;
  a.err = op->err;
  a.drop = op->drop;
  return a;
}

}  // namespace

extern "C" int ax_op_destroy(ax_op *op) {
  if (!op) return AX_EINVAL;
  if (op->gp) cudaFree(op->gp);
  if (op->coef) cudaFree(op->coef);
  if (op->err) cudaFree(op->err);
  if (op->hb) cudaFree(op->hb);
  delete op;
  return AX_OK;
}

extern "C" int ax_op_create(ax_op **out, int lx, int nelv, const double *dx, const double *dxt,
                            const double *h1, const double *g11, const double *g22,
                            const double *g33, const double *g12, const double *g13,
                            const double *g23, void *stream) {
  if (!out || lx < 2 || lx > 16 || nelv < 0 ||
      !ax::all_nonnull(dx, dxt, h1, g11, g22, g33, g12, g13, g23))
    return AX_EINVAL;
  *out = nullptr;
  ax_op *op = new (std::nothrow) ax_op();
  if (!op) return AX_ENOMEM;
  op->lx = lx;
  op->nelv = nelv;
  op->dx = dx;
  op->dxt = dxt;
  op->h1 = h1;
  const double *gg[6] = {g11, g22, g33, g12, g13, g23};
  for (int k = 0; k < 6; ++k) op->g[k] = gg[k];
  cudaStream_t st = (cudaStream_t)stream;
  if (op_prepares(lx) && nelv > 0) {
    // the even-odd split reads half the rows of dx and dxt: check them here,
    // once; matrices without the symmetry keep ax_helm's path
    std::vector<double> dh((size_t)lx * lx), dth((size_t)lx * lx);
    std::vector<unsigned char> cb(ax::eop_coef_bytes(lx));
    if (cudaMemcpyAsync(dh.data(), dx, dh.size() * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(dth.data(), dxt, dth.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      (void)cudaGetLastError();
      delete op;
      return AX_ELAUNCH;
    }
    if (ax::eop_coefficients(lx, dh.data(), dth.data(), cb.data(), &op->dfield)) {
      if (cudaMalloc((void **)&op->gp, ax::eo_prep_bytes(lx, nelv)) != cudaSuccess ||
          cudaMalloc((void **)&op->coef, cb.size()) != cudaSuccess ||
          cudaMalloc((void **)&op->err, sizeof(int)) != cudaSuccess) {
        (void)cudaGetLastError();
        ax_op_destroy(op);
        return AX_ENOMEM;
      }
      int rc = AX_OK;
      if (cudaMemcpyAsync(op->coef, cb.data(), cb.size(), cudaMemcpyHostToDevice, st) !=
              cudaSuccess ||
          cudaMemsetAsync(op->err, 0, sizeof(int), st) != cudaSuccess)
        rc = AX_ELAUNCH;
      if (rc == AX_OK)
        rc = ax::eop_prepare(lx, op->gp,
                             ax::guard::RawGeo{h1, g11, g22, g33, g12, g13, g23}, nelv, 0x7F,
                             op->dfield, st);
      if (rc == AX_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = AX_ELAUNCH;
      if (rc) {
        (void)cudaGetLastError();
        ax_op_destroy(op);
        return rc;
      }
    }
  }
  *out = op;
  return AX_OK;
}

extern "C" int ax_op_set_h1(ax_op *op, const double *h1, void *stream) {
  if (!op || !h1) return AX_EINVAL;
  op->h1 = h1;
  if (!op->gp) return AX_OK;
  const double *const *g = op->g;
  return ax::eop_prepare(op->lx, op->gp, ax::guard::RawGeo{h1, g[0], g[1], g[2], g[3], g[4], g[5]},
                         op->nelv, 0x40, op->dfield, (cudaStream_t)stream);
}

extern "C" int ax_op_set_h2(ax_op *op, const double *h2, const double *B, void *stream) {
  if (!op) return AX_EINVAL;
  if (!h2) {
    if (op->hb) cudaFree(op->hb);
    op->hb = nullptr;
    return AX_OK;
  }
  if (!B) return AX_EINVAL;
  const int64_t n = (int64_t)op->nelv * op->lx * op->lx * op->lx;
  if (!op->hb && cudaMalloc((void **)&op->hb, std::max<int64_t>(n, 1) * sizeof(double)) !=
                     cudaSuccess) {
    (void)cudaGetLastError();
    op->hb = nullptr;
    return AX_ENOMEM;
  }
  hb_kernel<<<608, 256, 0, (cudaStream_t)stream>>>(op->hb, h2, B, n);
  return ax::launch_status();
}

extern "C" int ax_op_apply(ax_op *op, double *w, const double *u, void *stream) {
  if (!op || (op->nelv > 0 && (!w || !u))) return AX_EINVAL;
  if (op->nelv == 0) return AX_OK;
  int rc;
  if (op->gp) {
    rc = ax::eop_launch(op->lx, eop_args(op, w, u), (cudaStream_t)stream);
  } else {
    const double *const *g = op->g;
    rc = ax_helm(w, u, op->dx, op->dxt, op->h1, g[0], g[1], g[2], g[3], g[4], g[5], op->lx,
                 op->nelv, stream);
  }
  if (rc || !op->hb) return rc;
  const int64_t n = (int64_t)op->nelv * op->lx * op->lx * op->lx;
  return ax::mass_add<double>(w, op->hb, u, n, nullptr, (cudaStream_t)stream);
}

namespace ax {

int op_dot_blocks(const ax_op *op) {
  return op && op->gp ? eop_blocks(op->lx, op->nelv, true) : 0;
}

int op_apply_dot(ax_op *op, double *w, const double *u, double *partials, cudaStream_t st) {
  if (!op || !op->gp || !partials) return AX_EINVAL;
  EopArgs a = eop_args(op, w, u);
  a.dotp = partials;
  return eop_launch(op->lx, a, st);
}

int op_update_apply_dot(ax_op *op, double *w, double *p, const double *r, const double *minv,
                        const double *beta, double *partials, cudaStream_t st,
                        const double *corr, const int *use_corr) {
  if (!op || !op->gp || !partials || !p || !r || !minv || !beta) return AX_EINVAL;
  EopArgs a = eop_args(op, w, nullptr);
  a.dotp = partials;
  a.pw = p;
  a.r = r;
  a.minv = minv;
  a.beta = beta;
  a.corr = corr;
  a.use_corr = use_corr;
  return eop_launch(op->lx, a, st);
}

}  // namespace ax

extern "C" int ax_op_info(const ax_op *op, int *prepared, int64_t *device_bytes) {
  if (!op) return AX_EINVAL;
  if (prepared) *prepared = op->gp != nullptr;
  if (device_bytes)
    *device_bytes = op->gp ? (int64_t)(ax::eo_prep_bytes(op->lx, op->nelv) +
                                       ax::eop_coef_bytes(op->lx) + sizeof(int))
                           : 0;
  return AX_OK;
}

extern "C" int ax_op_inject_copy_loss(ax_op *op, int64_t element) {
  if (!op || element < -1 || element >= op->nelv) return AX_EINVAL;
  op->drop = element;
  return AX_OK;
}

extern "C" int ax_op_error(const ax_op *op, int *flag) {
  if (!op || !flag) return AX_EINVAL;
  *flag = 0;
  if (!op->err) return AX_OK;
  if (cudaMemcpy(flag, op->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  return AX_OK;
}
