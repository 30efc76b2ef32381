// Jacobi-PCG on an element set split across ranks (SPMD): the scalar
// recurrences of the solve, with the rank-local vector work behind an ops
// table and the coupling between ranks behind a comm table.
//
// The element apply needs nothing from other elements; what couples the
// ranks is the gather-scatter sum at nodes that elements of two ranks share
// (the direct-stiffness summation after Ax named in Sec. "Neko and Small
// Tensor Kernel") and the global dot products of CG.  This driver issues no
// CUDA call itself: on a GPU rank the ops are the library's kernels on the
// rank's Poisson handle (ax_cg_solve_part_poisson), elsewhere any
// implementation of the same table.  Textbook PCG from x0 = 0 (the
// single-domain solver's recurrences), two all-sums per iteration (p.w, then
// r.r and r.z together), stopping at ||r|| <= tol ||r0||.
#include <cmath>

#include "../../include/axhelm.h"

extern "C" int ax_cg_solve_part(const ax_part_ops *ops, const ax_part_comm *comm, double *x,
                                const double *b, double *r, double *z, double *p, double *w,
                                double tol, int maxit, int *iters, double *relres,
                                void *stream) {
  if (!ops || !comm || !x || !b || !r || !z || !p || !w || maxit < 0 || !(tol >= 0.0) ||
      !ops->apply || !ops->precond || !ops->dot || !ops->axpby || !ops->copy || !ops->zero ||
      !comm->halo || !comm->allsum)
    return AX_EINVAL;
  void *oc = ops->ctx, *cc = comm->ctx;
  int rc;
#define AX_TRY(call)        \
  if ((rc = (call)) != 0) { \
    return rc;              \
  }
  if (iters) *iters = 0;
  if (relres) *relres = 0.0;
  AX_TRY(ops->zero(oc, x, stream));
  AX_TRY(ops->copy(oc, r, b, stream));
  AX_TRY(ops->precond(oc, z, r, stream));
  AX_TRY(ops->copy(oc, p, z, stream));
  double d[2];
  AX_TRY(ops->dot(oc, r, z, &d[0], stream));
  AX_TRY(ops->dot(oc, r, r, &d[1], stream));
  AX_TRY(comm->allsum(cc, d, 2));
  double rz = d[0];
  const double r0 = std::sqrt(d[1]);
  if (!std::isfinite(r0) || !std::isfinite(rz)) return AX_EBREAKDOWN;
  if (r0 == 0.0) return AX_OK;
  int it = 0;
  double rel = 1.0;
  while (it < maxit) {
    AX_TRY(ops->apply(oc, w, p, stream));
    AX_TRY(comm->halo(cc, w, stream));
    double pw;
    AX_TRY(ops->dot(oc, p, w, &pw, stream));
    AX_TRY(comm->allsum(cc, &pw, 1));
    if (!(pw > 0.0) || !std::isfinite(pw)) {
      if (iters) *iters = it;
      if (relres) *relres = rel;
      return AX_EBREAKDOWN;
    }
    const double alpha = rz / pw;
    AX_TRY(ops->axpby(oc, x, alpha, p, 1.0, stream));
    AX_TRY(ops->axpby(oc, r, -alpha, w, 1.0, stream));
    ++it;
    AX_TRY(ops->precond(oc, z, r, stream));
    AX_TRY(ops->dot(oc, r, r, &d[0], stream));
    AX_TRY(ops->dot(oc, r, z, &d[1], stream));
    AX_TRY(comm->allsum(cc, d, 2));
    rel = std::sqrt(d[0]) / r0;
    if (iters) *iters = it;
    if (relres) *relres = rel;
    if (!std::isfinite(rel)) return AX_EBREAKDOWN;
    if (rel <= tol) return AX_OK;
    const double beta = d[1] / rz;
    AX_TRY(ops->axpby(oc, p, 1.0, z, beta, stream));
    rz = d[1];
  }
#undef AX_TRY
  return AX_ENOTCONV;
}
