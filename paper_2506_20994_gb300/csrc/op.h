// Library-internal entry points of the operator handle (op.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/axhelm.h"

namespace ax {

// Partials that op_apply_dot writes (0 when the handle has no prepared
// geometry, where op_apply_dot returns AX_EINVAL).
int op_dot_blocks(const ax_op *op);
// w = Ax(u) as ax_op_apply, plus partials[b] = sum over block b's elements
// of u . w (element-local, before any gather-scatter; fixed order).
int op_apply_dot(ax_op *op, double *w, const double *u, double *partials, cudaStream_t st);
// The solver's direction update fused in front of the same apply:
// p = z + (*beta) p in place (fp64), z = minv .* r (+ corr when *use_corr),
// then w = Ax(p) and the partials of p . w.  beta, use_corr: device scalars.
int op_update_apply_dot(ax_op *op, double *w, double *p, const double *r, const double *minv,
                        const double *beta, double *partials, cudaStream_t st,
                        const double *corr = nullptr, const int *use_corr = nullptr);

// w += hb .* u over n points; partials (optional): kRedBlocks partial sums
// of u . hb . u (the mass term's share of a fused p . Ap).
template <typename T>
int mass_add(T *w, const T *hb, const T *u, int64_t n, double *partials, cudaStream_t st);
// w += (h2 .* B) .* u over n points (coefficient and mass given apart).
int mass_add2(double *w, const double *h2, const double *B, const double *u, int64_t n,
              cudaStream_t st);

}  // namespace ax
