// Declarations of the per-lx dispatchers; each is defined in its own
// translation unit so that the kernel instantiations compile in parallel.
#pragma once

#include "df64.cuh"
#include "guard.cuh"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace ax {

// Tuned elements per block for (AX_BATCH_F64 | AX_BATCH_F32, lx); 0 if untuned.
int tuned_epb(int dtype, int lx);

// Largest lx with a double-float instantiation (every lx the library takes).
constexpr int AX_DF64_LX_MAX = 16;

// k-loop kernel: fp64 storage and fp64 units.
int dispatch_kstep_f64(int lx, double *w, const double *u, const double *dx, const double *dxt,
                       const double *h1, const double *g11, const double *g22,
                       const double *g33, const double *g12, const double *g13,
                       const double *g23, int nelv, int epb, cudaStream_t st);
// k-loop kernel: fp32 storage and arithmetic.
int dispatch_kstep_f32(int lx, float *w, const float *u, const float *dx, const float *dxt,
                       const float *h1, const float *g11, const float *g22, const float *g33,
                       const float *g12, const float *g13, const float *g23, int nelv, int epb,
                       cudaStream_t st, double *dotp = nullptr);
// k-loop kernel: bf16 storage of u, h1, G; fp32 D, arithmetic and w.
int dispatch_kstep_bf16(int lx, float *w, const __nv_bfloat16 *u, const float *dx,
                        const float *dxt, const __nv_bfloat16 *h1, const __nv_bfloat16 *g11,
                        const __nv_bfloat16 *g22, const __nv_bfloat16 *g33,
                        const __nv_bfloat16 *g12, const __nv_bfloat16 *g13,
                        const __nv_bfloat16 *g23, int nelv, int epb, cudaStream_t st);

// k-loop kernel: fp32 u, bf16 h1 and G; fp32 D, arithmetic and w.
int dispatch_kstep_f32u_bf16(int lx, float *w, const float *u, const float *dx, const float *dxt,
                             const __nv_bfloat16 *h1, const __nv_bfloat16 *g11,
                             const __nv_bfloat16 *g22, const __nv_bfloat16 *g33,
                             const __nv_bfloat16 *g12, const __nv_bfloat16 *g13,
                             const __nv_bfloat16 *g23, int nelv, int epb, cudaStream_t st,
                             double *dotp = nullptr);
// Persistent even-odd operator with fp32 arithmetic (ax_eo32.cuh) for
// lx in {6, 8, 10, 12} (AX_EINVAL otherwise): u stored as fp32 or bf16,
// g = {h1, g11, g22, g33, g12, g13, g23} as fp32 or bf16, fp32 D and w.
// Every array must be 16-byte aligned (eo32_ok).  dotp: one partial of
// u . w per CTA, eo32_blocks_*(lx, nelv) of them (the same count with and
// without the fused update, up, which needs dotp).  err: device word set to
// 1 if a staged copy never arrived (may be null; the affected elements are
// then written as NaN).
// The solver's fused direction update for the fp32-vector forms: the kernel
// first forms pw = minv .* r + (*beta) pw in place (fp32) and applies the
// operator to it (u is then ignored).
struct E32Upd {
  float *pw = nullptr;
  const float *r = nullptr, *minv = nullptr;
  const double *beta = nullptr;
};
int dispatch_eo32_f32(int lx, float *w, const float *u, const float *dx, const float *dxt,
                      const float *const g[7], int nelv, int *err, double *dotp,
                      cudaStream_t st, const E32Upd *up = nullptr);
int dispatch_eo32_bf16(int lx, float *w, const __nv_bfloat16 *u, const float *dx,
                       const float *dxt, const __nv_bfloat16 *const g[7], int nelv, int *err,
                       double *dotp, cudaStream_t st, const E32Upd *up = nullptr);
int dispatch_eo32_f32u_bf16(int lx, float *w, const float *u, const float *dx,
                            const float *dxt, const __nv_bfloat16 *const g[7], int nelv,
                            int *err, double *dotp, cudaStream_t st,
                            const E32Upd *up = nullptr);
// The same operator at lx = 8 on bf16 geometry, one warp per element
// (ax_eo32w.cuh): u in bf16 (dispatch_eo32_bf16 takes it without dotp) or
// the solvers' fp32 vectors (dispatch_eo32_f32u_bf16 takes it at lx = 8 in
// every variant, the fused update included); w has the same bits as the
// octant kernel's.  dotp: one partial per CTA, eo32w_blocks_*(nelv) of them.
int dispatch_eo32w_bf16(float *w, const __nv_bfloat16 *u, const float *dx, const float *dxt,
                        const __nv_bfloat16 *const g[7], int nelv, int *err, double *dotp,
                        cudaStream_t st);
int dispatch_eo32w_f32u_bf16(float *w, const float *u, const float *dx, const float *dxt,
                             const __nv_bfloat16 *const g[7], int nelv, int *err, double *dotp,
                             cudaStream_t st, const E32Upd *up = nullptr);
int eo32w_blocks_bf16(int nelv);
int eo32w_blocks_f32u_bf16(int nelv);
int eo32_blocks_f32(int lx, int nelv);
int eo32_blocks_bf16(int lx, int nelv);
int eo32_blocks_f32u_bf16(int lx, int nelv);
// lx 4 stays on the k-loop kernel (measured faster there: 142 against 162 us
// for fp32 at 2^26 points)
inline bool eo32_lx(int lx) { return lx >= 6 && lx <= 12 && lx % 2 == 0; }
template <class... P>
inline bool eo32_ok(int lx, const P *...p) {
  return eo32_lx(lx) && ((((uintptr_t)p) % 16 == 0) && ...);
}
// Blocks (and dot partials) of a k-loop launch with the default elements per
// block.
inline int kstep_blocks(int lx, int nelv) {
  int e = 256 / (lx * lx);
  e = e < 1 ? 1 : e;
  return (nelv + e - 1) / e;
}
// Even-odd double-float kernel (lx in {4, 6, 8, 10, 12}; AX_EINVAL otherwise).
int dispatch_df64eo(int lx, double *w, const double *u, const double *dx, const double *dxt,
                    const double *h1, const double *g11, const double *g22, const double *g33,
                    const double *g12, const double *g13, const double *g23, int nelv, int epb,
                    cudaStream_t st);
inline bool df64eo_supported(int lx) { return lx >= 4 && lx <= 12 && lx % 2 == 0; }
// Persistent even-odd operator of the operator handle (ax_eo_persist.cuh),
// lx in {6, 8, 10, 12}.  gp: geometry prepared by eop_prepare (eo_prep_bytes
// bytes, the keys at its end); coef: the block eop_coefficients writes
// (eop_coef_bytes, device); dfield: its matrices' exponent field.  dotp:
// one partial of u . w per CTA, eop_blocks(lx, nelv, true) of them; pw, r,
// minv, beta (+ corr, use_corr): the fused direction update, pw = minv .* r
// (+ corr when *use_corr) + (*beta) pw formed in place before the apply.  err: device word set to 1 if a staged copy never
// arrived (may be null).
struct EopArgs {
  double *w = nullptr;
  const double *u = nullptr;
  const df::dd2 *coef = nullptr, *gp = nullptr;
  guard::RawGeo raw{};
  const double *dx = nullptr, *dxt = nullptr;
  int dfield = 0, nelv = 0;
  int *err = nullptr;
  double *dotp = nullptr, *pw = nullptr;
  const double *r = nullptr, *minv = nullptr, *beta = nullptr, *corr = nullptr;
  const int *use_corr = nullptr;
  long long drop = -1;  // testing aid: element whose geometry copy is not issued
};
bool eop_supported(int lx);
// The persistent even-odd kernel on the caller's fp64 arrays (ax_helm, no
// handle): lx in {6, 8, 10, 12} and 16-byte aligned geometry arrays, else
// AX_EINVAL (the caller then takes another kernel).
int eopr_launch(int lx, double *w, const double *u, const double *dx, const double *dxt,
                const guard::RawGeo &raw, int nelv, cudaStream_t st);
int eop_launch(int lx, const EopArgs &a, cudaStream_t st);
int eop_blocks(int lx, int nelv, bool dot);
// dfield: as eop_coefficients reports it (the per-element u ranges depend on it)
int eop_prepare(int lx, df::dd2 *gp, const guard::RawGeo &raw, int nelv, int fmask, int dfield,
                cudaStream_t st);
size_t eop_coef_bytes(int lx);
bool eop_coefficients(int lx, const double *dx_host, const double *dxt_host, void *out,
                      int *dfield);

// Bytes of a prepared-geometry buffer: 56 lx^3 per element of double-float
// pairs, then two exponent keys per element.
inline size_t eo_prep_bytes(int lx, int nelv) {
  return (size_t)nelv * 56 * lx * lx * lx + (size_t)nelv * 8;
}


// fp64-accurate double-float kernel, lx in 2..7 (a), 8..10 (b), 11..12 (c),
// 13..14 (d), 15..16 (e); AX_EINVAL above AX_DF64_LX_MAX.
#define AX_DF64_DECL(X)                                                                        \
  int dispatch_df64_##X(int lx, double *w, const double *u, const double *dx,                  \
                        const double *dxt, const double *h1, const double *g11,                \
                        const double *g22, const double *g33, const double *g12,               \
                        const double *g13, const double *g23, int nelv, int epb,               \
                        cudaStream_t st);
AX_DF64_DECL(a)
AX_DF64_DECL(b)
AX_DF64_DECL(c)
AX_DF64_DECL(d)
AX_DF64_DECL(e)
#undef AX_DF64_DECL

inline int dispatch_df64(int lx, double *w, const double *u, const double *dx, const double *dxt,
                  const double *h1, const double *g11, const double *g22, const double *g33,
                  const double *g12, const double *g13, const double *g23, int nelv, int epb,
                  cudaStream_t st) {
  if (lx > AX_DF64_LX_MAX) return AX_EINVAL;
  auto f = lx <= 7    ? dispatch_df64_a
           : lx <= 10 ? dispatch_df64_b
           : lx <= 12 ? dispatch_df64_c
           : lx <= 14 ? dispatch_df64_d
                      : dispatch_df64_e;
  return f(lx, w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nelv, epb, st);
}

}  // namespace ax

#define AX_LX_CASES(M) \
  M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12) M(13) M(14) M(15) M(16)
