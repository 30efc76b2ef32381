// Poisson solve built on the element operator: the assembled, masked
// operator A p = mask .* gs(Ax(p)) (the matrix-free evaluation of the weak
// Poisson form of Sec. "The Spectral Element Method", assembled by the
// gather-scatter of Sec. "Neko and Small Tensor Kernel"), the exact Jacobi
// diagonal, Jacobi-preconditioned conjugate gradients in fp64, and an
// iterative-refinement solve whose inner CG runs in fp32 (fp32 or bf16
// operator data) while the outer residual, inner products and updates stay
// fp64.  The paper prints no solver; the method is textbook PCG (Hestenes &
// Stiefel 1952) and mixed-precision iterative refinement (Wilkinson 1963;
// Carson & Higham 2018).
//
// Vectors are local (E * lx^3, element-major, continuous across shared
// nodes).  Inner products run over unique global nodes, i.e. the local sum
// weighted by 1/multiplicity.  The scalars of the iteration live on the
// device; the host reads the residual norm every `check_every` iterations.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "dispatch.h"
#include "op.h"
#include "mlp.cuh"
#include "reduce.cuh"

struct ax_gs;
extern "C" int ax_gs_sum(ax_gs *g, double *v, void *stream);
extern "C" int ax_gs_sum_f32(ax_gs *g, float *v, void *stream);
extern "C" const double *ax_gs_inverse_multiplicity(const ax_gs *g);

namespace {

using ax::kRedBlocks;
using ax::kRedThreads;

// Device-side scalars of one CG run.
struct CgScalars {
  double rz, rz_new, rr, rr0, pap, alpha, beta;
  int status;     // 0 ok, 1 breakdown (p.Ap <= 0 or non-finite)
  int use_corr;   // flexible CG: 1 if the learned correction is in z
  int fallbacks;  // flexible CG: steps that fell back to Jacobi
};

// ---------------------------------------------------------------- kernels
template <typename... P>
__device__ __forceinline__ bool aligned16(const P *...p) {
  return ((reinterpret_cast<uintptr_t>(p) | ...) & 15u) == 0;
}

__global__ void jacobi_diag_kernel(double *__restrict__ diag, const double *__restrict__ dx,
                                   const double *__restrict__ h1, const double *__restrict__ g11,
                                   const double *__restrict__ g22, const double *__restrict__ g33,
                                   const double *__restrict__ g12, const double *__restrict__ g13,
                                   const double *__restrict__ g23, int lx, int64_t n) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int n2 = lx * lx, n3 = n2 * lx;
  const int64_t e = q / n3;
  const int p = (int)(q - e * n3);
  const int k = p / n2, j = (p / lx) % lx, i = p % lx;
  const int64_t b = e * n3;
  // D_{ab} = dx[b*lx + a]
  double s = 0.0;
  for (int l = 0; l < lx; ++l) {
    const double dli = dx[i * lx + l], dlj = dx[j * lx + l], dlk = dx[k * lx + l];
    const int64_t qi = b + (k * lx + j) * lx + l, qj = b + (k * lx + l) * lx + i,
                  qk = b + (l * lx + j) * lx + i;
    s += dli * dli * h1[qi] * g11[qi] + dlj * dlj * h1[qj] * g22[qj] +
         dlk * dlk * h1[qk] * g33[qk];
  }
  const double di = dx[i * lx + i], dj = dx[j * lx + j], dk = dx[k * lx + k];
  s += 2.0 * h1[q] * (di * dj * g12[q] + di * dk * g13[q] + dj * dk * g23[q]);
  diag[q] = s;
}

// minv = mask / diag (0 where masked); cm = c * minv; also fp32 copies.
__global__ void precond_kernel(double *__restrict__ minv, double *__restrict__ cm,
                               const double *__restrict__ diag, const double *__restrict__ mask,
                               const double *__restrict__ c, int64_t n) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double m = (mask[q] != 0.0 && diag[q] != 0.0) ? 1.0 / diag[q] : 0.0;
  minv[q] = m;
  cm[q] = c[q] * m;
}

// sqm = sqrt(minv) in fp32 (the scale of the symmetric learned form)
__global__ void sqrt_minv_kernel(float *__restrict__ sqm, const double *__restrict__ minv,
                                 int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    sqm[q] = sqrtf(ax::df::split(minv[q]).hi);
}

// r = b (masked), p = minv r; partials: rz = sum cm r^2, rr = sum c r^2
template <typename T>
__global__ void cg_init_kernel(T *__restrict__ x, T *__restrict__ r, T *__restrict__ p,
                               const T *__restrict__ b, const T *__restrict__ mask,
                               const T *__restrict__ minv, const T *__restrict__ c,
                               double *__restrict__ partials, int64_t n) {
  __shared__ double sh[2 * kRedThreads / 32];
  T a_rz = 0, a_rr = 0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const T rv = b[q] * mask[q];
    x[q] = T(0);
    r[q] = rv;
    const T z = minv[q] * rv;
    p[q] = z;
    const T cq = c[q];
    a_rz += cq * rv * z;
    a_rr += cq * rv * rv;
  }
  double v[2] = {(double)a_rz, (double)a_rr};
  ax::block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = v[0];
    partials[gridDim.x + blockIdx.x] = v[1];
  }
}

// w = mask .* w; partial sum of c p w
template <typename T>
__global__ void mask_dot_kernel(T *__restrict__ w, const T *__restrict__ p,
                                const T *__restrict__ mask, const T *__restrict__ c,
                                double *__restrict__ partials, int64_t n) {
  __shared__ double sh[kRedThreads / 32];
  T a = 0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const T wv = w[q] * mask[q];
    w[q] = wv;
    a += c[q] * p[q] * wv;
  }
  double v[1] = {(double)a};
  ax::block_sum<1>(v, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

// alpha = rz / <p, Ap> from the partials (one warp for the fixed-grid
// partials; a whole block for the per-element-block partials of the fused
// apply)
__global__ void cg_alpha_kernel(const double *__restrict__ partials, int nblk,
                                CgScalars *__restrict__ s) {
  __shared__ double t[32];
  double pap_all;
  if (blockDim.x == 32) {
    ax::warp_sum_partials<1>(partials, nblk, t);
    __syncthreads();
    pap_all = t[0];
  } else {
    pap_all = ax::block_sum_partials(partials, nblk, t);
  }
  if (threadIdx.x == 0) {
    const double pap = pap_all;
    s->pap = pap;
    if (!(pap > 0.0) || !isfinite(pap) || !isfinite(s->rz)) {
      s->status = 1;
      s->alpha = 0.0;
    } else {
      s->alpha = s->rz / pap;
    }
  }
}

// x += alpha p; r -= alpha w; partials rz' = sum cm r^2, rr' = sum c r^2
// MASKW: w is not masked yet (fused apply); the Dirichlet rows, where
// cm = c * minv is 0, keep r = 0.  RR: also the rr partials; rr only feeds
// the host's convergence test, so iterations it does not check skip that sum
// and the read of c (their rr partials are written as 0).
template <typename T, bool MASKW = false, bool RR = true>
__global__ void cg_update_kernel(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p,
                                 const T *__restrict__ w, const T *__restrict__ cm,
                                 const T *__restrict__ c, const CgScalars *__restrict__ s,
                                 double *__restrict__ partials, int64_t n) {
  __shared__ double sh[2 * kRedThreads / 32];
  const T alpha = (T)s->alpha;
  T a_rz = 0, a_rr = 0;
  auto point = [&](T &xq, T &rq, T pq, T wq, T cmq, T cq) {
    xq += alpha * pq;
    const T rv = (MASKW && cmq == T(0)) ? rq : rq - alpha * wq;
    rq = rv;
    const T r2 = rv * rv;
    a_rz += cmq * r2;
    if constexpr (RR) a_rr += cq * r2;
  };
  int64_t q0 = 0;
  if constexpr (sizeof(T) == 4) {
    if (aligned16(x, r, p, w, cm, c)) {  // fp32: 16-byte accesses
      using V = float4;
      const int64_t n4 = n / 4;
      for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n4;
           v += (int64_t)gridDim.x * blockDim.x) {
        V xv = reinterpret_cast<V *>(x)[v], rv = reinterpret_cast<V *>(r)[v];
        const V pv = reinterpret_cast<const V *>(p)[v], wv = reinterpret_cast<const V *>(w)[v];
        const V mv = reinterpret_cast<const V *>(cm)[v];
        const V cv = RR ? reinterpret_cast<const V *>(c)[v] : V{0.f, 0.f, 0.f, 0.f};
        point(xv.x, rv.x, pv.x, wv.x, mv.x, cv.x);
        point(xv.y, rv.y, pv.y, wv.y, mv.y, cv.y);
        point(xv.z, rv.z, pv.z, wv.z, mv.z, cv.z);
        point(xv.w, rv.w, pv.w, wv.w, mv.w, cv.w);
        reinterpret_cast<V *>(x)[v] = xv;
        reinterpret_cast<V *>(r)[v] = rv;
      }
      q0 = n4 * 4;
    }
  } else if constexpr (!RR) {
    // fp64: 16-byte accesses, two points each (measured faster without the rr
    // sum, 174 vs 205 us at 16.8 M points; with it, slower: 245 vs 203 us)
    if (aligned16(x, r, p, w, cm, c)) {
      using V = double2;
      const int64_t n2 = n / 2;
      for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n2;
           v += (int64_t)gridDim.x * blockDim.x) {
        V xv = reinterpret_cast<V *>(x)[v], rv = reinterpret_cast<V *>(r)[v];
        const V pv = reinterpret_cast<const V *>(p)[v], wv = reinterpret_cast<const V *>(w)[v];
        const V mv = reinterpret_cast<const V *>(cm)[v];
        const V cv = RR ? reinterpret_cast<const V *>(c)[v] : V{0.0, 0.0};
        point(xv.x, rv.x, pv.x, wv.x, mv.x, cv.x);
        point(xv.y, rv.y, pv.y, wv.y, mv.y, cv.y);
        reinterpret_cast<V *>(x)[v] = xv;
        reinterpret_cast<V *>(r)[v] = rv;
      }
      q0 = n2 * 2;
    }
  }
  for (int64_t q = q0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    point(x[q], r[q], p[q], w[q], cm[q], RR ? c[q] : T(0));
  double v[2] = {(double)a_rz, (double)a_rr};
  ax::block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = v[0];
    partials[gridDim.x + blockIdx.x] = v[1];
  }
}

// first=1: rz = partial sums, rr0 = rr.  Otherwise beta = rz'/rz.
__global__ void cg_beta_kernel(const double *__restrict__ partials, int nblk,
                               CgScalars *__restrict__ s, int first) {
  __shared__ double t[2];
  ax::warp_sum_partials<2>(partials, nblk, t);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (first) {
      s->rz = t[0];
      s->rr = t[1];
      s->rr0 = t[1];
      s->beta = 0.0;
      s->status = 0;
    } else {
      s->beta = (s->rz != 0.0) ? t[0] / s->rz : 0.0;
      s->rz = t[0];
      s->rr = t[1];
      if (!isfinite(t[0]) || !isfinite(t[1])) s->status = 1;
    }
  }
}

// p = minv r + beta p
template <typename T>
__global__ void cg_p_kernel(T *__restrict__ p, const T *__restrict__ r,
                            const T *__restrict__ minv, const CgScalars *__restrict__ s,
                            int64_t n) {
  const T beta = (T)s->beta;
  int64_t q0 = 0;
  if constexpr (sizeof(T) == 4) {
    if (aligned16(p, r, minv)) {  // fp32: 16-byte accesses
      using V = float4;
      const int64_t n4 = n / 4;
      for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n4;
           v += (int64_t)gridDim.x * blockDim.x) {
        V pv = reinterpret_cast<V *>(p)[v];
        const V rv = reinterpret_cast<const V *>(r)[v], mv = reinterpret_cast<const V *>(minv)[v];
        pv.x = mv.x * rv.x + beta * pv.x;
        pv.y = mv.y * rv.y + beta * pv.y;
        pv.z = mv.z * rv.z + beta * pv.z;
        pv.w = mv.w * rv.w + beta * pv.w;
        reinterpret_cast<V *>(p)[v] = pv;
      }
      q0 = n4 * 4;
    }
  }
  for (int64_t q = q0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    p[q] = minv[q] * r[q] + beta * p[q];
}

// out = a .* b; out += a
__global__ void mul_kernel(double *__restrict__ out, const double *__restrict__ a,
                           const double *__restrict__ b, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = a[q] * b[q];
}
// out = a .* b where out may alias a or b
__global__ void mul_alias_kernel(double *out, const double *a, const double *b, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = a[q] * b[q];
}
__global__ void add_kernel(double *__restrict__ out, const double *__restrict__ a, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] += a[q];
}

// fp64 -> fp32 / bf16 conversions and the fp64 refinement updates
__global__ void to_f32_kernel(float *__restrict__ out, const double *__restrict__ in, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = (float)in[q];
}
__global__ void to_bf16_kernel(__nv_bfloat16 *__restrict__ out, const double *__restrict__ in,
                               int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = __double2bfloat16(in[q]);
}
// r = mask .* (b - w) (fp64), r32 = fp32(r) scaled by 1/s; partial rr = sum c r^2
__global__ void residual_kernel(double *__restrict__ r, float *__restrict__ r32,
                                const double *__restrict__ b, const double *__restrict__ w,
                                const double *__restrict__ mask, const double *__restrict__ c,
                                double *__restrict__ partials, int64_t n) {
  __shared__ double sh[kRedThreads / 32];
  double a = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double rv = (b[q] - w[q]) * mask[q];
    r[q] = rv;
    r32[q] = (float)rv;
    a += c[q] * rv * rv;
  }
  double v[1] = {a};
  ax::block_sum<1>(v, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}
__global__ void sum_partials_kernel(const double *__restrict__ partials, int nblk,
                                    double *__restrict__ out) {
  ax::warp_sum_partials<1>(partials, nblk, out);
}
// x += d (fp32 correction added in fp64)
__global__ void add_correction_kernel(double *__restrict__ x, const float *__restrict__ d,
                                      int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    x[q] += (double)d[q];
}

inline unsigned blocks_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

// ---------------------------------------------------------------- handle
struct ax_poisson {
  int lx = 0, nelv = 0;
  int64_t n = 0;
  const double *dx = nullptr, *dxt = nullptr, *h1 = nullptr, *g[6] = {};
  const double *mask = nullptr;
  ax_op *op = nullptr;  // the operator (prepared geometry where it applies)
  double *dotp = nullptr;  // per-block partials of p . Ap from the fused apply
  int ndot = 0;            // partials of the fp64 (prepared-geometry) apply
  int ndot32 = 0;          // partials of the fp32 / bf16-data apply
  bool lowp_eo32 = false;  // that apply runs the even-odd fp32 kernel
  float *sqm = nullptr;  // sqrt(minv) in fp32 for the symmetric learned form (lazily)
  double *hb = nullptr;  // h2 .* B of the Helmholtz problem, or null (Poisson)
  float *hb32 = nullptr;  // its fp32 copy for the mixed-precision solves
  ax_gs *gs = nullptr;
  const double *c = nullptr;  // 1/multiplicity (owned by gs)
  // owned fp64 work
  double *minv = nullptr, *cm = nullptr, *w = nullptr, *r = nullptr, *p = nullptr;
  double *partials = nullptr;
  CgScalars *scal = nullptr;
  CgScalars *scal_host = nullptr;  // pinned
  // owned fp32 data of the refinement solve (lazily allocated)
  int lowp_mode = 0;  // 0 none, 1 fp32, 2 bf16 operator data
  float *minv32 = nullptr, *mask32 = nullptr, *x32 = nullptr, *r32 = nullptr, *p32 = nullptr,
        *w32 = nullptr, *q32 = nullptr, *c32 = nullptr, *cm32 = nullptr, *dx32 = nullptr,
        *dxt32 = nullptr;
  void *h1lp = nullptr, *glp[6] = {};
  double *r64 = nullptr;  // outer residual
  int check_every = 1;
  // flexible-CG work (lazily allocated): previous residual, learned correction
  double *r_old = nullptr, *corr = nullptr;
  float *r_old32 = nullptr, *corr32 = nullptr;
};

namespace {

template <typename T>
int alloc(T **p, size_t count) {
  if (cudaMalloc((void **)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
    (void)cudaGetLastError();
    *p = nullptr;
    return AX_ENOMEM;
  }
  return AX_OK;
}

int apply_f64(ax_poisson *P, double *w, const double *u, cudaStream_t st) {
  int rc = ax_op_apply(P->op, w, u, st);
  if (rc == AX_OK && P->hb) rc = ax::mass_add<double>(w, P->hb, u, P->n, nullptr, st);
  if (rc) return rc;
  return ax_gs_sum(P->gs, w, st);
}

// dotp: also the per-block partials of u . Ax (P->ndot32 of them)
// up: the fused direction update (even-odd fp32 kernel only; u = up->pw)
int apply_lowp(ax_poisson *P, float *w, const float *u, cudaStream_t st,
               double *dotp = nullptr, const ax::E32Upd *up = nullptr) {
  int rc;
  if (up && !P->lowp_eo32) return AX_EINVAL;
  if (P->lowp_eo32 && P->lowp_mode == 2) {
    auto b = [](const void *x) { return reinterpret_cast<const __nv_bfloat16 *>(x); };
    const __nv_bfloat16 *g[7] = {b(P->h1lp), b(P->glp[0]), b(P->glp[1]), b(P->glp[2]),
                                 b(P->glp[3]), b(P->glp[4]), b(P->glp[5])};
    rc = ax::dispatch_eo32_f32u_bf16(P->lx, w, u, P->dx32, P->dxt32, g, P->nelv, nullptr, dotp,
                                     st, up);
  } else if (P->lowp_eo32) {
    auto f = [](const void *x) { return reinterpret_cast<const float *>(x); };
    const float *g[7] = {f(P->h1lp), f(P->glp[0]), f(P->glp[1]), f(P->glp[2]),
                         f(P->glp[3]), f(P->glp[4]), f(P->glp[5])};
    rc = ax::dispatch_eo32_f32(P->lx, w, u, P->dx32, P->dxt32, g, P->nelv, nullptr, dotp, st,
                               up);
  } else if (P->lowp_mode == 2) {
    auto b = [](const void *x) { return reinterpret_cast<const __nv_bfloat16 *>(x); };
    // u is fp32: the bf16 mode keeps vectors in fp32 and only G, h1 in bf16
    rc = ax::dispatch_kstep_f32u_bf16(P->lx, w, u, P->dx32, P->dxt32, b(P->h1lp), b(P->glp[0]),
                                      b(P->glp[1]), b(P->glp[2]), b(P->glp[3]), b(P->glp[4]),
                                      b(P->glp[5]), P->nelv, 0, st, dotp);
  } else {
    auto f = [](const void *x) { return reinterpret_cast<const float *>(x); };
    rc = ax::dispatch_kstep_f32(P->lx, w, u, P->dx32, P->dxt32, f(P->h1lp), f(P->glp[0]),
                                f(P->glp[1]), f(P->glp[2]), f(P->glp[3]), f(P->glp[4]),
                                f(P->glp[5]), P->nelv, 0, st, dotp);
  }
  if (rc == AX_OK && P->hb32)  // the mass term's partials follow the kernel's
    rc = ax::mass_add<float>(w, P->hb32, u, P->n, dotp ? dotp + P->ndot32 : nullptr, st);
  if (rc) return rc;
  return ax_gs_sum_f32(P->gs, w, st);
}

// The fused apply of a solver loop: w = gs(Ax(u)) (unmasked) and the
// partials of u . Ax in P->dotp; returns the number of partials, or 0 when
// this precision has no fused form (the caller masks and dots separately).
// (With a mass term its kRedBlocks partials follow the operator's.)
int fused_parts(const ax_poisson *P, const double *) {
  return P->dotp && P->ndot ? P->ndot + (P->hb ? kRedBlocks : 0) : 0;
}
int fused_parts(const ax_poisson *P, const float *) {
  return P->dotp ? P->ndot32 + (P->hb32 ? kRedBlocks : 0) : 0;
}
int mass_fused(ax_poisson *P, double *w, const double *u, cudaStream_t st) {
  return P->hb ? ax::mass_add<double>(w, P->hb, u, P->n, P->dotp + P->ndot, st) : AX_OK;
}
int apply_fused(ax_poisson *P, double *w, const double *u, cudaStream_t st) {
  int rc = ax::op_apply_dot(P->op, w, u, P->dotp, st);
  if (rc == AX_OK) rc = mass_fused(P, w, u, st);
  return rc ? rc : ax_gs_sum(P->gs, w, st);
}
int apply_fused(ax_poisson *P, float *w, const float *u, cudaStream_t st) {
  return apply_lowp(P, w, u, st, P->dotp);
}
// The direction update p = minv r + beta p folded into the apply that reads
// p next (fp64 with prepared geometry); false where no such kernel exists.
bool fuses_update(const ax_poisson *P, const double *) { return P->dotp && P->ndot > 0; }
bool fuses_update(const ax_poisson *P, const float *) { return P->dotp && P->lowp_eo32; }
int apply_fused_update(ax_poisson *P, double *w, double *p, const double *r,
                       const double *minv, const double *beta, cudaStream_t st,
                       const double *corr = nullptr, const int *use_corr = nullptr) {
  int rc = ax::op_update_apply_dot(P->op, w, p, r, minv, beta, P->dotp, st, corr, use_corr);
  if (rc == AX_OK) rc = mass_fused(P, w, p, st);
  return rc ? rc : ax_gs_sum(P->gs, w, st);
}
// fp32 vectors (the refinement's inner CG, even-odd fp32 kernel): the same
// fusion, p = minv .* r + beta p in fp32 inside the apply
int apply_fused_update(ax_poisson *P, float *w, float *p, const float *r, const float *minv,
                       const double *beta, cudaStream_t st, const float *corr = nullptr,
                       const int * = nullptr) {
  if (corr) return AX_EINVAL;  // the flexible loop keeps its own direction kernel
  ax::E32Upd up;
  up.pw = p;
  up.r = r;
  up.minv = minv;
  up.beta = beta;
  return apply_lowp(P, w, p, st, P->dotp, &up);
}

// Generic PCG loop on vectors of type T (fp64 with the fp64 operator, or
// fp32 with the low-precision operator).  x0 = 0.  Returns AX_OK when
// sqrt(rr/rr0) <= tol, AX_ENOTCONV at maxit, AX_EBREAKDOWN on breakdown.
template <typename T, typename Apply>
int pcg_loop(ax_poisson *P, T *x, const T *b, T *r, T *p, T *w, const T *mask, const T *minv,
             const T *c, const T *cm, Apply apply, double tol, int maxit, int *iters,
             double *relres, cudaStream_t st) {
  const int64_t n = P->n;
  const unsigned nb = kRedBlocks;
  cg_init_kernel<T><<<nb, kRedThreads, 0, st>>>(x, r, p, b, mask, minv, c, P->partials, n);
  cg_beta_kernel<<<1, 64, 0, st>>>(P->partials, nb, P->scal, 1);
  if (ax::launch_status()) return AX_ELAUNCH;
  if (cudaMemcpyAsync(P->scal_host, P->scal, sizeof(CgScalars), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return AX_ELAUNCH;
  const double rr0 = P->scal_host->rr0;
  int it = 0;
  double rel = rr0 > 0 ? 1.0 : 0.0;
  if (rr0 == 0.0 || tol >= 1.0) {
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return AX_OK;
  }
  int status = AX_ENOTCONV;
  // fp64 with prepared geometry: p . Ap comes out of the apply itself (for
  // a continuous, masked p the assembled dot equals the element-local sum
  // of p . A_e p), and the mask moves into the update
  const int nparts = fused_parts(P, (const T *)nullptr);
  const bool fused = nparts > 0;
  // after the first iteration the next direction is formed inside the apply
  const bool fused_p = fused && fuses_update(P, (const T *)nullptr);
  while (it < maxit) {
    int rc;
    if (fused) {
      // device address of the beta field (P->scal lives on the device)
      const double *beta_dev = reinterpret_cast<const double *>(
          reinterpret_cast<const char *>(P->scal) + offsetof(CgScalars, beta));
      rc = (fused_p && it > 0) ? apply_fused_update(P, w, p, r, minv, beta_dev, st)
                               : apply_fused(P, w, p, st);
      if (rc) return rc;
      cg_alpha_kernel<<<1, 1024, 0, st>>>(P->dotp, nparts, P->scal);
      // rr only where the host will test it (after this iteration)
      const bool checked = (it + 1) % P->check_every == 0 || it + 1 == maxit;
      if (checked)
        cg_update_kernel<T, true, true><<<nb, kRedThreads, 0, st>>>(x, r, p, w, cm, c, P->scal,
                                                                    P->partials, n);
      else
        cg_update_kernel<T, true, false><<<nb, kRedThreads, 0, st>>>(x, r, p, w, cm, c,
                                                                     P->scal, P->partials, n);
    } else {
      rc = apply(w, p, st);
      if (rc) return rc;
      mask_dot_kernel<T><<<nb, kRedThreads, 0, st>>>(w, p, mask, c, P->partials, n);
      cg_alpha_kernel<<<1, 32, 0, st>>>(P->partials, nb, P->scal);
      cg_update_kernel<T><<<nb, kRedThreads, 0, st>>>(x, r, p, w, cm, c, P->scal, P->partials,
                                                      n);
    }
    cg_beta_kernel<<<1, 64, 0, st>>>(P->partials, nb, P->scal, 0);
    ++it;
    if (it % P->check_every == 0 || it == maxit) {
      if (cudaMemcpyAsync(P->scal_host, P->scal, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                          st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return AX_ELAUNCH;
      if (P->scal_host->status) {
        status = AX_EBREAKDOWN;
        break;
      }
      rel = std::sqrt(std::max(P->scal_host->rr, 0.0) / rr0);
      if (rel <= tol) {
        status = AX_OK;
        break;
      }
    }
    if (!fused_p) cg_p_kernel<T><<<nb, kRedThreads, 0, st>>>(p, r, minv, P->scal, n);
  }
  if (ax::launch_status()) return AX_ELAUNCH;
  if (iters) *iters = it;
  if (relres) *relres = rel;
  return status;
}

int ensure_lowp(ax_poisson *P, int mode, cudaStream_t st) {
  if (P->lowp_mode == mode) return AX_OK;
  if (P->lowp_mode != 0) {  // switch modes: drop the old operator copies
    cudaFree(P->h1lp);
    for (auto &q : P->glp) cudaFree(q), q = nullptr;
    P->h1lp = nullptr;
  }
  const int64_t n = P->n;
  const size_t lx2 = (size_t)P->lx * P->lx;
  int rc = AX_OK;
  if (!P->x32) {
    rc |= alloc(&P->minv32, n) | alloc(&P->mask32, n) | alloc(&P->x32, n) | alloc(&P->r32, n) |
          alloc(&P->p32, n) | alloc(&P->w32, n) | alloc(&P->q32, n) | alloc(&P->c32, n) |
          alloc(&P->cm32, n) | alloc(&P->dx32, lx2) | alloc(&P->dxt32, lx2) | alloc(&P->r64, n);
    if (rc) return AX_ENOMEM;
  }
  const size_t es = mode == 2 ? sizeof(__nv_bfloat16) : sizeof(float);
  if (cudaMalloc(&P->h1lp, n * es) != cudaSuccess) return AX_ENOMEM;
  for (auto &q : P->glp)
    if (cudaMalloc(&q, n * es) != cudaSuccess) return AX_ENOMEM;
  const unsigned nb = kRedBlocks;
  auto conv = [&](void *out, const double *in, int64_t m) {
    if (mode == 2)
      to_bf16_kernel<<<nb, kRedThreads, 0, st>>>((__nv_bfloat16 *)out, in, m);
    else
      to_f32_kernel<<<nb, kRedThreads, 0, st>>>((float *)out, in, m);
  };
  conv(P->h1lp, P->h1, n);
  for (int k = 0; k < 6; ++k) conv(P->glp[k], P->g[k], n);
  to_f32_kernel<<<nb, kRedThreads, 0, st>>>(P->mask32, P->mask, n);
  to_f32_kernel<<<nb, kRedThreads, 0, st>>>(P->minv32, P->minv, n);
  to_f32_kernel<<<nb, kRedThreads, 0, st>>>(P->c32, P->c, n);
  to_f32_kernel<<<nb, kRedThreads, 0, st>>>(P->cm32, P->cm, n);
  to_f32_kernel<<<1, 256, 0, st>>>(P->dx32, P->dx, (int64_t)lx2);
  to_f32_kernel<<<1, 256, 0, st>>>(P->dxt32, P->dxt, (int64_t)lx2);
  if (P->hb) {  // the Helmholtz mass term of the inner operator
    if (!P->hb32 && alloc(&P->hb32, n)) return AX_ENOMEM;
    to_f32_kernel<<<nb, kRedThreads, 0, st>>>(P->hb32, P->hb, n);
  }
  if (ax::launch_status()) return AX_ELAUNCH;
  P->lowp_mode = mode;
  // the even-odd fp32 kernel where it applies (library buffers are aligned),
  // else the k-loop kernel; the fused dot's partial count follows
  const int ne = ax::eo32_lx(P->lx) ? (mode == 2 ? ax::eo32_blocks_f32u_bf16(P->lx, P->nelv)
                                                 : ax::eo32_blocks_f32(P->lx, P->nelv))
                                    : 0;
  P->lowp_eo32 = ne > 0;
  P->ndot32 = ne > 0 ? ne : ax::kstep_blocks(P->lx, P->nelv);
  return AX_OK;
}

}  // namespace

extern "C" {

int ax_poisson_destroy(ax_poisson *P) {
  if (!P) return AX_OK;
  double *d64[] = {P->minv, P->cm, P->w, P->r, P->p, P->partials, P->r64};
  for (double *q : d64) cudaFree(q);
  float *d32[] = {P->minv32, P->mask32, P->x32, P->r32, P->p32, P->w32,
                  P->q32,    P->c32,    P->cm32, P->dx32, P->dxt32};
  for (float *q : d32) cudaFree(q);
  cudaFree(P->h1lp);
  for (void *q : P->glp) cudaFree(q);
  cudaFree(P->r_old);
  cudaFree(P->corr);
  cudaFree(P->r_old32);
  cudaFree(P->corr32);
  if (P->op) ax_op_destroy(P->op);
  cudaFree(P->dotp);
  cudaFree(P->sqm);
  cudaFree(P->hb);
  cudaFree(P->hb32);
  cudaFree(P->scal);
  if (P->scal_host) cudaFreeHost(P->scal_host);
  delete P;
  return AX_OK;
}

int ax_poisson_create(ax_poisson **out, int lx, int nelv, const double *dx, const double *dxt,
                      const double *h1, const double *g11, const double *g22, const double *g33,
                      const double *g12, const double *g13, const double *g23,
                      const double *mask, ax_gs *gs, void *stream) {
  if (!out || !ax::lx_ok(lx) || nelv <= 0 ||
      !ax::all_nonnull(dx, dxt, h1, g11, g22, g33, g12, g13, g23, mask, gs))
    return AX_EINVAL;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  ax_poisson *P = new (std::nothrow) ax_poisson();
  if (!P) return AX_ENOMEM;
  P->lx = lx;
  P->nelv = nelv;
  P->n = (int64_t)nelv * lx * lx * lx;
  P->dx = dx;
  P->dxt = dxt;
  P->h1 = h1;
  const double *gg[6] = {g11, g22, g33, g12, g13, g23};
  for (int k = 0; k < 6; ++k) P->g[k] = gg[k];
  P->mask = mask;
  P->gs = gs;
  P->c = ax_gs_inverse_multiplicity(gs);
  const int64_t n = P->n;
  if (int rco = ax_op_create(&P->op, lx, nelv, dx, dxt, h1, g11, g22, g33, g12, g13, g23,
                             stream)) {
    ax_poisson_destroy(P);
    return rco;
  }
  P->ndot = ax::op_dot_blocks(P->op);
  P->ndot32 = ax::kstep_blocks(lx, nelv);
  // room for the partials of every reduced-precision apply (ensure_lowp
  // picks one)
  int nd32 = P->ndot32;
  if (ax::eo32_lx(lx))
    nd32 = std::max({nd32, ax::eo32_blocks_f32(lx, nelv), ax::eo32_blocks_f32u_bf16(lx, nelv)});
  if (alloc(&P->dotp, (size_t)std::max(P->ndot, nd32) + kRedBlocks)) {
    ax_poisson_destroy(P);
    return AX_ENOMEM;
  }
  int rc = alloc(&P->minv, n) | alloc(&P->cm, n) | alloc(&P->w, n) | alloc(&P->r, n) |
           alloc(&P->p, n) | alloc(&P->partials, 4 * (size_t)kRedBlocks) |
           alloc(&P->scal, 1);
  if (rc == AX_OK && cudaMallocHost((void **)&P->scal_host, sizeof(CgScalars)) != cudaSuccess)
    rc = AX_ENOMEM;
  if (rc) {
    ax_poisson_destroy(P);
    return AX_ENOMEM;
  }
  // exact Jacobi diagonal, assembled, then the masked inverse
  jacobi_diag_kernel<<<blocks_for(n, 256), 256, 0, st>>>(P->w, dx, h1, g11, g22, g33, g12, g13,
                                                         g23, lx, n);
  rc = ax_gs_sum(gs, P->w, st);
  precond_kernel<<<blocks_for(n, 256), 256, 0, st>>>(P->minv, P->cm, P->w, mask, P->c, n);
  if (rc == AX_OK) rc = ax::launch_status();
  if (rc == AX_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = AX_ELAUNCH;
  if (rc) {
    ax_poisson_destroy(P);
    return rc;
  }
  *out = P;
  return AX_OK;
}

int ax_poisson_set_check_every(ax_poisson *P, int every) {
  if (!P || every < 1) return AX_EINVAL;
  P->check_every = every;
  return AX_OK;
}

int ax_poisson_apply(ax_poisson *P, double *w, const double *u, void *stream) {
  if (!P || !w || !u) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = apply_f64(P, w, u, st);
  if (rc) return rc;
  // w = mask .* w (partials discarded)
  mask_dot_kernel<double><<<kRedBlocks, kRedThreads, 0, st>>>(w, u, P->mask, P->c, P->partials,
                                                              P->n);
  return ax::launch_status();
}

int ax_poisson_diag(const ax_poisson *P, double *diag, void *stream) {
  if (!P || !diag) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = P->n;
  jacobi_diag_kernel<<<blocks_for(n, 256), 256, 0, st>>>(diag, P->dx, P->h1, P->g[0], P->g[1],
                                                         P->g[2], P->g[3], P->g[4], P->g[5],
                                                         P->lx, n);
  int rc = ax::launch_status();
  if (rc == AX_OK) rc = ax_gs_sum(P->gs, diag, st);
  return rc;
}

int ax_poisson_set_diag(ax_poisson *P, const double *diag, void *stream) {
  if (!P || !diag) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = P->n;
  precond_kernel<<<blocks_for(n, 256), 256, 0, st>>>(P->minv, P->cm, diag, P->mask, P->c, n);
  if (P->sqm) sqrt_minv_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(P->sqm, P->minv, n);
  if (P->minv32) {  // fp32 copies of the refinement solve, if converted already
    to_f32_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(P->minv32, P->minv, n);
    to_f32_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(P->cm32, P->cm, n);
  }
  return ax::launch_status();
}

int ax_poisson_set_h2(ax_poisson *P, const double *h2, const double *B, void *stream) {
  if (!P || !h2 || !B) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = P->n;
  if (!P->hb && alloc(&P->hb, n)) return AX_ENOMEM;
  mul_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(P->hb, h2, B, n);
  // Jacobi diagonal: the stiffness diagonal plus h2 .* B, assembled
  jacobi_diag_kernel<<<blocks_for(n, 256), 256, 0, st>>>(P->w, P->dx, P->h1, P->g[0], P->g[1],
                                                         P->g[2], P->g[3], P->g[4], P->g[5],
                                                         P->lx, n);
  add_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(P->w, P->hb, n);
  int rc = ax_gs_sum(P->gs, P->w, st);
  if (rc == AX_OK) rc = ax_poisson_set_diag(P, P->w, stream);
  if (rc == AX_OK && P->lowp_mode) {
    if (!P->hb32 && alloc(&P->hb32, n)) return AX_ENOMEM;
    to_f32_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(P->hb32, P->hb, n);
  }
  if (rc == AX_OK) rc = ax::launch_status();
  if (rc == AX_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = AX_ELAUNCH;
  return rc;
}

int ax_poisson_jacobi(const ax_poisson *P, const double **minv) {
  if (!P || !minv) return AX_EINVAL;
  *minv = P->minv;
  return AX_OK;
}

int ax_cg_solve(ax_poisson *P, double *x, const double *b, double tol, int maxit, int *iters,
                double *relres, void *stream) {
  if (!P || !x || !b || maxit < 0 || !(tol >= 0)) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  auto A = [P](double *w, const double *u, cudaStream_t s) { return apply_f64(P, w, u, s); };
  return pcg_loop<double>(P, x, b, P->r, P->p, P->w, P->mask, P->minv, P->c, P->cm, A, tol,
                          maxit, iters, relres, st);
}

int ax_mpcg_solve(ax_poisson *P, int mode, double *x, const double *b, double tol,
                  double inner_tol, int max_outer, int max_inner, int *outer_iters,
                  int *inner_iters, double *relres, void *stream) {
  if (!P || !x || !b || (mode != AX_PREC_F32 && mode != AX_PREC_BF16) || max_outer < 1 ||
      max_inner < 1 || !(tol >= 0) || !(inner_tol > 0))
    return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_lowp(P, mode == AX_PREC_BF16 ? 2 : 1, st);
  if (rc) return rc;
  const int64_t n = P->n;
  const unsigned nb = kRedBlocks;
  double *sc = reinterpret_cast<double *>(P->scal);  // scratch scalar
  auto norm_r = [&](double *out_host) -> int {
    sum_partials_kernel<<<1, 32, 0, st>>>(P->partials, nb, sc);
    if (cudaMemcpyAsync(out_host, sc, sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return AX_ELAUNCH;
    return AX_OK;
  };
  // x = 0; r = mask .* b
  cudaMemsetAsync(x, 0, n * sizeof(double), st);
  cudaMemsetAsync(P->w, 0, n * sizeof(double), st);
  double rr0 = 0.0, rr = 0.0;
  residual_kernel<<<nb, kRedThreads, 0, st>>>(P->r64, P->r32, b, P->w, P->mask, P->c,
                                              P->partials, n);
  if ((rc = norm_r(&rr0))) return rc;
  int outer = 0, inner_total = 0;
  double rel = rr0 > 0 ? 1.0 : 0.0;
  int status = rr0 == 0.0 ? AX_OK : AX_ENOTCONV;
  auto A32 = [P](float *w, const float *u, cudaStream_t s) { return apply_lowp(P, w, u, s); };
  while (status != AX_OK && outer < max_outer) {
    // inner fp32 PCG on A d = r (r32 holds fp32(r))
    int its = 0;
    double irel = 0.0;
    // inner vectors: rhs r32, residual w32, direction p32, operator output q32
    rc = pcg_loop<float>(P, P->x32, P->r32, P->w32, P->p32, P->q32, P->mask32, P->minv32,
                         P->c32, P->cm32, A32, inner_tol, max_inner, &its, &irel, st);
    inner_total += its;
    if (rc != AX_OK && rc != AX_ENOTCONV) return rc;
    add_correction_kernel<<<nb, kRedThreads, 0, st>>>(x, P->x32, n);
    ++outer;
    // fp64 residual r = mask .* (b - A x)
    if ((rc = apply_f64(P, P->w, x, st))) return rc;
    residual_kernel<<<nb, kRedThreads, 0, st>>>(P->r64, P->r32, b, P->w, P->mask, P->c,
                                                P->partials, n);
    if ((rc = norm_r(&rr))) return rc;
    rel = std::sqrt(std::max(rr, 0.0) / rr0);
    if (!std::isfinite(rel)) return AX_EBREAKDOWN;
    if (rel <= tol) status = AX_OK;
  }
  if (outer_iters) *outer_iters = outer;
  if (inner_iters) *inner_iters = inner_total;
  if (relres) *relres = rel;
  return status;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free Jacobi refresh.
//
// Some callers must not allocate device memory at the point where they need
// the preconditioner: code that records work into a CUDA graph or runs
// inside a time-stepping loop with a fixed memory budget, or a host
// framework that owns every device allocation through its own pool.  When
// such a caller changes h1 (a variable coefficient) it still needs a fresh
// masked inverse Jacobi diagonal.  ax_poisson_create computes one, but it
// allocates; ax_jacobi_noalloc computes the same array into caller memory
// with its scratch (the un-assembled diagonal) in the fixed device array
// below, so it performs no allocation at all.
//
// The scratch holds at most AX_NOALLOC_MAX_POINTS doubles (4 MiB).  It is a
// file-scope __device__ array, so every GPU that loads this library keeps
// those 4 MiB reserved until the process exits.  Every call on a device
// shares the one array, and it keeps the previous call's contents; the
// kernel overwrites all n entries it later reads, so nothing needs clearing.
// Calls whose work overlaps on the GPU (two streams, or two host threads)
// race on the array and must be serialised by the caller.
// ---------------------------------------------------------------------------
#include <mutex>

#include <cuda.h>

static __device__ __align__(256) double g_noalloc_diag[AX_NOALLOC_MAX_POINTS];

namespace {

__global__ void noalloc_minv_kernel(double *__restrict__ minv, const double *__restrict__ diag,
                                    const double *__restrict__ mask, int64_t n) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  minv[q] = (mask[q] != 0.0 && diag[q] != 0.0) ? 1.0 / diag[q] : 0.0;
}

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
// Device address of the array per device, and the context it was resolved
// in: a context created after cudaDeviceReset may hold the module at another
// address, so the address is resolved again when the context changes.
double *g_noalloc_ptr[kNoallocMaxDevices];
unsigned long long g_noalloc_ctx[kNoallocMaxDevices];

// Id of the current context through the driver's entry points (cuCtxGetCurrent,
// cuCtxGetId; no link against the driver library); 0 when unavailable, in
// which case the address is resolved on every call.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static GetCurrent get_current = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      f = nullptr;
    (void)cudaGetLastError();
    return reinterpret_cast<GetCurrent>(f);
  }();
  static GetId get_id = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      f = nullptr;
    (void)cudaGetLastError();
    return reinterpret_cast<GetId>(f);
  }();
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c ||
      get_id(c, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch array on the current device (host code
// cannot use the symbol itself as an address): resolved once per device and
// context.
int noalloc_scratch(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  if (dev < 0 || dev >= kNoallocMaxDevices) return AX_EINVAL;
  // a runtime call makes sure the device's primary context is current
  if (cudaFree(nullptr) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev] || ctx == 0 || g_noalloc_ctx[dev] != ctx) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_diag) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return AX_ELAUNCH;
    }
    g_noalloc_ptr[dev] = static_cast<double *>(p);
    g_noalloc_ctx[dev] = ctx;
  }
  *out = g_noalloc_ptr[dev];
  return AX_OK;
}

}  // namespace

extern "C" int ax_gs_info(const ax_gs *g, int64_t *n_local, int64_t *n_shared,
                          int64_t *n_copies);

extern "C" int ax_jacobi_noalloc(double *minv, const double *dx, const double *h1,
                                 const double *g11, const double *g22, const double *g33,
                                 const double *g12, const double *g13, const double *g23,
                                 const double *mask, ax_gs *gs, int lx, int nelv, void *stream) {
  if (!ax::lx_ok(lx) || nelv < 0) return AX_EINVAL;
  const int64_t n = (int64_t)nelv * lx * lx * lx;
  if (n > AX_NOALLOC_MAX_POINTS) return AX_EINVAL;  // larger than the fixed scratch
  if (n == 0) return AX_OK;
  if (!ax::all_nonnull(minv, dx, h1, g11, g22, g33, g12, g13, g23, mask, gs)) return AX_EINVAL;
  int64_t n_gs = -1;
  if (ax_gs_info(gs, &n_gs, nullptr, nullptr) != AX_OK || n_gs != n) return AX_EINVAL;
  double *scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  jacobi_diag_kernel<<<blocks_for(n, 256), 256, 0, st>>>(scratch, dx, h1, g11, g22, g33, g12,
                                                         g13, g23, lx, n);
  if ((rc = ax::launch_status())) return rc;
  if ((rc = ax_gs_sum(gs, scratch, st))) return rc;
  noalloc_minv_kernel<<<blocks_for(n, 256), 256, 0, st>>>(minv, scratch, mask, n);
  return ax::launch_status();
}

// ---------------------------------------------------------------------------
// Flexible CG with the learned element preconditioner.
//
//   z = minv .* r + corr,   corr = gs(mask .* (1/mult) .* s_e * MLP(x_e))
//
// (mlp.cu).  A nonlinear preconditioner needs the flexible form of CG:
// beta_k = <z_{k+1}, r_{k+1} - r_k> / <z_k, r_k> (Notay 2000, "Flexible
// conjugate gradients").  If <r, z> is not positive or not finite the step
// falls back to z = minv .* r (counted); with no network every step is the
// Jacobi step.  All decisions are taken on the device; the host only reads
// the residual norm every check_every iterations.
// ---------------------------------------------------------------------------
namespace {

// x += alpha p; r_old = r; r -= alpha w; partial rr = sum c r^2.  MASKW: w is
// not masked yet (fused apply); rows where cm = c * minv is 0 keep r = 0.
// RR: the rr partials (read by the host's convergence test only); without
// it the kernel neither reads c nor reduces.
template <typename T, bool MASKW = false, bool RR = true>
__global__ void fcg_update_kernel(T *__restrict__ x, T *__restrict__ r, T *__restrict__ r_old,
                                  const T *__restrict__ p, const T *__restrict__ w,
                                  const T *__restrict__ c, const T *__restrict__ cm,
                                  const CgScalars *__restrict__ s,
                                  double *__restrict__ partials, int64_t n) {
  __shared__ double sh[kRedThreads / 32];
  const T alpha = (T)s->alpha;
  T a_rr = 0;
  auto point = [&](T &xq, T &rq, T &roq, T pq, T wq, T cq, T cmq) {
    xq += alpha * pq;
    roq = rq;
    rq = (MASKW && cmq == T(0)) ? rq : rq - alpha * wq;
    if constexpr (RR) a_rr += cq * rq * rq;
  };
  int64_t q0 = 0;
  if constexpr (sizeof(T) == 4) {
    if (aligned16(x, r, r_old, p, w, c, cm)) {  // fp32: 16-byte accesses
      using V = float4;
      const int64_t n4 = n / 4;
      for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n4;
           v += (int64_t)gridDim.x * blockDim.x) {
        V xv = reinterpret_cast<V *>(x)[v], rv = reinterpret_cast<V *>(r)[v], ov;
        const V pv = reinterpret_cast<const V *>(p)[v], wv = reinterpret_cast<const V *>(w)[v];
        const V cv = RR ? reinterpret_cast<const V *>(c)[v] : V{0.f, 0.f, 0.f, 0.f};
        const V mv = MASKW ? reinterpret_cast<const V *>(cm)[v] : V{1.f, 1.f, 1.f, 1.f};
        point(xv.x, rv.x, ov.x, pv.x, wv.x, cv.x, mv.x);
        point(xv.y, rv.y, ov.y, pv.y, wv.y, cv.y, mv.y);
        point(xv.z, rv.z, ov.z, pv.z, wv.z, cv.z, mv.z);
        point(xv.w, rv.w, ov.w, pv.w, wv.w, cv.w, mv.w);
        reinterpret_cast<V *>(x)[v] = xv;
        reinterpret_cast<V *>(r)[v] = rv;
        reinterpret_cast<V *>(r_old)[v] = ov;
      }
      q0 = n4 * 4;
    }
  } else {
    if (aligned16(x, r, r_old, p, w, c, cm)) {  // fp64: 16-byte accesses, two points each
      using V = double2;
      const int64_t n2 = n / 2;
      for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n2;
           v += (int64_t)gridDim.x * blockDim.x) {
        V xv = reinterpret_cast<V *>(x)[v], rv = reinterpret_cast<V *>(r)[v], ov;
        const V pv = reinterpret_cast<const V *>(p)[v], wv = reinterpret_cast<const V *>(w)[v];
        const V cv = RR ? reinterpret_cast<const V *>(c)[v] : V{0.0, 0.0};
        const V mv = MASKW ? reinterpret_cast<const V *>(cm)[v] : V{1.0, 1.0};
        point(xv.x, rv.x, ov.x, pv.x, wv.x, cv.x, mv.x);
        point(xv.y, rv.y, ov.y, pv.y, wv.y, cv.y, mv.y);
        reinterpret_cast<V *>(x)[v] = xv;
        reinterpret_cast<V *>(r)[v] = rv;
        reinterpret_cast<V *>(r_old)[v] = ov;
      }
      q0 = n2 * 2;
    }
  }
  for (int64_t q = q0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    point(x[q], r[q], r_old[q], p[q], w[q], RR ? c[q] : T(0), MASKW ? cm[q] : T(1));
  if constexpr (RR) {
    double v[1] = {(double)a_rr};
    ax::block_sum<1>(v, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
  }
}

// partials of <zj, r>, <corr, r>, <zj, r_old>, <corr, r_old> (zj = minv r),
// weighted by c; with cm = c * minv the Jacobi pair costs 3 multiply-adds and
// the correction pair 3 more (the fp64 pipe, not memory, bounds this kernel)
template <typename T>
__global__ void fcg_dots_kernel(const T *__restrict__ r, const T *__restrict__ r_old,
                                const T *__restrict__ corr, const T *__restrict__ cm,
                                const T *__restrict__ c, int have_corr,
                                double *__restrict__ partials, int64_t n) {
  __shared__ double sh[4 * kRedThreads / 32];
  T d0 = 0, d1 = 0, d2 = 0, d3 = 0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const T rv = r[q], ro = r_old[q];
    const T a = cm[q] * rv;
    d0 += a * rv;
    d2 += a * ro;
    if (have_corr) {
      const T e = c[q] * corr[q];
      d1 += e * rv;
      d3 += e * ro;
    }
  }
  double v[4] = {(double)d0, (double)d1, (double)d2, (double)d3};
  ax::block_sum<4>(v, sh);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) partials[k * gridDim.x + blockIdx.x] = v[k];
}

// first: rz from <z0, r0>; otherwise Notay's beta; choose learned or Jacobi
__global__ void fcg_beta_kernel(const double *__restrict__ partials, int nblk,
                                CgScalars *__restrict__ s, int first, int have_corr) {
  __shared__ double t[4];
  ax::warp_sum_partials<4>(partials, nblk, t);
  __syncthreads();
  if (threadIdx.x == 0) {
    const double rz_l = t[0] + t[1], rz_j = t[0];
    const double num_l = rz_l - (t[2] + t[3]), num_j = t[0] - t[2];
    const bool ok_l = have_corr && rz_l > 0.0 && isfinite(rz_l) && isfinite(num_l);
    if (have_corr && !ok_l) s->fallbacks += 1;
    const double rz = ok_l ? rz_l : rz_j;
    const double num = ok_l ? num_l : num_j;
    s->use_corr = ok_l ? 1 : 0;
    if (first) {
      s->beta = 0.0;
    } else {
      s->beta = (s->rz != 0.0) ? num / s->rz : 0.0;
    }
    s->rz = rz;
    if (!isfinite(rz)) s->status = 1;
  }
}

// p = minv r + use_corr * corr + beta p   (first: p = z)
template <typename T>
__global__ void fcg_p_kernel(T *__restrict__ p, const T *__restrict__ r,
                             const T *__restrict__ minv, const T *__restrict__ corr,
                             const CgScalars *__restrict__ s, int first, int64_t n) {
  const T beta = first ? T(0) : (T)s->beta;
  const bool uc = s->use_corr != 0;
  // explicit roundings: the Jacobi-only step is the same bits whether or not
  // a (zero) correction is present
  auto point = [&](T &pq, T mq, T rq, T cq) {
    T z = ax::mul_rn(mq, rq);
    if (uc) z = ax::add_rn(z, cq);
    pq = first ? z : ax::fma_rn(beta, pq, z);
  };
  int64_t q0 = 0;
  if constexpr (sizeof(T) == 4) {
    if (aligned16(p, r, minv, corr)) {  // fp32: 16-byte accesses
      using V = float4;
      const int64_t n4 = n / 4;
      for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n4;
           v += (int64_t)gridDim.x * blockDim.x) {
        V pv = first ? V{} : reinterpret_cast<V *>(p)[v];
        const V rv = reinterpret_cast<const V *>(r)[v], mv = reinterpret_cast<const V *>(minv)[v];
        const V cv = uc ? reinterpret_cast<const V *>(corr)[v] : V{};
        point(pv.x, mv.x, rv.x, cv.x);
        point(pv.y, mv.y, rv.y, cv.y);
        point(pv.z, mv.z, rv.z, cv.z);
        point(pv.w, mv.w, rv.w, cv.w);
        reinterpret_cast<V *>(p)[v] = pv;
      }
      q0 = n4 * 4;
    }
  }
  for (int64_t q = q0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    T pq = first ? T(0) : p[q];
    point(pq, minv[q], r[q], uc ? corr[q] : T(0));
    p[q] = pq;
  }
}

// init: x = 0, r = mask b, partial rr
template <typename T>
__global__ void fcg_init_kernel(T *__restrict__ x, T *__restrict__ r, T *__restrict__ r_old,
                                const T *__restrict__ b, const T *__restrict__ mask,
                                const T *__restrict__ c, double *__restrict__ partials,
                                int64_t n) {
  __shared__ double sh[kRedThreads / 32];
  T a = 0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const T rv = b[q] * mask[q];
    x[q] = T(0);
    r[q] = rv;
    r_old[q] = T(0);
    a += c[q] * rv * rv;
  }
  double v[1] = {(double)a};
  ax::block_sum<1>(v, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

__global__ void fcg_rr_kernel(const double *__restrict__ partials, int nblk,
                              CgScalars *__restrict__ s, int first) {
  __shared__ double t[1];
  ax::warp_sum_partials<1>(partials, nblk, t);
  __syncthreads();
  if (threadIdx.x == 0) {
    s->rr = t[0];
    if (first) {
      s->rr0 = t[0];
      s->status = 0;
      s->fallbacks = 0;
      s->use_corr = 0;
    }
  }
}

template <typename T>
int gs_sum_t(ax_gs *g, T *v, cudaStream_t st);
template <>
int gs_sum_t<double>(ax_gs *g, double *v, cudaStream_t st) {
  return ax_gs_sum(g, v, st);
}
template <>
int gs_sum_t<float>(ax_gs *g, float *v, cudaStream_t st) {
  return ax_gs_sum_f32(g, v, st);
}

// Flexible PCG loop (x0 = 0) with the learned correction when M != NULL.
template <typename T, typename Apply>
int fcg_loop(ax_poisson *P, const ax_mlp *M, T *x, const T *b, T *r, T *r_old, T *p, T *w,
             T *corr, const T *mask, const T *minv, const T *c, const T *cm, Apply apply,
             double tol, int maxit, int *iters, double *relres, int *fallbacks,
             cudaStream_t st) {
  const int64_t n = P->n;
  const unsigned nb = kRedBlocks;
  const int have = M != nullptr;
  // fp64 with prepared geometry: after the first step the direction update
  // p = z + beta p (+ the learned correction) runs inside the next apply (see
  // pcg_loop); the fp32 flexible loop keeps its direction kernel
  const bool fused_p = std::is_same_v<T, double> && fused_parts(P, (const T *)nullptr) > 0 &&
                       fuses_update(P, (const T *)nullptr);
  auto precondition = [&](int first) -> int {
    if (have) {
      int rc = ax::mlp_correction<T>(M, corr, r, minv, mask, c, P->nelv, st,
                                     M->arch == AX_MLP_SYM ? P->sqm : nullptr);
      if (rc) return rc;
      if ((rc = gs_sum_t<T>(P->gs, corr, st))) return rc;
    }
    fcg_dots_kernel<T><<<nb, kRedThreads, 0, st>>>(r, r_old, corr, cm, c, have, P->partials,
                                                   n);
    fcg_beta_kernel<<<1, 128, 0, st>>>(P->partials, nb, P->scal, first, have);
    if (first || !fused_p)
      fcg_p_kernel<T><<<nb, kRedThreads, 0, st>>>(p, r, minv, corr, P->scal, first, n);
    return ax::launch_status();
  };
  const char *scal_bytes = reinterpret_cast<const char *>(P->scal);
  const double *beta_dev =
      reinterpret_cast<const double *>(scal_bytes + offsetof(CgScalars, beta));
  const int *use_corr_dev = reinterpret_cast<const int *>(scal_bytes + offsetof(CgScalars, use_corr));
  auto read_scalars = [&]() -> int {
    if (cudaMemcpyAsync(P->scal_host, P->scal, sizeof(CgScalars), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return AX_ELAUNCH;
    return AX_OK;
  };
  fcg_init_kernel<T><<<nb, kRedThreads, 0, st>>>(x, r, r_old, b, mask, c, P->partials, n);
  fcg_rr_kernel<<<1, 32, 0, st>>>(P->partials, nb, P->scal, 1);
  int rc = precondition(1);
  if (rc) return rc;
  if ((rc = read_scalars())) return rc;
  const double rr0 = P->scal_host->rr0;
  double rel = rr0 > 0 ? 1.0 : 0.0;
  int it = 0, status = AX_ENOTCONV;
  if (rr0 == 0.0 || tol >= 1.0) status = AX_OK;
  // fp64 with prepared geometry: p . Ap from the apply itself (see pcg_loop)
  const int nparts = fused_parts(P, (const T *)nullptr);
  const bool fused = nparts > 0;
  int applied = 0;  // applies so far: the first uses the p formed above
  while (status != AX_OK && it < maxit) {
    const bool checked = (it + 1) % P->check_every == 0 || it + 1 == maxit;
    if (fused) {
      rc = (fused_p && applied > 0)
               ? apply_fused_update(P, w, p, r, minv, beta_dev, st, corr, use_corr_dev)
               : apply_fused(P, w, p, st);
      ++applied;
      if (rc) return rc;
      cg_alpha_kernel<<<1, 1024, 0, st>>>(P->dotp, nparts, P->scal);
      // rr only where the host will test it (after this iteration)
      if (checked)
        fcg_update_kernel<T, true, true><<<nb, kRedThreads, 0, st>>>(x, r, r_old, p, w, c, cm,
                                                                     P->scal, P->partials, n);
      else
        fcg_update_kernel<T, true, false><<<nb, kRedThreads, 0, st>>>(x, r, r_old, p, w, c, cm,
                                                                      P->scal, P->partials, n);
    } else {
      if ((rc = apply(w, p, st))) return rc;
      mask_dot_kernel<T><<<nb, kRedThreads, 0, st>>>(w, p, mask, c, P->partials, n);
      cg_alpha_kernel<<<1, 32, 0, st>>>(P->partials, nb, P->scal);
      fcg_update_kernel<T><<<nb, kRedThreads, 0, st>>>(x, r, r_old, p, w, c, cm, P->scal,
                                                       P->partials, n);
    }
    if (checked || !fused) fcg_rr_kernel<<<1, 32, 0, st>>>(P->partials, nb, P->scal, 0);
    ++it;
    if (it % P->check_every == 0 || it == maxit) {
      if ((rc = read_scalars())) return rc;
      if (P->scal_host->status) {
        status = AX_EBREAKDOWN;
        break;
      }
      rel = std::sqrt(std::max(P->scal_host->rr, 0.0) / rr0);
      if (rel <= tol) {
        status = AX_OK;
        break;
      }
    }
    if ((rc = precondition(0))) return rc;
  }
  if ((rc = read_scalars())) return rc;
  if (iters) *iters = it;
  if (relres) *relres = rel;
  if (fallbacks) *fallbacks = P->scal_host->fallbacks;
  return status;
}

int ensure_sqm(ax_poisson *P, cudaStream_t st) {
  if (P->sqm) return AX_OK;
  if (alloc(&P->sqm, P->n)) return AX_ENOMEM;
  sqrt_minv_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(P->sqm, P->minv, P->n);
  return ax::launch_status();
}

int ensure_fcg64(ax_poisson *P, cudaStream_t st) {
  if (int rc = ensure_sqm(P, st)) return rc;
  if (P->r_old) return AX_OK;
  return alloc(&P->r_old, P->n) | alloc(&P->corr, P->n) ? AX_ENOMEM : AX_OK;
}

}  // namespace

extern "C" int ax_fcg_solve(ax_poisson *P, const ax_mlp *M, double *x, const double *b,
                            double tol, int maxit, int *iters, double *relres, int *fallbacks,
                            void *stream) {
  if (!P || !x || !b || maxit < 0 || !(tol >= 0)) return AX_EINVAL;
  if (M && M->n_in != P->lx * P->lx * P->lx) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_fcg64(P, st);
  if (rc) return rc;
  auto A = [P](double *w, const double *u, cudaStream_t s) { return apply_f64(P, w, u, s); };
  return fcg_loop<double>(P, M, x, b, P->r, P->r_old, P->p, P->w, P->corr, P->mask, P->minv,
                          P->c, P->cm, A, tol, maxit, iters, relres, fallbacks, st);
}

extern "C" int ax_precondition(ax_poisson *P, const ax_mlp *M, double *z, const double *r,
                               void *stream) {
  if (!P || !z || !r) return AX_EINVAL;
  if (M && M->n_in != P->lx * P->lx * P->lx) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_fcg64(P, st);
  if (rc) return rc;
  if (M) {
    if ((rc = ax::mlp_correction<double>(M, P->corr, r, P->minv, P->mask, P->c, P->nelv, st,
                                        M->arch == AX_MLP_SYM ? P->sqm : nullptr)))
      return rc;
    if ((rc = ax_gs_sum(P->gs, P->corr, st))) return rc;
  }
  // z = minv r (+ corr): reuse the p-update kernel with beta = 0 (first = 1)
  cudaMemsetAsync(P->scal, 0, sizeof(CgScalars), st);
  if (M) {
    const int one = 1;
    cudaMemcpyAsync(&P->scal->use_corr, &one, sizeof(int), cudaMemcpyHostToDevice, st);
  }
  fcg_p_kernel<double><<<kRedBlocks, kRedThreads, 0, st>>>(z, r, P->minv, P->corr, P->scal, 1,
                                                           P->n);
  rc = ax::launch_status();
  if (rc == AX_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = AX_ELAUNCH;
  return rc;
}

extern "C" int ax_mpfcg_solve(ax_poisson *P, const ax_mlp *M, int mode, double *x,
                              const double *b, double tol, double inner_tol, int max_outer,
                              int max_inner, int *outer_iters, int *inner_iters, double *relres,
                              int *fallbacks, void *stream) {
  if (!P || !x || !b || (mode != AX_PREC_F32 && mode != AX_PREC_BF16) || max_outer < 1 ||
      max_inner < 1 || !(tol >= 0) || !(inner_tol > 0))
    return AX_EINVAL;
  if (M && M->n_in != P->lx * P->lx * P->lx) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_lowp(P, mode == AX_PREC_BF16 ? 2 : 1, st);
  if (rc) return rc;
  if (!P->r_old32 && (alloc(&P->r_old32, P->n) | alloc(&P->corr32, P->n))) return AX_ENOMEM;
  if ((rc = ensure_sqm(P, st))) return rc;
  const int64_t n = P->n;
  const unsigned nb = kRedBlocks;
  double *sc = reinterpret_cast<double *>(P->scal);
  auto norm_r = [&](double *out_host) -> int {
    sum_partials_kernel<<<1, 32, 0, st>>>(P->partials, nb, sc);
    if (cudaMemcpyAsync(out_host, sc, sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return AX_ELAUNCH;
    return AX_OK;
  };
  cudaMemsetAsync(x, 0, n * sizeof(double), st);
  cudaMemsetAsync(P->w, 0, n * sizeof(double), st);
  double rr0 = 0.0, rr = 0.0;
  residual_kernel<<<nb, kRedThreads, 0, st>>>(P->r64, P->r32, b, P->w, P->mask, P->c,
                                              P->partials, n);
  if ((rc = norm_r(&rr0))) return rc;
  int outer = 0, inner_total = 0, fb_total = 0;
  double rel = rr0 > 0 ? 1.0 : 0.0;
  int status = rr0 == 0.0 ? AX_OK : AX_ENOTCONV;
  auto A32 = [P](float *w, const float *u, cudaStream_t s) { return apply_lowp(P, w, u, s); };
  while (status != AX_OK && outer < max_outer) {
    int its = 0, fb = 0;
    double irel = 0.0;
    rc = fcg_loop<float>(P, M, P->x32, P->r32, P->w32, P->r_old32, P->p32, P->q32, P->corr32,
                         P->mask32, P->minv32, P->c32, P->cm32, A32, inner_tol, max_inner, &its,
                         &irel, &fb, st);
    inner_total += its;
    fb_total += fb;
    if (rc != AX_OK && rc != AX_ENOTCONV) return rc;
    add_correction_kernel<<<nb, kRedThreads, 0, st>>>(x, P->x32, n);
    ++outer;
    if ((rc = apply_f64(P, P->w, x, st))) return rc;
    residual_kernel<<<nb, kRedThreads, 0, st>>>(P->r64, P->r32, b, P->w, P->mask, P->c,
                                                P->partials, n);
    if ((rc = norm_r(&rr))) return rc;
    rel = std::sqrt(std::max(rr, 0.0) / rr0);
    if (!std::isfinite(rel)) return AX_EBREAKDOWN;
    if (rel <= tol) status = AX_OK;
  }
  if (outer_iters) *outer_iters = outer;
  if (inner_iters) *inner_iters = inner_total;
  if (relres) *relres = rel;
  if (fallbacks) *fallbacks = fb_total;
  return status;
}

// y = a x + b y on device vectors (training-data preparation and utilities).
namespace {
__global__ void axpby_kernel(double *__restrict__ y, double a, const double *__restrict__ x,
                             double b, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    y[q] = a * x[q] + b * y[q];
}
}  // namespace

extern "C" int ax_axpby(double *y, double a, const double *x, double b, int64_t n,
                        void *stream) {
  if (n < 0 || (n > 0 && (!y || !x))) return AX_EINVAL;
  if (n == 0) return AX_OK;
  axpby_kernel<<<kRedBlocks, kRedThreads, 0, (cudaStream_t)stream>>>(y, a, x, b, n);
  return ax::launch_status();
}

// ---------------------------------------------------------------------------
// Energy-norm training of the learned preconditioner.
//
// For CG iterates with residual r_k and error e_k the network is trained to
// make z(r_k) = minv .* r_k + corr(r_k) close to e_k in the energy norm,
//   L_k = ||e_k - z(r_k)||_A^2 / ||e_k||_A^2,
// the norm in which CG measures error.  Every element of the mesh is one
// training row (so each step uses nelv residual/error element pairs).  With
// d = e - z and q = mask .* gs(A_L d) the gradient with respect to the
// network output of element e is dL/dy_e = -2 mask .* c .* s_e .* q_e / ||e||_A^2
// (gs is self-adjoint, so the adjoint of z = gs(W y) is W gs(.)).
// ---------------------------------------------------------------------------
namespace {

__global__ void energy_features_kernel(float *__restrict__ X, double *__restrict__ s_out,
                                       const double *__restrict__ r,
                                       const double *__restrict__ minv, int N, int sym) {
  __shared__ double sh[kRedThreads / 32];
  __shared__ double s_b;
  const size_t base = (size_t)blockIdx.x * N;
  double ss = 0.0;
  auto scale = [&](double mv) { return sym ? sqrt(mv) : mv; };
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const double z = scale(minv[base + k]) * r[base + k];
    ss += z * z;
  }
  double v[1] = {ss};
  ax::block_sum<1>(v, sh);
  if (threadIdx.x == 0) {
    s_b = sqrt(v[0]);
    s_out[blockIdx.x] = s_b;
  }
  __syncthreads();
  const double inv = s_b > 0.0 ? 1.0 / s_b : 0.0;
  for (int k = threadIdx.x; k < N; k += blockDim.x)
    X[base + k] = (float)(scale(minv[base + k]) * r[base + k] * inv);
}

// d = e - minv r - corr, with corr = mask c s_e Y (corr assembled by gs before)
// output scale of the correction: 1/multiplicity (tanh form) or sqrt(minv)
// (symmetric form)
__device__ __forceinline__ double energy_out_scale(const double *c, const double *minv,
                                                   int64_t q, int sym) {
  return sym ? sqrt(minv[q]) : c[q];
}

__global__ void energy_corr_kernel(double *__restrict__ corr, const float *__restrict__ Y,
                                   const double *__restrict__ s, const double *__restrict__ mask,
                                   const double *__restrict__ c, const double *__restrict__ minv,
                                   int sym, int N, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    corr[q] = mask[q] * energy_out_scale(c, minv, q, sym) * s[q / N] * (double)Y[q];
}

__global__ void energy_diff_kernel(double *__restrict__ d, const double *__restrict__ e,
                                   const double *__restrict__ r, const double *__restrict__ minv,
                                   const double *__restrict__ corr, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    d[q] = e[q] - minv[q] * r[q] - corr[q];
}

__global__ void energy_dy_kernel(float *__restrict__ dY, const double *__restrict__ q,
                                 const double *__restrict__ s, const double *__restrict__ mask,
                                 const double *__restrict__ c, const double *__restrict__ minv,
                                 int sym, const double *__restrict__ eA, int N, int64_t n) {
  const double scale = eA[0] > 0.0 ? -2.0 / eA[0] : 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    dY[p] = (float)(scale * mask[p] * energy_out_scale(c, minv, p, sym) * s[p / N] * q[p]);
}

__global__ void store_partial_sum_kernel(const double *__restrict__ partials, int nblk,
                                         double *__restrict__ out) {
  ax::warp_sum_partials<1>(partials, nblk, out);
}

}  // namespace

extern "C" int ax_mlp_train_energy(ax_poisson *P, ax_mlp *M, const double *r_set,
                                   const double *e_set, int K, int epochs, float lr,
                                   double *final_loss, void *stream) {
  if (!P || !M || !r_set || !e_set || K < 1 || epochs < 1 || !(lr > 0)) return AX_EINVAL;
  const int N = P->lx * P->lx * P->lx;
  if (M->n_in != N) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = P->n;
  const unsigned nb = kRedBlocks;
  int rc = ax::mlp_reserve(M, P->nelv);
  if (rc) return rc;
  double *s = nullptr, *d = nullptr, *q = nullptr, *corr = nullptr, *eA = nullptr, *Lk = nullptr;
  rc = alloc(&s, P->nelv) | alloc(&d, n) | alloc(&q, n) | alloc(&corr, n) | alloc(&eA, K) |
       alloc(&Lk, K);
  auto cleanup = [&]() {
    cudaFree(s);
    cudaFree(d);
    cudaFree(q);
    cudaFree(corr);
    cudaFree(eA);
    cudaFree(Lk);
  };
  if (rc) {
    cleanup();
    return AX_ENOMEM;
  }
  // ||e_k||_A^2 once per pair
  for (int k = 0; k < K && rc == AX_OK; ++k) {
    const double *e = e_set + (size_t)k * n;
    rc = apply_f64(P, q, e, st);
    if (rc) break;
    mask_dot_kernel<double><<<nb, kRedThreads, 0, st>>>(q, e, P->mask, P->c, P->partials, n);
    store_partial_sum_kernel<<<1, 32, 0, st>>>(P->partials, nb, eA + k);
  }
  for (int ep = 0; ep < epochs && rc == AX_OK; ++ep) {
    for (int k = 0; k < K && rc == AX_OK; ++k) {
      const double *r = r_set + (size_t)k * n, *e = e_set + (size_t)k * n;
      const int sym = M->arch == AX_MLP_SYM;
      energy_features_kernel<<<P->nelv, kRedThreads, 0, st>>>(M->X, s, r, P->minv, N, sym);
      if ((rc = ax::mlp_train_forward(M, P->nelv, st))) break;
      energy_corr_kernel<<<nb, kRedThreads, 0, st>>>(corr, M->Y, s, P->mask, P->c, P->minv, sym,
                                                     N, n);
      if ((rc = ax_gs_sum(P->gs, corr, st))) break;
      energy_diff_kernel<<<nb, kRedThreads, 0, st>>>(d, e, r, P->minv, corr, n);
      if ((rc = apply_f64(P, q, d, st))) break;
      mask_dot_kernel<double><<<nb, kRedThreads, 0, st>>>(q, d, P->mask, P->c, P->partials, n);
      store_partial_sum_kernel<<<1, 32, 0, st>>>(P->partials, nb, Lk + k);
      energy_dy_kernel<<<nb, kRedThreads, 0, st>>>(M->dY, q, s, P->mask, P->c, P->minv, sym,
                                                   eA + k, N, n);
      if ((rc = ax::mlp_train_backward(M, P->nelv, st))) break;
      if (sym && (rc = ax::mlp_tie_grad(M, st))) break;
      if ((rc = ax::mlp_adam_step(M, lr, st))) break;
      if (sym && (rc = ax::mlp_tie_params(M, st))) break;
    }
  }
  if (rc == AX_OK) rc = ax::mlp_refresh(M, st);
  std::vector<double> hl(K), he(K);
  if (rc == AX_OK &&
      (cudaMemcpyAsync(hl.data(), Lk, K * sizeof(double), cudaMemcpyDeviceToHost, st) !=
           cudaSuccess ||
       cudaMemcpyAsync(he.data(), eA, K * sizeof(double), cudaMemcpyDeviceToHost, st) !=
           cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = AX_ELAUNCH;
  if (rc == AX_OK && final_loss) {
    double m = 0.0;
    for (int k = 0; k < K; ++k) m += he[k] > 0 ? hl[k] / he[k] : 0.0;
    *final_loss = m / K;  // mean relative energy error of the last epoch
  }
  cleanup();
  return rc;
}

extern "C" int ax_poisson_rhs(ax_poisson *P, const double *B, const double *f, double *b,
                              void *stream) {
  if (!P || !B || !f || !b) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  mul_alias_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(b, B, f, P->n);  // B .* f
  int rc = ax::launch_status();
  if (rc) return rc;
  if ((rc = ax_gs_sum(P->gs, b, st))) return rc;
  mul_alias_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(b, P->mask, b, P->n);  // mask .* gs(B f)
  return ax::launch_status();
}

// ---------------------------------------------------------------------------
// The partitioned solve's rank-local vector work on a GPU rank: this
// library's kernels on the rank's Poisson handle (the driver is part.cpp).
namespace {

struct PartNative {
  ax_poisson *P;
  const double *wgt;
  double *work;  // AX_DOT_WORK partials + the dot result
};

int pn_apply(void *c, double *w, const double *p, void *st) {
  return ax_poisson_apply(static_cast<PartNative *>(c)->P, w, p, st);
}
int pn_precond(void *c, double *z, const double *r, void *st) {
  return ax_precondition(static_cast<PartNative *>(c)->P, nullptr, z, r, st);
}
int pn_dot(void *c, const double *a, const double *b, double *out, void *st) {
  auto *n = static_cast<PartNative *>(c);
  int rc = ax_dot_weighted(a, b, n->wgt, n->P->n, n->work, n->work + AX_DOT_WORK, st);
  if (rc) return rc;
  if (cudaMemcpyAsync(out, n->work + AX_DOT_WORK, sizeof(double), cudaMemcpyDeviceToHost,
                      (cudaStream_t)st) != cudaSuccess ||
      cudaStreamSynchronize((cudaStream_t)st) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  return AX_OK;
}
int pn_axpby(void *c, double *y, double a, const double *x, double b, void *st) {
  return ax_axpby(y, a, x, b, static_cast<PartNative *>(c)->P->n, st);
}
int pn_copy(void *c, double *dst, const double *src, void *st) {
  const int64_t n = static_cast<PartNative *>(c)->P->n;
  if (cudaMemcpyAsync(dst, src, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice,
                      (cudaStream_t)st) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  return AX_OK;
}
int pn_zero(void *c, double *v, void *st) {
  const int64_t n = static_cast<PartNative *>(c)->P->n;
  if (cudaMemsetAsync(v, 0, (size_t)n * sizeof(double), (cudaStream_t)st) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  return AX_OK;
}

}  // namespace

extern "C" int ax_cg_solve_part_poisson(ax_poisson *P, const double *wgt,
                                        const ax_part_comm *comm, double *x, const double *b,
                                        double tol, int maxit, int *iters, double *relres,
                                        void *stream) {
  if (!P || !wgt || !comm || !x || !b) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  double *z = nullptr, *work = nullptr;
  if (alloc(&z, P->n) || alloc(&work, AX_DOT_WORK + 1)) {
    cudaFree(z);
    return AX_ENOMEM;
  }
  PartNative ctx{P, wgt, work};
  const ax_part_ops ops{&ctx, pn_apply, pn_precond, pn_dot, pn_axpby, pn_copy, pn_zero};
  int rc = ax_cg_solve_part(&ops, comm, x, b, P->r, z, P->p, P->w, tol, maxit, iters, relres,
                            stream);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == AX_OK) rc = AX_ELAUNCH;
  cudaFree(z);
  cudaFree(work);
  return rc;
}
