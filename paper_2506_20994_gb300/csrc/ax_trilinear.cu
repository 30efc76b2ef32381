// fp32 element operator with the geometric factors computed on the fly from
// each element's 8 corner vertices (trilinear hexahedra), instead of read as
// six stored fields.  Listing 2's contractions and pointwise step are
// unchanged; only where G comes from differs: per point,
//
//   J = dx/dr (3x3; column a the derivative along r, s, t),
//   G = w_i w_j w_k det(J) J^{-1} J^{-T} = (w_i w_j w_k / det J) adj(J) adj(J)^T,
//
// the factor of Listing 2 written out for a trilinear map (the same G that
// stored-geometry callers build from the GLL node coordinates, exact for a
// trilinear map since D differentiates degree-1 polynomials exactly).
//
// Per element: 36 edge coefficients in fp64 from the corners, rounded to
// fp32 (differences of nearby fp64 coordinates, so the fp32 values keep full
// relative precision).  Per thread (i, j) of the k-loop schedule: the t-column
// of J is constant over k and the r- and s-columns are linear in the
// k-position, so J costs 12 fp32 operations per point and G about 50 more.
// Reads u (and h1 unless it is constant 1) and writes w: 8 or 12 bytes per
// point against 36 for the stored-geometry fp32 kernel.
#include "common.cuh"
#include "dispatch.h"

namespace ax {
namespace {

// 1-D matrix tables in shared memory, rows padded to RS floats so that the
// 16-byte row loads of different rows fall in different banks
template <int LX>
constexpr int tri_rs() {
  return LX % 8 == 0 ? LX + 4 : LX;
}
template <int LX>
constexpr int tri_lxp() {  // small tables padded to whole 16-byte groups
  return (LX + 3) / 4 * 4;
}

template <int LX>
constexpr size_t tri_smem(int epb) {
  // three matrix tables; phi0, phi1, wq; per element u, wr, ws and 36 coefficients
  return (3 * (size_t)LX * tri_rs<LX>() + 3 * tri_lxp<LX>() +
          (size_t)epb * (3 * LX * LX * LX + 36)) *
         sizeof(float);
}

template <int LX, bool H1>
__global__ void __launch_bounds__(256, LX <= 8 ? 4 : LX <= 12 ? 3 : 2)
ax_tri_f32_kernel(float *__restrict__ w, const float *__restrict__ u,
                  const float *__restrict__ dx, const float *__restrict__ dxt,
                  const float *__restrict__ h1, const double *__restrict__ corners,
                  const double *__restrict__ xi, const double *__restrict__ wq, int nelv,
                  int epb) {
  constexpr int N2 = LX * LX;
  constexpr int N3 = LX * N2;
  // lx divisible by 4: rows of the tables, of u and of wr are read as float4
  constexpr bool VEC = LX % 4 == 0;
  constexpr int RS = tri_rs<LX>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // Fd[a][l] = dx[l*lx + a] (forward), Bd[a][l] = dxt[l*lx + a] and
  // Td[a][b] = dxt[a*lx + b] (transposed sum): each contraction reads a row
  float *Fd = reinterpret_cast<float *>(smem_raw);
  float *Bd = Fd + LX * RS;
  float *Td = Bd + LX * RS;
  float *phi0 = Td + LX * RS;          // (1 - xi_k) / 2
  float *phi1 = phi0 + tri_lxp<LX>();  // (1 + xi_k) / 2
  float *swq = phi1 + tri_lxp<LX>();   // GLL weights
  const bool own = (int)threadIdx.x < epb * N2;
  const int le = own ? (int)threadIdx.x / N2 : 0;
  const int p = (int)threadIdx.x - le * N2;
  const int i = p % LX;
  const int j = p / LX;
  float *su = swq + tri_lxp<LX>() + (size_t)le * (3 * N3 + 36);
  float *swr = su + N3;
  float *sws = swr + N3;
  float *cf = sws + N3;  // [dir r/s/t][coord x/y/z][pair], pair over the other two bits
  auto row4 = [](const float *r, int q) { return reinterpret_cast<const float4 *>(r)[q]; };

  const long long e0 = (long long)blockIdx.x * epb;
  const long long left = nelv - e0;
  const int nel = left < epb ? (int)left : epb;
  const bool active = own && le < nel;
  const long long e = active ? e0 + le : 0;
  const size_t base = (size_t)e * N3 + p;

  for (int t = threadIdx.x; t < N2; t += blockDim.x) {
    const int a = t / LX, b = t % LX;
    Fd[b * RS + a] = dx[t];
    Bd[b * RS + a] = dxt[t];
    Td[a * RS + b] = dxt[t];
  }
  for (int t = threadIdx.x; t < LX; t += blockDim.x) {
    const double x = xi[t];
    phi0[t] = (float)(0.5 * (1.0 - x));
    phi1[t] = (float)(0.5 * (1.0 + x));
    swq[t] = (float)wq[t];
  }
  // half edge vectors of the trilinear map, corner index ((c*2+b)*2+a)*3+coord
  for (int t = p; active && t < 36; t += N2) {  // lx < 6: fewer than 36 threads
    const int dir = t / 12, d = (t / 4) % 3, q = t % 4, hi = q >> 1, lo = q & 1;
    int c0, c1;  // corner pair differing in the bit of `dir`
    if (dir == 0) {        // r: bit a; pair (c, b)
      c0 = (hi * 2 + lo) * 2;
      c1 = c0 + 1;
    } else if (dir == 1) {  // s: bit b; pair (c, a)
      c0 = (hi * 2) * 2 + lo;
      c1 = c0 + 2;
    } else {                // t: bit c; pair (b, a)
      c0 = hi * 2 + lo;
      c1 = c0 + 4;
    }
    const double *x = corners + (size_t)e * 24;
    cf[t] = (float)(0.5 * (x[c1 * 3 + d] - x[c0 * 3 + d]));
  }

  float uk[LX];
  if (own) {
#pragma unroll
    for (int k = 0; k < LX; ++k) {
      uk[k] = active ? u[base + (size_t)k * N2] : 0.f;
      su[k * N2 + p] = uk[k];
    }
  }
  __syncthreads();

  // this thread's (i, j): r-column coefficients in c, s-column in c, t-column
  const float pj0 = phi0[j], pj1 = phi1[j], pi0 = phi0[i], pi1 = phi1[i];
  float P[3][2], Q[3][2], Jt[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      P[d][c] = __fmaf_rn(cf[d * 4 + c * 2 + 1], pj1, cf[d * 4 + c * 2] * pj0);
      Q[d][c] = __fmaf_rn(cf[12 + d * 4 + c * 2 + 1], pi1, cf[12 + d * 4 + c * 2] * pi0);
    }
    const float b0 = __fmaf_rn(cf[24 + d * 4 + 1], pi1, cf[24 + d * 4] * pi0);
    const float b1 = __fmaf_rn(cf[24 + d * 4 + 3], pi1, cf[24 + d * 4 + 2] * pi0);
    Jt[d] = __fmaf_rn(b1, pj1, b0 * pj0);
  }
  const float wij = swq[i] * swq[j];

  float wacc[LX];
  if (own) {
#pragma unroll
    for (int k = 0; k < LX; ++k) wacc[k] = 0.f;
#pragma unroll
    for (int k = 0; k < LX; ++k) {
      float ur = 0.f, us = 0.f, ut = 0.f;
      if constexpr (VEC) {
#pragma unroll
        for (int q = 0; q < LX / 4; ++q) {
          const float4 fi = row4(Fd + i * RS, q), fj = row4(Fd + j * RS, q);
          const float4 fk = row4(Fd + k * RS, q), v = row4(su + k * N2 + j * LX, q);
          const float *c = su + k * N2 + 4 * q * LX + i;
          ur = __fmaf_rn(fi.x, v.x, ur);
          us = __fmaf_rn(fj.x, c[0], us);
          ut = __fmaf_rn(fk.x, uk[4 * q], ut);
          ur = __fmaf_rn(fi.y, v.y, ur);
          us = __fmaf_rn(fj.y, c[LX], us);
          ut = __fmaf_rn(fk.y, uk[4 * q + 1], ut);
          ur = __fmaf_rn(fi.z, v.z, ur);
          us = __fmaf_rn(fj.z, c[2 * LX], us);
          ut = __fmaf_rn(fk.z, uk[4 * q + 2], ut);
          ur = __fmaf_rn(fi.w, v.w, ur);
          us = __fmaf_rn(fj.w, c[3 * LX], us);
          ut = __fmaf_rn(fk.w, uk[4 * q + 3], ut);
        }
      } else {
#pragma unroll
        for (int l = 0; l < LX; ++l) {
          ur = __fmaf_rn(Fd[i * RS + l], su[k * N2 + j * LX + l], ur);
          us = __fmaf_rn(Fd[j * RS + l], su[k * N2 + l * LX + i], us);
          ut = __fmaf_rn(Fd[k * RS + l], uk[l], ut);
        }
      }
      float wr = 0.f, ws = 0.f, wt = 0.f;
      if (active) {
        const float z0 = phi0[k], z1 = phi1[k];
        // J rows: coordinates x, y, z; columns r, s, t
        const float a = __fmaf_rn(P[0][1], z1, P[0][0] * z0);
        const float b = __fmaf_rn(Q[0][1], z1, Q[0][0] * z0);
        const float c = Jt[0];
        const float d = __fmaf_rn(P[1][1], z1, P[1][0] * z0);
        const float f = __fmaf_rn(Q[1][1], z1, Q[1][0] * z0);
        const float g = Jt[1];
        const float h = __fmaf_rn(P[2][1], z1, P[2][0] * z0);
        const float m = __fmaf_rn(Q[2][1], z1, Q[2][0] * z0);
        const float n = Jt[2];
        // adj(J) = det(J) J^{-1}: row r is det * grad r, and so on
        const float A00 = __fmaf_rn(f, n, -g * m), A01 = __fmaf_rn(c, m, -b * n);
        const float A02 = __fmaf_rn(b, g, -c * f), A10 = __fmaf_rn(g, h, -d * n);
        const float A11 = __fmaf_rn(a, n, -c * h), A12 = __fmaf_rn(c, d, -a * g);
        const float A20 = __fmaf_rn(d, m, -f * h), A21 = __fmaf_rn(b, h, -a * m);
        const float A22 = __fmaf_rn(a, f, -b * d);
        const float det = __fmaf_rn(a, A00, __fmaf_rn(b, A10, c * A20));
        float s = __fdividef(wij * swq[k], det);  // fp32 operator: ~2 ulp is ample
        if (H1) s *= h1[base + (size_t)k * N2];
        const float g11 = s * __fmaf_rn(A00, A00, __fmaf_rn(A01, A01, A02 * A02));
        const float g22 = s * __fmaf_rn(A10, A10, __fmaf_rn(A11, A11, A12 * A12));
        const float g33 = s * __fmaf_rn(A20, A20, __fmaf_rn(A21, A21, A22 * A22));
        const float g12 = s * __fmaf_rn(A00, A10, __fmaf_rn(A01, A11, A02 * A12));
        const float g13 = s * __fmaf_rn(A00, A20, __fmaf_rn(A01, A21, A02 * A22));
        const float g23 = s * __fmaf_rn(A10, A20, __fmaf_rn(A11, A21, A12 * A22));
        wr = __fmaf_rn(g11, ur, __fmaf_rn(g12, us, g13 * ut));
        ws = __fmaf_rn(g12, ur, __fmaf_rn(g22, us, g23 * ut));
        wt = __fmaf_rn(g13, ur, __fmaf_rn(g23, us, g33 * ut));
      }
      swr[k * N2 + p] = wr;
      sws[k * N2 + p] = ws;
      if constexpr (VEC) {
#pragma unroll
        for (int q = 0; q < LX / 4; ++q) {
          const float4 t4 = row4(Td + k * RS, q);
          wacc[4 * q] = __fmaf_rn(t4.x, wt, wacc[4 * q]);
          wacc[4 * q + 1] = __fmaf_rn(t4.y, wt, wacc[4 * q + 1]);
          wacc[4 * q + 2] = __fmaf_rn(t4.z, wt, wacc[4 * q + 2]);
          wacc[4 * q + 3] = __fmaf_rn(t4.w, wt, wacc[4 * q + 3]);
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < LX; ++kk) wacc[kk] = __fmaf_rn(Td[k * RS + kk], wt, wacc[kk]);
      }
    }
  }
  __syncthreads();

  if (own) {
#pragma unroll
    for (int k = 0; k < LX; ++k) {
      float acc = wacc[k];
      if constexpr (VEC) {
#pragma unroll
        for (int q = 0; q < LX / 4; ++q) {
          const float4 bi = row4(Bd + i * RS, q), bj = row4(Bd + j * RS, q);
          const float4 v = row4(swr + k * N2 + j * LX, q);
          const float *c = sws + k * N2 + 4 * q * LX + i;
          acc = __fmaf_rn(bi.x, v.x, acc);
          acc = __fmaf_rn(bj.x, c[0], acc);
          acc = __fmaf_rn(bi.y, v.y, acc);
          acc = __fmaf_rn(bj.y, c[LX], acc);
          acc = __fmaf_rn(bi.z, v.z, acc);
          acc = __fmaf_rn(bj.z, c[2 * LX], acc);
          acc = __fmaf_rn(bi.w, v.w, acc);
          acc = __fmaf_rn(bj.w, c[3 * LX], acc);
        }
      } else {
#pragma unroll
        for (int l = 0; l < LX; ++l) {
          acc = __fmaf_rn(Bd[i * RS + l], swr[k * N2 + j * LX + l], acc);
          acc = __fmaf_rn(Bd[j * RS + l], sws[k * N2 + l * LX + i], acc);
        }
      }
      if (active) w[base + (size_t)k * N2] = acc;
    }
  }
}

template <int LX>
int launch_tri(float *w, const float *u, const float *dx, const float *dxt, const float *h1,
               const double *corners, const double *xi, const double *wq, int nelv,
               cudaStream_t st) {
  const int epb = 256 / (LX * LX) < 1 ? 1 : 256 / (LX * LX);
  const size_t smem = tri_smem<LX>(epb);
  auto kern = h1 ? ax_tri_f32_kernel<LX, true> : ax_tri_f32_kernel<LX, false>;
  static std::atomic<size_t> granted[2][kMaxDevices];
  if (!grant_smem(kern, smem, granted[h1 != nullptr])) return AX_EINVAL;
  const unsigned grid = (unsigned)((nelv + epb - 1) / epb);
  kern<<<grid, epb * LX * LX, smem, st>>>(w, u, dx, dxt, h1, corners, xi, wq, nelv, epb);
  return launch_status();
}

}  // namespace
}  // namespace ax

extern "C" int ax_helm_trilinear_f32(float *w, const float *u, const float *dx, const float *dxt,
                                     const float *h1, const double *corners, const double *xi,
                                     const double *wq, int lx, int nelv, void *stream) {
  if (!ax::lx_ok(lx) || nelv < 0) return AX_EINVAL;
  if (nelv == 0) return AX_OK;
  if (!ax::all_nonnull(w, u, dx, dxt, corners, xi, wq)) return AX_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  switch (lx) {
#define AX_CASE(L) \
  case L:          \
    return ax::launch_tri<L>(w, u, dx, dxt, h1, corners, xi, wq, nelv, st);
    AX_LX_CASES(AX_CASE)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}
