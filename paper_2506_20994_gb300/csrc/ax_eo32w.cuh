// One warp per element: the fp32-arithmetic even-odd operator (ax_eo32.cuh)
// at lx = 8 on bf16 geometry (u in bf16, or the solvers' fp32 vectors), with
// the t-direction (along k) contracted in registers.
//
// Lane 4 j + i' owns the 16 points {i', 7 - i'} x {j} x {k = 0..7}.  Its two
// k-columns are whole, so the t-contractions (even-odd on the columns'
// mirror pairs) use no shared memory; only the r-lines (along i: the lane
// forms entry i' of line (k, j) itself) and the s-lines (along j: the mirror
// row 7 - j is lane ^ 28, one shuffle) pass through shared memory.  Every
// synchronisation is within the warp (__syncwarp): the warps of a CTA run
// independently, each with its own stage (u and the seven geometry fields of
// one element, bulk-copied under one mbarrier, waits bounded) and its own
// lines.  u and the geometry complete on two mbarriers: a warp issues its
// next element's u as soon as it holds this element's u in registers, and
// the next geometry once the pointwise step has read this one, so each copy
// overlaps most of an element's work.
//
// Same arithmetic as ax_eo32.cuh, operation for operation (chains over
// l = 0..3, y_i = E + O, y_{N-i} = O - E, pointwise h1 G, w = (r + s) + t;
// with the solver's fused direction update, p = minv r + beta p first): the
// two kernels give the same w.  The dot partial (DOT) sums the same products
// in another order.  Matrices that are not
// centro-antisymmetric take a second chain for the rows N - i, as there.
// Shared memory per element and warp: about 130 load and 64 store wavefronts
// for the lines (16-byte line reads; 8-byte entry writes) against about 450
// and 156 in the octant layout, whose t-lines are 32 distinct 16-byte units
// per warp access.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "ax_eo32.cuh"

namespace ax {
namespace e32w {

using df::u64;
using e32::fma2;
using e32::hi_;
using e32::lo_;
using e32::mul2;
using e32::pk;

constexpr int LX = 8, H = 4, N = 7, H2 = 16, N3 = 512;
constexpr int kWarps = 4;  // warps (elements in flight) per CTA

// PUPD (the solver's fused direction update, fp32 vectors): the u part of
// the stage holds r, minv and the old direction instead of u.
template <class SU, class SG, bool PUPD = false>
struct Cfg {
  static constexpr unsigned UBYTES = N3 * sizeof(SU);
  static constexpr unsigned GFBYTES = N3 * sizeof(SG);
  static constexpr int NU = PUPD ? 3 : 1;  // u-sized staged arrays
  static constexpr size_t SBYTES = e32::a128(NU * UBYTES + 7 * GFBYTES);
  static constexpr size_t LBYTES = 2 * 64 * H * 8;  // r-lines (k, j) and s-lines (k, i)
  static constexpr size_t WBYTES = SBYTES + LBYTES;
  // coefficients [m][rows i, rows N - i][H][H], as in ax_eo32.cuh
  static constexpr size_t OFF_W = e32::a128(2 * 2 * H2 * 8);
  static constexpr size_t OFF_BAR = OFF_W + kWarps * WBYTES;
  static constexpr size_t SMEM = OFF_BAR + kWarps * 16 + kWarps * 8;
};

// entry e of line L (4 entries of 8 bytes): the 16-byte halves swap with
// bit 2 of the line, so that lines L and L + 4 start in different banks
AX_D int rpos(int L, int e) { return L * 4 + ((((e >> 1) ^ (L >> 2)) & 1) << 1) + (e & 1); }

// Resident CTAs per SM the launch bounds ask for: 4 on bf16 data without
// the dot (128 registers); 3 where fp32 vectors or the dot partial add
// registers and shared memory.
template <class SU, bool DOT>
constexpr int minb() {
  return std::is_same_v<SU, float> || DOT ? 3 : 4;
}

template <class SU, class SG, bool DOT, bool PUPD = false>
__global__ void __launch_bounds__(kWarps * 32, (minb<SU, DOT>()))
ax_eo32w_kernel(const e32::Mesh<SU, SG> M, long long nelv, int *__restrict__ err,
                double *__restrict__ dotp, const E32Upd up) {
  static_assert(!PUPD || std::is_same_v<SU, float>, "the fused update keeps fp32 vectors");
  using C = Cfg<SU, SG, PUPD>;
  extern __shared__ __align__(128) unsigned char sm[];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int ip = lane & 3, j = lane >> 2;  // i in {i', 7 - i'}; this lane's j
  const bool lo = j < H;                   // s-lines: this lane forms entry jj of line (k, i)
  const int jj = lo ? j : N - j, is = lo ? ip : N - ip;
  u64 *cf = reinterpret_cast<u64 *>(sm);
  unsigned char *stg = sm + C::OFF_W + (size_t)wp * C::WBYTES;
  u64 *Lr = reinterpret_cast<u64 *>(stg + C::SBYTES);
  u64 *Ls = Lr + 64 * H;
  const uint32_t barU = eop::smem_u32(sm + C::OFF_BAR + wp * 16), barG = barU + 8;
  double *red = reinterpret_cast<double *>(sm + C::OFF_BAR + kWarps * 16);

  // even-odd coefficients of dx (m = 0) and dxt (m = 1): M(i, l) = D[l * 8 + i]
  bool ok = true;
  for (int q = threadIdx.x; q < 2 * H2; q += blockDim.x) {
    const int m = q / H2, i = (q / H) % H, l = q % H;
    const float *D = m ? M.dxt : M.dx;
    const float a = __ldg(D + l * LX + i), b = __ldg(D + (N - l) * LX + i);
    const float a2 = __ldg(D + l * LX + N - i), b2 = __ldg(D + (N - l) * LX + N - i);
    const float A = __fmul_rn(0.5f, __fadd_rn(a, b)), B = __fmul_rn(0.5f, __fsub_rn(a, b));
    const float A2 = __fmul_rn(0.5f, __fadd_rn(a2, b2));
    const float B2 = __fmul_rn(0.5f, __fsub_rn(a2, b2));
    cf[m * 2 * H2 + i * H + l] = pk(A, B);
    cf[m * 2 * H2 + H2 + i * H + l] = pk(A2, B2);
    ok = ok && A2 == -A && B2 == B;
  }
  if (lane == 0) {
    eop::mbar_init(barU, 1);
    eop::mbar_init(barG, 1);
  }
  // coefficients and barriers ready; from here on the warps are independent
  const bool gen_m = __syncthreads_and(ok) == 0;

  auto issue_u = [&](long long e) __attribute__((always_inline)) {
    const uint32_t dst = eop::smem_u32(stg);
    const size_t eo = (size_t)e * N3;
    eop::mbar_expect(barU, C::NU * C::UBYTES);
    if constexpr (PUPD) {
      eop::bulk_copy(dst, up.r + eo, C::UBYTES, barU);
      eop::bulk_copy(dst + C::UBYTES, up.minv + eo, C::UBYTES, barU);
      eop::bulk_copy(dst + 2 * C::UBYTES, up.pw + eo, C::UBYTES, barU);
    } else {
      eop::bulk_copy(dst, M.u + eo, C::UBYTES, barU);
    }
  };
  auto issue_g = [&](long long e) __attribute__((always_inline)) {
    const uint32_t dst = eop::smem_u32(stg) + C::NU * C::UBYTES;
    eop::mbar_expect(barG, 7 * C::GFBYTES);
#pragma unroll
    for (int f = 0; f < 7; ++f)
      eop::bulk_copy(dst + f * C::GFBYTES, M.g[f] + (size_t)e * N3, C::GFBYTES, barG);
  };
  const long long nw = (long long)gridDim.x * kWarps;
  long long e = (long long)blockIdx.x * kWarps + wp;
  if (lane == 0 && e < nelv) {
    issue_u(e);
    issue_g(e);
  }
  __syncwarp();

  // this lane's values of row (k, j) of one staged field at i' and 7 - i'.
  // bf16: the words holding them, each value moved into the high half of an
  // fp32 word by a byte permute.  fp32: the lanes with j >= 4 read 7 - i'
  // first (rows j and j + 4 share banks).
  const unsigned wsel0 = (ip & 1) ? 0x3244u : 0x1044u, wsel1 = (ip & 1) ? 0x1044u : 0x3244u;
  auto rowv = [&](const auto *F, int k, float &x0, float &x1) __attribute__((always_inline)) {
    using S = std::remove_cv_t<std::remove_pointer_t<decltype(F)>>;
    const int r = (k * LX + j) * LX;
    if constexpr (std::is_same_v<S, __nv_bfloat16>) {
      const unsigned *w = reinterpret_cast<const unsigned *>(F + r);
      x0 = __uint_as_float(__byte_perm(w[ip >> 1], 0u, wsel0));
      x1 = __uint_as_float(__byte_perm(w[3 - (ip >> 1)], 0u, wsel1));
    } else {
      const float f0 = F[r + (lo ? ip : N - ip)], f1 = F[r + (lo ? N - ip : ip)];
      x0 = lo ? f0 : f1;
      x1 = lo ? f1 : f0;
    }
  };
  auto eo = [](float v0, float v1) __attribute__((always_inline)) {
    return pk(__fadd_rn(v0, v1), __fsub_rn(v0, v1));
  };
  // (E, O) of coefficient row cr over line L of ln, l = 0..3 in order
  auto chainL = [](const u64 *ln, int L, const u64 (&cr)[H]) __attribute__((always_inline)) {
    const ulonglong2 h0 = *reinterpret_cast<const ulonglong2 *>(ln + rpos(L, 0));
    const ulonglong2 h1 = *reinterpret_cast<const ulonglong2 *>(ln + rpos(L, 2));
    u64 a = mul2(cr[0], h0.x);
    a = fma2(cr[1], h0.y, a);
    a = fma2(cr[2], h1.x, a);
    return fma2(cr[3], h1.y, a);
  };
  auto chainR = [](const u64 (&ln)[H], const u64 (&cr)[H]) __attribute__((always_inline)) {
    u64 a = mul2(cr[0], ln[0]);
    a = fma2(cr[1], ln[1], a);
    a = fma2(cr[2], ln[2], a);
    return fma2(cr[3], ln[3], a);
  };
  auto row = [&](const u64 *cof, int r, u64 (&cr)[H]) __attribute__((always_inline)) {
    const ulonglong2 c01 = *reinterpret_cast<const ulonglong2 *>(cof + r * H);
    const ulonglong2 c23 = *reinterpret_cast<const ulonglong2 *>(cof + r * H + 2);
    cr[0] = c01.x;
    cr[1] = c01.y;
    cr[2] = c23.x;
    cr[3] = c23.y;
  };

  // r-lines of field vr and s-lines of field vs
  auto publish = [&](const float (&vr)[LX][2], const float (&vs)[LX][2])
                     __attribute__((always_inline)) {
#pragma unroll
    for (int k = 0; k < LX; ++k) {
      Lr[rpos(k * LX + j, ip)] = eo(vr[k][0], vr[k][1]);
      // the lane with j < 4 forms the entry of line (k, i'), its mirror lane
      // (7 - j) that of line (k, 7 - i'); each sends the other the value it
      // needs
      const float mine = lo ? vs[k][0] : vs[k][1], other = lo ? vs[k][1] : vs[k][0];
      const float recv = __shfl_xor_sync(0xffffffffu, other, 28);
      Ls[rpos(k * LX + is, jj)] = lo ? eo(mine, recv) : eo(recv, mine);
    }
    __syncwarp();
  };
  // r-contractions: y at (k, j, i'), (k, j, 7 - i'); add: y += the result
  auto contract_r = [&](const u64 *cof, float (&y)[LX][2], bool add, auto gen)
                        __attribute__((always_inline)) {
    u64 cr[H];
    row(cof, ip, cr);
#pragma unroll
    for (int k = 0; k < LX; ++k) {
      const u64 a = chainL(Lr, k * LX + j, cr);
      const float y0 = __fadd_rn(lo_(a), hi_(a));
      float y1 = __fsub_rn(hi_(a), lo_(a));
      if constexpr (decltype(gen)::value) {
        u64 c2[H];
        row(cof + H2, ip, c2);
        const u64 b = chainL(Lr, k * LX + j, c2);
        y1 = __fadd_rn(lo_(b), hi_(b));
      }
      y[k][0] = add ? __fadd_rn(y[k][0], y0) : y0;
      y[k][1] = add ? __fadd_rn(y[k][1], y1) : y1;
    }
  };
  // s-contractions of line (k, i_s): rows jj and 7 - jj.  The lane keeps the
  // row at its own j and swaps the other with its mirror lane: the lo lane
  // (column i') sends y(7 - j) of column i', its mirror (column 7 - i')
  // sends back y(j) of column 7 - i'.
  auto contract_s = [&](const u64 *cof, float (&y)[LX][2], bool add, auto gen)
                        __attribute__((always_inline)) {
    u64 cr[H];
    row(cof, jj, cr);
#pragma unroll
    for (int k = 0; k < LX; ++k) {
      const u64 a = chainL(Ls, k * LX + is, cr);
      const float yj = __fadd_rn(lo_(a), hi_(a));
      float ym = __fsub_rn(hi_(a), lo_(a));
      if constexpr (decltype(gen)::value) {
        u64 c2[H];
        row(cof + H2, jj, c2);
        const u64 b = chainL(Ls, k * LX + is, c2);
        ym = __fadd_rn(lo_(b), hi_(b));
      }
      const float keep = lo ? yj : ym, send = lo ? ym : yj;
      const float got = __shfl_xor_sync(0xffffffffu, send, 28);
      const float y0 = lo ? keep : got, y1 = lo ? got : keep;
      y[k][0] = add ? __fadd_rn(y[k][0], y0) : y0;
      y[k][1] = add ? __fadd_rn(y[k][1], y1) : y1;
    }
  };
  // t-contractions of this lane's two columns, in registers (centro-
  // antisymmetric matrices: each coefficient row read once for both)
  auto contract_t = [&](const u64 *cof, const float (&v)[LX][2], float (&y)[LX][2], bool add,
                        auto gen) __attribute__((always_inline)) {
    auto put = [&](int kr, int a, float y0, float y1) __attribute__((always_inline)) {
      y[kr][a] = add ? __fadd_rn(y[kr][a], y0) : y0;
      y[N - kr][a] = add ? __fadd_rn(y[N - kr][a], y1) : y1;
    };
    if constexpr (decltype(gen)::value) {
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        u64 ln[H];
#pragma unroll
        for (int l = 0; l < H; ++l) ln[l] = eo(v[l][a], v[N - l][a]);
#pragma unroll
        for (int kr = 0; kr < H; ++kr) {
          u64 cr[H];
          row(cof, kr, cr);
          const u64 c = chainR(ln, cr);
          row(cof + H2, kr, cr);
          const u64 b = chainR(ln, cr);
          put(kr, a, __fadd_rn(lo_(c), hi_(c)), __fadd_rn(lo_(b), hi_(b)));
        }
      }
    } else {
      u64 ln[2][H];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int l = 0; l < H; ++l) ln[a][l] = eo(v[l][a], v[N - l][a]);
#pragma unroll
      for (int kr = 0; kr < H; ++kr) {
        u64 cr[H];
        row(cof, kr, cr);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const u64 c = chainR(ln[a], cr);
          put(kr, a, __fadd_rn(lo_(c), hi_(c)), __fsub_rn(hi_(c), lo_(c)));
        }
      }
    }
  };

  // a staged copy never completed: record it, write NaN into this warp's
  // elements from e on, wait once more (bounded) for the copies that may
  // still be in flight (phases pu of u, pg of the geometry)
  auto fail = [&](unsigned pu, unsigned pg) {
    if (lane == 0) {
      if (err) atomicExch(err, 1);
      (void)eop::mbar_wait(barU, pu, eop::kWaitLimit);
      (void)eop::mbar_wait(barG, pg, eop::kWaitLimit);
    }
    for (long long q = e; q < nelv; q += nw)
      for (int i = lane; i < N3; i += 32) M.w[(size_t)q * N3 + i] = __int_as_float(0x7fc00000);
  };

  double dsum = 0.0;
  const float beta = PUPD ? (float)*up.beta : 0.f;  // the solver's scalar, on the device
  // the element loop, compiled for both matrix forms (gen: CTA-uniform)
  auto run = [&](auto gen) __attribute__((always_inline)) {
    for (unsigned parity = 0u; e < nelv; e += nw, parity ^= 1u) {
      const bool more = e + nw < nelv;
      if (!__all_sync(0xffffffffu, eop::mbar_wait(barU, parity, eop::kWaitLimit))) {
        fail(parity, parity);
        break;
      }
      const SU *U = reinterpret_cast<const SU *>(stg);
      const SG *G = reinterpret_cast<const SG *>(stg + C::NU * C::UBYTES);
      const size_t eb = (size_t)e * N3;
      float v[LX][2];
#pragma unroll
      for (int k = 0; k < LX; ++k) rowv(U, k, v[k][0], v[k][1]);
      if constexpr (PUPD) {  // v = r here: p = minv .* r + beta p, stored
        const float *Mi = reinterpret_cast<const float *>(stg + C::UBYTES);
        const float *Po = reinterpret_cast<const float *>(stg + 2 * C::UBYTES);
#pragma unroll
        for (int k = 0; k < LX; ++k) {
          float mi[2], po[2];
          rowv(Mi, k, mi[0], mi[1]);
          rowv(Po, k, po[0], po[1]);
#pragma unroll
          for (int a = 0; a < 2; ++a) v[k][a] = __fmaf_rn(mi[a], v[k][a], __fmul_rn(beta, po[a]));
          up.pw[eb + (k * LX + j) * LX + ip] = v[k][0];
          up.pw[eb + (k * LX + j) * LX + N - ip] = v[k][1];
        }
      }
      __syncwarp();  // the staged vectors are read: the next element's may replace them
      if (lane == 0 && more) {
        eop::fence_async_smem();
        issue_u(e + nw);
      }

      // reference gradient
      float gr[LX][2], gs[LX][2], gt[LX][2];
      publish(v, v);
      contract_r(cf, gr, false, gen);
      contract_s(cf, gs, false, gen);
      contract_t(cf, v, gt, false, gen);
      __syncwarp();  // the lines are read

      // pointwise h1 G (the next u, if any, is in flight on phase parity ^ 1)
      if (!__all_sync(0xffffffffu, eop::mbar_wait(barG, parity, eop::kWaitLimit))) {
        fail(more ? parity ^ 1u : parity, parity);
        break;
      }
#pragma unroll
      for (int k = 0; k < LX; ++k) {
        float h[2], g11[2], g22[2], g33[2], g12[2], g13[2], g23[2];
        rowv(G, k, h[0], h[1]);
        rowv(G + N3, k, g11[0], g11[1]);
        rowv(G + 2 * N3, k, g22[0], g22[1]);
        rowv(G + 3 * N3, k, g33[0], g33[1]);
        rowv(G + 4 * N3, k, g12[0], g12[1]);
        rowv(G + 5 * N3, k, g13[0], g13[1]);
        rowv(G + 6 * N3, k, g23[0], g23[1]);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const float ur = gr[k][a], us = gs[k][a], ut = gt[k][a];
          gr[k][a] = __fmul_rn(
              h[a], __fmaf_rn(g13[a], ut, __fmaf_rn(g12[a], us, __fmul_rn(g11[a], ur))));
          gs[k][a] = __fmul_rn(
              h[a], __fmaf_rn(g23[a], ut, __fmaf_rn(g22[a], us, __fmul_rn(g12[a], ur))));
          gt[k][a] = __fmul_rn(
              h[a], __fmaf_rn(g33[a], ut, __fmaf_rn(g23[a], us, __fmul_rn(g13[a], ur))));
        }
      }
      __syncwarp();  // the geometry is read: the next element's may replace it
      if (lane == 0 && more) {
        eop::fence_async_smem();
        issue_g(e + nw);
      }

      // transposed contractions, w = (r + s) + t
      publish(gr, gs);
      float w[LX][2];
      contract_r(cf + 2 * H2, w, false, gen);
      contract_s(cf + 2 * H2, w, true, gen);
      contract_t(cf + 2 * H2, gt, w, true, gen);
      __syncwarp();  // the lines are read
      float el = 0.f;
#pragma unroll
      for (int k = 0; k < LX; ++k) {
        M.w[eb + (k * LX + j) * LX + ip] = w[k][0];
        M.w[eb + (k * LX + j) * LX + N - ip] = w[k][1];
        if constexpr (DOT) el = __fmaf_rn(v[k][1], w[k][1], __fmaf_rn(v[k][0], w[k][0], el));
      }
      if constexpr (DOT) dsum += (double)el;
    }
  };
  if (gen_m)
    run(std::true_type{});
  else
    run(std::false_type{});
  __syncwarp();
  if (lane == 0) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(barU) : "memory");
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(barG) : "memory");
  }
  if constexpr (DOT) {  // one partial per CTA: fixed shuffle tree, warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
    if (lane == 0) red[wp] = dsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int q = 0; q < kWarps; ++q) s += red[q];
      dotp[blockIdx.x] = s;
    }
  }
}

}  // namespace e32w
}  // namespace ax
