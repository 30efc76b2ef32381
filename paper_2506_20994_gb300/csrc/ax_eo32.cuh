// Persistent even-odd element operator (Listing 2) with fp32 arithmetic, for
// the reduced-precision storage modes: u and the geometry in fp32 or bf16,
// w in fp32.  It replaces the k-loop schedule (ax_kstep.cuh) for even lx,
// where that schedule is bound by the latency of its per-thread geometry
// loads and by its 6 lx multiply-adds per point.
//
//  * Each CTA loops over elements; one thread streams the next element's u
//    and its seven geometry fields (eight contiguous runs of lx^3 values)
//    into shared memory with `cp.async.bulk` while the CTA computes the
//    current one (two stage buffers, one mbarrier each, bounded waits).
//  * Each 1-D contraction y = M v of a line splits on the mirror pairs
//    (e_l, o_l) = (v_l + v_{N-l}, v_l - v_{N-l}), l < lx/2 (Solomonoff 1992):
//    y_i = sum_l A_il e_l + B_il o_l with A = (M_i,l + M_i,N-l)/2,
//    B = (M_i,l - M_i,N-l)/2, and y_{N-i} likewise with the rows N - i.  A
//    centro-antisymmetric M (the GLL derivative matrix) has A_{N-i} = -A_i
//    and B_{N-i} = B_i, so one chain of packed f32x2 multiply-adds over
//    (A, B) x (e, o) yields (E, O) and y_i = E + O, y_{N-i} = O - E: half the
//    multiply-adds of the direct sum.  The CTA checks the matrices when it
//    stages them; any other matrix takes the second chain (rows N - i), so
//    the result is the operator for every dx, dxt.
//  * The (lx/2)^3 mirror octants get two threads each, thread 2t + c owning
//    the points {i', N-i'} x {j} x {k', N-k'}, j = j' (c = 0) or N - j'
//    (c = 1): a warp's reads of a staged field then cover the eight rows of
//    one k-plane.  Pairs along i and k stay inside a thread; pairs along j
//    take one shuffle with the partner lane.  The two contractions of a
//    direction share their coefficient rows (held in registers at lx = 8).
//  * PUPD (the refinement's inner CG): the stage holds r, minv and the old
//    direction instead of u, and the kernel forms p = minv r + beta p first.
//  * The (e, o) lines of the three directions go to shared memory as 8-byte
//    entries, those of the gradient and those of the weighted gradient in
//    two separate sets: two barriers per element (after each publication)
//    order every reuse of a set or a stage buffer.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "ax_eo_persist.cuh"
#include "dispatch.h"

namespace ax {
namespace e32 {

using df::u64;
using eop::EopPos;

AX_D float ldf(const float *p) { return *p; }
AX_D float ldf(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

AX_D u64 pk(float x, float y) { return df::pk(x, y); }
AX_D float lo_(u64 v) { return df::lx_(v); }
AX_D float hi_(u64 v) { return df::ly_(v); }

constexpr size_t a128(size_t x) { return (x + 127) / 128 * 128; }

// PUPD: the stage holds r, minv and the old direction instead of u (the
// solver's fused direction update).
template <int LX, class SU, class SG, bool PUPD = false>
struct Cfg {
  static constexpr int H = LX / 2, N = LX - 1, H2 = H * H, H3 = H2 * H;
  static constexpr int NT = 2 * H3;                // threads per element
  static constexpr int NTB = (NT + 31) / 32 * 32;  // block size
  static constexpr int NW = NTB / 32;
  static constexpr int N3 = LX * LX * LX;
  static constexpr bool VEC = H % 2 == 0;          // lines read as 16-byte pairs
  static constexpr bool SWZ = H == 4;              // swizzled lines (lx = 8)
  static constexpr int DE = LX * LX * H;           // 8-byte entries per direction
  static constexpr int SETE = 3 * DE;              // entries per line set
  // coefficients [m = forward, transposed][rows i, rows N - i][H][H] (A, B)
  static constexpr size_t COEF_BYTES = 4 * (size_t)H2 * 8;
  static constexpr size_t OFF_LINES = a128(COEF_BYTES);
  static constexpr size_t LINE_BYTES = 2 * (size_t)SETE * 8;
  static constexpr unsigned UBYTES = N3 * sizeof(SU);
  static constexpr unsigned GFBYTES = N3 * sizeof(SG);  // one geometry field
  static constexpr int NU = PUPD ? 3 : 1;                // u-sized staged arrays
  static constexpr unsigned TXBYTES = NU * UBYTES + 7 * GFBYTES;
  static constexpr size_t SBYTES = a128(TXBYTES);        // one stage buffer
  static constexpr size_t OFF_STAGE = OFF_LINES + a128(LINE_BYTES);
  static constexpr size_t OFF_MISC = OFF_STAGE + 2 * SBYTES;
  // two mbarriers, one dot slot per warp
  static constexpr size_t SMEM = OFF_MISC + 16 + NW * 8;
  static_assert(LX % 2 == 0 && LX >= 4 && LX <= 12, "even lx, 4..12");
  static_assert(UBYTES % 16 == 0 && GFBYTES % 16 == 0, "bulk copies need 16-byte runs");
};

// At lx = 8 each thread keeps its coefficient rows of both matrices in
// registers (48 words) instead of reading them from shared memory in every
// contraction.
constexpr bool kE32CoefRegs = true;

// Resident CTAs per SM the launch bounds ask for.
template <int LX, class SU, class SG>
constexpr int minb() {
  return LX <= 4 ? 8 : LX == 6 ? 8 : LX == 8 ? (kE32CoefRegs ? 4 : 6) : LX == 10 ? 2 : 1;
}

// 8-byte entry `e` of line L of one direction.  At lx = 8 the 16-byte pairs
// of a line swap when bits 1 and 2 of L differ and lines swap in pairs when
// bit 3 is set: a model of the kernel's warp accesses gives 160 wavefronts
// per four warps against 304 unswizzled (lower bound 144).
template <int LX>
AX_D int lpos(int L, int e) {
  constexpr int H = LX / 2;
  if constexpr (H == 4) {
    return (L ^ (((L >> 3) & 1) << 1)) * 4 + ((((e >> 1) ^ ((L >> 1) ^ (L >> 2)) & 1)) << 1) +
           (e & 1);
  } else {
    return L * H + e;
  }
}

AX_D u64 fma2(u64 a, u64 b, u64 c) { return df::fma2(a, b, c); }
AX_D u64 mul2(u64 a, u64 b) { return df::mul2p(a, b); }

// Operands of one mesh: w = Ax(u); g = h1, g11, g22, g33, g12, g13, g23.
template <class SU, class SG>
struct Mesh {
  float *w;
  const SU *u;
  const SG *g[7];
  const float *dx, *dxt;
};

// Elements blockIdx.x, + gridDim.x, ... of one mesh (operands by value: the
// compiler reads them from the constant bank).
template <class SU, class SG>
struct SeqOne {
  Mesh<SU, SG> m;
  long long nelv;
  AX_D bool first(EopPos &p) const {
    p = EopPos{0, (long long)blockIdx.x};
    return p.off < nelv;
  }
  AX_D bool advance(const EopPos &p, EopPos &q) const {
    q = EopPos{0, p.off + (long long)gridDim.x};
    return q.off < nelv;
  }
  AX_D int mesh_of(const EopPos &) const { return 0; }
  AX_D long long elem(const EopPos &p) const { return p.off; }
  AX_D const Mesh<SU, SG> &mesh(int) const { return m; }
};

// Persistent body over `seq` for one group of NTB threads (`tid` in
// [0, NTB)), `sm` its shared memory (Cfg::SMEM bytes, 128-byte aligned),
// sync() / sync_and(p) its barriers.  DOT: adds this thread's share of
// u . w to dsum (fp32 per element, fp64 across elements).  err: set to 1 if
// a staged copy never arrived (the body then stops).
// CREG (lx = 8 only): coefficient rows in registers (same arithmetic, so
// the same bits, as reading them from shared memory).
template <int LX, class SU, class SG, bool DOT, bool PUPD, bool CREG, class Seq, class Sync,
          class SyncAnd>
AX_D void e32_run(unsigned char *sm, int tid, const Seq &seq, Sync sync, SyncAnd sync_and,
                  int *err, double &dsum, const E32Upd &up = E32Upd{}) {
  static_assert(!PUPD || std::is_same_v<SU, float>, "the fused update keeps fp32 vectors");
  using C = Cfg<LX, SU, SG, PUPD>;
  constexpr int H = C::H, N = C::N, H2 = C::H2, NT = C::NT, N3 = C::N3;
  constexpr bool kCoefRegs = CREG && LX == 8;
  u64 *cf = reinterpret_cast<u64 *>(sm);
  u64 *Lb = reinterpret_cast<u64 *>(sm + C::OFF_LINES);
  unsigned char *stg = sm + C::OFF_STAGE;
  const uint32_t bar0 = eop::smem_u32(sm + C::OFF_MISC);

  const bool real = tid < NT;
  const int t = real ? tid >> 1 : 0, c = tid & 1;
  const int ip = t % H, jp = (t / H) % H, kp = t / H2;
  const int jc = c ? N - jp : jp;  // this thread's j
  // point (i_a, j_c, k_b): a, b in {0, 1} pick i', N - i' and k', N - k'
  auto kb = [&](int b) __attribute__((always_inline)) { return b ? N - kp : kp; };
  auto ia = [&](int a) __attribute__((always_inline)) { return a ? N - ip : ip; };
  auto pidx = [&](int b, int a) __attribute__((always_inline)) {
    return (kb(b) * LX + jc) * LX + ia(a);
  };
  // lines: r along i at (k, j), entries ip; s along j at (k, i), entries jp;
  // t along k at (j, i), entries kp
  auto lineR = [&](int b) __attribute__((always_inline)) { return kb(b) * LX + jc; };
  auto lineS = [&](int b, int a) __attribute__((always_inline)) { return kb(b) * LX + ia(a); };
  auto lineT = [&](int a) __attribute__((always_inline)) { return jc * LX + ia(a); };
  auto eo = [](float v0, float v1) __attribute__((always_inline)) {
    return pk(__fadd_rn(v0, v1), __fsub_rn(v0, v1));
  };

  // chains over the (e, o) entries of two lines L0, L1 with the same
  // coefficient rows `cr` (read once for both)
  auto chain2 = [&](const u64 *ln, int L0, int L1, const u64 *cr, u64 &a0, u64 &a1)
                    __attribute__((always_inline)) {
    if constexpr (C::VEC) {
#pragma unroll
      for (int q = 0; q < H / 2; ++q) {
        const ulonglong2 cv = *reinterpret_cast<const ulonglong2 *>(cr + 2 * q);
        const ulonglong2 l0 = *reinterpret_cast<const ulonglong2 *>(ln + lpos<LX>(L0, 2 * q));
        const ulonglong2 l1 = *reinterpret_cast<const ulonglong2 *>(ln + lpos<LX>(L1, 2 * q));
        a0 = q == 0 ? mul2(cv.x, l0.x) : fma2(cv.x, l0.x, a0);
        a1 = q == 0 ? mul2(cv.x, l1.x) : fma2(cv.x, l1.x, a1);
        a0 = fma2(cv.y, l0.y, a0);
        a1 = fma2(cv.y, l1.y, a1);
      }
    } else {
      a0 = mul2(cr[0], ln[lpos<LX>(L0, 0)]);
      a1 = mul2(cr[0], ln[lpos<LX>(L1, 0)]);
#pragma unroll
      for (int l = 1; l < H; ++l) {
        a0 = fma2(cr[l], ln[lpos<LX>(L0, l)], a0);
        a1 = fma2(cr[l], ln[lpos<LX>(L1, l)], a1);
      }
    }
  };
  // the same with the coefficient row held in registers
  auto chain2r = [&](const u64 *ln, int L0, int L1, const u64 (&cr)[H], u64 &a0, u64 &a1)
                     __attribute__((always_inline)) {
#pragma unroll
    for (int q = 0; q < H / 2; ++q) {
      const ulonglong2 l0 = *reinterpret_cast<const ulonglong2 *>(ln + lpos<LX>(L0, 2 * q));
      const ulonglong2 l1 = *reinterpret_cast<const ulonglong2 *>(ln + lpos<LX>(L1, 2 * q));
      a0 = q == 0 ? mul2(cr[2 * q], l0.x) : fma2(cr[2 * q], l0.x, a0);
      a1 = q == 0 ? mul2(cr[2 * q], l1.x) : fma2(cr[2 * q], l1.x, a1);
      a0 = fma2(cr[2 * q + 1], l0.y, a0);
      a1 = fma2(cr[2 * q + 1], l1.y, a1);
    }
  };
  // y at rows (row, N - row) of lines L0 and L1; cof: one matrix's
  // [2][H][H] block; rr: row `row` of its first half, in registers (kCoefRegs)
  auto contract2 = [&](const u64 *ln, int L0, int L1, const u64 *cof, bool gen, int row,
                       const u64 (&rr)[H], float (&y0)[2], float (&y1)[2])
                       __attribute__((always_inline)) {
    u64 a0, a1;
    if constexpr (kCoefRegs)
      chain2r(ln, L0, L1, rr, a0, a1);
    else
      chain2(ln, L0, L1, cof + row * H, a0, a1);
    y0[0] = __fadd_rn(lo_(a0), hi_(a0));
    y0[1] = __fadd_rn(lo_(a1), hi_(a1));
    if (gen) {
      u64 b0, b1;
      chain2(ln, L0, L1, cof + H2 + row * H, b0, b1);
      y1[0] = __fadd_rn(lo_(b0), hi_(b0));
      y1[1] = __fadd_rn(lo_(b1), hi_(b1));
    } else {
      y1[0] = __fsub_rn(hi_(a0), lo_(a0));
      y1[1] = __fsub_rn(hi_(a1), lo_(a1));
    }
  };
  // lines of the three directions from this thread's values v[b][a] of one
  // field per direction
  auto publish = [&](u64 *Ar, float (&vr)[2][2], float (&vs)[2][2], float (&vt)[2][2])
                     __attribute__((always_inline)) {
    u64 *As = Ar + C::DE, *At = As + C::DE;
    // j-pairs: this thread forms the s-line entries at b = c; it needs the
    // partner's values there, the partner its values at b = 1 - c
    const float o0 = __shfl_xor_sync(0xffffffffu, c ? vs[0][0] : vs[1][0], 1);
    const float o1 = __shfl_xor_sync(0xffffffffu, c ? vs[0][1] : vs[1][1], 1);
    if (real) {
#pragma unroll
      for (int b = 0; b < 2; ++b) Ar[lpos<LX>(lineR(b), ip)] = eo(vr[b][0], vr[b][1]);
#pragma unroll
      for (int a = 0; a < 2; ++a) At[lpos<LX>(lineT(a), kp)] = eo(vt[0][a], vt[1][a]);
      As[lpos<LX>(lineS(c, 0), jp)] = c ? eo(o0, vs[1][0]) : eo(vs[0][0], o0);
      As[lpos<LX>(lineS(c, 1), jp)] = c ? eo(o1, vs[1][1]) : eo(vs[0][1], o1);
    }
  };
  // coefficient rows ip (r), kp (t), jp (s) of both matrices (kCoefRegs)
  u64 creg[2][3][H];
  auto contract_all = [&](const u64 *Ar, int m, bool gen, float (&yr)[2][2], float (&ys)[2][2],
                          float (&yt)[2][2]) __attribute__((always_inline)) {
    const u64 *cof = cf + m * 2 * H2;
    const u64 *As = Ar + C::DE, *At = As + C::DE;
    {  // r: lines (k_b, j_c), outputs at i', N - i'
      float y0[2], y1[2];
      contract2(Ar, lineR(0), lineR(1), cof, gen, ip, creg[m][0], y0, y1);
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        yr[b][0] = y0[b];
        yr[b][1] = y1[b];
      }
    }
    {  // t: lines (j_c, i_a), outputs at k', N - k'
      float y0[2], y1[2];
      contract2(At, lineT(0), lineT(1), cof, gen, kp, creg[m][1], y0, y1);
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        yt[0][a] = y0[a];
        yt[1][a] = y1[a];
      }
    }
    {  // s: lines (k_c, i_a), outputs at j', N - j'; keep this thread's j,
       // send the other to the partner, which owns it at k_c
      float y0[2], y1[2];
      contract2(As, lineS(c, 0), lineS(c, 1), cof, gen, jp, creg[m][2], y0, y1);
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const float own = c ? y1[a] : y0[a];
        const float recv = __shfl_xor_sync(0xffffffffu, c ? y0[a] : y1[a], 1);
        ys[0][a] = c ? recv : own;
        ys[1][a] = c ? own : recv;
      }
    }
  };
  // this thread's two values (a = 0, 1) of row (k_b, j_c) of one staged
  // field.  bf16 at lx = 8: the two 32-bit words holding i' and N - i', each
  // value moved into the high half of an fp32 word by one byte permute.
  // Otherwise the thread with c = 1 reads N - i' first: rows j and j + 4 of
  // a plane share banks at lx = 8, and this way the two halves of the warp
  // read different column halves in each load.
  const unsigned wsel0 = (ip & 1) ? 0x3244u : 0x1044u;  // value -> high half, zeros below
  const unsigned wsel1 = (ip & 1) ? 0x1044u : 0x3244u;  // (N - i' has the other parity)
  auto row_pair = [&](const auto *F, int b, float &x0, float &x1) __attribute__((always_inline)) {
    using S = std::remove_cv_t<std::remove_pointer_t<decltype(F)>>;
    const int r = real ? (kb(b) * LX + jc) * LX : 0;
    if constexpr (std::is_same_v<S, __nv_bfloat16> && LX == 8) {
      const unsigned *wr = reinterpret_cast<const unsigned *>(F + r);
      const unsigned w0 = wr[ip >> 1], w1 = wr[3 - (ip >> 1)];
      x0 = __uint_as_float(__byte_perm(w0, 0u, wsel0));
      x1 = __uint_as_float(__byte_perm(w1, 0u, wsel1));
    } else {
      const int i0 = real ? (c ? N - ip : ip) : 0, i1 = real ? (c ? ip : N - ip) : 0;
      const float f0 = ldf(F + r + i0), f1 = ldf(F + r + i1);
      x0 = c ? f1 : f0;
      x1 = c ? f0 : f1;
    }
  };
  // the even-odd coefficients of one mesh's matrices; returns true when a
  // matrix is not centro-antisymmetric (rows N - i need their own chain)
  auto load_coef = [&](const Mesh<SU, SG> &M) __attribute__((always_inline)) {
    sync();  // every thread is done with the previous coefficients
    bool ok = true;
    for (int q = tid; q < 2 * H2; q += C::NTB) {
      const int m = q / H2, i = (q / H) % H, l = q % H;
      const float *D = m ? M.dxt : M.dx;  // M(i, l) = D[l * lx + i]
      const float a = __ldg(D + l * LX + i), b = __ldg(D + (N - l) * LX + i);
      const float a2 = __ldg(D + l * LX + N - i), b2 = __ldg(D + (N - l) * LX + N - i);
      const float A = __fmul_rn(0.5f, __fadd_rn(a, b)), B = __fmul_rn(0.5f, __fsub_rn(a, b));
      const float A2 = __fmul_rn(0.5f, __fadd_rn(a2, b2));
      const float B2 = __fmul_rn(0.5f, __fsub_rn(a2, b2));
      cf[m * 2 * H2 + i * H + l] = pk(A, B);
      cf[m * 2 * H2 + H2 + i * H + l] = pk(A2, B2);
      ok = ok && A2 == -A && B2 == B;
    }
    const bool gen = !sync_and(ok);
    if constexpr (kCoefRegs) {
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int l = 0; l < H; ++l) {
          creg[m][0][l] = cf[m * 2 * H2 + ip * H + l];
          creg[m][1][l] = cf[m * 2 * H2 + kp * H + l];
          creg[m][2][l] = cf[m * 2 * H2 + jp * H + l];
        }
    }
    return gen;
  };
  // one thread: bulk copies of element p's u and geometry into stage `buf`
  auto issue = [&](const EopPos &p, int buf) __attribute__((always_inline)) {
    const Mesh<SU, SG> &M = seq.mesh(seq.mesh_of(p));
    const size_t eo = (size_t)seq.elem(p) * N3;
    const uint32_t bar = bar0 + 8u * (uint32_t)buf;
    const uint32_t dst = eop::smem_u32(stg + (size_t)buf * C::SBYTES);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(C::TXBYTES)
                 : "memory");
    auto copy = [&](uint32_t d, const void *src, uint32_t bytes) __attribute__((always_inline)) {
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
          "[%3];" ::"r"(d),
          "l"(src), "r"(bytes), "r"(bar)
          : "memory");
    };
    if constexpr (PUPD) {
      copy(dst, up.r + eo, C::UBYTES);
      copy(dst + C::UBYTES, up.minv + eo, C::UBYTES);
      copy(dst + 2 * C::UBYTES, up.pw + eo, C::UBYTES);
    } else {
      copy(dst, M.u + eo, C::UBYTES);
    }
#pragma unroll
    for (int f = 0; f < 7; ++f)
      copy(dst + C::NU * C::UBYTES + f * C::GFBYTES, M.g[f] + eo, C::GFBYTES);
  };

  if (tid == 0) {
    eop::mbar_init(bar0, 1);
    eop::mbar_init(bar0 + 8, 1);
  }
  EopPos pos;
  bool have = seq.first(pos);
  sync();  // the barriers are initialised before anyone waits on them
  if (tid == 0 && have) issue(pos, 0);

  const float beta = PUPD ? (float)*up.beta : 0.f;  // the solver's scalar, on the device
  unsigned n = 0;  // elements done by this group
  while (have) {
    const int cmesh = seq.mesh_of(pos);
    const bool gen = load_coef(seq.mesh(cmesh));
    for (; have && seq.mesh_of(pos) == cmesh; ++n) {
      EopPos nxp;
      const bool more = seq.advance(pos, nxp);
      const int buf = (int)(n & 1u);
      const uint32_t par = (n >> 1) & 1u;
      // stage buf ^ 1 was last read by the previous element, before its
      // second barrier (which this thread has passed)
      if (tid == 0 && more) {
        eop::fence_async_smem();
        issue(nxp, buf ^ 1);
      }
      const Mesh<SU, SG> &M = seq.mesh(cmesh);
      const size_t eb = (size_t)seq.elem(pos) * N3;
      const unsigned char *st = stg + (size_t)buf * C::SBYTES;
      const SU *U = reinterpret_cast<const SU *>(st);
      const SG *G = reinterpret_cast<const SG *>(st + C::NU * C::UBYTES);
      u64 *LA = Lb, *LB = Lb + C::SETE;  // gradient and weighted-gradient lines

      // ---- phase 1: this element's u, lines of the three directions
      const bool got = eop::mbar_wait(bar0 + 8u * (uint32_t)buf, par, eop::kWaitLimit);
      float v[2][2];
#pragma unroll
      for (int b = 0; b < 2; ++b) row_pair(U, b, v[b][0], v[b][1]);
      if constexpr (PUPD) {  // v = r here: p = minv .* r + beta p, stored
        const float *Mi = reinterpret_cast<const float *>(st + C::UBYTES);
        const float *Po = reinterpret_cast<const float *>(st + 2 * C::UBYTES);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          float mi[2], po[2];
          row_pair(Mi, b, mi[0], mi[1]);
          row_pair(Po, b, po[0], po[1]);
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            v[b][a] = __fmaf_rn(mi[a], v[b][a], __fmul_rn(beta, po[a]));
            if (real) up.pw[eb + pidx(b, a)] = v[b][a];
          }
        }
      }
      publish(LA, v, v, v);
      if (!sync_and(got)) {
        // a staged copy never completed: record it, write NaN into this
        // group's remaining elements (so that the failure cannot pass
        // unnoticed where no status word is given) and stop (group-uniform);
        // copies may still be in flight, so wait for them once more, bounded
        if (tid == 0) {
          if (err) atomicExch(err, 1);
          (void)eop::mbar_wait(bar0 + 8u * (uint32_t)buf, par, eop::kWaitLimit);
          if (more)
            (void)eop::mbar_wait(bar0 + 8u * (uint32_t)(buf ^ 1), ((n + 1) >> 1) & 1u,
                                 eop::kWaitLimit);
        }
        for (EopPos p = pos;;) {
          float *wp = seq.mesh(seq.mesh_of(p)).w + (size_t)seq.elem(p) * N3;
          for (int q = tid; q < N3; q += C::NTB) wp[q] = __int_as_float(0x7fc00000);
          EopPos p2;
          if (!seq.advance(p, p2)) break;
          p = p2;
        }
        have = false;
        break;
      }

      // ---- phase 2: reference gradient
      float gr[2][2], gs[2][2], gt[2][2];
      contract_all(LA, 0, gen, gr, gs, gt);

      // ---- phase 3: pointwise h1 G
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        float h[2], g11[2], g22[2], g33[2], g12[2], g13[2], g23[2];
        row_pair(G, b, h[0], h[1]);
        row_pair(G + N3, b, g11[0], g11[1]);
        row_pair(G + 2 * N3, b, g22[0], g22[1]);
        row_pair(G + 3 * N3, b, g33[0], g33[1]);
        row_pair(G + 4 * N3, b, g12[0], g12[1]);
        row_pair(G + 5 * N3, b, g13[0], g13[1]);
        row_pair(G + 6 * N3, b, g23[0], g23[1]);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const float ur = gr[b][a], us = gs[b][a], ut = gt[b][a];
          gr[b][a] = __fmul_rn(
              h[a], __fmaf_rn(g13[a], ut, __fmaf_rn(g12[a], us, __fmul_rn(g11[a], ur))));
          gs[b][a] = __fmul_rn(
              h[a], __fmaf_rn(g23[a], ut, __fmaf_rn(g22[a], us, __fmul_rn(g12[a], ur))));
          gt[b][a] = __fmul_rn(
              h[a], __fmaf_rn(g33[a], ut, __fmaf_rn(g23[a], us, __fmul_rn(g13[a], ur))));
        }
      }

      // ---- phase 4: lines of the weighted gradient (set B: its last
      // readers, the previous element's phase 5, are behind this element's
      // first barrier)
      publish(LB, gr, gs, gt);
      sync();

      // ---- phase 5: transposed contractions, summed, stored
      contract_all(LB, 1, gen, gr, gs, gt);
      if (real) {
        float el = 0.f;
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            const float wv = __fadd_rn(__fadd_rn(gr[b][a], gs[b][a]), gt[b][a]);
            M.w[eb + pidx(b, a)] = wv;
            if constexpr (DOT) el = __fmaf_rn(v[b][a], wv, el);
          }
        if constexpr (DOT) dsum += (double)el;
      }
      pos = nxp;
      have = more;
    }
  }
  sync();  // every wait has returned
  if (tid == 0) {  // no copy is pending here: the barriers may be reused as plain memory
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar0 + 8) : "memory");
  }
}

// One mesh, elements blockIdx.x + k gridDim.x.  DOT: one partial of u . w
// per CTA (fixed order) in dotp[blockIdx.x].
template <int LX, class SU, class SG, bool DOT, bool PUPD = false>
__global__ void __launch_bounds__(Cfg<LX, SU, SG>::NTB, (minb<LX, SU, SG>()))
ax_eo32_kernel(const Mesh<SU, SG> mesh, long long nelv, int *__restrict__ err,
               double *__restrict__ dotp, const E32Upd up) {
  using C = Cfg<LX, SU, SG, PUPD>;
  extern __shared__ __align__(128) unsigned char sm[];
  const SeqOne<SU, SG> seq{mesh, nelv};
  double dsum = 0.0;
  e32_run<LX, SU, SG, DOT, PUPD, kE32CoefRegs>(
      sm, (int)threadIdx.x, seq, [] { __syncthreads(); },
      [](bool p) { return __syncthreads_and(p) != 0; }, err, dsum, up);
  if constexpr (DOT) {  // one partial per CTA: fixed shuffle tree, warps in order
    double *red = reinterpret_cast<double *>(sm + C::OFF_MISC + 16);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int q = 0; q < C::NW; ++q) s += red[q];
      dotp[blockIdx.x] = s;
    }
  }
}

}  // namespace e32
}  // namespace ax

// ---------------------------------------------------------------------------
// Host side (instantiated by ax_eo32_*.cu).
#include <algorithm>
#include <atomic>

namespace ax {
namespace e32 {

// Resident CTAs of one kernel variant on the current device times its SMs
// (cached per device; the shared-memory limit is raised on first use).
template <int LX, class SU, class SG, bool DOT, bool PUPD>
int grid() {
  using C = Cfg<LX, SU, SG, PUPD>;
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return 0;
  }
  int g = cache[dev].load(std::memory_order_acquire);
  if (g > 0) return g;
  auto kern = ax_eo32_kernel<LX, SU, SG, DOT, PUPD>;
  int sms = 0, bps = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, C::NTB, C::SMEM) != cudaSuccess ||
      bps < 1) {
    (void)cudaGetLastError();
    return 0;
  }
  g = sms * bps;
  cache[dev].store(g, std::memory_order_release);
  return g;
}

// CTAs (and dot partials) of a launch over nelv elements: every variant of a
// storage pair launches the same grid, so that a solver sizes its partials
// once.
template <int LX, class SU, class SG>
int blocks(long long nelv) {
  int g = std::min(grid<LX, SU, SG, true, false>(), grid<LX, SU, SG, false, false>());
  if constexpr (std::is_same_v<SU, float>) g = std::min(g, grid<LX, SU, SG, true, true>());
  return g <= 0 ? 0 : (int)std::min<long long>(g, std::max(nelv, 1LL));
}

template <int LX, class SU, class SG>
int launch(float *w, const SU *u, const float *dx, const float *dxt, const SG *const g[7],
           int nelv, int *err, double *dotp, cudaStream_t st, const E32Upd *up) {
  const int nb = blocks<LX, SU, SG>(nelv);
  if (nb <= 0) return AX_ELAUNCH;
  Mesh<SU, SG> m;
  m.w = w;
  m.u = u;
  for (int f = 0; f < 7; ++f) m.g[f] = g[f];
  m.dx = dx;
  m.dxt = dxt;
  const E32Upd none{};
  if (up) {
    if constexpr (std::is_same_v<SU, float>) {
      if (!dotp || !up->pw || !up->r || !up->minv || !up->beta) return AX_EINVAL;
      using C = Cfg<LX, SU, SG, true>;
      ax_eo32_kernel<LX, SU, SG, true, true><<<nb, C::NTB, C::SMEM, st>>>(m, nelv, err, dotp,
                                                                          *up);
    } else {
      return AX_EINVAL;
    }
  } else if (dotp) {
    using C = Cfg<LX, SU, SG>;
    ax_eo32_kernel<LX, SU, SG, true><<<nb, C::NTB, C::SMEM, st>>>(m, nelv, err, dotp, none);
  } else {
    using C = Cfg<LX, SU, SG>;
    ax_eo32_kernel<LX, SU, SG, false><<<nb, C::NTB, C::SMEM, st>>>(m, nelv, err, dotp, none);
  }
  return launch_status();
}

}  // namespace e32
}  // namespace ax
