// fp64-accurate element operator (Listing 2) with the even-odd split of the
// 1-D contractions, for even lx.
//
// The GLL differentiation matrix is centro-antisymmetric,
// D[N-i][N-l] = -D[i][l] (N = lx-1), and so is its transpose.  With
// e_l = v_l + v_{N-l} and o_l = v_l - v_{N-l} (l < lx/2), a contraction
// y = D v splits into two half-size ones (Solomonoff 1992, "A fast algorithm
// for spectral differentiation"):
//   E_i = sum_l P_il e_l,  O_i = sum_l M_il o_l,   P = (D_il + D_i,N-l)/2,
//   M = (D_il - D_i,N-l)/2,  y_i = O_i + E_i,  y_{N-i} = O_i - E_i,
// halving the multiply-adds, which dominate the double-float cost.  E and O
// run as the two lanes of packed f32x2 double-float arithmetic (df64.cuh),
// so one packed step advances both half-size sums.
//
// Mapping: an element gets (lx/2)^3 threads; thread (i',j',k') owns the
// eight points {i',N-i'} x {j',N-j'} x {k',N-k'}, so every pair that the
// split needs sits in one thread.  Each thread forms (e, o) of its own
// values for all three directions and publishes them to shared memory as
// one 16-byte entry {e.hi, o.hi, e.lo, o.lo} per pair (one padded line per
// (outer, middle) index and direction); the contractions read whole lines
// back, broadcast across the threads sharing a line.  The same happens for
// the geometry-weighted gradient before the transposed contractions.  No
// fp64 instruction is issued.
//
// The geometry of the pointwise step comes either from the fp64 arrays
// (split on the fly, one point at a time) or from a prepared copy in this
// kernel's own order (eo_prepare_kernel), which the pointwise step consumes
// two points at a time (a = 0, 1: i' and N-i') as the two lanes of packed
// double-float arithmetic.  The prepared order is, per element, per
// corner pair (c, b), per field (g11, g22, g33, g12, g13, g23, h1), per
// thread, one 16-byte entry {hi(a=0), hi(a=1), lo(a=0), lo(a=1)}: the same
// 8 bytes per value and the same split, but no conversion instructions and
// coalesced 16-byte loads.  (The packed pointwise step rounds its tail sums
// in another order than the scalar one, so the two paths agree to ~1e-16
// relative, not bit for bit.)
#pragma once

#include <algorithm>

#include "common.cuh"
#include "df64.cuh"
#include "guard.cuh"

namespace ax {

namespace eo {

template <int LX>
constexpr int line_stride() {  // entries per line (16 B each), padded
  return LX / 2 + 1;
}
template <int LX>
constexpr int dir_entries() {
  return LX * LX * line_stride<LX>();
}

// 16-byte entries of one element's prepared geometry
template <int LX>
constexpr int prep_entries() {
  return 4 * 7 * (LX / 2) * (LX / 2) * (LX / 2);
}

// geometry in flight: 7 fields of one corner (fp64 arrays) or of one corner
// pair (prepared)
template <bool PREP>
struct GeoStage;
template <>
struct GeoStage<false> {
  double v[7];
};
template <>
struct GeoStage<true> {
  df::dd2 v[7];
};

}  // namespace eo

template <int LX>
constexpr size_t df64eo_smem(int epb) {
  // coefficients of D and D^T: (lx/2)^2 dd2 + (lx/2)^2 negated heads each;
  // three direction arrays of dd2 entries per element
  constexpr size_t H2 = (size_t)(LX / 2) * (LX / 2);
  return 2 * H2 * (16 + 8) + (size_t)epb * 3 * eo::dir_entries<LX>() * 16;
}

// PUPD (prepared geometry only): u is not an input; instead the kernel first
// forms the solver's next search direction in place, pw = z + (*beta) pw
// with z = minv .* r (+ corr when *use_corr, the flexible CG's learned
// step), in fp64 with explicit roundings, and applies the operator to it.
template <int LX, bool PREP = false, bool PUPD = false, bool NBAR = true>
__device__ __forceinline__ void df64eo_body(double *__restrict__ w, const double *__restrict__ u,
                                            const double *__restrict__ dx,
                                            const double *__restrict__ dxt,
                                            const double *__restrict__ h1,
                                            const double *__restrict__ g11,
                                            const double *__restrict__ g22,
                                            const double *__restrict__ g33,
                                            const double *__restrict__ g12,
                                            const double *__restrict__ g13,
                                            const double *__restrict__ g23,
                                            const df::dd2 *__restrict__ gp,
                                            const unsigned *__restrict__ gstat, long long e0,
                                            int nel, int epb, unsigned char *smem_raw,
                                            double *__restrict__ dotp = nullptr,
                                            double *__restrict__ pw = nullptr,
                                            const double *__restrict__ r_in = nullptr,
                                            const double *__restrict__ minv_in = nullptr,
                                            const double *__restrict__ beta_p = nullptr,
                                            const double *__restrict__ corr_in = nullptr,
                                            const int *__restrict__ use_corr_p = nullptr) {
  static_assert(LX % 2 == 0, "even-odd kernel needs an even lx");
  using namespace df;
  constexpr int H = LX / 2, N = LX - 1;
  constexpr int H2 = H * H, H3 = H2 * H;
  constexpr int N3 = LX * LX * LX;
  constexpr int LS = eo::line_stride<LX>();
  constexpr int DE = eo::dir_entries<LX>();

  dd2 *cf = reinterpret_cast<dd2 *>(smem_raw);  // [H][H] (P, M) of D
  dd2 *tf = cf + H2;                            // [H][H] (P, M) of D^T
  u64 *cn = reinterpret_cast<u64 *>(tf + H2);   // -heads of cf
  u64 *tn = cn + H2;                            // -heads of tf
  const bool own = (int)threadIdx.x < epb * H3;
  const int le = own ? (int)threadIdx.x / H3 : 0;
  const int t = (int)threadIdx.x - le * H3;
  const int ip = t % H, jp = (t / H) % H, kp = t / H2;
  dd2 *Ar = reinterpret_cast<dd2 *>(tn + H2) + (size_t)le * 3 * DE;  // lines [k][j]
  dd2 *As = Ar + DE;                                                    // lines [k][i]
  dd2 *At = As + DE;                                                    // lines [j][i]

  // range record of this block (guard.cuh), cleared before any thread notes
  __shared__ guard::Record rec;
  guard::clear(rec, epb);
  __syncthreads();

  // coefficients (dx[l*LX+i] = D_il, dxt[l*LX+i] = D_li); every entry of
  // both matrices is also checked against its centro-antisymmetric mirror
  for (int q = threadIdx.x; q < H2; q += blockDim.x) {
    const int i = q / H, l = q % H;
#pragma unroll
    for (int tr = 0; tr < 2; ++tr) {
      const double *m = tr ? dxt : dx;
      const double da = __ldg(m + l * LX + i), db = __ldg(m + (N - l) * LX + i);
      guard::note_pair(rec, da, __ldg(m + (N - l) * LX + (N - i)));
      guard::note_pair(rec, db, __ldg(m + l * LX + (N - i)));
      const df2 a = split(da), b = split(db);
      // lanes: x = (a + b)/2, y = (a - b)/2 (exact halving)
      dd2 s = dsum2(dd2{pk(a.hi, a.hi), pk(a.lo, a.lo)}, dd2{pk(b.hi, -b.hi), pk(b.lo, -b.lo)});
      const df2 P = norm(lx_(s.hi), lx_(s.lo)), M = norm(ly_(s.hi), ly_(s.lo));
      const dd2 c{pk(0.5f * P.hi, 0.5f * M.hi), pk(0.5f * P.lo, 0.5f * M.lo)};
      (tr ? tf : cf)[q] = c;
      (tr ? tn : cn)[q] = pk(-0.5f * P.hi, -0.5f * M.hi);
    }
  }

  // Phase barriers: with whole warps per element, every thread of the block
  // owning an element and at least four elements, each element synchronises
  // on its own named barrier, so the elements of a block do not wait for one
  // another (measured: faster with four elements per block, slower with two,
  // where the extra block barrier for the coefficients costs more).
  const bool elem_bar =
      NBAR && (H3 % 32 == 0) && (int)blockDim.x == epb * H3 && epb >= 4 && epb <= 8;
  auto phase_sync = [&]() {
    if (elem_bar)
      asm volatile("bar.sync %0, %1;" ::"r"(1 + le), "r"(H3) : "memory");
    else
      __syncthreads();
  };
  if (elem_bar) __syncthreads();  // the coefficients above are shared by all elements

  const bool active = own && le < nel;
  const size_t eb = (size_t)(active ? e0 + le : 0) * N3;
  // the geometry of this element is read only in phase 3: start it towards L2 now
  const size_t ep = (size_t)(active ? e0 + le : 0) * eo::prep_entries<LX>();
  if (active && t < 7) {
    if constexpr (PREP) {  // the element's prepared block, in 7 equal pieces
      prefetch_l2(gp + ep + (size_t)t * (eo::prep_entries<LX>() / 7),
                  (unsigned)(N3 * sizeof(double)));
    } else {
      const double *f = t == 0 ? g11 : t == 1 ? g22 : t == 2 ? g33 : t == 3 ? g12
                      : t == 4 ? g13 : t == 5 ? g23 : h1;
      prefetch_l2(f + eb, (unsigned)(N3 * sizeof(double)));
    }
  }
  auto gidx = [&](int c, int b, int a) {
    const int k = c ? N - kp : kp, j = b ? N - jp : jp, i = a ? N - ip : ip;
    return eb + (size_t)((k * LX + j) * LX + i);
  };
  auto lr = [&](int c, int b) { return ((c ? N - kp : kp) * LX + (b ? N - jp : jp)) * LS; };
  auto ls = [&](int c, int a) { return ((c ? N - kp : kp) * LX + (a ? N - ip : ip)) * LS; };
  auto lt = [&](int b, int a) { return ((b ? N - jp : jp) * LX + (a ? N - ip : ip)) * LS; };
  // (v0 + v1, v0 - v1) as one entry
  auto eo_pair = [](df2 v0, df2 v1) {
    return dsum2(dd2{pk(v0.hi, v0.hi), pk(v0.lo, v0.lo)},
                 dd2{pk_pm(v1.hi), pk_pm(v1.lo)});
  };
  auto publish = [&](df2 (&v)[2][2][2]) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b) Ar[lr(c, b) + ip] = eo_pair(v[c][b][0], v[c][b][1]);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int a = 0; a < 2; ++a) As[ls(c, a) + jp] = eo_pair(v[c][0][a], v[c][1][a]);
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) At[lt(b, a) + kp] = eo_pair(v[0][b][a], v[1][b][a]);
  };
  // half-size contractions of one line: (y at row, y at N-row)
  auto contract = [&](const dd2 *line, const dd2 *cof, const u64 *nco, int row, df2 &y_lo,
                      df2 &y_hi) {
    acc2 a = prod2(cof[row * H], nco[row * H], line[0]);
#pragma unroll
    for (int l = 1; l < H; ++l) mac2(a, cof[row * H + l], nco[row * H + l], line[l]);
    // lanes: x = E, y = O.  (O + E, O - E) in one packed sum
    const float Es = lx_(a.s), Ec = lx_(a.c), Os = ly_(a.s), Oc = ly_(a.c);
    const dd2 r = dsum2(dd2{pk(Os, Os), pk(Oc, Oc)}, dd2{pk_pm(Es), pk_pm(Ec)});
    y_lo = df2{lx_(r.hi), lx_(r.lo)};
    y_hi = df2{ly_(r.hi), ly_(r.lo)};
  };

  df2 gr[2][2][2], gs_[2][2][2], gt[2][2][2];
  unsigned ukey = 0u, gkey = 0u, hkey = 0u;  // exponent keys of u, G, h1 (guard.cuh)
  // ---- phase 1: own values of u, (e, o) along each direction
  if (own) {
    if constexpr (PUPD) {
      const double beta = *beta_p;
      // flexible CG: z = minv r + corr when its step took the correction
      const bool uc = corr_in != nullptr && *use_corr_p != 0;
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            gr[c][b][a] = df2{0.f, 0.f};
            if (active) {
              const size_t q = gidx(c, b, a);
              double z = __dmul_rn(__ldg(minv_in + q), __ldg(r_in + q));
              if (uc) z = __dadd_rn(z, __ldg(corr_in + q));
              const double pn = __fma_rn(beta, pw[q], z);
              pw[q] = pn;
              ukey = max(ukey, guard::key(pn));
              gr[c][b][a] = split(pn);
            }
          }
    } else {
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            const double x = active ? __ldg(u + gidx(c, b, a)) : 0.0;
            ukey = max(ukey, guard::key(x));
            gr[c][b][a] = split(x);
          }
    }
    if (active) atomicMax(&rec.ex[le][0], ukey);
    publish(gr);
  }
  phase_sync();

  // geometry of corner pair q = (c, b) (prepared) or of corner q = (c, b, a)
  // (fp64 arrays); two in flight
  auto load_geo = [&](int q, eo::GeoStage<PREP> &g) {
    if constexpr (PREP) {
      const dd2 *src = gp + ep + (size_t)q * 7 * H3 + t;
#pragma unroll
      for (int f = 0; f < 7; ++f) {
        const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(src + (size_t)f * H3));
        g.v[f] = dd2{v.x, v.y};
      }
    } else {
      const size_t x = gidx((q >> 2) & 1, (q >> 1) & 1, q & 1);
      const double *fld[7] = {g11, g22, g33, g12, g13, g23, h1};
#pragma unroll
      for (int f = 0; f < 7; ++f) g.v[f] = __ldg(fld[f] + x);
    }
  };
  eo::GeoStage<PREP> geo[2];
  if (active) load_geo(0, geo[0]);

  // ---- phase 2: reference gradient at the eight points
  if (own) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b) contract(Ar + lr(c, b), cf, cn, ip, gr[c][b][0], gr[c][b][1]);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int a = 0; a < 2; ++a)
        contract(As + ls(c, a), cf, cn, jp, gs_[c][0][a], gs_[c][1][a]);
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) contract(At + lt(b, a), cf, cn, kp, gt[0][b][a], gt[1][b][a]);
  }

  // ---- phase 3: pointwise h1 G, the next geometry loading meanwhile
  if constexpr (PREP) {  // point pairs a = 0, 1 as packed lanes
    if (active && t == 0) {  // the geometry's exponent keys, recorded when it was prepared
      atomicMax(&rec.ex[le][1], __ldg(gstat + 2 * (e0 + le)));
      atomicMax(&rec.ex[le][2], __ldg(gstat + 2 * (e0 + le) + 1));
    }
    if (own) {
      const u64 zero = pk(0.f, 0.f);
#pragma unroll
      for (int cp = 0; cp < 4; ++cp) {
        const int c = cp >> 1, b = cp & 1;
        if (active && cp + 1 < 4) load_geo(cp + 1, geo[(cp + 1) & 1]);
        dd2 WR{zero, zero}, WS{zero, zero}, WT{zero, zero};
        if (active) {
          const eo::GeoStage<PREP> &g = geo[cp & 1];
          const dd2 UR{pk(gr[c][b][0].hi, gr[c][b][1].hi), pk(gr[c][b][0].lo, gr[c][b][1].lo)};
          const dd2 US{pk(gs_[c][b][0].hi, gs_[c][b][1].hi),
                       pk(gs_[c][b][0].lo, gs_[c][b][1].lo)};
          const dd2 UT{pk(gt[c][b][0].hi, gt[c][b][1].hi), pk(gt[c][b][0].lo, gt[c][b][1].lo)};
          const u64 nR = neg2(UR.hi), nS = neg2(US.hi), nT = neg2(UT.hi);
          const dd2 &G11 = g.v[0], &G22 = g.v[1], &G33 = g.v[2];
          const dd2 &G12 = g.v[3], &G13 = g.v[4], &G23 = g.v[5], &HH = g.v[6];
          const u64 nH = neg2(HH.hi);
          acc2 a = prod2(UR, nR, G11);
          mac2(a, US, nS, G12);
          mac2(a, UT, nT, G13);
          acc2 m = prod2(HH, nH, dd2{a.s, a.c});
          WR = dd2{m.s, m.c};
          a = prod2(UR, nR, G12);
          mac2(a, US, nS, G22);
          mac2(a, UT, nT, G23);
          m = prod2(HH, nH, dd2{a.s, a.c});
          WS = dd2{m.s, m.c};
          a = prod2(UR, nR, G13);
          mac2(a, US, nS, G23);
          mac2(a, UT, nT, G33);
          m = prod2(HH, nH, dd2{a.s, a.c});
          WT = dd2{m.s, m.c};
        }
        gr[c][b][0] = df2{lx_(WR.hi), lx_(WR.lo)};
        gr[c][b][1] = df2{ly_(WR.hi), ly_(WR.lo)};
        gs_[c][b][0] = df2{lx_(WS.hi), lx_(WS.lo)};
        gs_[c][b][1] = df2{ly_(WS.hi), ly_(WS.lo)};
        gt[c][b][0] = df2{lx_(WT.hi), lx_(WT.lo)};
        gt[c][b][1] = df2{ly_(WT.hi), ly_(WT.lo)};
      }
    }
  } else {  // one point at a time, geometry split on the fly
    if (own) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = (q >> 2) & 1, b = (q >> 1) & 1, a = q & 1;
        if (active && q + 1 < 8) load_geo(q + 1, geo[(q + 1) & 1]);
        df2 wr{0.f, 0.f}, ws{0.f, 0.f}, wt{0.f, 0.f};
        if (active) {
          const double(&g)[7] = geo[q & 1].v;
#pragma unroll
          for (int f = 0; f < 6; ++f) gkey = max(gkey, guard::key(g[f]));
          hkey = max(hkey, guard::key(g[6]));
          const df2 a11 = split(g[0]), a22 = split(g[1]), a33 = split(g[2]);
          const df2 a12 = split(g[3]), a13 = split(g[4]), a23 = split(g[5]);
          const df2 hh = split(g[6]);
          const df2 ur = gr[c][b][a], us = gs_[c][b][a], ut = gt[c][b][a];
          acc sum = prod(a11, ur);
          mac(sum, a12, us);
          mac(sum, a13, ut);
          wr = mul2(hh, df2{sum.s, sum.c});
          sum = prod(a12, ur);
          mac(sum, a22, us);
          mac(sum, a23, ut);
          ws = mul2(hh, df2{sum.s, sum.c});
          sum = prod(a13, ur);
          mac(sum, a23, us);
          mac(sum, a33, ut);
          wt = mul2(hh, df2{sum.s, sum.c});
        }
        gr[c][b][a] = wr;
        gs_[c][b][a] = ws;
        gt[c][b][a] = wt;
      }
      if (active) {
        atomicMax(&rec.ex[le][1], gkey);
        atomicMax(&rec.ex[le][2], hkey);
      }
    }
  }
  phase_sync();  // every thread of the element has read its gradient lines

  // elements outside the double-float window, or matrices whose mirrored rows
  // the split below would misread, go to fp64 units after phase 5
  const bool bad = active && !(guard::elem_ok(rec, le) && guard::centro_ok(rec));

  // ---- phase 4: (e, o) of the weighted gradient, one direction each
  if (own) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b) Ar[lr(c, b) + ip] = eo_pair(gr[c][b][0], gr[c][b][1]);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int a = 0; a < 2; ++a) As[ls(c, a) + jp] = eo_pair(gs_[c][0][a], gs_[c][1][a]);
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) At[lt(b, a) + kp] = eo_pair(gt[0][b][a], gt[1][b][a]);
  }
  // the phase barrier also tells every thread whether its element (named
  // barriers) or block (block barrier) holds an element for the fallback
  bool any_bad;
  if (elem_bar) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)bad), "r"(1 + le), "r"(H3)
        : "memory");
    any_bad = r != 0u;
  } else {
    any_bad = __syncthreads_or(bad) != 0;
  }

  double dsum = 0.0;
  // ---- phase 5: transposed half-size contractions, summed, stored
  if (own) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b) contract(Ar + lr(c, b), tf, tn, ip, gr[c][b][0], gr[c][b][1]);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int a = 0; a < 2; ++a)
        contract(As + ls(c, a), tf, tn, jp, gs_[c][0][a], gs_[c][1][a]);
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) contract(At + lt(b, a), tf, tn, kp, gt[0][b][a], gt[1][b][a]);
    if (active && !bad) {
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          // points a = 0, 1 as the two lanes
          const df2 r0 = gr[c][b][0], r1 = gr[c][b][1];
          const df2 s0 = gs_[c][b][0], s1 = gs_[c][b][1];
          const df2 t0 = gt[c][b][0], t1 = gt[c][b][1];
          dd2 acc = dsum2(dd2{pk(r0.hi, r1.hi), pk(r0.lo, r1.lo)},
                          dd2{pk(s0.hi, s1.hi), pk(s0.lo, s1.lo)});
          acc = dsum2(acc, dd2{pk(t0.hi, t1.hi), pk(t0.lo, t1.lo)});
          const df2 w0 = norm(lx_(acc.hi), lx_(acc.lo)), w1 = norm(ly_(acc.hi), ly_(acc.lo));
          const double wd0 = join(w0.hi, w0.lo), wd1 = join(w1.hi, w1.lo);
          w[gidx(c, b, 0)] = wd0;
          w[gidx(c, b, 1)] = wd1;
          if (dotp) {  // u . Au of this element (u re-read from L2)
            if constexpr (PUPD) {  // written above by this thread: coherent loads
              dsum = __fma_rn(__ldcg(pw + gidx(c, b, 0)), wd0, dsum);
              dsum = __fma_rn(__ldcg(pw + gidx(c, b, 1)), wd1, dsum);
            } else {
              dsum = __fma_rn(__ldg(u + gidx(c, b, 0)), wd0, dsum);
              dsum = __fma_rn(__ldg(u + gidx(c, b, 1)), wd1, dsum);
            }
          }
        }
    }
  }
  if (any_bad) {  // fp64 units for the flagged elements (element- or block-uniform branch)
    const double *uu = PUPD ? pw : u;
    const int rank = (int)threadIdx.x - le * H3;
    if (elem_bar) {
      auto sync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(1 + le), "r"(H3) : "memory"); };
      sync();  // phase 5 has read the lines that serve as scratch
      guard::element_f64<LX>(true, w, uu, dx, dx, dx, dxt, dxt, dxt, h1, g11, g22, g33, g12, g13, g23,
                             eb, reinterpret_cast<double *>(Ar), rank, H3, sync,
                             dotp ? &dsum : nullptr);
    } else {
      auto sync = [&]() { __syncthreads(); };
      sync();
      // every thread takes part in the barriers; only flagged elements compute
      guard::element_f64<LX>(bad, w, uu, dx, dx, dx, dxt, dxt, dxt, h1, g11, g22, g33, g12,
                                g13, g23, eb, reinterpret_cast<double *>(Ar), own ? rank : 0,
                                H3, sync, dotp ? &dsum : nullptr);
    }
  }
  if (dotp) {  // one partial per block, fixed order (block-uniform branch)
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = dsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int k = 0; k < (int)((blockDim.x + 31) / 32); ++k) s += red[k];
      dotp[blockIdx.x] = s;
    }
  }
}

template <int LX>
__global__ void __launch_bounds__(256)
ax_df64eo_kernel(double *__restrict__ w, const double *__restrict__ u,
                 const double *__restrict__ dx, const double *__restrict__ dxt,
                 const double *__restrict__ h1, const double *__restrict__ g11,
                 const double *__restrict__ g22, const double *__restrict__ g33,
                 const double *__restrict__ g12, const double *__restrict__ g13,
                 const double *__restrict__ g23, int nelv, int epb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long e0 = (long long)blockIdx.x * epb;
  const long long left = nelv - e0;
  const int nel = left < epb ? (int)left : epb;
  df64eo_body<LX, false>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nullptr, nullptr, e0,
                         nel, epb, smem_raw);
}

// Same operator on geometry prepared by eo_prepare_kernel; DOT adds the
// per-block partials of u . w; PUPD forms u = pw = minv .* r + beta pw first
// (see df64eo_body).
template <int LX, bool DOT, bool PUPD = false>
__global__ void __launch_bounds__(256, 2)
ax_df64eo_prep_kernel(double *__restrict__ w, const double *__restrict__ u,
                      const double *__restrict__ dx, const double *__restrict__ dxt,
                      const df::dd2 *__restrict__ gp, const unsigned *__restrict__ gstat,
                      guard::RawGeo raw, int nelv, int epb,
                      double *__restrict__ dotp, double *__restrict__ pw,
                      const double *__restrict__ r_in, const double *__restrict__ minv_in,
                      const double *__restrict__ beta_p, const double *__restrict__ corr_in,
                      const int *__restrict__ use_corr_p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long e0 = (long long)blockIdx.x * epb;
  const long long left = nelv - e0;
  const int nel = left < epb ? (int)left : epb;
  df64eo_body<LX, true, PUPD, false>(w, u, dx, dxt, raw.h1, raw.g11, raw.g22, raw.g33, raw.g12,
                                     raw.g13, raw.g23, gp, gstat, e0, nel, epb, smem_raw,
                                     DOT ? dotp : nullptr, pw, r_in, minv_in, beta_p, corr_in,
                                     use_corr_p);
}

// Prepared geometry: entry ((e*4 + cp)*7 + f)*H3 + t holds field f at the
// two points a = 0, 1 of corner pair cp = (c, b) of thread t, split into
// double-float pairs exactly as the kernel above splits them.  fmask selects
// the fields to (re)write (bit f; bit 6 = h1).  The buffer ends with two
// exponent keys per element (largest of the six G fields, of h1; guard.cuh),
// written by geo_keys_kernel.
template <int LX>
__global__ void eo_prepare_kernel(df::dd2 *__restrict__ gp, const double *__restrict__ h1,
                                  const double *__restrict__ g11,
                                  const double *__restrict__ g22,
                                  const double *__restrict__ g33,
                                  const double *__restrict__ g12,
                                  const double *__restrict__ g13,
                                  const double *__restrict__ g23, int nelv, int fmask) {
  using namespace df;
  constexpr int H = LX / 2, N = LX - 1, H3 = H * H * H, N3 = LX * LX * LX;
  const int64_t total = (int64_t)nelv * eo::prep_entries<LX>();
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(q % H3);
    const int f = (int)((q / H3) % 7);
    if (!((fmask >> f) & 1)) continue;
    const int cp = (int)((q / (7 * H3)) % 4);
    const int64_t e = q / eo::prep_entries<LX>();
    const int ip = t % H, jp = (t / H) % H, kp = t / (H * H);
    const int k = (cp >> 1) ? N - kp : kp, j = (cp & 1) ? N - jp : jp;
    const double *fld = f == 0 ? g11 : f == 1 ? g22 : f == 2 ? g33 : f == 3 ? g12 : f == 4 ? g13
                      : f == 5 ? g23 : h1;
    const size_t row = (size_t)e * N3 + (size_t)(k * LX + j) * LX;
    const df2 a0 = split(fld[row + ip]), a1 = split(fld[row + N - ip]);
    gp[q] = dd2{pk(a0.hi, a1.hi), pk(a0.lo, a1.lo)};
  }
}

template <int LX>
int launch_df64eo(double *w, const double *u, const double *dx, const double *dxt,
                  const double *h1, const double *g11, const double *g22, const double *g33,
                  const double *g12, const double *g13, const double *g23, int nelv, int epb,
                  cudaStream_t stream) {
  constexpr int H3 = (LX / 2) * (LX / 2) * (LX / 2);
  if (epb <= 0) epb = 256 / H3 < 1 ? 1 : 256 / H3;
  if (epb * H3 > 256) return AX_EINVAL;
  const size_t smem = df64eo_smem<LX>(epb);
  auto kern = ax_df64eo_kernel<LX>;
  static std::atomic<size_t> granted[kMaxDevices];
  if (!grant_smem(kern, smem, granted)) return AX_EINVAL;
  const unsigned grid = (unsigned)((nelv + epb - 1) / epb);
  kern<<<grid, epb * H3, smem, stream>>>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nelv,
                                         epb);
  return launch_status();
}

// dotp (optional): one partial of sum u . w per block, gridDim = ceil(nelv /
// epb) of them (prep_blocks).
template <int LX>
int prep_blocks(int nelv, int epb) {
  constexpr int H3 = (LX / 2) * (LX / 2) * (LX / 2);
  if (epb <= 0) epb = 128 / H3 < 1 ? 1 : 128 / H3;
  return (nelv + epb - 1) / epb;
}

// pw (with dotp, r_in, minv_in, beta_p): the fused direction update.
template <int LX>
int launch_df64eo_prep(double *w, const double *u, const double *dx, const double *dxt,
                       const df::dd2 *gp, const guard::RawGeo &raw, int nelv, int epb,
                       cudaStream_t stream,
                       double *dotp = nullptr, double *pw = nullptr,
                       const double *r_in = nullptr, const double *minv_in = nullptr,
                       const double *beta_p = nullptr, const double *corr_in = nullptr,
                       const int *use_corr_p = nullptr) {
  if (pw && !(dotp && r_in && minv_in && beta_p)) return AX_EINVAL;
  if (corr_in && !use_corr_p) return AX_EINVAL;
  constexpr int H3 = (LX / 2) * (LX / 2) * (LX / 2);
  // measured on GB300 (E = 32768 at lx = 8, 13824 at lx = 10): blocks of
  // about 128 threads (4 per SM) beat 256-thread blocks by 8-9 %
  if (epb <= 0) epb = 128 / H3 < 1 ? 1 : 128 / H3;
  if (epb * H3 > 256) return AX_EINVAL;
  const size_t smem = df64eo_smem<LX>(epb);
  const int kind = pw ? 2 : dotp ? 1 : 0;
  auto kern = kind == 2   ? ax_df64eo_prep_kernel<LX, true, true>
              : kind == 1 ? ax_df64eo_prep_kernel<LX, true>
                          : ax_df64eo_prep_kernel<LX, false>;
  static std::atomic<size_t> granted[3][kMaxDevices];
  if (!grant_smem(kern, smem, granted[kind])) return AX_EINVAL;
  const unsigned grid = (unsigned)((nelv + epb - 1) / epb);
  const unsigned *gstat = reinterpret_cast<const unsigned *>(gp + (size_t)nelv * eo::prep_entries<LX>());
  kern<<<grid, epb * H3, smem, stream>>>(w, u, dx, dxt, gp, gstat, raw, nelv, epb, dotp, pw, r_in,
                                         minv_in, beta_p, corr_in, use_corr_p);
  return launch_status();
}

template <int LX>
int launch_eo_prepare(df::dd2 *gp, const double *h1, const double *g11, const double *g22,
                      const double *g33, const double *g12, const double *g13,
                      const double *g23, int nelv, int fmask, cudaStream_t stream) {
  const int64_t total = (int64_t)nelv * eo::prep_entries<LX>();
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
  eo_prepare_kernel<LX><<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, stream>>>(
      gp, h1, g11, g22, g33, g12, g13, g23, nelv, fmask);
  int rc = launch_status();
  if (rc) return rc;
  unsigned *keys = reinterpret_cast<unsigned *>(gp + (size_t)nelv * eo::prep_entries<LX>());
  geo_keys_kernel<<<(unsigned)std::max<int64_t>(((int64_t)nelv + 7) / 8, 1), 256, 0, stream>>>(
      keys, h1, g11, g22, g33, g12, g13, g23, nelv, LX * LX * LX);
  return launch_status();
}

}  // namespace ax
