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
// The geometry of the pointwise step comes from the fp64 arrays, split one
// point at a time (the operator handle's persistent kernel,
// ax_eo_persist.cuh, reads a copy prepared in its own order instead).
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

// geometry in flight: the 7 fields of one corner point
struct GeoStage {
  double v[7];
};

}  // namespace eo

template <int LX>
constexpr size_t df64eo_smem(int epb) {
  // coefficients of D and D^T: (lx/2)^2 dd2 + (lx/2)^2 negated heads each;
  // three direction arrays of dd2 entries per element
  constexpr size_t H2 = (size_t)(LX / 2) * (LX / 2);
  return 2 * H2 * (16 + 8) + (size_t)epb * 3 * eo::dir_entries<LX>() * 16;
}

template <int LX, bool NBAR = true>
__device__ __forceinline__ void df64eo_body(double *__restrict__ w, const double *__restrict__ u,
                                            const double *__restrict__ dx,
                                            const double *__restrict__ dxt,
                                            const double *__restrict__ h1,
                                            const double *__restrict__ g11,
                                            const double *__restrict__ g22,
                                            const double *__restrict__ g33,
                                            const double *__restrict__ g12,
                                            const double *__restrict__ g13,
                                            const double *__restrict__ g23, long long e0,
                                            int nel, int epb, unsigned char *smem_raw) {
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
  if (active && t < 7) {
    const double *f = t == 0 ? g11 : t == 1 ? g22 : t == 2 ? g33 : t == 3 ? g12
                    : t == 4 ? g13 : t == 5 ? g23 : h1;
    prefetch_l2(f + eb, (unsigned)(N3 * sizeof(double)));
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
    {
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

  // geometry of corner q = (c, b, a); two in flight
  auto load_geo = [&](int q, eo::GeoStage &g) {
    const size_t x = gidx((q >> 2) & 1, (q >> 1) & 1, q & 1);
    const double *fld[7] = {g11, g22, g33, g12, g13, g23, h1};
#pragma unroll
    for (int f = 0; f < 7; ++f) g.v[f] = __ldg(fld[f] + x);
  };
  eo::GeoStage geo[2];
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
  {  // one point at a time, geometry split on the fly
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
        }
    }
  }
  if (any_bad) {  // fp64 units for the flagged elements (element- or block-uniform branch)
    const double *uu = u;
    const int rank = (int)threadIdx.x - le * H3;
    if (elem_bar) {
      auto sync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(1 + le), "r"(H3) : "memory"); };
      sync();  // phase 5 has read the lines that serve as scratch
      guard::element_f64<LX>(true, w, uu, dx, dx, dx, dxt, dxt, dxt, h1, g11, g22, g33, g12, g13, g23,
                             eb, reinterpret_cast<double *>(Ar), rank, H3, sync, nullptr);
    } else {
      auto sync = [&]() { __syncthreads(); };
      sync();
      // every thread takes part in the barriers; only flagged elements compute
      guard::element_f64<LX>(bad, w, uu, dx, dx, dx, dxt, dxt, dxt, h1, g11, g22, g33, g12,
                                g13, g23, eb, reinterpret_cast<double *>(Ar), own ? rank : 0,
                                H3, sync, nullptr);
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
  df64eo_body<LX>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, e0, nel, epb, smem_raw);
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

}  // namespace ax
