// Host side of the persistent even-odd operator (ax_eo_persist.cuh): the
// per-lx instantiations, the persistent grid size, the geometry preparation
// and the coefficient block the kernel stages.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ax_eo_persist.cuh"
#include "dispatch.h"

namespace ax {

namespace {

template <int LX, bool DOT, bool PUPD>
auto eop_kernel() {
  return eop::ax_eop_kernel<LX, DOT, PUPD>;
}

// Resident CTAs of one kernel variant on the current device times its SMs
// (cached per device; the shared-memory limit is raised on first use).
template <int LX, bool DOT, bool PUPD>
int eop_grid() {
  using C = eop::Cfg<LX>;
  static std::atomic<int> grid[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return 0;
  }
  int g = grid[dev].load(std::memory_order_acquire);
  if (g > 0) return g;
  auto kern = eop_kernel<LX, DOT, PUPD>();
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
  grid[dev].store(g, std::memory_order_release);
  return g;
}

// The two variants that write dot partials launch the same grid, so that a
// solver sizes its partials once.
template <int LX>
int eop_grid_dot() {
  return std::min(eop_grid<LX, true, false>(), eop_grid<LX, true, true>());
}

template <int LX, bool DOT, bool PUPD>
int eop_launch_t(const EopArgs &a, cudaStream_t st) {
  using C = eop::Cfg<LX>;
  const int g = DOT ? eop_grid_dot<LX>() : eop_grid<LX, DOT, PUPD>();
  if (g <= 0) return AX_ELAUNCH;
  const unsigned grid = (unsigned)std::min<long long>(g, std::max(a.nelv, 1));
  eop::EopMesh m;
  m.w = a.w;
  m.u = a.u;
  m.coef = a.coef;
  m.gp = a.gp;
  m.urange = reinterpret_cast<const uint2 *>(a.gp + (size_t)a.nelv * C::GE);
  m.raw = a.raw;
  m.dx = a.dx;
  m.dxt = a.dxt;
  m.drop = a.drop;
  eop::EopUpd up{a.pw, a.r, a.minv, a.corr, 0.0, false};
  if constexpr (!DOT && !PUPD) {
    if (a.drop >= 0) {  // testing aid: same grid, its own instantiation
      cudaFuncSetAttribute(eop::ax_eop_kernel<LX, false, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
      eop::ax_eop_kernel<LX, false, false, true><<<grid, C::NTB, C::SMEM, st>>>(
          m, (long long)a.nelv, a.err, a.dotp, eop::EopUpd{a.pw, a.r, a.minv, a.corr, 0.0, false},
          a.beta, a.use_corr);
      return launch_status();
    }
  }
  eop::ax_eop_kernel<LX, DOT, PUPD><<<grid, C::NTB, C::SMEM, st>>>(m, (long long)a.nelv, a.err,
                                                                  a.dotp, up, a.beta,
                                                                  a.use_corr);
  return launch_status();
}

template <int LX>
int eop_launch_lx(const EopArgs &a, cudaStream_t st) {
  if (a.pw) return eop_launch_t<LX, true, true>(a, st);
  if (a.dotp) return eop_launch_t<LX, true, false>(a, st);
  return eop_launch_t<LX, false, false>(a, st);
}

// ax_helm on fp64 arrays (RAW body): grid of resident CTAs, cached per device
template <int LX>
int eopr_launch_lx(double *w, const double *u, const double *dx, const double *dxt,
                   const guard::RawGeo &raw, int nelv, cudaStream_t st) {
  using C = eop::Cfg<LX>;
  static std::atomic<int> grid[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  int g = grid[dev].load(std::memory_order_acquire);
  if (g <= 0) {
    auto kern = eop::ax_eopr_kernel<LX>;
    int sms = 0, bps = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, C::NTB, C::SMEM) !=
            cudaSuccess ||
        bps < 1) {
      (void)cudaGetLastError();
      return AX_ELAUNCH;
    }
    g = sms * bps;
    grid[dev].store(g, std::memory_order_release);
  }
  eop::EopMesh m{};
  m.w = w;
  m.u = u;
  m.raw = raw;
  m.dx = dx;
  m.dxt = dxt;
  const unsigned nb = (unsigned)std::min<long long>(g, std::max(nelv, 1));
  eop::ax_eopr_kernel<LX><<<nb, C::NTB, C::SMEM, st>>>(m, (long long)nelv);
  return launch_status();
}

template <int LX>
int eop_blocks_lx(int nelv, bool dot) {
  const int g = dot ? eop_grid_dot<LX>() : eop_grid<LX, false, false>();
  return std::min(g, std::max(nelv, 1));
}

template <int LX>
int eop_prepare_lx(df::dd2 *gp, const guard::RawGeo &r, int nelv, int fmask, int dfield,
                   cudaStream_t st) {
  using C = eop::Cfg<LX>;
  const int64_t total = (int64_t)nelv * C::GE;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
  eop::eop_prepare_kernel<LX><<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(
      gp, r.h1, r.g11, r.g22, r.g33, r.g12, r.g13, r.g23, nelv, fmask);
  int rc = launch_status();
  if (rc) return rc;
  unsigned *keys = reinterpret_cast<unsigned *>(gp + (size_t)nelv * C::GE);
  geo_keys_kernel<<<(unsigned)std::max<int64_t>(((int64_t)nelv + 7) / 8, 1), 256, 0, st>>>(
      keys, r.h1, r.g11, r.g22, r.g33, r.g12, r.g13, r.g23, nelv, LX * LX * LX);
  rc = launch_status();
  if (rc) return rc;
  geo_urange_kernel<<<(unsigned)std::max<int64_t>(((int64_t)nelv + 255) / 256, 1), 256, 0, st>>>(
      keys, nelv, dfield);
  return launch_status();
}

}  // namespace

__global__ void geo_urange_kernel(unsigned *__restrict__ keys, int nelv, int fd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nelv) return;
  unsigned packed, zero_ok;
  guard::u_range(guard::field(keys[2 * e]), guard::field(keys[2 * e + 1]), fd, packed, zero_ok);
  keys[2 * e] = packed;
  keys[2 * e + 1] = zero_ok;
}

bool eop_supported(int lx) { return lx == 6 || lx == 8 || lx == 10 || lx == 12; }

int eopr_launch(int lx, double *w, const double *u, const double *dx, const double *dxt,
                const guard::RawGeo &raw, int nelv, cudaStream_t st) {
  // the bulk copies read whole 16-byte aligned runs of every field
  auto al = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
  if (!(al(raw.h1) && al(raw.g11) && al(raw.g22) && al(raw.g33) && al(raw.g12) &&
        al(raw.g13) && al(raw.g23)))
    return AX_EINVAL;
  switch (lx) {
    case 6: return eopr_launch_lx<6>(w, u, dx, dxt, raw, nelv, st);
    case 8: return eopr_launch_lx<8>(w, u, dx, dxt, raw, nelv, st);
    case 10: return eopr_launch_lx<10>(w, u, dx, dxt, raw, nelv, st);
    case 12: return eopr_launch_lx<12>(w, u, dx, dxt, raw, nelv, st);
    default: return AX_EINVAL;
  }
}

int eop_launch(int lx, const EopArgs &a, cudaStream_t st) {
  if (a.pw && !(a.dotp && a.r && a.minv && a.beta)) return AX_EINVAL;
  if (a.corr && !a.use_corr) return AX_EINVAL;
  switch (lx) {
    case 6: return eop_launch_lx<6>(a, st);
    case 8: return eop_launch_lx<8>(a, st);
    case 10: return eop_launch_lx<10>(a, st);
    case 12: return eop_launch_lx<12>(a, st);
    default: return AX_EINVAL;
  }
}

int eop_blocks(int lx, int nelv, bool dot) {
  switch (lx) {
    case 6: return eop_blocks_lx<6>(nelv, dot);
    case 8: return eop_blocks_lx<8>(nelv, dot);
    case 10: return eop_blocks_lx<10>(nelv, dot);
    case 12: return eop_blocks_lx<12>(nelv, dot);
    default: return 0;
  }
}

int eop_prepare(int lx, df::dd2 *gp, const guard::RawGeo &r, int nelv, int fmask, int dfield,
                cudaStream_t st) {
  switch (lx) {
    case 6: return eop_prepare_lx<6>(gp, r, nelv, fmask, dfield, st);
    case 8: return eop_prepare_lx<8>(gp, r, nelv, fmask, dfield, st);
    case 10: return eop_prepare_lx<10>(gp, r, nelv, fmask, dfield, st);
    case 12: return eop_prepare_lx<12>(gp, r, nelv, fmask, dfield, st);
    default: return AX_EINVAL;
  }
}

size_t eop_coef_bytes(int lx) {
  const size_t h = lx / 2;
  return 2 * h * (h + 1) * 16 + 2 * h * h * 8;
}

// The half-size coefficients of D and D^T (even-odd split), formed in fp64
// and split into double-float pairs (split_rn): for row i < lx/2 and l < lx/2,
// P = (A[i][l] + A[i][N-l]) / 2 and M = (A[i][l] - A[i][N-l]) / 2 with
// A[i][l] = m[l * lx + i] (dx gives D, dxt gives D^T), stored as
// {P.hi, M.hi, P.lo, M.lo} in rows of lx/2 + 1 entries (the last one
// padding), then the negated heads {-P.hi, -M.hi} in rows of lx/2.
// Returns false when a matrix is not centro-antisymmetric to 2^-46 of its
// largest entry (the split would misread it); *dfield: biased fp64 exponent
// field of the largest |entry| of both matrices.
bool eop_coefficients(int lx, const double *dx_h, const double *dxt_h, void *out, int *dfield) {
  const int H = lx / 2, N = lx - 1, H2 = H * H;
  double dmax = 0.0, dev = 0.0;
  for (int q = 0; q < lx * lx; ++q) dmax = std::max({dmax, std::fabs(dx_h[q]), std::fabs(dxt_h[q])});
  for (int i = 0; i < lx; ++i)
    for (int l = 0; l < lx; ++l)
      for (const double *m : {dx_h, dxt_h})
        dev = std::max(dev, std::fabs(m[l * lx + i] + m[(N - l) * lx + (N - i)]));
  if (!(dev <= dmax * 0x1p-46) || !std::isfinite(dmax)) return false;
  int ex = 0;
  std::frexp(dmax, &ex);
  *dfield = dmax > 0.0 ? ex - 1 + 1023 : 0;
  auto bits = [](float f) { return (unsigned long long)df::f2u(f); };
  const int CS = H + 1;
  df::dd2 *cf = static_cast<df::dd2 *>(out);
  unsigned long long *cn = reinterpret_cast<unsigned long long *>(cf + 2 * H * CS);
  for (int q = 0; q < 2 * H * CS; ++q) cf[q] = df::dd2{0ull, 0ull};
  for (int tr = 0; tr < 2; ++tr) {
    const double *m = tr ? dxt_h : dx_h;
    for (int i = 0; i < H; ++i)
      for (int l = 0; l < H; ++l) {
        const double a = m[l * lx + i], b = m[(N - l) * lx + i];
        const df::df2 P = df::split_rn(0.5 * (a + b)), M = df::split_rn(0.5 * (a - b));
        df::dd2 &d = cf[(tr * H + i) * CS + l];
        d.hi = bits(P.hi) | (bits(M.hi) << 32);
        d.lo = bits(P.lo) | (bits(M.lo) << 32);
        cn[tr * H2 + i * H + l] = bits(-P.hi) | (bits(-M.hi) << 32);
      }
  }
  return true;
}

}  // namespace ax
