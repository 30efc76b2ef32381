// Host-side discretisation set-up of the library: GLL points and weights,
// the 1-D differentiation buffers, the geometric factors of a box mesh of
// trilinear hexahedra and its global numbering.  Plain C++ on the host; the
// results are uploaded by the caller.
//
// Formulas (Sec. "The Spectral Element Method"; Deville, Fischer & Mund,
// High-Order Methods for Incompressible Fluid Flow, 2002, Sec. 2.4):
//   * interior GLL nodes are the roots of L_N'; Newton's method on L_N' with
//     L_N'' from Legendre's equation (1-x^2) L'' = 2x L' - N(N+1) L;
//   * weights 2 / (N (N+1) L_N(x)^2);
//   * D from barycentric weights: D_ij = (b_j / b_i) / (x_i - x_j), i != j,
//     and D_ii = -sum_{j != i} D_ij (rows annihilate constants);
//   * the Jacobian of the trilinear map is evaluated in closed form from the
//     eight vertices; G = W * adj(J) adj(J)^T / det(J), the same matrix as
//     det(J) W J^{-1} J^{-T}.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <thread>
#include <vector>
#include <atomic>

#include "../../include/axhelm.h"
#include "df64.cuh"

namespace {

// L_n(x) and L_n'(x) by the recurrences
// (m+1) L_{m+1} = (2m+1) x L_m - m L_{m-1},  L_{m+1}' = L_{m-1}' + (2m+1) L_m.
void legendre_and_derivative(int n, double x, double *l, double *dl) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) {
    *l = 1.0;
    *dl = 0.0;
    return;
  }
  for (int m = 1; m < n; ++m) {
    const double p2 = ((2 * m + 1) * x * p1 - m * p0) / (m + 1);
    const double d2 = d0 + (2 * m + 1) * p1;
    p0 = p1;
    p1 = p2;
    d0 = d1;
    d1 = d2;
  }
  *l = p1;
  *dl = d1;
}

void gll_nodes_weights(int lx, double *x, double *w) {
  const int n = lx - 1;
  const double pi = 3.14159265358979323846;
  x[0] = -1.0;
  x[n] = 1.0;
  for (int i = 1; i < n; ++i) {
    // start between the Chebyshev-Lobatto point and a Gauss-like guess
    double t = -std::cos(pi * i / n);
    for (int it = 0; it < 60; ++it) {
      double l, dl;
      legendre_and_derivative(n, t, &l, &dl);
      const double ddl = (2.0 * t * dl - n * (n + 1.0) * l) / (1.0 - t * t);
      const double step = dl / ddl;
      t -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    x[i] = t;
  }
  // symmetrise: the node set is symmetric about 0
  for (int i = 0; i < lx / 2; ++i) {
    const double a = 0.5 * (x[n - i] - x[i]);
    x[i] = -a;
    x[n - i] = a;
  }
  if (lx % 2) x[n / 2] = 0.0;
  for (int i = 0; i < lx; ++i) {
    double l, dl;
    legendre_and_derivative(n, x[i], &l, &dl);
    w[i] = 2.0 / (n * (n + 1.0) * l * l);
  }
}

// D[i][j] (row-major) by barycentric weights.
void diff_matrix(int lx, const double *x, double *d) {
  std::vector<double> b(lx);
  for (int j = 0; j < lx; ++j) {
    double prod = 1.0;
    for (int k = 0; k < lx; ++k)
      if (k != j) prod *= (x[j] - x[k]);
    b[j] = 1.0 / prod;
  }
  for (int i = 0; i < lx; ++i) {
    double diag = 0.0;
    for (int j = 0; j < lx; ++j) {
      if (j == i) continue;
      const double v = (b[j] / b[i]) / (x[i] - x[j]);
      d[i * lx + j] = v;
      diag -= v;
    }
    d[i * lx + i] = diag;
  }
}

template <typename F>
void parallel_for(int64_t n, F f) {
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 1;
  if (nt > 64) nt = 64;
  if (n < 64 || nt == 1) {
    f(0, n);
    return;
  }
  std::vector<std::thread> th;
  const int64_t chunk = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    const int64_t a = t * chunk, b = std::min<int64_t>(n, a + chunk);
    if (a >= b) break;
    th.emplace_back([=] { f(a, b); });
  }
  for (auto &t : th) t.join();
}

}  // namespace

extern "C" {

int ax_gll(int lx, double *xi, double *wq) {
  if (lx < AX_LX_MIN || lx > AX_LX_MAX) return AX_EINVAL;
  std::vector<double> x(lx), w(lx);
  gll_nodes_weights(lx, x.data(), w.data());
  for (int i = 0; i < lx; ++i) {
    if (xi) xi[i] = x[i];
    if (wq) wq[i] = w[i];
  }
  return AX_OK;
}

int ax_dmat(int lx, double *dx, double *dxt) {
  if (lx < AX_LX_MIN || lx > AX_LX_MAX || !dx || !dxt) return AX_EINVAL;
  std::vector<double> x(lx), w(lx), d(lx * lx);
  gll_nodes_weights(lx, x.data(), w.data());
  diff_matrix(lx, x.data(), d.data());
  for (int l = 0; l < lx; ++l)
    for (int i = 0; i < lx; ++i) {
      dx[l * lx + i] = d[i * lx + l];   // D_{i l}
      dxt[l * lx + i] = d[l * lx + i];  // D_{l i}
    }
  return AX_OK;
}

int ax_box_geometry(int nx, int ny, int nz, int lx, const double *vertices, double *g11,
                    double *g22, double *g33, double *g12, double *g13, double *g23,
                    double *mass, double *xyz) {
  if (lx < AX_LX_MIN || lx > AX_LX_MAX || nx < 1 || ny < 1 || nz < 1 || !vertices || !g11 ||
      !g22 || !g33 || !g12 || !g13 || !g23)
    return AX_EINVAL;
  std::vector<double> xi(lx), wq(lx);
  gll_nodes_weights(lx, xi.data(), wq.data());
  const int64_t nel = (int64_t)nx * ny * nz;
  const int64_t n3 = (int64_t)lx * lx * lx;
  std::atomic<int> bad{0};
  auto vtx = [&](int a, int b, int c, int d) {
    return vertices[(((int64_t)c * (ny + 1) + b) * (nx + 1) + a) * 3 + d];
  };
  parallel_for(nel, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) {
      const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
      double X[2][2][2][3];
      for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a)
            for (int d = 0; d < 3; ++d) X[c][b][a][d] = vtx(ex + a, ey + b, ez + c, d);
      for (int k = 0; k < lx; ++k)
        for (int j = 0; j < lx; ++j)
          for (int i = 0; i < lx; ++i) {
            const double r = xi[i], s = xi[j], t = xi[k];
            const double fr[2] = {0.5 * (1 - r), 0.5 * (1 + r)};
            const double fs[2] = {0.5 * (1 - s), 0.5 * (1 + s)};
            const double ft[2] = {0.5 * (1 - t), 0.5 * (1 + t)};
            const double dfd[2] = {-0.5, 0.5};
            double J[3][3] = {{0}}, pos[3] = {0, 0, 0};
            for (int c = 0; c < 2; ++c)
              for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a)
                  for (int d = 0; d < 3; ++d) {
                    const double v = X[c][b][a][d];
                    pos[d] += v * fr[a] * fs[b] * ft[c];
                    J[d][0] += v * dfd[a] * fs[b] * ft[c];
                    J[d][1] += v * fr[a] * dfd[b] * ft[c];
                    J[d][2] += v * fr[a] * fs[b] * dfd[c];
                  }
            // adj(J)[a][d] = cofactor of J[d][a]
            double adj[3][3];
            adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
            adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
            adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
            adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
            adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
            adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
            adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
            adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
            adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
            if (!(det > 0)) {
              bad.store(1);
              continue;
            }
            const double W = wq[i] * wq[j] * wq[k];
            const double f = W / det;
            auto gg = [&](int a, int b) {
              return f * (adj[a][0] * adj[b][0] + adj[a][1] * adj[b][1] + adj[a][2] * adj[b][2]);
            };
            const int64_t q = e * n3 + ((int64_t)k * lx + j) * lx + i;
            g11[q] = gg(0, 0);
            g22[q] = gg(1, 1);
            g33[q] = gg(2, 2);
            g12[q] = gg(0, 1);
            g13[q] = gg(0, 2);
            g23[q] = gg(1, 2);
            if (mass) mass[q] = det * W;
            if (xyz)
              for (int d = 0; d < 3; ++d) xyz[3 * q + d] = pos[d];
          }
    }
  });
  return bad.load() ? AX_EINVAL : AX_OK;
}

int ax_box_numbering(int nx, int ny, int nz, int lx, int64_t *glob) {
  if (lx < AX_LX_MIN || lx > AX_LX_MAX || nx < 1 || ny < 1 || nz < 1 || !glob) return AX_EINVAL;
  const int64_t n = lx - 1, NX = (int64_t)nx * n + 1, NY = (int64_t)ny * n + 1;
  const int64_t nel = (int64_t)nx * ny * nz;
  parallel_for(nel, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) {
      const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
      int64_t q = e * lx * lx * lx;
      for (int k = 0; k < lx; ++k)
        for (int j = 0; j < lx; ++j)
          for (int i = 0; i < lx; ++i)
            glob[q++] = (ex * n + i) + NX * ((ey * n + j) + NY * (ez * n + k));
    }
  });
  return AX_OK;
}

int ax_box_mask(int nx, int ny, int nz, int lx, const int *dirichlet, double *mask) {
  if (lx < AX_LX_MIN || lx > AX_LX_MAX || nx < 1 || ny < 1 || nz < 1 || !dirichlet || !mask)
    return AX_EINVAL;
  const int64_t n = lx - 1, NX = (int64_t)nx * n + 1, NY = (int64_t)ny * n + 1;
  const int64_t NZ = (int64_t)nz * n + 1;
  const int64_t nel = (int64_t)nx * ny * nz;
  const bool fx0 = dirichlet[0], fx1 = dirichlet[1], fy0 = dirichlet[2], fy1 = dirichlet[3];
  const bool fz0 = dirichlet[4], fz1 = dirichlet[5];
  parallel_for(nel, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) {
      const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
      int64_t q = e * lx * lx * lx;
      for (int k = 0; k < lx; ++k)
        for (int j = 0; j < lx; ++j)
          for (int i = 0; i < lx; ++i) {
            const int64_t X = ex * n + i, Y = ey * n + j, Z = ez * n + k;
            const bool on = (fx0 && X == 0) || (fx1 && X == NX - 1) || (fy0 && Y == 0) ||
                            (fy1 && Y == NY - 1) || (fz0 && Z == 0) || (fz1 && Z == NZ - 1);
            mask[q++] = on ? 0.0 : 1.0;
          }
    }
  });
  return AX_OK;
}

int ax_box_corners(int nx, int ny, int nz, const double *vertices, double *corners) {
  if (nx < 1 || ny < 1 || nz < 1 || !vertices || !corners) return AX_EINVAL;
  const int64_t nel = (int64_t)nx * ny * nz;
  for (int64_t e = 0; e < nel; ++e) {
    const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const int64_t v = ((ez + c) * (ny + 1) + (ey + b)) * (nx + 1) + (ex + a);
          for (int d = 0; d < 3; ++d)
            corners[e * 24 + ((c * 2 + b) * 2 + a) * 3 + d] = vertices[v * 3 + d];
        }
  }
  return AX_OK;
}

int ax_tune_save(const char *path) {
  if (!path) return AX_EINVAL;
  FILE *f = std::fopen(path, "w");
  if (!f) return AX_EIO;
  bool ok = std::fprintf(f, "# axhelm tuning table: epb <dtype> <lx> <n> | variant <lx> <v>\n") > 0;
  for (int dtype : {AX_BATCH_F64, AX_BATCH_F32})
    for (int lx = AX_LX_MIN; lx <= AX_LX_MAX; ++lx) {
      int v = 0;
      if (ax_tune_get(dtype, lx, &v) == AX_OK && v > 0)
        ok = ok && std::fprintf(f, "epb %d %d %d\n", dtype, lx, v) > 0;
    }
  for (int lx = AX_LX_MIN; lx <= AX_LX_MAX; ++lx) {
    int v = 0;
    if (ax_tune_variant_get(lx, &v) == AX_OK && v > 0)
      ok = ok && std::fprintf(f, "variant %d %d\n", lx, v) > 0;
  }
  if (std::fclose(f) != 0) ok = false;
  return ok ? AX_OK : AX_EIO;
}

int ax_tune_load(const char *path) {
  if (!path) return AX_EINVAL;
  FILE *f = std::fopen(path, "r");
  if (!f) return AX_EIO;
  struct Entry {
    bool epb;
    int a, b, c;
  };
  std::vector<Entry> entries;
  char line[256];
  bool bad = false;
  while (!bad && std::fgets(line, sizeof line, f)) {
    char kw[16] = {0};
    if (std::sscanf(line, "%15s", kw) != 1 || kw[0] == '#') continue;  // blank or comment
    int a = 0, b = 0, c = 0;
    char extra[2];
    if (!std::strcmp(kw, "epb") && std::sscanf(line, "epb %d %d %d %1s", &a, &b, &c, extra) == 3)
      entries.push_back({true, a, b, c});
    else if (!std::strcmp(kw, "variant") && std::sscanf(line, "variant %d %d %1s", &a, &b, extra) == 2)
      entries.push_back({false, a, b, 0});
    else
      bad = true;
  }
  const bool read_error = std::ferror(f) != 0;
  std::fclose(f);
  if (read_error) return AX_EIO;
  if (bad) return AX_EINVAL;
  // the setters' rules, checked for every entry before any is applied
  for (const Entry &e : entries) {
    if (e.epb) {
      if ((e.a != AX_BATCH_F64 && e.a != AX_BATCH_F32) || e.b < AX_LX_MIN || e.b > AX_LX_MAX ||
          e.c < 0 || e.c * e.b * e.b > 256)
        return AX_EINVAL;
    } else if (e.a < AX_LX_MIN || e.a > AX_LX_MAX || e.b < AX_VARIANT_AUTO ||
               e.b > AX_VARIANT_F64_DF_EO) {
      return AX_EINVAL;
    }
  }
  for (const Entry &e : entries) {
    const int rc = e.epb ? ax_tune_set(e.a, e.b, e.c) : ax_tune_variant_set(e.a, e.b);
    if (rc != AX_OK) return rc;
  }
  return AX_OK;
}

// Host twin of the device fp64 <-> double-float conversions, so that their
// bit manipulation can be checked without a GPU.
int ax_df64_roundtrip(const double *x, float *hi, float *lo, double *back, int64_t n) {
  if (n < 0 || (n > 0 && (!x || !hi || !lo || !back))) return AX_EINVAL;
  for (int64_t p = 0; p < n; ++p) {
    const ax::df::df2 v = ax::df::split(x[p]);
    hi[p] = v.hi;
    lo[p] = v.lo;
    const ax::df::df2 r = ax::df::norm(v.hi, v.lo);
    back[p] = ax::df::join(r.hi, r.lo);
  }
  return AX_OK;
}

}  // extern "C"
