// Gather-scatter ("dssum", the second main ingredient of the spectral
// element method named in Sec. "Neko and Small Tensor Kernel"): every local
// copy of a global node receives the sum over all of that node's copies.
//
// Design: the host builds, once, a CSR list of the shared global nodes
// (multiplicity > 1) and the local indices of their copies, ordered by the
// first copy's local index so that neighbouring threads touch neighbouring
// face points.  The kernel gives one thread to each shared node; it sums the
// copies in ascending local-index order (deterministic, no atomics) and
// writes the sum back to every copy.  Points with multiplicity 1 are not
// touched.  Nodes with exactly two copies (the face points, most of the
// shared nodes) keep their two local indices as one 8-byte pair, so their
// thread does one index load instead of the offset-then-index chain; the
// summation order is the same.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

struct ax_gs {
  int64_t n_local = 0;
  int64_t n_shared = 0;   // global nodes with more than one copy
  int64_t n_copies = 0;   // local points that belong to a shared node
  int64_t n_pairs = 0;    // shared nodes with exactly two copies
  int2 *d_pairs = nullptr;  // [n_pairs] (first, second) copy, ascending
  int64_t n_multi = 0;    // shared nodes with more than two copies
  int *d_off = nullptr;   // [n_multi + 1]
  int *d_idx = nullptr;   // copies of the n_multi nodes
  double *d_invmult = nullptr;  // [n_local] 1/multiplicity
  int device = 0;
};

namespace {

// threads [0, n_pairs): two-copy nodes; then one thread per other node
template <typename T>
__global__ void gs_sum_kernel(T *__restrict__ v, const int2 *__restrict__ pairs,
                              int64_t n_pairs, const int *__restrict__ off,
                              const int *__restrict__ idx, int64_t n_multi) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n_pairs) {
    const int2 q = __ldg(pairs + s);
    const T acc = v[q.x] + v[q.y];
    v[q.x] = acc;
    v[q.y] = acc;
    return;
  }
  const int64_t m = s - n_pairs;
  if (m >= n_multi) return;
  const int b = __ldg(off + m), e = __ldg(off + m + 1);
  T acc = v[__ldg(idx + b)];
  for (int k = b + 1; k < e; ++k) acc += v[__ldg(idx + k)];
  for (int k = b; k < e; ++k) v[__ldg(idx + k)] = acc;
}

template <typename T>
int gs_sum_launch(ax_gs *g, T *v, cudaStream_t st) {
  if (!g) return AX_EINVAL;
  if (g->n_shared == 0) return AX_OK;
  if (!v) return AX_EINVAL;
  const int threads = 256;
  const unsigned grid = (unsigned)((g->n_shared + threads - 1) / threads);
  gs_sum_kernel<T><<<grid, threads, 0, st>>>(v, g->d_pairs, g->n_pairs, g->d_off, g->d_idx,
                                             g->n_multi);
  return ax::launch_status();
}

}  // namespace

extern "C" {

int ax_gs_setup(ax_gs **out, const int64_t *glob, int64_t n_local, void *stream) {
  if (!out || n_local < 0 || (n_local > 0 && !glob) || n_local >= (int64_t)1 << 31)
    return AX_EINVAL;
  *out = nullptr;
  int64_t gmax = -1;
  for (int64_t p = 0; p < n_local; ++p) {
    if (glob[p] < 0) return AX_EINVAL;
    gmax = std::max(gmax, glob[p]);
  }
  // group the local copies of every global id, in ascending local order
  std::vector<int> order(n_local);
  std::vector<int64_t> start;
  const bool dense = gmax < 4 * std::max<int64_t>(n_local, 1);
  std::vector<int> count;
  std::vector<int64_t> key;  // global id of each group, by first-copy order
  std::vector<int> gstart, gsize;
  if (dense) {
    count.assign((size_t)gmax + 1, 0);
    for (int64_t p = 0; p < n_local; ++p) ++count[glob[p]];
    std::vector<int64_t> pos((size_t)gmax + 2, 0);
    for (int64_t g = 0; g <= gmax; ++g) pos[g + 1] = pos[g] + count[g];
    std::vector<int64_t> fill(pos.begin(), pos.end() - 1);
    for (int64_t p = 0; p < n_local; ++p) order[fill[glob[p]]++] = (int)p;
    // groups ordered by their first copy
    for (int64_t p = 0; p < n_local; ++p) {
      const int64_t g = glob[p];
      if (count[g] > 1 && order[pos[g]] == (int)p) {
        gstart.push_back((int)pos[g]);
        gsize.push_back(count[g]);
      }
    }
  } else {
    for (int64_t p = 0; p < n_local; ++p) order[p] = (int)p;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return glob[a] < glob[b]; });
    std::vector<std::pair<int, int>> groups;  // (first copy, start in order)
    for (int64_t a = 0; a < n_local;) {
      int64_t b = a + 1;
      while (b < n_local && glob[order[b]] == glob[order[a]]) ++b;
      if (b - a > 1) groups.push_back({order[a], (int)a});
      a = b;
    }
    std::sort(groups.begin(), groups.end());
    for (auto &gr : groups) {
      int64_t b = gr.second + 1;
      while (b < n_local && glob[order[b]] == glob[order[gr.second]]) ++b;
      gstart.push_back(gr.second);
      gsize.push_back((int)(b - gr.second));
    }
  }
  // two-copy nodes as pairs, the rest as CSR; each list keeps the order of
  // first copies
  std::vector<int2> pairs;
  std::vector<int> off(1, 0), idx;
  std::vector<double> invmult(n_local, 1.0);
  int64_t n_copies = 0;
  for (size_t s = 0; s < gstart.size(); ++s) {
    const int *cp = order.data() + gstart[s];
    for (int k = 0; k < gsize[s]; ++k) invmult[cp[k]] = 1.0 / gsize[s];
    n_copies += gsize[s];
    if (gsize[s] == 2) {
      pairs.push_back(make_int2(cp[0], cp[1]));
    } else {
      for (int k = 0; k < gsize[s]; ++k) idx.push_back(cp[k]);
      off.push_back((int)idx.size());
    }
  }

  ax_gs *g = new (std::nothrow) ax_gs();
  if (!g) return AX_ENOMEM;
  g->n_local = n_local;
  g->n_shared = (int64_t)gstart.size();
  g->n_copies = n_copies;
  g->n_pairs = (int64_t)pairs.size();
  g->n_multi = (int64_t)off.size() - 1;
  cudaGetDevice(&g->device);
  cudaStream_t st = (cudaStream_t)stream;
  bool ok = cudaMalloc(&g->d_off, off.size() * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&g->d_idx, std::max<size_t>(idx.size(), 1) * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&g->d_pairs, std::max<size_t>(pairs.size(), 1) * sizeof(int2)) ==
                cudaSuccess &&
            cudaMalloc(&g->d_invmult, std::max<int64_t>(n_local, 1) * sizeof(double)) ==
                cudaSuccess;
  if (ok)
    ok = cudaMemcpyAsync(g->d_off, off.data(), off.size() * sizeof(int),
                         cudaMemcpyHostToDevice, st) == cudaSuccess &&
         (idx.empty() || cudaMemcpyAsync(g->d_idx, idx.data(), idx.size() * sizeof(int),
                                         cudaMemcpyHostToDevice, st) == cudaSuccess) &&
         (pairs.empty() || cudaMemcpyAsync(g->d_pairs, pairs.data(),
                                           pairs.size() * sizeof(int2),
                                           cudaMemcpyHostToDevice, st) == cudaSuccess) &&
         (n_local == 0 || cudaMemcpyAsync(g->d_invmult, invmult.data(),
                                          n_local * sizeof(double), cudaMemcpyHostToDevice,
                                          st) == cudaSuccess) &&
         cudaStreamSynchronize(st) == cudaSuccess;
  if (!ok) {
    (void)cudaGetLastError();
    cudaFree(g->d_off);
    cudaFree(g->d_idx);
    cudaFree(g->d_pairs);
    cudaFree(g->d_invmult);
    delete g;
    return AX_ENOMEM;
  }
  *out = g;
  return AX_OK;
}

int ax_gs_sum(ax_gs *g, double *v, void *stream) {
  return gs_sum_launch<double>(g, v, (cudaStream_t)stream);
}

int ax_gs_sum_f32(ax_gs *g, float *v, void *stream) {
  return gs_sum_launch<float>(g, v, (cudaStream_t)stream);
}

int ax_gs_info(const ax_gs *g, int64_t *n_local, int64_t *n_shared, int64_t *n_copies) {
  if (!g) return AX_EINVAL;
  if (n_local) *n_local = g->n_local;
  if (n_shared) *n_shared = g->n_shared;
  if (n_copies) *n_copies = g->n_copies;
  return AX_OK;
}

const double *ax_gs_inverse_multiplicity(const ax_gs *g) { return g ? g->d_invmult : nullptr; }

int ax_gs_free(ax_gs *g) {
  if (!g) return AX_OK;
  cudaFree(g->d_off);
  cudaFree(g->d_idx);
  cudaFree(g->d_pairs);
  cudaFree(g->d_invmult);
  delete g;
  return AX_OK;
}

}  // extern "C"
