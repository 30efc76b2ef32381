// Learned element preconditioner: a two-layer perceptron per element,
//   x = (minv .* r)_e / s_e,  h = tanh(x W1 + b1),  y = h W2 + b2,
// whose output, scaled back by s_e, is added to the Jacobi step (see the
// flexible CG in cg.cu).  The paper has no learned component; this follows
// the project's learned-preconditioner workload.
//
// * Apply (inference): both layers are small dense GEMMs over a tile of 64
//   elements, run on the tensor cores with bf16 operands and fp32
//   accumulation (mma.sync m16n8k16); x is staged in shared memory chunk by
//   chunk, the hidden layer stays in shared memory, and the output goes
//   through shared memory in 128-column slabs so that every global access
//   is a coalesced row segment.
// * Training: fp32 SIMT kernels with one thread per output and a fixed
//   summation order (deterministic, no atomics): forward, mean-squared loss,
//   backpropagation, Adam (Kingma & Ba 2015).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "df64.cuh"
#include "mlp.cuh"
#include "reduce.cuh"

namespace {

constexpr int kTE = 64;     // elements per inference block
constexpr int kKC = 64;     // k-chunk of the first layer
constexpr int kThreads = 256;

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// fp32 -> fp64 bits without the fp64 pipe: normal numbers exactly, Inf and
// NaN to Inf and NaN, subnormals and zero to signed zero.
AX_D double f2d(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  uint64_t d = ((uint64_t)(b & 0x80000000u) << 32);
  if (e == 0xFFu)
    d |= (0x7FFull << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29);
  else if (e != 0u)
    d |= ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}
AX_D float to_f32(double x) { return ax::df::split(x).hi; }
AX_D float to_f32(float x) { return x; }
template <typename T>
AX_D T from_f32(float y);
template <>
AX_D double from_f32<double>(float y) { return f2d(y); }
template <>
AX_D float from_f32<float>(float y) { return y; }

AX_D uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low half)
  return *reinterpret_cast<uint32_t *>(&v);
}

AX_D void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Inference over a tile of kTE elements.  Weights (bf16, padded with
// zeros): W1T [HP][NP] (k contiguous per hidden unit), b1 [HP] (fp32),
// W2T [NP][HP] (k contiguous per output), b2 [NP] (fp32).
// Global memory is touched only by coalesced row-contiguous passes: the
// input chunk is loaded one row segment per warp into xs, and each 128-wide
// output slab goes through ys before it is scaled and stored.
// Shared memory: xs [kTE][kKC+8] bf16, hs [kTE][HP+8] bf16,
// ys [kTE][kYC+4] fp32, s [kTE] fp32, s_part [kTE][2] fp32.
constexpr int kYC = 128;  // output columns per epilogue slab

inline size_t apply_smem(int HP) {
  return (size_t)kTE * (kKC + 8) * 2 + (size_t)kTE * (HP + 8) * 2 + (size_t)kTE * (kYC + 4) * 4 +
         (size_t)kTE * 3 * 4;
}

template <typename T, bool SYM>
__global__ void __launch_bounds__(kThreads)
mlp_apply_kernel(T *__restrict__ corr, const T *__restrict__ r, const T *__restrict__ minv,
                 const T *__restrict__ mask, const T *__restrict__ cw,
                 const float *__restrict__ sc, const __nv_bfloat16 *__restrict__ W1T,
                 const float *__restrict__ b1, const __nv_bfloat16 *__restrict__ W2T,
                 const float *__restrict__ b2, int N, int NP, int HP, int nelv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int XS = kKC + 8, HS = HP + 8, YS = kYC + 4;  // row strides, padded
  __nv_bfloat16 *xs = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
  __nv_bfloat16 *hs = xs + kTE * XS;
  float *ys = reinterpret_cast<float *>(hs + kTE * HS);
  float *s_sh = ys + kTE * YS;
  float *s_part = s_sh + kTE;  // [kTE][2]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  const long long e0 = (long long)blockIdx.x * kTE;
  // input scale of the residual and activation of the hidden layer; the
  // symmetric form is linear, so its per-element normalisation cancels and
  // is skipped, and its scale sqrt(minv) comes precomputed in sc if given
  auto in_scale = [&](size_t q) {
    return SYM ? (sc ? sc[q] : sqrtf(to_f32(minv[q]))) : to_f32(minv[q]);
  };
  auto act = [](float a) { return SYM ? a : tanhf(a); };
  const int nel = (int)min((long long)kTE, nelv - e0);

  // ---- layer 1: acc = x W1 over k chunks (and ||x||^2 per row, tanh form)
  const int mt = warp & 3;        // rows mt*16 .. +15
  const int nh = warp >> 2;       // n-tiles nh, nh+2, ...
  const int n_tiles1 = HP / 8;
  float acc1[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc1[a][b] = 0.f;
  const int lcol = tid & 63;      // loader: column of the chunk
  const int lrow0 = tid >> 6;     // loader: rows lrow0 + 4 i
  float ss[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) ss[i] = 0.f;
  for (int kc = 0; kc < NP; kc += kKC) {
    __syncthreads();
    const int k = kc + lcol;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int row = lrow0 + 4 * i;
      float v = 0.f;
      if (row < nel && k < N) {
        const size_t q = (size_t)(e0 + row) * N + k;
        v = in_scale(q) * to_f32(r[q]);
      }
      if (!SYM) ss[i] = fmaf(v, v, ss[i]);
      xs[row * XS + lcol] = __float2bfloat16_rn(v);
    }
    __syncthreads();
    const int kmax = min(kKC, NP - kc);
#pragma unroll
    for (int ks = 0; ks < kKC; ks += 16) {
      if (ks >= kmax) break;
      uint32_t a[4];
      const __nv_bfloat16 *x0 = xs + (mt * 16 + g) * XS + ks + 2 * t4;
      const __nv_bfloat16 *x1 = x0 + 8 * XS;
      a[0] = *reinterpret_cast<const uint32_t *>(x0);
      a[1] = *reinterpret_cast<const uint32_t *>(x1);
      a[2] = *reinterpret_cast<const uint32_t *>(x0 + 8);
      a[3] = *reinterpret_cast<const uint32_t *>(x1 + 8);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int nt = nh + 2 * j;
        if (nt < n_tiles1) {
          const __nv_bfloat16 *w = W1T + (size_t)(nt * 8 + g) * NP + kc + ks + 2 * t4;
          const uint32_t b0 = __ldg(reinterpret_cast<const unsigned int *>(w));
          const uint32_t b1r = __ldg(reinterpret_cast<const unsigned int *>(w + 8));
          mma_bf16(acc1[j], a, b0, b1r);
        }
      }
    }
  }
  // row norms: each warp holds 32 columns of its rows; fixed-order sums
  if (!SYM) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float v = ss[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) s_part[(lrow0 + 4 * i) * 2 + (warp & 1)] = v;
    }
  }
  __syncthreads();
  if (tid < kTE) s_sh[tid] = SYM ? 1.f : sqrtf(s_part[2 * tid] + s_part[2 * tid + 1]);
  __syncthreads();
  // hidden layer: h = act(acc / s + b1) -> shared memory (bf16)
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int nt = nh + 2 * j;
    if (nt < n_tiles1) {
      const int col = nt * 8 + 2 * t4;
      const int r0 = mt * 16 + g, r1 = r0 + 8;
      const float i0 = s_sh[r0] > 0.f ? 1.f / s_sh[r0] : 0.f;
      const float i1 = s_sh[r1] > 0.f ? 1.f / s_sh[r1] : 0.f;
      const float bb0 = b1[col], bb1 = b1[col + 1];
      *reinterpret_cast<uint32_t *>(&hs[r0 * HS + col]) =
          pack_bf16(act(acc1[j][0] * i0 + bb0), act(acc1[j][1] * i0 + bb1));
      *reinterpret_cast<uint32_t *>(&hs[r1 * HS + col]) =
          pack_bf16(act(acc1[j][2] * i1 + bb0), act(acc1[j][3] * i1 + bb1));
    }
  }
  __syncthreads();

  // ---- layer 2: y = h W2 + b2 in slabs of kYC outputs, epilogue
  // corr = mask * c * s * y (tanh form) or sqrt(minv) * y (symmetric form)
  const int half = warp >> 2;
  const int n_tiles2 = NP / 8;
  const int r0 = mt * 16 + g, r1 = r0 + 8;
  const int ocol = tid & (kYC - 1), orow0 = tid / kYC;  // epilogue mapping
  for (int nb0 = 0; nb0 < n_tiles2; nb0 += kYC / 8) {
    float acc2[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc2[a][b] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 64; ks += 16) {  // HP <= 64
      if (ks >= HP) break;
      uint32_t a[4];
      const __nv_bfloat16 *h0 = hs + r0 * HS + ks + 2 * t4;
      const __nv_bfloat16 *h1 = hs + r1 * HS + ks + 2 * t4;
      a[0] = *reinterpret_cast<const uint32_t *>(h0);
      a[1] = *reinterpret_cast<const uint32_t *>(h1);
      a[2] = *reinterpret_cast<const uint32_t *>(h0 + 8);
      a[3] = *reinterpret_cast<const uint32_t *>(h1 + 8);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int nt = nb0 + half * 8 + j;
        if (nt < n_tiles2) {
          const __nv_bfloat16 *w = W2T + (size_t)(nt * 8 + g) * HP + ks + 2 * t4;
          const uint32_t b0 = __ldg(reinterpret_cast<const unsigned int *>(w));
          const uint32_t b1r = __ldg(reinterpret_cast<const unsigned int *>(w + 8));
          mma_bf16(acc2[j], a, b0, b1r);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = (half * 8 + j) * 8 + 2 * t4;  // within the slab
      *reinterpret_cast<float2 *>(&ys[r0 * YS + col]) = make_float2(acc2[j][0], acc2[j][1]);
      *reinterpret_cast<float2 *>(&ys[r1 * YS + col]) = make_float2(acc2[j][2], acc2[j][3]);
    }
    __syncthreads();
    const int o = nb0 * 8 + ocol;
    if (o < N) {
      const float bo = b2[o];
      // fixed trip count, unrolled: the loads of several rows are in flight
      // together instead of one latency per row
#pragma unroll 8
      for (int j = 0; j < kTE / (kThreads / kYC); ++j) {
        const int row = orow0 + j * (kThreads / kYC);
        if (row < nel) {
          const size_t q = (size_t)(e0 + row) * N + o;
          const float y = ys[row * YS + ocol] + bo;
          const float osc = SYM ? in_scale(q) : to_f32(mask[q]) * to_f32(cw[q]);
          corr[q] = from_f32<T>(osc * s_sh[row] * y);
        }
      }
    }
    __syncthreads();
  }
}

// Symmetric form with its scale precomputed (sc = sqrt(minv), fp32) and an
// even number of points per element: one warp streams 16 elements through
// both layers with no shared memory and no block barrier.  Layer 1 loads the
// mma A-fragments straight from r and sc (rows g, g+8, columns k+2t4 and
// k+2t4+8: 16-byte and 8-byte pairs, full sectors), one k-step ahead;
// its accumulators are re-packed in registers as the A-fragments of
// layer 2 (n-tiles 2q, 2q+1 of layer 1 are k-step q of layer 2); the
// epilogue stores corr = sc * y as pairs.  Weights come through L1/L2.
constexpr int kSymWarps = 4;  // warps per block

template <typename T>
struct Pair;  // two consecutive values of T
template <>
struct Pair<double> {
  using V = double2;
};
template <>
struct Pair<float> {
  using V = float2;
};

template <typename T, int NT1>  // NT1 = HP / 8 hidden n-tiles
__global__ void __launch_bounds__(kSymWarps * 32)
mlp_sym_apply_kernel(T *__restrict__ corr, const T *__restrict__ r,
                     const float *__restrict__ sc, const __nv_bfloat16 *__restrict__ W1T,
                     const __nv_bfloat16 *__restrict__ W2T, int N, int NP, int nelv) {
  using V = typename Pair<T>::V;
  constexpr int HP = NT1 * 8;
  const int lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
  const long long ew = ((long long)blockIdx.x * kSymWarps + (threadIdx.x >> 5)) * 16;
  if (ew >= nelv) return;  // warp-uniform
  const bool ok0 = ew + g < nelv, ok1 = ew + g + 8 < nelv;
  const size_t row0 = (size_t)(ok0 ? ew + g : 0) * N, row1 = (size_t)(ok1 ? ew + g + 8 : 0) * N;

  // A-fragment inputs of one k-step: x at (row, k + 2 t4 + {0, 1, 8, 9})
  struct In {
    V r[4];
    float2 s[4];
  };
  auto load = [&](int ks, In &in) {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int k = ks + 2 * t4 + ((h & 2) ? 8 : 0);
      const bool okr = (h & 1) ? ok1 : ok0;
      const size_t q = ((h & 1) ? row1 : row0) + k;
      if (okr && k < N) {  // N even: the pair (k, k + 1) is inside the element
        in.r[h] = *reinterpret_cast<const V *>(r + q);
        in.s[h] = *reinterpret_cast<const float2 *>(sc + q);
      } else {
        in.r[h] = V{};
        in.s[h] = make_float2(0.f, 0.f);
      }
    }
  };
  float acc1[NT1][4];
#pragma unroll
  for (int j = 0; j < NT1; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc1[j][q] = 0.f;
  In cur, nxt;
  load(0, nxt);
  for (int ks = 0; ks < NP; ks += 16) {
    cur = nxt;
    if (ks + 16 < NP) load(ks + 16, nxt);
    uint32_t a[4];
#pragma unroll
    for (int h = 0; h < 4; ++h)  // fragment order: (g, k), (g+8, k), (g, k+8), (g+8, k+8)
      a[h] = pack_bf16(cur.s[h].x * to_f32(cur.r[h].x), cur.s[h].y * to_f32(cur.r[h].y));
#pragma unroll
    for (int j = 0; j < NT1; ++j) {
      const __nv_bfloat16 *w = W1T + (size_t)(j * 8 + g) * NP + ks + 2 * t4;
      mma_bf16(acc1[j], a, __ldg(reinterpret_cast<const unsigned int *>(w)),
               __ldg(reinterpret_cast<const unsigned int *>(w + 8)));
    }
  }
  // layer-1 accumulators (rows g, g+8; hidden 8j + 2t4 + {0, 1}) as layer-2
  // A-fragments: k-step q takes n-tiles 2q (k) and 2q + 1 (k + 8)
  uint32_t a2[NT1 / 2][4];
#pragma unroll
  for (int q = 0; q < NT1 / 2; ++q) {
    a2[q][0] = pack_bf16(acc1[2 * q][0], acc1[2 * q][1]);
    a2[q][1] = pack_bf16(acc1[2 * q][2], acc1[2 * q][3]);
    a2[q][2] = pack_bf16(acc1[2 * q + 1][0], acc1[2 * q + 1][1]);
    a2[q][3] = pack_bf16(acc1[2 * q + 1][2], acc1[2 * q + 1][3]);
  }
  for (int nt = 0; nt < NP / 8; ++nt) {
    float acc2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < NT1 / 2; ++q) {
      const __nv_bfloat16 *w = W2T + (size_t)(nt * 8 + g) * HP + 16 * q + 2 * t4;
      mma_bf16(acc2, a2[q], __ldg(reinterpret_cast<const unsigned int *>(w)),
               __ldg(reinterpret_cast<const unsigned int *>(w + 8)));
    }
    const int col = nt * 8 + 2 * t4;
    if (col < N) {
      if (ok0) {
        const float2 sv = *reinterpret_cast<const float2 *>(sc + row0 + col);
        V o;
        o.x = from_f32<T>(sv.x * acc2[0]);
        o.y = from_f32<T>(sv.y * acc2[1]);
        *reinterpret_cast<V *>(corr + row0 + col) = o;
      }
      if (ok1) {
        const float2 sv = *reinterpret_cast<const float2 *>(sc + row1 + col);
        V o;
        o.x = from_f32<T>(sv.x * acc2[2]);
        o.y = from_f32<T>(sv.y * acc2[3]);
        *reinterpret_cast<V *>(corr + row1 + col) = o;
      }
    }
  }
}

// ---------------------------------------------------------------- training
// X[b][k] = (minv r)_e / s, T[b][k] = (err - minv r)_e / s for e = idx[b]
__global__ void gather_pairs_kernel(float *__restrict__ X, float *__restrict__ Tt,
                                    const double *__restrict__ r, const double *__restrict__ err,
                                    const double *__restrict__ minv, const int *__restrict__ idx,
                                    int N) {
  __shared__ double sh[kThreads / 32];
  const int b = blockIdx.x;
  const size_t base = (size_t)idx[b] * N;
  double ss = 0.0;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const double z = minv[base + k] * r[base + k];
    ss += z * z;
  }
  double v[1] = {ss};
  ax::block_sum<1>(v, sh);
  __shared__ double s_b;
  if (threadIdx.x == 0) s_b = sqrt(v[0]);
  __syncthreads();
  const double inv = s_b > 0.0 ? 1.0 / s_b : 0.0;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const double z = minv[base + k] * r[base + k];
    X[(size_t)b * N + k] = (float)(z * inv);
    Tt[(size_t)b * N + k] = (float)((err[base + k] - z) * inv);
  }
}

// H[b][h] = tanh(sum_k X[b][k] W1[k][h] + b1[h])
__global__ void fwd_hidden_kernel(float *__restrict__ H, const float *__restrict__ X,
                                  const float *__restrict__ theta, int B, int N, int Hd,
                                  int sym) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)B * Hd) return;
  const int b = (int)(q / Hd), h = (int)(q % Hd);
  const float *W1 = theta, *b1 = theta + (size_t)N * Hd;
  float a = 0.f;
  for (int k = 0; k < N; ++k) a = fmaf(X[(size_t)b * N + k], W1[(size_t)k * Hd + h], a);
  H[q] = sym ? a + b1[h] : tanhf(a + b1[h]);
}

// Y = H W2 + b2; dY = 2 (Y - T) / (B N); per-block partial of sum (Y-T)^2
__global__ void fwd_out_loss_kernel(float *__restrict__ Y, float *__restrict__ dY,
                                    const float *__restrict__ H, const float *__restrict__ Tt,
                                    const float *__restrict__ theta, int B, int N, int Hd,
                                    double *__restrict__ partials) {
  __shared__ double sh[kThreads / 32];
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (q < (int64_t)B * N) {
    const int b = (int)(q / N), o = (int)(q % N);
    const float *W2 = theta + (size_t)N * Hd + Hd, *b2 = W2 + (size_t)Hd * N;
    float a = 0.f;
    for (int h = 0; h < Hd; ++h) a = fmaf(H[(size_t)b * Hd + h], W2[(size_t)h * N + o], a);
    const float y = a + b2[o];
    Y[q] = y;
    const float res = y - Tt[q];
    dY[q] = 2.f * res / ((float)B * (float)N);
    l = (double)res * (double)res;
  }
  double v[1] = {l};
  ax::block_sum<1>(v, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

// Y = H W2 + b2 (training forward without a target)
__global__ void fwd_out_kernel(float *__restrict__ Y, const float *__restrict__ H,
                               const float *__restrict__ theta, int B, int N, int Hd) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)B * N) return;
  const int b = (int)(q / N), o = (int)(q % N);
  const float *W2 = theta + (size_t)N * Hd + Hd, *b2 = W2 + (size_t)Hd * N;
  float a = 0.f;
  for (int h = 0; h < Hd; ++h) a = fmaf(H[(size_t)b * Hd + h], W2[(size_t)h * N + o], a);
  Y[q] = a + b2[o];
}

// gW2[h][o] = sum_b H[b][h] dY[b][o]; gb2[o] = sum_b dY[b][o]
__global__ void grad_w2_kernel(float *__restrict__ grad, const float *__restrict__ H,
                               const float *__restrict__ dY, int B, int N, int Hd) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float *gW2 = grad + (size_t)N * Hd + Hd, *gb2 = gW2 + (size_t)Hd * N;
  if (q < (int64_t)Hd * N) {
    const int h = (int)(q / N), o = (int)(q % N);
    float a = 0.f;
    for (int b = 0; b < B; ++b) a = fmaf(H[(size_t)b * Hd + h], dY[(size_t)b * N + o], a);
    gW2[q] = a;
  } else if (q < (int64_t)Hd * N + N) {
    const int o = (int)(q - (int64_t)Hd * N);
    float a = 0.f;
    for (int b = 0; b < B; ++b) a += dY[(size_t)b * N + o];
    gb2[o] = a;
  }
}

// dP[b][h] = (sum_o dY[b][o] W2[h][o]) (1 - H[b][h]^2)
__global__ void back_hidden_kernel(float *__restrict__ dP, const float *__restrict__ dY,
                                   const float *__restrict__ H, const float *__restrict__ theta,
                                   int B, int N, int Hd, int sym) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)B * Hd) return;
  const int b = (int)(q / Hd), h = (int)(q % Hd);
  const float *W2 = theta + (size_t)N * Hd + Hd;
  float a = 0.f;
  for (int o = 0; o < N; ++o) a = fmaf(dY[(size_t)b * N + o], W2[(size_t)h * N + o], a);
  const float hv = H[q];
  dP[q] = sym ? a : a * (1.f - hv * hv);
}

// gW1[k][h] = sum_b X[b][k] dP[b][h]; gb1[h] = sum_b dP[b][h]
__global__ void grad_w1_kernel(float *__restrict__ grad, const float *__restrict__ X,
                               const float *__restrict__ dP, int B, int N, int Hd) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float *gb1 = grad + (size_t)N * Hd;
  if (q < (int64_t)N * Hd) {
    const int k = (int)(q / Hd), h = (int)(q % Hd);
    float a = 0.f;
    for (int b = 0; b < B; ++b) a = fmaf(X[(size_t)b * N + k], dP[(size_t)b * Hd + h], a);
    grad[q] = a;
  } else if (q < (int64_t)N * Hd + Hd) {
    const int h = (int)(q - (int64_t)N * Hd);
    float a = 0.f;
    for (int b = 0; b < B; ++b) a += dP[(size_t)b * Hd + h];
    gb1[h] = a;
  }
}

__global__ void adam_kernel(float *__restrict__ theta, float *__restrict__ m,
                            float *__restrict__ v, const float *__restrict__ g, int64_t n,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float gq = g[q];
  const float mq = b1 * m[q] + (1.f - b1) * gq;
  const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
  m[q] = mq;
  v[q] = vq;
  theta[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

// bf16 inference copy: W1T [HP][NP], b1 [HP] (fp32), W2T [NP][HP], b2 [NP] (fp32)
__global__ void refresh_bf16_kernel(__nv_bfloat16 *__restrict__ W1T, float *__restrict__ b1p,
                                    __nv_bfloat16 *__restrict__ W2T, float *__restrict__ b2p,
                                    const float *__restrict__ theta, int N, int Hd, int NP,
                                    int HP) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const float *W1 = theta, *b1 = theta + (size_t)N * Hd;
  const float *W2 = b1 + Hd, *b2 = W2 + (size_t)Hd * N;
  const int64_t n1 = (int64_t)HP * NP;
  if (q < n1) {
    const int h = (int)(q / NP), k = (int)(q % NP);
    W1T[q] = __float2bfloat16_rn((h < Hd && k < N) ? W1[(size_t)k * Hd + h] : 0.f);
  }
  if (q < (int64_t)NP * HP) {
    const int o = (int)(q / HP), h = (int)(q % HP);
    W2T[q] = __float2bfloat16_rn((h < Hd && o < N) ? W2[(size_t)h * N + o] : 0.f);
  }
  if (q < HP) b1p[q] = q < Hd ? b1[q] : 0.f;
  if (q < NP) b2p[q] = q < N ? b2[q] : 0.f;
}

struct Layout {
  int NP, HP;
  size_t w1t, b1p, w2t, b2p;  // offsets (bytes) in theta_bf's allocation
  size_t bytes;
};

Layout layout(const ax_mlp *M) {
  Layout L;
  L.NP = round_up(M->n_in, 16);
  L.HP = round_up(M->n_hid, 16);
  L.w1t = 0;
  L.b1p = L.w1t + (size_t)L.HP * L.NP * 2;
  L.w2t = L.b1p + (size_t)L.HP * 4;
  L.b2p = L.w2t + (size_t)L.NP * L.HP * 2;
  L.bytes = L.b2p + (size_t)L.NP * 4;
  return L;
}

int refresh_bf16(ax_mlp *M, cudaStream_t st) {
  const Layout L = layout(M);
  char *base = reinterpret_cast<char *>(M->theta_bf);
  const int64_t n = std::max<int64_t>((int64_t)L.HP * L.NP, (int64_t)L.NP);
  refresh_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<__nv_bfloat16 *>(base + L.w1t), reinterpret_cast<float *>(base + L.b1p),
      reinterpret_cast<__nv_bfloat16 *>(base + L.w2t), reinterpret_cast<float *>(base + L.b2p),
      M->theta, M->n_in, M->n_hid, L.NP, L.HP);
  return ax::launch_status();
}

int ensure_capacity(ax_mlp *M, int B) {
  if (B <= M->cap) return AX_OK;
  cudaFree(M->X);
  cudaFree(M->T);
  cudaFree(M->H);
  cudaFree(M->Y);
  cudaFree(M->dY);
  cudaFree(M->dP);
  cudaFree(M->partials);
  M->cap = 0;
  const size_t bn = (size_t)B * M->n_in, bh = (size_t)B * M->n_hid;
  const size_t nblk = (bn + kThreads - 1) / kThreads;
  if (cudaMalloc(&M->X, bn * 4) != cudaSuccess || cudaMalloc(&M->T, bn * 4) != cudaSuccess ||
      cudaMalloc(&M->Y, bn * 4) != cudaSuccess || cudaMalloc(&M->dY, bn * 4) != cudaSuccess ||
      cudaMalloc(&M->H, bh * 4) != cudaSuccess || cudaMalloc(&M->dP, bh * 4) != cudaSuccess ||
      cudaMalloc(&M->partials, nblk * 8) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ENOMEM;
  }
  M->cap = B;
  return AX_OK;
}

// tied weights: gW1[k][h] += gW2[h][k]; gb1 = 0
__global__ void tie_grad_kernel(float *__restrict__ grad, int N, int Hd) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const float *gW2 = grad + (size_t)N * Hd + Hd;
  if (q < (int64_t)N * Hd) {
    const int k = (int)(q / Hd), h = (int)(q % Hd);
    grad[q] += gW2[(size_t)h * N + k];
  } else if (q < (int64_t)N * Hd + Hd) {
    grad[q] = 0.f;
  }
}
// zero the W2 and b2 gradients (after tie_grad_kernel has read them)
__global__ void zero_tail_kernel(float *__restrict__ grad, int64_t from, int64_t n) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n - from) grad[from + q] = 0.f;
}
// W2 = W1^T, b1 = b2 = 0
__global__ void tie_params_kernel(float *__restrict__ theta, int N, int Hd) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float *b1 = theta + (size_t)N * Hd, *W2 = b1 + Hd, *b2 = W2 + (size_t)Hd * N;
  if (q < (int64_t)N * Hd) {
    const int k = (int)(q / Hd), h = (int)(q % Hd);
    W2[(size_t)h * N + k] = theta[q];
  }
  if (q < Hd) b1[q] = 0.f;
  if (q < N) b2[q] = 0.f;
}

// rows perm[b] of the sample set -> the batch buffers
__global__ void gather_rows_kernel(float *__restrict__ X, float *__restrict__ Tt,
                                   const float *__restrict__ Xa, const float *__restrict__ Ta,
                                   const int *__restrict__ perm, int N) {
  const size_t src = (size_t)perm[blockIdx.x] * N, dst = (size_t)blockIdx.x * N;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    X[dst + k] = Xa[src + k];
    Tt[dst + k] = Ta[src + k];
  }
}

__global__ void sum_partials_kernel2(const double *__restrict__ p, int n, double *__restrict__ out) {
  ax::warp_sum_partials<1>(p, n, out);
}

// forward + loss + full gradient on M->X / M->T (B samples)
int loss_grad_dev(ax_mlp *M, int B, cudaStream_t st) {
  const int N = M->n_in, Hd = M->n_hid;
  auto blocks = [](int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); };
  const int64_t bn = (int64_t)B * N, bh = (int64_t)B * Hd;
  fwd_hidden_kernel<<<blocks(bh), kThreads, 0, st>>>(M->H, M->X, M->theta, B, N, Hd, M->arch);
  fwd_out_loss_kernel<<<blocks(bn), kThreads, 0, st>>>(M->Y, M->dY, M->H, M->T, M->theta, B, N,
                                                       Hd, M->partials);
  sum_partials_kernel2<<<1, 32, 0, st>>>(M->partials, (int)blocks(bn), M->loss_dev);
  grad_w2_kernel<<<blocks((int64_t)Hd * N + N), kThreads, 0, st>>>(M->grad, M->H, M->dY, B, N,
                                                                    Hd);
  back_hidden_kernel<<<blocks(bh), kThreads, 0, st>>>(M->dP, M->dY, M->H, M->theta, B, N, Hd,
                                                     M->arch);
  grad_w1_kernel<<<blocks((int64_t)N * Hd + Hd), kThreads, 0, st>>>(M->grad, M->X, M->dP, B, N,
                                                                    Hd);
  return ax::launch_status();
}

int adam_dev(ax_mlp *M, float lr, float b1, float b2, float eps, cudaStream_t st) {
  M->adam_step += 1;
  const float c1 = 1.f - powf(b1, (float)M->adam_step);
  const float c2 = 1.f - powf(b2, (float)M->adam_step);
  adam_kernel<<<(unsigned)((M->nparam + 255) / 256), 256, 0, st>>>(
      M->theta, M->m, M->v, M->grad, M->nparam, lr, b1, b2, eps, c1, c2);
  return ax::launch_status();
}

}  // namespace

namespace ax {

int mlp_reserve(ax_mlp *M, int B) { return ensure_capacity(M, B); }

// H, Y from M->X for B rows (fp32 training forward)
int mlp_train_forward(ax_mlp *M, int B, cudaStream_t st) {
  const int N = M->n_in, Hd = M->n_hid;
  auto blocks = [](int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); };
  fwd_hidden_kernel<<<blocks((int64_t)B * Hd), kThreads, 0, st>>>(M->H, M->X, M->theta, B, N,
                                                                  Hd, M->arch);
  fwd_out_kernel<<<blocks((int64_t)B * N), kThreads, 0, st>>>(M->Y, M->H, M->theta, B, N, Hd);
  return launch_status();
}

// gradient from M->X, M->H and the output gradient M->dY (B rows)
int mlp_train_backward(ax_mlp *M, int B, cudaStream_t st) {
  const int N = M->n_in, Hd = M->n_hid;
  auto blocks = [](int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); };
  grad_w2_kernel<<<blocks((int64_t)Hd * N + N), kThreads, 0, st>>>(M->grad, M->H, M->dY, B, N,
                                                                    Hd);
  back_hidden_kernel<<<blocks((int64_t)B * Hd), kThreads, 0, st>>>(M->dP, M->dY, M->H, M->theta,
                                                                   B, N, Hd, M->arch);
  grad_w1_kernel<<<blocks((int64_t)N * Hd + Hd), kThreads, 0, st>>>(M->grad, M->X, M->dP, B, N,
                                                                    Hd);
  return launch_status();
}

int mlp_adam_step(ax_mlp *M, float lr, cudaStream_t st) {
  return adam_dev(M, lr, 0.9f, 0.999f, 1e-8f, st);
}

int mlp_refresh(ax_mlp *M, cudaStream_t st) { return refresh_bf16(M, st); }

int mlp_tie_grad(ax_mlp *M, cudaStream_t st) {
  const int N = M->n_in, Hd = M->n_hid;
  const int64_t n1 = (int64_t)N * Hd + Hd;
  tie_grad_kernel<<<(unsigned)((n1 + 255) / 256), 256, 0, st>>>(M->grad, N, Hd);
  const int64_t rest = M->nparam - n1;
  zero_tail_kernel<<<(unsigned)((rest + 255) / 256), 256, 0, st>>>(M->grad, n1, M->nparam);
  return launch_status();
}

int mlp_tie_params(ax_mlp *M, cudaStream_t st) {
  const int N = M->n_in, Hd = M->n_hid;
  const int64_t n = std::max<int64_t>((int64_t)N * Hd, N);
  tie_params_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M->theta, N, Hd);
  return launch_status();
}

template <typename T>
int mlp_correction(const ax_mlp *M, T *corr, const T *r, const T *minv, const T *mask,
                   const T *c, int nelv, cudaStream_t st, const float *sc) {
  if (nelv <= 0) return AX_OK;
  const Layout L = layout(M);
  const char *base = reinterpret_cast<const char *>(M->theta_bf);
  if (M->arch == AX_MLP_SYM && sc && M->n_in % 2 == 0 && (L.HP == 16 || L.HP == 32 ||
                                                          L.HP == 48 || L.HP == 64)) {
    auto w1 = reinterpret_cast<const __nv_bfloat16 *>(base + L.w1t);
    auto w2 = reinterpret_cast<const __nv_bfloat16 *>(base + L.w2t);
    const unsigned grid = (unsigned)((nelv + 16 * kSymWarps - 1) / (16 * kSymWarps));
    const int th = kSymWarps * 32;
    switch (L.HP) {
      case 16: mlp_sym_apply_kernel<T, 2><<<grid, th, 0, st>>>(corr, r, sc, w1, w2, M->n_in, L.NP, nelv); break;
      case 32: mlp_sym_apply_kernel<T, 4><<<grid, th, 0, st>>>(corr, r, sc, w1, w2, M->n_in, L.NP, nelv); break;
      case 48: mlp_sym_apply_kernel<T, 6><<<grid, th, 0, st>>>(corr, r, sc, w1, w2, M->n_in, L.NP, nelv); break;
      default: mlp_sym_apply_kernel<T, 8><<<grid, th, 0, st>>>(corr, r, sc, w1, w2, M->n_in, L.NP, nelv); break;
    }
    return launch_status();
  }
  const size_t smem = apply_smem(L.HP);
  auto kern = M->arch == AX_MLP_SYM ? mlp_apply_kernel<T, true> : mlp_apply_kernel<T, false>;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
    (void)cudaGetLastError();
    return AX_EINVAL;
  }
  const unsigned grid = (unsigned)((nelv + kTE - 1) / kTE);
  kern<<<grid, kThreads, smem, st>>>(
      corr, r, minv, mask, c, sc, reinterpret_cast<const __nv_bfloat16 *>(base + L.w1t),
      reinterpret_cast<const float *>(base + L.b1p),
      reinterpret_cast<const __nv_bfloat16 *>(base + L.w2t),
      reinterpret_cast<const float *>(base + L.b2p), M->n_in, L.NP, L.HP, nelv);
  return launch_status();
}

template int mlp_correction<double>(const ax_mlp *, double *, const double *, const double *,
                                    const double *, const double *, int, cudaStream_t,
                                    const float *);
template int mlp_correction<float>(const ax_mlp *, float *, const float *, const float *,
                                   const float *, const float *, int, cudaStream_t,
                                   const float *);

}  // namespace ax

extern "C" {

int ax_mlp_destroy(ax_mlp *M) {
  if (!M) return AX_OK;
  float *f[] = {M->theta, M->grad, M->m, M->v, M->X, M->T, M->H, M->Y, M->dY, M->dP};
  for (float *p : f) cudaFree(p);
  cudaFree(M->theta_bf);
  cudaFree(M->partials);
  cudaFree(M->loss_dev);
  delete M;
  return AX_OK;
}

int ax_mlp_create_ex(ax_mlp **out, int n_in, int n_hid, int arch) {
  if (!out || n_in < 1 || n_in > 4096 || n_hid < 1 || n_hid > 64 ||
      (arch != AX_MLP_TANH && arch != AX_MLP_SYM))
    return AX_EINVAL;
  *out = nullptr;
  ax_mlp *M = new (std::nothrow) ax_mlp();
  if (!M) return AX_ENOMEM;
  M->n_in = n_in;
  M->n_hid = n_hid;
  M->arch = arch;
  M->nparam = (int64_t)n_in * n_hid + n_hid + (int64_t)n_hid * n_in + n_in;
  const Layout L = layout(M);
  const size_t pb = (size_t)M->nparam * 4;
  if (cudaMalloc(&M->theta, pb) != cudaSuccess || cudaMalloc(&M->grad, pb) != cudaSuccess ||
      cudaMalloc(&M->m, pb) != cudaSuccess || cudaMalloc(&M->v, pb) != cudaSuccess ||
      cudaMalloc(&M->theta_bf, L.bytes) != cudaSuccess ||
      cudaMalloc(&M->loss_dev, sizeof(double)) != cudaSuccess ||
      cudaMemset(M->theta, 0, pb) != cudaSuccess || cudaMemset(M->grad, 0, pb) != cudaSuccess ||
      cudaMemset(M->m, 0, pb) != cudaSuccess || cudaMemset(M->v, 0, pb) != cudaSuccess ||
      cudaMemset(M->theta_bf, 0, L.bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    ax_mlp_destroy(M);
    return AX_ENOMEM;
  }
  *out = M;
  return AX_OK;
}

int ax_mlp_create(ax_mlp **out, int n_in, int n_hid) {
  return ax_mlp_create_ex(out, n_in, n_hid, AX_MLP_TANH);
}

int ax_mlp_nparams(const ax_mlp *M, int64_t *n) {
  if (!M || !n) return AX_EINVAL;
  *n = M->nparam;
  return AX_OK;
}

int ax_mlp_set_params(ax_mlp *M, const float *host, int64_t count, void *stream) {
  if (!M || !host || count != M->nparam) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(M->theta, host, count * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(M->m, 0, count * 4, st) != cudaSuccess ||
      cudaMemsetAsync(M->v, 0, count * 4, st) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  M->adam_step = 0;
  int rc = M->arch == AX_MLP_SYM ? ax::mlp_tie_params(M, st) : AX_OK;
  if (rc == AX_OK) rc = refresh_bf16(M, st);
  if (rc == AX_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = AX_ELAUNCH;
  return rc;
}

int ax_mlp_get_params(const ax_mlp *M, float *host, int64_t count, void *stream) {
  if (!M || !host || count != M->nparam) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(host, M->theta, count * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  return AX_OK;
}

int ax_mlp_loss_grad(ax_mlp *M, const float *X, const float *T, int B, double *loss,
                     float *grad_host, void *stream) {
  if (!M || !X || !T || B < 1) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_capacity(M, B);
  if (rc) return rc;
  const size_t bn = (size_t)B * M->n_in * 4;
  if (cudaMemcpyAsync(M->X, X, bn, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(M->T, T, bn, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return AX_ELAUNCH;
  if ((rc = loss_grad_dev(M, B, st))) return rc;
  if (M->arch == AX_MLP_SYM && (rc = ax::mlp_tie_grad(M, st))) return rc;
  double l = 0.0;
  if (cudaMemcpyAsync(&l, M->loss_dev, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return AX_ELAUNCH;
  if (grad_host && cudaMemcpyAsync(grad_host, M->grad, M->nparam * 4, cudaMemcpyDeviceToHost,
                                   st) != cudaSuccess)
    return AX_ELAUNCH;
  if (cudaStreamSynchronize(st) != cudaSuccess) return AX_ELAUNCH;
  if (loss) *loss = l / ((double)B * M->n_in);
  return AX_OK;
}

int ax_mlp_adam(ax_mlp *M, float lr, float beta1, float beta2, float eps, void *stream) {
  if (!M || !(lr >= 0)) return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = adam_dev(M, lr, beta1, beta2, eps, st);
  if (rc) return rc;
  if (M->arch == AX_MLP_SYM && (rc = ax::mlp_tie_params(M, st))) return rc;
  return refresh_bf16(M, st);
}

int ax_mlp_forward(const ax_mlp *M, const float *r, const float *minv, const float *mask,
                   const float *c, float *corr, int nelv, void *stream) {
  if (!M || nelv < 0 || (nelv > 0 && !ax::all_nonnull(r, minv, mask, c, corr)))
    return AX_EINVAL;
  return ax::mlp_correction<float>(M, corr, r, minv, mask, c, nelv, (cudaStream_t)stream);
}

int ax_mlp_train(ax_mlp *M, const float *X_all, const float *T_all, int nsamples,
                 const int *perm, int epochs, int batch, float lr, double *final_loss,
                 void *stream) {
  if (!M || !X_all || !T_all || !perm || nsamples < 1 || batch < 1 || epochs < 1 || !(lr > 0))
    return AX_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  batch = std::min(batch, nsamples);
  int rc = ensure_capacity(M, batch);
  if (rc) return rc;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int s0 = 0; s0 + batch <= nsamples; s0 += batch) {
      gather_rows_kernel<<<batch, kThreads, 0, st>>>(M->X, M->T, X_all, T_all,
                                                     perm + (size_t)ep * nsamples + s0, M->n_in);
      if ((rc = loss_grad_dev(M, batch, st))) return rc;
      if (M->arch == AX_MLP_SYM && (rc = ax::mlp_tie_grad(M, st))) return rc;
      if ((rc = adam_dev(M, lr, 0.9f, 0.999f, 1e-8f, st))) return rc;
      if (M->arch == AX_MLP_SYM && (rc = ax::mlp_tie_params(M, st))) return rc;
    }
  }
  if ((rc = refresh_bf16(M, st))) return rc;
  double last = 0.0;
  if (cudaMemcpyAsync(&last, M->loss_dev, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return AX_ELAUNCH;
  if (final_loss) *final_loss = last / ((double)batch * M->n_in);
  return AX_OK;
}

int ax_mlp_gather_pairs(const ax_mlp *M, const double *r, const double *err, const double *minv,
                        const int *idx, int nsamples, float *X, float *T, void *stream) {
  if (!M || !r || !err || !minv || !idx || nsamples < 0 || !X || !T) return AX_EINVAL;
  if (nsamples == 0) return AX_OK;
  gather_pairs_kernel<<<nsamples, kThreads, 0, (cudaStream_t)stream>>>(X, T, r, err, minv, idx,
                                                                       M->n_in);
  return ax::launch_status();
}

}  // extern "C"
