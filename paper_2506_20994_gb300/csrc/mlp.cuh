// Learned element preconditioner: the network state shared by mlp.cu (its
// kernels) and cg.cu (the flexible CG that applies it).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

struct ax_mlp {
  int n_in = 0, n_hid = 0;       // n_out == n_in
  int arch = 0;                  // AX_MLP_TANH or AX_MLP_SYM
  int64_t nparam = 0;
  float *theta = nullptr;        // fp32 master parameters [W1, b1, W2, b2]
  float *grad = nullptr;         // last gradient
  float *m = nullptr, *v = nullptr;  // Adam moments
  __nv_bfloat16 *theta_bf = nullptr;  // inference copy (bf16)
  int adam_step = 0;
  // training workspace for batches up to cap samples
  int cap = 0;
  float *X = nullptr, *T = nullptr, *H = nullptr, *Y = nullptr, *dY = nullptr, *dP = nullptr;
  double *partials = nullptr;
  double *loss_dev = nullptr;
};

namespace ax {

// Offsets of the parameter blocks in theta.
inline int64_t mlp_off_b1(const ax_mlp *M) { return (int64_t)M->n_in * M->n_hid; }
inline int64_t mlp_off_w2(const ax_mlp *M) { return mlp_off_b1(M) + M->n_hid; }
inline int64_t mlp_off_b2(const ax_mlp *M) { return mlp_off_w2(M) + (int64_t)M->n_hid * M->n_in; }

// Training internals (fp32, on the workspace of ax_mlp):
int mlp_reserve(ax_mlp *M, int B);                          // workspace for B rows
int mlp_train_forward(ax_mlp *M, int B, cudaStream_t st);   // X -> H, Y
int mlp_train_backward(ax_mlp *M, int B, cudaStream_t st);  // X, H, dY -> grad
int mlp_adam_step(ax_mlp *M, float lr, cudaStream_t st);    // theta -= Adam(grad)
int mlp_refresh(ax_mlp *M, cudaStream_t st);                // bf16 inference copy
// Symmetric form: fold the W2 gradient into W1 (tied weights), zero the rest;
// and re-tie the parameters (W2 = W1^T, zero biases) after an update.
int mlp_tie_grad(ax_mlp *M, cudaStream_t st);
int mlp_tie_params(ax_mlp *M, cudaStream_t st);

// corr[q] = mask[q] * c[q] * s_e * y_e[q - e*n] for every element e, where
// y_e = MLP(x_e), x_e = (minv .* r)_e / s_e, s_e = ||(minv .* r)_e||_2
// (bf16 tensor-core apply, fp32 accumulation).  T is double or float.
// For the symmetric form (arch AX_MLP_SYM) the scale sqrt(minv) replaces
// minv on the input and c on the output, and the activation is the identity;
// sc, if not null, holds that scale precomputed in fp32 (mask and c unused).
template <typename T>
int mlp_correction(const ax_mlp *M, T *corr, const T *r, const T *minv, const T *mask,
                   const T *c, int nelv, cudaStream_t st, const float *sc = nullptr);

}  // namespace ax
