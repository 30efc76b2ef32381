/*
 * axhelm.h - C ABI of libaxhelm.so, a GB300 (sm_103a) implementation of the
 * matrix-free spectral-element stiffness apply ("Ax") of
 * "Portable High-Performance Kernel Generation for a CFD Code with DaCe"
 * (Andersson, Karp, Jansson, Markidis), and of the gather-scatter and
 * conjugate-gradient Poisson solve built on it.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Element fields are element-major fp arrays of nelv*lx^3 values laid out
 *    [e][k][j][i] with i fastest (the dtype[nel,lx,lx,lx] arrays of
 *    Listing 2).  lx = N+1 is the number of GLL points per direction.
 *  - The 1-D differentiation buffers follow Listing 2's indexing:
 *        dx [l*lx + i] = D_{i l}   (derivative at GLL node i of basis l)
 *        dxt[l*lx + i] = D_{l i}   (the transpose).
 *  - The six geometric factors are the entries of the symmetric 3x3 matrix
 *    G (Listing 2's pointwise step): g11 = G_rr, g22 = G_ss, g33 = G_tt,
 *    g12 = G_rs, g13 = G_rt, g23 = G_st, passed in the order of Listing 1:
 *    g11, g22, g33, g12, g13, g23.
 *  - Device pointers are caller-owned CUDA global memory; the library never
 *    frees them.  Every device call is asynchronous on `stream` (a
 *    cudaStream_t passed as void*; NULL is the legacy default stream); it
 *    neither allocates nor synchronises unless its comment says so.
 *  - Output buffers must not alias inputs.
 *  - Devices: a call runs on the device current on the calling host thread
 *    (cudaSetDevice), and its pointers and stream must belong to that
 *    device.  A handle (ax_op, ax_gs, ax_poisson, ax_mlp, ax_batch) owns
 *    memory on the device current at its creation and is used and destroyed
 *    with that device current.  Several devices may be driven from one
 *    process; per-kernel launch settings are kept per device.
 *  - Return value: AX_OK (0) on success or a negative AX_E* code.  Launch
 *    failures are reported from cudaPeekAtLastError (AX_ELAUNCH); nothing
 *    aborts the process.
 */
#ifndef AXHELM_H
#define AXHELM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AX_OK 0
#define AX_EINVAL (-1)     /* bad size, unsupported lx, or NULL pointer   */
#define AX_ELAUNCH (-3)    /* the CUDA launch (or a CUDA call) failed     */
#define AX_ENOMEM (-4)     /* an allocation the call documents failed     */
#define AX_ENOTCONV (-5)   /* a solver hit maxit before its tolerance     */
#define AX_EBREAKDOWN (-6) /* a solver met p.Ap <= 0 or a non-finite value */
#define AX_EIO (-7)        /* a file could not be opened, read or written  */

#define AX_LX_MIN 2
#define AX_LX_MAX 16

/* bf16 values are passed as their 16-bit patterns (IEEE bfloat16). */
typedef uint16_t ax_bf16;

/* Human-readable name of an AX_* code (static storage). */
const char *ax_strerror(int code);

/* Library version string, e.g. "axhelm 0.1 sm_103a". */
const char *ax_version(void);

/* ------------------------------------------------------------------------
 * Element operator (Listing 2, Sec. "The Kernel Expressed in DaCe"):
 *
 *   w_e = D_r^T wr + D_s^T ws + D_t^T wt,
 *   [wr ws wt]^T = h1 * G * [D_r u_e, D_s u_e, D_t u_e]^T,
 *
 * for every element e independently (no assembly).  nelv == 0 is a no-op.
 * Errors: AX_EINVAL if lx is outside [AX_LX_MIN, AX_LX_MAX], nelv < 0, or
 * any pointer is NULL while nelv > 0; AX_ELAUNCH if the launch fails.
 * ------------------------------------------------------------------------ */

/* fp64 in, fp64 out, fp64-accurate (relative L2 error against exact fp64
 * arithmetic below 1e-12).  Dispatches to the fastest fp64-accurate variant
 * for lx (see ax_helm_variant).
 * Range: any fp64 input and any dx, dxt.  The double-float variants carry
 * each value as two fp32 numbers; per element they record the largest
 * exponent of u, of G and of h1, and an element whose product chain
 * D, u, G, h1 leaves the fp32 exponent window with room for the tails (for
 * example |u| beyond ~1e27 or below ~1e-23 with O(1) geometry, or any Inf or
 * NaN) is recomputed with fp64 units, with IEEE fp64 semantics (Inf and NaN
 * propagate as in the loop nest of Listing 2).  The even-odd variant reads
 * only half the rows of dx and dxt, which is exact for centro-antisymmetric
 * matrices (D[N-i][N-l] = -D[i][l], as the GLL matrix is); it checks that
 * property to 2^-46 of the largest entry on every launch, and when it does
 * not hold every element runs on fp64 units (correct, several times slower).
 * fp64 values below 2^-1022 (subnormals) may be flushed to zero. */
int ax_helm(double *w, const double *u, const double *dx, const double *dxt,
            const double *h1, const double *g11, const double *g22,
            const double *g33, const double *g12, const double *g13,
            const double *g23, int lx, int nelv, void *stream);

/* Explicit fp64 variants (same arguments, errors and range as ax_helm).
 * AUTO: the even-odd kernel for lx 6, 8, 10, 12, the double-float k-loop
 * kernel for every other lx, unless ax_tune_variant_run / _set recorded
 * another.  The even-odd variant runs a persistent kernel that streams each
 * element's geometry into shared memory with bulk copies when lx is 6-12,
 * elems_per_block is 0 and the seven geometry arrays are 16-byte aligned;
 * otherwise its per-block form (elems_per_block elements per block). */
#define AX_VARIANT_AUTO 0
#define AX_VARIANT_F64_NATIVE 1 /* fp64 FMA units                           */
#define AX_VARIANT_F64_DF 2     /* pairs of fp32 (double-float) arithmetic   */
#define AX_VARIANT_F64_DF_EO 3  /* double-float with the even-odd split of D  */
                                /* (even lx in 4..12; AX_EINVAL otherwise)    */
int ax_helm_variant(int variant, double *w, const double *u, const double *dx,
                    const double *dxt, const double *h1, const double *g11,
                    const double *g22, const double *g33, const double *g12,
                    const double *g13, const double *g23, int lx, int nelv,
                    int elems_per_block, void *stream);

/* fp32 storage and fp32 arithmetic (the mixed-precision inner operator). */
int ax_helm_f32(float *w, const float *u, const float *dx, const float *dxt,
                const float *h1, const float *g11, const float *g22,
                const float *g33, const float *g12, const float *g13,
                const float *g23, int lx, int nelv, void *stream);

/* bf16 storage of u, h1 and G; fp32 D, fp32 arithmetic, fp32 w. */
int ax_helm_bf16(float *w, const ax_bf16 *u, const float *dx, const float *dxt,
                 const ax_bf16 *h1, const ax_bf16 *g11, const ax_bf16 *g22,
                 const ax_bf16 *g33, const ax_bf16 *g12, const ax_bf16 *g13,
                 const ax_bf16 *g23, int lx, int nelv, void *stream);

/* The full argument list of the paper's interface and kernel (Listings 1
 * and 2): one lx x lx matrix per direction, dx, dy, dz for the forward
 * gradient (ur from dx along i, us from dy along j, ut from dz along k) and
 * dxt, dyt, dzt for the transposed contractions, each in the same layout as
 * ax_helm's dx (entry [l * lx + i] multiplies the value at l to give the
 * one at i).  All six are read as given (no relation between them is
 * assumed).  The paper orders its last two arguments (nelv, lx) and passes a
 * handle first; here the order is ax_helm's and the operator handle is
 * ax_op.  fp64-accurate as ax_helm (double-float k-loop kernel for lx <= 12,
 * fp64 units above).  If dy == dz == dx and dyt == dzt == dxt (the same
 * pointers) the call is exactly ax_helm.  Device arrays, borrowed;
 * asynchronous on `stream`.  Errors as ax_helm (the four extra matrices
 * must not be NULL when nelv > 0). */
int ax_helm_xyz(double *w, const double *u, const double *dx, const double *dy,
                const double *dz, const double *dxt, const double *dyt, const double *dzt,
                const double *h1, const double *g11, const double *g22, const double *g33,
                const double *g12, const double *g13, const double *g23, int lx, int nelv,
                void *stream);

/* fp32 operator with the geometric factors computed on the fly from each
 * element's trilinear map instead of read from six stored fields (u and w,
 * plus h1 unless it is NULL, are the only per-point streams: 8 or 12 bytes
 * per point against 36).  corners: nelv * 24 fp64 values, the element's
 * 8 vertices as written by ax_box_corners; xi, wq: the lx GLL nodes and
 * weights (ax_gll); all device arrays, borrowed.  h1 == NULL means h1 = 1.
 * Per point G = (w_i w_j w_k / det J) adj(J) adj(J)^T with J the Jacobian of
 * the trilinear map, the same factors ax_box_geometry writes, then Listing
 * 2's contractions, all in fp32 (edge vectors formed in fp64, rounded).
 * Asynchronous on `stream`.  Errors as ax_helm (AX_EINVAL for a NULL
 * pointer other than h1 when nelv > 0). */
int ax_helm_trilinear_f32(float *w, const float *u, const float *dx, const float *dxt,
                          const float *h1, const double *corners, const double *xi,
                          const double *wq, int lx, int nelv, void *stream);

/* The operator on host buffers (the paper's interface passes device
 * arrays; this serves callers whose fields live in host memory): w, u, h1
 * and G are host arrays of nelv * lx^3 doubles, dx and dxt host arrays of
 * lx^2; they should be page-locked (pinned) for the copies to run
 * asynchronously.  The elements stream through the device in chunks of
 * `chunk` elements (0 picks about 4 M points per field), the copies in,
 * the apply (as ax_helm) and the copies out of different chunks overlapping
 * on three streams; the device staging buffers are kept per device for the
 * next call.  Work starts after the work queued on `stream`; the call
 * returns when w is written (synchronises).  Calls are serialised per
 * process.  Errors as ax_helm; AX_ENOMEM if staging cannot be allocated. */
int ax_helm_host(double *w, const double *u, const double *dx, const double *dxt,
                 const double *h1, const double *g11, const double *g22, const double *g33,
                 const double *g12, const double *g13, const double *g23, int lx, int nelv,
                 int chunk, void *stream);

/* Helmholtz form: w = Ax(u) + h2 .* B .* u, the stiffness apply above plus
 * the mass term with a coefficient h2 (B the diagonal mass matrix, jac *
 * w_i w_j w_k, in the element-major layout).  The paper's listing is
 * h1-only; the h2 term is the other half of Neko's Helmholtz operator.
 * fp64-accurate stiffness part, fp64 mass part (one extra pass).  Same
 * errors as ax_helm (h2 and B must not be NULL when nelv > 0). */
int ax_helm_h2(double *w, const double *u, const double *dx, const double *dxt,
               const double *h1, const double *g11, const double *g22, const double *g33,
               const double *g12, const double *g13, const double *g23, const double *h2,
               const double *B, int lx, int nelv, void *stream);
/* w += hb .* u over n points (device fp64 / fp32): the mass term with its
 * coefficient folded in (hb = h2 .* B).  Asynchronous; n == 0 is a no-op;
 * AX_EINVAL for n < 0 or a NULL pointer with n > 0. */
int ax_mass_add(double *w, const double *hb, const double *u, int64_t n, void *stream);
int ax_mass_add_f32(float *w, const float *hb, const float *u, int64_t n, void *stream);

/* ------------------------------------------------------------------------
 * Operator handle for repeated applies on one mesh (the paper's interface
 * passes an opaque handle first, Listing 1; here it owns per-mesh state).
 * The operator is ax_helm's: w = Ax(u) in fp64 (element-local, no gs).
 * ------------------------------------------------------------------------ */
typedef struct ax_op ax_op;

/* Creates the handle.  dx, dxt, h1 and G are borrowed device arrays in
 * ax_helm's conventions and must outlive the handle.  For lx in {6, 8, 10,
 * 12}, when dx and dxt are centro-antisymmetric (checked here, to 2^-46 of
 * their largest entry), the handle converts the geometry once into the
 * order of the persistent even-odd kernel that ax_op_apply then runs (device
 * memory, owned: 56 lx^3 + 8 bytes per element - the same 8 bytes per value,
 * split into double-float pairs, plus two exponent records - and
 * 32 h (h + 1) + 16 h^2 + 4 bytes of coefficients and status, h = lx/2).  That kernel streams
 * each element's geometry into shared memory with one bulk copy, one element
 * ahead; results agree with AX_VARIANT_F64_DF_EO to ~1e-16 relative.  Range
 * as ax_helm: elements outside the double-float window are computed from the
 * borrowed fp64 arrays with fp64 units; other lx, and matrices without the
 * symmetry, apply through ax_helm.  Synchronises stream.  Returns AX_EINVAL
 * on bad arguments, AX_ENOMEM when an allocation fails, AX_ELAUNCH when a
 * copy or launch fails. */
int ax_op_create(ax_op **op, int lx, int nelv, const double *dx, const double *dxt,
                 const double *h1, const double *g11, const double *g22, const double *g33,
                 const double *g12, const double *g13, const double *g23, void *stream);
/* w = Ax(u) (device, nelv lx^3 doubles; w must not alias u); asynchronous. */
int ax_op_apply(ax_op *op, double *w, const double *u, void *stream);
/* New coefficient h1 (borrowed; the prepared copy is refreshed on stream). */
int ax_op_set_h1(ax_op *op, const double *h1, void *stream);
/* Adds the Helmholtz mass term: apply becomes w = Ax(u) + h2 .* B .* u.  The
 * handle keeps hb = h2 .* B (device, owned; computed on stream); h2 = NULL
 * removes the term.  Returns AX_ENOMEM if hb cannot be allocated. */
int ax_op_set_h2(ax_op *op, const double *h2, const double *B, void *stream);
/* Whether the geometry is prepared and how many device bytes that holds. */
int ax_op_info(const ax_op *op, int *prepared, int64_t *device_bytes);
/* *flag = 1 if an apply on the prepared path gave up waiting for the
 * bulk copy that stages an element's geometry in shared memory (every wait
 * is bounded, to about 2 s, so a lost copy ends the launch with this flag
 * set instead of hanging; the elements the affected CTA had left are then
 * written as NaN), else 0.  Synchronises the device; the flag stays set for
 * the life of the handle. */
int ax_op_error(const ax_op *op, int *flag);
/* Testing aid for that path: later plain applies (ax_op_apply) on the
 * prepared path run a kernel that does not issue the geometry copy of
 * `element` (0 <= element < nelv), so its wait runs out; element = -1 turns
 * this off.  AX_EINVAL otherwise. */
int ax_op_inject_copy_loss(ax_op *op, int64_t element);
int ax_op_destroy(ax_op *op);

/* ------------------------------------------------------------------------
 * Gather-scatter (direct-stiffness summation; Sec. "Neko and Small Tensor
 * Kernel" names it as the second main ingredient beside the small matrix
 * products): every local copy of a global node receives the sum over all
 * copies of that node.
 * ------------------------------------------------------------------------ */
typedef struct ax_gs ax_gs;

/* Builds the handle from the global id of every local point (host array
 * glob[n_local], ids >= 0, n_local < 2^31).  Allocates device memory
 * (the CSR list of shared nodes and 1/multiplicity per point) and
 * synchronises `stream`.  AX_EINVAL on bad arguments, AX_ENOMEM if an
 * allocation or copy fails. */
int ax_gs_setup(ax_gs **gs, const int64_t *glob, int64_t n_local, void *stream);
/* v[n_local] (device) <- summed over shared copies; deterministic order. */
int ax_gs_sum(ax_gs *gs, double *v, void *stream);
int ax_gs_sum_f32(ax_gs *gs, float *v, void *stream);
/* Sizes of the handle (any pointer may be NULL). */
int ax_gs_info(const ax_gs *gs, int64_t *n_local, int64_t *n_shared, int64_t *n_copies);
/* Device array of 1/multiplicity per local point, owned by the handle. */
const double *ax_gs_inverse_multiplicity(const ax_gs *gs);
int ax_gs_free(ax_gs *gs);

/* ------------------------------------------------------------------------
 * Poisson solve: A p = mask .* gs(Ax(p)), the assembled stiffness operator
 * of the weak form in Sec. "The Spectral Element Method" with homogeneous
 * Dirichlet rows masked out.  Vectors are local (nelv*lx^3, continuous
 * across shared nodes); inner products and norms are over unique global
 * nodes (local sums weighted by 1/multiplicity).
 * ------------------------------------------------------------------------ */
typedef struct ax_poisson ax_poisson;

#define AX_PREC_F32 1  /* inner solve: fp32 G, h1, D and fp32 vectors       */
#define AX_PREC_BF16 2 /* inner solve: bf16 G, h1; fp32 D and fp32 vectors */

/* Creates the operator handle.  dx..g23 and mask (1 interior, 0 on the
 * Dirichlet boundary) are caller-owned device arrays that must outlive the
 * handle; gs is borrowed likewise.  Allocates the work vectors and computes
 * the exact assembled Jacobi diagonal on the device; synchronises stream. */
int ax_poisson_create(ax_poisson **P, int lx, int nelv, const double *dx, const double *dxt,
                      const double *h1, const double *g11, const double *g22,
                      const double *g33, const double *g12, const double *g13,
                      const double *g23, const double *mask, ax_gs *gs, void *stream);
int ax_poisson_destroy(ax_poisson *P);
/* w = mask .* gs(Ax(u)), fp64-accurate; asynchronous. */
int ax_poisson_apply(ax_poisson *P, double *w, const double *u, void *stream);
/* Device array of the masked inverse Jacobi diagonal, owned by P. */
int ax_poisson_jacobi(const ax_poisson *P, const double **minv);
/* Makes the problem Helmholtz, -div(h1 grad u) + h2 u = f: the operator
 * gains h2 .* B .* u (B the diagonal mass, device fp64 arrays of n points,
 * read here; the handle keeps h2 .* B) and the Jacobi diagonal h2 .* B.
 * Every solver then solves the Helmholtz system; the fused p.Ap of the fp64
 * solvers stays on (the mass part's u . hb . u is added by the mass pass).
 * Call before the first mixed-precision solve or again after it (the fp32
 * copies are refreshed).  Synchronises stream. */
int ax_poisson_set_h2(ax_poisson *P, const double *h2, const double *B, void *stream);
/* The assembled Jacobi diagonal before masking and inversion:
 * diag = gs(diag_e(A)) over this handle's gather-scatter (exact element
 * diagonal, reading of the Jacobi preconditioner in the oracle).  diag is a
 * caller-owned device array of n local points; asynchronous.  With the mesh
 * split across ranks this is the rank's partial sum at nodes it shares with
 * another rank; ax_poisson_set_diag takes the fully assembled one back. */
int ax_poisson_diag(const ax_poisson *P, double *diag, void *stream);
/* Replaces the handle's inverse Jacobi diagonal by mask ./ diag (0 where
 * masked or diag == 0) from a caller-assembled diag (device, n points);
 * also refreshes the fp32 copy if a mixed-precision solve converted it
 * already.  Asynchronous; the solvers called afterwards on the same stream
 * use it. */
int ax_poisson_set_diag(ax_poisson *P, const double *diag, void *stream);
/* How often the solvers read the residual norm back (default 1). */
int ax_poisson_set_check_every(ax_poisson *P, int every);

/* Allocation-free refresh of the masked inverse Jacobi diagonal (the paper
 * has no counterpart; it serves callers that may not allocate device memory
 * where they need it: work recorded into a CUDA graph, a time loop with a
 * fixed memory budget, a host framework that owns all device allocations).
 * Writes into minv[nelv*lx^3] (caller's device memory) the same array that
 * ax_poisson_create computes (ax_poisson_jacobi) for the given dx, h1, G,
 * mask (1 interior / 0 Dirichlet) and gather-scatter handle.  Its scratch is
 * a fixed device array inside the library of AX_NOALLOC_MAX_POINTS doubles
 * (4 MiB, reserved on every GPU that loads the library until exit); larger
 * problems return AX_EINVAL, as does a gs handle of another size.  Calls no
 * cudaMalloc/cudaFree.  The first call on a device, and the first after
 * the device's context changed (cudaDeviceReset), resolves the array's
 * device address (cudaGetSymbolAddress); make that call before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race
 * and must be serialised by the caller.  Asynchronous on stream. */
#define AX_NOALLOC_MAX_POINTS (1 << 19)
int ax_jacobi_noalloc(double *minv, const double *dx, const double *h1, const double *g11,
                      const double *g22, const double *g33, const double *g12,
                      const double *g13, const double *g23, const double *mask, ax_gs *gs,
                      int lx, int nelv, void *stream);

/* Jacobi-preconditioned CG in fp64 from x0 = 0 until ||r|| <= tol ||b||
 * (b is masked first).  Writes the iteration count and the final relative
 * residual.  Synchronises stream.  Returns AX_OK, AX_ENOTCONV (maxit
 * reached), AX_EBREAKDOWN (p.Ap <= 0 or non-finite) or AX_EINVAL. */
int ax_cg_solve(ax_poisson *P, double *x, const double *b, double tol, int maxit, int *iters,
                double *relres, void *stream);

/* Mixed-precision iterative refinement: outer loop r = b - A x in fp64
 * (fp64-accurate operator), inner Jacobi-PCG on A d = r in fp32 with the
 * operator data in fp32 (AX_PREC_F32) or bf16 (AX_PREC_BF16) to the
 * relative tolerance inner_tol, x += d in fp64; stops when the fp64
 * residual satisfies ||r|| <= tol ||b||.  The first call per mode converts
 * the operator data (allocates).  Synchronises stream. */
int ax_mpcg_solve(ax_poisson *P, int mode, double *x, const double *b, double tol,
                  double inner_tol, int max_outer, int max_inner, int *outer_iters,
                  int *inner_iters, double *relres, void *stream);

/* ------------------------------------------------------------------------
 * Learned element preconditioner.  The paper has no learned component (it
 * studies the operator only); this is the project's learned form:
 *   z = minv .* r + gs(mask .* (1/mult) .* s_e * MLP(x_e)),
 *   x_e = (minv .* r)_e / s_e,  s_e = ||(minv .* r)_e||_2,
 *   MLP(x) = tanh(x W1 + b1) W2 + b2   (n_in = n_out = lx^3 per element),
 * applied with bf16 weights on the tensor cores (fp32 accumulation) and
 * trained with fp32 kernels on pairs (x_e, (err_e - (minv .* r)_e)/s_e)
 * of element residuals and errors.  Parameters are one flat fp32 vector
 * [W1 (n_in x n_hid, row-major), b1, W2 (n_hid x n_in), b2].
 * ------------------------------------------------------------------------ */
typedef struct ax_mlp ax_mlp;

#define AX_MLP_TANH 0 /* the two-layer tanh network above                  */
#define AX_MLP_SYM 1  /* symmetric linear form (below)                      */

/* Allocates the network (device; parameters start at zero, which makes the
 * preconditioner exactly Jacobi).  n_in in [1, 4096], n_hid in [1, 64].
 * ax_mlp_create makes an AX_MLP_TANH network. */
int ax_mlp_create(ax_mlp **M, int n_in, int n_hid);
/* Same, with the architecture chosen.  AX_MLP_SYM is the symmetric linear
 * form with one basis W = W1 (n_in x n_hid) per element and S = sqrt(minv):
 *   z = minv .* r + gs(mask .* S .* s_e * (x_e W) W^T),
 *   x_e = (S .* r)_e / s_e,  s_e = ||(S .* r)_e||_2,
 * i.e. z = B r with B = diag(minv) + sum_e (R_e S)^T W W^T (R_e S), which is
 * symmetric positive definite for every W (s_e cancels: the map is linear).
 * It keeps the parameter layout; set_params, adam and train keep W2 = W1^T
 * and b1 = b2 = 0, and gradients are folded onto W1 (tied weights).
 * Returns AX_EINVAL for an unknown arch. */
int ax_mlp_create_ex(ax_mlp **M, int n_in, int n_hid, int arch);
int ax_mlp_destroy(ax_mlp *M);
int ax_mlp_nparams(const ax_mlp *M, int64_t *n);
/* Host fp32 parameter vector in / out (count must equal nparams); set
 * resets the Adam state and refreshes the bf16 inference copy.  Both
 * synchronise stream. */
int ax_mlp_set_params(ax_mlp *M, const float *host, int64_t count, void *stream);
int ax_mlp_get_params(const ax_mlp *M, float *host, int64_t count, void *stream);
/* Training pieces on device fp32 batches X, T [B x n_in]: loss (mean
 * squared error, written to *loss on the host) and its gradient (copied to
 * grad_host if not NULL); then one Adam step on the last gradient.
 * loss_grad allocates the batch workspace when B grows; synchronises. */
int ax_mlp_loss_grad(ax_mlp *M, const float *X, const float *T, int B, double *loss,
                     float *grad_host, void *stream);
int ax_mlp_adam(ax_mlp *M, float lr, float beta1, float beta2, float eps, void *stream);
/* Sample set from fp64 local vectors: for each idx[s] (element id, device
 * int32) writes X[s] = (minv .* r)_e / s_e and T[s] = (err - minv .* r)_e / s_e
 * (device fp32 [nsamples x n_in]). */
int ax_mlp_gather_pairs(const ax_mlp *M, const double *r, const double *err, const double *minv,
                        const int *idx, int nsamples, float *X, float *T, void *stream);
/* Minibatch Adam over a sample set: epoch e visits rows perm[e*nsamples ..]
 * (device int32, epochs*nsamples entries, any order) in batches of `batch`;
 * lr fixed, beta1 0.9, beta2 0.999, eps 1e-8.  Writes the last batch loss;
 * synchronises stream. */
int ax_mlp_train(ax_mlp *M, const float *X_all, const float *T_all, int nsamples,
                 const int *perm, int epochs, int batch, float lr, double *final_loss,
                 void *stream);
/* corr = mask .* c .* s_e * MLP(x_e) for fp32 local vectors (no gs);
 * the element-local part of the preconditioner, asynchronous. */
int ax_mlp_forward(const ax_mlp *M, const float *r, const float *minv, const float *mask,
                   const float *c, float *corr, int nelv, void *stream);

/* ------------------------------------------------------------------------
 * Batched operator over many independent meshes of uneven size and mixed
 * lx in one persistent launch.  The paper applies Listing 2 to one mesh per
 * launch and Neko picks its kernel variant by run-time timing (Sec.
 * "Methodology"); the plan below generalises both: one kernel per dtype
 * whose CTAs walk statically balanced work items, grouped by lx and thread
 * layout, with each group run by the single-mesh body of that layout.
 * ------------------------------------------------------------------------ */
typedef struct ax_batch ax_batch;

#define AX_BATCH_F64 1 /* fp64 data, fp64-accurate double-float arithmetic */
#define AX_BATCH_F32 2 /* fp32 data and arithmetic                         */

/* One mesh of a batch: device pointers (double* for AX_BATCH_F64, float*
 * for AX_BATCH_F32) in the conventions above; lx in [2, 12]. */
typedef struct {
  int lx, nelv;
  void *w;
  const void *u, *dx, *dxt, *h1, *g11, *g22, *g33, *g12, *g13, *g23;
} ax_batch_mesh;

/* Builds the plan (host array meshes[nmesh], copied; the device arrays are
 * borrowed and must outlive the plan).  blocks_per_sm <= 0 picks the
 * kernel's full residency.  Allocates the device work list; synchronises
 * stream.  Thread layout per mesh: for AX_BATCH_F64 meshes with lx in
 * {6, 8, 10} the persistent even-odd body of the operator handle,
 * unless the variant table (ax_tune_variant_*) records a k-loop variant for
 * that lx or the mesh's dx / dxt are not centro-antisymmetric; the plan then
 * keeps h1 and G prepared as ax_op_create does (56 lx^3 + 8 bytes per
 * element plus the coefficient block; results equal ax_op_apply's bit for
 * bit; a change of those meshes' h1 or G needs a new plan).  Every other
 * mesh runs the k-loop body (double-float or fp32) in chunks of
 * 256 / lx^2 elements, with the bits of ax_helm / ax_helm_f32. */
int ax_batch_create(ax_batch **B, int dtype, int nmesh, const ax_batch_mesh *meshes,
                    int blocks_per_sm, void *stream);
/* All meshes of the plan in one persistent kernel launch (asynchronous). */
int ax_batch_launch(ax_batch *B, void *stream);
/* The same launch replayed from a CUDA graph captured on the first call. */
int ax_batch_graph_launch(ax_batch *B, void *stream);
/* Plan sizes and the algorithmic flops / bytes of one launch. */
int ax_batch_info(const ax_batch *B, int *nitems, int *nblocks, int64_t *smem_bytes,
                  double *flops, double *bytes);
/* *flag = 1 if a launch gave up waiting for a staged geometry copy (every
 * wait is bounded; the output is then incomplete), else 0.  Synchronises
 * the device. */
int ax_batch_error(const ax_batch *B, int *flag);
int ax_batch_destroy(ax_batch *B);

/* Autotuner: elements per block for (dtype, lx), process-wide.  ax_tune_run
 * times every admissible value on the caller's buffers (nelv elements of
 * the given dtype; w is overwritten; reps timed launches each) and records
 * the fastest; ax_tune_set / ax_tune_get read and write the table (0 means
 * the built-in default).  The single-mesh k-loop dispatch uses the table;
 * the batched kernel sizes its k-loop chunks to its 256-thread CTAs. */
int ax_tune_run(int dtype, int lx, int nelv, void *w, const void *u, const void *dx,
                const void *dxt, const void *h1, const void *g11, const void *g22,
                const void *g33, const void *g12, const void *g13, const void *g23, int reps,
                int *best_epb, float *best_ms, void *stream);
int ax_tune_set(int dtype, int lx, int elems_per_block);
int ax_tune_get(int dtype, int lx, int *elems_per_block);

/* Variant selection for AX_VARIANT_AUTO, process-wide (Neko times its
 * kernel variants at run time and keeps the fastest, Sec. "Methodology").
 * ax_tune_variant_run times AX_VARIANT_F64_NATIVE, AX_VARIANT_F64_DF (every
 * lx) and AX_VARIANT_F64_DF_EO (even lx in 4..12) with default elements per
 * block on the caller's fp64 buffers (w is overwritten; reps timed launches
 * each, after one warm-up), records the fastest for lx and returns it.
 * ax_tune_variant_set / _get write and read the table (0 = the built-in
 * choice, which ax_helm uses until a variant is recorded). */
int ax_tune_variant_run(int lx, int nelv, double *w, const double *u, const double *dx,
                        const double *dxt, const double *h1, const double *g11,
                        const double *g22, const double *g33, const double *g12,
                        const double *g13, const double *g23, int reps, int *best_variant,
                        float *best_ms, void *stream);
int ax_tune_variant_set(int lx, int variant);
int ax_tune_variant_get(int lx, int *variant);

/* The two tuning tables above as a text file (host only, no GPU needed):
 * one line per recorded entry, "epb <dtype> <lx> <elems_per_block>" and
 * "variant <lx> <variant>", '#' lines are comments; entries at 0 (built-in
 * choice) are not written.  ax_tune_load reads the whole file, checks every
 * entry against the rules of ax_tune_set / ax_tune_variant_set and only then
 * applies them (tables not named in the file keep their values).  Errors:
 * AX_EINVAL for a NULL path, an unknown line or an entry the setters would
 * refuse (nothing applied); AX_EIO if the file cannot be opened, read or
 * written. */
int ax_tune_save(const char *path);
int ax_tune_load(const char *path);

/* y = a x + b y on device fp64 vectors of n values (asynchronous). */
int ax_axpby(double *y, double a, const double *x, double b, int64_t n, void *stream);

/* ------------------------------------------------------------------------
 * Vector kernels of the partitioned solve (the paper runs one mesh on one
 * device; splitting the element set across ranks couples them only through
 * the gather-scatter sum at shared nodes and the dot products of CG).
 * ------------------------------------------------------------------------ */
#define AX_DOT_WORK 608 /* doubles of device scratch ax_dot_weighted needs */

/* *out = sum_q wgt[q] a[q] b[q] (device arrays of n doubles; out a device
 * double; work caller-owned device scratch of AX_DOT_WORK doubles).  Fixed
 * grid and order: bitwise reproducible.  Asynchronous; n == 0 writes 0. */
int ax_dot_weighted(const double *a, const double *b, const double *wgt, int64_t n,
                    double *work, double *out, void *stream);
/* out[q] = v[idx[q]], q < n (device arrays; idx int64 in range).  Packs the
 * values at shared nodes (one representative local copy each) to send. */
int ax_gather(double *out, const double *v, const int64_t *idx, int64_t n, void *stream);
/* v[idx[q]] += vals[pos[q]], q < n (device arrays): adds the received
 * values of shared nodes to every local copy.  idx must hold distinct
 * entries (no two threads update one point). */
int ax_scatter_add(double *v, const double *vals, const int64_t *idx, const int64_t *pos,
                   int64_t n, void *stream);

/* Right-hand side of the weak form: b = mask .* gs(B .* f) for the nodal
 * source f and mass B = jac * w_i w_j w_k (device arrays of the handle's
 * local points; b may alias f).  Asynchronous on stream. */
int ax_poisson_rhs(ax_poisson *P, const double *B, const double *f, double *b, void *stream);

/* Partitioned Jacobi-PCG (one rank's part of an SPMD solve).  The element
 * set is split across ranks; they are coupled only by the gather-scatter sum
 * at nodes shared between ranks and by the global dot products.  The driver
 * runs the scalar recurrences (textbook PCG from x0 = 0, stopping at
 * ||r|| <= tol ||r0||, norms over unique global nodes) and does everything
 * else through two caller tables:
 *   ops:  the rank-local vector work on this rank's vectors (all of one
 *         length): w = mask .* gs(A p) with the rank-local gather-scatter,
 *         z = M^-1 r, the rank-local weighted dot (weights 1 / global
 *         multiplicity) returned as a host double, y = a x + b y, copy, zero;
 *   comm: halo(v) adds the other ranks' partial sums at the shared nodes of
 *         a rank-locally summed vector; allsum(vals, count) sums host doubles
 *         over the ranks in place (every rank must get the same bits).
 * Each callback returns 0 on success; any other value ends the solve and is
 * returned.  Two all-sums per iteration.  x, b, r, z, p, w: this rank's
 * vectors (device or host memory, as the ops expect); b is the rank's part of
 * the assembled, masked right-hand side.  Returns AX_OK, AX_ENOTCONV (maxit
 * reached), AX_EBREAKDOWN (p.Ap <= 0 or a non-finite value), AX_EINVAL, or a
 * callback's code.  The driver itself makes no CUDA call. */
typedef struct {
  void *ctx;
  int (*apply)(void *ctx, double *w, const double *p, void *stream);
  int (*precond)(void *ctx, double *z, const double *r, void *stream);
  int (*dot)(void *ctx, const double *a, const double *b, double *out, void *stream);
  int (*axpby)(void *ctx, double *y, double a, const double *x, double b, void *stream);
  int (*copy)(void *ctx, double *dst, const double *src, void *stream);
  int (*zero)(void *ctx, double *v, void *stream);
} ax_part_ops;
typedef struct {
  void *ctx;
  int (*halo)(void *ctx, double *v, void *stream);
  int (*allsum)(void *ctx, double *vals, int count);
} ax_part_comm;
int ax_cg_solve_part(const ax_part_ops *ops, const ax_part_comm *comm, double *x,
                     const double *b, double *r, double *z, double *p, double *w, double tol,
                     int maxit, int *iters, double *relres, void *stream);
/* The same solve on a GPU rank with this library's kernels as the ops: the
 * rank's Poisson handle P (its operator, rank-local gather-scatter, mask and
 * Jacobi diagonal, set by ax_poisson_set_diag to the diagonal assembled
 * across ranks), wgt = 1 / global multiplicity per local point (device).
 * x, b: device vectors of the rank.  Uses the handle's work vectors plus one
 * vector and the dot scratch it allocates for the call; synchronises stream
 * at every dot.  AX_ENOMEM if that allocation fails. */
int ax_cg_solve_part_poisson(ax_poisson *P, const double *wgt, const ax_part_comm *comm,
                             double *x, const double *b, double tol, int maxit, int *iters,
                             double *relres, void *stream);

/* Preconditioner application z = minv .* r (+ learned correction if M is
 * not NULL; M's n_in must be lx^3) for fp64 local vectors; synchronises. */
int ax_precondition(ax_poisson *P, const ax_mlp *M, double *z, const double *r, void *stream);

/* Flexible CG (Notay 2000: beta = <z_new, r_new - r_old> / <z_old, r_old>)
 * with the learned preconditioner in fp64 from x0 = 0; M == NULL gives the
 * Jacobi preconditioner.  A step whose <r, z> is not positive or finite
 * falls back to Jacobi (counted in *fallbacks).  Status codes as
 * ax_cg_solve; allocates its work vectors on first use; synchronises. */
int ax_fcg_solve(ax_poisson *P, const ax_mlp *M, double *x, const double *b, double tol,
                 int maxit, int *iters, double *relres, int *fallbacks, void *stream);

/* Energy-norm training of the learned preconditioner on K residual/error
 * pairs of the operator P (device fp64, K consecutive local vectors each in
 * r_set and e_set, e.g. CG iterates r_k = b - A x_k and e_k = x* - x_k):
 * Adam (fixed lr) on L_k = ||e_k - z(r_k)||_A^2 / ||e_k||_A^2 with z the
 * preconditioner of ax_precondition, every element one training row, the
 * K pairs visited in order for `epochs` passes.  Writes the mean L_k of the
 * last pass.  Allocates scratch (freed on return); synchronises stream. */
int ax_mlp_train_energy(ax_poisson *P, ax_mlp *M, const double *r_set, const double *e_set,
                        int K, int epochs, float lr, double *final_loss, void *stream);

/* ax_mpcg_solve with the flexible CG and the learned preconditioner (in
 * fp32) as the inner solver; fallbacks summed over the inner solves. */
int ax_mpfcg_solve(ax_poisson *P, const ax_mlp *M, int mode, double *x, const double *b,
                   double tol, double inner_tol, int max_outer, int max_inner, int *outer_iters,
                   int *inner_iters, double *relres, int *fallbacks, void *stream);

/* ------------------------------------------------------------------------
 * Host-side discretisation set-up (no GPU needed; plain host memory).
 * ------------------------------------------------------------------------ */

/* GLL nodes xi[lx] (ascending, on [-1,1]) and weights wq[lx] (the
 * quadrature points of Sec. "The Spectral Element Method").  Either pointer
 * may be NULL.  AX_EINVAL if lx is outside [AX_LX_MIN, AX_LX_MAX]. */
int ax_gll(int lx, double *xi, double *wq);

/* The dx and dxt buffers (lx*lx each, convention above) for lx points. */
int ax_dmat(int lx, double *dx, double *dxt);

/* Geometry of a structured box mesh of nx*ny*nz trilinear hexahedra whose
 * vertex positions are given as vertices[((c*(ny+1)+b)*(nx+1)+a)*3 + d]
 * (vertex (a,b,c), coordinate d).  Elements are numbered e = ex+nx*(ey+ny*ez).
 * Writes, per local point, G = jac * W * J^{-1} J^{-T} (six factors, order of
 * Listing 1), the mass jac*W (if mass != NULL) and the node coordinates
 * xyz[3*p + d] (if xyz != NULL); W = w_i w_j w_k.  AX_EINVAL on bad sizes
 * or if an element is inverted (jac <= 0 at a node). */
int ax_box_geometry(int nx, int ny, int nz, int lx, const double *vertices,
                    double *g11, double *g22, double *g33, double *g12,
                    double *g13, double *g23, double *mass, double *xyz);

/* The 8 corner vertices of every element of the same box, corners[e*24 +
 * ((c*2+b)*2+a)*3 + d] = vertex (ex+a, ey+b, ez+c), coordinate d: the input
 * of ax_helm_trilinear_f32.  AX_EINVAL on bad sizes or NULL pointers. */
int ax_box_corners(int nx, int ny, int nz, const double *vertices, double *corners);

/* Global node id of every local point of the structured box (x fastest):
 * glob = X + NX*(Y + NY*Z), X = ex*(lx-1)+i, NX = nx*(lx-1)+1, ... */
int ax_box_numbering(int nx, int ny, int nz, int lx, int64_t *glob);

/* Dirichlet mask of the structured box (host array of nelv lx^3 doubles):
 * 0 at every local point on a face marked in dirichlet[6] (faces x = 0,
 * x = 1, y = 0, y = 1, z = 0, z = 1; nonzero = homogeneous Dirichlet), 1
 * elsewhere.  A face left open is an interface to another partition. */
int ax_box_mask(int nx, int ny, int nz, int lx, const int *dirichlet, double *mask);

/* Host diagnostic of the fp64 <-> fp32-pair conversions that the
 * AX_VARIANT_F64_DF kernels use on the device (same source): splits each
 * x[p] into hi[p] + lo[p] and writes the re-assembled fp64 value to back[p].
 * No counterpart in the paper; it exists so the integer bit manipulation can
 * be checked without a GPU.  All pointers are host memory. */
int ax_df64_roundtrip(const double *x, float *hi, float *lo, double *back, int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* AXHELM_H */
