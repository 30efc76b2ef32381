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
 * for lx (see ax_helm_variant). */
int ax_helm(double *w, const double *u, const double *dx, const double *dxt,
            const double *h1, const double *g11, const double *g22,
            const double *g33, const double *g12, const double *g13,
            const double *g23, int lx, int nelv, void *stream);

/* Explicit fp64 variants (same arguments and errors as ax_helm). */
#define AX_VARIANT_AUTO 0
#define AX_VARIANT_F64_NATIVE 1 /* fp64 FMA units                           */
#define AX_VARIANT_F64_DF 2     /* pairs of fp32 (double-float) arithmetic   */
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

/* Global node id of every local point of the structured box (x fastest):
 * glob = X + NX*(Y + NY*Z), X = ex*(lx-1)+i, NX = nx*(lx-1)+1, ... */
int ax_box_numbering(int nx, int ny, int nz, int lx, int64_t *glob);

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
