/*
 * Oracle for the matrix-free spectral-element stiffness apply ("Ax").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code with the CUDA library and nothing here is tuned.
 *
 * What it computes (Sec. "The Kernel Expressed in DaCe", Listing 2, and the
 * weak form of Poisson's equation in Sec. "The Spectral Element Method"): for
 * every element e, independently,
 *
 *   grad:  ur = D_r u,  us = D_s u,  ut = D_t u        (reference gradient)
 *   geom:  [wr ws wt]^T = h1 * G * [ur us ut]^T       (G symmetric 3x3)
 *   div:   w = D_r^T wr + D_s^T ws + D_t^T wt         (transposed gradient)
 *
 * where D_r applies the 1-D GLL differentiation matrix along i, D_s along j
 * and D_t along k of an element stored [k][j][i] (i fastest).
 *
 * Buffer convention for the 1-D matrices, read from Listing 2 (the r-sum
 * multiplies dxd[l,i] by u[e,k,j,l]; the transposed sum multiplies
 * dxtd[l,i] by urtmp[e,k,j,l]):
 *     dx[l*lx + i]  = D_{i l}   (derivative at node i of the l-th basis
 *                                 function),
 *     dxt[l*lx + i] = D_{l i}.
 * The same holds for dy/dyt along j and dz/dzt along k.
 *
 * Everything is plain fp64 with a straightforward l-ascending sum; the
 * element loop carries an OpenMP pragma and nothing else.
 */
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the element loop (timing only; results do not depend on it). */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static size_t at(int lx, size_t e, int k, int j, int i)
{
    return ((e * (size_t)lx + (size_t)k) * (size_t)lx + (size_t)j) * (size_t)lx + (size_t)i;
}

/* Returns 0 on success, -1 on bad sizes, -2 if the scratch allocation fails. */
int oracle_ax_helm(double *w, const double *u,
                   const double *dx, const double *dy, const double *dz,
                   const double *dxt, const double *dyt, const double *dzt,
                   const double *h1,
                   const double *g11, const double *g22, const double *g33,
                   const double *g12, const double *g13, const double *g23,
                   int lx, int nel)
{
    if (lx < 1 || nel < 0)
        return -1;
    const size_t n3 = (size_t)lx * lx * lx;
    int status = 0;

#pragma omp parallel
    {
        /* element-local transients: the reference gradient and the
           geometry-weighted gradient of one element */
        double *ur = (double *)malloc(6 * n3 * sizeof(double));
        if (!ur) {
#pragma omp atomic write
            status = -2;
        } else {
            double *us = ur + n3, *ut = us + n3;
            double *wr = ut + n3, *ws = wr + n3, *wt = ws + n3;
#pragma omp for schedule(static)
            for (long long el = 0; el < (long long)nel; ++el) {
                const size_t e = (size_t)el;
                /* reference gradient: one 1-D derivative per direction */
                for (int k = 0; k < lx; ++k)
                    for (int j = 0; j < lx; ++j)
                        for (int i = 0; i < lx; ++i) {
                            double r = 0.0, s = 0.0, t = 0.0;
                            for (int l = 0; l < lx; ++l) {
                                r += dx[l * lx + i] * u[at(lx, e, k, j, l)];
                                s += dy[l * lx + j] * u[at(lx, e, k, l, i)];
                                t += dz[l * lx + k] * u[at(lx, e, l, j, i)];
                            }
                            const size_t p = ((size_t)k * lx + j) * lx + i;
                            ur[p] = r;
                            us[p] = s;
                            ut[p] = t;
                        }
                /* pointwise metric tensor times the coefficient */
                for (size_t p = 0; p < n3; ++p) {
                    const size_t q = e * n3 + p;
                    const double a = ur[p], b = us[p], c = ut[p];
                    wr[p] = h1[q] * (g11[q] * a + g12[q] * b + g13[q] * c);
                    ws[p] = h1[q] * (g12[q] * a + g22[q] * b + g23[q] * c);
                    wt[p] = h1[q] * (g13[q] * a + g23[q] * b + g33[q] * c);
                }
                /* transposed gradient, summed over the three directions */
                for (int k = 0; k < lx; ++k)
                    for (int j = 0; j < lx; ++j)
                        for (int i = 0; i < lx; ++i) {
                            double acc_r = 0.0, acc_s = 0.0, acc_t = 0.0;
                            for (int l = 0; l < lx; ++l) {
                                acc_r += dxt[l * lx + i] * wr[((size_t)k * lx + j) * lx + l];
                                acc_s += dyt[l * lx + j] * ws[((size_t)k * lx + l) * lx + i];
                                acc_t += dzt[l * lx + k] * wt[((size_t)l * lx + j) * lx + i];
                            }
                            w[at(lx, e, k, j, i)] = acc_r + acc_s + acc_t;
                        }
            }
            free(ur);
        }
    }
    return status;
}

/*
 * Direct-stiffness summation (gather-scatter "dssum", the second main
 * ingredient named in Sec. "Neko and Small Tensor Kernel"): every local copy
 * of a global node receives the sum over all local copies of that node.
 * glob[p] in [0, nglob) is the global id of local point p.  Plain dense
 * scatter-add into a global array, then gather.  Returns 0, or -2 if the
 * scratch allocation fails.
 */
int oracle_gs_sum(double *v, const long long *glob, long long n, long long nglob)
{
    double *acc = (double *)calloc((size_t)(nglob > 0 ? nglob : 1), sizeof(double));
    if (!acc)
        return -2;
    for (long long p = 0; p < n; ++p)
        acc[glob[p]] += v[p];
    for (long long p = 0; p < n; ++p)
        v[p] = acc[glob[p]];
    free(acc);
    return 0;
}
