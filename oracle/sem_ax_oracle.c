/*
 * Plain FP64 CPU oracle for the element-local spectral-element Laplacian
 * operator ("Ax").  TEST INFRASTRUCTURE ONLY: it is used by the tests, by the
 * smoke check and by the benchmark's CPU-baseline leg, never by the library.
 * It shares no source with the CUDA path.
 *
 * Definition (textbook SEM, Deville, Fischer & Mund 2002, Sec. 4.4; the kind
 * of Fortran PDE array kernel the paper's Section 3 front-end ingests and its
 * Section 1 names as a use case): for each element e with u_e of n^3 nodal
 * values stored [k][j][i] (i fastest, the Fortran u(i,j,k,e) order),
 *
 *   ur[k][j][i] = sum_l D[i][l] u[k][j][l]
 *   us[k][j][i] = sum_l D[j][l] u[k][l][i]
 *   ut[k][j][i] = sum_l D[k][l] u[l][j][i]
 *
 *   [wr ws wt]^T = G_p [ur us ut]^T,  G_p symmetric 3x3 from the six stored
 *   components (rr, rs, rt, ss, st, tt), layout G[e][6][k][j][i]
 *
 *   w[k][j][i] = sum_l D[l][i] wr[k][j][l] + sum_l D[l][j] ws[k][l][i]
 *              + sum_l D[l][k] wt[l][j][i]
 *
 * i.e. w_e = sum_{a,b} D_a^T diag(G_ab) D_b u_e.  w is overwritten.
 * Written as the literal loop nest, in that order, in double precision; build
 * with -O2 -ffp-contract=off so no fused multiply-add changes the rounding.
 */
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static void ax_one_element(int n, const double *u, const double *G,
                           const double *D, double *w, double *scratch)
{
    const int n3 = n * n * n;
    double *ur = scratch, *us = scratch + n3, *ut = scratch + 2 * n3;
    const double *Grr = G, *Grs = G + n3, *Grt = G + 2 * n3;
    const double *Gss = G + 3 * n3, *Gst = G + 4 * n3, *Gtt = G + 5 * n3;

    /* gradient in reference coordinates */
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double a = 0.0, b = 0.0, c = 0.0;
                for (int l = 0; l < n; ++l) {
                    a += D[i * n + l] * u[(k * n + j) * n + l];
                    b += D[j * n + l] * u[(k * n + l) * n + i];
                    c += D[k * n + l] * u[(l * n + j) * n + i];
                }
                const int p = (k * n + j) * n + i;
                ur[p] = a; us[p] = b; ut[p] = c;
            }

    /* multiply by the symmetric geometric factor, in place */
    for (int p = 0; p < n3; ++p) {
        const double r = ur[p], s = us[p], t = ut[p];
        ur[p] = Grr[p] * r + Grs[p] * s + Grt[p] * t;
        us[p] = Grs[p] * r + Gss[p] * s + Gst[p] * t;
        ut[p] = Grt[p] * r + Gst[p] * s + Gtt[p] * t;
    }

    /* transposed derivative, summed over the three directions */
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double acc = 0.0;
                for (int l = 0; l < n; ++l) acc += D[l * n + i] * ur[(k * n + j) * n + l];
                for (int l = 0; l < n; ++l) acc += D[l * n + j] * us[(k * n + l) * n + i];
                for (int l = 0; l < n; ++l) acc += D[l * n + k] * ut[(l * n + j) * n + i];
                w[(k * n + j) * n + i] = acc;
            }
}

/* Apply Ax to E elements of order N (n = N+1 nodes per direction).
 * nthreads <= 0 uses the OpenMP default.  Returns the number of threads used,
 * or -1 on bad arguments or allocation failure. */
int oracle_sem_ax(int64_t E, int N, const double *u, const double *G,
                  const double *D, double *w, int nthreads)
{
    if (E < 0 || N < 1 || N > 63) return -1;
    const int n = N + 1;
    const int64_t n3 = (int64_t)n * n * n;
    int used = 1, failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel reduction(+ : failed)
    {
#pragma omp single
        used = omp_get_num_threads();
#else
    (void)nthreads;
    {
#endif
        double *scratch = (double *)malloc(sizeof(double) * 3 * (size_t)n3);
        if (!scratch) failed = 1;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t e = 0; e < E; ++e)
            if (scratch)
                ax_one_element(n, u + e * n3, G + e * 6 * n3, D, w + e * n3, scratch);
        free(scratch);
    }
    return failed ? -1 : used;
}

/* Helmholtz form w = h1 A u + h2 B u, B the diagonal mass matrix (one value
 * per node): the operator above followed by the diagonal term, as defined. */
int oracle_sem_helmholtz(int64_t E, int N, const double *u, const double *G, const double *B,
                         const double *D, double h1, double h2, double *w, int nthreads)
{
    int used = oracle_sem_ax(E, N, u, G, D, w, nthreads);
    if (used < 0) return used;
    const int64_t count = E * (int64_t)(N + 1) * (N + 1) * (N + 1);
    for (int64_t p = 0; p < count; ++p) w[p] = h1 * w[p] + h2 * B[p] * u[p];
    return used;
}
