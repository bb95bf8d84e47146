/*
 * oracle.c -- plain, slow, obviously correct FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * CPU legs of bench.py, never by the CUDA library.  See oracle.h for the
 * conventions.  Every function follows a passage of the paper or the plain
 * mathematical definition; each says which.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* element (i, j) of a column-major matrix with leading dimension ld */
#define CM(A, ld, i, j) ((A)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

/* ------------------------------------------------------------------------ */
/* Unblocked Cholesky-Crout: the plain definition of the factor.              */
/*   L_jj = sqrt(A_jj - sum_{k<j} L_jk^2)                                     */
/*   L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj,   i > j                      */
/* A working copy W holds the lower triangle row-major (row i contiguous), so  */
/* the inner products run over contiguous memory; the arithmetic and its order */
/* are exactly the two formulas above.                                        */
/* ------------------------------------------------------------------------ */
int64_t oracle_potrf_unblocked(int64_t n, double *A, int64_t lda)
{
    if (n <= 0) return 0;
    double *W = (double *)malloc((size_t)n * (size_t)n * sizeof(double));
    if (!W) return -1;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = 0; k <= i; ++k) W[i * n + k] = CM(A, lda, i, k);

    int64_t info = 0;
    for (int64_t j = 0; j < n && info == 0; ++j) {
        const double *Lj = W + j * n;
        double d = W[j * n + j];
        for (int64_t k = 0; k < j; ++k) d -= Lj[k] * Lj[k];
        if (!(d > 0.0)) {           /* pivot <= 0 or NaN */
            info = j + 1;
            break;
        }
        const double ljj = sqrt(d);
        W[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            const double *Li = W + i * n;
            double s = Li[j];
            for (int64_t k = 0; k < j; ++k) s -= Li[k] * Lj[k];
            W[i * n + j] = s / ljj;
        }
    }
    /* write back the columns that were completed (all of them on success) */
    const int64_t done = info ? info - 1 : n;
    for (int64_t j = 0; j < done; ++j)
        for (int64_t i = j; i < n; ++i) CM(A, lda, i, j) = W[i * n + j];
    free(W);
    return info;
}

/* ------------------------------------------------------------------------ */
/* Tile operations (Section 3.1), tiles row-major: T[r * nb + c].             */
/* ------------------------------------------------------------------------ */
#define RM(T, nb, r, c) ((T)[(size_t)(r) * (size_t)(nb) + (size_t)(c)])

/* POTRF: A_JJ <- chol(A_JJ).  The same Crout formulas as above on one tile. */
int64_t oracle_potrf_tile(int64_t nb, double *T)
{
    for (int64_t j = 0; j < nb; ++j) {
        double d = RM(T, nb, j, j);
        for (int64_t k = 0; k < j; ++k) d -= RM(T, nb, j, k) * RM(T, nb, j, k);
        if (!(d > 0.0)) return j + 1;
        const double ljj = sqrt(d);
        RM(T, nb, j, j) = ljj;
        for (int64_t i = j + 1; i < nb; ++i) {
            double s = RM(T, nb, i, j);
            for (int64_t k = 0; k < j; ++k) s -= RM(T, nb, i, k) * RM(T, nb, j, k);
            RM(T, nb, i, j) = s / ljj;
        }
    }
    return 0;
}

/* TRSM: A_IJ <- A_IJ A_JJ^{-T}, i.e. solve X L^T = B for X (L = A_JJ lower).
 * Row r of X satisfies L x_r^T = b_r^T: forward substitution over columns. */
void oracle_trsm_tile(int64_t nb, const double *L, double *B)
{
    for (int64_t r = 0; r < nb; ++r) {
        for (int64_t j = 0; j < nb; ++j) {
            double x = RM(B, nb, r, j);
            for (int64_t k = 0; k < j; ++k) x -= RM(B, nb, r, k) * RM(L, nb, j, k);
            RM(B, nb, r, j) = x / RM(L, nb, j, j);
        }
    }
}

/* SYRK: A_II <- A_II - A_IJ A_IJ^T, lower triangle of A_II only. */
void oracle_syrk_tile(int64_t nb, const double *A, double *C)
{
    for (int64_t i = 0; i < nb; ++i)
        for (int64_t j = 0; j <= i; ++j) {
            double s = RM(C, nb, i, j);
            for (int64_t k = 0; k < nb; ++k) s -= RM(A, nb, i, k) * RM(A, nb, j, k);
            RM(C, nb, i, j) = s;
        }
}

/* GEMM: A_IK <- A_IK - A_IJ A_KJ^T. */
void oracle_gemm_tile(int64_t nb, const double *A, const double *B, double *C)
{
    for (int64_t i = 0; i < nb; ++i)
        for (int64_t j = 0; j < nb; ++j) {
            double s = RM(C, nb, i, j);
            for (int64_t k = 0; k < nb; ++k) s -= RM(A, nb, i, k) * RM(B, nb, j, k);
            RM(C, nb, i, j) = s;
        }
}

/* ------------------------------------------------------------------------ */
/* Tile storage (Section 3.1: only diagonal and strictly lower tiles).       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n, nb, M;
    double *t;            /* M(M+1)/2 tiles of nb*nb, tile (I,J) at index I(I+1)/2+J */
} tiles_t;

static double *tile(const tiles_t *S, int64_t I, int64_t J)
{
    return S->t + (size_t)(I * (I + 1) / 2 + J) * (size_t)(S->nb * S->nb);
}

/* Copy lower(A) into tiles; entries beyond n are the identity (diagonal 1,
 * everything else 0), so the padded matrix is diag(A, I). */
static int tiles_pack(tiles_t *S, int64_t n, int64_t nb, const double *A, int64_t lda)
{
    S->n = n;
    S->nb = nb;
    S->M = (n + nb - 1) / nb;
    const size_t count = (size_t)(S->M * (S->M + 1) / 2) * (size_t)(nb * nb);
    S->t = (double *)calloc(count, sizeof(double));
    if (!S->t) return -1;
    for (int64_t I = 0; I < S->M; ++I)
        for (int64_t J = 0; J <= I; ++J) {
            double *T = tile(S, I, J);
            for (int64_t r = 0; r < nb; ++r)
                for (int64_t c = 0; c < nb; ++c) {
                    const int64_t i = I * nb + r, j = J * nb + c;
                    double v = 0.0;
                    if (i < n && j < n) {
                        if (j <= i) v = CM(A, lda, i, j);
                        else v = CM(A, lda, j, i); /* upper half of a diagonal tile: mirror of lower */
                    } else if (i == j) {
                        v = 1.0;
                    }
                    RM(T, nb, r, c) = v;
                }
        }
    return 0;
}

/* Copy the lower triangle of the first `cols` columns back into A. */
static void tiles_unpack(const tiles_t *S, double *A, int64_t lda, int64_t cols)
{
    const int64_t nb = S->nb;
    for (int64_t j = 0; j < cols; ++j)
        for (int64_t i = j; i < S->n; ++i)
            CM(A, lda, i, j) = RM(tile(S, i / nb, j / nb), nb, i % nb, j % nb);
}

/* Fig. 1, line by line in meaning: for each block column J, POTRF on the
 * diagonal tile, TRSM on every tile below it, then SYRK on each trailing
 * diagonal tile and GEMM on each trailing off-diagonal tile. */
int64_t oracle_potrf_tiled(int64_t n, int64_t nb, double *A, int64_t lda,
                           int64_t counts[4], int32_t *log)
{
    if (counts) counts[0] = counts[1] = counts[2] = counts[3] = 0;
    if (n <= 0) return 0;
    if (nb <= 0) return -1;
    tiles_t S;
    if (tiles_pack(&S, n, nb, A, lda)) return -1;
    const int64_t M = S.M;
    int64_t ntask = 0;
#define LOG(ty, I, K, J)                                   \
    do {                                                  \
        if (log) {                                        \
            log[4 * ntask + 0] = (ty);                    \
            log[4 * ntask + 1] = (int32_t)(I);            \
            log[4 * ntask + 2] = (int32_t)(K);            \
            log[4 * ntask + 3] = (int32_t)(J);            \
        }                                                 \
        ++ntask;                                          \
        if (counts) counts[ty] += 1;                      \
    } while (0)

    int64_t info = 0;
    for (int64_t J = 0; J < M; ++J) {
        LOG(0, J, J, J);
        const int64_t ti = oracle_potrf_tile(nb, tile(&S, J, J));
        if (ti) {
            info = J * nb + ti;
            break;
        }
        for (int64_t I = J + 1; I < M; ++I) {
            LOG(1, I, J, J);
            oracle_trsm_tile(nb, tile(&S, J, J), tile(&S, I, J));
        }
        for (int64_t I = J + 1; I < M; ++I) {
            LOG(2, I, I, J);
            oracle_syrk_tile(nb, tile(&S, I, J), tile(&S, I, I));
            for (int64_t K = J + 1; K < I; ++K) {
                LOG(3, I, K, J);
                oracle_gemm_tile(nb, tile(&S, I, J), tile(&S, K, J), tile(&S, I, K));
            }
        }
    }
#undef LOG
    tiles_unpack(&S, A, lda, info ? (info - 1) / nb * nb : n);
    free(S.t);
    return info;
}

/* The same task graph with OpenMP 4.0 task dependencies (Section 3.2, "Task
 * asynchronous"): each task names the tiles it reads (in) and the tile it
 * writes (inout).  Tasks that write the same tile run in the order they were
 * created, i.e. ascending J, which is the order of the sequential version. */
int64_t oracle_potrf_tiled_tasks(int64_t n, int64_t nb, double *A, int64_t lda,
                                 int nthreads)
{
    if (n <= 0) return 0;
    if (nb <= 0) return -1;
    tiles_t S;
    if (tiles_pack(&S, n, nb, A, lda)) return -1;
    const int64_t M = S.M;
    int64_t *tinfo = (int64_t *)calloc((size_t)M, sizeof(int64_t));
    if (!tinfo) {
        free(S.t);
        return -1;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
#pragma omp single
    {
        for (int64_t J = 0; J < M; ++J) {
            double *Tjj = tile(&S, J, J);
#pragma omp task depend(inout : Tjj[0]) firstprivate(J, Tjj)
            tinfo[J] = oracle_potrf_tile(nb, Tjj);
            for (int64_t I = J + 1; I < M; ++I) {
                double *Tij = tile(&S, I, J);
#pragma omp task depend(in : Tjj[0]) depend(inout : Tij[0]) firstprivate(Tjj, Tij)
                oracle_trsm_tile(nb, Tjj, Tij);
            }
            for (int64_t I = J + 1; I < M; ++I) {
                double *Tij = tile(&S, I, J), *Tii = tile(&S, I, I);
#pragma omp task depend(in : Tij[0]) depend(inout : Tii[0]) firstprivate(Tij, Tii)
                oracle_syrk_tile(nb, Tij, Tii);
                for (int64_t K = J + 1; K < I; ++K) {
                    double *Tkj = tile(&S, K, J), *Tik = tile(&S, I, K);
#pragma omp task depend(in : Tij[0], Tkj[0]) depend(inout : Tik[0]) firstprivate(Tij, Tkj, Tik)
                    oracle_gemm_tile(nb, Tij, Tkj, Tik);
                }
            }
        }
    }
    int64_t info = 0;
    for (int64_t J = 0; J < M; ++J)
        if (tinfo[J]) {
            info = J * nb + tinfo[J];
            break;
        }
    tiles_unpack(&S, A, lda, info ? (info - 1) / nb * nb : n);
    free(tinfo);
    free(S.t);
    return info;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Solve A X = B with A = L L^T: L Y = B (forward), L^T X = Y (backward).     */
/* ------------------------------------------------------------------------ */
void oracle_potrs(int64_t n, int64_t nrhs, const double *L, int64_t ldl,
                  double *B, int64_t ldb)
{
    for (int64_t c = 0; c < nrhs; ++c) {
        double *b = B + (size_t)c * (size_t)ldb;
        for (int64_t i = 0; i < n; ++i) {          /* y_i = (b_i - sum_{k<i} L_ik y_k) / L_ii */
            double s = b[i];
            for (int64_t k = 0; k < i; ++k) s -= CM(L, ldl, i, k) * b[k];
            b[i] = s / CM(L, ldl, i, i);
        }
        for (int64_t i = n - 1; i >= 0; --i) {     /* x_i = (y_i - sum_{k>i} L_ki x_k) / L_ii */
            double s = b[i];
            for (int64_t k = i + 1; k < n; ++k) s -= CM(L, ldl, k, i) * b[k];
            b[i] = s / CM(L, ldl, i, i);
        }
    }
}

/* symmetric A from its lower triangle */
static double sym(const double *A, int64_t lda, int64_t i, int64_t j)
{
    return i >= j ? CM(A, lda, i, j) : CM(A, lda, j, i);
}

double oracle_residual_fro(int64_t n, const double *A, int64_t lda,
                           const double *L, int64_t ldl)
{
    double num = 0.0, den = 0.0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) {
            /* (L L^T)_ij = sum_{k <= min(i,j)} L_ik L_jk */
            const int64_t m = i < j ? i : j;
            double s = 0.0;
            for (int64_t k = 0; k <= m; ++k) s += CM(L, ldl, i, k) * CM(L, ldl, j, k);
            const double a = sym(A, lda, i, j);
            num += (a - s) * (a - s);
            den += a * a;
        }
    return den > 0.0 ? sqrt(num / den) : sqrt(num);
}

double oracle_residual_probe(int64_t n, const double *A, int64_t lda,
                             const double *L, int64_t ldl, int64_t k,
                             const double *X)
{
    double *t = (double *)malloc((size_t)n * sizeof(double));
    if (!t) return -1.0;
    double num = 0.0, den = 0.0;
    for (int64_t c = 0; c < k; ++c) {
        const double *x = X + (size_t)c * (size_t)n;
        /* t = L^T x:  t_j = sum_{i >= j} L_ij x_i */
        for (int64_t j = 0; j < n; ++j) {
            double s = 0.0;
            for (int64_t i = j; i < n; ++i) s += CM(L, ldl, i, j) * x[i];
            t[j] = s;
        }
        for (int64_t i = 0; i < n; ++i) {
            double ax = 0.0, llx = 0.0;
            for (int64_t j = 0; j < n; ++j) ax += sym(A, lda, i, j) * x[j];
            for (int64_t j = 0; j <= i; ++j) llx += CM(L, ldl, i, j) * t[j];
            num += (ax - llx) * (ax - llx);
            den += ax * ax;
        }
    }
    free(t);
    return den > 0.0 ? sqrt(num / den) : sqrt(num);
}

double oracle_backward_error(int64_t n, int64_t nrhs, const double *A,
                             int64_t lda, const double *X, int64_t ldx,
                             const double *B, int64_t ldb)
{
    double anorm = 0.0;                        /* ||A||_inf = max row sum of |A| */
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s += fabs(sym(A, lda, i, j));
        if (s > anorm) anorm = s;
    }
    double worst = 0.0;
    for (int64_t c = 0; c < nrhs; ++c) {
        const double *x = X + (size_t)c * (size_t)ldx;
        const double *b = B + (size_t)c * (size_t)ldb;
        double rn = 0.0, xn = 0.0, bn = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double r = b[i];
            for (int64_t j = 0; j < n; ++j) r -= sym(A, lda, i, j) * x[j];
            if (fabs(r) > rn) rn = fabs(r);
            if (fabs(x[i]) > xn) xn = fabs(x[i]);
            if (fabs(b[i]) > bn) bn = fabs(b[i]);
        }
        const double den = anorm * xn + bn;
        const double e = den > 0.0 ? rn / den : rn;
        if (e > worst) worst = e;
    }
    return worst;
}
