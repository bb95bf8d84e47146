/*
 * oracle.h -- plain FP64 CPU oracle for the tiled right-looking Cholesky
 * factorization (paper Section 3.1, Fig. 1) and the SPD solve built on it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this code: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py use it.  It shares no source with the CUDA
 * library under paper_2606_11937_gb300/csrc.
 *
 * Conventions (shared by every function here):
 *   - matrices are column-major with a leading dimension (LAPACK uplo='L');
 *     element (i, j) of A lives at A[j * lda + i];
 *   - only the lower triangle including the diagonal is read or written; the
 *     strict upper triangle is never touched (Section 3.1: only the diagonal
 *     and the strictly lower part are stored);
 *   - failures are reported LAPACK-style: info = 1-based index of the first
 *     column whose pivot is not positive (or is NaN), 0 on success.
 *   - arithmetic is IEEE binary64, one rounding per + - * / sqrt, in the order
 *     written; the build passes -ffp-contract=off so no FMA contraction occurs.
 */
#ifndef CHOL_ORACLE_H
#define CHOL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Unblocked Cholesky-Crout, column by column (the plain definition A = L L^T,
 * L lower with a positive diagonal).  Sums run in ascending k. */
int64_t oracle_potrf_unblocked(int64_t n, double *A, int64_t lda);

/* Tile operations of Section 3.1 on nb x nb tiles stored ROW-major
 * (element (r, c) at T[r * nb + c]).  Each is the formula of the paper with
 * scalar loops:
 *   potrf: T <- chol(T) (lower), returns tile-local info
 *   trsm:  B <- B * L^{-T}        (right side, L lower, non-unit)
 *   syrk:  C <- C - A * A^T       (lower triangle of C only)
 *   gemm:  C <- C - A * B^T                                              */
int64_t oracle_potrf_tile(int64_t nb, double *T);
void oracle_trsm_tile(int64_t nb, const double *L, double *B);
void oracle_syrk_tile(int64_t nb, const double *A, double *C);
void oracle_gemm_tile(int64_t nb, const double *A, const double *B, double *C);

/* Fig. 1 transcribed: tiles of order nb, M = ceil(n / nb) per dimension, the
 * ragged last tile padded with the identity on its padded diagonal (the
 * factor of diag(A, I) is diag(L, I)).  counts[0..3] receive the number of
 * POTRF, TRSM, SYRK and GEMM tasks executed (may be NULL).  If log is not
 * NULL, each executed task appends 4 int32 values (type 0..3, I, K, J) to it;
 * log must hold 4 * (number of tasks) entries. */
int64_t oracle_potrf_tiled(int64_t n, int64_t nb, double *A, int64_t lda,
                           int64_t counts[4], int32_t *log);

/* The same Fig. 1 task graph expressed with OpenMP task dependencies on the
 * tiles (Section 3.2, "Task asynchronous"), run on nthreads threads.  Used
 * only as the timed CPU baseline; every tile sees its updates in ascending J,
 * so its result is bitwise that of oracle_potrf_tiled. */
int64_t oracle_potrf_tiled_tasks(int64_t n, int64_t nb, double *A, int64_t lda,
                                 int nthreads);
int oracle_max_threads(void);

/* B <- A^{-1} B given the factor L (lower, column-major): forward substitution
 * L Y = B, then backward substitution L^T X = Y, column by column. */
void oracle_potrs(int64_t n, int64_t nrhs, const double *L, int64_t ldl,
                  double *B, int64_t ldb);

/* ||A - L L^T||_F / ||A||_F with A symmetric, given by its lower triangle.
 * O(n^3). */
double oracle_residual_fro(int64_t n, const double *A, int64_t lda,
                           const double *L, int64_t ldl);

/* Randomized residual estimate: ||A X - L (L^T X)||_F / ||A X||_F for the k
 * probe columns X (n x k, column-major, ld n).  O(n^2 k). */
double oracle_residual_probe(int64_t n, const double *A, int64_t lda,
                             const double *L, int64_t ldl, int64_t k,
                             const double *X);

/* Normwise backward error of a solve (Rigal-Gaches), max over columns:
 *   ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf).
 * A symmetric, given by its lower triangle. */
double oracle_backward_error(int64_t n, int64_t nrhs, const double *A,
                             int64_t lda, const double *X, int64_t ldx,
                             const double *B, int64_t ldb);

#ifdef __cplusplus
}
#endif
#endif
