/*
 * chol_testing.h -- test hooks of libchol.so.  Not part of the factorization
 * API; they expose single kernels so tests can check them in isolation.
 */
#ifndef CHOL_TESTING_H
#define CHOL_TESTING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One tcgen05 SYRK/GEMM tile update, the tensor-core kernel of the
 * mixed-precision trailing update (Section 3.1 SYRK and GEMM formulas,
 * A_IK <- A_IK - A_IJ A_KJ^T), run twice by one CTA:
 *     C[r] <- C[r] - 2^-eA 2^-eB sum_p A_p B_p^T,   r = 0, 1
 * precision: CHOL_BF16 / CHOL_FP16 (one product of 16-bit operands),
 * CHOL_TF32 (one product of tf32-valued binary32 operands) or CHOL_FP32
 * (three products hi*hi + hi*lo + lo*hi).  nb in {128, 256, 512, 1024}.
 * ops (device): the hi operand array of 2*nb rows x nb columns, row-major
 * (rows [0, nb) = A, rows [nb, 2 nb) = B), 2-byte elements for BF16/FP16 and
 * 4-byte for TF32/FP32; for CHOL_FP32 the lo array of the same shape follows.
 * C (device): two row-major nb x nb binary32 tiles, contiguous.  lower != 0:
 * only the sub-tiles on or below the diagonal are updated (SYRK).
 * Returns CHOL_OK, CHOL_ERR_ARG, CHOL_ERR_CUDA or CHOL_ERR_TIMEOUT (a bounded
 * wait expired). */
int chol_test_tc_update(int32_t precision, int64_t nb, const void *ops, int32_t eA, int32_t eB, float *C,
                        int32_t lower);

/* One binary64-accurate tensor-core tile update (the CHOL_FLAG_FP64_TC GEMM,
 * Section 3.1 GEMM formula), run twice by one CTA after the operands are
 * split into bf16 slices on the device:
 *     C[r] <- C[r] - A B^T,   r = 0, 1
 * A, B: 128 x 128 row-major binary64 tiles; C: two contiguous 128 x 128
 * row-major binary64 tiles; all device pointers.  Returns CHOL_OK,
 * CHOL_ERR_CUDA or CHOL_ERR_TIMEOUT. */
int chol_test_ozaki_update(const double *A, const double *B, double *C);

/* The refinement residual on the tensor cores alone: R = B - A X (B may be
 * NULL: R = -A X) with binary64 accuracy from exact bf16 slicing of A (every
 * 128 x 128 tile, rows scaled per tile) and X (per 128-row block and column).
 * A: n x n symmetric, only its lower triangle is read (column-major, lda);
 * X, B, R: n x nrhs column-major; all device pointers.  Allocates and frees
 * its own scratch (about n^2 / 2 bytes x 8 for the slices).  Returns CHOL_OK,
 * CHOL_ERR_ARG, CHOL_ERR_CUDA or CHOL_ERR_TIMEOUT. */
int chol_test_oz_residual(int64_t n, const double *A, int64_t lda, const double *X, int64_t ldx,
                          const double *B, int64_t ldb, double *R, int64_t ldr, int64_t nrhs);

/* Memory the current device has in use, for tests that check that a call
 * allocates nothing: the device's free bytes (cudaMemGetInfo) and the bytes in
 * use and reserved by its default stream-ordered pool (the pool the library's
 * workspaces come from).  Returns CHOL_OK or CHOL_ERR_CUDA. */
int chol_test_device_memory(uint64_t *free_bytes, uint64_t *pool_used, uint64_t *pool_reserved);

#ifdef __cplusplus
}
#endif
#endif
