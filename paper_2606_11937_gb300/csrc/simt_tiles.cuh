// simt_tiles.cuh -- CTA-wide tile kernels of Section 3.1 on CUDA cores
// (DFMA for binary64, FFMA for binary32), for 256-thread CTAs.
//
// Tiles are nb x nb, row-major (element (r, c) at r * ld + c).  Every routine
// is executed by the first 256 threads of the CTA (all of it for 256-thread
// bodies) and ends with a barrier among them (named barrier 2, simt_sync).
//   tile_potrf : A_JJ <- chol(A_JJ)                   (lower; returns local info)
//   tile_trsm  : A_IJ <- A_IJ A_JJ^{-T}
//   tile_syrk  : A_II <- A_II - A_IJ A_IJ^T           (lower triangle only)
//   tile_gemm  : A_IK <- A_IK - A_IJ A_KJ^T
// All of them reduce to one primitive, block_nt_update, which subtracts a
// 64 x 64 block of A B^T from C with operand chunks staged through shared
// memory.  The arithmetic order inside each routine is fixed, so every
// schedule that runs the same tasks in the same per-tile order produces the
// same bits.
#pragma once

#include "common.cuh"

namespace chol {

constexpr int kThreads = 256;

// Barrier among threads 0..255: the tile routines below synchronise with it,
// so a body with more threads runs them on its first 256 threads only.
__device__ __forceinline__ void simt_sync() { asm volatile("bar.sync 2, 256;" ::: "memory"); }
constexpr int kBlk = 64;   // output block edge of block_nt_update
constexpr int kBK = 16;    // k-chunk staged per iteration
constexpr int kIB = 32;    // panel width of the blocked POTRF / TRSM

template <typename T>
struct SimtSmem {
    T As[kBK][kBlk + 1];
    T Bs[kBK][kBlk + 1];
    T D[kIB][kIB + 1];     // diagonal block of the blocked POTRF / TRSM
    T Dinv[kIB];           // reciprocals of its diagonal
    int flag;
};

// loads of tile data bypass L1 (L2 is the coherence point between SMs that
// exchange tiles inside one persistent kernel)
template <typename T>
__device__ __forceinline__ T ldg_cg(const T *p) { return __ldcg(p); }

template <typename T> __device__ __forceinline__ T t_sqrt(T x);
template <> __device__ __forceinline__ double t_sqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float t_sqrt<float>(float x) { return sqrtf(x); }

// C[0:m, 0:n] -= A[0:m, 0:k] * B[0:n, 0:k]^T  (m, n <= 16 * MI).
// LOWER: only entries with column <= row are written (diagonal blocks of SYRK).
// The 256 threads form a 16 x 16 grid; thread (ty, tx) owns the MI x MI
// outputs (ty + 16 i, tx + 16 j).  MI = 4 gives 64 x 64 blocks, MI = 2 gives
// 32 x 32 blocks (used for tiles of order <= 32 so no lane computes padding).
template <typename T, bool LOWER, int MI>
__device__ void block_nt_update(T *C, int ldc, const T *A, int lda, const T *B, int ldb,
                                int m, int n, int k, SimtSmem<T> &sm) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[MI][MI];
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < MI; ++j) acc[i][j] = T(0);

    // binary32: the next k-chunk's operands are loaded into registers while the
    // current one is applied (FFMA leaves the loads' latency exposed); binary64
    // keeps the register budget that lets two CTAs share an SM (DFMA-bound)
    constexpr bool kPipe = sizeof(T) == 4;
    constexpr int NQ = (16 * MI * kBK) / kThreads;
    T pa[NQ], pb[NQ];
    auto load_chunk = [&](int k0) {
        const int kc = min(kBK, k - k0);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int e = threadIdx.x + kThreads * q;
            const int r = e / kBK, kk = e % kBK;
            pa[q] = (r < m && kk < kc) ? ldg_cg(A + (size_t)r * lda + k0 + kk) : T(0);
            pb[q] = (r < n && kk < kc) ? ldg_cg(B + (size_t)r * ldb + k0 + kk) : T(0);
        }
    };
    if (kPipe && k > 0) load_chunk(0);
    for (int k0 = 0; k0 < k; k0 += kBK) {
        if (!kPipe) load_chunk(k0);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int e = threadIdx.x + kThreads * q;
            const int r = e / kBK, kk = e % kBK;
            sm.As[kk][r] = pa[q];
            sm.Bs[kk][r] = pb[q];
        }
        simt_sync();
        if (kPipe && k0 + kBK < k) load_chunk(k0 + kBK);
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            T a[MI], b[MI];
#pragma unroll
            for (int i = 0; i < MI; ++i) a[i] = sm.As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < MI; ++j) b[j] = sm.Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int j = 0; j < MI; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        simt_sync();
    }
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < MI; ++j) {
            const int r = ty + 16 * i, c = tx + 16 * j;
            if (r < m && c < n && (!LOWER || c <= r)) {
                T *p = C + (size_t)r * ldc + c;
                *p = ldg_cg(p) - acc[i][j];
            }
        }
    simt_sync();
}

// Subtract A B^T from the block region C[0:m, 0:n] (any m, n) by 64 x 64 (or
// 32 x 32 when both tile edges are <= 32) blocks; LOWER_DIAG: the region is
// square and only its lower triangle is updated.
template <typename T, bool LOWER_DIAG>
__device__ void region_nt_update(T *C, int ldc, const T *A, int lda, const T *B, int ldb,
                                 int m, int n, int k, SimtSmem<T> &sm) {
    if (m <= 32 && n <= 32) {
        block_nt_update<T, LOWER_DIAG, 2>(C, ldc, A, lda, B, ldb, m, n, k, sm);
        return;
    }
    for (int bi = 0; bi < m; bi += kBlk)
        for (int bj = 0; bj < n && (!LOWER_DIAG || bj <= bi); bj += kBlk) {
            T *c = C + (size_t)bi * ldc + bj;
            const T *a = A + (size_t)bi * lda, *b = B + (size_t)bj * ldb;
            const int mm = min(kBlk, m - bi), nn = min(kBlk, n - bj);
            if (LOWER_DIAG && bi == bj) block_nt_update<T, true, 4>(c, ldc, a, lda, b, ldb, mm, nn, k, sm);
            else block_nt_update<T, false, 4>(c, ldc, a, lda, b, ldb, mm, nn, k, sm);
        }
}

// A_IK <- A_IK - A_IJ A_KJ^T
template <typename T>
__device__ void tile_gemm(T *C, const T *A, const T *B, int nb, SimtSmem<T> &sm) {
    region_nt_update<T, false>(C, nb, A, nb, B, nb, nb, nb, nb, sm);
}

// A_II <- A_II - A_IJ A_IJ^T on the lower triangle
template <typename T>
__device__ void tile_syrk(T *C, const T *A, int nb, SimtSmem<T> &sm) {
    region_nt_update<T, true>(C, nb, A, nb, A, nb, nb, nb, nb, sm);
}

// Stage the w x w diagonal block of L starting at (jb, jb) into sm.D (lower;
// identity beyond w) and the reciprocals of its diagonal into sm.Dinv.
template <typename T>
__device__ void stage_diag(const T *L, int ld, int jb, int w, SimtSmem<T> &sm) {
    for (int e = threadIdx.x; e < kIB * kIB; e += kThreads) {
        const int r = e / kIB, c = e % kIB;
        T v = T(0);
        if (r < w && c < w) {
            if (c <= r) v = ldg_cg(L + (size_t)(jb + r) * ld + jb + c);
        } else if (r == c) {
            v = T(1);
        }
        sm.D[r][c] = v;
    }
    simt_sync();
    if (threadIdx.x < kIB) sm.Dinv[threadIdx.x] = T(1) / sm.D[threadIdx.x][threadIdx.x];
    simt_sync();
}

// Rows [r0, r1) of P (columns jb .. jb+w) <- P * D^{-T}: each thread runs the
// forward substitution of whole rows with the block held in registers.
template <typename T>
__device__ void rows_trsm(T *P, int ld, int jb, int w, int r0, int r1, SimtSmem<T> &sm) {
    for (int r = r0 + threadIdx.x; r < r1; r += kThreads) {
        T *row = P + (size_t)r * ld + jb;
        T x[kIB];
#pragma unroll
        for (int j = 0; j < kIB; ++j) x[j] = j < w ? ldg_cg(row + j) : T(0);
#pragma unroll
        for (int j = 0; j < kIB; ++j) {
            T s = x[j];
#pragma unroll
            for (int q = 0; q < j; ++q) s = fma(-x[q], sm.D[j][q], s);
            x[j] = s * sm.Dinv[j];
        }
#pragma unroll
        for (int j = 0; j < kIB; ++j)
            if (j < w) row[j] = x[j];
    }
    simt_sync();
}

// A_IJ <- A_IJ L^{-T}: blocked right-looking over panels of kIB columns.
template <typename T>
__device__ void tile_trsm(T *B, const T *L, int nb, SimtSmem<T> &sm) {
    for (int jb = 0; jb < nb; jb += kIB) {
        const int w = min(kIB, nb - jb);
        stage_diag(L, nb, jb, w, sm);
        rows_trsm(B, nb, jb, w, 0, nb, sm);
        const int c0 = jb + w;
        if (c0 < nb)
            region_nt_update<T, false>(B + c0, nb, B + jb, nb, L + (size_t)c0 * nb + jb, nb, nb, nb - c0, w, sm);
    }
}

// In-place Cholesky of the lower triangle of a diagonal tile: blocked
// right-looking with panels of kIB columns; each diagonal block is factored
// by the Crout formulas by warp 0 in shared memory.  Returns 0 or the 1-based
// tile-local column whose pivot is not positive (or NaN); on failure the
// tile is left partially factored.
template <typename T>
__device__ int tile_potrf(T *A, int nb, SimtSmem<T> &sm) {
    for (int jb = 0; jb < nb; jb += kIB) {
        const int w = min(kIB, nb - jb);
        // load the diagonal block (lower part; identity padding)
        for (int e = threadIdx.x; e < kIB * kIB; e += kThreads) {
            const int r = e / kIB, c = e % kIB;
            T v = T(0);
            if (r < w && c < w) {
                if (c <= r) v = ldg_cg(A + (size_t)(jb + r) * nb + jb + c);
            } else if (r == c) {
                v = T(1);
            }
            sm.D[r][c] = v;
        }
        if (threadIdx.x == 0) sm.flag = 0;
        simt_sync();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int fail = 0;
            for (int j = 0; j < kIB; ++j) {
                if (lane == j) {
                    T d = sm.D[j][j];
                    for (int q = 0; q < j; ++q) d = fma(-sm.D[j][q], sm.D[j][q], d);
                    if (!(d > T(0))) fail = j + 1;
                    else sm.D[j][j] = t_sqrt(d);
                }
                fail = __shfl_sync(0xffffffffu, fail, j);
                __syncwarp();
                if (fail) break;
                if (lane > j) {
                    T s = sm.D[lane][j];
                    for (int q = 0; q < j; ++q) s = fma(-sm.D[lane][q], sm.D[j][q], s);
                    sm.D[lane][j] = s / sm.D[j][j];
                }
                __syncwarp();
            }
            if (lane == 0) sm.flag = fail;
        }
        simt_sync();
        if (sm.flag) {
            const int f = sm.flag;
            simt_sync();
            return jb + f;
        }
        // write back the factored block, reciprocals of its diagonal
        for (int e = threadIdx.x; e < w * w; e += kThreads) {
            const int r = e / w, c = e % w;
            if (c <= r) A[(size_t)(jb + r) * nb + jb + c] = sm.D[r][c];
        }
        if (threadIdx.x < kIB) sm.Dinv[threadIdx.x] = T(1) / sm.D[threadIdx.x][threadIdx.x];
        simt_sync();
        const int r0 = jb + w;
        if (r0 < nb) {
            rows_trsm(A, nb, jb, w, r0, nb, sm);
            const T *P = A + (size_t)r0 * nb + jb;
            region_nt_update<T, true>(A + (size_t)r0 * nb + r0, nb, P, nb, P, nb, nb - r0, nb - r0, w, sm);
        }
    }
    return 0;
}

}  // namespace chol
