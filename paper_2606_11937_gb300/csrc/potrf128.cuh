// potrf128.cuh -- binary64 Cholesky of one 128 x 128 diagonal tile held in
// shared memory (the POTRF of Section 3.1 for the tensor-core engines, whose
// CTAs have the shared memory of a whole SM).
#pragma once

#include "common.cuh"

namespace chol {

constexpr int kPotrfNb = 128;
// padded 128 x 129 binary64 tile + (i, k) table of the lower triangle
constexpr size_t kPotrf128SmemBytes = (size_t)kPotrfNb * (kPotrfNb + 1) * 8 + (size_t)kPotrfNb * (kPotrfNb + 1);

// Cholesky, in binary64, of a 128 x 128 diagonal tile (row-major, lower part
// read and written; T = double, or float widened on load and rounded on
// store) in shared memory, right-looking: columns are factored four at a
// time (the panel by one warp, with warp barriers only) and each block of four
// is applied to the trailing lower triangle as one rank-4 update by all
// threads.  Every element sees the same operations in the same
// order as the Crout formulas (fused multiply-subtracts in ascending column
// order), the division by the pivot being a multiplication by its reciprocal.  The trailing elements are visited through a
// table of (i, k) in column-major lower order, so the active ones form a
// contiguous suffix and all threads stay busy.  All threads; smem holds
// kPotrf128SmemBytes (the padded tile stays there for the caller); returns 0
// or the 1-based local column whose pivot is not positive (or NaN).  Ends with
// a barrier.
template <typename T>
__device__ int smem_potrf128(T *A, uint8_t *smem) {
    constexpr int N = kPotrfNb;
    constexpr int P = N + 1;  // padded row
    double *S = reinterpret_cast<double *>(smem);
    uint16_t *tab = reinterpret_cast<uint16_t *>(smem + N * P * 8);
    const int t = threadIdx.x, nt = blockDim.x;
    constexpr int kTri = N * (N + 1) / 2;
    for (int e = t; e < N * N; e += nt) {
        const int i = e / N, k = e % N;
        if (k <= i) S[i * P + k] = (double)__ldcg(A + e);
    }
    for (int k = t; k < N; k += nt) {
        const int off = k * N - k * (k - 1) / 2;
        for (int i = k; i < N; ++i) tab[off + i - k] = (uint16_t)((i << 8) | k);
    }
    __syncthreads();
    __shared__ int s_fail;
    const int warp = t / 32, lane = t % 32;
    for (int j0 = 0; j0 < N; j0 += 4) {
        // the panel (columns j0 .. j0+3, rows j0 .. N-1) by warp 0 alone: lane l
        // owns rows l, l+32, ...; only warp barriers between the columns
        if (warp == 0) {
            int fail = 0;
            for (int q = 0; q < 4 && !fail; ++q) {
                const int j = j0 + q;
                const double djj = S[j * P + j];
                __syncwarp();
                if (!(djj > 0.0)) {  // uniform: every lane read the same value
                    fail = j + 1;
                    break;
                }
                const double d = sqrt(djj), rd = 1.0 / d;
                if (lane == 0) S[j * P + j] = d;
                for (int i = j + 1 + lane; i < N; i += 32) S[i * P + j] *= rd;
                __syncwarp();
                for (int c = j + 1; c < j0 + 4; ++c) {
                    const double scj = S[c * P + j];
                    for (int i = c + lane; i < N; i += 32) S[i * P + c] = fma(-S[i * P + j], scj, S[i * P + c]);
                }
                __syncwarp();
            }
            if (lane == 0) s_fail = fail;
        }
        __syncthreads();
        if (s_fail) {
            const int f = s_fail;
            __syncthreads();
            return f;
        }
        // trailing rank-4 update of the elements (i, k), j0 + 4 <= k <= i
        const int k0 = j0 + 4;
        const int off = k0 * N - k0 * (k0 - 1) / 2;
        for (int e = off + t; e < kTri; e += nt) {
            const int ik = tab[e], i = ik >> 8, k = ik & 255;
            double v = S[i * P + k];
#pragma unroll
            for (int q = 0; q < 4; ++q) v = fma(-S[i * P + j0 + q], S[k * P + j0 + q], v);
            S[i * P + k] = v;
        }
        __syncthreads();
    }
    for (int e = t; e < N * N; e += nt) {
        const int i = e / N, k = e % N;
        if (k <= i) A[e] = (T)S[i * P + k];
    }
    __syncthreads();
    return 0;
}

}  // namespace chol
