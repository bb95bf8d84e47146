// potrf128.cuh -- binary64 Cholesky of one 128 x 128 diagonal tile held in
// shared memory (the POTRF of Section 3.1 for the tensor-core engines, whose
// CTAs have the shared memory of a whole SM).
#pragma once

#include "common.cuh"

namespace chol {

constexpr int kPotrfNb = 128;
// padded 128 x 129 binary64 tile + (i, k) table of the lower triangle + the
// reciprocals of the factor's diagonal
constexpr size_t kPotrf128TabOff = (size_t)kPotrfNb * (kPotrfNb + 1) * 8;
constexpr size_t kPotrf128RcpOff = kPotrf128TabOff + (size_t)kPotrfNb * (kPotrfNb + 1);
constexpr size_t kPotrf128SmemBytes = kPotrf128RcpOff + (size_t)kPotrfNb * 8;
constexpr int kPotrfPanelThreads = 128;  // warps 0..3, one per SM sub-partition

// the panel threads' named barrier (id 4; no other code of a task uses it)
__device__ __forceinline__ void potrf_panel_sync() { asm volatile("bar.sync 4, 128;" ::: "memory"); }

// Cholesky, in the compute type C (binary64 by default; binary32 for the
// binary32 batches), of a 128 x 128 diagonal tile (row-major, lower part read
// and written; T = double, or float widened on load and rounded on store) in
// shared memory, right-looking: columns are factored four at a
// time and each block of four is applied to the trailing lower triangle as
// one rank-4 update.  With lookahead: while warps 4.. apply panel p to the
// columns right of panel p + 1, warps 0..3 (one per SM sub-partition, so the
// panel has the binary64 pipes of all four) apply it to panel p + 1's four
// columns and factor them (a named barrier between columns), so the panels'
// sequential work overlaps the trailing updates.  Every element sees the same operations
// in the same order as the Crout formulas (fused multiply-subtracts in
// ascending column order), the division by the pivot being a multiplication
// by its reciprocal.  The trailing elements are visited through a table of
// (i, k) in column-major lower order, so the active ones form a contiguous
// suffix and all threads stay busy.  All threads (at least 256); A has row
// pitch ld; smem holds kPotrf128SmemBytes (the padded tile and the
// reciprocals of its diagonal, at kPotrf128RcpOff, stay there for the
// caller); returns 0 or the 1-based local column whose pivot is not positive
// (or NaN).  Ends with a barrier.
template <typename T, typename C = double>
__device__ int smem_potrf128(T *A, uint8_t *smem, int ld = kPotrfNb) {
    constexpr int N = kPotrfNb;
    constexpr int P = N + 1;  // padded row
    C *S = reinterpret_cast<C *>(smem);
    uint16_t *tab = reinterpret_cast<uint16_t *>(smem + kPotrf128TabOff);
    C *rcp = reinterpret_cast<C *>(smem + kPotrf128RcpOff);
    const int t = threadIdx.x, nt = blockDim.x;
    constexpr int kTri = N * (N + 1) / 2;
    // eight loads in flight per thread before their shared-memory stores
    constexpr int U = 8;
    for (int e0 = t; e0 < N * N; e0 += nt * U) {
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * nt, i = e / N, k = e % N;
            v[u] = (e < N * N && k <= i) ? __ldcg(A + (size_t)i * ld + k) : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * nt, i = e / N, k = e % N;
            if (e < N * N && k <= i) S[i * P + k] = (C)v[u];
        }
    }
    for (int k = t; k < N; k += nt) {
        const int off = k * N - k * (k - 1) / 2;
        for (int i = k; i < N; ++i) tab[off + i - k] = (uint16_t)((i << 8) | k);
    }
    __syncthreads();
    // failure of the panel factored in step it (it = j0 / 4) at s_fail[it & 1]:
    // read at the top of step it + 1 while the panel threads write the other slot
    __shared__ int s_fail[2];
    // table offset of column k's first element (k <= N)
    auto col_off = [](int k) { return k * N - k * (k - 1) / 2; };
    constexpr int PT = kPotrfPanelThreads;
    // the panel (columns j0 .. j0+3, rows j0 .. N-1) by the panel threads
    // (thread t < 128 owns row j + 1 + t of column j): every one computes the
    // pivot's root and reciprocal, a named barrier separates the columns
    auto factor_panel = [&](int j0) -> int {
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + q;
            const C djj = S[j * P + j];
            potrf_panel_sync();
            if (!(djj > C(0))) return j + 1;  // uniform: every thread read the same value
            const C d = sqrt(djj), rd = C(1) / d;
            if (t == 0) {
                S[j * P + j] = d;
                rcp[j] = rd;
            }
            for (int i = j + 1 + t; i < N; i += PT) S[i * P + j] *= rd;
            potrf_panel_sync();
            for (int c = j + 1; c < j0 + 4; ++c) {
                const C scj = S[c * P + j];
                for (int i = c + t; i < N; i += PT) S[i * P + c] = fma(-S[i * P + j], scj, S[i * P + c]);
            }
            potrf_panel_sync();
        }
        return 0;
    };
    // rank-4 update of the table entries [e0, e1) with panel j0 by threads
    // first .. first + count - 1 (the thread's index relative to first is r)
    auto rank4 = [&](int j0, int e0, int e1, int r, int count) {
        for (int e = e0 + r; e < e1; e += count) {
            const int ik = tab[e], i = ik >> 8, k = ik & 255;
            C v = S[i * P + k];
#pragma unroll
            for (int q = 0; q < 4; ++q) v = fma(-S[i * P + j0 + q], S[k * P + j0 + q], v);
            S[i * P + k] = v;
        }
    };
    if (t < PT) {
        const int f = factor_panel(0);
        if (t == 0) s_fail[0] = f;
    }
    __syncthreads();
    for (int j0 = 0; j0 < N; j0 += 4) {
        const int it = j0 / 4;
        const int fl = s_fail[it & 1];
        if (fl) {
            __syncthreads();
            return fl;
        }
        const int k0 = j0 + 4;  // the next panel
        if (k0 >= N) break;
        const int k1 = k0 + 4 < N ? k0 + 4 : N;
        if (t < PT) {
            // panel j0 applied to the next panel's columns, then that panel factored
            rank4(j0, col_off(k0), col_off(k1), t, PT);
            potrf_panel_sync();
            const int f = factor_panel(k0);
            if (t == 0) s_fail[(it + 1) & 1] = f;
        } else {
            rank4(j0, col_off(k1), kTri, t - PT, nt - PT);
        }
        __syncthreads();
    }
    for (int e = t; e < N * N; e += nt) {
        const int i = e / N, k = e % N;
        if (k <= i) A[(size_t)i * ld + k] = (T)S[i * P + k];
    }
    __syncthreads();
    return 0;
}

}  // namespace chol
