// solve_impl.cuh -- triangular solves with the Cholesky factor:
// forward substitution L Y = B, then backward substitution L^T X = Y.
//
// Each sweep is one persistent "wavefront" launch over row blocks of 64.  A
// CTA takes a ticket (atomic counter), which fixes the block it solves in
// ticket order, so it only ever waits for blocks owned by CTAs that started
// before it (no deadlock whatever the residency).  It accumulates the
// contributions of the finished blocks as their ready flags appear (acquire),
// solves its diagonal block (loaded before the waits; one warp per pair of
// right-hand sides, shuffles instead of block barriers), stores the result
// and releases its own flag.
// Every wait is bounded by a %globaltimer deadline after which the kernel
// records CHOL_ERR_TIMEOUT and returns.  grid.y splits the right-hand sides
// into slices of kRC columns, each with its own tickets and flags.
#pragma once

#include "common.cuh"

namespace chol {

constexpr int kSB = 64;  // row block of the solve
constexpr int kRC = 16;  // right-hand-side columns per CTA

// Factor accessors: element (i, j), i >= j, of L.
template <typename T>
struct ColMajorL {
    const T *p;
    int64_t ld;
    static constexpr bool kRowsFastest = true;  // consecutive i are contiguous
    __device__ __forceinline__ T operator()(int64_t i, int64_t j) const { return __ldcg(p + j * ld + i); }
};

template <typename T>
struct TileMajorL {
    const T *p;   // tile store, row-major tiles of order nb
    int64_t nb;
    static constexpr bool kRowsFastest = false;  // consecutive j are contiguous
    __device__ __forceinline__ T operator()(int64_t i, int64_t j) const {
        const int64_t I = i / nb, K = j / nb;
        return __ldcg(p + (size_t)tile_index(I, K) * nb * nb + (i - I * nb) * nb + (j - K * nb));
    }
};

struct SolveCtl {
    int32_t status;
    int32_t where;
    unsigned int tickets[2 * 4096];  // per rhs slice: forward, backward (grid.y <= 4096)
};

template <typename T>
struct SolveSmem {
    T Ls[kSB][kSB + 1];   // off-diagonal block being applied
    T Ld[kSB][kSB + 1];   // this CTA's diagonal block, loaded before the wait loop
    T rinv[kSB];          // reciprocals of its diagonal
    T Xs[kSB][kRC + 1];
    int I;
};

// Load the diagonal block (rows and columns [r0, r0+64)) into Ld and the
// reciprocals of its diagonal into rinv; ends with a barrier.
template <typename T, class Acc>
__device__ void load_diag(const Acc &L, int64_t n, int64_t r0, SolveSmem<T> &sm) {
    for (int e = threadIdx.x; e < kSB * kSB; e += blockDim.x) {
        int r, c;
        if (Acc::kRowsFastest) { r = e % kSB; c = e / kSB; }
        else { r = e / kSB; c = e % kSB; }
        const int64_t i = r0 + r, j = r0 + c;
        T v = T(0);
        if (i < n && j < n) {
            if (j <= i) v = L(i, j);
        } else if (i == j) {
            v = T(1);
        }
        sm.Ld[r][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < kSB) sm.rinv[threadIdx.x] = T(1) / sm.Ld[threadIdx.x][threadIdx.x];
    __syncthreads();
}

// Solve with the diagonal block in place on sm.Xs (64 rows x 16 columns):
// L_II y = x (forward) or L_II^T y = x (backward).  Warp w owns columns 2w
// and 2w+1; lane l owns rows l and l+32 and receives each solved entry by a
// shuffle, so the 64 steps need no block barrier.  Ends with a barrier.
template <typename T, bool FWD>
__device__ void diag_solve(SolveSmem<T> &sm) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int c0 = 2 * warp, c1 = 2 * warp + 1;
    T a0 = sm.Xs[lane][c0], a1 = sm.Xs[lane][c1], b0 = sm.Xs[lane + 32][c0], b1 = sm.Xs[lane + 32][c1];
#pragma unroll 4
    for (int s = 0; s < kSB; ++s) {
        const int k = FWD ? s : kSB - 1 - s;
        const int owner = k & 31;
        const bool hi = k >= 32;
        if (lane == owner) {
            if (hi) { b0 *= sm.rinv[k]; b1 *= sm.rinv[k]; }
            else { a0 *= sm.rinv[k]; a1 *= sm.rinv[k]; }
        }
        const T x0 = __shfl_sync(0xffffffffu, hi ? b0 : a0, owner);
        const T x1 = __shfl_sync(0xffffffffu, hi ? b1 : a1, owner);
        // FWD: rows i > k get -L(i, k) x_k; backward: rows i < k get -L(k, i) x_k
        const int i0 = lane, i1 = lane + 32;
        if (FWD ? i0 > k : i0 < k) {
            const T l = FWD ? sm.Ld[i0][k] : sm.Ld[k][i0];
            a0 = fma(-l, x0, a0);
            a1 = fma(-l, x1, a1);
        }
        if (FWD ? i1 > k : i1 < k) {
            const T l = FWD ? sm.Ld[i1][k] : sm.Ld[k][i1];
            b0 = fma(-l, x0, b0);
            b1 = fma(-l, x1, b1);
        }
    }
    sm.Xs[lane][c0] = a0;
    sm.Xs[lane][c1] = a1;
    sm.Xs[lane + 32][c0] = b0;
    sm.Xs[lane + 32][c1] = b1;
    __syncthreads();
}

// Load the 64 x 64 block of L with rows [r0, r0+64) and columns [c0, c0+64)
// (rows / columns beyond n read as the identity) into Ls[r][c] (transpose=false)
// or Ls[c][r] (transpose=true).
template <typename T, class Acc>
__device__ void load_Lblock(const Acc &L, int64_t n, int64_t r0, int64_t c0, SolveSmem<T> &sm, bool transpose) {
    for (int e = threadIdx.x; e < kSB * kSB; e += blockDim.x) {
        int r, c;
        if (Acc::kRowsFastest) { r = e % kSB; c = e / kSB; }
        else { r = e / kSB; c = e % kSB; }
        const int64_t i = r0 + r, j = c0 + c;
        T v = T(0);
        if (i < n && j < n) {
            if (j <= i) v = L(i, j);
        } else if (i == j) {
            v = T(1);
        }
        if (transpose) sm.Ls[c][r] = v;
        else sm.Ls[r][c] = v;
    }
}

__device__ __forceinline__ bool wait_flag(const int32_t *flag, uint64_t deadline, SolveCtl *ctl, int where) {
    while (!ld_acquire_s32(flag)) {
        if (ld_relaxed_s32(&ctl->status)) return false;
        if (global_ns() > deadline) {
            if (atomicCAS(&ctl->status, 0, (int32_t)CHOL_ERR_TIMEOUT) == 0) ctl->where = where;
            return false;
        }
        nanosleep_ns(128);
    }
    return true;
}

// Forward sweep: Y = L^{-1} B in place (B column-major, ldb).
template <typename T, class Acc>
__global__ void __launch_bounds__(256) solve_fwd_kernel(Acc L, T *B, int64_t ldb, int64_t n, int64_t nrhs,
                                                        int32_t *flags, SolveCtl *ctl, uint64_t timeout_ns) {
    __shared__ SolveSmem<T> sm;
    const int nblk = (int)((n + kSB - 1) / kSB);
    const int y = blockIdx.y;
    if (threadIdx.x == 0) sm.I = (int)atomicAdd(&ctl->tickets[2 * y], 1u);
    __syncthreads();
    const int I = sm.I;
    if (I >= nblk) return;
    const int64_t c0 = (int64_t)y * kRC;
    const int c = threadIdx.x % kRC, rq = threadIdx.x / kRC;  // rows rq + 16 q
    int32_t *fl = flags + (size_t)y * nblk;
    const uint64_t deadline = global_ns() + timeout_ns;
    load_diag<T>(L, n, (int64_t)I * kSB, sm);
    T acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = (int64_t)I * kSB + rq + 16 * q;
        acc[q] = (i < n && c0 + c < nrhs) ? B[(c0 + c) * ldb + i] : T(0);
    }
    for (int J = 0; J < I; ++J) {
        if (threadIdx.x == 0) {
            if (!wait_flag(fl + J, deadline, ctl, 10)) sm.I = -1;
            else fence_acq_rel();
        }
        __syncthreads();
        if (sm.I < 0) return;
        load_Lblock<T>(L, n, (int64_t)I * kSB, (int64_t)J * kSB, sm, false);
        for (int e = threadIdx.x; e < kSB * kRC; e += blockDim.x) {
            const int k = e / kRC, cc = e % kRC;
            const int64_t i = (int64_t)J * kSB + k;
            sm.Xs[k][cc] = (i < n && c0 + cc < nrhs) ? __ldcg(B + (c0 + cc) * ldb + i) : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kSB; ++k) {
            const T yk = sm.Xs[k][c];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(-sm.Ls[rq + 16 * q][k], yk, acc[q]);
        }
        __syncthreads();
    }
    // diagonal block: L_II y = acc
#pragma unroll
    for (int q = 0; q < 4; ++q) sm.Xs[rq + 16 * q][c] = acc[q];
    __syncthreads();
    diag_solve<T, true>(sm);
    for (int e = threadIdx.x; e < kSB * kRC; e += blockDim.x) {
        const int k = e / kRC, cc = e % kRC;
        const int64_t i = (int64_t)I * kSB + k;
        if (i < n && c0 + cc < nrhs) B[(c0 + cc) * ldb + i] = sm.Xs[k][cc];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_acq_rel();
        st_release_s32(fl + I, 1);
    }
}

// Backward sweep: X = L^{-T} Y in place; tickets run the blocks from the last.
template <typename T, class Acc>
__global__ void __launch_bounds__(256) solve_bwd_kernel(Acc L, T *B, int64_t ldb, int64_t n, int64_t nrhs,
                                                        int32_t *flags, SolveCtl *ctl, uint64_t timeout_ns) {
    __shared__ SolveSmem<T> sm;
    const int nblk = (int)((n + kSB - 1) / kSB);
    const int y = blockIdx.y;
    if (threadIdx.x == 0) sm.I = (int)atomicAdd(&ctl->tickets[2 * y + 1], 1u);
    __syncthreads();
    const int t = sm.I;
    if (t >= nblk) return;
    const int I = nblk - 1 - t;
    const int64_t c0 = (int64_t)y * kRC;
    const int c = threadIdx.x % kRC, rq = threadIdx.x / kRC;
    int32_t *fl = flags + (size_t)y * nblk;
    const uint64_t deadline = global_ns() + timeout_ns;
    load_diag<T>(L, n, (int64_t)I * kSB, sm);
    T acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = (int64_t)I * kSB + rq + 16 * q;
        acc[q] = (i < n && c0 + c < nrhs) ? B[(c0 + c) * ldb + i] : T(0);
    }
    for (int J = nblk - 1; J > I; --J) {
        if (threadIdx.x == 0) {
            if (!wait_flag(fl + J, deadline, ctl, 20)) sm.I = -1;
            else fence_acq_rel();
        }
        __syncthreads();
        if (sm.I < 0) return;
        // Ls[r][k] = L(J*64 + k, I*64 + r): the transpose of block (J, I)
        load_Lblock<T>(L, n, (int64_t)J * kSB, (int64_t)I * kSB, sm, true);
        for (int e = threadIdx.x; e < kSB * kRC; e += blockDim.x) {
            const int k = e / kRC, cc = e % kRC;
            const int64_t i = (int64_t)J * kSB + k;
            sm.Xs[k][cc] = (i < n && c0 + cc < nrhs) ? __ldcg(B + (c0 + cc) * ldb + i) : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kSB; ++k) {
            const T xk = sm.Xs[k][c];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(-sm.Ls[rq + 16 * q][k], xk, acc[q]);
        }
        __syncthreads();
    }
    // diagonal block: L_II^T x = acc  (Ld[r][c] = L_II(r, c), lower)
#pragma unroll
    for (int q = 0; q < 4; ++q) sm.Xs[rq + 16 * q][c] = acc[q];
    __syncthreads();
    diag_solve<T, false>(sm);
    for (int e = threadIdx.x; e < kSB * kRC; e += blockDim.x) {
        const int k = e / kRC, cc = e % kRC;
        const int64_t i = (int64_t)I * kSB + k;
        if (i < n && c0 + cc < nrhs) B[(c0 + cc) * ldb + i] = sm.Xs[k][cc];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_acq_rel();
        st_release_s32(fl + I, 1);
    }
}

// Workspace bytes for a solve of order n with nrhs right-hand sides.
inline size_t solve_ws_bytes(int64_t n, int64_t nrhs) {
    const int64_t nblk = (n + kSB - 1) / kSB, ny = (nrhs + kRC - 1) / kRC;
    return sizeof(SolveCtl) + (size_t)2 * nblk * ny * sizeof(int32_t);
}

// Forward + backward sweep on stream st using the caller-provided workspace
// (solve_ws_bytes).  Does not synchronize; the status is left in ws.
template <typename T, class Acc>
int launch_solve(const Acc &L, T *B, int64_t ldb, int64_t n, int64_t nrhs, void *ws, double timeout_s,
                 cudaStream_t st) {
    const int64_t nblk = (n + kSB - 1) / kSB, ny = (nrhs + kRC - 1) / kRC;
    if (ny > 4096) {
        set_error("argument: nrhs > %d", 4096 * kRC);
        return CHOL_ERR_ARG;
    }
    SolveCtl *ctl = (SolveCtl *)ws;
    int32_t *flags = (int32_t *)((char *)ws + sizeof(SolveCtl));
    CHOL_CUDA(cudaMemsetAsync(ws, 0, solve_ws_bytes(n, nrhs), st));
    const uint64_t tns = (uint64_t)(timeout_s * 1e9);
    const dim3 grid((unsigned)nblk, (unsigned)ny);
    solve_fwd_kernel<T, Acc><<<grid, 256, 0, st>>>(L, B, ldb, n, nrhs, flags, ctl, tns);
    solve_bwd_kernel<T, Acc><<<grid, 256, 0, st>>>(L, B, ldb, n, nrhs, flags + nblk * ny, ctl, tns);
    CHOL_CUDA(cudaGetLastError());
    return CHOL_OK;
}

}  // namespace chol
