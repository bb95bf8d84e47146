// solve_impl.cuh -- triangular solves with the Cholesky factor:
// forward substitution L Y = B, then backward substitution L^T X = Y.
//
// Each sweep is one "wavefront" launch over row blocks of 64.  A CTA takes a
// ticket (atomic counter), which fixes the block it solves in ticket order,
// so it only ever waits for blocks owned by CTAs that started before it (no
// deadlock whatever the residency).  It accumulates the contributions of the
// finished blocks in order as their ready flags appear (acquire): the next
// factor block is loaded into registers while the current one is applied, and
// one flag poll also takes note of the further blocks that are already
// finished, whose solution values are then prefetched the same way.  Before
// its waits it inverts its diagonal block (W = L_II^{-1}, one column per
// thread), so that on the sweep's critical path the diagonal step is the
// product W y (or W^T x) rather than 64 dependent substitution steps; a block
// whose kappa_inf = ||L_II|| ||W|| exceeds kSolveKappa keeps the substitution
// (one warp per pair of right-hand sides, shuffles instead of block
// barriers).  It stores the result and releases its own flag.
// Every wait is bounded by a %globaltimer deadline after which the kernel
// records CHOL_ERR_TIMEOUT and returns.  grid.y splits the right-hand sides
// into slices of RC columns (16, or 4 when there are at most 4, so a thread
// works on one row instead of four and no arithmetic goes to empty columns),
// each slice with its own tickets and flags.
#pragma once

#include "common.cuh"

namespace chol {

constexpr int kSB = 64;  // row block of the solve
constexpr int kRC = 16;  // right-hand-side columns per CTA (the binary64 residual kernel's slices too)

// columns per slice of a solve with nrhs right-hand sides
inline int solve_rc(int64_t nrhs) { return nrhs <= 4 ? 4 : kRC; }

// Factor accessors: element (i, j), i >= j, of L.
// block(r0, c0) gives the address of element (r0, c0) of a 64 x 64 block that
// lies in one contiguous piece of storage (valid when blocked() is true): element
// (r0 + r, c0 + c) is at p + r * rs + c * cs.
template <typename T>
struct BlockRef {
    const T *p;
    int64_t rs, cs;
};

template <typename T>
struct ColMajorL {
    const T *p;
    int64_t ld;
    static constexpr bool kRowsFastest = true;  // consecutive i are contiguous
    __device__ __forceinline__ T operator()(int64_t i, int64_t j) const { return __ldcg(p + j * ld + i); }
    __device__ __forceinline__ bool blocked() const { return true; }
    __device__ __forceinline__ BlockRef<T> block(int64_t r0, int64_t c0) const { return {p + c0 * ld + r0, 1, ld}; }
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
    // a 64 x 64 block at a multiple of 64 stays inside one tile when 64 divides nb
    __device__ __forceinline__ bool blocked() const { return nb % 64 == 0; }
    __device__ __forceinline__ BlockRef<T> block(int64_t r0, int64_t c0) const {
        const int64_t I = r0 / nb, K = c0 / nb;
        return {p + (size_t)tile_index(I, K) * nb * nb + (r0 - I * nb) * nb + (c0 - K * nb), nb, 1};
    }
};

struct SolveCtl {
    int32_t status;
    int32_t where;
    unsigned int tickets[2 * 4096];  // per rhs slice: forward, backward (grid.y <= 4096)
};

constexpr double kSolveKappa = 65536.0;  // largest kappa_inf of a diagonal block applied by its inverse

template <typename T, int RC = kRC>
struct SolveSmem {
    T Ls[kSB][kSB + 1];   // off-diagonal block being applied (first the diagonal block)
    T W[kSB][kSB + 1];    // inverse of the diagonal block, or the block itself (substitution)
    T rinv[kSB];          // reciprocals of the diagonal block's diagonal
    T Xs[kSB][RC + 1];
    T nrm[2][2];          // per warp of the first two: max row sums of |L_II| and |W|
    int I;
    int known;            // leading blocks of the sweep known to be finished
    int subst;            // diagonal block too ill-conditioned for its inverse
};

// Register share of one 64 x 64 block: thread t holds 16 elements, (r, c)
// with r = t % 64, c = t / 64 + 4 q when consecutive rows are contiguous in
// memory, else r = t / 64 + 4 q, c = t % 64 (coalesced either way).
constexpr int kBlkPer = kSB * kSB / 256;

template <class Acc>
__device__ __forceinline__ void blk_coord(int q, int &r, int &c) {
    if (Acc::kRowsFastest) {
        r = threadIdx.x % kSB;
        c = threadIdx.x / kSB + 4 * q;
    } else {
        r = threadIdx.x / kSB + 4 * q;
        c = threadIdx.x % kSB;
    }
}

// Issue the loads of block (r0, c0) of L into registers.  diag: the diagonal
// block (upper part zero, identity beyond n); otherwise entries beyond n are 0.
template <typename T, class Acc>
__device__ __forceinline__ void load_block_regs(const Acc &L, int64_t n, int64_t r0, int64_t c0, bool diag,
                                                T (&v)[kBlkPer]) {
    const bool fast = L.blocked();
    BlockRef<T> b{nullptr, 0, 0};
    if (fast) b = L.block(r0, c0);
#pragma unroll
    for (int q = 0; q < kBlkPer; ++q) {
        int r, c;
        blk_coord<Acc>(q, r, c);
        const int64_t i = r0 + r, j = c0 + c;
        T x = T(0);
        if (i < n && j < n) {
            if (!diag || j <= i) x = fast ? __ldcg(b.p + r * b.rs + c * b.cs) : L(i, j);
        } else if (diag && i == j) {
            x = T(1);
        }
        v[q] = x;
    }
}

// Store a register block into S[r][c] (transpose=false) or S[c][r].
template <typename T, class Acc>
__device__ __forceinline__ void store_block_regs(const T (&v)[kBlkPer], T (*S)[kSB + 1], bool transpose) {
#pragma unroll
    for (int q = 0; q < kBlkPer; ++q) {
        int r, c;
        blk_coord<Acc>(q, r, c);
        if (transpose) S[c][r] = v[q];
        else S[r][c] = v[q];
    }
}

// Solve with the diagonal block in place on sm.Xs (64 rows x 16 columns):
// L_II y = x (forward) or L_II^T y = x (backward).  Warp w owns columns 2w
// and 2w+1; lane l owns rows l and l+32 and receives each solved entry by a
// shuffle, so the 64 steps need no block barrier.  Ends with a barrier.
template <typename T, bool FWD, int RC>
__device__ void diag_solve(SolveSmem<T, RC> &sm, const T (*Ld)[kSB + 1]) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (warp >= RC / 2) {  // no columns for this warp
        __syncthreads();
        return;
    }
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
            const T l = FWD ? Ld[i0][k] : Ld[k][i0];
            a0 = fma(-l, x0, a0);
            a1 = fma(-l, x1, a1);
        }
        if (FWD ? i1 > k : i1 < k) {
            const T l = FWD ? Ld[i1][k] : Ld[k][i1];
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

// One sweep.  FWD: Y = L^{-1} B in place, blocks in increasing order, the
// block row I gets -L(I, J) y_J for J < I.  Backward: X = L^{-T} Y in place,
// blocks from the last, block I gets -L(J, I)^T x_J for J > I.  The u-th update
// of a CTA uses block J(u) = u (forward) or nblk - 1 - u (backward), which the
// sweep finishes in that same order.
template <typename T, class Acc, bool FWD, int RC>
__global__ void __launch_bounds__(256) solve_sweep_kernel(Acc L, T *B, int64_t ldb, int64_t n, int64_t nrhs,
                                                          int32_t *flags, SolveCtl *ctl, uint64_t timeout_ns) {
    static_assert(RC == 4 || RC == 16, "slices of 4 or 16 columns");
    constexpr int RS = 256 / RC;        // row stride of a thread's rows
    constexpr int RPT = kSB / RS;       // rows per thread (4 for RC = 16, 1 for RC = 4)
    __shared__ SolveSmem<T, RC> sm;
    const int nblk = (int)((n + kSB - 1) / kSB);
    const int y = blockIdx.y;
    if (threadIdx.x == 0) {
        sm.I = (int)atomicAdd(&ctl->tickets[2 * y + (FWD ? 0 : 1)], 1u);
        sm.known = 0;
    }
    __syncthreads();
    const int t = sm.I;
    if (t >= nblk) return;
    const int I = FWD ? t : nblk - 1 - t;
    const int nupd = t;
    auto Jof = [&](int u) { return FWD ? u : nblk - 1 - u; };
    const int64_t c0 = (int64_t)y * RC;
    const int c = threadIdx.x % RC, rq = threadIdx.x / RC;  // rows rq + RS q
    int32_t *fl = flags + (size_t)y * nblk;
    const uint64_t deadline = global_ns() + timeout_ns;
    const int64_t rI = (int64_t)I * kSB;
    T lr[kBlkPer];
    // the first off-diagonal block, then the diagonal block (through Ld)
    if (nupd > 0) {
        const int64_t rJ = (int64_t)Jof(0) * kSB;
        load_block_regs<T>(L, n, FWD ? rI : rJ, FWD ? rJ : rI, false, lr);
    }
    {
        T dr[kBlkPer];
        load_block_regs<T>(L, n, rI, rI, true, dr);
        store_block_regs<T, Acc>(dr, sm.Ls, false);
    }
    T acc[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int64_t i = rI + rq + RS * q;
        acc[q] = (i < n && c0 + c < nrhs) ? B[(c0 + c) * ldb + i] : T(0);
    }
    __syncthreads();
    if (threadIdx.x < kSB) sm.rinv[threadIdx.x] = T(1) / sm.Ls[threadIdx.x][threadIdx.x];
    __syncthreads();
    // W = L_II^{-1} by forward substitution on the identity, column c by thread c
    if (threadIdx.x < kSB) {
        const int cw = threadIdx.x;
        for (int i = 0; i < cw; ++i) sm.W[i][cw] = T(0);
        sm.W[cw][cw] = sm.rinv[cw];
        for (int i = cw + 1; i < kSB; ++i) {
            T t = T(0);
            for (int k = cw; k < i; ++k) t = fma(sm.Ls[i][k], sm.W[k][cw], t);
            sm.W[i][cw] = -t * sm.rinv[i];
        }
    }
    __syncthreads();
    // kappa_inf = ||L_II||_inf ||W||_inf (row sums, thread r for row r)
    if (threadIdx.x < kSB) {
        T sl = T(0), sw = T(0);
        for (int k = 0; k < kSB; ++k) {
            sl += fabs(sm.Ls[threadIdx.x][k]);
            sw += fabs(sm.W[threadIdx.x][k]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            sl = fmax(sl, __shfl_xor_sync(0xffffffffu, sl, o));
            sw = fmax(sw, __shfl_xor_sync(0xffffffffu, sw, o));
        }
        if (threadIdx.x % 32 == 0) {
            sm.nrm[threadIdx.x / 32][0] = sl;
            sm.nrm[threadIdx.x / 32][1] = sw;
        }
    }
    __syncthreads();
    {
        const double kap = (double)fmax(sm.nrm[0][0], sm.nrm[1][0]) * (double)fmax(sm.nrm[0][1], sm.nrm[1][1]);
        const bool subst = !(kap <= kSolveKappa);  // also on NaN / Inf
        if (subst) {  // keep the block itself for the substitution
            for (int e = threadIdx.x; e < kSB * kSB; e += blockDim.x) sm.W[e / kSB][e % kSB] = sm.Ls[e / kSB][e % kSB];
        }
        if (threadIdx.x == 0) sm.subst = subst;
    }
    // solution values of the next finished block, prefetched into registers
    constexpr int kXPer = kSB * RC / 256;
    T xr[kXPer];
    bool xpre = false;
    for (int u = 0; u < nupd; ++u) {
        const int J = Jof(u);
        if (threadIdx.x == 0) {
            int known = sm.known;
            if (u >= known) {
                if (!wait_flag(fl + J, deadline, ctl, FWD ? 10 : 20)) {
                    sm.I = -1;
                } else {
                    known = u + 1;
                    // note the further blocks that are already finished
                    while (known < nupd && known < u + 32 && ld_acquire_s32(fl + Jof(known))) ++known;
                }
                sm.known = known;
            }
        }
        __syncthreads();
        if (sm.I < 0) return;
        store_block_regs<T, Acc>(lr, sm.Ls, !FWD);
        const int64_t rJ = (int64_t)J * kSB;
#pragma unroll
        for (int q = 0; q < kXPer; ++q) {
            const int e = threadIdx.x + 256 * q, k = e / RC, cc = e % RC;
            if (!xpre) {
                const int64_t i = rJ + k;
                xr[q] = (i < n && c0 + cc < nrhs) ? __ldcg(B + (c0 + cc) * ldb + i) : T(0);
            }
            sm.Xs[k][cc] = xr[q];
        }
        if (u + 1 < nupd) {
            const int64_t rN = (int64_t)Jof(u + 1) * kSB;
            load_block_regs<T>(L, n, FWD ? rI : rN, FWD ? rN : rI, false, lr);
            xpre = u + 1 < sm.known;
            if (xpre) {
#pragma unroll
                for (int q = 0; q < kXPer; ++q) {
                    const int e = threadIdx.x + 256 * q, k = e / RC, cc = e % RC;
                    const int64_t i = rN + k;
                    xr[q] = (i < n && c0 + cc < nrhs) ? __ldcg(B + (c0 + cc) * ldb + i) : T(0);
                }
            }
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kSB; ++k) {
            const T xk = sm.Xs[k][c];
#pragma unroll
            for (int q = 0; q < RPT; ++q) acc[q] = fma(-sm.Ls[rq + RS * q][k], xk, acc[q]);
        }
    }
    __syncthreads();
    // diagonal block: L_II y = acc (forward) or L_II^T x = acc (backward)
#pragma unroll
    for (int q = 0; q < RPT; ++q) sm.Xs[rq + RS * q][c] = acc[q];
    __syncthreads();
    if (!sm.subst) {
        // y = W acc (forward), x = W^T acc (backward); W is zero above its diagonal
        T y[RPT];
#pragma unroll
        for (int q = 0; q < RPT; ++q) y[q] = T(0);
#pragma unroll 8
        for (int k = 0; k < kSB; ++k) {
            const T xk = sm.Xs[k][c];
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int r = rq + RS * q;
                y[q] = fma(FWD ? sm.W[r][k] : sm.W[k][r], xk, y[q]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < RPT; ++q) sm.Xs[rq + RS * q][c] = y[q];
        __syncthreads();
    } else {
        diag_solve<T, FWD, RC>(sm, sm.W);
    }
    for (int e = threadIdx.x; e < kSB * RC; e += blockDim.x) {
        const int k = e / RC, cc = e % RC;
        const int64_t i = rI + k;
        if (i < n && c0 + cc < nrhs) B[(c0 + cc) * ldb + i] = sm.Xs[k][cc];
    }
    __syncthreads();
    // the barrier orders every thread's stores before this release (cumulative)
    if (threadIdx.x == 0) st_release_s32(fl + I, 1);
}

// Workspace bytes for a solve of order n with nrhs right-hand sides.
inline size_t solve_ws_bytes(int64_t n, int64_t nrhs) {
    const int rc = solve_rc(nrhs);
    const int64_t nblk = (n + kSB - 1) / kSB, ny = (nrhs + rc - 1) / rc;
    return sizeof(SolveCtl) + (size_t)2 * nblk * ny * sizeof(int32_t);
}

// Forward + backward sweep on stream st using the caller-provided workspace
// (solve_ws_bytes).  Does not synchronize; the status is left in ws.
template <typename T, class Acc>
int launch_solve(const Acc &L, T *B, int64_t ldb, int64_t n, int64_t nrhs, void *ws, double timeout_s,
                 cudaStream_t st) {
    const int rc = solve_rc(nrhs);
    const int64_t nblk = (n + kSB - 1) / kSB, ny = (nrhs + rc - 1) / rc;
    if (ny > 4096) {
        set_error("argument: nrhs > %d", 4096 * kRC);
        return CHOL_ERR_ARG;
    }
    SolveCtl *ctl = (SolveCtl *)ws;
    int32_t *flags = (int32_t *)((char *)ws + sizeof(SolveCtl));
    CHOL_CUDA(cudaMemsetAsync(ws, 0, solve_ws_bytes(n, nrhs), st));
    const uint64_t tns = (uint64_t)(timeout_s * 1e9);
    const dim3 grid((unsigned)nblk, (unsigned)ny);
    if (rc == 4) {
        solve_sweep_kernel<T, Acc, true, 4><<<grid, 256, 0, st>>>(L, B, ldb, n, nrhs, flags, ctl, tns);
        solve_sweep_kernel<T, Acc, false, 4><<<grid, 256, 0, st>>>(L, B, ldb, n, nrhs, flags + nblk * ny, ctl, tns);
    } else {
        solve_sweep_kernel<T, Acc, true, kRC><<<grid, 256, 0, st>>>(L, B, ldb, n, nrhs, flags, ctl, tns);
        solve_sweep_kernel<T, Acc, false, kRC><<<grid, 256, 0, st>>>(L, B, ldb, n, nrhs, flags + nblk * ny, ctl, tns);
    }
    CHOL_CUDA(cudaGetLastError());
    return CHOL_OK;
}

}  // namespace chol
