// fp64tc_body.cuh -- the task bodies of the FP64 factorization on the tensor
// cores (binary64 accuracy by exact bf16 slicing, ozaki.cuh): arguments, the
// shared-memory POTRF and inverse of a diagonal block, and OzBodyT, whose two
// instantiations (tile order 128; tile orders 128 r, r > 1) are launched from
// fp64tc.cu and fp64tc_blocks.cu.
#pragma once

#include <cuda.h>
#include <string.h>

#include "common.cuh"
#include "factor_impl.cuh"
#include "ozaki.cuh"
#include "potrf128.cuh"

namespace chol {

struct OzArgs {
    CUtensorMap mapA;   // slice store, 128-row boxes
    CUtensorMap mapB;   // slice store, 32-row boxes (one quarter of a tile)
    CUtensorMap mapW;   // slices of the inverted diagonal tiles, 32-row boxes
    TileStore<double> S;
    __nv_bfloat16 *slices;  // per tile: 8 slices of 128 x 128
    int32_t *rexp;          // per tile: 128 row exponents
    __nv_bfloat16 *wslices; // per block column J: 8 slices of W_J = L_JJ^{-1}
    int32_t *wexp;          // per block column J: 128 row exponents of W_J
    double *wbuf;           // per block column J: L_JJ^{-T} in binary64 (row-major)
    int32_t *wflag;         // per block column J: 1 if its TRSMs use W_J (kappa_inf(L_JJ) <= kTrsmKappa)
    uint64_t timeout_ns;
    int32_t r;              // the task's tile order is 128 r (r x r subtiles of order 128)
    int32_t Ml;             // tiles of order 128 r per dimension (S.M counts the subtiles)
    // early output (dataflow schedule; null when unused): every final tile is
    // written to the column-major out (leading dimension out_ld, order n) as
    // soon as it is final; out_flag[K] becomes 1 once all tiles of block
    // column K are there (out_cnt counts them)
    double *out;
    int64_t out_ld;
    int64_t n;
    int32_t *out_cnt;
    int32_t *out_flag;
};

// Early output of the host-buffer path: destination and per-block-column
// counters and flags (factor.cu).
struct EarlyOut {
    double *out;
    int64_t ld;
    int32_t *cnt;
    int32_t *flag;
};

// The FP64 diagonal factorization in shared memory (potrf128.cuh) over the B
// and A regions of the tile-update staging area.
static_assert(kPotrf128SmemBytes <= sizeof(OzSmem::B) + sizeof(OzSmem::A),
              "the padded tile and its index table must fit in the B and A regions");
__device__ __forceinline__ int oz_potrf128(double *A, OzSmem &sm) {
    return smem_potrf128<double>(A, reinterpret_cast<uint8_t *>(sm.B));
}

// Inverse W = L^{-1} of the lower triangular factor that oz_potrf128 left in
// shared memory (lower part of the padded square S, kept intact), by forward
// substitution on the identity in blocks of four rows: the rows k0..k0+3 of
// W are finished one after the other (entry (k, c) = (R(k, c) - sum over
// m = k0..k-1 of L(k, m) W(m, c)) / L(k, k), R the updated right-hand side),
// then the rows below receive them as one rank-4 update R(i, c) -=
// sum_q L(i, k0+q) W(k0+q, c) (the next block's rows by warps 0..3, which
// then finish that block, the others by the remaining warps).  The
// reciprocals of L's diagonal come from the POTRF (its shared memory).  W(i, c), c < i, is stored transposed in the
// strict upper part of S (S(c, i)), its diagonal in a separate vector.  Writes
// W (row-major, zero above the diagonal) to Wout and returns
// kappa_inf = ||L||_inf ||W||_inf.  All threads; ends with a barrier.
__device__ inline double oz_trtri128(OzSmem &sm, double *Wout) {
    constexpr int P = kOzNb + 1;
    double *S = reinterpret_cast<double *>(sm.B);
    double *wd = sm.xp[0];           // diagonal of W
    double *red = sm.xp[1];          // row-sum maxima
    const int t = threadIdx.x, nt = blockDim.x, warp = t / 32, lane = t % 32, nw = nt / 32;
    // ||L||_inf (row sums of |L|); R = I in the strict upper part (zeros)
    double m = 0.0;
    for (int i = t; i < kOzNb; i += nt) {
        double r = 0.0;
        for (int k = 0; k <= i; ++k) r += fabs(S[i * P + k]);
        m = fmax(m, r);
    }
    for (int e = t; e < kOzNb * kOzNb; e += nt) {
        const int c = e / kOzNb, i = e % kOzNb;
        if (c < i) S[c * P + i] = 0.0;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red[warp] = m;
    __syncthreads();
    double nL = 0.0;
    for (int w = 0; w < nw; ++w) nL = fmax(nL, red[w]);
    // the reciprocals of L's diagonal, left by the shared-memory POTRF
    const double *rcp = reinterpret_cast<const double *>(reinterpret_cast<const uint8_t *>(sm.B) + kPotrf128RcpOff);
    // rows k0 .. k0+3 of W by the 128 panel threads: thread c owns column c, so
    // the rows of a block depend on each other only within a thread (the
    // diagonal entry W(c, c) included)
    auto w_block = [&](int k0) {
        const int c = t;
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + q;
            const double rk = rcp[k];
            if (c == k) {
                wd[k] = rk;
            } else if (c < k) {
                double v = S[c * P + k];
                for (int mm = k0; mm < k; ++mm) {
                    const double wmc = c < mm ? S[c * P + mm] : (c == mm ? wd[mm] : 0.0);
                    v = fma(-S[k * P + mm], wmc, v);
                }
                S[c * P + k] = v * rk;
            }
        }
    };
    // W(r, c) of a finished block row r (zero above the diagonal)
    auto wrc = [&](int r, int c) { return c < r ? S[c * P + r] : (c == r ? wd[r] : 0.0); };
    if (t < kPotrfPanelThreads) w_block(0);
    __syncthreads();
    // With lookahead: while warps 4.. apply block k0 to the rows below the next
    // block, warps 0..3 apply it to the next block's four rows and compute them.
    // R(i, c) -= sum_q L(i, k0+q) W(k0+q, c) for rows i >= k0 + 4, columns
    // c <= k0 + 3; every element receives the blocks in ascending order.
    for (int k0 = 0; k0 < kOzNb; k0 += 4) {
        const int i0 = k0 + 4;
        if (i0 >= kOzNb) break;
        const int i1 = i0 + 4 < kOzNb ? i0 + 4 : kOzNb;
        if (t < kPotrfPanelThreads) {
            for (int e = t; e < 4 * i0; e += kPotrfPanelThreads) {
                const int i = i0 + (e & 3), c = e >> 2;
                if (i < i1) {
                    double v = S[c * P + i];
#pragma unroll
                    for (int q = 0; q < 4; ++q) v = fma(-S[i * P + k0 + q], wrc(k0 + q, c), v);
                    S[c * P + i] = v;
                }
            }
            potrf_panel_sync();
            w_block(i0);
        } else {
            constexpr int pw = kPotrfPanelThreads / 32;
            for (int c = warp - pw; c < i0; c += nw - pw) {
                double wq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) wq[q] = wrc(k0 + q, c);
                for (int i = i1 + lane; i < kOzNb; i += 32) {
                    double v = S[c * P + i];
#pragma unroll
                    for (int q = 0; q < 4; ++q) v = fma(-S[i * P + k0 + q], wq[q], v);
                    S[c * P + i] = v;
                }
            }
        }
        __syncthreads();
    }
    // ||W||_inf, and W out
    m = 0.0;
    for (int i = t; i < kOzNb; i += nt) {
        double r = fabs(wd[i]);
        for (int c = 0; c < i; ++c) r += fabs(S[c * P + i]);
        m = fmax(m, r);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red[16 + warp] = m;
    for (int e = t; e < kOzNb * kOzNb; e += nt) {
        const int i = e / kOzNb, c = e % kOzNb;
        Wout[e] = c < i ? S[c * P + i] : (c == i ? wd[i] : 0.0);
    }
    __syncthreads();
    double nW = 0.0;
    for (int w = 0; w < nw; ++w) nW = fmax(nW, red[16 + w]);
    __syncthreads();
    return nL * nW;
}

// Largest infinity-norm condition number ||L_JJ|| ||L_JJ^{-1}|| for which the
// TRSMs of block column J multiply by the inverse (the error of X W^T grows
// with it); a worse-conditioned diagonal tile keeps the substitution TRSM.
constexpr double kTrsmKappa = 65536.0;

// Word of a deferred quarter that completes no task: an update inside a
// multi-update task (tile order 128 r, r > 1) whose last quarter the next
// update of the same task applies.
constexpr uint64_t kOzNoTask = ~0ull;

// Task bodies on tiles of order nb = 128 r.  The tile store, the slices and
// the inverted diagonal blocks stay on 128 x 128 blocks ("subtiles"); a task
// on a tile of order 128 r runs the operations of its subtiles in the order
// the tiled algorithm gives them at tile order 128 (every subtile receives
// its updates in ascending subtile column), so every tile order gives the
// same bits.  Subtiles past the matrix's last 128-block are skipped.
template <bool kBlocks>
struct OzBodyT {
    using Args = OzArgs;
    using Smem = OzSmem;
    static constexpr bool kSolveTask = false;
    static constexpr int kCtasPerSm = 1;
    static constexpr int kBlock = kOzThreads;
    static constexpr size_t kSmemBytes = sizeof(OzSmem);
    // In the dataflow kernel a SYRK/GEMM leaves the epilogue of its last
    // quarter to the next tile update on this CTA (which applies it while its
    // own first quarter is on the tensor cores) or to flush(); the task
    // completes (successors released) when that quarter is stored.
    static constexpr bool kLag = true;
    static __device__ __forceinline__ bool lagging(Smem &sm) { return sm.os.pend != 0; }
    static __device__ __forceinline__ bool absorbs(const Args &g, int I, int K, int J) {
        const int type = task_type(I, K, J);
        if (type == T_POTRF) return false;
        if (type == T_TRSM) return g.r == 1 && __ldcg(g.wflag + J) != 0;  // the emulated TRSM is a tile update
        return true;
    }
    static __device__ void fail_timeout(const SchedArgs &a) {
        if (atomicCAS(&a.ctl->status, 0, (int32_t)CHOL_ERR_TIMEOUT) == 0) a.ctl->timeout_where = 4;
        st_release_s32(&a.ctl->abort, 1);
    }
    static __device__ void flush(const Args &g, const SchedArgs &a, Smem &sm) {
        const bool ok = ozaki_flush(sm, g.timeout_ns, Done{g, a});
        if (!ok && threadIdx.x == 0) fail_timeout(a);
    }
    // apply a deferred quarter inside a task (all threads); false if a wait expired
    static __device__ bool flush_sub(const Args &g, const SchedArgs &a, Smem &sm) {
        return ozaki_flush(sm, g.timeout_ns, Done{g, a});
    }
    // completion of a deferred update (one epilogue thread)
    struct Done {
        const Args &g;
        const SchedArgs &a;
        __device__ void operator()(uint64_t w, uint64_t t0) const {
            if (w == kOzNoTask) return;
            df_complete_lagged<OzBodyT>(g, a, (int)(w >> 48), (int)((w >> 32) & 0xffff), (int)((w >> 16) & 0xffff),
                                       (int)(w & 0xffff), t0);
        }
    };
    static __device__ __forceinline__ void cta_init(const Args &, Smem &sm) { oz_cta_init(sm.os); }
    static __device__ __forceinline__ void cta_fini(const Args &, Smem &sm) { oz_cta_fini(sm.os); }
    static __device__ __forceinline__ int tiles(const Args &g, int) { return g.Ml; }
    static __device__ __forceinline__ int64_t task_base(const Args &, int) { return 0; }

    // POTRF of diagonal subtile j, then (unless it is the last) the inverse
    // W_j = L_jj^{-1} from the factor still in shared memory and, when it is
    // well conditioned, its slices.  False (uniform) if a pivot failed; the
    // failing column is reported.
    static __device__ bool potrf_sub(const Args &g, const SchedArgs &a, int j, Smem &sm) {
        const TileStore<double> &S = g.S;
        const int li = oz_potrf128(S.tile(j, j), sm);
        if (li) {
            if (threadIdx.x == 0) {
                report_info(a.ctl, (int64_t)j * kOzNb + li);
                st_release_s32(&a.ctl->abort, 1);
            }
            return false;
        }
        if (j < S.M - 1) {
            double *W = g.wbuf + (size_t)j * kOzNb * kOzNb;
            const double kappa = oz_trtri128(sm, W);
            const bool use_w = kappa <= kTrsmKappa;  // false also for a NaN
            if (use_w) ozaki_split(W, g.wslices + (size_t)j * kOzS * kOzNb * kOzNb, g.wexp + (size_t)j * kOzNb);
            if (threadIdx.x == 0) g.wflag[j] = use_w ? 1 : 0;
            __syncthreads();
        }
        return true;
    }
    // The producer's hook after its last load: in the dataflow kernel, take
    // the next task from the queues ahead of time (when `on`).
    struct TakeAhead {
        const SchedArgs *a;
        bool on;
        __device__ void operator()() const {
            if (on) df_take_ahead(*a);
        }
    };
    // Every tile update of the body goes through this one out-of-line copy of
    // the update (a single instance keeps the kernel's register count down).
    static __device__ __noinline__ bool tile_update(const Args &g, const SchedArgs &a, Smem &sm, const CUtensorMap *mapB,
                                                    double *C, int aRow0, int bRow0, const int32_t *expA,
                                                    const int32_t *expB, bool take, bool defer, uint64_t word,
                                                    uint64_t t0) {
        return ozaki_tile_update(sm, &g.mapA, mapB, C, aRow0, bRow0, expA, expB, g.timeout_ns, TakeAhead{&a, take},
                                 Done{g, a}, defer, word, t0);
    }
    // TRSM of subtile (i, j): substitution on the CUDA cores, or the emulated
    // product with W_j on the tensor cores; then the solution's slices.
    // False if a wait expired.
    static __device__ bool trsm_sub(const Args &g, const SchedArgs &a, int i, int j, Smem &sm, bool take) {
        const TileStore<double> &S = g.S;
        const int64_t t = tile_index(i, j);
        double *X = S.tile(i, j);
        __nv_bfloat16 *sl = g.slices + (size_t)t * kOzS * kOzNb * kOzNb;
        if (!__ldcg(g.wflag + j)) {  // substitution on the CUDA cores (threads 0..255)
            SimtSmem<double> &ss = *reinterpret_cast<SimtSmem<double> *>(sm.B);
            if (threadIdx.x < kThreads) tile_trsm(X, S.tile(j, j), kOzNb, ss);
            __syncthreads();
            ozaki_split(X, sl, g.rexp + t * kOzNb);
            return true;
        }
        // A_ij L_jj^{-T} = A_ij W_j^T on the tensor cores: the slices of -A_ij
        // go to this subtile's slice slot, the subtile is cleared, the emulated
        // update C -= (-A_ij) W_j^T leaves the solution in it, and the
        // solution's own slices replace those of -A_ij.
        ozaki_split(X, sl, g.rexp + t * kOzNb, true, false);
        for (int e = threadIdx.x; e < kOzNb * kOzNb; e += blockDim.x) X[e] = 0.0;
        __syncthreads();
        const bool ok = tile_update(g, a, sm, &g.mapW, X, (int)(t * kOzS * kOzNb), (int)((int64_t)j * kOzS * kOzNb),
                                    g.rexp + t * kOzNb, g.wexp + (size_t)j * kOzNb, take, false, 0, 0);
        if (ok) ozaki_split(X, sl, g.rexp + t * kOzNb);
        return ok;
    }
    // C(i, k) -= L(i, j) L(k, j)^T on the tensor cores; with `defer` its last
    // quarter is left to the next update (tagged with `word`).
    static __device__ bool update_sub(const Args &g, const SchedArgs &a, int i, int k, int j, Smem &sm, bool take,
                                      bool defer, uint64_t word, uint64_t t0) {
        const int64_t ta = tile_index(i, j), tb = tile_index(k, j);
        return tile_update(g, a, sm, &g.mapB, g.S.tile(i, k), (int)(ta * kOzS * kOzNb), (int)(tb * kOzS * kOzNb),
                           g.rexp + ta * kOzNb, g.rexp + tb * kOzNb, take, defer, word, t0);
    }

    // Tile order 128 (r = 1): one block per task.
    static __device__ __forceinline__ void run_order128(const Args &g, const SchedArgs &a, int m, int I, int K, int J,
                                                        Smem &sm) {
        const int type = task_type(I, K, J);
        uint64_t t0 = 0;
        if (a.trace && threadIdx.x == 0) t0 = global_ns();
        const TileStore<double> &S = g.S;
        SimtSmem<double> &ss = *reinterpret_cast<SimtSmem<double> *>(sm.B);
        // the TMA producer (thread 0) takes the next task from the queues once
        // its loads are issued, while the tensor cores and the epilogue finish
        const auto take_ahead = [&a]() { df_take_ahead(a); };
        if (!(a.flags & CHOL_FLAG_NOOP)) {
            switch (type) {
            case T_POTRF: {
                const int li = oz_potrf128(S.tile(J, J), sm);
                if (li) {
                    if (threadIdx.x == 0) {
                        report_info(a.ctl, (int64_t)J * kOzNb + li);
                        st_release_s32(&a.ctl->abort, 1);
                    }
                } else if (J < S.M - 1) {
                    // W_J = L_JJ^{-1} for the TRSMs of this block column, from
                    // the factor still in shared memory; its slices (rows of W_J)
                    // when it is well conditioned
                    double *W = g.wbuf + (size_t)J * kOzNb * kOzNb;
                    const double kappa = oz_trtri128(sm, W);
                    const bool use_w = kappa <= kTrsmKappa;  // false also for a NaN
                    if (use_w)
                        ozaki_split(W, g.wslices + (size_t)J * kOzS * kOzNb * kOzNb, g.wexp + (size_t)J * kOzNb);
                    if (threadIdx.x == 0) g.wflag[J] = use_w ? 1 : 0;
                }
            } break;
            case T_TRSM: {
                if (!__ldcg(g.wflag + J)) {  // substitution on the CUDA cores (threads 0..255)
                    if (threadIdx.x < kThreads) tile_trsm(S.tile(I, J), S.tile(J, J), kOzNb, ss);
                    __syncthreads();
                    const int64_t t = tile_index(I, J);
                    ozaki_split(S.tile(I, J), g.slices + (size_t)t * kOzS * kOzNb * kOzNb, g.rexp + t * kOzNb);
                    break;
                }
                // A_IJ L_JJ^{-T} = A_IJ W_J^T on the tensor cores: the slices of
                // -A_IJ go to this tile's slice slot, the tile is cleared, the
                // emulated update C -= (-A_IJ) W_J^T leaves the solution in it,
                // and the solution's own slices replace those of -A_IJ.
                const int64_t t = tile_index(I, J);
                double *X = S.tile(I, J);
                __nv_bfloat16 *sl = g.slices + (size_t)t * kOzS * kOzNb * kOzNb;
                ozaki_split(X, sl, g.rexp + t * kOzNb, true, false);
                for (int e = threadIdx.x; e < kOzNb * kOzNb; e += blockDim.x) X[e] = 0.0;
                __syncthreads();
                const bool ok = ozaki_tile_update(sm, &g.mapA, &g.mapW, X, (int)(t * kOzS * kOzNb),
                                                  (int)((int64_t)J * kOzS * kOzNb), g.rexp + t * kOzNb,
                                                  g.wexp + (size_t)J * kOzNb, g.timeout_ns, take_ahead, Done{g, a});
                if (ok) {
                    ozaki_split(X, sl, g.rexp + t * kOzNb);
                } else if (threadIdx.x == 0) {
                    if (atomicCAS(&a.ctl->status, 0, (int32_t)CHOL_ERR_TIMEOUT) == 0) a.ctl->timeout_where = 4;
                    st_release_s32(&a.ctl->abort, 1);
                }
            } break;
            default: {
                const int64_t ta = tile_index(I, J), tb = tile_index(K, J);
                const bool ok = ozaki_tile_update(sm, &g.mapA, &g.mapB, S.tile(I, K), (int)(ta * kOzS * kOzNb),
                                                  (int)(tb * kOzS * kOzNb), g.rexp + ta * kOzNb,
                                                  g.rexp + tb * kOzNb, g.timeout_ns, take_ahead, Done{g, a},
                                                  a.dfl != nullptr, pack_task(m, I, K, J), t0);
                if (!ok && threadIdx.x == 0) {
                    if (atomicCAS(&a.ctl->status, 0, (int32_t)CHOL_ERR_TIMEOUT) == 0) a.ctl->timeout_where = 4;
                    st_release_s32(&a.ctl->abort, 1);
                }
            } break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && !sm.os.pend) task_done_bookkeeping(a, type, m, I, K, J, t0);
    }
    // Tile order 128 r, r > 1: the blocks of the task in the order of tile
    // order 128.
    static __device__ __forceinline__ void run_blocks(const Args &g, const SchedArgs &a, int m, int I, int K, int J,
                                                      Smem &sm) {
        const int type = task_type(I, K, J);
        uint64_t t0 = 0;
        if (a.trace && threadIdx.x == 0) t0 = global_ns();
        // the TMA producer (thread 0) takes the next task from the queues once
        // its loads are issued (dataflow kernel, the task's last update), while
        // the tensor cores and the epilogue finish
        const int r = g.r, Mp = g.S.M;
        const bool df = a.dfl != nullptr;
        bool ok = true;
        if (!(a.flags & CHOL_FLAG_NOOP)) {
            switch (type) {
            case T_POTRF: {
                // right-looking over the subtiles of the diagonal tile
                for (int c = 0; c < r && ok; ++c) {
                    const int j = J * r + c;
                    if (j >= Mp) break;
                    if (!potrf_sub(g, a, j, sm)) break;  // info reported
                    for (int q = c + 1; q < r && ok; ++q)
                        if (J * r + q < Mp) ok = trsm_sub(g, a, J * r + q, j, sm, false);
                    for (int q = c + 1; q < r && ok; ++q)
                        for (int p = c + 1; p <= q && ok; ++p)
                            if (J * r + q < Mp) ok = update_sub(g, a, J * r + q, J * r + p, j, sm, false, df,
                                                                kOzNoTask, 0);
                    if (ok) ok = flush_sub(g, a, sm);
                }
            } break;
            case T_TRSM: {
                if (r == 1) {
                    ok = trsm_sub(g, a, I, J, sm, df);
                    break;
                }
                // per subtile column c of block column J: the TRSMs of the
                // block row's subtiles, then their updates of the columns right
                // of c inside the tile
                for (int c = 0; c < r && ok; ++c) {
                    const int j = J * r + c;
                    for (int q = 0; q < r && ok; ++q) {
                        if (I * r + q >= Mp) break;
                        ok = trsm_sub(g, a, I * r + q, j, sm, false);
                    }
                    for (int q = 0; q < r && ok; ++q)
                        for (int p = c + 1; p < r && ok; ++p) {
                            if (I * r + q >= Mp) break;
                            ok = update_sub(g, a, I * r + q, J * r + p, j, sm, false, df, kOzNoTask, 0);
                        }
                    if (ok) ok = flush_sub(g, a, sm);
                }
            } break;
            default: {
                // SYRK (K == I: the subtiles on or below the diagonal) or GEMM;
                // subtile column c of J outermost, so each subtile receives
                // its updates in ascending column; the task's last update
                // defers its last quarter (the task completes with it)
                int last_q = -1, last_p = -1;
                for (int q = 0; q < r; ++q)
                    for (int p = 0; p < r; ++p)
                        if (I * r + q < Mp && K * r + p < Mp && (I != K || p <= q)) last_q = q, last_p = p;
                for (int c = 0; c < r && ok; ++c)
                    for (int q = 0; q < r && ok; ++q) {
                        if (I * r + q >= Mp) break;
                        for (int p = 0; p < r && ok; ++p) {
                            if (K * r + p >= Mp || (I == K && p > q)) break;
                            const bool last = c == r - 1 && q == last_q && p == last_p;
                            ok = update_sub(g, a, I * r + q, K * r + p, J * r + c, sm, last && df, df,
                                            last ? pack_task(m, I, K, J) : kOzNoTask, last ? t0 : 0);
                        }
                    }
            } break;
            }
        }
        if (!ok && threadIdx.x == 0) fail_timeout(a);
        __syncthreads();
        if (threadIdx.x == 0 && !sm.os.pend) task_done_bookkeeping(a, type, m, I, K, J, t0);
    }
    // (two instantiations, one per path, so that the order-128 kernel keeps
    // the register allocation of its own path: a call would spill around it)
    static __device__ void run(const Args &g, const SchedArgs &a, int m, int I, int K, int J, Smem &sm) {
        if constexpr (kBlocks) run_blocks(g, a, m, I, K, J, sm);
        else run_order128(g, a, m, I, K, J, sm);
    }
    static __device__ void solve(const Args &, const SchedArgs &, int, Smem &) {}

    // Early output: tile (I, K) (order 128 r) is final; write its lower part
    // to the column-major destination (32 x 32 blocks transposed through
    // shared memory: rows read and columns written 256 bytes at a time), then
    // count it for its block column and flag the column when it is complete
    // (system-scope release: a copy engine reads the column after the flag).
    static constexpr bool kFinalHook = true;
    static __device__ __forceinline__ void final_hook(const Args &g, const SchedArgs &, int, int I, int K, Smem &sm) {
        if (!g.out) return;
        const int r = g.r, Mp = g.S.M;
        const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
        double(*buf)[33] = reinterpret_cast<double(*)[33]>(sm.B) + warp * 32;
        for (int a = 0; a < r; ++a) {
            const int i = I * r + a;
            if (i >= Mp) break;
            for (int b = 0; b < r; ++b) {
                const int k = K * r + b;
                if (k >= Mp || k > i) break;
                const double *T = g.S.tile(i, k);
                for (int blk = warp; blk < 16; blk += nw) {
                    const int br = (blk >> 2) * 32, bc = (blk & 3) * 32;
                    const int64_t row0 = (int64_t)i * kOzNb + br, col0 = (int64_t)k * kOzNb + bc;
                    if (row0 + 31 < col0 || row0 >= g.n || col0 >= g.n) continue;  // above the diagonal / padding
                    for (int rr = 0; rr < 32; ++rr) buf[rr][lane] = __ldcg(T + (size_t)(br + rr) * kOzNb + bc + lane);
                    __syncwarp();
                    const int64_t row = row0 + lane;
                    for (int cc = 0; cc < 32; ++cc) {
                        const int64_t col = col0 + cc;
                        if (row >= col && row < g.n && col < g.n) g.out[col * g.out_ld + row] = buf[lane][cc];
                    }
                    __syncwarp();
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("fence.acq_rel.sys;" ::: "memory");
            if (atomicAdd(g.out_cnt + K, 1) + 1 == g.Ml - K)
                asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(g.out_flag + K), "r"(1) : "memory");
        }
    }
};

using OzBody = OzBodyT<false>;       // tile order 128
using OzBodyBlocks = OzBodyT<true>;  // tile orders 128 r, r > 1

// Launch of the multi-block instantiation (fp64tc_blocks.cu): the dataflow
// kernel (d != null) or the launch-ordered schedule `variant` over Ml tiles.
int fp64tc_launch_blocks(const OzArgs &g, const SchedArgs &a, const DFArgs *d, int Ml, int variant,
                         const chol_opts &o, cudaStream_t st, int *launches, cudaEvent_t e0);

}  // namespace chol
