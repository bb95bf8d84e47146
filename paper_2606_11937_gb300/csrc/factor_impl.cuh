// factor_impl.cuh -- the schedule machinery shared by the FP64, FP32-batched
// and mixed-precision factorizations: tile-store repack/unpack, fork-join
// kernels, and the persistent dataflow kernel with its ready queues.
//
// A "Body" policy supplies the task bodies (which engine runs POTRF, TRSM,
// SYRK and GEMM) and the geometry of the matrices it factors:
//   using Args; using Smem;
//   static __device__ int  tiles(const Args &, int m);          // M of matrix m
//   static __device__ int64_t task_base(const Args &, int m);   // offset of m's task ids
//   static __device__ void run(const Args &, const SchedArgs &, int m, int I, int K, int J, Smem &);
//   static constexpr bool kSolveTask;  // a SOLVE task follows POTRF(M-1) of every matrix
//   static constexpr int kCtasPerSm;   // default persistent CTAs per SM
//   static constexpr int kBlock;       // threads per CTA (the tile routines use the first 256)
//   static constexpr bool kLag;        // a task may complete after run() returns: then
//     static bool lagging(Smem &);     //   true while the last run's completion is deferred,
//     static bool absorbs(g, I, K, J); //   whether task (I,K,J) can start with it deferred,
//     static void flush(g, a, Smem &); //   complete it now (all threads; df_complete_lagged)
//   static __device__ void solve(const Args &, const SchedArgs &, int m, Smem &);
#pragma once

#include <type_traits>

#include "common.cuh"
#include "simt_tiles.cuh"

namespace chol {

template <typename T>
struct TileStore {
    T *base;
    int32_t nb;
    int32_t M;
    __device__ __forceinline__ T *tile(int I, int K) const {
        return base + (size_t)tile_index(I, K) * (size_t)nb * (size_t)nb;
    }
};

struct DFLocal;

struct SchedArgs {
    Control *ctl;
    chol_trace_rec *trace;
    int64_t trace_cap;
    int32_t flags;
    int32_t pad;
    DFLocal *dfl;  // dataflow kernel: this CTA's scheduler state (shared memory); else null
};

struct DFArgs {
    unsigned long long *queue;   // 2 * capacity slots: [0, cap) priority, [cap, 2 cap) normal
    int32_t *deps;               // one counter per task
    int64_t capacity;            // slots per queue (>= total tasks)
    int64_t total;               // tasks to run before the kernel ends
    uint64_t timeout_ns;
    int32_t num_matrices;
    int32_t pad;
};

// Per-CTA scheduler state of the dataflow kernel, in shared memory and used
// by thread 0 only: the claimed queue slots and a task taken ahead of time.
struct DFLocal {
    DFArgs d;
    unsigned long long tk[2];  // claimed slots (priority, normal), or kNoTicket
    uint64_t next;             // a ready task held for the next iteration, or kEmptySlot
    uint64_t lagcont;          // ready chain successor released by a deferred completion, or kEmptySlot
};

constexpr int kSolveJ = 0xFFFF;  // J marker of the fused SOLVE task (batched)

// Optional body hook, run by the dataflow kernel with all threads once a
// tile's final task (POTRF or TRSM) has completed and released its
// successors: Body::kFinalHook and Body::final_hook(g, a, m, I, K, sm).
template <class B, class = void>
struct BodyFinalHook : std::false_type {};
template <class B>
struct BodyFinalHook<B, std::void_t<decltype(B::kFinalHook)>> : std::integral_constant<bool, B::kFinalHook> {};

// ----------------------------------------------------------------- repack / unpack
// (I, K) of lower tile index t = I (I + 1) / 2 + K
__device__ __forceinline__ void tile_of(int64_t t, int &I, int &K) {
    int64_t i = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    I = (int)i;
    K = (int)(t - i * (i + 1) / 2);
}

// Column-major lower(A) -> row-major tiles; entries outside the n x n matrix
// are the identity; the strict upper triangle of diagonal tiles is set to 0
// (A's upper triangle is never read).  grid.x = tile, grid.y = (32-row strip,
// group of kRpW 32-column blocks): each thread moves 4 kRpW elements, all of
// its loads in flight before the transposes through shared memory.
constexpr int kRpW = 4;

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) repack_kernel(const Tin *A, int64_t lda, int64_t n, Tout *store,
                                                     int nb, int64_t tile0) {
    __shared__ Tout buf[kRpW][32][33];
    int I, K;
    const int64_t t = tile0 + blockIdx.x;
    tile_of(t, I, K);
    const int nsb = (nb + 31) / 32, ngr = (nsb + kRpW - 1) / kRpW;
    const int sr = blockIdx.y / ngr, sc0 = (blockIdx.y % ngr) * kRpW;
    Tout *tile = store + (size_t)t * nb * nb;
#pragma unroll
    for (int w = 0; w < kRpW; ++w) {
        const int sc = sc0 + w;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int yy = threadIdx.y + 8 * q;
            const int r = sr * 32 + threadIdx.x, c = sc * 32 + yy;
            const int64_t i = (int64_t)I * nb + r, j = (int64_t)K * nb + c;
            Tout v = Tout(0);
            if (sc < nsb && r < nb && c < nb) {
                if (i < n && j < n) v = j <= i ? (Tout)A[j * lda + i] : Tout(0);
                else v = i == j ? Tout(1) : Tout(0);
            }
            buf[w][yy][threadIdx.x] = v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < kRpW; ++w) {
        const int sc = sc0 + w;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int yy = threadIdx.y + 8 * q;
            const int r = sr * 32 + yy, c = sc * 32 + threadIdx.x;
            if (sc < nsb && r < nb && c < nb) tile[(size_t)r * nb + c] = buf[w][threadIdx.x][yy];
        }
    }
}

// Row-major tiles -> lower triangle of column-major A (i >= j, i, j < n);
// the same blocking as repack_kernel.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) unpack_kernel(const Tin *store, int nb, Tout *A, int64_t lda, int64_t n,
                                                     int64_t tile0) {
    __shared__ Tin buf[kRpW][32][33];
    int I, K;
    const int64_t t = tile0 + blockIdx.x;
    tile_of(t, I, K);
    const int nsb = (nb + 31) / 32, ngr = (nsb + kRpW - 1) / kRpW;
    const int sr = blockIdx.y / ngr, sc0 = (blockIdx.y % ngr) * kRpW;
    const Tin *tile = store + (size_t)t * nb * nb;
#pragma unroll
    for (int w = 0; w < kRpW; ++w) {
        const int sc = sc0 + w;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int yy = threadIdx.y + 8 * q;
            const int r = sr * 32 + yy, c = sc * 32 + threadIdx.x;
            buf[w][yy][threadIdx.x] = (sc < nsb && r < nb && c < nb) ? tile[(size_t)r * nb + c] : Tin(0);
        }
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < kRpW; ++w) {
        const int sc = sc0 + w;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int yy = threadIdx.y + 8 * q;
            const int r = sr * 32 + threadIdx.x, c = sc * 32 + yy;
            const int64_t i = (int64_t)I * nb + r, j = (int64_t)K * nb + c;
            if (sc < nsb && r < nb && c < nb && i < n && j < n && j <= i) A[j * lda + i] = (Tout)buf[w][threadIdx.x][yy];
        }
    }
}

template <typename Tin, typename Tout>
int launch_repack(const Tin *A, int64_t lda, int64_t n, Tout *store, int nb, int64_t M, cudaStream_t st) {
    const int nsb = (nb + 31) / 32, ngr = (nsb + kRpW - 1) / kRpW;
    const int64_t tiles = num_tiles(M);
    for (int64_t t0 = 0; t0 < tiles; t0 += 1ll << 30) {
        const int64_t cnt = tiles - t0 < (1ll << 30) ? tiles - t0 : (1ll << 30);
        repack_kernel<Tin, Tout><<<dim3((unsigned)cnt, nsb * ngr), dim3(32, 8), 0, st>>>(A, lda, n, store, nb, t0);
    }
    CHOL_CUDA(cudaGetLastError());
    return CHOL_OK;
}

template <typename Tin, typename Tout>
int launch_unpack(const Tin *store, int nb, int64_t M, Tout *A, int64_t lda, int64_t n, cudaStream_t st) {
    const int nsb = (nb + 31) / 32, ngr = (nsb + kRpW - 1) / kRpW;
    const int64_t tiles = num_tiles(M);
    for (int64_t t0 = 0; t0 < tiles; t0 += 1ll << 30) {
        const int64_t cnt = tiles - t0 < (1ll << 30) ? tiles - t0 : (1ll << 30);
        unpack_kernel<Tin, Tout><<<dim3((unsigned)cnt, nsb * ngr), dim3(32, 8), 0, st>>>(store, nb, A, lda, n, t0);
    }
    CHOL_CUDA(cudaGetLastError());
    return CHOL_OK;
}

// ----------------------------------------------------------------- task bookkeeping
__device__ __forceinline__ void task_done_bookkeeping(const SchedArgs &a, int type, int m, int I, int K, int J,
                                                      uint64_t t0) {
    // thread 0 only
    atomicAdd(&a.ctl->tasks[type & 3], 1ull);
    if (a.trace) {
        const unsigned long long slot = atomicAdd(&a.ctl->trace_count, 1ull);
        if ((int64_t)slot < a.trace_cap) {
            chol_trace_rec r;
            r.type = type;
            r.I = I;
            r.K = K;
            r.J = J;
            r.sm = (int32_t)smid();
            r.matrix = m;
            r.t_start = t0;
            r.t_end = global_ns();
            a.trace[slot] = r;
        }
    }
}

// ----------------------------------------------------------------- SIMT body (FP64 / FP32)
template <typename T>
struct SimtBody {
    struct Args {
        TileStore<T> S;
    };
    using Smem = SimtSmem<T>;
    static constexpr bool kSolveTask = false;
    static constexpr int kCtasPerSm = 4;  // DFMA latency is hidden by several task CTAs per SM
    static constexpr int kBlock = kThreads;
    static constexpr bool kLag = false;
    static constexpr size_t kSmemBytes = sizeof(SimtSmem<T>);
    static __device__ __forceinline__ void cta_init(const Args &, Smem &) {}
    static __device__ __forceinline__ void cta_fini(const Args &, Smem &) {}
    static __device__ __forceinline__ int tiles(const Args &a, int) { return a.S.M; }
    static __device__ __forceinline__ int64_t task_base(const Args &, int) { return 0; }
    static __device__ void run(const Args &g, const SchedArgs &a, int m, int I, int K, int J, Smem &sm) {
        const int type = task_type(I, K, J);
        uint64_t t0 = 0;
        if (a.trace && threadIdx.x == 0) t0 = global_ns();
        const TileStore<T> &S = g.S;
        if (!(a.flags & CHOL_FLAG_NOOP)) {
            switch (type) {
            case T_POTRF: {
                const int li = tile_potrf(S.tile(J, J), S.nb, sm);
                if (li && threadIdx.x == 0) {
                    report_info(a.ctl, (int64_t)J * S.nb + li);
                    st_release_s32(&a.ctl->abort, 1);
                }
            } break;
            case T_TRSM: tile_trsm(S.tile(I, J), S.tile(J, J), S.nb, sm); break;
            case T_SYRK: tile_syrk(S.tile(I, I), S.tile(I, J), S.nb, sm); break;
            default: tile_gemm(S.tile(I, K), S.tile(I, J), S.tile(K, J), S.nb, sm); break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) task_done_bookkeeping(a, type, m, I, K, J, t0);
    }
    static __device__ void solve(const Args &, const SchedArgs &, int, Smem &) {}
};

// ----------------------------------------------------------------- fork-join kernels
// Dynamic shared memory, aligned to 1024 bytes (the tcgen05 bodies stage
// swizzled operand tiles in it); launched with Body::kSmemBytes + 1024.
template <class Body>
__device__ __forceinline__ typename Body::Smem &body_smem() {
    extern __shared__ uint8_t dyn_smem[];
    const uintptr_t p = (reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~uintptr_t(1023);
    return *reinterpret_cast<typename Body::Smem *>(p);
}
template <class Body>
constexpr size_t body_smem_bytes() { return Body::kSmemBytes + 1024; }

// Whether the launch has been aborted, read once by thread 0 and shared with
// the CTA (all threads call it; it ends with a barrier), so the whole CTA
// returns or none of it does: a CTA whose thread 0 left early would never
// initialise the barriers and tensor memory the other threads then use.
__device__ __forceinline__ bool fj_cta_aborted(const SchedArgs &a) {
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = ld_acquire_s32(&a.ctl->abort);
    __syncthreads();
    return s_abort != 0;
}

template <class Body>
__global__ void __launch_bounds__(Body::kBlock) fj_potrf_kernel(const __grid_constant__ typename Body::Args g, SchedArgs a,
                                                       int J) {
    typename Body::Smem &sm = body_smem<Body>();
    if (fj_cta_aborted(a)) return;
    Body::cta_init(g, sm);
    Body::run(g, a, 0, J, J, J, sm);
    Body::cta_fini(g, sm);
}

template <class Body>
__global__ void __launch_bounds__(Body::kBlock) fj_trsm_kernel(const __grid_constant__ typename Body::Args g, SchedArgs a,
                                                      int J) {
    typename Body::Smem &sm = body_smem<Body>();
    if (fj_cta_aborted(a)) return;
    Body::cta_init(g, sm);
    Body::run(g, a, 0, J + 1 + (int)blockIdx.x, J, J, sm);
    Body::cta_fini(g, sm);
}

// collapsed: one CTA per trailing lower tile (I, K), J < K <= I
template <class Body>
__global__ void __launch_bounds__(Body::kBlock) fj_update_kernel(const __grid_constant__ typename Body::Args g, SchedArgs a,
                                                        int J) {
    typename Body::Smem &sm = body_smem<Body>();
    if (fj_cta_aborted(a)) return;
    int i, k;
    tile_of(blockIdx.x, i, k);
    Body::cta_init(g, sm);
    Body::run(g, a, 0, J + 1 + i, J + 1 + k, J, sm);
    Body::cta_fini(g, sm);
}

// naive: one CTA per block row I walks K = J+1 .. I (SYRK last)
template <class Body>
__global__ void __launch_bounds__(Body::kBlock) fj_update_naive_kernel(const __grid_constant__ typename Body::Args g,
                                                              SchedArgs a, int J) {
    typename Body::Smem &sm = body_smem<Body>();
    if (fj_cta_aborted(a)) return;
    const int I = J + 1 + (int)blockIdx.x;
    Body::cta_init(g, sm);
    for (int K = J + 1; K <= I; ++K) Body::run(g, a, 0, I, K, J, sm);
    Body::cta_fini(g, sm);
}

// left-looking: for block column K one CTA per tile (I, K), I >= K, applies
// all of the tile's updates J = 0 .. K-1 in ascending order (SYRK for I == K)
template <class Body>
__global__ void __launch_bounds__(Body::kBlock) fj_left_update_kernel(const __grid_constant__ typename Body::Args g,
                                                             SchedArgs a, int K) {
    typename Body::Smem &sm = body_smem<Body>();
    if (fj_cta_aborted(a)) return;
    const int I = K + (int)blockIdx.x;
    Body::cta_init(g, sm);
    for (int J = 0; J < K; ++J) Body::run(g, a, 0, I, K, J, sm);
    Body::cta_fini(g, sm);
}

// top-looking: block row I in one launch of I + 1 CTAs.  A CTA takes a ticket
// (the row's tiles K = 0 .. I in ticket order), applies the updates J < K of
// tile (I, K) as the tiles (I, J) of the same row become final (their flag
// reaches the row's epoch I + 1, acquire), then its TRSM (or, for K = I, the
// POTRF), and publishes its own flag (release).  A CTA only waits for tiles
// of earlier tickets, whose CTAs are already resident, so the waits end
// whatever the residency (the tensor-memory bodies hold a whole SM's shared
// memory, so no CTA's tensor-memory allocation waits for another CTA of the
// launch); each wait is bounded by the timeout (CHOL_ERR_TIMEOUT).
template <class Body>
__global__ void __launch_bounds__(Body::kBlock) fj_top_row_kernel(const __grid_constant__ typename Body::Args g,
                                                         SchedArgs a, int I, int32_t *fin, uint64_t timeout_ns) {
    typename Body::Smem &sm = body_smem<Body>();
    __shared__ int s_k, s_ok;
    if (threadIdx.x == 0) {
        s_k = (int)(atomicAdd(&a.ctl->ticket, 1ull) - (unsigned long long)I * (I + 1) / 2);
        s_ok = ld_acquire_s32(&a.ctl->abort) ? 0 : 1;
    }
    __syncthreads();
    const int K = s_k;
    if (!s_ok) return;  // the whole CTA, on the one value thread 0 read
    Body::cta_init(g, sm);
    const uint64_t deadline = global_ns() + timeout_ns;
    for (int J = 0; J < K; ++J) {
        if (threadIdx.x == 0) {
            while (ld_acquire_s32(fin + J) != I + 1) {
                if (ld_relaxed_s32(&a.ctl->abort)) {
                    s_ok = 0;
                    break;
                }
                if (global_ns() > deadline) {
                    if (atomicCAS(&a.ctl->status, 0, (int32_t)CHOL_ERR_TIMEOUT) == 0) a.ctl->timeout_where = 30;
                    st_release_s32(&a.ctl->abort, 1);
                    s_ok = 0;
                    break;
                }
                nanosleep_ns(256);
            }
        }
        __syncthreads();
        if (!s_ok) break;
        Body::run(g, a, 0, I, K, J, sm);  // GEMM (K < I) or SYRK (K == I)
    }
    if (s_ok) Body::run(g, a, 0, I, K, K, sm);  // TRSM (K < I) or POTRF (K == I)
    __syncthreads();
    // the barrier orders every thread's stores of the tile before the release
    // (test hook: tile (I, 0) of the last block row is never published)
    const bool withhold = (a.flags & CHOL_FLAG_TEST_WITHHOLD) && I > 0 && I == Body::tiles(g, 0) - 1 && K == 0;
    if (threadIdx.x == 0 && s_ok && !withhold) st_release_s32(fin + K, I + 1);
    Body::cta_fini(g, sm);
}

// The launch-ordered schedules: right-looking fork-join (collapsed update
// grid, or one CTA per block row), left-looking, top-looking.
enum FjVariant : int { FJ_COLLAPSED = 0, FJ_NAIVE = 1, FJ_LEFT = 2, FJ_TOP = 3 };

inline int fj_variant(int sched) {
    return sched == CHOL_SCHED_FORK_JOIN_NAIVE ? FJ_NAIVE
           : sched == CHOL_SCHED_LEFT_LOOKING  ? FJ_LEFT
           : sched == CHOL_SCHED_TOP_LOOKING   ? FJ_TOP
                                               : FJ_COLLAPSED;
}

template <class Body, typename KernelT>
int set_smem_attr(KernelT kernel) {
    CHOL_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)body_smem_bytes<Body>()));
    return CHOL_OK;
}

// Issue the launches of a launch-ordered schedule on st; returns their count.
template <class Body>
int fj_issue(const typename Body::Args &g, const SchedArgs &a, int M, int variant, cudaStream_t st, int32_t *fin,
             uint64_t timeout_ns) {
    const size_t smem = body_smem_bytes<Body>();
    int L = 0;
    if (variant == FJ_TOP) {
        for (int I = 0; I < M; ++I) fj_top_row_kernel<Body><<<I + 1, Body::kBlock, smem, st>>>(g, a, I, fin, timeout_ns);
        return M;
    }
    if (variant == FJ_LEFT) {
        // per block column K: the updates from the left, POTRF, the TRSM grid
        for (int K = 0; K < M; ++K) {
            if (K > 0) {
                fj_left_update_kernel<Body><<<M - K, Body::kBlock, smem, st>>>(g, a, K);
                ++L;
            }
            fj_potrf_kernel<Body><<<1, Body::kBlock, smem, st>>>(g, a, K);
            ++L;
            if (M - K - 1 > 0) {
                fj_trsm_kernel<Body><<<M - K - 1, Body::kBlock, smem, st>>>(g, a, K);
                ++L;
            }
        }
        return L;
    }
    for (int J = 0; J < M; ++J) {
        fj_potrf_kernel<Body><<<1, Body::kBlock, smem, st>>>(g, a, J);
        ++L;
        const int rest = M - J - 1;
        if (rest > 0) {
            fj_trsm_kernel<Body><<<rest, Body::kBlock, smem, st>>>(g, a, J);
            if (variant == FJ_NAIVE)
                fj_update_naive_kernel<Body><<<rest, Body::kBlock, smem, st>>>(g, a, J);
            else
                fj_update_kernel<Body><<<(unsigned)((int64_t)rest * (rest + 1) / 2), Body::kBlock, smem, st>>>(g, a, J);
            L += 2;
        }
    }
    return L;
}

// Launch-ordered schedule (variant: FJ_*).  e0 (may be null) is recorded on st
// right before the first kernel.  With CHOL_FLAG_GRAPH the launches are
// captured into a CUDA graph, which is instantiated and then launched as one
// unit (the host's launch latency leaves the critical path); the call then
// waits for the graph before destroying it.
template <class Body>
int run_fork_join(const typename Body::Args &g, const SchedArgs &a, int M, int variant, cudaStream_t st,
                  int *launches, cudaEvent_t e0, double timeout_s) {
    int rc;
    if ((rc = set_smem_attr<Body>(fj_potrf_kernel<Body>)) || (rc = set_smem_attr<Body>(fj_trsm_kernel<Body>)) ||
        (rc = set_smem_attr<Body>(fj_update_kernel<Body>)) || (rc = set_smem_attr<Body>(fj_update_naive_kernel<Body>)) ||
        (rc = set_smem_attr<Body>(fj_left_update_kernel<Body>)) || (rc = set_smem_attr<Body>(fj_top_row_kernel<Body>)))
        return rc;
    const uint64_t tns = (uint64_t)(timeout_s * 1e9);
    // top-looking: one "final" flag per tile of the current block row (epoch I + 1)
    int32_t *fin = nullptr;
    if (variant == FJ_TOP) {
        CHOL_CUDA(cudaMallocAsync(&fin, (size_t)M * 4, st));
        CHOL_CUDA(cudaMemsetAsync(fin, 0, (size_t)M * 4, st));
    }
    struct FinFree {
        int32_t *p;
        cudaStream_t s;
        ~FinFree() {
            if (p) cudaFreeAsync(p, s);
        }
    } fin_free{fin, st};
    if (!(a.flags & CHOL_FLAG_GRAPH)) {
        if (e0) CHOL_CUDA(cudaEventRecord(e0, st));
        *launches = fj_issue<Body>(g, a, M, variant, st, fin, tns);
        CHOL_CUDA(cudaGetLastError());
        return CHOL_OK;
    }
    // captured on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); nothing runs during the capture
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    CHOL_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t ec = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int L = 0;
    if (ec == cudaSuccess) {
        L = fj_issue<Body>(g, a, M, variant, cs, fin, tns);
        ec = cudaStreamEndCapture(cs, &graph);
    }
    cudaStreamDestroy(cs);
    if (ec != cudaSuccess) return cuda_fail(ec, "fork-join graph capture", __FILE__, __LINE__);
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess && e0) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "fork-join graph", __FILE__, __LINE__);
    *launches = L;
    return CHOL_OK;
}

// ----------------------------------------------------------------- dataflow scheduler
__device__ __forceinline__ void df_timeout(Control *ctl, int where) {
    if (atomicCAS(&ctl->status, 0, (int32_t)CHOL_ERR_TIMEOUT) == 0) ctl->timeout_where = where;
    st_release_s32(&ctl->abort, 1);
}

__device__ __forceinline__ void df_push(Control *ctl, const DFArgs &d, int q, uint64_t v) {
    const unsigned long long slot = atomicAdd(&ctl->tail[q], 1ull);
    st_release_u64(&d.queue[(size_t)q * d.capacity + slot], v);
}

// Pop one task (thread 0).  Returns 1 (task in *out), 0 (all tasks done) or
// -1 (abort, failure elsewhere, or a wait longer than the timeout).
//
// Both queues are popped by ticket: a CTA takes the next slot index of a
// queue with one fetch-and-add and keeps it (tk[q]) until a push fills that
// slot -- no compare-and-swap retry storm on a contended head.  A CTA holds
// at most one ticket per queue; it claims a priority ticket only when the
// priority queue has unclaimed entries, serves a filled priority slot first,
// and runs normal tasks while its priority ticket is still unfilled.  Slots
// are handed out in push order, so each queue stays FIFO; a ticket past the
// last push is never filled and is dropped when every task has completed.
constexpr unsigned long long kNoTicket = ~0ull;
constexpr int kLookahead = 16;  // panel columns ahead whose updates are prioritized

static __device__ int df_pop(Control *ctl, const DFArgs &d, uint64_t *out, unsigned long long *tk) {
    const uint64_t t0 = global_ns();
    const unsigned long long cap = (unsigned long long)d.capacity;
    uint32_t backoff = 32;
    for (;;) {
        // independent loads, issued together (one round trip to L2)
        const int32_t ab = ld_acquire_s32(&ctl->abort);
        const unsigned long long done = ld_relaxed_u64(&ctl->completed);
        const unsigned long long h = ld_relaxed_u64(&ctl->head[0]);
        const unsigned long long t = ld_relaxed_u64(&ctl->tail[0]);
        const uint64_t vp = tk[0] < cap ? ld_acquire_u64(&d.queue[tk[0]]) : kEmptySlot;
        const uint64_t vn = tk[1] < cap ? ld_acquire_u64(&d.queue[cap + tk[1]]) : kEmptySlot;
        if (ab) return -1;
        if (done >= (uint64_t)d.total) return 0;
        if (vp != kEmptySlot) {
            tk[0] = kNoTicket;
            *out = vp;
            return 1;
        }
        if (tk[0] == kNoTicket && h < t) {
            tk[0] = atomicAdd(&ctl->head[0], 1ull);
            continue;
        }
        if (vn != kEmptySlot) {
            tk[1] = kNoTicket;
            *out = vn;
            return 1;
        }
        if (tk[1] == kNoTicket) {
            tk[1] = atomicAdd(&ctl->head[1], 1ull);
            continue;
        }
        if (global_ns() - t0 > d.timeout_ns) {
            df_timeout(ctl, 1);
            return -1;
        }
        nanosleep_ns(backoff);
        backoff = backoff < 512 ? backoff * 2 : 512;
    }
}

// One non-blocking attempt (thread 0): take a filled claimed slot, or claim
// a slot for later.  True with the task in *out.
static __device__ bool df_try_pop(Control *ctl, DFLocal &L, uint64_t *out) {
    const unsigned long long cap = (unsigned long long)L.d.capacity;
    const unsigned long long h = ld_relaxed_u64(&ctl->head[0]);
    const unsigned long long t = ld_relaxed_u64(&ctl->tail[0]);
    const uint64_t vp = L.tk[0] < cap ? ld_acquire_u64(&L.d.queue[L.tk[0]]) : kEmptySlot;
    const uint64_t vn = L.tk[1] < cap ? ld_acquire_u64(&L.d.queue[cap + L.tk[1]]) : kEmptySlot;
    if (vp != kEmptySlot) {
        L.tk[0] = kNoTicket;
        *out = vp;
        return true;
    }
    if (L.tk[0] == kNoTicket && h < t) L.tk[0] = atomicAdd(&ctl->head[0], 1ull);
    if (vn != kEmptySlot) {
        L.tk[1] = kNoTicket;
        *out = vn;
        return true;
    }
    if (L.tk[1] == kNoTicket) L.tk[1] = atomicAdd(&ctl->head[1], 1ull);
    return false;
}

// Called by a body's thread 0 while it has nothing else to do inside a task
// (the TMA producer after its last load): take the next task ahead of time,
// so that the queue round trips overlap the task.  No-op outside the
// dataflow kernel or when a task is already held.
__device__ __forceinline__ void df_take_ahead(const SchedArgs &a) {
    if (a.dfl && a.dfl->next == kEmptySlot) {
        uint64_t v;
        if (df_try_pop(a.ctl, *a.dfl, &v)) a.dfl->next = v;
    }
}

// Priority class (with CHOL_FLAG_PRIORITY): the tasks that lead to the next
// POTRFs -- POTRF, TRSM, SYRK and the GEMMs that update one of the next
// kLookahead panel columns (K <= J + kLookahead).
__device__ __forceinline__ bool df_is_priority(int flags, int I, int K, int J) {
    return (flags & CHOL_FLAG_PRIORITY) && (task_type(I, K, J) != T_GEMM || K <= J + kLookahead);
}

// Count one finished predecessor of the tile-chain successor (I, K, J) and
// return its packed word if that made it ready (the caller runs it next, on
// the same CTA, without a trip through the queue), else kEmptySlot.
template <class Body>
__device__ __forceinline__ uint64_t df_release_chain(const typename Body::Args &g, const SchedArgs &a,
                                                     const DFArgs &d, int m, int M, int I, int K, int J) {
    if ((a.flags & CHOL_FLAG_TEST_WITHHOLD) && I == M - 1 && K == M - 1 && J == M - 1) return kEmptySlot;
    const int64_t id = Body::task_base(g, m) + task_id(I, K, J);
    const int32_t old = atom_add_acqrel_s32(&d.deps[id], 1);
    return old + 1 == task_needs(I, K, J) ? pack_task(m, I, K, J) : kEmptySlot;
}

// Completion of a task whose epilogue finished after its run() returned (one
// thread, after a barrier that orders the task's tile writes): bookkeeping,
// release of its tile-chain successor (held in lagcont for the CTA, or queued
// when a successor is already held), and the completed count.
template <class Body>
__device__ void df_complete_lagged(const typename Body::Args &g, const SchedArgs &a, int m, int I, int K, int J,
                                   uint64_t t0) {
    DFLocal &L = *a.dfl;
    task_done_bookkeeping(a, task_type(I, K, J), m, I, K, J, t0);
    if (!ld_relaxed_s32(&a.ctl->abort) && J < K) {
        const uint64_t c = df_release_chain<Body>(g, a, L.d, m, Body::tiles(g, m), I, K, J + 1);
        if (c != kEmptySlot) {
            if (L.lagcont == kEmptySlot) L.lagcont = c;
            else df_push(a.ctl, L.d, df_is_priority(a.flags, I, K, J + 1) ? 0 : 1, c);
        }
    }
    atomicAdd(&a.ctl->completed, 1ull);
}

template <class Body>
__device__ __forceinline__ void df_notify_one(const typename Body::Args &g, const SchedArgs &a, const DFArgs &d,
                                              int m, int M, int I, int K, int J) {
    if ((a.flags & CHOL_FLAG_TEST_WITHHOLD) && I == M - 1 && K == M - 1 && J == M - 1) return;
    const int32_t need = task_needs(I, K, J);
    const int64_t id = Body::task_base(g, m) + task_id(I, K, J);
    const int32_t old = atom_add_acqrel_s32(&d.deps[id], 1);
    if (old + 1 == need) df_push(a.ctl, d, df_is_priority(a.flags, I, K, J) ? 0 : 1, pack_task(m, I, K, J));
}

// Successors of task (I, K, J) of matrix m, released by the 32 lanes of warp 0.
// The successor of an update on its tile's chain is not queued when it
// becomes ready: lane 0 gets it in *cont and the CTA runs it next.
template <class Body>
__device__ void df_notify(const typename Body::Args &g, const SchedArgs &a, const DFArgs &d, int m, int I, int K,
                          int J, int lane, uint64_t *cont) {
    const int M = Body::tiles(g, m);
    if (J < K) {                       // an update: the next task of the tile's chain
        if (lane == 0) *cont = df_release_chain<Body>(g, a, d, m, M, I, K, J + 1);
    } else if (I == K) {               // POTRF(K): every TRSM(I2, K)
        for (int I2 = K + 1 + lane; I2 < M; I2 += 32) df_notify_one<Body>(g, a, d, m, M, I2, K, K);
        if (Body::kSolveTask && K == M - 1 && lane == 0) df_push(a.ctl, d, 0, pack_task(m, M, M, kSolveJ));
    } else {                           // TRSM(I, K): SYRK(I,I,K), GEMM(I,K2,K) for K<K2<I, GEMM(I2,I,K) for I2>I
        const int cnt = 1 + (I - K - 1) + (M - I - 1);
        for (int idx = lane; idx < cnt; idx += 32) {
            if (idx == 0) df_notify_one<Body>(g, a, d, m, M, I, I, K);
            else if (idx < I - K) df_notify_one<Body>(g, a, d, m, M, I, K + idx, K);
            else df_notify_one<Body>(g, a, d, m, M, I + 1 + (idx - (I - K)), I, K);
        }
    }
}

template <class Body>
__global__ void __launch_bounds__(Body::kBlock) df_kernel(const __grid_constant__ typename Body::Args g, SchedArgs a0,
                                                 DFArgs d) {
    typename Body::Smem &sm = body_smem<Body>();
    __shared__ unsigned long long s_task;
    __shared__ int s_cmd;
    __shared__ DFLocal s_local;
    Control *ctl = a0.ctl;
    SchedArgs a = a0;
    a.dfl = &s_local;
    if (threadIdx.x == 0) {
        s_local.d = d;
        s_local.tk[0] = s_local.tk[1] = kNoTicket;
        s_local.next = kEmptySlot;
        s_local.lagcont = kEmptySlot;
    }
    Body::cta_init(g, sm);
    uint64_t cont = kEmptySlot;  // thread 0: ready chain successor of the last task
    int32_t aborted = 0;         // thread 0: abort flag seen after the last task
    __shared__ int s_flush;
    for (;;) {
        if (threadIdx.x == 0) {
            uint64_t v = 0;
            int cmd = 0;
            DFLocal &L = s_local;
            bool lag = false;
            if constexpr (Body::kLag) lag = Body::lagging(sm);
            if (aborted) {
                cmd = -1;
            } else {
                // candidates: the chain successor of the last task (cont), one
                // released by a deferred completion (lagcont), a task taken ahead
                // (next).  Run a priority-class one first, else a chain successor
                // (its tile is hot in L2); hold one other, queue a third.
                uint64_t c[3] = {cont, L.lagcont, L.next};
                cont = kEmptySlot;
                L.lagcont = kEmptySlot;
                L.next = kEmptySlot;
                int pick = -1;
                for (int i = 0; i < 3 && pick < 0; ++i)
                    if (c[i] != kEmptySlot && df_is_priority(a.flags, (int)((c[i] >> 32) & 0xffff),
                                                              (int)((c[i] >> 16) & 0xffff), (int)(c[i] & 0xffff)))
                        pick = i;
                for (int i = 0; i < 3 && pick < 0; ++i)
                    if (c[i] != kEmptySlot) pick = i;
                int held = 0;
                for (int i = 0; i < 3; ++i) {
                    if (i == pick || c[i] == kEmptySlot) continue;
                    if (!held++) L.next = c[i];
                    else df_push(ctl, d, df_is_priority(a.flags, (int)((c[i] >> 32) & 0xffff),
                                                        (int)((c[i] >> 16) & 0xffff), (int)(c[i] & 0xffff)) ? 0 : 1,
                                 c[i]);
                }
                if (pick >= 0) {
                    cmd = 1;
                    v = c[pick];
                    // a normal-class successor, nothing held, priority work
                    // waiting: it goes to the normal queue
                    if (!held && (a.flags & CHOL_FLAG_PRIORITY) &&
                        !df_is_priority(a.flags, (int)((v >> 32) & 0xffff), (int)((v >> 16) & 0xffff),
                                        (int)(v & 0xffff))) {
                        const unsigned long long h = ld_relaxed_u64(&ctl->head[0]);
                        const unsigned long long t = ld_relaxed_u64(&ctl->tail[0]);
                        if (h < t) {
                            df_push(ctl, d, 1, v);
                            cmd = 0;
                        }
                    }
                }
                if (cmd == 0) {
                    if (lag) {
                        // a deferred completion may release what we would wait
                        // for: only a non-blocking attempt, else complete it first
                        cmd = df_try_pop(ctl, L, &v) ? 1 : 2;
                    } else {
                        cmd = df_pop(ctl, d, &v, L.tk);
                    }
                }
            }
            int fl = 0;
            if constexpr (Body::kLag) {
                if (lag && cmd == 1)
                    fl = !Body::absorbs(g, (int)((v >> 32) & 0xffff), (int)((v >> 16) & 0xffff), (int)(v & 0xffff));
                if (lag && cmd < 0) fl = 1;
            }
            if (cmd == 1) fence_acq_rel();
            s_task = v;
            s_cmd = cmd;
            s_flush = fl;
        }
        __syncthreads();
        const int cmd = s_cmd;
        const uint64_t v = s_task;
        const int fl = s_flush;
        __syncthreads();
        if constexpr (Body::kLag) {
            if (cmd == 2 || fl) {
                Body::flush(g, a, sm);  // all threads
                if (cmd == 2) continue;
            }
        }
        if (cmd != 1) break;
        const int J = (int)(v & 0xffff), K = (int)((v >> 16) & 0xffff), I = (int)((v >> 32) & 0xffff);
        const int m = (int)(v >> 48);
        if (J == kSolveJ) {
            Body::solve(g, a, m, sm);
        } else {
            Body::run(g, a, m, I, K, J, sm);   // ends with __syncthreads()
        }
        bool lagged = false;
        if constexpr (Body::kLag) lagged = Body::lagging(sm);
        if (threadIdx.x < 32 && !lagged) {
            // No separate fence: every way a successor is published is a
            // release at GPU scope (the acq_rel counter update, the release
            // store of a queue slot) by a warp-0 thread that passed the
            // barrier ending the task, so the CTA's tile writes are ordered
            // before it.
            __syncwarp();
            const int32_t ab = ld_relaxed_s32(&ctl->abort);
            if (J != kSolveJ && !ab) df_notify<Body>(g, a, d, m, I, K, J, threadIdx.x, &cont);
            __syncwarp();
            if (threadIdx.x == 0) {
                atomicAdd(&ctl->completed, 1ull);
                aborted = ab;
            }
        } else if (threadIdx.x == 0 && lagged) {
            aborted = ld_relaxed_s32(&ctl->abort);
        }
        if constexpr (BodyFinalHook<Body>::value) {
            if (J == K) {  // POTRF / TRSM: tile (I, K) is final
                __syncthreads();
                Body::final_hook(g, a, m, I, K, sm);
            }
        }
    }
    Body::cta_fini(g, sm);
}

// Seed the queues with POTRF(0) of every matrix.
static __global__ void df_seed_kernel(Control *ctl, DFArgs d, int flags) {
    const int q = (flags & CHOL_FLAG_PRIORITY) ? 0 : 1;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < d.num_matrices; m += gridDim.x * blockDim.x)
        d.queue[(size_t)q * d.capacity + m] = pack_task(m, 0, 0, 0);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->tail[q] = (unsigned long long)d.num_matrices;
}

// Persistent grid size.  The occupancy query runs once per body (never inside
// a stream capture: batched plans prime it before capturing) and a failed
// query leaves no error state behind.
template <class Body>
int df_grid(int num_ctas) {
    static int occ_cached = 0;
    int occ = occ_cached;
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, df_kernel<Body>, Body::kBlock, body_smem_bytes<Body>()) !=
                cudaSuccess ||
            occ < 1) {
            cudaGetLastError();
            occ = 1;
        }
        occ_cached = occ;
    }
    const int sms = num_sms();
    const int maxg = sms * occ;
    if (num_ctas <= 0) return sms * (occ < Body::kCtasPerSm ? occ : Body::kCtasPerSm);
    return num_ctas < maxg ? num_ctas : maxg;
}

// Prepare counters and queues (stream-ordered), then launch the persistent
// kernel; `e0` (if not null) is recorded between the two, so events around
// the launch time the schedule alone.
template <class Body>
int launch_dataflow(const typename Body::Args &g, const SchedArgs &a, DFArgs d, const chol_opts &o,
                    cudaStream_t st, int *launches, cudaEvent_t e0 = nullptr) {
    CHOL_CUDA(cudaMemsetAsync(d.queue, 0xFF, (size_t)2 * d.capacity * sizeof(unsigned long long), st));
    CHOL_CUDA(cudaMemsetAsync(d.deps, 0, (size_t)d.total * sizeof(int32_t), st));
    d.timeout_ns = (uint64_t)(o.timeout_s * 1e9);
    df_seed_kernel<<<(d.num_matrices + 255) / 256, 256, 0, st>>>(a.ctl, d, a.flags);
    int rc;
    if ((rc = set_smem_attr<Body>(df_kernel<Body>))) return rc;
    if (e0) CHOL_CUDA(cudaEventRecord(e0, st));
    df_kernel<Body><<<df_grid<Body>(o.num_ctas), Body::kBlock, body_smem_bytes<Body>(), st>>>(g, a, d);
    *launches = 2;
    CHOL_CUDA(cudaGetLastError());
    return CHOL_OK;
}

// single-matrix FP64 / FP32 helpers used by factor.cu
template <typename T>
int run_fork_join(const TileStore<T> &S, const SchedArgs &a, int variant, cudaStream_t st, int *launches,
                  cudaEvent_t e0, double timeout_s) {
    typename SimtBody<T>::Args g{S};
    return run_fork_join<SimtBody<T>>(g, a, S.M, variant, st, launches, e0, timeout_s);
}

template <typename T>
int run_dataflow(const TileStore<T> &S, const SchedArgs &a, unsigned long long *queue, int32_t *deps,
                 const chol_opts &o, cudaStream_t st, int *launches, cudaEvent_t e0) {
    typename SimtBody<T>::Args g{S};
    DFArgs d{};
    d.queue = queue;
    d.deps = deps;
    d.capacity = num_tasks(S.M);
    d.total = num_tasks(S.M);
    d.num_matrices = 1;
    return launch_dataflow<SimtBody<T>>(g, a, d, o, st, launches, e0);
}

}  // namespace chol
