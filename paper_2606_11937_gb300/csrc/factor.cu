// factor.cu -- FP64 tiled right-looking Cholesky (Section 3.1, Fig. 1) under
// the two GPU schedules of Section 3.2:
//
//  * fork-join: for each block column J, one launch for POTRF(J), one grid
//    with a CTA per TRSM(I, J), one grid with a CTA per trailing tile
//    (collapsed: every (I, K) with J < K <= I, SYRK when I == K, else GEMM) or
//    a CTA per block row I (naive: the CTA walks K = J+1 .. I).  Stream order
//    is the barrier between the phases.
//  * dataflow: one persistent kernel.  Every task (I, K, J) owns a counter of
//    finished predecessors; a finished task increments the counters of its
//    successors and pushes those that became ready onto a global ready queue
//    that the CTAs pop.  No barrier ends a step.  Each tile receives its
//    updates in ascending J (the chain dependency), exactly as under
//    fork-join, so the two schedules produce identical bits.
#include <atomic>
#include <chrono>
#include <functional>
#include <mutex>
#include <thread>

#include "common.cuh"
#include "factor_impl.cuh"

namespace chol {

template struct TileStore<double>;

// Early output of the dataflow schedule on the tensor-core engine (fp64tc.cu).
struct EarlyOut {
    double *out;
    int64_t ld;
    int32_t *cnt;
    int32_t *flag;
};
int fp64tc_schedule(double *store, int64_t n, int64_t nb, Control *ctl, unsigned long long *queue, int32_t *deps,
                    int sched, const chol_opts &o, cudaStream_t st, int *launches, cudaEvent_t e0,
                    const EarlyOut *eo);

// The FP64 engine a call runs, a pure function of (n, nb, flags): the
// tensor-core engine (SYRK/GEMM/TRSM as exact bf16 slice products) when asked
// for, or by default above order 1024 (where it is faster: measured equal at
// n = 1024, 1.5x at 1536, 4x at 6144) for tile orders that are multiples of
// 128; otherwise the DFMA engine.
bool fp64_uses_tc(int64_t n, int64_t nb, int32_t flags) {
    if (flags & CHOL_FLAG_FP64_SIMT) return false;
    if (flags & CHOL_FLAG_FP64_TC) return true;
    return n > kFp64TcMinN && (nb == 0 || (nb % 128 == 0 && nb <= kFp64TcMaxNb));
}

// Allocation layout of one FP64 factorization.
struct FactorWs {
    void *base = nullptr;
    double *store = nullptr;
    Control *ctl = nullptr;
    unsigned long long *queue = nullptr;
    int32_t *deps = nullptr;
};

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Repack A into `store` (tile order nb; the tensor-core engine stores tiles
// of order 128 and runs tasks on tiles of order tc_nb), run the schedule,
// optionally unpack the factor into A_out, read back the control block and
// synchronize.
static int fp64_core(int64_t n, const double *A, int64_t lda, const chol_opts &o, double *store, int64_t nb,
                     int64_t tc_nb, int64_t *info, chol_stats *stats, double *A_out, int64_t lda_out,
                     const EarlyOut *eo = nullptr, const std::function<void(cudaEvent_t)> *while_running = nullptr) {
    const int64_t M = (n + nb - 1) / nb;
    const int sched = o.schedule == CHOL_SCHED_AUTO ? CHOL_SCHED_DATAFLOW : o.schedule;
    CHOL_CHECK_ARG(sched >= CHOL_SCHED_FORK_JOIN && sched <= CHOL_SCHED_TOP_LOOKING, "unknown schedule");
    cudaStream_t st = (cudaStream_t)o.stream;
    const int64_t Mt = tc_nb ? (n + tc_nb - 1) / tc_nb : M;  // tiles per dimension of the tasks
    const int64_t ntasks = num_tasks(Mt);
    const size_t ctl_bytes = align256(sizeof(Control));
    const size_t q_bytes = sched == CHOL_SCHED_DATAFLOW ? align256((size_t)2 * ntasks * 8) : 0;
    const size_t d_bytes = sched == CHOL_SCHED_DATAFLOW ? align256((size_t)ntasks * 4) : 0;
    FactorWs ws;
    CHOL_CUDA(cudaMallocAsync(&ws.base, ctl_bytes + q_bytes + d_bytes, st));
    char *p = (char *)ws.base;
    ws.store = store;
    ws.ctl = (Control *)p;
    ws.queue = (unsigned long long *)(p + ctl_bytes);
    ws.deps = (int32_t *)(p + ctl_bytes + q_bytes);

    int rc = CHOL_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Control h{};
    int launches = 0;
    do {
        if ((rc = launch_repack<double, double>(A, lda, n, ws.store, (int)nb, M, st)) != CHOL_OK) break;
        if (cudaMemsetAsync(ws.ctl, 0, sizeof(Control), st) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__); break; }
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "event", __FILE__, __LINE__); break; }
        TileStore<double> S{ws.store, (int32_t)nb, (int32_t)M};
        SchedArgs a{ws.ctl, o.trace, o.trace_capacity, o.flags, 0};
        if (tc_nb) {
            rc = fp64tc_schedule(ws.store, n, tc_nb, ws.ctl, ws.queue, ws.deps, sched, o, st, &launches, e0,
                                 sched == CHOL_SCHED_DATAFLOW ? eo : nullptr);
        } else if (sched == CHOL_SCHED_DATAFLOW) {
            rc = run_dataflow<double>(S, a, ws.queue, ws.deps, o, st, &launches, e0);
        } else {
            rc = run_fork_join<double>(S, a, fj_variant(sched), st, &launches, e0, o.timeout_s);
        }
        if (rc != CHOL_OK) break;
        cudaEventRecord(e1, st);
        // (with early output the dataflow kernel already wrote every final tile)
        if (A_out && !(eo && tc_nb && sched == CHOL_SCHED_DATAFLOW) &&
            (rc = launch_unpack<double, double>(ws.store, (int)nb, M, A_out, lda_out, n, st)) != CHOL_OK)
            break;
        // work of the caller that overlaps the schedule (e1: the schedule's
        // end); before the readback below, whose copy into pageable memory
        // blocks this thread until the stream gets there
        if (while_running) (*while_running)(e1);
        if (cudaMemcpyAsync(&h, ws.ctl, sizeof(Control), cudaMemcpyDeviceToHost, st) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "readback", __FILE__, __LINE__); break; }
        if (cudaStreamSynchronize(st) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "sync", __FILE__, __LINE__); break; }
    } while (0);
    cudaFreeAsync(ws.base, st);
    if (rc == CHOL_OK) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *info = h.info;
        if (stats) {
            for (int i = 0; i < 4; ++i) stats->tasks[i] = (int64_t)h.tasks[i];
            stats->nb = tc_nb ? tc_nb : nb;
            stats->schedule = sched;
            stats->launches = launches + (A_out ? 2 : 1);
            stats->trace_records = (int64_t)h.trace_count;
            stats->device_ms = ms;
        }
        if (h.status != 0) {
            set_error("device-side wait expired after %.3f s (site %d)", o.timeout_s, h.timeout_where);
            rc = h.status;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

// Tile order of the tasks: the caller's nb, else the default (128 on the
// tensor-core engine, chol_default_nb on the DFMA engine).
static int64_t task_nb(int64_t n, const chol_opts &o, bool tc) {
    if (o.nb > 0) return o.nb;
    return tc ? 128 : chol_default_nb(n, CHOL_FP64);
}

size_t fp64_store_bytes(int64_t n, int64_t nb) {
    const int64_t M = (n + nb - 1) / nb;
    return align256((size_t)num_tiles(M) * nb * nb * sizeof(double));
}

static int check_tc_nb(int64_t nb) {
    CHOL_CHECK_ARG(nb % 128 == 0 && nb >= 128 && nb <= kFp64TcMaxNb,
                   "the tensor-core FP64 engine takes tile orders that are multiples of 128, up to 2048");
    return CHOL_OK;
}

static int factor_fp64_device(int64_t n, double *A, int64_t lda, const chol_opts &o, int64_t *info,
                              chol_stats *stats, const EarlyOut *eo = nullptr,
                              const std::function<void(cudaEvent_t)> *while_running = nullptr) {
    const bool tc = fp64_uses_tc(n, o.nb, o.flags);
    const int64_t tnb = task_nb(n, o, tc);
    CHOL_CHECK_ARG(tnb >= 1 && tnb <= 2048, "nb must be in [1, 2048]");
    if (tc && check_tc_nb(tnb) != CHOL_OK) return CHOL_ERR_ARG;
    const int64_t nb = tc ? 128 : tnb;  // tile order of the store
    CHOL_CHECK_ARG((n + nb - 1) / nb < 65536, "too many tiles per dimension (n / nb must be < 65536)");
    cudaStream_t st = (cudaStream_t)o.stream;
    prepare_pool();
    double *store = nullptr;
    CHOL_CUDA(cudaMallocAsync((void **)&store, fp64_store_bytes(n, nb), st));
    const int rc = fp64_core(n, A, lda, o, store, nb, tc ? tnb : 0, info, stats, A, lda, eo, while_running);
    cudaFreeAsync(store, st);
    return rc;
}

// Factor into a tile store that the caller keeps (freed with cudaFreeAsync);
// used by the server for resident factors.  *nb_out is the store's tile
// order (128 on the tensor-core engine).
int fp64_factor_store(int64_t n, const double *A, int64_t lda, const chol_opts &o, double **store_out,
                      int64_t *nb_out, int64_t *info) {
    *store_out = nullptr;
    const bool tc = fp64_uses_tc(n, o.nb, o.flags);
    const int64_t tnb = task_nb(n, o, tc);
    if (tc && check_tc_nb(tnb) != CHOL_OK) return CHOL_ERR_ARG;
    const int64_t nb = tc ? 128 : tnb;
    CHOL_CHECK_ARG(nb >= 1 && nb <= 2048 && (n + nb - 1) / nb < 65536, "bad tile order");
    cudaStream_t st = (cudaStream_t)o.stream;
    prepare_pool();
    double *store = nullptr;
    CHOL_CUDA(cudaMallocAsync((void **)&store, fp64_store_bytes(n, nb), st));
    const int rc = fp64_core(n, A, lda, o, store, nb, tc ? tnb : 0, info, nullptr, nullptr, 0);
    if (rc != CHOL_OK) {
        cudaFreeAsync(store, st);
        return rc;
    }
    *store_out = store;
    *nb_out = nb;
    return CHOL_OK;
}

}  // namespace chol

using namespace chol;

static thread_local int64_t g_last_info = 0;

extern "C" {

int chol_factor_ex(int64_t n, double *A, int64_t lda, const chol_opts *opts, int64_t *info,
                   chol_stats *stats) {
    CHOL_CHECK_ARG(info != nullptr, "info is NULL");
    *info = 0;
    CHOL_CHECK_ARG(n >= 0, "n < 0");
    CHOL_CHECK_ARG(lda >= (n > 1 ? n : 1), "lda < max(1, n)");
    chol_opts o = resolve_opts(opts);
    CHOL_CHECK_ARG(o.precision == CHOL_FP64, "chol_factor_ex computes in FP64; use chol_mixed_factor");
    cudaGetLastError();  // errors left by earlier, unrelated runtime calls are not ours to report
    if (stats) memset(stats, 0, sizeof(*stats));
    if (n == 0) return CHOL_OK;
    CHOL_CHECK_ARG(A != nullptr, "A is NULL");
    return factor_fp64_device(n, A, lda, o, info, stats);
}

int chol_factor(int64_t n, int64_t nb, double *A, int64_t lda) {
    chol_opts o;
    chol_opts_init(&o);
    o.nb = nb;
    o.schedule = CHOL_SCHED_DATAFLOW;
    CHOL_CHECK_ARG(nb >= 1, "nb < 1");
    int64_t info = 0;
    const int rc = chol_factor_ex(n, A, lda, &o, &info, nullptr);
    g_last_info = info;
    if (rc == CHOL_OK && info > 0) {
        set_error("matrix is not positive definite: leading minor %lld", (long long)info);
        return CHOL_ERR_NOT_SPD;
    }
    return rc;
}

int64_t chol_last_info(void) { return g_last_info; }

int chol_factor_host(int64_t n, double *A_host, int64_t lda, const chol_opts *opts, int64_t *info,
                     chol_stats *stats) {
    CHOL_CHECK_ARG(info != nullptr, "info is NULL");
    *info = 0;
    CHOL_CHECK_ARG(n >= 0, "n < 0");
    CHOL_CHECK_ARG(lda >= (n > 1 ? n : 1), "lda < max(1, n)");
    if (n == 0) return CHOL_OK;
    CHOL_CHECK_ARG(A_host != nullptr, "A is NULL");
    chol_opts o = resolve_opts(opts);
    CHOL_CHECK_ARG(o.precision == CHOL_FP64, "chol_factor_host computes in FP64");
    cudaStream_t st = (cudaStream_t)o.stream;
    cudaGetLastError();  // errors left by earlier, unrelated runtime calls are not ours to report
    prepare_pool();
    double *dA = nullptr;
    CHOL_CUDA(cudaMallocAsync(&dA, (size_t)n * n * sizeof(double), st));
    int rc = CHOL_OK;
    // only the lower triangle travels: per block of columns from c0, rows
    // c0 .. n-1 (the few entries above the diagonal inside a block's diagonal
    // square come along; the factorization never reads them, and on the way
    // back they are the caller's own values)
    auto copy_lower = [&](double *dst, int64_t ldd, const double *src, int64_t lds, cudaMemcpyKind kind, int64_t c0,
                          int64_t c1, int64_t bw, cudaStream_t s) {
        for (int64_t j0 = c0; j0 < c1; j0 += bw) {
            const int64_t w = c1 - j0 < bw ? c1 - j0 : bw;
            const cudaError_t e = cudaMemcpy2DAsync(dst + j0 * ldd + j0, ldd * sizeof(double), src + j0 * lds + j0,
                                                    lds * sizeof(double), (size_t)(n - j0) * sizeof(double), (size_t)w,
                                                    kind, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    constexpr int64_t kCopyCols = 512;
    if (copy_lower(dA, n, A_host, lda, cudaMemcpyHostToDevice, 0, n, kCopyCols, st) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "H2D", __FILE__, __LINE__);
        cudaFreeAsync(dA, st);
        return rc;
    }
    // The dataflow schedule on the tensor-core engine writes each tile of
    // the factor to dA as soon as it is final and, once a block column is
    // complete, sets that column's flag in page-locked host memory.  This
    // thread polls the flags while the schedule runs and queues each
    // column's copy back on a copy stream, so the copies overlap the
    // factorization; whatever is not flagged when the schedule ends is copied
    // then.  Other schedules and engines copy back after the factorization.
    const int sched = o.schedule == CHOL_SCHED_AUTO ? CHOL_SCHED_DATAFLOW : o.schedule;
    const bool tc = fp64_uses_tc(n, o.nb, o.flags);
    const int64_t tnb = task_nb(n, o, tc);
    const int64_t Mt = (n + tnb - 1) / tnb;
    bool early = tc && sched == CHOL_SCHED_DATAFLOW && !(o.flags & CHOL_FLAG_NOOP) && tnb % 128 == 0 &&
                 tnb <= kFp64TcMaxNb;
    int32_t *cnt = nullptr, *hflag = nullptr, *dflag = nullptr;
    cudaStream_t cs = nullptr;
    if (early) {
        early = cudaMallocAsync(&cnt, (size_t)Mt * sizeof(int32_t), st) == cudaSuccess &&
                cudaMemsetAsync(cnt, 0, (size_t)Mt * sizeof(int32_t), st) == cudaSuccess &&
                cudaHostAlloc(&hflag, (size_t)Mt * sizeof(int32_t), cudaHostAllocMapped) == cudaSuccess &&
                cudaHostGetDevicePointer((void **)&dflag, hflag, 0) == cudaSuccess &&
                cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
        if (!early) cudaGetLastError();
    }
    if (early) {
        for (int64_t K = 0; K < Mt; ++K) reinterpret_cast<volatile int32_t *>(hflag)[K] = 0;
        EarlyOut eo{dA, n, cnt, dflag};
        cudaError_t ce = cudaSuccess;
        const std::function<void(cudaEvent_t)> overlap = [&](cudaEvent_t sched_end) {
            // the schedule was enqueued on st after the flags were cleared;
            // queue each block column's copy once its flag is set, the rest
            // once the schedule has ended (its end event is recorded on st)
            int64_t next = 0;
            while (next < Mt && ce == cudaSuccess) {
                // (any answer but "not ready", an error included, ends the polling)
                const bool ended = cudaEventQuery(sched_end) != cudaErrorNotReady;
                int64_t upto = next;
                while (upto < Mt && (ended || reinterpret_cast<volatile int32_t *>(hflag)[upto] != 0)) ++upto;
                if (upto > next) {
                    std::atomic_thread_fence(std::memory_order_acquire);
                    if (ended) ce = cudaStreamWaitEvent(cs, sched_end, 0);  // the rest: after the schedule
                    if (ce == cudaSuccess)
                        ce = copy_lower(A_host, lda, dA, n, cudaMemcpyDeviceToHost, next * tnb,
                                        upto * tnb < n ? upto * tnb : n, tnb, cs);
                    next = upto;
                } else {
                    std::this_thread::sleep_for(std::chrono::microseconds(50));
                }
            }
        };
        rc = factor_fp64_device(n, dA, n, o, info, stats, &eo, &overlap);
        if (cudaStreamSynchronize(cs) != cudaSuccess || ce != cudaSuccess) {
            if (rc == CHOL_OK) rc = cuda_fail(ce != cudaSuccess ? ce : cudaGetLastError(), "D2H", __FILE__, __LINE__);
        }
    } else {
        rc = chol_factor_ex(n, dA, n, &o, info, stats);
        if (rc == CHOL_OK && copy_lower(A_host, lda, dA, n, cudaMemcpyDeviceToHost, 0, n, kCopyCols, st) != cudaSuccess)
            rc = cuda_fail(cudaGetLastError(), "D2H", __FILE__, __LINE__);
        if (cudaStreamSynchronize(st) != cudaSuccess && rc == CHOL_OK)
            rc = cuda_fail(cudaGetLastError(), "sync", __FILE__, __LINE__);
    }
    if (cnt) cudaFreeAsync(cnt, st);
    cudaFreeAsync(dA, st);
    cudaStreamSynchronize(st);
    if (cs) cudaStreamDestroy(cs);
    if (hflag) cudaFreeHost(hflag);
    return rc;
}

}  // extern "C"
