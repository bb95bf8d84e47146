// batched.cu -- factor + solve of many independent SPD systems of uneven
// order in ONE persistent dataflow launch, captured once into a CUDA graph.
//
// Every matrix keeps its own tile store, task counters (at an offset of the
// shared counter array) and tile order; one ready queue spans all of them, so
// CTAs run whatever task of whichever matrix is ready.  A matrix whose POTRF
// fails records its info and turns its remaining tasks into no-ops (the other
// matrices are unaffected).  After POTRF(M-1) of a matrix its SOLVE task runs
// the forward and backward substitution for its right-hand side in one CTA.
// The graph holds: descriptor upload (from pinned host memory), repack of all
// matrices, queue/counter reset, queue seeding, the persistent kernel, unpack
// of the factors and the info download.  In FP64 batches the matrices of
// order above 1024 (where a single factorization runs on the tensor cores)
// form a part of their own: tiles of order 128 and one persistent kernel of
// the tensor-core engine for all of them (batched_tc.cu), before the
// persistent kernel of the others; in FP32 batches the same split puts the
// larger matrices on the tensor-core bodies of the mixed-precision engine in
// its FP32 mode (batched_mixed.cu).  Internally the smaller matrices come
// first (a permutation maps them back to the caller's order).
#include <string.h>

#include <vector>

#include "batched_impl.cuh"

namespace chol {

template <typename T>
struct BatchSmem {
    SimtSmem<T> simt;
    T y[2048];          // right-hand side of the SOLVE task (n <= 2048)
};

static_assert(sizeof(SolveScratch<double>) <= sizeof(SimtSmem<double>) &&
                  sizeof(SolveScratch<float>) <= sizeof(SimtSmem<float>),
              "the SOLVE task's scratch fits in the tile bodies' scratch");

template <typename T>
struct BatchBody {
    struct Args {
        const MatDesc *desc;
        int64_t *info;     // per matrix
        int32_t *failed;   // per matrix
    };
    using Smem = BatchSmem<T>;
    static constexpr bool kSolveTask = true;
    static constexpr int kCtasPerSm = 4;
    static constexpr int kBlock = kThreads;
    static constexpr bool kLag = false;
    static constexpr size_t kSmemBytes = sizeof(BatchSmem<T>);
    static __device__ __forceinline__ void cta_init(const Args &, Smem &) {}
    static __device__ __forceinline__ void cta_fini(const Args &, Smem &) {}
    static __device__ __forceinline__ int tiles(const Args &g, int m) { return g.desc[m].M; }
    static __device__ __forceinline__ int64_t task_base(const Args &g, int m) { return g.desc[m].task_base; }

    static __device__ __forceinline__ T *tile(const MatDesc &d, int I, int K) {
        return reinterpret_cast<T *>(d.store) + (size_t)tile_index(I, K) * d.nb * d.nb;
    }

    static __device__ void run(const Args &g, const SchedArgs &a, int m, int I, int K, int J, Smem &sm) {
        const int type = task_type(I, K, J);
        uint64_t t0 = 0;
        if (a.trace && threadIdx.x == 0) t0 = global_ns();
        const MatDesc d = g.desc[m];
        const bool skip = batch_skip(a, g.failed, m);
        if (!skip) {
            switch (type) {
            case T_POTRF: {
                const int li = tile_potrf(tile(d, J, J), d.nb, sm.simt);
                if (li && threadIdx.x == 0) {
                    g.info[m] = (int64_t)J * d.nb + li;
                    st_release_s32(g.failed + m, 1);
                }
            } break;
            case T_TRSM: tile_trsm(tile(d, I, J), tile(d, J, J), d.nb, sm.simt); break;
            case T_SYRK: tile_syrk(tile(d, I, I), tile(d, I, J), d.nb, sm.simt); break;
            default: tile_gemm(tile(d, I, K), tile(d, I, J), tile(d, K, J), d.nb, sm.simt); break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) task_done_bookkeeping(a, type, m, I, K, J, t0);
    }

    // L L^T x = b for matrix m, one CTA: forward and backward substitution
    // blocked by chunks of 32 rows (tiles_solve).
    static __device__ void solve(const Args &g, const SchedArgs &a, int m, Smem &sm) {
        const MatDesc d = g.desc[m];
        uint64_t t0 = 0;
        if (a.trace && threadIdx.x == 0) t0 = global_ns();
        const bool skip = batch_skip(a, g.failed, m);
        const int n = d.n, nb = d.nb;
        if (!skip) {
            tiles_solve<T>(reinterpret_cast<const T *>(d.store), nb, n, d.b, sm.y,
                           *reinterpret_cast<SolveScratch<T> *>(&sm.simt));
        }
        __syncthreads();
        if (threadIdx.x == 0 && a.trace) {
            const unsigned long long slot = atomicAdd(&a.ctl->trace_count, 1ull);
            if ((int64_t)slot < a.trace_cap) {
                chol_trace_rec r;
                r.type = 4;
                r.I = r.K = r.J = d.M;
                r.sm = (int32_t)smid();
                r.matrix = m;
                r.t_start = t0;
                r.t_end = global_ns();
                a.trace[slot] = r;
            }
        }
    }
};

}  // namespace chol

using namespace chol;

struct chol_batch_s {
    int32_t batch = 0;
    int32_t precision = CHOL_FP64;
    std::vector<int64_t> n, nb, M;      // internal order: matrices of the CUDA-core part, then the tensor-core part
    std::vector<int32_t> perm;          // perm[k] = caller's index of internal matrix k
    int32_t small = 0;                  // matrices of the CUDA-core part
    OzBatchPart *tc = nullptr;          // FP64 tensor-core part (matrices small .. batch-1), or null
    MixedBatchPart *mtc = nullptr;      // FP32 tensor-core part (matrices small .. batch-1), or null
    void *tc_ws = nullptr;
    chol_opts opts{};
    int64_t total_tasks = 0, total_tiles = 0;
    int max_nsb2 = 1;
    // device
    void *ws = nullptr;
    MatDesc *d_desc = nullptr;
    TileRef *d_list = nullptr;
    int64_t *d_info = nullptr;
    int32_t *d_failed = nullptr;
    Control *d_ctl = nullptr;
    unsigned long long *d_queue = nullptr;
    int32_t *d_deps = nullptr;
    // host (pinned)
    MatDesc *h_desc = nullptr;
    int64_t *h_info = nullptr;
    Control *h_ctl = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;  // recorded inside the graph (not timed)
    cudaEvent_t t0 = nullptr, t1 = nullptr;  // around the graph launch
    int launches = 0;
};

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

template <typename T>
static int record_batch(chol_batch_s *p) {
    cudaStream_t st = p->stream;
    const size_t dbytes = sizeof(MatDesc) * p->batch;
    CHOL_CUDA(cudaMemcpyAsync(p->d_desc, p->h_desc, dbytes, cudaMemcpyHostToDevice, st));
    CHOL_CUDA(cudaMemsetAsync(p->d_ctl, 0, sizeof(Control), st));
    CHOL_CUDA(cudaMemsetAsync(p->d_info, 0, sizeof(int64_t) * p->batch, st));
    CHOL_CUDA(cudaMemsetAsync(p->d_failed, 0, sizeof(int32_t) * p->batch, st));
    const dim3 rgrid((unsigned)p->total_tiles, (unsigned)((p->max_nsb2 + kSubPer - 1) / kSubPer));
    batch_repack_kernel<T><<<rgrid, dim3(32, 8), 0, st>>>(p->d_desc, p->d_list);
    CHOL_CUDA(cudaGetLastError());
    int launches = 0, rc = CHOL_OK;
    CHOL_CUDA(cudaEventRecord(p->e0, st));
    if (p->tc) {
        int l = 0;
        if ((rc = oz_batch_record(p->tc, p->d_desc + p->small, p->d_info + p->small, p->d_failed + p->small, st,
                                  &l)) != CHOL_OK)
            return rc;
        launches += l;
    }
    if (p->mtc) {
        int l = 0;
        if ((rc = mixed_batch_record(p->mtc, p->d_desc + p->small, p->d_info + p->small, p->d_failed + p->small, st,
                                     &l)) != CHOL_OK)
            return rc;
        launches += l;
    }
    if (p->small > 0) {
        typename BatchBody<T>::Args g{p->d_desc, p->d_info, p->d_failed};
        SchedArgs a{p->d_ctl, p->opts.trace, p->opts.trace_capacity, p->opts.flags, 0};
        DFArgs d{};
        d.queue = p->d_queue;
        d.deps = p->d_deps;
        d.capacity = p->total_tasks;
        d.total = p->total_tasks;
        d.num_matrices = p->small;
        int l = 0;
        if ((rc = launch_dataflow<BatchBody<T>>(g, a, d, p->opts, st, &l)) != CHOL_OK) return rc;
        launches += l;
    }
    CHOL_CUDA(cudaEventRecord(p->e1, st));
    batch_unpack_kernel<T><<<rgrid, dim3(32, 8), 0, st>>>(p->d_desc, p->d_list);
    CHOL_CUDA(cudaGetLastError());
    CHOL_CUDA(cudaMemcpyAsync(p->h_info, p->d_info, sizeof(int64_t) * p->batch, cudaMemcpyDeviceToHost, st));
    CHOL_CUDA(cudaMemcpyAsync(p->h_ctl, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
    p->launches = launches + 2;
    return CHOL_OK;
}

extern "C" {

void chol_batch_free(chol_batch_h p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->ws) cudaFree(p->ws);
    if (p->tc) oz_batch_destroy(p->tc);
    if (p->mtc) mixed_batch_destroy(p->mtc);
    if (p->tc_ws) cudaFree(p->tc_ws);
    if (p->h_desc) cudaFreeHost(p->h_desc);
    if (p->h_info) cudaFreeHost(p->h_info);
    if (p->h_ctl) cudaFreeHost(p->h_ctl);
    if (p->e0) cudaEventDestroy(p->e0);
    if (p->e1) cudaEventDestroy(p->e1);
    if (p->t0) cudaEventDestroy(p->t0);
    if (p->t1) cudaEventDestroy(p->t1);
    if (p->stream) cudaStreamDestroy(p->stream);
    delete p;
}

int chol_batch_plan(int32_t batch, const int64_t *n, const chol_opts *opts, chol_batch_h *out) {
    CHOL_CHECK_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    CHOL_CHECK_ARG(batch >= 1 && batch < 65536, "batch must be in [1, 65535]");
    CHOL_CHECK_ARG(n != nullptr, "n is NULL");
    chol_opts o = resolve_opts(opts);
    CHOL_CHECK_ARG(o.precision == CHOL_FP64 || o.precision == CHOL_FP32, "batched precision must be FP64 or FP32");
    cudaGetLastError();  // start from a clean error state
    chol_batch_s *p = new chol_batch_s();
    p->batch = batch;
    p->precision = o.precision;
    p->opts = o;
    const size_t esz = o.precision == CHOL_FP64 ? 8 : 4;
    size_t store_bytes = 0;
    int64_t tasks = 0, tiles = 0;
    for (int i = 0; i < batch; ++i) {
        if (n[i] < 1 || n[i] > 2048) {
            delete p;
            set_error("argument: batched orders must be in [1, 2048] (matrix %d has n=%lld)", i, (long long)n[i]);
            return CHOL_ERR_ARG;
        }
    }
    // matrices above order 1024 (or opts->tc_min_order) go to the
    // tensor-core part (1024: the choice of a single FP64 factorization with
    // the default tile order), unless CHOL_FLAG_FP64_SIMT keeps an FP64 batch
    // on the CUDA cores; the others keep the CUDA-core bodies with the tile
    // order (cap) of opts->nb
    const int64_t tc_min = o.tc_min_order > 0 ? o.tc_min_order : kFp64TcMinN;
    auto on_tc = [&](int64_t nn) {
        return !(o.precision == CHOL_FP64 && (o.flags & CHOL_FLAG_FP64_SIMT)) && nn > tc_min;
    };
    for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < batch; ++i)
            if (on_tc(n[i]) == (pass == 1)) p->perm.push_back(i);
    std::vector<int64_t> tc_n;
    for (int k = 0; k < batch; ++k) {
        const int64_t ni = n[p->perm[k]];
        const bool tc = on_tc(ni);
        int64_t nb = tc ? 128 : (o.nb > 0 ? o.nb : chol_default_nb(ni, o.precision));
        if (!tc && nb > ni) nb = ni;  // a matrix smaller than the tile is one tile of its own order
        const int64_t M = (ni + nb - 1) / nb;
        p->n.push_back(ni);
        p->nb.push_back(nb);
        p->M.push_back(M);
        store_bytes += al256((size_t)num_tiles(M) * nb * nb * esz);
        if (tc) tc_n.push_back(ni);
        else {
            tasks += num_tasks(M) + 1;  // + SOLVE
            p->small = k + 1;
        }
        tiles += num_tiles(M);
        const int nsb = (int)((nb + 31) / 32);
        p->max_nsb2 = nsb * nsb > p->max_nsb2 ? nsb * nsb : p->max_nsb2;
    }
    p->total_tasks = tasks;
    p->total_tiles = tiles;
    const size_t b_desc = al256(sizeof(MatDesc) * batch), b_list = al256(sizeof(TileRef) * tiles);
    const size_t b_info = al256(8 * (size_t)batch), b_failed = al256(4 * (size_t)batch);
    const size_t b_ctl = al256(sizeof(Control)), b_q = al256((size_t)2 * tasks * 8), b_d = al256((size_t)tasks * 4);
    int rc = CHOL_OK;
    do {
        if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&p->e0) != cudaSuccess || cudaEventCreate(&p->e1) != cudaSuccess ||
            cudaEventCreate(&p->t0) != cudaSuccess || cudaEventCreate(&p->t1) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "batch stream", __FILE__, __LINE__);
            break;
        }
        if (cudaMalloc(&p->ws, store_bytes + b_desc + b_list + b_info + b_failed + b_ctl + b_q + b_d) != cudaSuccess) {
            cudaGetLastError();
            set_error("batched plan: device allocation of %zu bytes failed",
                      store_bytes + b_desc + b_list + b_info + b_failed + b_ctl + b_q + b_d);
            rc = CHOL_ERR_NOMEM;
            break;
        }
        if (cudaMallocHost(&p->h_desc, sizeof(MatDesc) * batch) != cudaSuccess ||
            cudaMallocHost(&p->h_info, 8 * (size_t)batch) != cudaSuccess ||
            cudaMallocHost(&p->h_ctl, sizeof(Control)) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "pinned host buffers", __FILE__, __LINE__);
            break;
        }
        char *w = (char *)p->ws;
        char *stores = w;
        w += store_bytes;
        p->d_desc = (MatDesc *)w;
        w += b_desc;
        p->d_list = (TileRef *)w;
        w += b_list;
        p->d_info = (int64_t *)w;
        w += b_info;
        p->d_failed = (int32_t *)w;
        w += b_failed;
        p->d_ctl = (Control *)w;
        w += b_ctl;
        p->d_queue = (unsigned long long *)w;
        w += b_q;
        p->d_deps = (int32_t *)w;
        // descriptors (pointers to caller data are filled by chol_batch_run) and the tile list
        std::vector<TileRef> list;
        list.reserve(tiles);
        size_t off = 0;
        int64_t tb = 0;
        for (int i = 0; i < batch; ++i) {
            MatDesc &d = p->h_desc[i];
            memset(&d, 0, sizeof(d));
            d.store = stores + off;
            d.task_base = tb;
            d.n = (int32_t)p->n[i];
            d.nb = (int32_t)p->nb[i];
            d.M = (int32_t)p->M[i];
            off += al256((size_t)num_tiles(p->M[i]) * p->nb[i] * p->nb[i] * esz);
            tb += num_tasks(p->M[i]);
            for (int64_t t = 0; t < num_tiles(p->M[i]); ++t) list.push_back(TileRef{i, (int32_t)t});
        }
        if (cudaMemcpy(p->d_list, list.data(), sizeof(TileRef) * tiles, cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "tile list", __FILE__, __LINE__);
            break;
        }
        if (!tc_n.empty()) {
            const bool fp64 = p->precision == CHOL_FP64;
            const size_t tcb = fp64 ? oz_batch_bytes((int)tc_n.size(), tc_n.data(), nullptr)
                                    : mixed_batch_bytes((int)tc_n.size(), tc_n.data(), nullptr);
            if (cudaMalloc(&p->tc_ws, tcb) != cudaSuccess) {
                cudaGetLastError();
                set_error("batched plan: device allocation of %zu bytes (tensor-core part) failed", tcb);
                rc = CHOL_ERR_NOMEM;
                break;
            }
            rc = fp64 ? oz_batch_create(&p->tc, (int)tc_n.size(), tc_n.data(), p->tc_ws, p->h_desc + p->small, p->opts)
                      : mixed_batch_create(&p->mtc, (int)tc_n.size(), tc_n.data(), p->tc_ws, p->opts);
            if (rc != CHOL_OK) break;
        }
        // kernel attributes and the occupancy query are settled before the capture starts
        if ((rc = p->precision == CHOL_FP64 ? set_smem_attr<BatchBody<double>>(df_kernel<BatchBody<double>>)
                                            : set_smem_attr<BatchBody<float>>(df_kernel<BatchBody<float>>)) != CHOL_OK)
            break;
        if (p->precision == CHOL_FP64) df_grid<BatchBody<double>>(0);
        else df_grid<BatchBody<float>>(0);
        // capture the whole launch sequence once
        if (cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "capture", __FILE__, __LINE__);
            break;
        }
        rc = p->precision == CHOL_FP64 ? record_batch<double>(p) : record_batch<float>(p);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(p->stream, &graph);
        if (rc != CHOL_OK) {
            if (graph) cudaGraphDestroy(graph);
            break;
        }
        if (ce != cudaSuccess) {
            rc = cuda_fail(ce, "end capture", __FILE__, __LINE__);
            break;
        }
        p->graph = graph;
        if (cudaGraphInstantiate(&p->exec, graph, 0) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "graph instantiate", __FILE__, __LINE__);
            break;
        }
    } while (0);
    if (rc != CHOL_OK) {
        chol_batch_free(p);
        return rc;
    }
    *out = p;
    return CHOL_OK;
}

int chol_batch_run(chol_batch_h p, double *const *A, const int64_t *lda, double *const *B, int64_t *info) {
    if (!p || !p->exec) {
        set_error("invalid batch plan");
        return CHOL_ERR_HANDLE;
    }
    CHOL_CHECK_ARG(A && lda && B && info, "NULL array argument");
    for (int k = 0; k < p->batch; ++k) {
        const int i = p->perm[k];
        CHOL_CHECK_ARG(A[i] && B[i] && lda[i] >= p->n[k], "matrix / rhs pointer NULL or lda < n");
        p->h_desc[k].A = A[i];
        p->h_desc[k].lda = lda[i];
        p->h_desc[k].b = B[i];
    }
    CHOL_CUDA(cudaEventRecord(p->t0, p->stream));
    CHOL_CUDA(cudaGraphLaunch(p->exec, p->stream));
    CHOL_CUDA(cudaEventRecord(p->t1, p->stream));
    CHOL_CUDA(cudaStreamSynchronize(p->stream));
    for (const Control *c : {(const Control *)p->h_ctl, p->tc ? oz_batch_control(p->tc) : nullptr,
                             p->mtc ? mixed_batch_control(p->mtc) : nullptr}) {
        if (c && c->status) {
            set_error("batched: device-side wait expired (site %d)", c->timeout_where);
            return c->status;
        }
    }
    for (int k = 0; k < p->batch; ++k) info[p->perm[k]] = p->h_info[k];
    return CHOL_OK;
}

int chol_batch_stats(chol_batch_h p, chol_stats *st) {
    if (!p) {
        set_error("invalid batch plan");
        return CHOL_ERR_HANDLE;
    }
    CHOL_CHECK_ARG(st != nullptr, "stats is NULL");
    memset(st, 0, sizeof(*st));
    const Control *tcc = p->tc ? oz_batch_control(p->tc) : p->mtc ? mixed_batch_control(p->mtc) : nullptr;
    for (int i = 0; i < 4; ++i) st->tasks[i] = (int64_t)p->h_ctl->tasks[i] + (tcc ? (int64_t)tcc->tasks[i] : 0);
    st->nb = p->batch ? p->nb[0] : 0;
    st->schedule = CHOL_SCHED_DATAFLOW;
    st->launches = p->launches;
    st->trace_records = (int64_t)p->h_ctl->trace_count + (tcc ? (int64_t)tcc->trace_count : 0);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->t0, p->t1) == cudaSuccess) st->device_ms = ms;
    return CHOL_OK;
}

}  // extern "C"
