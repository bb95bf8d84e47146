// batched_tc.cu -- the tensor-core FP64 part of a batched factor + solve plan:
// every matrix of order above 1024 is factored on tiles of order 128 with
// SYRK/GEMM/TRSM as exact bf16 slice products (the engine of a single FP64
// factorization at those orders, fp64tc_body.cuh) and then solved, all of
// them in ONE persistent dataflow kernel with one ready queue, so the
// critical paths of the matrices overlap.  The matrices' tiles live in the
// batch's tile stores; their bf16 slices in one arena (one tensor map serves
// every matrix), the inverted diagonal blocks in a second one.  A matrix
// whose POTRF fails records its info and turns its remaining tasks into
// no-ops; the other matrices are unaffected.  Each matrix gets the bits of a
// single FP64 factorization of it on this engine (same block operations in
// the same order).
#include <string.h>

#include <vector>

#include "batched_impl.cuh"
#include "fp64tc_body.cuh"

namespace chol {

int make_operand_map(CUtensorMap *map, void *base, int fmt, int64_t rows, int64_t nb, int box_rows);

struct OzBatchDesc {
    int64_t task_base;  // offset of its task counters
    int64_t tile_off;   // arena index of its tile (0, 0) (slices, row exponents)
    int64_t col_off;    // arena index of its block column 0 (inverted diagonal blocks)
    int32_t n, M;
};

struct OzBatchArgs {
    CUtensorMap mapA;         // slice arena, 128-row boxes
    CUtensorMap mapB;         // slice arena, 32-row boxes
    CUtensorMap mapW;         // inverse-slice arena, 32-row boxes
    const OzBatchDesc *desc;  // per matrix of this part
    const MatDesc *mdesc;     // the batch's descriptors of these matrices (store, right-hand side)
    __nv_bfloat16 *slices;
    int32_t *rexp;
    __nv_bfloat16 *wslices;
    int32_t *wexp;
    double *wbuf;
    int32_t *wflag;
    int64_t *info;    // per matrix of this part
    int32_t *failed;  // per matrix of this part
    uint64_t timeout_ns;
};

struct OzBatchBody {
    using Args = OzBatchArgs;
    using Smem = OzSmem;
    static constexpr bool kSolveTask = true;
    static constexpr int kCtasPerSm = 1;
    static constexpr int kBlock = kOzThreads;
    static constexpr size_t kSmemBytes = sizeof(OzSmem);
    // a SYRK/GEMM defers the epilogue of its last quarter to the next update
    // on this CTA (as in the single-matrix body)
    static constexpr bool kLag = true;
    static __device__ __forceinline__ bool lagging(Smem &sm) { return sm.os.pend != 0; }
    static __device__ __forceinline__ bool absorbs(const Args &, int I, int K, int J) {
        if (J == kSolveJ) return false;
        const int type = task_type(I, K, J);
        return type == T_SYRK || type == T_GEMM;
    }
    static __device__ void fail_timeout(const SchedArgs &a) {
        if (atomicCAS(&a.ctl->status, 0, (int32_t)CHOL_ERR_TIMEOUT) == 0) a.ctl->timeout_where = 6;
        st_release_s32(&a.ctl->abort, 1);
    }
    struct Done {
        const Args &g;
        const SchedArgs &a;
        __device__ void operator()(uint64_t w, uint64_t t0) const {
            df_complete_lagged<OzBatchBody>(g, a, (int)(w >> 48), (int)((w >> 32) & 0xffff),
                                            (int)((w >> 16) & 0xffff), (int)(w & 0xffff), t0);
        }
    };
    static __device__ void flush(const Args &g, const SchedArgs &a, Smem &sm) {
        const bool ok = ozaki_flush(sm, g.timeout_ns, Done{g, a});
        if (!ok && threadIdx.x == 0) fail_timeout(a);
    }
    static __device__ __forceinline__ void cta_init(const Args &, Smem &sm) { oz_cta_init(sm.os); }
    static __device__ __forceinline__ void cta_fini(const Args &, Smem &sm) { oz_cta_fini(sm.os); }
    static __device__ __forceinline__ int tiles(const Args &g, int m) { return g.desc[m].M; }
    static __device__ __forceinline__ int64_t task_base(const Args &g, int m) { return g.desc[m].task_base; }

    static __device__ void run(const Args &g, const SchedArgs &a, int m, int I, int K, int J, Smem &sm) {
        const int type = task_type(I, K, J);
        uint64_t t0 = 0;
        if (a.trace && threadIdx.x == 0) t0 = global_ns();
        const OzBatchDesc od = g.desc[m];
        double *store = reinterpret_cast<double *>(g.mdesc[m].store);
        auto tile = [&](int i, int k) { return store + (size_t)tile_index(i, k) * kOzNb * kOzNb; };
        const bool skip = batch_skip(a, g.failed, m);
        const auto take_ahead = [&a]() { df_take_ahead(a); };
        bool ok = true;
        if (skip && sm.os.pend) {
            // a task of a failed matrix that may start with an epilogue
            // deferred: complete that one first, so that this task completes
            // on return like any other
            ok = ozaki_flush(sm, g.timeout_ns, Done{g, a});
        } else if (!skip) {
            switch (type) {
            case T_POTRF: {
                const int li = oz_potrf128(tile(J, J), sm);
                if (li) {
                    if (threadIdx.x == 0) {
                        g.info[m] = (int64_t)J * kOzNb + li;
                        st_release_s32(g.failed + m, 1);
                    }
                } else if (J < od.M - 1) {
                    // W_J = L_JJ^{-1} for the TRSMs of this block column and,
                    // when it is well conditioned, its slices
                    const int64_t c = od.col_off + J;
                    double *W = g.wbuf + (size_t)c * kOzNb * kOzNb;
                    const double kappa = oz_trtri128(sm, W);
                    const bool use_w = kappa <= kTrsmKappa;  // false also for a NaN
                    if (use_w) ozaki_split(W, g.wslices + (size_t)c * kOzS * kOzNb * kOzNb, g.wexp + (size_t)c * kOzNb);
                    if (threadIdx.x == 0) g.wflag[c] = use_w ? 1 : 0;
                }
            } break;
            case T_TRSM: {
                const int64_t t = od.tile_off + tile_index(I, J), c = od.col_off + J;
                double *X = tile(I, J);
                __nv_bfloat16 *sl = g.slices + (size_t)t * kOzS * kOzNb * kOzNb;
                if (!__ldcg(g.wflag + c)) {  // substitution on the CUDA cores (threads 0..255)
                    SimtSmem<double> &ss = *reinterpret_cast<SimtSmem<double> *>(sm.B);
                    if (threadIdx.x < kThreads) tile_trsm(X, tile(J, J), kOzNb, ss);
                    __syncthreads();
                    ozaki_split(X, sl, g.rexp + t * kOzNb);
                    break;
                }
                // X = A_IJ W_J^T as the emulated update C -= (-A_IJ) W_J^T of a cleared tile
                ozaki_split(X, sl, g.rexp + t * kOzNb, true, false);
                for (int e = threadIdx.x; e < kOzNb * kOzNb; e += blockDim.x) X[e] = 0.0;
                __syncthreads();
                ok = ozaki_tile_update(sm, &g.mapA, &g.mapW, X, (int)(t * kOzS * kOzNb), (int)(c * kOzS * kOzNb),
                                       g.rexp + t * kOzNb, g.wexp + (size_t)c * kOzNb, g.timeout_ns, take_ahead,
                                       Done{g, a});
                if (ok) ozaki_split(X, sl, g.rexp + t * kOzNb);
            } break;
            default: {
                const int64_t ta = od.tile_off + tile_index(I, J), tb = od.tile_off + tile_index(K, J);
                ok = ozaki_tile_update(sm, &g.mapA, &g.mapB, tile(I, K), (int)(ta * kOzS * kOzNb),
                                       (int)(tb * kOzS * kOzNb), g.rexp + ta * kOzNb, g.rexp + tb * kOzNb,
                                       g.timeout_ns, take_ahead, Done{g, a}, a.dfl != nullptr, pack_task(m, I, K, J),
                                       t0);
            } break;
            }
        }
        if (!ok && threadIdx.x == 0) fail_timeout(a);
        __syncthreads();
        if (threadIdx.x == 0 && !sm.os.pend) task_done_bookkeeping(a, type, m, I, K, J, t0);
    }

    // forward and backward substitution with the matrix's factor (one CTA;
    // the pending quarter, if any, was flushed before: absorbs() is false)
    static __device__ void solve(const Args &g, const SchedArgs &a, int m, Smem &sm) {
        uint64_t t0 = 0;
        if (a.trace && threadIdx.x == 0) t0 = global_ns();
        const MatDesc d = g.mdesc[m];
        const bool skip = batch_skip(a, g.failed, m);
        double *y = reinterpret_cast<double *>(sm.B);
        if (!skip) tiles_solve<double>(reinterpret_cast<const double *>(d.store), kOzNb, d.n, d.b, y,
                                       *reinterpret_cast<SolveScratch<double> *>(y + 2048));
        __syncthreads();
        if (threadIdx.x == 0 && a.trace) {
            const unsigned long long slot = atomicAdd(&a.ctl->trace_count, 1ull);
            if ((int64_t)slot < a.trace_cap) {
                chol_trace_rec r;
                r.type = 4;
                r.I = r.K = r.J = g.desc[m].M;
                r.sm = (int32_t)smid();
                r.matrix = m;
                r.t_start = t0;
                r.t_end = global_ns();
                a.trace[slot] = r;
            }
        }
    }
};

static_assert(2048 * sizeof(double) + sizeof(SolveScratch<double>) <= sizeof(OzSmem::B),
              "the SOLVE task's right-hand side and scratch fit in the B region");

struct OzBatchPart {
    int count = 0;
    int64_t tasks = 0, tiles = 0, cols = 0;
    chol_opts o{};
    OzBatchArgs g{};
    OzBatchDesc *d_desc = nullptr;
    Control *d_ctl = nullptr;
    unsigned long long *d_queue = nullptr;
    int32_t *d_deps = nullptr;
    Control *h_ctl = nullptr;  // pinned
};

static size_t a256b(size_t x) { return (x + 255) & ~size_t(255); }

// Arena sizes of a part with `count` matrices of orders n[0 .. count-1].
struct OzBatchLayout {
    int64_t tiles = 0, cols = 0, tasks = 0;
    size_t b_desc, b_sl, b_rexp, b_wsl, b_wexp, b_wbuf, b_wflag, b_ctl, b_q, b_d;
    size_t total() const { return b_desc + b_sl + b_rexp + b_wsl + b_wexp + b_wbuf + b_wflag + b_ctl + b_q + b_d; }
};

static OzBatchLayout oz_layout(int count, const int64_t *n) {
    OzBatchLayout L;
    for (int i = 0; i < count; ++i) {
        const int64_t M = (n[i] + kOzNb - 1) / kOzNb;
        L.tiles += num_tiles(M);
        L.cols += M;
        L.tasks += num_tasks(M) + 1;  // + SOLVE
    }
    const size_t sl = (size_t)kOzS * kOzNb * kOzNb * 2;
    L.b_desc = a256b(sizeof(OzBatchDesc) * count);
    L.b_sl = a256b((size_t)L.tiles * sl);
    L.b_rexp = a256b((size_t)L.tiles * kOzNb * 4);
    L.b_wsl = a256b((size_t)L.cols * sl);
    L.b_wexp = a256b((size_t)L.cols * kOzNb * 4);
    L.b_wbuf = a256b((size_t)L.cols * kOzNb * kOzNb * 8);
    L.b_wflag = a256b((size_t)L.cols * 4);
    L.b_ctl = a256b(sizeof(Control));
    L.b_q = a256b((size_t)2 * L.tasks * 8);
    L.b_d = a256b((size_t)L.tasks * 4);
    return L;
}

size_t oz_batch_bytes(int count, const int64_t *n, int64_t *tasks_out) {
    const OzBatchLayout L = oz_layout(count, n);
    if (tasks_out) *tasks_out = L.tasks;
    return L.total();
}

int oz_batch_create(OzBatchPart **out, int count, const int64_t *n, void *ws, const MatDesc *, const chol_opts &o) {
    *out = nullptr;
    const OzBatchLayout L = oz_layout(count, n);
    CHOL_CHECK_ARG(L.tiles * kOzS * kOzNb < (1ll << 31) && L.cols * kOzS * kOzNb < (1ll << 31),
                   "batched: too many tiles of order 128 for the slice maps");
    OzBatchPart *p = new OzBatchPart();
    p->count = count;
    p->tiles = L.tiles;
    p->cols = L.cols;
    p->tasks = L.tasks;
    p->o = o;
    char *w = (char *)ws;
    p->d_desc = (OzBatchDesc *)w;
    w += L.b_desc;
    OzBatchArgs &g = p->g;
    memset(&g, 0, sizeof(g));
    g.slices = (__nv_bfloat16 *)w;
    w += L.b_sl;
    g.rexp = (int32_t *)w;
    w += L.b_rexp;
    g.wslices = (__nv_bfloat16 *)w;
    w += L.b_wsl;
    g.wexp = (int32_t *)w;
    w += L.b_wexp;
    g.wbuf = (double *)w;
    w += L.b_wbuf;
    g.wflag = (int32_t *)w;
    w += L.b_wflag;
    p->d_ctl = (Control *)w;
    w += L.b_ctl;
    p->d_queue = (unsigned long long *)w;
    w += L.b_q;
    p->d_deps = (int32_t *)w;
    g.desc = p->d_desc;
    g.timeout_ns = (uint64_t)(o.timeout_s * 1e9);
    std::vector<OzBatchDesc> hd(count);
    int64_t tb = 0, to = 0, co = 0;
    for (int i = 0; i < count; ++i) {
        const int64_t M = (n[i] + kOzNb - 1) / kOzNb;
        hd[i].task_base = tb;
        hd[i].tile_off = to;
        hd[i].col_off = co;
        hd[i].n = (int32_t)n[i];
        hd[i].M = (int32_t)M;
        tb += num_tasks(M);
        to += num_tiles(M);
        co += M;
    }
    int rc = CHOL_OK;
    do {
        if (cudaMemcpy(p->d_desc, hd.data(), sizeof(OzBatchDesc) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMallocHost(&p->h_ctl, sizeof(Control)) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "batched tensor-core part", __FILE__, __LINE__);
            break;
        }
        memset(p->h_ctl, 0, sizeof(Control));
        if ((rc = make_operand_map(&g.mapA, g.slices, OP_BF16, L.tiles * kOzS * kOzNb, kOzNb, 128)) != CHOL_OK) break;
        if ((rc = make_operand_map(&g.mapB, g.slices, OP_BF16, L.tiles * kOzS * kOzNb, kOzNb, kOzQ)) != CHOL_OK) break;
        if ((rc = make_operand_map(&g.mapW, g.wslices, OP_BF16, L.cols * kOzS * kOzNb, kOzNb, kOzQ)) != CHOL_OK) break;
        // kernel attributes and the occupancy query are settled before the batch's capture
        if ((rc = set_smem_attr<OzBatchBody>(df_kernel<OzBatchBody>)) != CHOL_OK) break;
        df_grid<OzBatchBody>(0);
    } while (0);
    if (rc != CHOL_OK) {
        oz_batch_destroy(p);
        return rc;
    }
    *out = p;
    return CHOL_OK;
}

int oz_batch_record(OzBatchPart *p, const MatDesc *d_desc_part, int64_t *d_info_part, int32_t *d_failed_part,
                    cudaStream_t st, int *launches) {
    OzBatchArgs g = p->g;
    g.mdesc = d_desc_part;
    g.info = d_info_part;
    g.failed = d_failed_part;
    CHOL_CUDA(cudaMemsetAsync(p->d_ctl, 0, sizeof(Control), st));
    SchedArgs a{p->d_ctl, p->o.trace, p->o.trace_capacity, p->o.flags, 0};
    DFArgs d{};
    d.queue = p->d_queue;
    d.deps = p->d_deps;
    d.capacity = p->tasks;
    d.total = p->tasks;
    d.num_matrices = p->count;
    chol_opts o = p->o;
    o.num_ctas = 0;
    int rc = launch_dataflow<OzBatchBody>(g, a, d, o, st, launches);
    if (rc != CHOL_OK) return rc;
    CHOL_CUDA(cudaMemcpyAsync(p->h_ctl, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
    return CHOL_OK;
}

const Control *oz_batch_control(const OzBatchPart *p) { return p->h_ctl; }

void oz_batch_destroy(OzBatchPart *p) {
    if (!p) return;
    if (p->h_ctl) cudaFreeHost(p->h_ctl);
    delete p;
}

}  // namespace chol
