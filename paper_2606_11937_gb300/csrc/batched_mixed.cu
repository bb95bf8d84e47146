// batched_mixed.cu -- the tensor-core part of a binary32 batched factor +
// solve plan (many independent factorizations of Section 3.1 in one
// dataflow launch of Section 3.2): every matrix of order above the split order is factored on
// tiles of order 128 with the task bodies of the mixed-precision engine in
// its FP32 mode (TRSM in binary32, SYRK/GEMM as three TF32 products with
// binary32 accumulation in tensor memory, mixed_body.cuh), the diagonal tiles
// factored in binary32 as in the rest of a binary32 batch (shared memory, the
// same right-looking order as the engine's binary64 one), and then solved in
// binary32, all of them in ONE
// persistent dataflow kernel with one ready queue.  The matrices' binary32
// tiles live in the batch's tile stores; their TF32 operand copies (hi and
// lo) in one arena each, so one pair of tensor maps serves every matrix.  A
// matrix whose POTRF fails records its info and turns its remaining tasks
// into no-ops; the other matrices are unaffected.  The bits of a matrix do
// not depend on the rest of the batch (every tile receives its operations in
// the same order).
#include <string.h>

#include <vector>

#include "batched_impl.cuh"
#include "mixed_body.cuh"

namespace chol {

int make_operand_map(CUtensorMap *map, void *base, int fmt, int64_t rows, int64_t nb, int box_rows);

constexpr int kMbNb = 128;  // tile order of this part

struct MixedBatchDesc {
    int64_t task_base;  // offset of its task counters
    int64_t tile_off;   // arena index of its tile (0, 0) (operand copies)
    int32_t n, M;
};

struct MixedBatchArgs {
    MixedArgs mx;                 // operand maps over the arenas, format, precision, wait bound
    const MixedBatchDesc *desc;   // per matrix of this part
    const MatDesc *mdesc;         // the batch's descriptors of these matrices (store, right-hand side)
    int64_t *info;                // per matrix of this part
    int32_t *failed;              // per matrix of this part
};

struct MixedBatchBody {
    using Args = MixedBatchArgs;
    using Smem = MixedSmem;
    static constexpr bool kSolveTask = true;
    static constexpr int kCtasPerSm = 1;
    static constexpr int kBlock = kThreads;
    static constexpr size_t kSmemBytes = sizeof(MixedSmem);
    // a SYRK/GEMM leaves its epilogue to the next update on this CTA (as in
    // the single-matrix body)
    static constexpr bool kLag = true;
    static __device__ __forceinline__ bool lagging(Smem &sm) { return sm.ts.pend != 0; }
    static __device__ __forceinline__ bool absorbs(const Args &, int I, int K, int J) {
        if (J == kSolveJ) return false;
        const int type = task_type(I, K, J);
        return type == T_SYRK || type == T_GEMM;
    }
    static __device__ void fail_timeout(const SchedArgs &a) {
        if (atomicCAS(&a.ctl->status, 0, (int32_t)CHOL_ERR_TIMEOUT) == 0) a.ctl->timeout_where = 7;
        st_release_s32(&a.ctl->abort, 1);
    }
    struct Done {
        const Args &g;
        const SchedArgs &a;
        __device__ void operator()(uint64_t w, uint64_t t0) const {
            df_complete_lagged<MixedBatchBody>(g, a, (int)(w >> 48), (int)((w >> 32) & 0xffff),
                                               (int)((w >> 16) & 0xffff), (int)(w & 0xffff), t0);
        }
    };
    static __device__ void flush(const Args &g, const SchedArgs &a, Smem &sm) {
        const bool ok = tc_flush(sm.ts, g.mx.timeout_ns, Done{g, a});
        if (!ok && threadIdx.x == 0) fail_timeout(a);
    }
    static __device__ __forceinline__ void cta_init(const Args &, Smem &sm) { tc_cta_init(sm.ts); }
    static __device__ __forceinline__ void cta_fini(const Args &, Smem &sm) { tc_cta_fini(sm.ts); }
    static __device__ __forceinline__ int tiles(const Args &g, int m) { return g.desc[m].M; }
    static __device__ __forceinline__ int64_t task_base(const Args &g, int m) { return g.desc[m].task_base; }

    static __device__ void run(const Args &g, const SchedArgs &a, int m, int I, int K, int J, Smem &sm) {
        uint64_t t0 = 0;
        if (a.trace && threadIdx.x == 0) t0 = global_ns();
        const bool skip = batch_skip(a, g.failed, m);
        bool ok = true;
        if (skip && sm.ts.pend) {
            // a task of a failed matrix that may start with an epilogue
            // deferred: complete that one first, so that this task completes
            // on return like any other
            ok = tc_flush(sm.ts, g.mx.timeout_ns, Done{g, a});
        } else if (!skip) {
            const auto fail = [&g, m](int64_t col) {
                g.info[m] = col;
                st_release_s32(g.failed + m, 1);
            };
            ok = mixed_task<true>(g.mx, a, m, I, K, J, sm, reinterpret_cast<float *>(g.mdesc[m].store),
                                  g.desc[m].tile_off, t0, Done{g, a}, fail);
        }
        if (!ok && threadIdx.x == 0) fail_timeout(a);
        __syncthreads();
        if (threadIdx.x == 0 && !sm.ts.pend) task_done_bookkeeping(a, task_type(I, K, J), m, I, K, J, t0);
    }

    // forward and backward substitution in binary32 with the matrix's factor
    // (one CTA; a deferred epilogue was completed before: absorbs() is false)
    static __device__ void solve(const Args &g, const SchedArgs &a, int m, Smem &sm) {
        uint64_t t0 = 0;
        if (a.trace && threadIdx.x == 0) t0 = global_ns();
        const MatDesc d = g.mdesc[m];
        const bool skip = batch_skip(a, g.failed, m);
        float *y = reinterpret_cast<float *>(&sm.stages[0][0]);
        if (!skip) tiles_solve<float>(reinterpret_cast<const float *>(d.store), kMbNb, d.n, d.b, y,
                                      *reinterpret_cast<SolveScratch<float> *>(y + 2048));
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

static_assert(2048 * sizeof(float) + sizeof(SolveScratch<float>) <= sizeof(MixedSmem::stages),
              "the SOLVE task's right-hand side and scratch fit in the stages");

struct MixedBatchPart {
    int count = 0;
    int64_t tasks = 0, tiles = 0;
    chol_opts o{};
    MixedBatchArgs g{};
    MixedBatchDesc *d_desc = nullptr;
    Control *d_ctl = nullptr;
    unsigned long long *d_queue = nullptr;
    int32_t *d_deps = nullptr;
    Control *h_ctl = nullptr;  // pinned
};

static size_t a256m(size_t x) { return (x + 255) & ~size_t(255); }

// Arena sizes of a part with `count` matrices of orders n[0 .. count-1].
struct MixedBatchLayout {
    int64_t tiles = 0, tasks = 0;
    size_t b_desc, b_hi, b_lo, b_ctl, b_q, b_d;
    size_t total() const { return b_desc + b_hi + b_lo + b_ctl + b_q + b_d; }
};

static MixedBatchLayout mb_layout(int count, const int64_t *n) {
    MixedBatchLayout L;
    for (int i = 0; i < count; ++i) {
        const int64_t M = (n[i] + kMbNb - 1) / kMbNb;
        L.tiles += num_tiles(M);
        L.tasks += num_tasks(M) + 1;  // + SOLVE
    }
    const size_t op = (size_t)kMbNb * kMbNb * 4;  // one TF32 tile
    L.b_desc = a256m(sizeof(MixedBatchDesc) * count);
    L.b_hi = a256m((size_t)L.tiles * op);
    L.b_lo = a256m((size_t)L.tiles * op);
    L.b_ctl = a256m(sizeof(Control));
    L.b_q = a256m((size_t)2 * L.tasks * 8);
    L.b_d = a256m((size_t)L.tasks * 4);
    return L;
}

size_t mixed_batch_bytes(int count, const int64_t *n, int64_t *tasks_out) {
    const MixedBatchLayout L = mb_layout(count, n);
    if (tasks_out) *tasks_out = L.tasks;
    return L.total();
}

int mixed_batch_create(MixedBatchPart **out, int count, const int64_t *n, void *ws, const chol_opts &o) {
    *out = nullptr;
    const MixedBatchLayout L = mb_layout(count, n);
    CHOL_CHECK_ARG(L.tiles * kMbNb < (1ll << 31), "batched: too many tiles of order 128 for the operand maps");
    MixedBatchPart *p = new MixedBatchPart();
    p->count = count;
    p->tiles = L.tiles;
    p->tasks = L.tasks;
    p->o = o;
    char *w = (char *)ws;
    p->d_desc = (MixedBatchDesc *)w;
    w += L.b_desc;
    MixedBatchArgs &g = p->g;
    memset(&g, 0, sizeof(g));
    g.mx.op_hi = w;
    w += L.b_hi;
    g.mx.op_lo = (float *)w;
    w += L.b_lo;
    p->d_ctl = (Control *)w;
    w += L.b_ctl;
    p->d_queue = (unsigned long long *)w;
    w += L.b_q;
    p->d_deps = (int32_t *)w;
    // the tile order is the only field of the tile store the bodies read
    g.mx.S = TileStore<float>{nullptr, kMbNb, 0};
    g.mx.precision = CHOL_FP32;
    g.mx.fmt = OP_TF32;
    g.mx.timeout_ns = (uint64_t)(o.timeout_s * 1e9);
    g.desc = p->d_desc;
    std::vector<MixedBatchDesc> hd(count);
    int64_t tb = 0, to = 0;
    for (int i = 0; i < count; ++i) {
        const int64_t M = (n[i] + kMbNb - 1) / kMbNb;
        hd[i].task_base = tb;
        hd[i].tile_off = to;
        hd[i].n = (int32_t)n[i];
        hd[i].M = (int32_t)M;
        tb += num_tasks(M);
        to += num_tiles(M);
    }
    int rc = CHOL_OK;
    do {
        if (cudaMemcpy(p->d_desc, hd.data(), sizeof(MixedBatchDesc) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMallocHost(&p->h_ctl, sizeof(Control)) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "batched tensor-core part", __FILE__, __LINE__);
            break;
        }
        memset(p->h_ctl, 0, sizeof(Control));
        if ((rc = make_operand_map(&g.mx.map_hi, g.mx.op_hi, OP_TF32, L.tiles * kMbNb, kMbNb, kBoxRows)) != CHOL_OK)
            break;
        if ((rc = make_operand_map(&g.mx.map_lo, g.mx.op_lo, OP_TF32, L.tiles * kMbNb, kMbNb, kBoxRows)) != CHOL_OK)
            break;
        // kernel attributes and the occupancy query are settled before the batch's capture
        if ((rc = set_smem_attr<MixedBatchBody>(df_kernel<MixedBatchBody>)) != CHOL_OK) break;
        df_grid<MixedBatchBody>(0);
    } while (0);
    if (rc != CHOL_OK) {
        mixed_batch_destroy(p);
        return rc;
    }
    *out = p;
    return CHOL_OK;
}

int mixed_batch_record(MixedBatchPart *p, const MatDesc *d_desc_part, int64_t *d_info_part, int32_t *d_failed_part,
                       cudaStream_t st, int *launches) {
    MixedBatchArgs g = p->g;
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
    int rc = launch_dataflow<MixedBatchBody>(g, a, d, o, st, launches);
    if (rc != CHOL_OK) return rc;
    CHOL_CUDA(cudaMemcpyAsync(p->h_ctl, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
    return CHOL_OK;
}

const Control *mixed_batch_control(const MixedBatchPart *p) { return p->h_ctl; }

void mixed_batch_destroy(MixedBatchPart *p) {
    if (!p) return;
    if (p->h_ctl) cudaFreeHost(p->h_ctl);
    delete p;
}

}  // namespace chol
