// fp64tc.cu -- FP64 factorization whose SYRK/GEMM run on the tensor cores with
// binary64 accuracy (exact bf16 slicing, ozaki.cuh).  POTRF stays on the CUDA
// cores in binary64 (the tile in shared memory) and also forms the inverse
// W_J = L_JJ^{-1} there; the TRSMs of block column J are then one emulated
// product A_IJ W_J^T each on the tensor cores, unless L_JJ is ill-conditioned
// (kappa_inf above kTrsmKappa), when they keep the substitution kernel.
// Selected with CHOL_FLAG_FP64_TC (the default above order 1024); tile orders
// 128 r (the bodies are in fp64tc_body.cuh; r > 1 launches from
// fp64tc_blocks.cu).  Every schedule of Section 3.2 runs these bodies
// unchanged.
#include "fp64tc_body.cuh"

namespace chol {

int make_operand_map(CUtensorMap *map, void *base, int fmt, int64_t rows, int64_t nb, int box_rows);

// 2-D map over the slice store (rows x 128 bf16) with boxes of 64 columns x box_rows.
static int make_slice_map(CUtensorMap *map, void *base, int64_t rows, int box_rows) {
    return make_operand_map(map, base, OP_BF16, rows, kOzNb, box_rows);
}

// After the schedule: every block column flagged (a copy stream waiting on
// the flags always proceeds, whatever happened to the factorization).
__global__ void early_out_release_kernel(int32_t *flag, int M) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x)
        asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(flag + i), "r"(1) : "memory");
}

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace bytes beyond the FP64 tile store for an order-n factorization.
size_t fp64tc_extra_bytes(int64_t n) {
    const int64_t M = (n + kOzNb - 1) / kOzNb;
    const size_t tiles = (size_t)num_tiles(M);
    return a256(tiles * kOzS * kOzNb * kOzNb * 2) + a256(tiles * kOzNb * 4) +   // tile slices, exponents
           a256((size_t)M * kOzS * kOzNb * kOzNb * 2) + a256((size_t)M * kOzNb * 4) +  // W_J slices, exponents
           a256((size_t)M * kOzNb * kOzNb * 8) + a256((size_t)M * 4);               // L_JJ^{-T}, flags
}

// Run the schedule with the tensor-core FP64 body on a store repacked at
// tile order 128; the tasks work on tiles of order nb = 128 r (Ml per
// dimension), whose counters and queues the caller sized.
int fp64tc_schedule(double *store, int64_t n, int64_t nb, Control *ctl, unsigned long long *queue, int32_t *deps,
                    int sched, const chol_opts &o, cudaStream_t st, int *launches, cudaEvent_t e0,
                    const EarlyOut *eo) {
    CHOL_CHECK_ARG(nb >= kOzNb && nb % kOzNb == 0, "the tensor-core FP64 engine takes tile orders 128 r");
    const int64_t M = (n + kOzNb - 1) / kOzNb;
    const int r = (int)(nb / kOzNb);
    const int64_t Ml = (M + r - 1) / r;
    const int64_t tiles = num_tiles(M);
    const size_t b_sl = a256((size_t)tiles * kOzS * kOzNb * kOzNb * 2);
    CHOL_CHECK_ARG(tiles * kOzS * kOzNb < (1ll << 31), "matrix too large for the slice maps");
    void *ws = nullptr;
    CHOL_CUDA(cudaMallocAsync(&ws, fp64tc_extra_bytes(n), st));
    OzArgs g;
    memset(&g, 0, sizeof(g));
    g.S = TileStore<double>{store, kOzNb, (int32_t)M};
    g.slices = (__nv_bfloat16 *)ws;
    char *p = (char *)ws + b_sl;
    g.rexp = (int32_t *)p;
    p += a256((size_t)tiles * kOzNb * 4);
    g.wslices = (__nv_bfloat16 *)p;
    p += a256((size_t)M * kOzS * kOzNb * kOzNb * 2);
    g.wexp = (int32_t *)p;
    p += a256((size_t)M * kOzNb * 4);
    g.wbuf = (double *)p;
    p += a256((size_t)M * kOzNb * kOzNb * 8);
    g.wflag = (int32_t *)p;
    g.timeout_ns = (uint64_t)(o.timeout_s * 1e9);
    g.r = r;
    g.Ml = (int32_t)Ml;
    g.n = n;
    if (eo && sched == CHOL_SCHED_DATAFLOW) {
        g.out = eo->out;
        g.out_ld = eo->ld;
        g.out_cnt = eo->cnt;
        g.out_flag = eo->flag;
    }
    int rc = make_slice_map(&g.mapA, g.slices, tiles * kOzS * kOzNb, 128);
    if (rc == CHOL_OK) rc = make_slice_map(&g.mapB, g.slices, tiles * kOzS * kOzNb, kOzQ);
    if (rc == CHOL_OK) rc = make_slice_map(&g.mapW, g.wslices, M * kOzS * kOzNb, kOzQ);
    SchedArgs a{ctl, o.trace, o.trace_capacity, o.flags, 0};
    if (rc == CHOL_OK) {
        if (sched == CHOL_SCHED_DATAFLOW) {
            DFArgs d{};
            d.queue = queue;
            d.deps = deps;
            d.capacity = num_tasks(Ml);
            d.total = num_tasks(Ml);
            d.num_matrices = 1;
            rc = r == 1 ? launch_dataflow<OzBody>(g, a, d, o, st, launches, e0)
                        : fp64tc_launch_blocks(g, a, &d, (int)Ml, 0, o, st, launches, e0);
            if (rc == CHOL_OK && g.out) {
                early_out_release_kernel<<<(unsigned)((Ml + 255) / 256), 256, 0, st>>>(g.out_flag, (int)Ml);
                if (cudaGetLastError() != cudaSuccess) rc = cuda_fail(cudaErrorLaunchFailure, "early output", __FILE__, __LINE__);
            }
        } else {
            rc = r == 1 ? run_fork_join<OzBody>(g, a, (int)Ml, fj_variant(sched), st, launches, e0, o.timeout_s)
                        : fp64tc_launch_blocks(g, a, nullptr, (int)Ml, fj_variant(sched), o, st, launches, e0);
        }
    }
    cudaFreeAsync(ws, st);
    return rc;
}

// ------------------------------------------------------------------ test hook
__global__ void __launch_bounds__(256) oz_split_kernel(const double *T, __nv_bfloat16 *slices, int32_t *rexp) {
    ozaki_split(T + (size_t)blockIdx.x * kOzNb * kOzNb, slices + (size_t)blockIdx.x * kOzS * kOzNb * kOzNb,
                rexp + blockIdx.x * kOzNb);
}

struct OzTestArgs {
    CUtensorMap mapA, mapB;
    double *C;
    const int32_t *rexp;
    int32_t *ok;
};

__global__ void __launch_bounds__(kOzThreads) oz_test_kernel(const __grid_constant__ OzTestArgs g) {
    extern __shared__ uint8_t dyn[];
    OzSmem &sm = *reinterpret_cast<OzSmem *>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
    oz_cta_init(sm.os);
    bool ok = true;
    // two updates in a row (C[0], C[1]) exercise the barrier phases across tasks
    for (int rep = 0; rep < 2 && ok; ++rep)
        ok = ozaki_tile_update(sm, &g.mapA, &g.mapB, g.C + (size_t)rep * kOzNb * kOzNb, 0, kOzS * kOzNb, g.rexp,
                               g.rexp + kOzNb, 2000000000ull);
    if (threadIdx.x == 0) *g.ok = ok ? 1 : 0;
    oz_cta_fini(sm.os);
}

}  // namespace chol

using namespace chol;

extern "C" {

int chol_test_ozaki_update(const double *A, const double *B, double *C) {
    CHOL_CHECK_ARG(A && B && C, "NULL pointer");
    const size_t tile = (size_t)kOzNb * kOzNb;
    double *T = nullptr;
    __nv_bfloat16 *sl = nullptr;
    int32_t *rexp = nullptr, *dok = nullptr;
    CHOL_CUDA(cudaMalloc(&T, 2 * tile * 8));
    CHOL_CUDA(cudaMalloc(&sl, 2 * kOzS * tile * 2));
    CHOL_CUDA(cudaMalloc(&rexp, 2 * kOzNb * 4 + 16));
    dok = rexp + 2 * kOzNb;
    CHOL_CUDA(cudaMemcpy(T, A, tile * 8, cudaMemcpyDeviceToDevice));
    CHOL_CUDA(cudaMemcpy(T + tile, B, tile * 8, cudaMemcpyDeviceToDevice));
    oz_split_kernel<<<2, 256>>>(T, sl, rexp);
    OzTestArgs g;
    memset(&g, 0, sizeof(g));
    int rc = make_slice_map(&g.mapA, sl, 2 * kOzS * kOzNb, 128);
    if (rc == CHOL_OK) rc = make_slice_map(&g.mapB, sl, 2 * kOzS * kOzNb, kOzQ);
    if (rc == CHOL_OK) {
        g.C = C;
        g.rexp = rexp;
        g.ok = dok;
        const size_t smem = sizeof(OzSmem) + 1024;
        CHOL_CUDA(cudaFuncSetAttribute(oz_test_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        oz_test_kernel<<<1, kOzThreads, smem>>>(g);
        int32_t ok = 0;
        const cudaError_t e = cudaMemcpy(&ok, dok, 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "ozaki test", __FILE__, __LINE__);
        else if (!ok) {
            set_error("ozaki tile update: wait expired");
            rc = CHOL_ERR_TIMEOUT;
        }
    }
    cudaFree(T);
    cudaFree(sl);
    cudaFree(rexp);
    return rc;
}

}  // extern "C"
