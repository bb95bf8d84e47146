// mixed.cu -- mixed-precision tiled Cholesky with FP64 iterative refinement.
//
// The tiles are kept in binary32.  POTRF of each diagonal tile runs in
// binary64 on its 128 x 128 diagonal blocks (each block widened, factored in
// shared memory, rounded back; for tile orders above 128 the blocks below
// and right of it are solved and updated in binary32 in between), TRSM in
// binary32 on the CUDA cores, and its epilogue writes the tensor-core operand copies of
// the panel tile: bf16 / fp16 after an exact power-of-two scaling that puts
// the tile's largest magnitude in [2^14, 2^15), or tf32-rounded values (hi,
// and lo = tf32(x - hi) for the 3-product FP32 mode).  SYRK and GEMM run on
// tcgen05 with binary32 accumulation in tensor memory (tc_gemm.cuh).  Both
// schedules of Section 3.2 run these bodies unchanged.
//
// Solves refine in FP64: r = b - A x with the caller's FP64 A, stop when the
// normwise backward error reaches the tolerance, else correct x += d with
// L^ L^T d = r solved in binary32 on the tile store.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "factor_impl.cuh"
#include "solve_impl.cuh"
#include "mixed_body.cuh"

namespace chol {

// ------------------------------------------------------------------ tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// 2-D map over `rows` rows of nb elements (row pitch nb * elem bytes), boxes of
// 128 bytes of K x box_rows rows, 128-byte swizzle.
size_t ozr_a_bytes(int64_t n);
bool ozr_supported(int64_t n);
int ozr_prepare_a(const double *A, int64_t lda, int64_t n, void *abuf, cudaStream_t st);
size_t ozr_ws_bytes(int64_t n, int64_t nrhs, int num_ctas);
int ozr_residual(const void *abuf, int64_t n, const double *X, int64_t ldx, const double *B, int64_t ldb, double *R,
                 int64_t ldr, int64_t nrhs, void *ws, double timeout_s, cudaStream_t st);

int make_operand_map(CUtensorMap *map, void *base, int fmt, int64_t rows, int64_t nb, int box_rows) {
    auto enc = tensor_map_encoder();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return CHOL_ERR_CUDA;
    }
    const int eb = fmt == OP_TF32 ? 4 : 2;
    const CUtensorMapDataType dt = fmt == OP_TF32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : fmt == OP_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                    : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    cuuint64_t dims[2] = {(cuuint64_t)nb, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(nb * eb)};
    cuuint32_t box[2] = {(cuuint32_t)(128 / eb), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    memset(map, 0, sizeof(*map));
    CUresult r = enc(map, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return CHOL_ERR_CUDA;
    }
    return CHOL_OK;
}

static int op_fmt(int precision) {
    return precision == CHOL_BF16 ? OP_BF16 : precision == CHOL_FP16 ? OP_F16 : OP_TF32;
}

// ------------------------------------------------------------------ task bodies
struct MixedBody {
    using Args = MixedArgs;
    using Smem = MixedSmem;
    static constexpr bool kSolveTask = false;
    static constexpr int kCtasPerSm = 1;  // one CTA owns the SM's shared memory and tensor memory
    static constexpr int kBlock = kThreads;
    static constexpr size_t kSmemBytes = sizeof(MixedSmem);
    // In the dataflow kernel a SYRK/GEMM on tiles of order 128 leaves its
    // epilogue to the next tile update on this CTA (its accumulator is one of
    // two tensor-memory buffers) or to flush(); the task completes when that
    // epilogue has stored the tile.
    static constexpr bool kLag = true;
    static __device__ __forceinline__ bool lagging(Smem &sm) { return sm.ts.pend != 0; }
    static __device__ __forceinline__ bool absorbs(const Args &, int I, int K, int J) {
        const int type = task_type(I, K, J);
        return type == T_SYRK || type == T_GEMM;
    }
    struct Done {
        const Args &g;
        const SchedArgs &a;
        __device__ void operator()(uint64_t w, uint64_t t0) const {
            df_complete_lagged<MixedBody>(g, a, (int)(w >> 48), (int)((w >> 32) & 0xffff), (int)((w >> 16) & 0xffff),
                                          (int)(w & 0xffff), t0);
        }
    };
    static __device__ void flush(const Args &g, const SchedArgs &a, Smem &sm) {
        const bool ok = tc_flush(sm.ts, g.timeout_ns, Done{g, a});
        if (!ok && threadIdx.x == 0) {
            if (atomicCAS(&a.ctl->status, 0, (int32_t)CHOL_ERR_TIMEOUT) == 0) a.ctl->timeout_where = 3;
            st_release_s32(&a.ctl->abort, 1);
        }
    }
    static __device__ __forceinline__ void cta_init(const Args &, Smem &sm) { tc_cta_init(sm.ts); }
    static __device__ __forceinline__ void cta_fini(const Args &, Smem &sm) { tc_cta_fini(sm.ts); }
    static __device__ __forceinline__ int tiles(const Args &g, int) { return g.S.M; }
    static __device__ __forceinline__ int64_t task_base(const Args &, int) { return 0; }

    static __device__ void run(const Args &g, const SchedArgs &a, int m, int I, int K, int J, Smem &sm) {
        uint64_t t0 = 0;
        if (a.trace && threadIdx.x == 0) t0 = global_ns();
        const auto fail = [&a](int64_t col) {
            report_info(a.ctl, col);
            st_release_s32(&a.ctl->abort, 1);
        };
        const bool ok = mixed_task<false>(g, a, m, I, K, J, sm, g.S.base, 0, t0, Done{g, a}, fail);
        if (!ok && threadIdx.x == 0) {
            if (atomicCAS(&a.ctl->status, 0, (int32_t)CHOL_ERR_TIMEOUT) == 0) a.ctl->timeout_where = 3;
            st_release_s32(&a.ctl->abort, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0 && !sm.ts.pend) task_done_bookkeeping(a, task_type(I, K, J), m, I, K, J, t0);
    }
    static __device__ void solve(const Args &, const SchedArgs &, int, Smem &) {}
};

// ------------------------------------------------------------------ refinement kernels
// R = B - A X for symmetric A given by its lower triangle (column-major, lda):
// one CTA per (64-row block, 16-column slice), FP64.
__global__ void __launch_bounds__(256) residual_kernel(const double *A, int64_t lda, int64_t n, const double *X,
                                                       int64_t ldx, const double *B, int64_t ldb, double *R,
                                                       int64_t ldr, int64_t nrhs) {
    __shared__ double As[kSB][kSB + 1];
    __shared__ double Xs[kSB][kRC + 1];
    const int I = blockIdx.x, nblk = (int)((n + kSB - 1) / kSB);
    const int64_t c0 = (int64_t)blockIdx.y * kRC;
    const int c = threadIdx.x % kRC, rq = threadIdx.x / kRC;
    double acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = (int64_t)I * kSB + rq + 16 * q;
        acc[q] = (i < n && c0 + c < nrhs) ? B[(c0 + c) * ldb + i] : 0.0;
    }
    for (int J = 0; J < nblk; ++J) {
        // As[r][k] = Asym(I*64 + r, J*64 + k)
        for (int e = threadIdx.x; e < kSB * kSB; e += blockDim.x) {
            int r, k;
            if (J <= I) { r = e % kSB; k = e / kSB; }   // read lower block (I, J): rows contiguous
            else { k = e % kSB; r = e / kSB; }          // read lower block (J, I): its rows are our columns
            const int64_t i = (int64_t)I * kSB + r, j = (int64_t)J * kSB + k;
            double v = 0.0;
            if (i < n && j < n) v = i >= j ? A[j * lda + i] : A[i * lda + j];
            As[r][k] = v;
        }
        for (int e = threadIdx.x; e < kSB * kRC; e += blockDim.x) {
            const int k = e / kRC, cc = e % kRC;
            const int64_t j = (int64_t)J * kSB + k;
            Xs[k][cc] = (j < n && c0 + cc < nrhs) ? X[(c0 + cc) * ldx + j] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kSB; ++k) {
            const double xk = Xs[k][c];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(-As[rq + 16 * q][k], xk, acc[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = (int64_t)I * kSB + rq + 16 * q;
        if (i < n && c0 + c < nrhs) R[(c0 + c) * ldr + i] = acc[q];
    }
}

// ||A||_inf of the symmetric matrix: row sums of |A|, one thread per row.
// rows[i] = sum_j |A(i, j)| of the symmetric A given by its lower triangle
// (column-major, lda): the lower part of row i (j <= i) by thread i, the loads
// of a warp on consecutive rows of one column, then the part right of the
// diagonal, which is column i below it, by one warp per column (lanes on
// consecutive rows) in the second kernel.
__global__ void anorm_rows_kernel(const double *A, int64_t lda, int64_t n, double *rows) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int64_t j = 0; j <= i; ++j) s += fabs(A[j * lda + i]);  // lower part of row i
    rows[i] = s;
}
__global__ void anorm_cols_kernel(const double *A, int64_t lda, int64_t n, double *rows) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (i >= n) return;
    double s = 0.0;
    for (int64_t j = i + 1 + lane; j < n; j += 32) s += fabs(A[i * lda + j]);  // column i below the diagonal
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rows[i] += s;
}

// Column maxima of |R|, |X|, |B| (non-negative doubles, so their bit patterns
// order like the values): reduced over the warp, then the block (256
// threads), then one atomic per block and quantity.
__global__ void __launch_bounds__(256) colmax_kernel(const double *R, int64_t ldr, const double *X, int64_t ldx,
                                                     const double *B, int64_t ldb, int64_t n, int64_t nrhs,
                                                     unsigned long long *out) {
    __shared__ double red[3][8];
    const int64_t c = blockIdx.y;
    double m[3] = {0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        m[0] = fmax(m[0], fabs(R[c * ldr + i]));
        m[1] = fmax(m[1], fabs(X[c * ldx + i]));
        m[2] = fmax(m[2], fabs(B[c * ldb + i]));
    }
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        for (int o = 16; o > 0; o >>= 1) m[q] = fmax(m[q], __shfl_xor_sync(0xffffffffu, m[q], o));
        if (lane == 0) red[q][warp] = m[q];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) v = fmax(v, red[threadIdx.x][w]);
        atomicMax(out + 3 * c + threadIdx.x, (unsigned long long)__double_as_longlong(v));
    }
}

__global__ void to_f32_kernel(const double *R, int64_t ldr, float *D, int64_t n, int64_t nrhs) {
    const int64_t c = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        D[c * n + i] = (float)R[c * ldr + i];
}

__global__ void axpy_kernel(double *X, int64_t ldx, const float *D, int64_t n, int64_t nrhs) {
    const int64_t c = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        X[c * ldx + i] += (double)D[c * n + i];
}

__global__ void __launch_bounds__(256) max_kernel(const double *v, int64_t n, unsigned long long *out) {
    __shared__ double red[8];
    double m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, v[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x / 32); ++w) m = fmax(m, red[w]);
        atomicMax(out, (unsigned long long)__double_as_longlong(m));
    }
}

// ------------------------------------------------------------------ GMRES-based refinement helpers
// Column-wise operations on n x nrhs column-major FP64 blocks (leading
// dimension n).  The dot products reduce in a fixed order (per-block partial
// sums, then one thread per column), so results do not depend on timing.
constexpr int kDotParts = 128;

__global__ void cols_dot_partial(const double *U, const double *V, int64_t n, double *part) {
    const int64_t c = blockIdx.y, chunk = (n + kDotParts - 1) / kDotParts;
    const int64_t i0 = blockIdx.x * chunk, i1 = i0 + chunk < n ? i0 + chunk : n;
    double s = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s = fma(U[c * n + i], V[c * n + i], s);
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[c * kDotParts + blockIdx.x] = red[0];
}

// out[c] = sum of the partials (sqrt of it with take_sqrt)
__global__ void cols_dot_final(const double *part, int64_t nrhs, double *out, int take_sqrt) {
    const int64_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    double s = 0.0;
    for (int b = 0; b < kDotParts; ++b) s += part[c * kDotParts + b];
    out[c] = take_sqrt ? sqrt(s) : s;
}

// W[:, c] += sgn * coef[c] * V[:, c]
__global__ void cols_axpy(double *W, const double *V, const double *coef, double sgn, int64_t n, int64_t nrhs) {
    const int64_t c = blockIdx.y;
    const double a = sgn * coef[c];
    for (int64_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        W[c * n + i] = fma(a, V[c * n + i], W[c * n + i]);
}

// X[:, c] += coef[c] * V[:, c] for X with leading dimension ldx
__global__ void cols_axpy_ld(double *X, int64_t ldx, const double *V, const double *coef, int64_t n, int64_t nrhs) {
    const int64_t c = blockIdx.y;
    const double a = coef[c];
    for (int64_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        X[c * ldx + i] = fma(a, V[c * n + i], X[c * ldx + i]);
}

// V[:, c] = V[:, c] / nrm[c] (zero column when nrm[c] == 0)
__global__ void cols_normalize(double *V, const double *nrm, int64_t n, int64_t nrhs) {
    const int64_t c = blockIdx.y;
    const double r = nrm[c] > 0.0 ? 1.0 / nrm[c] : 0.0;
    for (int64_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        V[c * n + i] *= r;
}

// W = sgn * (double)D (binary32 solve result back to binary64)
__global__ void f32_to_f64_kernel(const float *D, double *W, double sgn, int64_t n, int64_t nrhs) {
    const int64_t c = blockIdx.y;
    for (int64_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        W[c * n + i] = sgn * (double)D[c * n + i];
}

}  // namespace chol

// ------------------------------------------------------------------ handle
struct chol_factor_s {
    int64_t n = 0, nb = 0, M = 0;
    const double *A = nullptr;  // caller's FP64 matrix (referenced)
    int64_t lda = 0;
    float *store = nullptr;     // binary32 factor tiles
    chol_opts opts{};
    double anorm = -1.0;        // ||A||_inf, computed on first solve
    int64_t info = 0;           // factorization info (> 0: broke down at that column)
    void *ozr_a = nullptr;      // slices of A for the tensor-core residual (built on first solve)
    bool ozr_tried = false;
};

// order from which the refinement residual runs on the tensor cores
constexpr int64_t kOzrMinN = 1024;

namespace chol {
// Device bytes a mixed handle of order n keeps for the tensor-core residual
// once it has solved (the slices of A), and the per-solve workspace of that
// residual; 0 where the binary64 CUDA-core residual is used.  (The serving
// layer's memory budget.)
size_t mixed_residual_keep_bytes(int64_t n) { return n >= kOzrMinN && ozr_supported(n) ? ozr_a_bytes(n) : 0; }
size_t mixed_residual_ws_bytes(int64_t n, int64_t nrhs) {
    return n >= kOzrMinN && ozr_supported(n) ? (ozr_ws_bytes(n, nrhs, num_sms()) + 255) / 256 * 256 : 0;
}
}  // namespace chol

namespace chol {

// Residual R = B - A X of the refinement (B null: R = -A X): on the tensor
// cores with binary64 accuracy (ozres.cu) when the handle holds the slices of
// A, else by the binary64 CUDA-core kernel (zero: an n x nrhs zero block for
// its B operand).
struct ResidualOp {
    chol_factor_s *h;
    void *ozws;
    const double *zero;
    cudaStream_t st;
    int operator()(const double *X, int64_t ldx, const double *B, int64_t ldb, double *R, int64_t nrhs) const {
        const int64_t n = h->n;
        if (h->ozr_a) return ozr_residual(h->ozr_a, n, X, ldx, B, ldb, R, n, nrhs, ozws, h->opts.timeout_s, st);
        const int nblk = (int)((n + kSB - 1) / kSB), ny = (int)((nrhs + kRC - 1) / kRC);
        residual_kernel<<<dim3(nblk, ny), 256, 0, st>>>(h->A, h->lda, n, X, ldx, B ? B : zero, B ? ldb : n, R, n,
                                                         nrhs);
        return CHOL_OK;
    }
};

}  // namespace chol

using namespace chol;

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

static int mixed_factor_impl(int64_t n, const double *A, int64_t lda, const chol_opts &o, chol_factor_s *h,
                             int64_t *info, chol_stats *stats) {
    const int64_t nb = o.nb > 0 ? o.nb : chol_default_nb(n, o.precision);
    CHOL_CHECK_ARG(nb >= 128 && nb <= 1024 && nb % 128 == 0, "mixed precision needs nb in {128, 256, ..., 1024}");
    const int64_t M = (n + nb - 1) / nb;
    CHOL_CHECK_ARG(M < 65536 && num_tiles(M) * nb < (1ll << 31), "matrix too large for the operand maps");
    const int sched = o.schedule == CHOL_SCHED_AUTO ? CHOL_SCHED_DATAFLOW : o.schedule;
    CHOL_CHECK_ARG(sched >= CHOL_SCHED_FORK_JOIN && sched <= CHOL_SCHED_TOP_LOOKING, "unknown schedule");
    cudaStream_t st = (cudaStream_t)o.stream;
    prepare_pool();
    const int fmt = op_fmt(o.precision);
    const int64_t tiles = num_tiles(M);
    const size_t tile_elems = (size_t)nb * nb;
    const int grid = df_grid<MixedBody>(o.num_ctas);
    const int64_t ntasks = num_tasks(M);

    const size_t b_store = a256(tiles * tile_elems * 4);
    const size_t b_hi = a256(tiles * tile_elems * (fmt == OP_TF32 ? 4 : 2));
    const size_t b_lo = o.precision == CHOL_FP32 ? a256(tiles * tile_elems * 4) : 0;
    const size_t b_exp = a256(tiles * 4);
    const size_t b_ctl = a256(sizeof(Control));
    const size_t b_q = sched == CHOL_SCHED_DATAFLOW ? a256((size_t)2 * ntasks * 8) : 0;
    const size_t b_d = sched == CHOL_SCHED_DATAFLOW ? a256((size_t)ntasks * 4) : 0;

    float *store = nullptr;
    void *ws = nullptr;
    CHOL_CUDA(cudaMallocAsync((void **)&store, b_store, st));
    if (cudaMallocAsync(&ws, b_hi + b_lo + b_exp + b_ctl + b_q + b_d, st) != cudaSuccess) {
        cudaFreeAsync(store, st);
        set_error("device allocation of the mixed-precision workspace failed");
        return CHOL_ERR_NOMEM;
    }
    char *p = (char *)ws;
    MixedArgs g;
    memset(&g, 0, sizeof(g));
    g.S = TileStore<float>{store, (int32_t)nb, (int32_t)M};
    g.op_hi = p;
    g.op_lo = b_lo ? (float *)(p + b_hi) : nullptr;
    g.exps = (int32_t *)(p + b_hi + b_lo);
    Control *ctl = (Control *)(p + b_hi + b_lo + b_exp);
    unsigned long long *queue = (unsigned long long *)(p + b_hi + b_lo + b_exp + b_ctl);
    int32_t *deps = (int32_t *)(p + b_hi + b_lo + b_exp + b_ctl + b_q);
    g.precision = o.precision;
    g.fmt = fmt;
    g.timeout_ns = (uint64_t)(o.timeout_s * 1e9);

    int rc = make_operand_map(&g.map_hi, g.op_hi, fmt, tiles * nb, nb, kBoxRows);
    if (rc == CHOL_OK) rc = make_operand_map(&g.map_lo, g.op_lo ? (void *)g.op_lo : g.op_hi, fmt, tiles * nb, nb, kBoxRows);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Control hc{};
    int launches = 0;
    if (rc == CHOL_OK) do {
        if ((rc = launch_repack<double, float>(A, lda, n, store, (int)nb, M, st)) != CHOL_OK) break;
        if (cudaMemsetAsync(ctl, 0, sizeof(Control), st) != cudaSuccess ||
            cudaMemsetAsync(g.exps, 0, tiles * 4, st) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__);
            break;
        }
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "event", __FILE__, __LINE__);
            break;
        }
        SchedArgs a{ctl, o.trace, o.trace_capacity, o.flags, 0};
        if (sched == CHOL_SCHED_DATAFLOW) {
            DFArgs d{};
            d.queue = queue;
            d.deps = deps;
            d.capacity = ntasks;
            d.total = ntasks;
            d.num_matrices = 1;
            chol_opts oo = o;
            oo.num_ctas = grid;
            rc = launch_dataflow<MixedBody>(g, a, d, oo, st, &launches, e0);
        } else {
            rc = run_fork_join<MixedBody>(g, a, (int)M, fj_variant(sched), st, &launches, e0, o.timeout_s);
        }
        if (rc != CHOL_OK) break;
        cudaEventRecord(e1, st);
        if (cudaMemcpyAsync(&hc, ctl, sizeof(Control), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "mixed factor", __FILE__, __LINE__);
            break;
        }
    } while (0);
    cudaFreeAsync(ws, st);
    if (rc == CHOL_OK && hc.status) {
        set_error("mixed factorization: device-side wait expired (site %d)", hc.timeout_where);
        rc = hc.status;
    }
    if (rc != CHOL_OK) {
        cudaFreeAsync(store, st);
    } else {
        *info = hc.info;
        h->info = hc.info;
        h->n = n;
        h->nb = nb;
        h->M = M;
        h->A = A;
        h->lda = lda;
        h->store = store;
        h->opts = o;
        if (stats) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            for (int i = 0; i < 4; ++i) stats->tasks[i] = (int64_t)hc.tasks[i];
            stats->nb = nb;
            stats->schedule = sched;
            stats->launches = launches;
            stats->trace_records = (int64_t)hc.trace_count;
            stats->device_ms = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

// ------------------------------------------------------------------ GMRES-based refinement
// One correction X += d with d ~ A^{-1} R, by GMRES(m) on the left-
// preconditioned system M^{-1} A d = M^{-1} R, M = L^ L^T the binary32 factor
// (Carson and Higham's GMRES-IR): Arnoldi with modified Gram-Schmidt in
// binary64, A v in binary64, M^{-1} by the binary32 triangular solves, Givens
// rotations per right-hand side on the host.  The inner iteration stops when
// every column's preconditioned residual has dropped by rtol, or after m
// steps.  *napply counts the preconditioner applications.
struct GmresWs {
    double *V;      // (m + 1) blocks of n x nrhs
    double *zero;   // n x nrhs zeros (right-hand side of the A v product)
    double *U;      // n x nrhs
    float *D;       // n x nrhs, binary32 solves
    double *part;   // nrhs x kDotParts partial dot products
    double *hcol;   // (m + 2) x nrhs Hessenberg column / coefficients
    void *sws;      // solve workspace
};

constexpr int kGmresMaxM = 32;

static int gmres_correction(chol_factor_s *h, const double *R, double *X, int64_t ldx, int64_t nrhs, const GmresWs &w,
                            const ResidualOp &resid, cudaStream_t st, int m, double rtol, int *napply) {
    const int64_t n = h->n;
    const chol_opts &o = h->opts;
    if (m > kGmresMaxM) m = kGmresMaxM;
    const int nblk = (int)((n + kSB - 1) / kSB), ny = (int)((nrhs + kRC - 1) / kRC);
    const unsigned gx = (unsigned)((n + 255) / 256 < 512 ? (n + 255) / 256 : 512);
    const dim3 vg(gx, (unsigned)nrhs), vgrid((unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), (unsigned)nrhs);
    const size_t blk = (size_t)n * nrhs;
    int rc = CHOL_OK;
    auto precond = [&](const double *Y, double *Out, double sgn) {
        to_f32_kernel<<<vgrid, 256, 0, st>>>(Y, n, w.D, n, nrhs);
        rc = launch_solve<float, TileMajorL<float>>(TileMajorL<float>{h->store, h->nb}, w.D, n, n, nrhs, w.sws,
                                                    o.timeout_s, st);
        f32_to_f64_kernel<<<vg, 256, 0, st>>>(w.D, Out, sgn, n, nrhs);
        ++*napply;
    };
    auto dot = [&](const double *Ap, const double *Bp, double *out, int take_sqrt) {
        cols_dot_partial<<<dim3(kDotParts, (unsigned)nrhs), 256, 0, st>>>(Ap, Bp, n, w.part);
        cols_dot_final<<<(unsigned)((nrhs + 127) / 128), 128, 0, st>>>(w.part, nrhs, out, take_sqrt);
    };
    std::vector<double> hc((size_t)(m + 2) * nrhs), beta(nrhs), g((size_t)(m + 1) * nrhs, 0.0);
    std::vector<double> Rm((size_t)(m + 1) * m * nrhs, 0.0), cs((size_t)m * nrhs), sn((size_t)m * nrhs);
    // v0 = M^{-1} r / ||M^{-1} r||
    precond(R, w.V, 1.0);
    if (rc != CHOL_OK) return rc;
    dot(w.V, w.V, w.hcol, 1);
    cols_normalize<<<vg, 256, 0, st>>>(w.V, w.hcol, n, nrhs);
    CHOL_CUDA(cudaMemcpyAsync(beta.data(), w.hcol, nrhs * 8, cudaMemcpyDeviceToHost, st));
    CHOL_CUDA(cudaStreamSynchronize(st));
    for (int64_t c = 0; c < nrhs; ++c) g[c] = beta[c];
    int kend = -1;
    for (int k = 0; k < m; ++k) {
        double *Vk = w.V + (size_t)k * blk, *Vk1 = w.V + (size_t)(k + 1) * blk;
        // Vk1 = M^{-1} A Vk (the residual kernel gives U = 0 - A Vk)
        rc = resid(Vk, n, nullptr, n, w.U, nrhs);
        if (rc != CHOL_OK) return rc;
        precond(w.U, Vk1, -1.0);
        if (rc != CHOL_OK) return rc;
        for (int j = 0; j <= k; ++j) {
            dot(Vk1, w.V + (size_t)j * blk, w.hcol + (size_t)j * nrhs, 0);
            cols_axpy<<<vg, 256, 0, st>>>(Vk1, w.V + (size_t)j * blk, w.hcol + (size_t)j * nrhs, -1.0, n, nrhs);
        }
        dot(Vk1, Vk1, w.hcol + (size_t)(k + 1) * nrhs, 1);
        cols_normalize<<<vg, 256, 0, st>>>(Vk1, w.hcol + (size_t)(k + 1) * nrhs, n, nrhs);
        CHOL_CUDA(cudaMemcpyAsync(hc.data(), w.hcol, (size_t)(k + 2) * nrhs * 8, cudaMemcpyDeviceToHost, st));
        CHOL_CUDA(cudaStreamSynchronize(st));
        double worst = 0.0;
        for (int64_t c = 0; c < nrhs; ++c) {
            double col[kGmresMaxM + 1];
            for (int j = 0; j <= k + 1; ++j) col[j] = hc[(size_t)j * nrhs + c];
            for (int j = 0; j < k; ++j) {  // previous rotations
                const double a = col[j], b = col[j + 1];
                col[j] = cs[j * nrhs + c] * a + sn[j * nrhs + c] * b;
                col[j + 1] = -sn[j * nrhs + c] * a + cs[j * nrhs + c] * b;
            }
            const double a = col[k], b = col[k + 1], r = hypot(a, b);
            const double cc = r > 0.0 ? a / r : 1.0, ss = r > 0.0 ? b / r : 0.0;
            cs[k * nrhs + c] = cc;
            sn[k * nrhs + c] = ss;
            col[k] = r;
            col[k + 1] = 0.0;
            for (int j = 0; j <= k; ++j) Rm[((size_t)j * m + k) * nrhs + c] = col[j];
            const double gk = g[(size_t)k * nrhs + c];
            g[(size_t)k * nrhs + c] = cc * gk;
            g[(size_t)(k + 1) * nrhs + c] = -ss * gk;
            const double rel = beta[c] > 0.0 ? fabs(g[(size_t)(k + 1) * nrhs + c]) / beta[c] : 0.0;
            worst = rel > worst ? rel : worst;
        }
        kend = k;
        if (!(worst > rtol)) break;  // also stops on a NaN
    }
    // y = R^{-1} g per column, X += sum_j y_j v_j
    std::vector<double> y((size_t)(kend + 1) * nrhs, 0.0);
    for (int64_t c = 0; c < nrhs; ++c)
        for (int j = kend; j >= 0; --j) {
            double v = g[(size_t)j * nrhs + c];
            for (int l = j + 1; l <= kend; ++l) v -= Rm[((size_t)j * m + l) * nrhs + c] * y[(size_t)l * nrhs + c];
            const double d = Rm[((size_t)j * m + j) * nrhs + c];
            y[(size_t)j * nrhs + c] = d != 0.0 ? v / d : 0.0;
        }
    CHOL_CUDA(cudaMemcpyAsync(w.hcol, y.data(), y.size() * 8, cudaMemcpyHostToDevice, st));
    for (int j = 0; j <= kend; ++j)
        cols_axpy_ld<<<vg, 256, 0, st>>>(X, ldx, w.V + (size_t)j * blk, w.hcol + (size_t)j * nrhs, n, nrhs);
    CHOL_CUDA(cudaStreamSynchronize(st));  // y lives on the host stack
    return rc;
}

static thread_local chol_stats g_mixed_stats;

extern "C" {

int chol_mixed_factor(int64_t n, const double *A, int64_t lda, const chol_opts *opts, chol_factor_h *out,
                      int64_t *info) {
    CHOL_CHECK_ARG(out != nullptr && info != nullptr, "out or info is NULL");
    *out = nullptr;
    *info = 0;
    CHOL_CHECK_ARG(n >= 1, "n < 1");
    CHOL_CHECK_ARG(lda >= n, "lda < n");
    CHOL_CHECK_ARG(A != nullptr, "A is NULL");
    chol_opts o = resolve_opts(opts);
    CHOL_CHECK_ARG(o.precision >= CHOL_FP32 && o.precision <= CHOL_FP16, "precision must be FP32, TF32, BF16 or FP16");
    cudaGetLastError();  // errors left by earlier, unrelated runtime calls are not ours to report
    chol_factor_s *h = new chol_factor_s();
    memset(&g_mixed_stats, 0, sizeof(g_mixed_stats));
    const int rc = mixed_factor_impl(n, A, lda, o, h, info, &g_mixed_stats);
    if (rc != CHOL_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return CHOL_OK;
}

// statistics of the last chol_mixed_factor on this thread
int chol_mixed_last_stats(chol_stats *st) {
    CHOL_CHECK_ARG(st != nullptr, "stats is NULL");
    *st = g_mixed_stats;
    return CHOL_OK;
}

int chol_mixed_get_factor(chol_factor_h h, double *L, int64_t ldl) {
    if (!h || !h->store) {
        set_error("invalid factor handle");
        return CHOL_ERR_HANDLE;
    }
    CHOL_CHECK_ARG(L != nullptr && ldl >= h->n, "L is NULL or ldl < n");
    cudaStream_t st = (cudaStream_t)h->opts.stream;
    int rc = launch_unpack<float, double>(h->store, (int)h->nb, h->M, L, ldl, h->n, st);
    if (rc != CHOL_OK) return rc;
    CHOL_CUDA(cudaStreamSynchronize(st));
    return CHOL_OK;
}

int chol_mixed_solve(chol_factor_h h, int64_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx,
                     int32_t *iters_out, double *berr_out) {
    if (!h || !h->store) {
        set_error("invalid factor handle");
        return CHOL_ERR_HANDLE;
    }
    const int64_t n = h->n;
    CHOL_CHECK_ARG(nrhs >= 1 && B && X && ldb >= n && ldx >= n, "bad B / X arguments");
    if (h->info > 0) {
        set_error("the factorization broke down at column %lld (not positive definite in this precision)",
                  (long long)h->info);
        return CHOL_ERR_NOT_SPD;
    }
    const chol_opts &o = h->opts;
    cudaStream_t st = (cudaStream_t)o.stream;
    prepare_pool();
    if (!h->ozr_tried) {
        // slices of A for the tensor-core residual, once per handle (A stays
        // unchanged while the handle lives); without the memory for them the
        // binary64 CUDA-core residual is used
        h->ozr_tried = true;
        if (n >= kOzrMinN && ozr_supported(n)) {
            if (cudaMallocAsync(&h->ozr_a, ozr_a_bytes(n), st) != cudaSuccess) {
                cudaGetLastError();
                h->ozr_a = nullptr;
            } else if (ozr_prepare_a(h->A, h->lda, n, h->ozr_a, st) != CHOL_OK) {
                cudaFreeAsync(h->ozr_a, st);
                h->ozr_a = nullptr;
                cudaGetLastError();
            }
        }
    }
    const size_t b_oz = h->ozr_a ? a256(ozr_ws_bytes(n, nrhs, num_sms())) : 0;
    const size_t b_r = a256((size_t)n * nrhs * 8), b_d = a256((size_t)n * nrhs * 4);
    const size_t b_max = a256((size_t)3 * nrhs * 8 + 8), b_rows = a256((size_t)n * 8);
    const size_t b_sws = a256(solve_ws_bytes(n, nrhs));
    const bool gmres = (o.flags & CHOL_FLAG_GMRES_IR) != 0;
    // GMRES(20); the inner iteration stops once the preconditioned residual has
    // dropped by max(1e-6, 0.1 tol / berr): below about 1e-6 the binary32
    // rounding of the preconditioner's input limits what one correction can
    // gain, and near the target a smaller reduction suffices.
    constexpr int kGmresM = 20;
    const size_t b_g = gmres ? (size_t)(kGmresM + 3) * b_r + a256((size_t)nrhs * kDotParts * 8) +
                                   a256((size_t)(kGmresM + 2) * nrhs * 8)
                             : 0;
    void *ws = nullptr;
    CHOL_CUDA(cudaMallocAsync(&ws, b_r + b_d + b_max + b_rows + b_sws + b_g + b_oz, st));
    char *p = (char *)ws;
    double *R = (double *)p;
    float *D = (float *)(p + b_r);
    unsigned long long *mx = (unsigned long long *)(p + b_r + b_d);
    double *rows = (double *)(p + b_r + b_d + b_max);
    void *sws = p + b_r + b_d + b_max + b_rows;
    GmresWs gw{};
    if (gmres) {
        char *q = p + b_r + b_d + b_max + b_rows + b_sws;
        gw.V = (double *)q;
        q += (size_t)(kGmresM + 1) * b_r;
        gw.zero = (double *)q;
        q += b_r;
        gw.U = (double *)q;
        q += b_r;
        gw.part = (double *)q;
        q += a256((size_t)nrhs * kDotParts * 8);
        gw.hcol = (double *)q;
        gw.D = D;
        gw.sws = sws;
    }
    void *ozws = b_oz ? (void *)(p + b_r + b_d + b_max + b_rows + b_sws + b_g) : nullptr;
    const ResidualOp resid{h, ozws, gw.zero, st};
    int napply = 0;
    const int nblk = (int)((n + kSB - 1) / kSB), ny = (int)((nrhs + kRC - 1) / kRC);
    const dim3 vgrid((unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), (unsigned)nrhs);
    int rc = CHOL_OK;
    std::vector<unsigned long long> hm(3 * nrhs + 1);
    int it = 0;
    double berr = 1.0;
    do {
        if (h->anorm < 0) {
            anorm_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(h->A, h->lda, n, rows);
            anorm_cols_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(h->A, h->lda, n, rows);
            if (cudaMemsetAsync(mx + 3 * nrhs, 0, 8, st) != cudaSuccess) { rc = CHOL_ERR_CUDA; break; }
            max_kernel<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, st>>>(rows, n, mx + 3 * nrhs);
            unsigned long long v = 0;
            if (cudaMemcpyAsync(&v, mx + 3 * nrhs, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = cuda_fail(cudaGetLastError(), "anorm", __FILE__, __LINE__);
                break;
            }
            memcpy(&h->anorm, &v, 8);
        }
        if (cudaMemset2DAsync(X, ldx * 8, 0, n * 8, nrhs, st) != cudaSuccess ||
            (gmres && cudaMemsetAsync(gw.zero, 0, b_r, st) != cudaSuccess)) {
            rc = cuda_fail(cudaGetLastError(), "zero X", __FILE__, __LINE__);
            break;
        }
        for (it = 0;; ++it) {
            // r = b - A x (FP64) and the backward error (x = 0 at the start: r = b)
            if (it == 0) {
                if (cudaMemcpy2DAsync(R, n * 8, B, ldb * 8, n * 8, nrhs, cudaMemcpyDeviceToDevice, st) !=
                    cudaSuccess) {
                    rc = cuda_fail(cudaGetLastError(), "refinement", __FILE__, __LINE__);
                    break;
                }
            } else {
                rc = resid(X, ldx, B, ldb, R, nrhs);
                if (rc != CHOL_OK) break;
            }
            if (cudaMemsetAsync(mx, 0, 3 * nrhs * 8, st) != cudaSuccess) { rc = CHOL_ERR_CUDA; break; }
            colmax_kernel<<<vgrid, 256, 0, st>>>(R, n, X, ldx, B, ldb, n, nrhs, mx);
            if (cudaMemcpyAsync(hm.data(), mx, 3 * nrhs * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = cuda_fail(cudaGetLastError(), "refinement", __FILE__, __LINE__);
                break;
            }
            berr = 0.0;
            bool finite = true;
            for (int64_t c = 0; c < nrhs; ++c) {
                double r, x, b;
                memcpy(&r, &hm[3 * c], 8);
                memcpy(&x, &hm[3 * c + 1], 8);
                memcpy(&b, &hm[3 * c + 2], 8);
                const double den = h->anorm * x + b;
                const double e = den > 0 ? r / den : r;
                if (!(e <= 1e300)) finite = false;  // NaN or Inf: the iterate is unusable
                else berr = e > berr ? e : berr;
            }
            if (!finite) berr = __builtin_nan("");
            if (berr <= o.refine_tol || it >= o.max_iter || !(berr == berr)) break;
            if (gmres) {
                const double rt = std::min(0.5, std::max(1e-6, 0.1 * o.refine_tol / berr));
                rc = gmres_correction(h, R, X, ldx, nrhs, gw, resid, st, kGmresM, rt, &napply);
                if (rc != CHOL_OK) break;
                continue;
            }
            // d = L^-T L^-1 r in binary32 on the tile store; x += d
            to_f32_kernel<<<vgrid, 256, 0, st>>>(R, n, D, n, nrhs);
            rc = launch_solve<float, TileMajorL<float>>(TileMajorL<float>{h->store, h->nb}, D, n, n, nrhs, sws,
                                                        o.timeout_s, st);
            if (rc != CHOL_OK) break;
            axpy_kernel<<<vgrid, 256, 0, st>>>(X, ldx, D, n, nrhs);
        }
        if (rc == CHOL_OK && cudaGetLastError() != cudaSuccess) rc = CHOL_ERR_CUDA;
        if (rc == CHOL_OK) {
            int32_t sst = 0, ost = 0;
            if (cudaMemcpyAsync(&sst, sws, 4, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                (!ozws || cudaMemcpyAsync(&ost, ozws, 4, cudaMemcpyDeviceToHost, st) == cudaSuccess) &&
                cudaStreamSynchronize(st) == cudaSuccess && (sst != 0 || ost != 0)) {
                set_error("refinement %s: device-side wait expired", sst ? "solve" : "residual");
                rc = sst ? sst : ost;
            }
        }
    } while (0);
    cudaFreeAsync(ws, st);
    if (iters_out) *iters_out = gmres ? napply : it;
    if (berr_out) *berr_out = berr;
    if (rc == CHOL_OK && !(berr <= o.refine_tol)) {
        set_error("refinement stopped at backward error %.3e after %d iterations", berr, it);
        rc = CHOL_ERR_NOT_CONVERGED;
    }
    return rc;
}

void chol_factor_free(chol_factor_h h) {
    if (!h) return;
    if (h->store) cudaFreeAsync(h->store, (cudaStream_t)h->opts.stream);
    if (h->ozr_a) cudaFreeAsync(h->ozr_a, (cudaStream_t)h->opts.stream);
    h->store = nullptr;
    h->ozr_a = nullptr;
    delete h;
}

}  // extern "C"

// ------------------------------------------------------------------ test hook: one tcgen05 tile update
namespace chol {

struct TcTestArgs {
    CUtensorMap map_hi;
    CUtensorMap map_lo;
    float *C;
    int32_t nb, precision, fmt, eA, eB, lower;
    int32_t *ok;
};

__global__ void __launch_bounds__(256) tc_test_kernel(const __grid_constant__ TcTestArgs g) {
    extern __shared__ uint8_t dyn[];
    MixedSmem &sm = *reinterpret_cast<MixedSmem *>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
    tc_cta_init(sm.ts);
    TcGemmArgs ga;
    const bool three = g.precision == CHOL_FP32;
    ga.passes = three ? 3 : 1;
    ga.tf32 = g.fmt == OP_TF32;
    for (int p = 0; p < 3; ++p) {
        ga.mapA[p] = (three && p == 2) ? &g.map_lo : &g.map_hi;
        ga.mapB[p] = (three && p == 1) ? &g.map_lo : &g.map_hi;
    }
    ga.idesc = make_idesc((uint32_t)g.fmt, 128, (uint32_t)tc_sub_cols(g.nb));
    // two updates in a row exercise the barrier phases across tasks
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep)
        ok = tc_tile_update(sm.ts, &sm.stages[0][0], ga, g.C + (size_t)rep * g.nb * g.nb, g.nb, 0, g.nb,
                            ldexpf(1.f, -g.eA), ldexpf(1.f, -g.eB), g.lower != 0, 2000000000ull);
    if (threadIdx.x == 0) *g.ok = ok ? 1 : 0;
    tc_cta_fini(sm.ts);
}

}  // namespace chol

extern "C" {

// C[0] and C[1] (two nb x nb FP32 tiles, row-major, contiguous) each receive
// C -= 2^-eA 2^-eB * sum_p A_p B_p^T with operands from `ops`: rows [0, nb) of
// each operand array are A, rows [nb, 2 nb) are B; `ops` holds the hi array
// and, for CHOL_FP32, the lo array right after it.  Returns CHOL_OK, or
// CHOL_ERR_TIMEOUT if a wait expired.
int chol_test_tc_update(int32_t precision, int64_t nb, const void *ops, int32_t eA, int32_t eB, float *C,
                        int32_t lower) {
    CHOL_CHECK_ARG(precision >= CHOL_FP32 && precision <= CHOL_FP16, "precision");
    CHOL_CHECK_ARG(nb >= 128 && nb <= 1024 && nb % 128 == 0, "nb");
    CHOL_CHECK_ARG(ops && C, "NULL pointer");
    TcTestArgs g;
    memset(&g, 0, sizeof(g));
    g.fmt = op_fmt(precision);
    const size_t eb = g.fmt == OP_TF32 ? 4 : 2;
    int rc = make_operand_map(&g.map_hi, (void *)ops, g.fmt, 2 * nb, nb, kBoxRows);
    if (rc == CHOL_OK && precision == CHOL_FP32)
        rc = make_operand_map(&g.map_lo, (char *)ops + 2 * nb * nb * eb, g.fmt, 2 * nb, nb, kBoxRows);
    else if (rc == CHOL_OK)
        g.map_lo = g.map_hi;
    if (rc != CHOL_OK) return rc;
    g.C = C;
    g.nb = (int32_t)nb;
    g.precision = precision;
    g.eA = eA;
    g.eB = eB;
    g.lower = lower;
    int32_t *dok = nullptr;
    CHOL_CUDA(cudaMalloc(&dok, 4));
    const size_t smem = sizeof(MixedSmem) + 1024;
    CHOL_CUDA(cudaFuncSetAttribute(tc_test_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    g.ok = dok;
    tc_test_kernel<<<1, 256, smem>>>(g);
    int32_t ok = 0;
    cudaError_t e = cudaMemcpy(&ok, dok, 4, cudaMemcpyDeviceToHost);
    cudaFree(dok);
    if (e != cudaSuccess) return cuda_fail(e, "tc test", __FILE__, __LINE__);
    if (!ok) {
        set_error("tcgen05 tile update: wait expired");
        return CHOL_ERR_TIMEOUT;
    }
    return CHOL_OK;
}

}  // extern "C"
