// ozres.cu -- the refinement residual R = B - A X in binary64 on the bf16
// tensor cores (the exact slicing of ozaki.cuh applied to a matrix times a
// block of vectors).
//
// Iterative refinement (Section 1's use of the factor: solving with it)
// needs R = B - A X in the working precision.  As a dot-product kernel on the
// CUDA cores it costs n^2 nrhs binary64 FMAs, and GB300's binary64 rate
// (about 1.2 TFLOP/s) makes that the largest part of a refinement step.
// Here A is split once per factor handle into 8 bf16 slices per 128 x 128
// tile (every tile of the full symmetric matrix, rows scaled per tile), X is
// split per call into slices per 128-row block and right-hand-side column,
// and the 36 slice products of each (tile, block) pair are accumulated
// exactly in FP32 tensor memory, combined exactly into two int64 values and
// added into binary64 registers.  The kernel streams the A slices once per
// call (256 KB per tile): HBM-bound, where the CUDA-core kernel was bound by
// binary64 arithmetic.
//
// Work: a persistent kernel over units (16-column chunk ch, row block I,
// column range jc); each unit sums A_IJ X_J over its J range into a partial
// result, and a second kernel forms R = B - sum of the partials in a fixed
// order (deterministic).  CTA roles: thread 0 issues the TMA loads (X slices
// of block J, then the 8 A slices of tile (I, J) through a ring of stages),
// thread 32 issues the MMAs (for A slice s one MMA of N = 16 (8 - s) covers
// the X slices t = 0 .. 7 - s, whose accumulators are the groups s + t),
// warps 4..7 run the epilogue (one row per thread, 16 columns), with the two
// halves of the 256 tensor-memory columns alternating between K-tiles.
// Every wait is bounded; on expiry the kernel records CHOL_ERR_TIMEOUT.
#include <cuda.h>
#include <string.h>

#include "common.cuh"
#include "ozaki.cuh"

namespace chol {

int make_operand_map(CUtensorMap *map, void *base, int fmt, int64_t rows, int64_t nb, int box_rows);

constexpr int kOzrCols = 16;                            // right-hand-side columns per chunk
constexpr int kOzrStages = 4;                           // A-slice ring
constexpr int kOzrABytes = 2 * kOzNb * 128;             // one A slice, both K-chunks of 64
constexpr int kOzrXChunk = kOzS * kOzrCols * 128;       // X slices of one K-chunk: 128 rows x 128 B
constexpr int kOzrThreads = 256;

struct OzrArgs {
    CUtensorMap mapA;      // A slices: rows ((I Mt + J) 8 + s) 128 + r, 128-row boxes
    CUtensorMap mapX;      // X slices: rows ((ch Mt + J) 8 + s) 16 + c, 128-row boxes
    const int32_t *expA;   // [(I Mt + J) 128 + r]
    const int32_t *expX;   // [(ch Mt + J) 16 + c]
    double *Rp;            // [((jc nch + ch) Mt 128 + i) 16 + c] partial sums of A X
    int32_t *status;
    int Mt, nJc, Lc, nch, units;
    uint64_t timeout_ns;
};

struct OzrSmem {
    uint8_t X[2][2][kOzrXChunk];            // 64 KB: buffer, K-chunk
    uint8_t A[kOzrStages][kOzrABytes];      // 128 KB
    uint64_t full[kOzrStages], empty[kOzrStages], xfull[2], xfree[2], acc_full[2], tmem_empty[2], drain;
    uint32_t tmem_base;
    int32_t fail;
};

// ------------------------------------------------------------------ splitting
// Slices of every tile (I, J) of the symmetric A, given by its lower triangle
// (column-major, lda): element (r, c) of tile (I, J) is A(I 128 + r, J 128 + c),
// zero beyond n.  One CTA per half tile (64 rows), staged through shared
// memory so that both triangles are read along their contiguous direction.
__global__ void __launch_bounds__(256) ozr_split_a_kernel(const double *A, int64_t lda, int64_t n, int Mt,
                                                          __nv_bfloat16 *slices, int32_t *expA) {
    extern __shared__ double T[];  // [64][129]
    constexpr int P = kOzNb + 1;
    const int64_t t = blockIdx.x >> 1;
    const int hb = blockIdx.x & 1;
    const int64_t I = t / Mt, J = t % Mt;
    const int64_t r0 = I * kOzNb + hb * 64, c0 = J * kOzNb;
    for (int e = threadIdx.x; e < 64 * kOzNb; e += blockDim.x) {
        int r, c;
        if (J > I) { c = e % kOzNb; r = e / kOzNb; }  // upper tile: A(gj, gi) is contiguous along c
        else { r = e % 64; c = e / 64; }             // lower (and diagonal) tile: contiguous along r
        const int64_t gi = r0 + r, gj = c0 + c;
        double v = 0.0;
        if (gi < n && gj < n) v = gi >= gj ? __ldcs(A + gj * lda + gi) : __ldcs(A + gi * lda + gj);
        T[r * P + c] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    uint16_t *out = reinterpret_cast<uint16_t *>(slices) + (size_t)t * kOzS * kOzNb * kOzNb;
    for (int r = warp; r < 64; r += 8) {
        double v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = T[r * P + oz_col(lane, q)];
        const int row = hb * 64 + r;
        const int e = ozaki_split_row(v, out + (size_t)row * kOzNb, (size_t)kOzNb * kOzNb, false);
        if (lane == 0) expA[t * kOzNb + row] = e;
    }
}

// Slices of X (n x nrhs, column-major): for column chunk ch, row block J and
// column c one warp splits the 128 values X(J 128 + k, 16 ch + c) (zero beyond
// n or nrhs) into rows ((ch Mt + J) 8 + s) 16 + c of the slice store.
__global__ void __launch_bounds__(256) ozr_split_x_kernel(const double *X, int64_t ldx, int64_t n, int64_t nrhs,
                                                          int Mt, int nch, __nv_bfloat16 *slices, int32_t *expX) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (w >= (int64_t)nch * Mt * kOzrCols) return;
    const int c = (int)(w % kOzrCols);
    const int64_t chJ = w / kOzrCols;  // ch Mt + J
    const int64_t J = chJ % Mt, ch = chJ / Mt;
    const int64_t col = ch * kOzrCols + c;
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = J * kOzNb + oz_col(lane, q);
        v[q] = (col < nrhs && i < n) ? X[col * ldx + i] : 0.0;
    }
    uint16_t *out = reinterpret_cast<uint16_t *>(slices) + ((size_t)chJ * kOzS * kOzrCols + c) * kOzNb;
    const int e = ozaki_split_row(v, out, (size_t)kOzrCols * kOzNb, false);
    if (lane == 0) expX[chJ * kOzrCols + c] = e;
}

// ------------------------------------------------------------------ product
__device__ __forceinline__ void ozr_fail(OzrSmem &sm, const OzrArgs &g) {
    *(volatile int32_t *)&sm.fail = 1;
    atomicCAS(g.status, 0, (int32_t)CHOL_ERR_TIMEOUT);
}
__device__ __forceinline__ bool ozr_failed(OzrSmem &sm) { return *(volatile int32_t *)&sm.fail != 0; }

__device__ __forceinline__ void ozr_unit(const OzrArgs &g, int u, int &ch, int &I, int &J0, int &J1, int &jc) {
    ch = u / (g.Mt * g.nJc);
    const int rem = u % (g.Mt * g.nJc);
    I = rem / g.nJc;
    jc = rem % g.nJc;
    J0 = jc * g.Lc;
    J1 = J0 + g.Lc < g.Mt ? J0 + g.Lc : g.Mt;
}

__global__ void __launch_bounds__(kOzrThreads, 1) ozr_product_kernel(const __grid_constant__ OzrArgs g) {
    extern __shared__ uint8_t dyn[];
    OzrSmem &sm = *reinterpret_cast<OzrSmem *>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kOzrStages; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sm.xfull[b], 1);
            mbar_init(&sm.xfree[b], 1);
            mbar_init(&sm.acc_full[b], 1);
            mbar_init(&sm.tmem_empty[b], 4);
        }
        mbar_init(&sm.drain, 1);
        sm.fail = 0;
        mbar_fence_init();
    }
    if (warp == 1) {
        tmem_alloc(&sm.tmem_base, 256);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint64_t deadline = global_ns() + g.timeout_ns;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        uint32_t f = 0, kt = 0;
        for (int u = blockIdx.x; u < g.units && !ozr_failed(sm); u += gridDim.x) {
            int ch, I, J0, J1, jc;
            ozr_unit(g, u, ch, I, J0, J1, jc);
            for (int J = J0; J < J1 && !ozr_failed(sm); ++J, ++kt) {
                const uint32_t b = kt & 1;
                if (kt >= 2 && !mbar_wait(&sm.xfree[b], ((kt >> 1) - 1) & 1, deadline)) {
                    ozr_fail(sm, g);
                    break;
                }
                mbar_arrive_expect_tx(&sm.xfull[b], 2 * kOzrXChunk);
                for (int kc = 0; kc < 2; ++kc)
                    tma_load_2d(smem_u32(sm.X[b][kc]), &g.mapX, &sm.xfull[b], kc * 64, (ch * g.Mt + J) * kOzS * kOzrCols);
                const int arow = ((I * g.Mt + J) * kOzS) * kOzNb;
                for (int s = 0; s < kOzS; ++s, ++f) {
                    const int st = (int)(f % kOzrStages);
                    if (f >= (uint32_t)kOzrStages &&
                        !mbar_wait(&sm.empty[st], ((f / kOzrStages) & 1) ^ 1, deadline)) {
                        ozr_fail(sm, g);
                        break;
                    }
                    mbar_arrive_expect_tx(&sm.full[st], kOzrABytes);
                    for (int kc = 0; kc < 2; ++kc)
                        tma_load_2d(smem_u32(sm.A[st]) + kc * (kOzrABytes / 2), &g.mapA, &sm.full[st], kc * 64,
                                    arow + s * kOzNb);
                }
            }
        }
        // copies still in flight land before the CTA exits: wait for the last
        // fill of every stage and X buffer (already complete unless a wait failed)
        for (uint32_t k = 0; k < kOzrStages && k < f; ++k) {
            const uint32_t last = f - 1 - k;
            mbar_wait(&sm.full[last % kOzrStages], (last / kOzrStages) & 1, global_ns() + 1000000000ull);
        }
        for (uint32_t k = 0; k < 2 && k < kt; ++k) {
            const uint32_t last = kt - 1 - k;
            mbar_wait(&sm.xfull[last & 1], (last >> 1) & 1, global_ns() + 1000000000ull);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        constexpr uint32_t kIdescN[kOzS + 1] = {
            0u, make_idesc(OP_BF16, 128, 16), make_idesc(OP_BF16, 128, 32), make_idesc(OP_BF16, 128, 48),
            make_idesc(OP_BF16, 128, 64), make_idesc(OP_BF16, 128, 80), make_idesc(OP_BF16, 128, 96),
            make_idesc(OP_BF16, 128, 112), make_idesc(OP_BF16, 128, 128)};
        uint32_t f = 0, kt = 0;
        for (int u = blockIdx.x; u < g.units && !ozr_failed(sm); u += gridDim.x) {
            int ch, I, J0, J1, jc;
            ozr_unit(g, u, ch, I, J0, J1, jc);
            for (int J = J0; J < J1 && !ozr_failed(sm); ++J, ++kt) {
                const uint32_t b = kt & 1;
                if (!mbar_wait(&sm.xfull[b], (kt >> 1) & 1, deadline)) {
                    ozr_fail(sm, g);
                    break;
                }
                if (kt >= 2 && !mbar_wait(&sm.tmem_empty[b], ((kt >> 1) - 1) & 1, deadline)) {
                    ozr_fail(sm, g);
                    break;
                }
                tc_fence_after();
                const uint64_t xdesc[2] = {sdesc_sw128(smem_u32(sm.X[b][0])), sdesc_sw128(smem_u32(sm.X[b][1]))};
                const uint32_t dbase = sm.tmem_base + b * (uint32_t)(kOzS * kOzrCols);
                for (int s = 0; s < kOzS; ++s, ++f) {
                    const int st = (int)(f % kOzrStages);
                    if (!mbar_wait(&sm.full[st], (f / kOzrStages) & 1, deadline)) {
                        ozr_fail(sm, g);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = dbase + (uint32_t)(s * kOzrCols);
#pragma unroll
                    for (int kc = 0; kc < 2; ++kc) {
                        const uint64_t adesc = sdesc_sw128(smem_u32(sm.A[st]) + kc * (kOzrABytes / 2));
#pragma unroll
                        for (int k4 = 0; k4 < 4; ++k4)
                            tc_mma<false>(d, adesc + 2 * k4, xdesc[kc] + 2 * k4, kIdescN[kOzS - s],
                                          (s == 0 && kc == 0 && k4 == 0) ? 0u : 1u);
                    }
                    tc_commit(&sm.empty[st]);
                }
                tc_commit(&sm.acc_full[b]);
                tc_commit(&sm.xfree[b]);
            }
        }
    } else if (warp >= 4) {
        // ---------------- epilogue: one row per thread, 16 columns
        const int q = warp & 3, row = q * 32 + lane;
        double acc[kOzrCols];
#pragma unroll
        for (int c = 0; c < kOzrCols; ++c) acc[c] = 0.0;
        uint32_t kt = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
            int ch, I, J0, J1, jc;
            ozr_unit(g, u, ch, I, J0, J1, jc);
            for (int J = J0; J < J1 && ok; ++J, ++kt) {
                const uint32_t b = kt & 1;
                bool got = true;
                if (lane == 0) got = mbar_wait(&sm.acc_full[b], (kt >> 1) & 1, deadline);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    if (lane == 0) ozr_fail(sm, g);
                    ok = false;
                    break;
                }
                tc_fence_after();
                // groups g = s + t (d = g + 2) at columns 16 g of this half; the
                // same exact int64 combination as the tile update (ozaki.cuh)
                long long hi[kOzrCols], lo[kOzrCols];
                const uint32_t tb = sm.tmem_base + ((uint32_t)(q * 32) << 16) + b * (uint32_t)(kOzS * kOzrCols);
#pragma unroll
                for (int half4 = 0; half4 < 2; ++half4) {
                    uint32_t r0[16], r1[16], r2[16], r3[16];
                    const int gg = half4 * 4;
                    tmem_ld16(tb + (uint32_t)(gg * kOzrCols), r0);
                    tmem_ld16(tb + (uint32_t)((gg + 1) * kOzrCols), r1);
                    tmem_ld16(tb + (uint32_t)((gg + 2) * kOzrCols), r2);
                    tmem_ld16(tb + (uint32_t)((gg + 3) * kOzrCols), r3);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < kOzrCols; ++j) {
                        const int32_t t01 =
                            __float2int_rn(__uint_as_float(r0[j])) * 128 + __float2int_rn(__uint_as_float(r1[j]));
                        const int32_t t23 =
                            __float2int_rn(__uint_as_float(r2[j])) * 128 + __float2int_rn(__uint_as_float(r3[j]));
                        const long long w = ((long long)t01 << 14) + (long long)t23;
                        if (half4 == 0) hi[j] = w;
                        else lo[j] = w;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.tmem_empty[b]);
                const int ea = __ldg(g.expA + ((size_t)I * g.Mt + J) * kOzNb + row);
                const int32_t *eb = g.expX + ((size_t)ch * g.Mt + J) * kOzrCols;
#pragma unroll
                for (int j = 0; j < kOzrCols; ++j) {
                    const int e = ea + __ldg(eb + j);
                    acc[j] = (acc[j] + int_scaled(hi[j], e - 35)) + int_scaled(lo[j], e - 63);
                }
            }
            if (!ok) break;
            double *dst = g.Rp + (((size_t)jc * g.nch + ch) * g.Mt * kOzNb + (size_t)I * kOzNb + row) * kOzrCols;
#pragma unroll
            for (int j = 0; j < kOzrCols; j += 2) {
                *reinterpret_cast<double2 *>(dst + j) = make_double2(acc[j], acc[j + 1]);
                acc[j] = 0.0;
                acc[j + 1] = 0.0;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 32) {
        tc_commit(&sm.drain);
        mbar_wait(&sm.drain, 0, global_ns() + 1000000000ull);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(sm.tmem_base, 256);
}

// R = B - sum over jc of the partials (B may be null: R = -A X).
__global__ void ozr_reduce_kernel(const double *Rp, int nJc, int nch, int Mt, const double *B, int64_t ldb,
                                  double *R, int64_t ldr, int64_t n, int64_t nrhs) {
    const int64_t c = blockIdx.y;
    const int64_t ch = c / kOzrCols, cc = c % kOzrCols;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int jc = 0; jc < nJc; ++jc) s += Rp[(((size_t)jc * nch + ch) * Mt * kOzNb + i) * kOzrCols + cc];
        R[c * ldr + i] = (B ? B[c * ldb + i] : 0.0) - s;
    }
}

// ------------------------------------------------------------------ host side
size_t ozr_a_bytes(int64_t n) {
    const int64_t Mt = (n + kOzNb - 1) / kOzNb;
    return ((size_t)Mt * Mt * kOzS * kOzNb * kOzNb * 2 + 255) / 256 * 256 + (size_t)Mt * Mt * kOzNb * 4;
}

bool ozr_supported(int64_t n) {
    const int64_t Mt = (n + kOzNb - 1) / kOzNb;
    return n > 0 && Mt * Mt * kOzS * kOzNb < (1ll << 31);
}

// Split A into the slice store `abuf` (ozr_a_bytes(n) bytes).
int ozr_prepare_a(const double *A, int64_t lda, int64_t n, void *abuf, cudaStream_t st) {
    CHOL_CHECK_ARG(ozr_supported(n), "matrix too large for the residual slice maps");
    const int Mt = (int)((n + kOzNb - 1) / kOzNb);
    __nv_bfloat16 *sl = (__nv_bfloat16 *)abuf;
    int32_t *ex = (int32_t *)((char *)abuf + ((size_t)Mt * Mt * kOzS * kOzNb * kOzNb * 2 + 255) / 256 * 256);
    const size_t smem = 64 * (kOzNb + 1) * sizeof(double);
    CHOL_CUDA(cudaFuncSetAttribute(ozr_split_a_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ozr_split_a_kernel<<<(unsigned)((int64_t)Mt * Mt * 2), 256, smem, st>>>(A, lda, n, Mt, sl, ex);
    CHOL_CUDA(cudaGetLastError());
    return CHOL_OK;
}

// Workspace of ozr_residual for (n, nrhs).
size_t ozr_ws_bytes(int64_t n, int64_t nrhs, int num_ctas) {
    const int64_t Mt = (n + kOzNb - 1) / kOzNb, nch = (nrhs + kOzrCols - 1) / kOzrCols;
    const int64_t target = 6 * (int64_t)num_ctas;  // units for load balance
    int64_t nJc = (target + Mt * nch - 1) / (Mt * nch);
    if (nJc < 1) nJc = 1;
    if (nJc > Mt) nJc = Mt;
    return 256 + ((size_t)nch * Mt * kOzS * kOzrCols * kOzNb * 2 + 255) / 256 * 256 +
           ((size_t)nch * Mt * kOzrCols * 4 + 255) / 256 * 256 + (size_t)nJc * nch * Mt * kOzNb * kOzrCols * 8;
}

// R = B - A X (B may be null: R = -A X) with A given by its slice store
// (ozr_prepare_a).  X, B, R: n x nrhs column-major, device.  Stream-ordered;
// the status word (first 4 bytes of ws) is CHOL_ERR_TIMEOUT if a wait expired.
int ozr_residual(const void *abuf, int64_t n, const double *X, int64_t ldx, const double *B, int64_t ldb, double *R,
                 int64_t ldr, int64_t nrhs, void *ws, double timeout_s, cudaStream_t st) {
    CHOL_CHECK_ARG(ozr_supported(n), "matrix too large for the residual slice maps");
    const int Mt = (int)((n + kOzNb - 1) / kOzNb);
    const int nch = (int)((nrhs + kOzrCols - 1) / kOzrCols);
    CHOL_CHECK_ARG((int64_t)nch * Mt * kOzS * kOzrCols < (1ll << 31) && nrhs <= 65535, "too many right-hand sides");
    const int sms = num_sms();
    const int64_t target = 6 * (int64_t)sms;
    int nJc = (int)((target + (int64_t)Mt * nch - 1) / ((int64_t)Mt * nch));
    if (nJc < 1) nJc = 1;
    if (nJc > Mt) nJc = Mt;
    const int Lc = (Mt + nJc - 1) / nJc;
    nJc = (Mt + Lc - 1) / Lc;
    OzrArgs g;
    memset(&g, 0, sizeof(g));
    char *p = (char *)ws;
    g.status = (int32_t *)p;
    p += 256;
    __nv_bfloat16 *xs = (__nv_bfloat16 *)p;
    p += ((size_t)nch * Mt * kOzS * kOzrCols * kOzNb * 2 + 255) / 256 * 256;
    int32_t *ex = (int32_t *)p;
    p += ((size_t)nch * Mt * kOzrCols * 4 + 255) / 256 * 256;
    g.Rp = (double *)p;
    g.expA = (const int32_t *)((const char *)abuf + ((size_t)Mt * Mt * kOzS * kOzNb * kOzNb * 2 + 255) / 256 * 256);
    g.expX = ex;
    g.Mt = Mt;
    g.nJc = nJc;
    g.Lc = Lc;
    g.nch = nch;
    g.units = nch * Mt * nJc;
    g.timeout_ns = (uint64_t)(timeout_s * 1e9);
    int rc = make_operand_map(&g.mapA, const_cast<void *>(abuf), OP_BF16, (int64_t)Mt * Mt * kOzS * kOzNb, kOzNb, 128);
    if (rc == CHOL_OK)
        rc = make_operand_map(&g.mapX, xs, OP_BF16, (int64_t)nch * Mt * kOzS * kOzrCols, kOzNb, kOzS * kOzrCols);
    if (rc != CHOL_OK) return rc;
    CHOL_CUDA(cudaMemsetAsync(g.status, 0, 4, st));
    const int64_t warps = (int64_t)nch * Mt * kOzrCols;
    ozr_split_x_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(X, ldx, n, nrhs, Mt, nch, xs, ex);
    const size_t smem = sizeof(OzrSmem) + 1024;
    CHOL_CUDA(cudaFuncSetAttribute(ozr_product_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = g.units < sms ? g.units : sms;
    ozr_product_kernel<<<grid, kOzrThreads, smem, st>>>(g);
    const unsigned gx = (unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    ozr_reduce_kernel<<<dim3(gx, (unsigned)nrhs), 256, 0, st>>>(g.Rp, nJc, nch, Mt, B, ldb, R, ldr, n, nrhs);
    CHOL_CUDA(cudaGetLastError());
    return CHOL_OK;
}

}  // namespace chol

using namespace chol;

extern "C" {

int chol_test_oz_residual(int64_t n, const double *A, int64_t lda, const double *X, int64_t ldx, const double *B,
                          int64_t ldb, double *R, int64_t ldr, int64_t nrhs) {
    CHOL_CHECK_ARG(n > 0 && nrhs > 0 && A && X && R, "bad argument");
    CHOL_CHECK_ARG(ldx >= n && ldr >= n && lda >= n && (!B || ldb >= n), "leading dimension < n");
    CHOL_CHECK_ARG(ozr_supported(n), "matrix too large");
    void *abuf = nullptr, *ws = nullptr;
    CHOL_CUDA(cudaMalloc(&abuf, ozr_a_bytes(n)));
    const size_t wb = ozr_ws_bytes(n, nrhs, num_sms());
    if (cudaMalloc(&ws, wb) != cudaSuccess) {
        cudaFree(abuf);
        return cuda_fail(cudaGetLastError(), "cudaMalloc", __FILE__, __LINE__);
    }
    int rc = ozr_prepare_a(A, lda, n, abuf, 0);
    if (rc == CHOL_OK) rc = ozr_residual(abuf, n, X, ldx, B, ldb, R, ldr, nrhs, ws, 10.0, 0);
    if (rc == CHOL_OK) {
        int32_t status = 0;
        const cudaError_t e = cudaMemcpy(&status, ws, 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "residual", __FILE__, __LINE__);
        else if (status) {
            set_error("residual: device-side wait expired");
            rc = status;
        }
    }
    cudaFree(abuf);
    cudaFree(ws);
    return rc;
}

}  // extern "C"
