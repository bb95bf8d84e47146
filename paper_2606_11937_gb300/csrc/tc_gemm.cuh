// tc_gemm.cuh -- SYRK/GEMM tile updates on the 5th-generation tensor cores
// (tcgen05) for the mixed-precision factorization:
//
//     C (FP32 tile, row-major nb x nb)  -=  scale * sum_p A_p B_p^T
//
// where A_p, B_p are low-precision copies (bf16, fp16 or tf32-rounded fp32)
// of two panel tiles A_IJ, A_KJ written by the TRSM epilogue, and p runs over
// one product (BF16, FP16, TF32) or three (FP32 = hi*hi + hi*lo + lo*hi).
//
// Operands are staged by TMA (cp.async.bulk.tensor, 128-byte swizzle, K-major)
// into a ring of shared-memory stages, one thread issues tcgen05.mma with the
// FP32 accumulator in tensor memory (M = 128 rows per MMA, N = min(nb, 256)),
// and four epilogue warps read the accumulator with tcgen05.ld and update C.
// Every mbarrier wait is bounded by a %globaltimer deadline; an expired wait
// raises the CTA's abort flag and the roles unwind.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace chol {

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for the completion of the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, uint64_t deadline) {
    while (!mbar_test(b, parity)) {
        if (global_ns() > deadline) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint64_t *bar, int32_t x,
                                            int32_t y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(dst), "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T ; kind f16 (bf16 / fp16 operands) or tf32
template <bool TF32>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    if (TF32)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
            : "memory");
}
// 32 TMEM lanes (one per thread of the warp) x 32 consecutive 32-bit columns
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes in 8-row (1024-byte) groups; the buffer is 1024-byte aligned.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulate, A/B format (0 fp16, 1 bf16, 2 tf32),
// both K-major, M x N.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// ------------------------------------------------------------------ configuration
constexpr int kTcStages = 3;
constexpr int kBoxRows = 128;              // rows per TMA box
constexpr int kBoxBytes = kBoxRows * 128;  // 128 bytes of K per row
constexpr int kStageBytes = 4 * kBoxBytes; // up to 2 A boxes + 2 B boxes (or A hi/lo + B hi/lo)
// The staging area (kTcStages x kStageBytes) is cut into ring slots of the
// size one K-chunk of the update needs: 3 slots of 4 boxes, or 6 of 2 boxes
// (tile order 128, one product), so more loads are in flight.
constexpr int kTcMaxSlots = 6;

// Operand formats of the mixed precisions
enum OpFmt : int32_t { OP_F16 = 0, OP_BF16 = 1, OP_TF32 = 2 };

struct TcShared {
    uint64_t full[kTcMaxSlots];
    uint64_t empty[kTcMaxSlots];
    uint64_t acc_full[2];   // per accumulator buffer (two when a sub-tile takes <= 256 columns)
    uint64_t tmem_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    uint32_t ring;       // stage fills issued (== consumed) before the current task
    uint32_t acc_uses;   // accumulator uses completed before the current task
    uint32_t drains;     // drain barrier completions
    int32_t fail;        // an mbarrier wait expired in this CTA
    // a single-sub-tile update whose epilogue was deferred (tc_tile_update with
    // defer_last) to the next call or to tc_flush
    int32_t pend;
    uint32_t pend_u;     // its accumulator use
    float *pend_C;
    float pend_sa, pend_sb;
    int32_t pend_nb, pend_ri, pend_ci;  // the tile's order and the sub-tile's position
    uint64_t pend_task, pend_t0;
};

struct TcGemmArgs {
    const CUtensorMap *mapA[3];  // per product p: map of the A operand
    const CUtensorMap *mapB[3];
    int32_t passes;              // products per update (1 or 3)
    int32_t tf32;                // kind::tf32 (else kind::f16)
    uint32_t idesc;
};

// One CTA (256 threads) initialises its barriers and allocates 512 TMEM columns.
__device__ inline void tc_cta_init(TcShared &ts) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcMaxSlots; ++s) {
            mbar_init(&ts.full[s], 1);
            mbar_init(&ts.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ts.acc_full[b], 1);
            mbar_init(&ts.tmem_empty[b], 4);
        }
        mbar_init(&ts.drain, 1);
        ts.ring = 0;
        ts.acc_uses = 0;
        ts.drains = 0;
        ts.fail = 0;
        ts.pend = 0;
        mbar_fence_init();
    }
    if (threadIdx.x / 32 == 1) {
        tmem_alloc(&ts.tmem_base, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Wait (bounded) for every MMA this CTA issued, then free the TMEM columns.
__device__ inline void tc_cta_fini(TcShared &ts) {
    __syncthreads();
    if (threadIdx.x == 32) {
        tc_commit(&ts.drain);
        mbar_wait(&ts.drain, ts.drains & 1, global_ns() + 2000000000ull);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x / 32 == 1) tmem_dealloc(ts.tmem_base, 512);
}

__device__ __forceinline__ int tc_failed(const TcShared &ts) { return *(volatile const int32_t *)&ts.fail; }

// Accumulator use u of a sub-tile of 'cols' tensor-memory columns: buffer and
// phase.  Sub-tiles of up to 256 columns alternate between two buffers (so
// the epilogue of one overlaps the MMAs of the next); wider ones use one.
__device__ __forceinline__ uint32_t tc_buf(uint32_t u, int cols) { return cols <= 256 ? (u & 1) : 0; }
__device__ __forceinline__ uint32_t tc_phase(uint32_t u, int cols) { return cols <= 256 ? (u >> 1) : u; }

// Sub-tiles of a tile of order nb (a multiple of 128): 128 rows (one MMA of
// M = 128) by NN = 256 columns when 256 divides nb, else 128; 'cols'
// tensor-memory columns each, so two accumulators fit and alternate.
__host__ __device__ __forceinline__ int tc_sub_cols(int nb) { return nb % 256 == 0 ? 256 : 128; }

// Epilogue of one sub-tile (rows ri*SR.., columns ci*NN..) from accumulator use
// u, by the 4 epilogue warps: TMEM -> registers -> C.  A lane holds one row of
// a 32 x 32 chunk (the tensor-memory lane layout) and reads and writes that
// row's 32 consecutive entries of C with four 32-byte accesses, each warp
// access touching 32 whole sectors.  False if a wait expired.
__device__ __forceinline__ void ld_global_v8(const float *p, float *v) {
    asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p));
}
__device__ __forceinline__ void st_global_v8(float *p, const float *v) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}

__device__ inline bool tc_epilogue_sub(TcShared &ts, float *C, int nb, int ri, int ci, float sa, float sb, uint32_t u,
                                       uint64_t deadline) {
    const int NN = tc_sub_cols(nb), SR = 128, cols = NN;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int q = warp - 4;  // TMEM lane quadrant of this warp
    const uint32_t b = tc_buf(u, cols), k = tc_phase(u, cols);
    // this lane's row of the sub-tile: 32-byte aligned (nb a multiple of 128)
    float *cr = C + (size_t)(ri * SR + q * 32 + lane) * nb + ci * NN;
    for (int l = 0; l < NN; l += 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(cr + l));  // into L2
    bool got = true;
    if (lane == 0) got = mbar_wait(&ts.acc_full[b], k & 1, deadline);
    got = __shfl_sync(0xffffffffu, got, 0);
    if (!got) return false;
    tc_fence_after();
    const uint32_t tcol = b * (uint32_t)cols;
    for (int c = 0; c < NN; c += 32) {
        // the row's 32 entries of C are requested first, so their latency
        // overlaps the tensor-memory load
        float cv[32];
#pragma unroll
        for (int v = 0; v < 4; ++v) ld_global_v8(cr + c + 8 * v, cv + 8 * v);
        uint32_t r[32];
        tmem_ld32(ts.tmem_base + ((uint32_t)(q * 32) << 16) + tcol + (uint32_t)c, r);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) cv[j] -= (__uint_as_float(r[j]) * sa) * sb;
#pragma unroll
        for (int v = 0; v < 4; ++v) st_global_v8(cr + c + 8 * v, cv + 8 * v);
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ts.tmem_empty[b]);
    return true;
}

struct TcNoDone {
    __device__ void operator()(uint64_t, uint64_t) const {}
};

// The epilogue warps apply a deferred sub-tile, if any, then one thread hands
// its word to on_done (after all 4 warps' stores: the named barrier).
template <class Done>
__device__ inline bool tc_epilogue_pending(TcShared &ts, uint64_t deadline, const Done &on_done) {
    if (!ts.pend) return true;
    const bool ok =
        tc_epilogue_sub(ts, ts.pend_C, ts.pend_nb, ts.pend_ri, ts.pend_ci, ts.pend_sa, ts.pend_sb, ts.pend_u, deadline);
    asm volatile("bar.sync 1, 128;" ::: "memory");  // the 4 epilogue warps only
    if (threadIdx.x == 128 && ok) on_done(ts.pend_task, ts.pend_t0);
    return ok;
}

// Apply a deferred sub-tile now (all threads; ends with a barrier).  False if
// a wait expired.
template <class Done>
__device__ inline bool tc_flush(TcShared &ts, uint64_t timeout_ns, const Done &on_done) {
    bool ok = true;
    if (threadIdx.x >= 128) ok = tc_epilogue_pending(ts, global_ns() + timeout_ns, on_done);
    if (!ok) *(volatile int32_t *)&ts.fail = 1;
    __syncthreads();
    ok = !tc_failed(ts);
    __syncthreads();
    if (threadIdx.x == 0) ts.pend = 0;
    __syncthreads();
    return ok;
}

// C[nb x nb] -= sa * sb * sum_p A_p B_p^T (sa, sb powers of two, applied one
// after the other so their product never underflows on its own), A rows
// starting at row aRow0 of the operand maps, B rows at bRow0.  lower: skip
// sub-tiles strictly above the diagonal (SYRK).  Called by all 256 threads;
// returns false if a wait expired.  A deferred sub-tile of the previous call
// is applied first by the epilogue warps (its completion handed to on_done);
// with defer_last the epilogue of this call's last sub-tile is left for the
// next call or tc_flush, tagged with task / t0.  The producer thread calls
// producer_idle() after its last load.
struct TcNoHook {
    __device__ void operator()() const {}
};

template <class Done = TcNoDone, class Hook = TcNoHook>
__device__ inline bool tc_tile_update(TcShared &ts, uint8_t *stages, const TcGemmArgs &g, float *C,
                                      int nb, int aRow0, int bRow0, float sa, float sb, bool lower,
                                      uint64_t timeout_ns, const Done &on_done = Done(), bool defer_last = false,
                                      uint64_t task = 0, uint64_t t0 = 0, const Hook &producer_idle = Hook()) {
    const int MH = 1;                          // 128-row halves per sub-tile
    const int NN = tc_sub_cols(nb);            // MMA N
    const int SR = MH * 128;                   // sub-tile rows
    const int cols = MH * NN;                  // tensor-memory columns of a sub-tile
    const int nsr = nb / SR, nsc = nb / NN;
    const int kchunks = nb / (g.tf32 ? 32 : 64);
    // the three products hi.hi, hi.lo, lo.hi read one K-chunk of A hi, A lo,
    // B hi and B lo from one slot (each box loaded once)
    const bool fused = g.passes == 3;
    const int NB = NN / 128;                   // B boxes of one operand
    const int boxes = fused ? 2 * MH + 2 * NB : MH + NB;
    const uint32_t stage_bytes = (uint32_t)boxes * kBoxBytes;
    const int nst_fit = (kTcStages * kStageBytes) / (int)stage_bytes;
    const uint32_t nst = (uint32_t)(nst_fit < kTcMaxSlots ? nst_fit : kTcMaxSlots);  // ring slots
    const int npass = fused ? 1 : g.passes;  // loads per K-chunk: per product, or once
    const uint32_t ring0 = ts.ring, acc0 = ts.acc_uses;
    const uint64_t deadline = global_ns() + timeout_ns;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    auto skip = [&](int ri, int ci) { return lower && ci * NN >= (ri + 1) * SR; };
    int nsub = 0;
    for (int ri = 0; ri < nsr; ++ri)
        for (int ci = 0; ci < nsc; ++ci) nsub += skip(ri, ci) ? 0 : 1;
    const uint32_t iters_per_sub = (uint32_t)(npass * kchunks);
    const bool defer = defer_last && cols <= 256;
    int last_ri = 0, last_ci = 0;  // the last sub-tile (the one deferred)
    for (int ri = 0; ri < nsr; ++ri)
        for (int ci = 0; ci < nsc; ++ci)
            if (!skip(ri, ci)) {
                last_ri = ri;
                last_ci = ci;
            }

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        fence_proxy_async_global();
        uint32_t f = ring0;
        for (int ri = 0; ri < nsr && !tc_failed(ts); ++ri)
            for (int ci = 0; ci < nsc && !tc_failed(ts); ++ci) {
                if (skip(ri, ci)) continue;
                for (int p = 0; p < npass && !tc_failed(ts); ++p)
                    for (int kc = 0; kc < kchunks; ++kc, ++f) {
                        const int s = (int)(f % nst);
                        if (f >= nst && !mbar_wait(&ts.empty[s], ((f / nst) & 1) ^ 1, deadline)) {
                            *(volatile int32_t *)&ts.fail = 1;
                            break;
                        }
                        mbar_arrive_expect_tx(&ts.full[s], stage_bytes);
                        const uint32_t dst = smem_u32(stages + (size_t)s * stage_bytes);
                        const int x = kc * (g.tf32 ? 32 : 64);
                        if (fused) {
                            // A hi, A lo, B hi (NB boxes), B lo (NB boxes); products 0 and 2
                            // name the A maps, 0 and 1 the B maps
                            const int ar = aRow0 + ri * SR, br = bRow0 + ci * NN;
                            tma_load_2d(dst, g.mapA[0], &ts.full[s], x, ar);
                            tma_load_2d(dst + kBoxBytes, g.mapA[2], &ts.full[s], x, ar);
                            for (int q = 0; q < NB; ++q) {
                                tma_load_2d(dst + (2 + q) * kBoxBytes, g.mapB[0], &ts.full[s], x, br + q * 128);
                                tma_load_2d(dst + (2 + NB + q) * kBoxBytes, g.mapB[1], &ts.full[s], x, br + q * 128);
                            }
                            continue;
                        }
                        for (int h = 0; h < MH; ++h)
                            tma_load_2d(dst + h * kBoxBytes, g.mapA[p], &ts.full[s], x, aRow0 + ri * SR + h * 128);
                        for (int q = 0; q < NN / 128; ++q)
                            tma_load_2d(dst + (MH + q) * kBoxBytes, g.mapB[p], &ts.full[s], x,
                                        bRow0 + ci * NN + q * 128);
                    }
            }
        producer_idle();
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        uint32_t f = ring0, u = acc0;
        for (int ri = 0; ri < nsr && !tc_failed(ts); ++ri)
            for (int ci = 0; ci < nsc && !tc_failed(ts); ++ci) {
                if (skip(ri, ci)) continue;
                const uint32_t b = tc_buf(u, cols), k = tc_phase(u, cols);
                // the epilogue of the previous use of this buffer must have read it
                if (k > 0 && !mbar_wait(&ts.tmem_empty[b], (k - 1) & 1, deadline)) {
                    *(volatile int32_t *)&ts.fail = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t tcol = b * (uint32_t)cols;
                bool first = true;
                for (int p = 0; p < npass && !tc_failed(ts); ++p)
                    for (int kc = 0; kc < kchunks; ++kc, ++f) {
                        const int s = (int)(f % nst);
                        if (!mbar_wait(&ts.full[s], (f / nst) & 1, deadline)) {
                            *(volatile int32_t *)&ts.fail = 1;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t base = smem_u32(stages + (size_t)s * stage_bytes);
                        if (fused) {
                            // hi.hi + hi.lo + lo.hi per K step (tf32)
                            const uint32_t d = ts.tmem_base + tcol;
#pragma unroll
                            for (int k4 = 0; k4 < 4; ++k4) {
                                const uint64_t ahi = sdesc_sw128(base + k4 * 32);
                                const uint64_t alo = sdesc_sw128(base + kBoxBytes + k4 * 32);
                                const uint64_t bhi = sdesc_sw128(base + 2 * kBoxBytes + k4 * 32);
                                const uint64_t blo = sdesc_sw128(base + (2 + NB) * kBoxBytes + k4 * 32);
                                tc_mma<true>(d, ahi, bhi, g.idesc, first ? 0u : 1u);
                                tc_mma<true>(d, ahi, blo, g.idesc, 1u);
                                tc_mma<true>(d, alo, bhi, g.idesc, 1u);
                                first = false;
                            }
                            tc_commit(&ts.empty[s]);
                            continue;
                        }
#pragma unroll
                        for (int k4 = 0; k4 < 4; ++k4) {
                            const uint64_t bdesc = sdesc_sw128(base + MH * kBoxBytes + k4 * 32);
                            for (int h = 0; h < MH; ++h) {
                                const uint64_t adesc = sdesc_sw128(base + h * kBoxBytes + k4 * 32);
                                const uint32_t d = ts.tmem_base + tcol + (uint32_t)(h * NN);
                                if (g.tf32) tc_mma<true>(d, adesc, bdesc, g.idesc, first ? 0u : 1u);
                                else tc_mma<false>(d, adesc, bdesc, g.idesc, first ? 0u : 1u);
                            }
                            first = false;
                        }
                        tc_commit(&ts.empty[s]);
                    }
                tc_commit(&ts.acc_full[b]);
                ++u;
            }
    } else if (warp >= 4) {
        // ---------------- epilogue (a deferred sub-tile of the previous call first)
        bool ok = tc_epilogue_pending(ts, deadline, on_done);
        uint32_t u = acc0;
        for (int ri = 0; ri < nsr && ok; ++ri)
            for (int ci = 0; ci < nsc && ok; ++ci) {
                if (skip(ri, ci)) continue;
                if (!(defer && ri == last_ri && ci == last_ci))
                    ok = tc_epilogue_sub(ts, C, nb, ri, ci, sa, sb, u, deadline);
                ++u;
            }
        if (!ok) *(volatile int32_t *)&ts.fail = 1;
    }
    __syncthreads();
    const bool ok = !tc_failed(ts);
    __syncthreads();
    if (threadIdx.x == 0 && ok) {
        ts.ring = ring0 + (uint32_t)nsub * iters_per_sub;
        ts.acc_uses = acc0 + (uint32_t)nsub;
        ts.pend = defer ? 1 : 0;
        if (defer) {
            ts.pend_u = acc0 + (uint32_t)nsub - 1;
            ts.pend_C = C;
            ts.pend_sa = sa;
            ts.pend_sb = sb;
            ts.pend_nb = nb;
            ts.pend_ri = last_ri;
            ts.pend_ci = last_ci;
            ts.pend_task = task;
            ts.pend_t0 = t0;
        }
    }
    __syncthreads();
    return ok;
}

}  // namespace chol
