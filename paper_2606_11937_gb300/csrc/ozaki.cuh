// ozaki.cuh -- binary64-accurate SYRK/GEMM tile updates on the bf16 tensor
// cores by exact splitting (the Ozaki scheme: Ozaki, Ogita, Oishi, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59, 2012), for tiles of order 128:
//
//  * split: every row r of a binary64 tile is scaled by 2^-e_r (e_r = the
//    exponent of the row's largest magnitude, so the scaled row lies in
//    (-1, 1)) and cut into S = 8 slices of 7 bits:
//        x = sum_{s=1..8} a_s 2^{-7 s} + delta,  a_s integer, |a_s| <= 127,
//    |delta| < 2^-56; every a_s is exact in bf16;
//  * product: A B^T = 2^{e_r + e_c} sum_d 2^{-7 d} G_d with
//        G_d = sum_{s + t = d} a_s b_t^T,  d = 2 .. 9  (36 slice products;
//    the omitted d >= 10 terms are below 2^-53 relative to the row scales).
//    |sum_k a_s(k) b_t(k)| <= 128 * 127^2 < 2^21 and a group has at most 8
//    products, so every partial sum of G_d is an integer below 2^24 and the
//    FP32 accumulation in tensor memory is exact in any order;
//  * the epilogue combines the 8 groups exactly into two int64 values, scales
//    them back by 2^{e_r + e_c} by building the binary64 encodings, and
//    subtracts both from the FP64 tile (two binary64 roundings per element; the
//    FP64 pipe does nothing else).
//
// The output tile is processed in four quarters of 32 columns.  A quarter's 8
// group accumulators take 8 x 32 = 256 tensor-memory columns, so two quarters
// alternate between the two halves of the 512 columns: the epilogue of one
// quarter runs while the tensor cores accumulate the next.  The 8 B slices of
// a quarter's 32 rows (64 KB) are double-buffered in shared memory as well;
// the A slices stream through a ring of stages.  The CTA has 12 warps: TMA
// producer (thread 0), MMA issuer (warp 1), and 8 epilogue warps, two per
// tensor-memory lane quadrant, each converting 16 of a quarter's 32 columns
// (two warps per SM sub-partition hide the latency of the integer and
// binary64 epilogue arithmetic).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace chol {

constexpr int kOzNb = 128;      // tile order of the emulated path
constexpr int kOzS = 8;         // slices per value
constexpr int kOzStages = 2;    // A-slice ring (one stage = one slice, both K-chunks)
constexpr int kOzThreads = 384; // 12 warps: producer, MMA issuer, 2 idle, 8 epilogue
constexpr int kOzEpiWarps = 8;
constexpr int kOzQ = 32;        // output columns per quarter (B rows per slice and quarter)
constexpr int kOzAChunk = 128 * 128;  // one A slice, one K-chunk of 64 (bf16): 128 rows x 128 B
constexpr int kOzABytes = 2 * kOzAChunk;  // one ring stage: a whole A slice
constexpr int kOzBBytes = kOzQ * 128; // one B slice, one K-chunk, one quarter's 32 rows

struct OzShared {
    uint64_t full[kOzStages];
    uint64_t empty[kOzStages];
    uint64_t bfull[2], bfree[2], acc_full[2], tmem_empty[2], drain;
    uint32_t tmem_base;
    uint32_t ring;      // A-stage fills before the current task
    uint32_t quarters;  // quarters (B loads / accumulations) before the current task
    int32_t fail;
    // the last quarter of an update whose epilogue was deferred to the next
    // call (ozaki_tile_update with defer_last) or to ozaki_flush
    int32_t pend;
    uint32_t pend_u;             // its quarter index
    double *pend_C;
    uint64_t pend_task;          // opaque word handed to the completion callback
    uint64_t pend_t0;
};

struct OzSmem {
    uint8_t B[2][2 * kOzS][kOzBBytes];     // 128 KB: buffer b, K-chunk kc, slice t at [b][kc * 8 + t] (the
                                           // 8 slices of a K-chunk form one 256-row K-major operand)
    uint8_t A[kOzStages][kOzABytes];       // 64 KB
    double xp[kOzEpiWarps][32 * 16];       // 32 KB: per epilogue warp, a 32 x 16 block of C
    int32_t ex[2][kOzNb];                  // column exponents (rows of B): [1] current update, [0] deferred quarter
    int32_t pea[kOzNb];                    // row exponents (rows of A) of the deferred quarter
    OzShared os;
};

__device__ __forceinline__ int oz_failed(const OzShared &s) { return *(volatile const int32_t *)&s.fail; }
__device__ __forceinline__ void oz_fail(OzShared &s) { *(volatile int32_t *)&s.fail = 1; }

__device__ __forceinline__ double pow2d(int e) {
    if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(1023 + e) << 52);
    return ldexp(1.0, e);
}

// bf16 bits of a small integer |a| <= 127 with sign `neg` (exact), integer ops only.
__device__ __forceinline__ uint16_t small_int_bf16(uint32_t a, uint32_t neg) {
    if (a == 0) return 0;
    const uint32_t msb = 31u - __clz(a);
    const uint32_t mant = (a << (7u - msb)) & 0x7Fu;
    return (uint16_t)((neg << 15) | ((127u + msb) << 7) | mant);
}

// Column of a row that lane `lane` holds in v[q] for ozaki_split_row: each
// lane owns the column pairs (2 lane, 2 lane + 1) and (64 + 2 lane, 65 + 2 lane),
// so every slice is written as packed bf16 pairs.
__device__ __forceinline__ int oz_col(int lane, int q) { return 2 * lane + (q & 1) + 64 * (q >> 1); }

// Split one row of 128 binary64 values (v[q] is column oz_col(lane, q); one
// warp) into 8 bf16 slices and return the row exponent e (|row| < 2^e).
// With x = v 2^-e in (-1, 1) and X = floor(|x| 2^56), slice s (1-based) is
// sign(x) times bits [56 - 7s, 63 - 7s) of X -- the digits the recursion
// t = 128 x, a = trunc(t), x = t - a produces -- computed with integer
// operations on the binary64 encoding.  Slice s (0-based) of column c goes
// to o[s * sstride + c] (o and sstride even); `negate` splits -v.
__device__ __forceinline__ int ozaki_split_row(const double (&v)[4], uint16_t *o, size_t sstride, bool negate) {
    const int lane = threadIdx.x % 32;
    // e = the frexp exponent of the row's largest magnitude m (m = f 2^e,
    // f in [0.5, 1), so |row| < 2^e), NaNs ignored, 0 if m is 0 or infinite;
    // found on the integer pipes: the magnitude bits of non-negative doubles
    // order like the values (GB300's binary64 pipe is the scarce one)
    unsigned long long mb = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v[q]) & 0x7FFFFFFFFFFFFFFFull;
        const unsigned long long mag = b > 0x7FF0000000000000ull ? 0ull : b;  // NaN
        mb = mag > mb ? mag : mb;
    }
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, mb, off);
        mb = o > mb ? o : mb;
    }
    int e = 0;
    const int emax = (int)(mb >> 52);
    if (mb != 0 && emax != 2047) e = emax ? emax - 1022 : (63 - __clzll((long long)mb)) - 1073;
    unsigned long long Xq[4];
    uint32_t ng[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned long long bits = (unsigned long long)__double_as_longlong(v[q]);
        ng[q] = (uint32_t)(bits >> 63) ^ (negate ? 1u : 0u);
        const int expo = (int)((bits >> 52) & 0x7FF);
        unsigned long long M = bits & ((1ull << 52) - 1);
        int qexp;                      // |v| = M 2^qexp
        if (expo == 0) qexp = -1074;   // subnormal or zero
        else {
            M |= 1ull << 52;
            qexp = expo - 1075;
        }
        const int sh = qexp - e + 56;  // X = floor(M 2^sh) < 2^56
        if (sh >= 0) Xq[q] = M << sh;
        else Xq[q] = sh <= -64 ? 0ull : (M >> (-sh));
    }
    // slice s of the two columns of a pair, stored as one packed bf16 word
#pragma unroll
    for (int s = 0; s < kOzS; ++s) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t lo = small_int_bf16((uint32_t)((Xq[2 * h] >> (49 - 7 * s)) & 127u), ng[2 * h]);
            const uint32_t hi = small_int_bf16((uint32_t)((Xq[2 * h + 1] >> (49 - 7 * s)) & 127u), ng[2 * h + 1]);
            *reinterpret_cast<uint32_t *>(o + (size_t)s * sstride + 2 * lane + 64 * h) = lo | (hi << 16);
        }
    }
    return e;
}

// Split a 128 x 128 binary64 tile into 8 bf16 slices ([s][r][c], 32 KB each)
// and one exponent per row (ozaki_split_row per row).  Element (r, c) is
// T[r * 128 + c], or T[c * 128 + r] with `transpose`; `negate` splits -T.
// All threads of the CTA; ends with a barrier.
__device__ inline void ozaki_split(const double *T, __nv_bfloat16 *slices, int32_t *rexp, bool negate = false,
                                   bool transpose = false) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nwarps = blockDim.x / 32;
    uint16_t *out = reinterpret_cast<uint16_t *>(slices);
    // four rows per warp at a time: their loads are in flight together
    constexpr int kRows = 4;
    for (int r0 = warp; r0 < kOzNb; r0 += kRows * nwarps) {
        double v[kRows][4];
#pragma unroll
        for (int j = 0; j < kRows; ++j) {
            const int r = r0 + j * nwarps;
            if (r >= kOzNb) {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[j][q] = 0.0;
            } else if (!transpose) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const double2 p = __ldcg(reinterpret_cast<const double2 *>(T + (size_t)r * kOzNb + oz_col(lane, 2 * h)));
                    v[j][2 * h] = p.x;
                    v[j][2 * h + 1] = p.y;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[j][q] = __ldcg(T + (size_t)oz_col(lane, q) * kOzNb + r);
            }
        }
#pragma unroll
        for (int j = 0; j < kRows; ++j) {
            const int r = r0 + j * nwarps;
            if (r < kOzNb) {
                const int e = ozaki_split_row(v[j], out + (size_t)r * kOzNb, (size_t)kOzNb * kOzNb, negate);
                if (lane == 0) rexp[r] = e;
            }
        }
    }
    fence_proxy_async_global();
    __syncthreads();
}

// binary64 value of the integer x (|x| < 2^53) times 2^scale, built from the
// bit pattern with integer operations (exact unless the result leaves the
// normal range, handled by ldexp).
__device__ __forceinline__ double int_scaled(long long x, int scale) {
    if (x == 0) return 0.0;
    const unsigned long long sign = x < 0 ? (1ull << 63) : 0ull;
    const unsigned long long ax = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
    const int msb = 63 - __clzll((long long)ax);
    const int biased = msb + scale + 1023;
    if (biased < 1 || biased > 2046) return ldexp((double)x, scale);
    const unsigned long long mant = (ax << (52 - msb)) & ((1ull << 52) - 1);
    return __longlong_as_double((long long)(sign | ((unsigned long long)biased << 52) | mant));
}

// As int_scaled for |x| < 2^47 when the caller knows 1 <= msb + scale + 1023 <= 2046.
__device__ __forceinline__ double int_scaled_fast(long long x, int scale) {
    const unsigned long long sign = (unsigned long long)x & (1ull << 63);
    const unsigned long long ax = (unsigned long long)(x < 0 ? -x : x);
    const int msb = 63 - __clzll((long long)ax);
    const unsigned long long mant = (ax << (52 - msb)) & ((1ull << 52) - 1);
    const unsigned long long bits = sign | ((unsigned long long)(msb + scale + 1023) << 52) | mant;
    return ax == 0 ? 0.0 : __longlong_as_double((long long)bits);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
// L2 policy that makes the lines it touches the first to be evicted: the C
// tiles stream through L2 once per update, the slices of a block column are
// reused by many updates
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void cp_async16_hint(uint32_t dst, const void *src, uint64_t pol) {
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_f64x2_hint(double *p, double2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(v.x), "d"(v.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}
// index of element (r, j) of a warp's 32 x 16 double block in shared memory,
// 16-byte segments XOR-swizzled by row so row- and column-wise accesses spread
__device__ __forceinline__ int xp_idx(int r, int j) { return r * 16 + ((((j >> 1) ^ (r & 7)) << 1) | (j & 1)); }

inline __device__ void oz_cta_init(OzShared &os) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < kOzStages; ++s) {
            mbar_init(&os.full[s], 1);
            mbar_init(&os.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&os.bfull[b], 1);
            mbar_init(&os.bfree[b], 1);
            mbar_init(&os.acc_full[b], 1);
            mbar_init(&os.tmem_empty[b], kOzEpiWarps);
        }
        mbar_init(&os.drain, 1);
        os.ring = 0;
        os.quarters = 0;
        os.fail = 0;
        os.pend = 0;
        mbar_fence_init();
    }
    if (threadIdx.x / 32 == 1) {
        tmem_alloc(&os.tmem_base, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

inline __device__ void oz_cta_fini(OzShared &os) {
    __syncthreads();
    if (threadIdx.x == 32) {
        tc_commit(&os.drain);
        mbar_wait(&os.drain, 0, global_ns() + 2000000000ull);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x / 32 == 1) tmem_dealloc(os.tmem_base, 512);
}

// One quarter of the epilogue for one epilogue warp (ew = warp - 4): rows of
// lane quadrant q = warp & 3, columns col0 .. col0 + 15 with col0 = 32 qq +
// 16 (ew >> 2), accumulators in tensor-memory half u & 1 of quarter u.  ea is
// the exponent of this lane's row, exB the column exponents of the tile (in
// shared memory).
// Returns false if the wait for the accumulators expired.
__device__ inline bool oz_epilogue_quarter(OzSmem &sm, double *C, int qq, uint32_t u, int ea, const int32_t *exB,
                                           uint64_t deadline) {
    OzShared &os = sm.os;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int ew = warp - 4, q = warp & 3, ch = ew >> 2;
    const uint32_t b = u & 1;
    double *xp = sm.xp[ew];
    const int col0 = qq * kOzQ + ch * 16;
    // stage this warp's 32 x 16 block of C in shared memory (async, coalesced
    // 16-byte copies) while the accumulators are produced
    double *cblk = C + (size_t)(q * 32) * kOzNb + col0;
    const uint64_t pol = l2_evict_first();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int idx = i * 32 + lane, rr = idx >> 3, seg = idx & 7;
        cp_async16_hint(smem_u32(xp + xp_idx(rr, 2 * seg)), cblk + (size_t)rr * kOzNb + 2 * seg, pol);
    }
    // one lane polls, the others wait at the shuffle
    bool got = true;
    if (lane == 0) got = mbar_wait(&os.acc_full[b], (u >> 1) & 1, deadline);
    got = __shfl_sync(0xffffffffu, got, 0);
    if (!got) {
        cp_async_wait_all();
        return false;
    }
    tc_fence_after();
    // group d = g + 2 holds at most d - 1 products below 2^21 each, so
    // G_{2k} 128 + G_{2k+1} fits in int32; hi = (t01 << 14) + t23 and
    // lo = (t45 << 14) + t67 are exact int64.
    long long hi[16], lo[16];
    const uint32_t tb = os.tmem_base + ((uint32_t)(q * 32) << 16) + b * (uint32_t)(kOzS * kOzQ) + (uint32_t)(ch * 16);
#pragma unroll
    for (int half4 = 0; half4 < 2; ++half4) {
        uint32_t r0[16], r1[16], r2[16], r3[16];
        const int g = half4 * 4;
        tmem_ld16(tb + (uint32_t)(g * kOzQ), r0);
        tmem_ld16(tb + (uint32_t)((g + 1) * kOzQ), r1);
        tmem_ld16(tb + (uint32_t)((g + 2) * kOzQ), r2);
        tmem_ld16(tb + (uint32_t)((g + 3) * kOzQ), r3);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int32_t t01 = __float2int_rn(__uint_as_float(r0[j])) * 128 + __float2int_rn(__uint_as_float(r1[j]));
            const int32_t t23 = __float2int_rn(__uint_as_float(r2[j])) * 128 + __float2int_rn(__uint_as_float(r3[j]));
            const long long w = ((long long)t01 << 14) + (long long)t23;
            if (half4 == 0) hi[j] = w;
            else lo[j] = w;
        }
    }
    // the accumulators are in registers: release this half of tensor memory
    // to the MMAs of quarter u + 2 before updating C
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&os.tmem_empty[b]);
    // one vote per quarter: exponents of the scaled values stay normal
    // (|hi|, |lo| < 2^47) unless a row or column scale is extreme
    bool ok_range = true;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int e = ea + exB[col0 + j];
        ok_range &= (e >= -900 && e <= 900);
    }
    cp_async_wait_all();
    __syncwarp();
    // this lane's row of the block: C <- (C - hi 2^(eab-35)) - lo 2^(eab-63)
    if (__all_sync(0xffffffffu, ok_range)) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int e = ea + exB[col0 + j];
            double &cv = xp[xp_idx(lane, j)];
            cv = (cv - int_scaled_fast(hi[j], e - 35)) - int_scaled_fast(lo[j], e - 63);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int e = ea + exB[col0 + j];
            double &cv = xp[xp_idx(lane, j)];
            cv = (cv - int_scaled(hi[j], e - 35)) - int_scaled(lo[j], e - 63);
        }
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int idx = i * 32 + lane, rr = idx >> 3, seg = idx & 7;
        const double2 v = *reinterpret_cast<const double2 *>(xp + xp_idx(rr, 2 * seg));
        st_f64x2_hint(cblk + (size_t)rr * kOzNb + 2 * seg, v, pol);
    }
    __syncwarp();
    return true;
}

// The epilogue warps apply the deferred quarter, if any (its exponents were
// left in shared memory by the call that deferred it: pea, ex[0]).  Its
// completion is handed to on_done after all 8 warps' stores: with
// done_by_warp2 the epilogue warps only arrive on named barrier 3 and warp 2
// (idle in the tile update) waits there and calls on_done, so the epilogue
// goes on without the completion's round trips; otherwise thread 128 calls
// it after a barrier of the epilogue warps.
template <class Done>
__device__ inline bool oz_epilogue_pending(OzSmem &sm, uint64_t deadline, const Done &on_done, bool done_by_warp2) {
    OzShared &os = sm.os;
    if (!os.pend) return true;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int row = (warp & 3) * 32 + lane;
    const bool ok = oz_epilogue_quarter(sm, os.pend_C, kOzNb / kOzQ - 1, os.pend_u, sm.pea[row], sm.ex[0], deadline);
    if (!ok) oz_fail(os);
    if (done_by_warp2) {
        asm volatile("bar.arrive 3, 288;" ::: "memory");  // 8 epilogue warps + warp 2
    } else {
        asm volatile("bar.sync 1, 256;" ::: "memory");  // the 8 epilogue warps only
        if (warp == 4 && lane == 0 && ok) on_done(os.pend_task, os.pend_t0);
    }
    return ok;
}

struct OzNoDone {
    __device__ void operator()(uint64_t, uint64_t) const {}
};

// Apply a deferred last quarter now (all threads of the CTA; ends with a
// barrier).  False if a wait expired.
template <class Done>
__device__ inline bool ozaki_flush(OzSmem &sm, uint64_t timeout_ns, const Done &on_done) {
    OzShared &os = sm.os;
    bool ok = true;
    if (threadIdx.x >= 128) ok = oz_epilogue_pending(sm, global_ns() + timeout_ns, on_done, false);
    if (!ok) oz_fail(os);
    __syncthreads();
    ok = !oz_failed(os);
    __syncthreads();
    if (threadIdx.x == 0) os.pend = 0;
    __syncthreads();
    return ok;
}

// C (row-major 128 x 128 binary64) -= A B^T where A, B are given by their
// slices: rows [aRow0, aRow0 + 8*128) and [bRow0, ...) of the slice maps
// (slice s of a tile at rows base + 128 s) and their row exponents.  mapA has
// 128-row boxes, mapB 32-row boxes.  Called by all kOzThreads threads; false
// if a bounded wait expired.
//
// Quarter u (counted across tasks) uses B buffer and tensor-memory half
// b = u & 1; the k-th use of a buffer waits on its barriers with parity k & 1.
// The producer thread (thread 0) calls producer_idle() after its last load.
struct OzNoHook {
    __device__ void operator()() const {}
};

//
// A deferred quarter of the previous call is applied first by the epilogue
// warps (its completion handed to on_done); with defer_last this call's last
// quarter is left for the next call or ozaki_flush, tagged with `task`/t0.
template <class Hook = OzNoHook, class Done = OzNoDone>
__device__ inline bool ozaki_tile_update(OzSmem &sm, const CUtensorMap *mapA, const CUtensorMap *mapB, double *C,
                                         int aRow0, int bRow0, const int32_t *expA, const int32_t *expB,
                                         uint64_t timeout_ns, const Hook &producer_idle = Hook(),
                                         const Done &on_done = Done(), bool defer_last = false, uint64_t task = 0,
                                         uint64_t t0 = 0) {
    OzShared &os = sm.os;
    const uint32_t ring0 = os.ring, q0 = os.quarters;
    const uint64_t deadline = global_ns() + timeout_ns;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    constexpr int kQuarters = kOzNb / kOzQ;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        fence_proxy_async_global();
        uint32_t f = ring0;
        for (int qq = 0; qq < kQuarters && !oz_failed(os); ++qq) {
            const uint32_t u = q0 + qq, b = u & 1;
            // the MMAs of quarter u - 2 must have finished reading buffer b
            if (u >= 2 && !mbar_wait(&os.bfree[b], ((u >> 1) - 1) & 1, deadline)) {
                oz_fail(os);
                break;
            }
            mbar_arrive_expect_tx(&os.bfull[b], 2 * kOzS * kOzBBytes);
            for (int t = 0; t < kOzS; ++t)
                for (int kc = 0; kc < 2; ++kc)
                    tma_load_2d(smem_u32(sm.B[b][kc * kOzS + t]), mapB, &os.bfull[b], kc * 64,
                                bRow0 + t * 128 + qq * kOzQ);
            for (int s = 0; s < kOzS && !oz_failed(os); ++s, ++f) {
                const int st = (int)(f % kOzStages);
                if (f >= (uint32_t)kOzStages && !mbar_wait(&os.empty[st], ((f / kOzStages) & 1) ^ 1, deadline)) {
                    oz_fail(os);
                    break;
                }
                mbar_arrive_expect_tx(&os.full[st], kOzABytes);
                for (int kc = 0; kc < 2; ++kc)
                    tma_load_2d(smem_u32(sm.A[st]) + kc * kOzAChunk, mapA, &os.full[st], kc * 64, aRow0 + s * 128);
            }
        }
        producer_idle();
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        // For A slice s, the products with B slices t = 0 .. 7-s go to groups
        // g = s + t, whose accumulators sit at tensor-memory columns 32 g of the
        // quarter's half: contiguous, so with the 8 B slices of a K-chunk stored
        // as one 256-row operand a single MMA of N = 32 (8 - s) covers them all.
        // Advancing K by 16 bf16 (32 bytes) adds 2 to the descriptor's
        // start-address field (16-byte units).
        constexpr uint32_t kIdescN[kOzS + 1] = {
            0u, make_idesc(OP_BF16, 128, 32), make_idesc(OP_BF16, 128, 64), make_idesc(OP_BF16, 128, 96),
            make_idesc(OP_BF16, 128, 128), make_idesc(OP_BF16, 128, 160), make_idesc(OP_BF16, 128, 192),
            make_idesc(OP_BF16, 128, 224), make_idesc(OP_BF16, 128, 256)};
        uint32_t f = ring0;
        for (int qq = 0; qq < kQuarters && !oz_failed(os); ++qq) {
            const uint32_t u = q0 + qq, b = u & 1;
            if (!mbar_wait(&os.bfull[b], (u >> 1) & 1, deadline)) {
                oz_fail(os);
                break;
            }
            // the epilogue of quarter u - 2 must have read this half of tensor memory
            if (u >= 2 && !mbar_wait(&os.tmem_empty[b], ((u >> 1) - 1) & 1, deadline)) {
                oz_fail(os);
                break;
            }
            tc_fence_after();
            const uint64_t bdesc[2] = {sdesc_sw128(smem_u32(sm.B[b][0])), sdesc_sw128(smem_u32(sm.B[b][kOzS]))};
            const uint32_t dbase = os.tmem_base + b * (uint32_t)(kOzS * kOzQ);
            for (int s = 0; s < kOzS && !oz_failed(os); ++s, ++f) {
                const int st = (int)(f % kOzStages);
                if (!mbar_wait(&os.full[st], (f / kOzStages) & 1, deadline)) {
                    oz_fail(os);
                    break;
                }
                tc_fence_after();
                const uint32_t idesc = kIdescN[kOzS - s];
                const uint32_t d = dbase + (uint32_t)(s * kOzQ);
#pragma unroll
                for (int kc = 0; kc < 2; ++kc) {
                    const uint64_t adesc = sdesc_sw128(smem_u32(sm.A[st]) + kc * kOzAChunk);
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4)
                        tc_mma<false>(d, adesc + 2 * k4, bdesc[kc] + 2 * k4, idesc,
                                      (s == 0 && kc == 0 && k4 == 0) ? 0u : 1u);
                }
                tc_commit(&os.empty[st]);
            }
            tc_commit(&os.acc_full[b]);
            tc_commit(&os.bfree[b]);
        }
    } else if (warp >= 4) {
        // ---------------- epilogue: 8 exact FP32 group sums -> binary64
        // G_g (d = g + 2) are integers below 2^24.  hi = sum_{g<4} G_g 2^{7(3-g)}
        // and lo = sum_{g>=4} G_g 2^{7(7-g)} are exact int64 (< 2^46); the
        // update is A B^T = 2^{e_r + e_c} (hi 2^-35 + lo 2^-63).  Warp w owns
        // the 32 rows of lane quadrant w % 4 and columns 16 ((w - 4) / 4) ..
        // +15 of each quarter (oz_epilogue_quarter).
        const int row = (warp & 3) * 32 + lane;
        // pull this row of C into L2 while the MMAs run (8 lines of 128 bytes)
        if (warp < 8) {
#pragma unroll
            for (int l = 0; l < 8; ++l)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(C + (size_t)row * kOzNb + l * 16));
        }
        // the previous call's deferred quarter (its accumulators are in the
        // other tensor-memory half than this call's first quarter)
        const int ea = __ldcg(expA + row);
        bool ok = oz_epilogue_pending(sm, deadline, on_done, true);
        for (int i = threadIdx.x - 128; i < kOzNb; i += 32 * kOzEpiWarps) sm.ex[1][i] = __ldcg(expB + i);
        asm volatile("bar.sync 1, 256;" ::: "memory");  // the 8 epilogue warps only
        const int nq = defer_last ? kQuarters - 1 : kQuarters;
#pragma unroll 1
        for (int qq = 0; qq < nq && ok; ++qq) ok = oz_epilogue_quarter(sm, C, qq, q0 + qq, ea, sm.ex[1], deadline);
        if (!ok) oz_fail(os);
        if (defer_last) {
            // leave the deferred quarter's exponents for the call that applies it
            if (warp < 8) sm.pea[row] = ea;
            const int i = (int)threadIdx.x - 128;
            if (i < kOzQ) sm.ex[0][kOzNb - kOzQ + i] = sm.ex[1][kOzNb - kOzQ + i];
        }
    } else if (warp == 2) {
        // ---------------- completion of the previous call's deferred quarter
        if (os.pend) {
            asm volatile("bar.sync 3, 288;" ::: "memory");
            if (lane == 0 && !oz_failed(os)) on_done(os.pend_task, os.pend_t0);
        }
    }
    __syncthreads();
    const bool ok = !oz_failed(os);
    __syncthreads();
    if (threadIdx.x == 0 && ok) {
        os.ring = ring0 + kQuarters * kOzS;
        os.quarters = q0 + kQuarters;
        os.pend = defer_last ? 1 : 0;
        if (defer_last) {
            os.pend_u = q0 + kQuarters - 1;
            os.pend_C = C;
            os.pend_task = task;
            os.pend_t0 = t0;
        }
    }
    __syncthreads();
    return ok;
}

}  // namespace chol
