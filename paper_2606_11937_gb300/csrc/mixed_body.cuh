// mixed_body.cuh -- the task bodies of the mixed-precision factorization,
// shared by the single-matrix engine (mixed.cu) and the tensor-core part of
// binary32 batches (batched_mixed.cu): the arguments and shared memory of a
// CTA, the operand copies of a panel tile, the binary32 TRSM of a tile of
// order 128 and one task of the tiled right-looking algorithm (Section 3.1,
// Fig. 1: POTRF in binary64, TRSM in binary32, SYRK/GEMM on tcgen05 with
// binary32 accumulation in tensor memory).
#pragma once

#include <cuda.h>
#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "factor_impl.cuh"
#include "tc_gemm.cuh"
#include "potrf128.cuh"

namespace chol {

struct MixedArgs {
    CUtensorMap map_hi;        // operand copies (bf16 / fp16 / tf32-hi)
    CUtensorMap map_lo;        // tf32-lo (FP32 mode)
    TileStore<float> S;        // binary32 tiles
    void *op_hi;               // operand stores, same tile indexing as S
    float *op_lo;
    int32_t *exps;             // per-tile scaling exponent (bf16 / fp16)
    int32_t precision;
    int32_t fmt;
    uint64_t timeout_ns;
};

struct MixedSmem {
    uint8_t stages[kTcStages][kStageBytes];
    TcShared ts;
};
static_assert(sizeof(SimtSmem<double>) <= sizeof(MixedSmem::stages), "SIMT scratch must fit in the stage area");
static_assert(kPotrf128SmemBytes <= sizeof(MixedSmem::stages), "the shared-memory POTRF must fit in the stage area");
static_assert(2 * 128 * 129 * sizeof(float) <= sizeof(MixedSmem::stages), "the shared-memory TRSM must fit in the stage area");

__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float pow2f(int e) { return ldexpf(1.0f, e); }

// CTA-wide max of |x| over a tile of nb*nb floats (count a multiple of 4,
// T 16-byte aligned: float4 loads, four in flight per thread)
__device__ inline float tile_absmax(const float *T, int64_t count, float *red) {
    float m = 0.f;
    const float4 *T4 = reinterpret_cast<const float4 *>(T);
    const int64_t n4 = count / 4;
#pragma unroll 4
    for (int64_t i = threadIdx.x; i < n4; i += blockDim.x) {
        const float4 v = __ldcg(T4 + i);
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) red[0] = m;
    }
    __syncthreads();
    const float r = red[0];
    __syncthreads();
    return r;
}

// exponent e with max * 2^e in [2^14, 2^15) (0 for an all-zero tile), clamped
__device__ __forceinline__ int scale_exponent(float mx) {
    if (!(mx > 0.f) || !isfinite(mx)) return 0;
    int E;
    frexpf(mx, &E);  // mx = f * 2^E, f in [0.5, 1)
    int e = 15 - E;
    return e < -126 ? -126 : (e > 126 ? 126 : e);
}

// Write the tensor-core operand copies of tile t (binary32 values in T).
// Four consecutive elements per thread and step (16-byte loads, several in
// flight: the tile was just written by this CTA and is read back from L2).
__device__ inline void write_operands(const MixedArgs &g, int64_t t, const float *T, float *red) {
    const int nb = g.S.nb;
    const int64_t cnt = (int64_t)nb * nb, n4 = cnt / 4;
    const size_t off = (size_t)t * cnt;
    const float4 *T4 = reinterpret_cast<const float4 *>(T);
    if (g.fmt == OP_TF32) {
        uint4 *hi = reinterpret_cast<uint4 *>(reinterpret_cast<uint32_t *>(g.op_hi) + off);
        uint4 *lo = g.op_lo ? reinterpret_cast<uint4 *>(reinterpret_cast<uint32_t *>(g.op_lo) + off) : nullptr;
#pragma unroll 4
        for (int64_t i = threadIdx.x; i < n4; i += blockDim.x) {
            const float4 x = __ldcg(T4 + i);
            const uint4 h = make_uint4(f32_to_tf32(x.x), f32_to_tf32(x.y), f32_to_tf32(x.z), f32_to_tf32(x.w));
            hi[i] = h;
            if (lo)
                lo[i] = make_uint4(f32_to_tf32(x.x - __uint_as_float(h.x)), f32_to_tf32(x.y - __uint_as_float(h.y)),
                                   f32_to_tf32(x.z - __uint_as_float(h.z)), f32_to_tf32(x.w - __uint_as_float(h.w)));
        }
    } else {
        const int e = scale_exponent(tile_absmax(T, cnt, red));
        const float s = pow2f(e);
        if (threadIdx.x == 0) g.exps[t] = e;
        if (g.fmt == OP_BF16) {
            __nv_bfloat162 *o = reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(g.op_hi) + off);
#pragma unroll 4
            for (int64_t i = threadIdx.x; i < n4; i += blockDim.x) {
                const float4 x = __ldcg(T4 + i);
                o[2 * i] = __floats2bfloat162_rn(x.x * s, x.y * s);
                o[2 * i + 1] = __floats2bfloat162_rn(x.z * s, x.w * s);
            }
        } else {
            __half2 *o = reinterpret_cast<__half2 *>(reinterpret_cast<__half *>(g.op_hi) + off);
#pragma unroll 4
            for (int64_t i = threadIdx.x; i < n4; i += blockDim.x) {
                const float4 x = __ldcg(T4 + i);
                o[2 * i] = __floats2half2_rn(x.x * s, x.y * s);
                o[2 * i + 1] = __floats2half2_rn(x.z * s, x.w * s);
            }
        }
    }
    fence_proxy_async_global();  // make the generic-proxy writes visible to later TMA reads
    __syncthreads();
}

// TRSM of a tile of order 128 in binary32 with both tiles in shared memory:
// B <- B L^{-T} (row-major tiles), right-looking over panels of 16 columns.
// A panel is solved row by row (thread r owns row r; x_c = (b_c - sum over
// k < c of x_k L(c, k)) / L(c, c), the division a multiplication by the
// reciprocal), then applied to the columns right of it as one rank-16 update
// by the 256 threads, each holding an 8-row x (up to 7)-column block of
// accumulators.  The solved tile is stored back and left in shared memory
// (Bs, padded rows) for the operand copies.  B and L have row pitches ldb
// and ldl (multiples of 4).  smem: 2 x 128 x 129 floats.
constexpr int kTrsmP = 129;
__device__ inline void smem_trsm128_f32(float *B, const float *L, float *smem, int ldb = 128, int ldl = 128) {
    constexpr int N = 128, P = kTrsmP, W = 16;
    float *Bs = smem, *Ls = smem + N * P;
    __shared__ float rinv[N];
    const int t = threadIdx.x;
    // four 16-byte loads of each tile in flight per thread before the stores
    constexpr int U = 4;
    for (int e0 = t; e0 < N * N / 4; e0 += blockDim.x * U) {
        float4 b[U], l[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x, r = (4 * e) / N, c = (4 * e) % N;
            if (e < N * N / 4) {
                b[u] = __ldcg(reinterpret_cast<const float4 *>(B + (size_t)r * ldb + c));
                l[u] = __ldcg(reinterpret_cast<const float4 *>(L + (size_t)r * ldl + c));
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x, r = (4 * e) / N, c = (4 * e) % N;
            if (e < N * N / 4) {
                Bs[r * P + c] = b[u].x; Bs[r * P + c + 1] = b[u].y; Bs[r * P + c + 2] = b[u].z; Bs[r * P + c + 3] = b[u].w;
                Ls[r * P + c] = l[u].x; Ls[r * P + c + 1] = l[u].y; Ls[r * P + c + 2] = l[u].z; Ls[r * P + c + 3] = l[u].w;
            }
        }
    }
    __syncthreads();
    if (t < N) rinv[t] = 1.0f / Ls[t * P + t];
    __syncthreads();
    const int tx = t & 15, ty = t >> 4;
    for (int jb = 0; jb < N; jb += W) {
        if (t < N) {
            float x[W];
#pragma unroll
            for (int c = 0; c < W; ++c) x[c] = Bs[t * P + jb + c];
#pragma unroll
            for (int c = 0; c < W; ++c) {
                float v = x[c];
#pragma unroll
                for (int k = 0; k < c; ++k) v = fmaf(-x[k], Ls[(jb + c) * P + jb + k], v);
                x[c] = v * rinv[jb + c];
            }
#pragma unroll
            for (int c = 0; c < W; ++c) Bs[t * P + jb + c] = x[c];
        }
        __syncthreads();
        const int c0 = jb + W, nj = (N - c0) / 16;  // column blocks of 16 right of the panel
        if (nj > 0) {
            float acc[8][7];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 7; ++j) acc[i][j] = 0.f;
#pragma unroll 4
            for (int k = 0; k < W; ++k) {
                float a[8], b[7];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = Bs[(ty * 8 + i) * P + jb + k];
#pragma unroll
                for (int j = 0; j < 7; ++j) b[j] = j < nj ? Ls[(c0 + tx + 16 * j) * P + jb + k] : 0.f;
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 7; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 7; ++j)
                    if (j < nj) Bs[(ty * 8 + i) * P + c0 + tx + 16 * j] -= acc[i][j];
        }
        __syncthreads();
    }
    for (int e = t; e < N * N / 4; e += blockDim.x) {
        const int r = (4 * e) / N, c = (4 * e) % N;
        *reinterpret_cast<float4 *>(B + (size_t)r * ldb + c) =
            make_float4(Bs[r * P + c], Bs[r * P + c + 1], Bs[r * P + c + 2], Bs[r * P + c + 3]);
    }
    __syncthreads();
}

// One task (I, K, J) of matrix m of the mixed-precision factorization: the
// matrix's binary32 tiles (order g.S.nb) are at `store`, its operand copies
// and scaling exponents at arena tile `toff` onwards (the operand maps span the
// arena); fail(col) records a non-positive pivot at 1-based column col and
// Done completes a deferred epilogue.  kPotrf32: the diagonal blocks are
// factored in binary32 (binary32 batches) instead of binary64.  Returns false
// if a wait expired.
template <bool kPotrf32, class Done, class Fail>
__device__ bool mixed_task(const MixedArgs &g, const SchedArgs &a, int m, int I, int K, int J, MixedSmem &sm,
                           float *store, int64_t toff, uint64_t t0, const Done &done, const Fail &fail) {
    const int type = task_type(I, K, J);
    const int nb = g.S.nb;
    auto tile = [&](int i, int k) { return store + (size_t)tile_index(i, k) * nb * nb; };
    bool ok = true;
    if (!(a.flags & CHOL_FLAG_NOOP)) {
        switch (type) {
        case T_POTRF: {
            // binary64 POTRF of each 128 x 128 diagonal block in shared memory
            // (the stage area); for tile orders above 128, blocked over those
            // blocks: TRSM of the blocks below and the update of the trailing
            // blocks in binary32, as the tiles of order 128 would see them
            float *T = tile(J, J);
            const int r = nb / kPotrfNb;
            SimtSmem<float> &ss = *reinterpret_cast<SimtSmem<float> *>(sm.stages);
            for (int j = 0; j < r; ++j) {
                float *Tjj = T + (size_t)j * kPotrfNb * nb + j * kPotrfNb;
                const int li = smem_potrf128<float, typename std::conditional<kPotrf32, float, double>::type>(
                    Tjj, &sm.stages[0][0], nb);
                if (li) {
                    if (threadIdx.x == 0) fail((int64_t)J * nb + j * kPotrfNb + li);
                    break;
                }
                for (int i = j + 1; i < r; ++i)
                    smem_trsm128_f32(T + (size_t)i * kPotrfNb * nb + j * kPotrfNb, Tjj,
                                     reinterpret_cast<float *>(sm.stages), nb, nb);
                for (int i = j + 1; i < r; ++i)
                    for (int k = j + 1; k <= i; ++k) {
                        float *C = T + (size_t)i * kPotrfNb * nb + k * kPotrfNb;
                        const float *Ai = T + (size_t)i * kPotrfNb * nb + j * kPotrfNb;
                        const float *Ak = T + (size_t)k * kPotrfNb * nb + j * kPotrfNb;
                        if (i == k) region_nt_update<float, true>(C, nb, Ai, nb, Ai, nb, kPotrfNb, kPotrfNb, kPotrfNb, ss);
                        else region_nt_update<float, false>(C, nb, Ai, nb, Ak, nb, kPotrfNb, kPotrfNb, kPotrfNb, ss);
                    }
                __syncthreads();
            }
        } break;
        case T_TRSM: {
            // B <- B L^{-T} by column blocks of 128: each block solved in
            // shared memory, then subtracted from the blocks right of it
            float *B = tile(I, J);
            const float *L = tile(J, J);
            const int r = nb / 128;
            SimtSmem<float> &ss = *reinterpret_cast<SimtSmem<float> *>(sm.stages);
            for (int j = 0; j < r; ++j) {
                const float *Ljj = L + (size_t)j * 128 * nb + j * 128;
                for (int i = 0; i < r; ++i)
                    smem_trsm128_f32(B + (size_t)i * 128 * nb + j * 128, Ljj, reinterpret_cast<float *>(sm.stages),
                                     nb, nb);
                for (int c = j + 1; c < r; ++c)
                    region_nt_update<float, false>(B + c * 128, nb, B + j * 128, nb, L + (size_t)c * 128 * nb + j * 128,
                                                   nb, nb, 128, 128, ss);
                __syncthreads();
            }
            write_operands(g, toff + tile_index(I, J), B, reinterpret_cast<float *>(sm.stages));
        } break;
        default: {
            // SYRK (K == I) or GEMM: C(I,K) -= A(I,J) A(K,J)^T on the tensor cores
            const int64_t ta = toff + tile_index(I, J), tb = toff + tile_index(K, J);
            float sa = 1.f, sb = 1.f;
            if (g.fmt != OP_TF32) {
                sa = pow2f(-__ldcg(g.exps + ta));
                sb = pow2f(-__ldcg(g.exps + tb));
            }
            TcGemmArgs ga;
            const bool three = g.precision == CHOL_FP32;
            ga.passes = three ? 3 : 1;
            ga.tf32 = g.fmt == OP_TF32;
            for (int p = 0; p < 3; ++p) {
                ga.mapA[p] = (three && p == 2) ? &g.map_lo : &g.map_hi;
                ga.mapB[p] = (three && p == 1) ? &g.map_lo : &g.map_hi;
            }
            ga.idesc = make_idesc((uint32_t)g.fmt, 128, (uint32_t)tc_sub_cols(nb));
            // the producer takes the next task from the queues once its
            // loads are issued, while the tensor cores and the epilogue finish
            const auto take_ahead = [&a]() { df_take_ahead(a); };
            ok = tc_tile_update(sm.ts, &sm.stages[0][0], ga, tile(I, K), nb, (int)(ta * nb),
                                (int)(tb * nb), sa, sb, type == T_SYRK, g.timeout_ns, done, a.dfl != nullptr,
                                pack_task(m, I, K, J), t0, take_ahead);
        } break;
        }
    }
    return ok;
}

}  // namespace chol
