// batched_impl.cuh -- definitions shared by the batched factor + solve
// plans (batched.cu) and their tensor-core parts (batched_tc.cu for FP64,
// batched_mixed.cu for FP32): matrix
// descriptors, the repack / unpack over a flat tile list, and the SOLVE
// task's substitutions.
#pragma once

#include "common.cuh"
#include "factor_impl.cuh"

namespace chol {

struct MatDesc {
    void *store;        // tiles of this matrix (double or float)
    int64_t task_base;  // offset of its task counters
    double *A;          // caller's matrix (input, factor output)
    int64_t lda;
    double *b;          // caller's right-hand side (input, solution output)
    int32_t n, nb, M, pad;
};

struct TileRef {
    int32_t m;
    int32_t t;  // lower tile index inside matrix m
};

// Whether the tasks of matrix m are no-ops (the matrix failed, or a no-op
// run): read once by thread 0 and shared, so that every thread of the CTA
// takes the same branch even when the matrix fails while this task starts.
// All threads; contains a barrier.
__device__ inline bool batch_skip(const SchedArgs &a, const int32_t *failed, int m) {
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = ((a.flags & CHOL_FLAG_NOOP) || ld_acquire_s32(failed + m)) ? 1 : 0;
    __syncthreads();
    return s_skip != 0;
}

// Scratch of tiles_solve besides y: a staged 32 x 32 diagonal block of L
// (row pitch 33), the reciprocals of its diagonal and the offsets of the
// rows of the current chunk in the tile store.
template <typename T>
struct SolveScratch {
    T D[32][33];
    T dinv[32];
    int64_t rb[32];  // row r of the chunk: offset of element (r, 0) if tile column 0 held it
};

// Stage chunk [c0, c0 + w) of the diagonal: D (lower part), 1 / L_ii, rb.
// All threads; ends with a barrier.
template <typename T>
__device__ void solve_stage_chunk(const T *store, int nb, int c0, int w, SolveScratch<T> &s) {
    const int64_t nb2 = (int64_t)nb * nb;
    if (threadIdx.x < 32) {
        const int r = threadIdx.x, i = c0 + r, I = i / nb;
        s.rb[r] = r < w ? ((int64_t)I * (I + 1) / 2) * nb2 + (int64_t)(i - I * nb) * nb : 0;
    }
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int r = e >> 5, c = e & 31;
        T v = T(0);
        if (r < w && c <= r) {
            const int i = c0 + r, k = c0 + c, I = i / nb, K = k / nb;
            v = __ldcg(store + ((int64_t)I * (I + 1) / 2 + K) * nb2 + (int64_t)(i - I * nb) * nb + (k - K * nb));
        }
        s.D[r][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) s.dinv[threadIdx.x] = threadIdx.x < w ? T(1) / s.D[threadIdx.x][threadIdx.x] : T(0);
    __syncthreads();
}

template <typename T, int V> struct SolveVec;
template <> struct SolveVec<float, 4> { using type = float4; };
template <> struct SolveVec<double, 2> { using type = double2; };
template <typename T> struct SolveVec<T, 1> { using type = T; };

template <typename T, int V>
__device__ __forceinline__ void solve_load(const T *p, T (&v)[V]) {
    if constexpr (V == 1) {
        v[0] = __ldcg(p);
    } else {
        const typename SolveVec<T, V>::type x = __ldcg(reinterpret_cast<const typename SolveVec<T, V>::type *>(p));
        if constexpr (V == 4) { v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w; }
        else { v[0] = x.x; v[1] = x.y; }
    }
}

// L L^T x = b (the use of the factor the paper motivates in Section 1) with
// L in a tile store (row-major tiles of order nb, tile
// (I, K) at index I (I + 1) / 2 + K), one CTA, blocked by chunks of 32 rows.
// Forward, chunk by chunk: y_c -= L(c, 0:c0) y(0:c0) (one warp per row, its
// lanes along the row in V-element loads, a warp sum), then y_c = L_cc^{-1}
// y_c by column-oriented substitution in one warp (y_k = y_k / L_kk, then
// y_i -= L_ik y_k for i > k).  Backward, last chunk first: x_c = L_cc^{-T}
// y_c by column-oriented substitution (x_k = y_k / L_kk, then y_j -= L_kj x_k
// for j < k), then y(0:c0) -= L(c, 0:c0)^T x_c (each thread owns V columns
// and sums over the chunk's rows).  Both sweeps read each element of L once.
// y: n values in shared memory; b is read and overwritten with x.  Needs nb
// a multiple of V and a 16-byte aligned store when V > 1.  All threads; ends
// with a barrier.  Not inlined: the persistent kernels that run it keep
// the register allocation of their task bodies.
template <typename T, int V>
__device__ __noinline__ void tiles_solve_v(const T *store, int nb, int n, double *b, T *y, SolveScratch<T> &s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int64_t nb2 = (int64_t)nb * nb;
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = (T)b[i];
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += 32) {
        const int w = min(32, n - c0);
        solve_stage_chunk(store, nb, c0, w, s);
        // y_c -= L(c, 0:c0) y(0:c0): warp `warp` takes rows warp, warp + W, ...
        if (c0 > 0) {
            for (int r0 = warp; r0 < w; r0 += 4 * W) {
                T acc[4] = {T(0), T(0), T(0), T(0)};
                int K = (lane * V) / nb, kl = lane * V - K * nb;
                for (int k = lane * V; k < c0; k += 32 * V) {
                    T yv[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) yv[v] = y[k + v];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int r = r0 + q * W;
                        if (r < w) {
                            T lv[V];
                            solve_load<T, V>(store + s.rb[r] + K * nb2 + kl, lv);
#pragma unroll
                            for (int v = 0; v < V; ++v) acc[q] = fma(lv[v], yv[v], acc[q]);
                        }
                    }
                    kl += 32 * V;
                    while (kl >= nb) { kl -= nb; ++K; }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    T a = acc[q];
                    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                    const int r = r0 + q * W;
                    if (lane == 0 && r < w) y[c0 + r] -= a;
                }
            }
            __syncthreads();
        }
        if (warp == 0) {
            T yi = lane < w ? y[c0 + lane] : T(0);
            for (int k = 0; k < w; ++k) {
                const T yk = __shfl_sync(0xffffffffu, yi, k) * s.dinv[k];
                if (lane == k) yi = yk;
                else if (lane > k) yi = fma(-s.D[lane][k], yk, yi);
            }
            if (lane < w) y[c0 + lane] = yi;
        }
        __syncthreads();
    }
    const int last = ((n - 1) / 32) * 32;
    for (int c0 = last; c0 >= 0; c0 -= 32) {
        const int w = min(32, n - c0);
        solve_stage_chunk(store, nb, c0, w, s);
        if (warp == 0) {
            T zj = lane < w ? y[c0 + lane] : T(0);
            for (int k = w - 1; k >= 0; --k) {
                const T xk = __shfl_sync(0xffffffffu, zj, k) * s.dinv[k];
                if (lane == k) zj = xk;
                else if (lane < k) zj = fma(-s.D[k][lane], xk, zj);
            }
            if (lane < w) y[c0 + lane] = zj;
        }
        __syncthreads();
        // y(0:c0) -= L(c, 0:c0)^T x_c: thread t owns columns t V .. t V + V - 1,
        // then every blockDim V-th column after them
        for (int j = threadIdx.x * V; j < c0; j += blockDim.x * V) {
            const int K = j / nb, kl = j - K * nb;
            T acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = T(0);
#pragma unroll 4
            for (int r = 0; r < w; ++r) {
                T lv[V];
                solve_load<T, V>(store + s.rb[r] + K * nb2 + kl, lv);
                const T xr = y[c0 + r];
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = fma(lv[v], xr, acc[v]);
            }
#pragma unroll
            for (int v = 0; v < V; ++v) y[j + v] -= acc[v];
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = (double)y[i];
    __syncthreads();
}

// The vector width is the widest 16-byte load the tile order allows.
template <typename T>
__device__ void tiles_solve(const T *store, int nb, int n, double *b, T *y, SolveScratch<T> &s) {
    constexpr int V = 16 / sizeof(T);
    if (nb % V == 0 && (reinterpret_cast<uintptr_t>(store) & 15) == 0) tiles_solve_v<T, V>(store, nb, n, b, y, s);
    else tiles_solve_v<T, 1>(store, nb, n, b, y, s);
}

// Repack / unpack over a flat list of (matrix, tile): a CTA (32 x 8 threads)
// moves kSubPer consecutive 32 x 32 sub-blocks of one tile (grid.y = groups of
// kSubPer sub-blocks), all its loads issued before the shared-memory
// transposes (16 per thread), so that enough bytes are in flight per SM.
constexpr int kSubPer = 4;

template <typename T>
__global__ void __launch_bounds__(256) batch_repack_kernel(const MatDesc *desc, const TileRef *list) {
    __shared__ T buf[kSubPer][32][33];
    const TileRef tr = list[blockIdx.x];
    const MatDesc d = desc[tr.m];
    const int nb = d.nb, nsb = (nb + 31) / 32, sb0 = blockIdx.y * kSubPer;
    if (sb0 >= nsb * nsb) return;
    int I, K;
    tile_of(tr.t, I, K);
    T *tile = reinterpret_cast<T *>(d.store) + (size_t)tr.t * nb * nb;
    T v[kSubPer][4];
#pragma unroll
    for (int s = 0; s < kSubPer; ++s) {
        const int sb = sb0 + s, sr = sb / nsb, sc = sb % nsb;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int yy = threadIdx.y + 8 * q;
            const int r = sr * 32 + threadIdx.x, c = sc * 32 + yy;
            const int64_t i = (int64_t)I * nb + r, j = (int64_t)K * nb + c;
            T x = T(0);
            if (sb < nsb * nsb && r < nb && c < nb) {
                if (i < d.n && j < d.n) x = j <= i ? (T)d.A[j * d.lda + i] : T(0);
                else x = i == j ? T(1) : T(0);
            }
            v[s][q] = x;
        }
    }
#pragma unroll
    for (int s = 0; s < kSubPer; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) buf[s][threadIdx.y + 8 * q][threadIdx.x] = v[s][q];
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kSubPer; ++s) {
        const int sb = sb0 + s, sr = sb / nsb, sc = sb % nsb;
        if (sb >= nsb * nsb) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int yy = threadIdx.y + 8 * q;
            const int r = sr * 32 + yy, c = sc * 32 + threadIdx.x;
            if (r < nb && c < nb) tile[(size_t)r * nb + c] = buf[s][threadIdx.x][yy];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) batch_unpack_kernel(const MatDesc *desc, const TileRef *list) {
    __shared__ T buf[kSubPer][32][33];
    const TileRef tr = list[blockIdx.x];
    const MatDesc d = desc[tr.m];
    const int nb = d.nb, nsb = (nb + 31) / 32, sb0 = blockIdx.y * kSubPer;
    if (sb0 >= nsb * nsb) return;
    int I, K;
    tile_of(tr.t, I, K);
    const T *tile = reinterpret_cast<const T *>(d.store) + (size_t)tr.t * nb * nb;
    T v[kSubPer][4];
#pragma unroll
    for (int s = 0; s < kSubPer; ++s) {
        const int sb = sb0 + s, sr = sb / nsb, sc = sb % nsb;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int yy = threadIdx.y + 8 * q;
            const int r = sr * 32 + yy, c = sc * 32 + threadIdx.x;
            v[s][q] = (sb < nsb * nsb && r < nb && c < nb) ? tile[(size_t)r * nb + c] : T(0);
        }
    }
#pragma unroll
    for (int s = 0; s < kSubPer; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) buf[s][threadIdx.y + 8 * q][threadIdx.x] = v[s][q];
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kSubPer; ++s) {
        const int sb = sb0 + s, sr = sb / nsb, sc = sb % nsb;
        if (sb >= nsb * nsb) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int yy = threadIdx.y + 8 * q;
            const int r = sr * 32 + threadIdx.x, c = sc * 32 + yy;
            const int64_t i = (int64_t)I * nb + r, j = (int64_t)K * nb + c;
            if (r < nb && c < nb && i < d.n && j < d.n && j <= i) d.A[j * d.lda + i] = (double)buf[s][threadIdx.x][yy];
        }
    }
}


// The tensor-core FP64 part of a batch (batched_tc.cu): matrices of order
// above 1024 factored (and solved) in one persistent dataflow kernel of
// their own, on tiles of order 128 with SYRK/GEMM/TRSM as exact bf16 slice
// products.  Their tile stores are part of the batch's descriptors
// (index base .. base + count - 1 of desc).
struct OzBatchPart;
size_t oz_batch_bytes(int count, const int64_t *n, int64_t *tasks_out);
int oz_batch_create(OzBatchPart **out, int count, const int64_t *n, void *ws, const MatDesc *h_desc_part,
                    const chol_opts &o);
int oz_batch_record(OzBatchPart *p, const MatDesc *d_desc_part, int64_t *d_info_part, int32_t *d_failed_part,
                    cudaStream_t st, int *launches);
void oz_batch_destroy(OzBatchPart *p);
const Control *oz_batch_control(const OzBatchPart *p);

// The tensor-core part of a binary32 batch (batched_mixed.cu): matrices of
// order above the split order factored (and solved) in one persistent
// dataflow kernel of their own, on tiles of order 128 with SYRK/GEMM as three
// TF32 products on tcgen05 (the mixed-precision engine's FP32 mode).
struct MixedBatchPart;
size_t mixed_batch_bytes(int count, const int64_t *n, int64_t *tasks_out);
int mixed_batch_create(MixedBatchPart **out, int count, const int64_t *n, void *ws, const chol_opts &o);
int mixed_batch_record(MixedBatchPart *p, const MatDesc *d_desc_part, int64_t *d_info_part, int32_t *d_failed_part,
                       cudaStream_t st, int *launches);
void mixed_batch_destroy(MixedBatchPart *p);
const Control *mixed_batch_control(const MixedBatchPart *p);

}  // namespace chol
