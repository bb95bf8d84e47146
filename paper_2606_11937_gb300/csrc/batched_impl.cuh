// batched_impl.cuh -- definitions shared by the batched factor + solve
// plans (batched.cu) and their tensor-core FP64 part (batched_tc.cu): matrix
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

// L L^T x = b with L in a tile store (row-major tiles of order nb, tile
// (I, K) at index I (I + 1) / 2 + K), one CTA: column-oriented forward
// substitution (y_k = y_k / L_kk, then y_i -= L_ik y_k for i > k) and
// row-oriented backward substitution (x_k = (y_k - sum_{i>k} L_ik x_i) / L_kk,
// the sum a warp-parallel dot product).  y: n values in shared memory; b is
// read and overwritten with x.  All threads; ends with a barrier.
template <typename T>
__device__ void tiles_solve(const T *store, int nb, int n, double *b, T *y) {
    auto tile = [&](int I, int K) { return store + (size_t)tile_index(I, K) * nb * nb; };
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = (T)b[i];
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const T *Lk = tile(k / nb, k / nb);
        if (threadIdx.x == 0) y[k] = y[k] / __ldcg(Lk + (size_t)(k % nb) * nb + k % nb);
        __syncthreads();
        const T yk = y[k];
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
            const T *t = tile(i / nb, k / nb);
            y[i] = fma(-__ldcg(t + (size_t)(i % nb) * nb + k % nb), yk, y[i]);
        }
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {
        T s = T(0);
        if (threadIdx.x < 32) {
            for (int i = k + 1 + threadIdx.x; i < n; i += 32) {
                const T *t = tile(i / nb, k / nb);
                s = fma(__ldcg(t + (size_t)(i % nb) * nb + k % nb), y[i], s);
            }
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (threadIdx.x == 0) {
                const T *Lk = tile(k / nb, k / nb);
                y[k] = (y[k] - s) / __ldcg(Lk + (size_t)(k % nb) * nb + k % nb);
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = (double)y[i];
    __syncthreads();
}

// Repack / unpack over a flat list of (matrix, tile); grid.y = 32 x 32 sub-block.
template <typename T>
__global__ void __launch_bounds__(256) batch_repack_kernel(const MatDesc *desc, const TileRef *list) {
    __shared__ T buf[32][33];
    const TileRef tr = list[blockIdx.x];
    const MatDesc d = desc[tr.m];
    const int nb = d.nb, nsb = (nb + 31) / 32;
    if ((int)blockIdx.y >= nsb * nsb) return;
    int I, K;
    tile_of(tr.t, I, K);
    const int sr = blockIdx.y / nsb, sc = blockIdx.y % nsb;
    T *tile = reinterpret_cast<T *>(d.store) + (size_t)tr.t * nb * nb;
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
        const int r = sr * 32 + threadIdx.x, c = sc * 32 + yy;
        const int64_t i = (int64_t)I * nb + r, j = (int64_t)K * nb + c;
        T v = T(0);
        if (r < nb && c < nb) {
            if (i < d.n && j < d.n) v = j <= i ? (T)d.A[j * d.lda + i] : T(0);
            else v = i == j ? T(1) : T(0);
        }
        buf[yy][threadIdx.x] = v;
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
        const int r = sr * 32 + yy, c = sc * 32 + threadIdx.x;
        if (r < nb && c < nb) tile[(size_t)r * nb + c] = buf[threadIdx.x][yy];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) batch_unpack_kernel(const MatDesc *desc, const TileRef *list) {
    __shared__ T buf[32][33];
    const TileRef tr = list[blockIdx.x];
    const MatDesc d = desc[tr.m];
    const int nb = d.nb, nsb = (nb + 31) / 32;
    if ((int)blockIdx.y >= nsb * nsb) return;
    int I, K;
    tile_of(tr.t, I, K);
    const int sr = blockIdx.y / nsb, sc = blockIdx.y % nsb;
    const T *tile = reinterpret_cast<const T *>(d.store) + (size_t)tr.t * nb * nb;
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
        const int r = sr * 32 + yy, c = sc * 32 + threadIdx.x;
        buf[yy][threadIdx.x] = (r < nb && c < nb) ? tile[(size_t)r * nb + c] : T(0);
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
        const int r = sr * 32 + threadIdx.x, c = sc * 32 + yy;
        const int64_t i = (int64_t)I * nb + r, j = (int64_t)K * nb + c;
        if (r < nb && c < nb && i < d.n && j < d.n && j <= i) d.A[j * d.lda + i] = (double)buf[threadIdx.x][yy];
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

}  // namespace chol
