// common.cuh -- shared definitions of the CUDA library: error reporting, tile
// geometry of the tile-major store, device-side control block and the memory
// ordering primitives the schedulers use.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/chol.h"

namespace chol {

// ----------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define CHOL_CUDA(call)                                                     \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return ::chol::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define CHOL_CHECK_ARG(cond, msg)                  \
    do {                                           \
        if (!(cond)) {                             \
            ::chol::set_error("argument: %s", msg); \
            return CHOL_ERR_ARG;                   \
        }                                          \
    } while (0)

// ----------------------------------------------------------------- options
chol_opts resolve_opts(const chol_opts *opts);
int num_sms();

// FP64 engine choice (factor.cu): the tensor-core engine by default above
// order kFp64TcMinN for tile orders that are multiples of 128 up to
// kFp64TcMaxNb; CHOL_FLAG_FP64_TC / CHOL_FLAG_FP64_SIMT force one engine.
constexpr int64_t kFp64TcMinN = 1024;
constexpr int64_t kFp64TcMaxNb = 2048;
bool fp64_uses_tc(int64_t n, int64_t nb, int32_t flags);

// ----------------------------------------------------------------- tile store
// Lower tiles (I, K), K <= I, of order nb, each stored contiguously and
// ROW-major inside (element (r, c) at r * nb + c); tile (I, K) has index
// I (I + 1) / 2 + K.  The ragged last block row / column is padded with the
// identity, so the padded matrix is diag(A, I) and its factor diag(L, I).
__host__ __device__ __forceinline__ int64_t tile_index(int64_t I, int64_t K) {
    return I * (I + 1) / 2 + K;
}
__host__ __device__ __forceinline__ int64_t num_tiles(int64_t M) { return M * (M + 1) / 2; }
__host__ __device__ __forceinline__ int64_t num_tasks(int64_t M) {
    return M * (M + 1) * (M + 2) / 6;
}
// Tasks are numbered along per-tile chains: the chain of tile (I, K) holds
// its K updates (J = 0 .. K-1: SYRK if I == K, else GEMM) followed by its
// final task at J = K (POTRF if I == K, else TRSM).
__host__ __device__ __forceinline__ int64_t task_id(int64_t I, int64_t K, int64_t J) {
    return I * (I + 1) * (I + 2) / 6 + K * (K + 1) / 2 + J;
}

enum TaskType : int32_t { T_POTRF = 0, T_TRSM = 1, T_SYRK = 2, T_GEMM = 3 };

__host__ __device__ __forceinline__ int32_t task_type(int64_t I, int64_t K, int64_t J) {
    if (J == K) return I == K ? T_POTRF : T_TRSM;
    return I == K ? T_SYRK : T_GEMM;
}
// number of predecessor tasks that must finish before (I, K, J) may run
__host__ __device__ __forceinline__ int32_t task_needs(int64_t I, int64_t K, int64_t J) {
    const int32_t prev = J > 0 ? 1 : 0;  // previous task in the tile's chain
    if (J == K) return I == K ? prev : 1 + prev;  // POTRF: chain; TRSM: POTRF(K) + chain
    return (I == K ? 1 : 2) + prev;               // SYRK: TRSM(I,J); GEMM: TRSM(I,J), TRSM(K,J)
}

// packed queue entry: J | K << 16 | I << 32 | matrix << 48 (all < 65536)
__host__ __device__ __forceinline__ uint64_t pack_task(int64_t m, int64_t I, int64_t K, int64_t J) {
    return (uint64_t)J | ((uint64_t)K << 16) | ((uint64_t)I << 32) | ((uint64_t)m << 48);
}
constexpr uint64_t kEmptySlot = ~0ull;

// ----------------------------------------------------------------- device control block
// One per factorization (or per batched launch), zeroed before the schedule runs.
struct Control {
    int64_t info;           // 0 or 1-based failing column (first failure wins)
    int32_t abort;          // set on failure or timeout: every CTA stops
    int32_t status;         // 0 or a chol_status (CHOL_ERR_TIMEOUT)
    unsigned long long tasks[4];
    unsigned long long head[2], tail[2];  // ready queues: [0] priority, [1] normal
    unsigned long long completed;         // tasks finished (termination test)
    unsigned long long trace_count;
    unsigned long long ticket;            // solve wavefront ticket
    int32_t timeout_where;                // debug: where a wait expired
    int32_t pad;
};

// ----------------------------------------------------------------- memory ordering
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t smid() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint64_t ld_acquire_u64(const unsigned long long *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int32_t ld_acquire_s32(const int32_t *p) {
    int32_t v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int32_t ld_relaxed_s32(const int32_t *p) {
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const unsigned long long *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_s32(int32_t *p, int32_t v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int32_t atom_add_acqrel_s32(int32_t *p, int32_t v) {
    int32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void nanosleep_ns(uint32_t ns) { asm volatile("nanosleep.u32 %0;" ::"r"(ns)); }

// Record a failing pivot (1-based column); the smallest column wins.
__device__ __forceinline__ void report_info(Control *ctl, int64_t col1) {
    unsigned long long *p = reinterpret_cast<unsigned long long *>(&ctl->info);
    unsigned long long cur = *p;
    while (cur == 0ull || (unsigned long long)col1 < cur) {
        const unsigned long long prev = atomicCAS(p, cur, (unsigned long long)col1);
        if (prev == cur) break;
        cur = prev;
    }
}

// Keep stream-ordered allocations pooled between calls (per device, once).
void prepare_pool();

}  // namespace chol
