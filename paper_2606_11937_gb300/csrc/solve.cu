// solve.cu -- FP64 SPD solve with a factor from chol_factor: forward then
// backward substitution (the use the paper motivates in Section 1).
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "solve_impl.cuh"

using namespace chol;

// ------------------------------------------------------------------ allocation-free solve
// Scratch of chol_solve_noalloc: the solve's control block (tickets, status)
// and its per-block ready flags, in device memory that exists as soon as the
// library is loaded on a device (every device that loads the library keeps
// these 4 MiB until the process exits).  Host code cannot use the symbol's
// name as a device address; the address is looked up once per device.
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
std::mutex g_noalloc_mu;
void *g_noalloc_addr[256] = {};
}  // namespace

namespace chol {

// X <- A^{-1} X with the factor held in a row-major FP64 tile store (server).
int fp64_solve_store(const double *store, int64_t n, int64_t nb, double *X, int64_t ldx, int64_t nrhs,
                     cudaStream_t st, double timeout_s) {
    void *ws = nullptr;
    CHOL_CUDA(cudaMallocAsync(&ws, solve_ws_bytes(n, nrhs), st));
    int rc = launch_solve<double, TileMajorL<double>>(TileMajorL<double>{store, nb}, X, ldx, n, nrhs, ws, timeout_s,
                                                      st);
    int32_t h[2] = {0, 0};
    if (rc == CHOL_OK) {
        if (cudaMemcpyAsync(h, ws, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = cuda_fail(cudaGetLastError(), "solve readback", __FILE__, __LINE__);
        else if (h[0]) {
            set_error("solve: device-side wait expired (site %d)", h[1]);
            rc = h[0];
        }
    }
    cudaFreeAsync(ws, st);
    return rc;
}

}  // namespace chol

extern "C" {

int chol_solve_ex(int64_t n, int64_t nrhs, const double *L, int64_t ldl, double *B, int64_t ldb,
                  const chol_opts *opts) {
    CHOL_CHECK_ARG(n >= 0 && nrhs >= 0, "n < 0 or nrhs < 0");
    CHOL_CHECK_ARG(ldl >= (n > 1 ? n : 1) && ldb >= (n > 1 ? n : 1), "ldl or ldb < max(1, n)");
    if (n == 0 || nrhs == 0) return CHOL_OK;
    CHOL_CHECK_ARG(L != nullptr && B != nullptr, "L or B is NULL");
    chol_opts o = resolve_opts(opts);
    cudaStream_t st = (cudaStream_t)o.stream;
    cudaGetLastError();  // errors left by earlier, unrelated runtime calls are not ours to report
    prepare_pool();
    void *ws = nullptr;
    const size_t bytes = solve_ws_bytes(n, nrhs);
    CHOL_CUDA(cudaMallocAsync(&ws, bytes, st));
    int rc = launch_solve<double, ColMajorL<double>>(ColMajorL<double>{L, ldl}, B, ldb, n, nrhs, ws, o.timeout_s, st);
    SolveCtl h;
    if (rc == CHOL_OK) {
        if (cudaMemcpyAsync(&h, ws, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = cuda_fail(cudaGetLastError(), "solve readback", __FILE__, __LINE__);
        else if (h.status) {
            set_error("solve: device-side wait expired (site %d)", h.where);
            rc = h.status;
        }
    }
    cudaFreeAsync(ws, st);
    return rc;
}

int chol_solve(int64_t n, int64_t nrhs, const double *L, double *B) {
    return chol_solve_ex(n, nrhs, L, n > 1 ? n : 1, B, n > 1 ? n : 1, nullptr);
}

int chol_solve_noalloc(int64_t n, int64_t nrhs, const double *L, int64_t ldl, double *B, int64_t ldb,
                       void *stream) {
    CHOL_CHECK_ARG(n >= 0 && nrhs >= 0, "n < 0 or nrhs < 0");
    CHOL_CHECK_ARG(ldl >= (n > 1 ? n : 1) && ldb >= (n > 1 ? n : 1), "ldl or ldb < max(1, n)");
    if (n == 0 || nrhs == 0) return CHOL_OK;
    CHOL_CHECK_ARG(L != nullptr && B != nullptr, "L or B is NULL");
    const size_t need = solve_ws_bytes(n, nrhs);
    if (need > kNoAllocScratchBytes) {
        set_error("argument: chol_solve_noalloc needs %zu bytes of scratch for n=%lld, nrhs=%lld; its fixed "
                  "scratch holds %zu bytes (use chol_solve_ex)",
                  need, (long long)n, (long long)nrhs, kNoAllocScratchBytes);
        return CHOL_ERR_ARG;
    }
    int dev = 0;
    CHOL_CUDA(cudaGetDevice(&dev));
    CHOL_CHECK_ARG(dev >= 0 && dev < 256, "device ordinal out of range");
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            // first call on this device: look up the device address of the array
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
            g_noalloc_addr[dev] = p;
        }
        scratch = g_noalloc_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaGetLastError();  // errors left by earlier, unrelated runtime calls are not ours to report
    // launch_solve clears the control block and flags it uses before the sweeps
    int rc = launch_solve<double, ColMajorL<double>>(ColMajorL<double>{L, ldl}, B, ldb, n, nrhs, scratch, 60.0, st);
    int32_t h[2] = {0, 0};
    if (rc == CHOL_OK && cudaMemcpyAsync(h, scratch, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), "solve readback", __FILE__, __LINE__);
    // whatever happened, return only once the work queued on the stream has
    // finished: a caller that retries after an error must not overlap kernels
    // of this call that still write B and the shared scratch
    const cudaError_t es = cudaStreamSynchronize(st);
    if (rc != CHOL_OK) return rc;
    if (es != cudaSuccess) return cuda_fail(es, "solve sync", __FILE__, __LINE__);
    if (h[0]) {
        set_error("solve: device-side wait expired (site %d)", h[1]);
        return h[0];
    }
    return CHOL_OK;
}

}  // extern "C"
