// solve.cu -- FP64 SPD solve with a factor from chol_factor: forward then
// backward substitution (the use the paper motivates in Section 1).
#include <string.h>

#include "common.cuh"
#include "solve_impl.cuh"

using namespace chol;

extern "C" {

int chol_solve_ex(int64_t n, int64_t nrhs, const double *L, int64_t ldl, double *B, int64_t ldb,
                  const chol_opts *opts) {
    CHOL_CHECK_ARG(n >= 0 && nrhs >= 0, "n < 0 or nrhs < 0");
    CHOL_CHECK_ARG(ldl >= (n > 1 ? n : 1) && ldb >= (n > 1 ? n : 1), "ldl or ldb < max(1, n)");
    if (n == 0 || nrhs == 0) return CHOL_OK;
    CHOL_CHECK_ARG(L != nullptr && B != nullptr, "L or B is NULL");
    chol_opts o = resolve_opts(opts);
    cudaStream_t st = (cudaStream_t)o.stream;
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

}  // extern "C"
