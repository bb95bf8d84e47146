// runtime.cu -- error reporting, option defaults, device queries.
#include <stdarg.h>
#include <string.h>

#include <mutex>

#include "common.cuh"

namespace chol {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
    return CHOL_ERR_CUDA;
}

chol_opts resolve_opts(const chol_opts *opts) {
    chol_opts o;
    chol_opts_init(&o);
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = 30;
    if (!(o.refine_tol > 0.0)) o.refine_tol = 1e-14;
    if (!(o.timeout_s > 0.0)) o.timeout_s = 60.0;
    return o;
}

int num_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

// Keep stream-ordered allocations in the device's default pool between calls
// (the pool would otherwise release them at every synchronization).
void prepare_pool() {
    static std::once_flag once[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::call_once(once[dev], [dev]() {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

}  // namespace chol

extern "C" {

void chol_opts_init(chol_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->schedule = CHOL_SCHED_AUTO;
    o->precision = CHOL_FP64;
    o->nb = 0;
    o->flags = 0;
    o->max_iter = 30;
    o->refine_tol = 1e-14;
    o->timeout_s = 60.0;
    o->stream = nullptr;
    o->num_ctas = 0;
    o->trace = nullptr;
    o->trace_capacity = 0;
}

const char *chol_last_error(void) { return chol::g_err; }

const char *chol_version(void) { return "gb300-cholesky 0.1 (sm_103a)"; }

}  // extern "C"

extern "C" int chol_test_device_memory(uint64_t *free_bytes, uint64_t *pool_used, uint64_t *pool_reserved) {
    CHOL_CHECK_ARG(free_bytes && pool_used && pool_reserved, "NULL pointer");
    int dev = 0;
    CHOL_CUDA(cudaGetDevice(&dev));
    size_t fr = 0, tot = 0;
    CHOL_CUDA(cudaMemGetInfo(&fr, &tot));
    cudaMemPool_t pool;
    CHOL_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t used = 0, res = 0;
    CHOL_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
    CHOL_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &res));
    *free_bytes = fr;
    *pool_used = used;
    *pool_reserved = res;
    return CHOL_OK;
}
