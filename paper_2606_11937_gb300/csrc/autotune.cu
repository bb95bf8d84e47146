// autotune.cu -- tile order and schedule selection.
//
// chol_default_nb is a fixed table (a pure function of n and precision), so
// the batched and served paths give a matrix the same nb alone and in a mix.
// chol_autotune replaces the paper's manual tile-size sweep (Section 4.1):
// it times candidate (nb, schedule) pairs on a synthetic SPD matrix of the
// requested order and keeps the fastest, cached per (device, precision,
// power-of-two bucket of n) in memory and optionally in a JSON file.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace {

// A(i, j) = exp(-((i - j) / (0.05 n))^2 / 2) + delta_ij: a Gaussian kernel on
// equispaced points (positive semidefinite) plus the identity.
__global__ void synth_spd_kernel(double *A, int64_t n) {
    const int64_t total = n * n;
    const double s = 0.05 * (double)n + 1.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, j = e / n;
        const double d = (double)(i - j) / s;
        A[e] = exp(-0.5 * d * d) + (i == j ? 1.0 : 0.0);
    }
}

struct Entry {
    int64_t nb;
    int32_t schedule;
    double ms;
};

std::mutex g_mu;
std::map<std::string, Entry> g_cache;

std::string device_name() {
    int dev = 0;
    cudaDeviceProp p;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    return p.name;
}

int64_t bucket(int64_t n) {
    int64_t b = 1;
    while (b < n) b <<= 1;
    return b;
}

std::string key_of(int64_t n, int32_t precision) {
    return device_name() + "|p" + std::to_string(precision) + "|n" + std::to_string(bucket(n));
}

// minimal reader/writer of {"entries": [{"key": "...", "nb": N, "schedule": S, "ms": T}, ...]}
void load_file(const char *path) {
    FILE *f = fopen(path, "r");
    if (!f) return;
    std::string s;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, k);
    fclose(f);
    size_t pos = 0;
    while ((pos = s.find("\"key\"", pos)) != std::string::npos) {
        const size_t q0 = s.find('"', s.find(':', pos) + 1);
        const size_t q1 = s.find('"', q0 + 1);
        if (q0 == std::string::npos || q1 == std::string::npos) break;
        const std::string key = s.substr(q0 + 1, q1 - q0 - 1);
        Entry e{0, CHOL_SCHED_DATAFLOW, 0.0};
        const size_t pnb = s.find("\"nb\"", q1), psc = s.find("\"schedule\"", q1), pms = s.find("\"ms\"", q1);
        if (pnb == std::string::npos || psc == std::string::npos || pms == std::string::npos) break;
        e.nb = atoll(s.c_str() + s.find(':', pnb) + 1);
        e.schedule = atoi(s.c_str() + s.find(':', psc) + 1);
        e.ms = atof(s.c_str() + s.find(':', pms) + 1);
        if (e.nb > 0 && !g_cache.count(key)) g_cache[key] = e;
        pos = q1;
    }
}

void save_file(const char *path) {
    FILE *f = fopen(path, "w");
    if (!f) return;
    fprintf(f, "{\"entries\": [\n");
    size_t i = 0;
    for (auto &kv : g_cache)
        fprintf(f, "  {\"key\": \"%s\", \"nb\": %lld, \"schedule\": %d, \"ms\": %.6f}%s\n", kv.first.c_str(),
                (long long)kv.second.nb, kv.second.schedule, kv.second.ms, ++i < g_cache.size() ? "," : "");
    fprintf(f, "]}\n");
    fclose(f);
}

}  // namespace

using namespace chol;

extern "C" {

int64_t chol_default_nb(int64_t n, int32_t precision) {
    if (precision == CHOL_FP64) {
        // binary64 runs on the CUDA cores at a low per-SM rate: small tiles
        // shorten the POTRF->TRSM->SYRK critical path, which dominates small n
        if (n <= 1024) return 32;
        if (n <= 4096) return 64;
        if (n <= 16384) return 128;
        return 256;
    }
    // tensor-core precisions: tiles are multiples of the 128-row MMA; 128
    // keeps the critical path short (binary64 POTRF in shared memory) up to
    // order 32768, larger orders amortise per-task costs over 256 tiles
    if (n <= 32768) return 128;
    if (n <= 65536) return 256;
    return 512;
}

int chol_autotune(int64_t n, int32_t precision, const char *cache_path, double budget_s, chol_opts *opts_out) {
    CHOL_CHECK_ARG(opts_out != nullptr, "opts_out is NULL");
    CHOL_CHECK_ARG(n >= 1 && n <= 65536, "n must be in [1, 65536]");
    CHOL_CHECK_ARG(precision >= CHOL_FP64 && precision <= CHOL_FP16, "unknown precision");
    if (!(budget_s > 0)) budget_s = 5.0;
    const std::string key = key_of(n, precision);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (cache_path) load_file(cache_path);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            chol_opts_init(opts_out);
            opts_out->precision = precision;
            opts_out->nb = it->second.nb;
            opts_out->schedule = it->second.schedule;
            return CHOL_OK;
        }
    }
    std::vector<int64_t> nbs;
    if (precision == CHOL_FP64) {
        // 32 and 64 run on the DFMA engine; multiples of 128 above order 1024
        // on the tensor-core engine (the default engine is a function of n, nb)
        for (int64_t c : {32, 64, 128, 256, 512, 1024})
            if (c <= n || nbs.empty()) nbs.push_back(c);
    } else {
        for (int64_t c : {128, 256, 512})
            if (c <= n || nbs.empty()) nbs.push_back(c);
    }
    const int32_t scheds[2] = {CHOL_SCHED_DATAFLOW, CHOL_SCHED_FORK_JOIN};
    double *A = nullptr, *W = nullptr;
    CHOL_CUDA(cudaMalloc(&A, (size_t)n * n * 8));
    if (cudaMalloc(&W, (size_t)n * n * 8) != cudaSuccess) {
        cudaFree(A);
        set_error("autotune: allocation failed");
        return CHOL_ERR_NOMEM;
    }
    synth_spd_kernel<<<1024, 256>>>(A, n);
    Entry best{0, CHOL_SCHED_DATAFLOW, 1e300};
    const auto t_start = std::chrono::steady_clock::now();
    int rc = CHOL_OK;
    for (int64_t nb : nbs) {
        for (int32_t sc : scheds) {
            chol_opts o;
            chol_opts_init(&o);
            o.nb = nb;
            o.schedule = sc;
            o.precision = precision;
            double ms = 1e300;
            for (int rep = 0; rep < 2; ++rep) {  // the first run warms up
                cudaMemcpy(W, A, (size_t)n * n * 8, cudaMemcpyDeviceToDevice);
                chol_stats st;
                int64_t info = 0;
                const auto t0 = std::chrono::steady_clock::now();
                if (precision == CHOL_FP64) {
                    rc = chol_factor_ex(n, W, n, &o, &info, &st);
                } else {
                    chol_factor_h h = nullptr;
                    rc = chol_mixed_factor(n, W, n, &o, &h, &info);
                    chol_factor_free(h);
                }
                const double t = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
                if (rc != CHOL_OK) break;
                ms = t < ms ? t : ms;
            }
            if (rc != CHOL_OK) break;
            if (ms < best.ms) best = Entry{nb, sc, ms};
            const double spent = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
            if (spent > budget_s) break;
        }
        if (rc != CHOL_OK) break;
        const double spent = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if (spent > budget_s) break;
    }
    cudaFree(A);
    cudaFree(W);
    if (rc != CHOL_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = best;
        if (cache_path) save_file(cache_path);
    }
    chol_opts_init(opts_out);
    opts_out->precision = precision;
    opts_out->nb = best.nb;
    opts_out->schedule = best.schedule;
    return CHOL_OK;
}

}  // extern "C"
