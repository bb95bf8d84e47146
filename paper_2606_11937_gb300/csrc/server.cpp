// server.cpp -- continuous-batching SPD solve server.
//
// Requests (factor + solve, or solve against a resident factor) are queued in
// arrival order.  `slots` worker threads each own a CUDA stream; a request is
// admitted to a free slot as soon as its workspace fits in the device-memory
// budget (least-recently-used resident factors that no running request holds
// are evicted to make room), so requests that arrive while others run on the
// GPU start as slots and memory free up and their kernels overlap on the
// device.  Factors requested with a nonzero factor_id stay resident for
// repeat right-hand sides.  The tile order is a fixed function of (n,
// precision), so a request gives the same bits alone and in a mix.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/chol.h"

namespace chol {
void set_error(const char *fmt, ...);
int fp64_factor_store(int64_t n, const double *A, int64_t lda, const chol_opts &o, double **store_out,
                      int64_t *nb_out, int64_t *info);
int fp64_solve_store(const double *store, int64_t n, int64_t nb, double *X, int64_t ldx, int64_t nrhs,
                     cudaStream_t st, double timeout_s);
size_t fp64_store_bytes(int64_t n, int64_t nb);
size_t fp64tc_extra_bytes(int64_t n);
bool fp64_uses_tc(int64_t n, int64_t nb, int32_t flags);
size_t mixed_residual_keep_bytes(int64_t n);
size_t mixed_residual_ws_bytes(int64_t n, int64_t nrhs);
}  // namespace chol

using Clock = std::chrono::steady_clock;

namespace {

struct Resident {
    int64_t n = 0, nb = 0;
    int32_t precision = CHOL_FP64;
    double *store = nullptr;          // FP64 tile store
    chol_factor_h mixed = nullptr;    // mixed-precision handle (references the caller's A)
    size_t bytes = 0;
    int refs = 0;
    uint64_t last_use = 0;
    cudaStream_t stream = nullptr;    // stream the store was allocated on
};

struct Request {
    uint64_t ticket = 0;
    chol_request req{};
    Clock::time_point t_submit, t_admit, t_done;
    chol_result res{};
    bool done = false;
    size_t reserve = 0;
    int slot = -1;
    bool reuse = false;
    // produced by execution
    double *new_store = nullptr;
    int64_t new_nb = 0;
    chol_factor_h new_mixed = nullptr;
    size_t keep_bytes = 0;
};

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

int64_t tasks_of(int64_t M) { return M * (M + 1) * (M + 2) / 6; }

// FP64 requests of order above this factor with SYRK/GEMM/TRSM on the tensor
// cores (binary64 accuracy, tiles of 128); smaller ones on the FP64 pipe.
// Measured single factorizations (dataflow): n = 1024 3.5 ms on both engines,
// n = 1536 5.5 against 8.2 ms, n = 4096 15.6 against 31.5 ms.  A pure function
// of n, so a request gives the same bits alone and in a mix.
bool fp64_on_tensor_cores(int64_t n) { return chol::fp64_uses_tc(n, 0, 0); }
int64_t fp64_nb(int64_t n) { return fp64_on_tensor_cores(n) ? 128 : chol_default_nb(n, CHOL_FP64); }

// Persistent grid of a served factorization: the device's SMs shared among
// the slots (a served factorization of order <= 8192 is bound by its chain of
// diagonal-tile tasks more than by its updates, so the slots' chains overlap
// instead of each kernel holding every SM), and no more CTAs than tiles in
// the lower triangle (the widest a step of the task graph gets).  The bits do
// not depend on the grid (every tile receives its updates in the same order).
int served_grid(int64_t n, int64_t nb, int sms, int slots) {
    const int64_t M = (n + nb - 1) / nb, tiles = M * (M + 1) / 2;
    int64_t g = sms / (slots > 0 ? slots : 1);
    if (g < 8) g = 8;
    if (tiles < g) g = tiles < 4 ? 4 : tiles;
    return (int)g;
}

// upper bound of the device bytes a request needs while it runs
size_t need_bytes(const chol_request &r, bool reuse) {
    const int64_t n = r.n, nrhs = r.nrhs;
    const size_t solve_ws = 32768 + 2 * (size_t)((n + 63) / 64) * ((nrhs + 15) / 16) * 4 + 1024;
    if (r.precision == CHOL_FP64) {
        if (reuse) return a256(solve_ws);
        const int64_t nb = fp64_nb(n), M = (n + nb - 1) / nb;
        return chol::fp64_store_bytes(n, nb) + a256((size_t)tasks_of(M) * 20 + 1024) + a256(solve_ws) +
               (fp64_on_tensor_cores(n) ? chol::fp64tc_extra_bytes(n) : 0);
    }
    // refinement workspace, including the tensor-core residual's (its slices of
    // A are counted with the kept factor: the handle holds them once built)
    const size_t ir = a256((size_t)n * nrhs * 12 + (size_t)n * 8 + 3 * (size_t)nrhs * 8 + 1024) + a256(solve_ws) +
                      chol::mixed_residual_ws_bytes(n, nrhs);
    if (reuse) return ir;
    const int64_t nb = chol_default_nb(n, r.precision), M = (n + nb - 1) / nb;
    const size_t tiles = (size_t)M * (M + 1) / 2, te = (size_t)nb * nb;
    const size_t per = r.precision == CHOL_FP32 ? 12 : (r.precision == CHOL_TF32 ? 8 : 6);
    return tiles * te * per + (size_t)tasks_of(M) * 20 + ir + 4096 + chol::mixed_residual_keep_bytes(n);
}

size_t keep_bytes_of(const chol_request &r) {
    if (r.precision == CHOL_FP64) return chol::fp64_store_bytes(r.n, fp64_nb(r.n));
    const int64_t nb = chol_default_nb(r.n, r.precision), M = (r.n + nb - 1) / nb;
    return a256((size_t)M * (M + 1) / 2 * nb * nb * 4) + chol::mixed_residual_keep_bytes(r.n);
}

}  // namespace

struct chol_server_s {
    size_t budget = 0, in_use = 0;
    int nslots = 0;
    chol_opts opts{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> tickets;
    std::unordered_map<uint64_t, Resident> resident;
    std::unordered_set<uint64_t> creating;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    std::vector<Request *> slot_req;
    bool stop = false;
    uint64_t next_ticket = 1, use_clock = 0;
    int device = 0;
    int sms = 152;  // the device's SM count
    // statistics
    std::vector<double> lat_ms;
    int64_t completed = 0, failed = 0, rejected = 0;
    bool any_submit = false;
    Clock::time_point first_submit, last_done;

    void finish_locked(Request *r, int status) {
        r->res.status = status;
        r->t_done = Clock::now();
        r->res.latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
        r->done = true;
        if (status == CHOL_OK) {
            ++completed;
            lat_ms.push_back(r->res.latency_ms);
        } else if (status == CHOL_ERR_NOMEM) {
            ++rejected;
        } else {
            ++failed;
        }
        last_done = r->t_done;
        cv_done.notify_all();
    }

    bool evict_one_locked(uint64_t keep_id) {
        uint64_t best = 0, best_use = ~0ull;
        for (auto &kv : resident)
            if (kv.second.refs == 0 && kv.first != keep_id && kv.second.last_use < best_use) {
                best = kv.first;
                best_use = kv.second.last_use;
            }
        if (best_use == ~0ull) return false;
        Resident &f = resident[best];
        if (f.store) cudaFreeAsync(f.store, f.stream);
        if (f.mixed) chol_factor_free(f.mixed);
        in_use -= f.bytes;
        resident.erase(best);
        return true;
    }

    // Admit pending requests in arrival order while a slot is free and the budget allows.
    void admit_locked() {
        while (!pending.empty()) {
            int slot = -1;
            for (int s = 0; s < nslots; ++s)
                if (!slot_req[s]) {
                    slot = s;
                    break;
                }
            if (slot < 0) return;
            Request *r = pending.front();
            const uint64_t id = r->req.factor_id;
            r->reuse = r->req.A == nullptr;
            if (r->reuse) {
                if (creating.count(id)) return;  // its factor is still being computed: wait
                auto it = resident.find(id);
                if (id == 0 || it == resident.end() || it->second.precision != r->req.precision ||
                    it->second.n != r->req.n) {
                    pending.pop_front();
                    r->t_admit = Clock::now();
                    finish_locked(r, CHOL_ERR_HANDLE);
                    continue;
                }
            } else if (id != 0 && (creating.count(id) || resident.count(id))) {
                if (creating.count(id)) return;
                // a new factor replaces a resident one with the same id once nobody uses it
                Resident &old = resident[id];
                if (old.refs > 0) return;
                if (old.store) cudaFreeAsync(old.store, old.stream);
                if (old.mixed) chol_factor_free(old.mixed);
                in_use -= old.bytes;
                resident.erase(id);
            }
            const size_t need = need_bytes(r->req, r->reuse) + (r->reuse || id == 0 ? 0 : keep_bytes_of(r->req));
            while (in_use + need > budget && evict_one_locked(r->reuse ? id : 0)) {
            }
            if (in_use + need > budget) {
                bool busy = false;
                for (int s = 0; s < nslots; ++s) busy |= slot_req[s] != nullptr;
                if (busy) return;  // wait for running requests to free memory
                pending.pop_front();
                r->t_admit = Clock::now();
                chol::set_error("request needs %zu bytes, budget %zu", need, budget);
                finish_locked(r, CHOL_ERR_NOMEM);
                continue;
            }
            pending.pop_front();
            in_use += need;
            r->reserve = need;
            r->slot = slot;
            r->t_admit = Clock::now();
            r->res.queue_ms = std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
            r->res.slot = slot;
            if (r->reuse) {
                Resident &f = resident[id];
                f.refs++;
                f.last_use = ++use_clock;
            } else if (id != 0) {
                creating.insert(id);
            }
            slot_req[slot] = r;
            cv_work.notify_all();
        }
    }

    // Runs on the worker thread of the request's slot (no lock held).
    void execute(Request *r, cudaStream_t st, const Resident *f) {
        const chol_request &q = r->req;
        chol_opts o = opts;
        o.stream = st;
        o.precision = q.precision;
        o.nb = 0;
        o.schedule = CHOL_SCHED_DATAFLOW;
        o.num_ctas = served_grid(q.n, q.precision == CHOL_FP64 ? fp64_nb(q.n) : chol_default_nb(q.n, q.precision),
                                 sms, nslots);
        int rc = CHOL_OK;
        r->res.berr = -1.0;
        r->res.reused_factor = r->reuse ? 1 : 0;
        if (q.precision == CHOL_FP64) {
            const double *store = f ? f->store : nullptr;
            int64_t nb = f ? f->nb : 0;
            if (!r->reuse) {
                double *s = nullptr;
                int64_t info = 0;
                if (fp64_on_tensor_cores(q.n)) o.flags |= CHOL_FLAG_FP64_TC | CHOL_FLAG_PRIORITY;
                rc = chol::fp64_factor_store(q.n, q.A, q.lda, o, &s, &nb, &info);
                r->res.info = info;
                if (rc == CHOL_OK && info > 0) rc = CHOL_ERR_NOT_SPD;
                if (rc != CHOL_OK && s) {
                    cudaFreeAsync(s, st);
                    s = nullptr;
                }
                store = s;
                r->new_store = s;
                r->new_nb = nb;
            }
            if (rc == CHOL_OK) {
                if (cudaMemcpy2DAsync(q.X, q.ldx * 8, q.B, q.ldb * 8, q.n * 8, q.nrhs, cudaMemcpyDeviceToDevice, st) !=
                    cudaSuccess)
                    rc = CHOL_ERR_CUDA;
                else
                    rc = chol::fp64_solve_store(store, q.n, nb, q.X, q.ldx, q.nrhs, st, o.timeout_s);
            }
            if (!r->reuse && (q.factor_id == 0 || rc != CHOL_OK) && r->new_store) {
                cudaFreeAsync(r->new_store, st);
                cudaStreamSynchronize(st);
                r->new_store = nullptr;
            }
        } else {
            chol_factor_h h = f ? f->mixed : nullptr;
            if (!r->reuse) {
                int64_t info = 0;
                rc = chol_mixed_factor(q.n, q.A, q.lda, &o, &h, &info);
                r->res.info = info;
                if (rc == CHOL_OK && info > 0) rc = CHOL_ERR_NOT_SPD;
                r->new_mixed = rc == CHOL_OK ? h : nullptr;
                if (rc != CHOL_OK && h) {
                    chol_factor_free(h);
                    h = nullptr;
                }
            }
            if (rc == CHOL_OK) {
                int32_t it = 0;
                double be = -1;
                rc = chol_mixed_solve(h, q.nrhs, q.B, q.ldb, q.X, q.ldx, &it, &be);
                r->res.iters = it;
                r->res.berr = be;
            }
            if (!r->reuse && (q.factor_id == 0 || rc != CHOL_OK) && r->new_mixed) {
                chol_factor_free(r->new_mixed);
                r->new_mixed = nullptr;
            }
        }
        r->res.status = rc;
    }

    void worker(int slot) {
        cudaSetDevice(device);
        cudaStream_t st = streams[slot];
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv_work.wait(lk, [&] { return stop || slot_req[slot] != nullptr; });
            if (!slot_req[slot]) {
                if (stop) return;
                continue;
            }
            Request *r = slot_req[slot];
            const Resident *f = nullptr;
            Resident copy;
            if (r->reuse) {
                copy = resident[r->req.factor_id];
                f = &copy;
            }
            lk.unlock();
            execute(r, st, f);
            lk.lock();
            in_use -= r->reserve;
            const uint64_t id = r->req.factor_id;
            if (r->reuse) {
                auto it = resident.find(id);
                if (it != resident.end()) it->second.refs--;
            } else if (id != 0) {
                creating.erase(id);
                if (r->res.status == CHOL_OK && (r->new_store || r->new_mixed)) {
                    Resident nf;
                    nf.n = r->req.n;
                    nf.nb = r->new_nb;
                    nf.precision = r->req.precision;
                    nf.store = r->new_store;
                    nf.mixed = r->new_mixed;
                    nf.bytes = keep_bytes_of(r->req);
                    nf.last_use = ++use_clock;
                    nf.stream = st;
                    resident[id] = nf;
                    in_use += nf.bytes;
                }
            }
            slot_req[slot] = nullptr;
            finish_locked(r, r->res.status);
            admit_locked();
        }
    }
};

extern "C" {

int chol_server_create(size_t mem_budget_bytes, int32_t slots, const chol_opts *opts, chol_server_h *out) {
    if (!out) {
        chol::set_error("argument: out is NULL");
        return CHOL_ERR_ARG;
    }
    *out = nullptr;
    if (mem_budget_bytes == 0 || slots < 0 || slots > 64) {
        chol::set_error("argument: budget must be > 0 and slots in [0, 64]");
        return CHOL_ERR_ARG;
    }
    chol_server_s *s = new chol_server_s();
    s->budget = mem_budget_bytes;
    s->nslots = slots ? slots : 4;
    chol_opts_init(&s->opts);
    if (opts) s->opts = *opts;
    if (!(s->opts.refine_tol > 0)) s->opts.refine_tol = 1e-14;
    if (s->opts.max_iter <= 0) s->opts.max_iter = 30;
    if (!(s->opts.timeout_s > 0)) s->opts.timeout_s = 60.0;
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    s->slot_req.assign(s->nslots, nullptr);
    for (int i = 0; i < s->nslots; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            chol::set_error("cudaStreamCreate failed");
            for (auto x : s->streams) cudaStreamDestroy(x);
            delete s;
            return CHOL_ERR_CUDA;
        }
        s->streams.push_back(st);
    }
    for (int i = 0; i < s->nslots; ++i) s->workers.emplace_back([s, i] { s->worker(i); });
    *out = s;
    return CHOL_OK;
}

int chol_server_submit(chol_server_h s, const chol_request *req, uint64_t *ticket) {
    if (!s) {
        chol::set_error("invalid server handle");
        return CHOL_ERR_HANDLE;
    }
    if (!req || !ticket || req->n < 1 || req->nrhs < 1 || !req->B || !req->X || req->ldb < req->n ||
        req->ldx < req->n || (req->A && req->lda < req->n) || (!req->A && req->factor_id == 0) ||
        req->precision < CHOL_FP64 || req->precision > CHOL_FP16) {
        chol::set_error("argument: invalid request");
        return CHOL_ERR_ARG;
    }
    Request *r = new Request();
    r->req = *req;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->any_submit) {
        s->any_submit = true;
        s->first_submit = r->t_submit;
    }
    r->ticket = s->next_ticket++;
    s->tickets[r->ticket] = r;
    s->pending.push_back(r);
    *ticket = r->ticket;
    s->admit_locked();
    return CHOL_OK;
}

int chol_server_poll(chol_server_h s, uint64_t ticket, chol_result *res) {
    if (!s || !res) {
        chol::set_error("invalid server handle or result pointer");
        return CHOL_ERR_HANDLE;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        chol::set_error("unknown ticket %llu", (unsigned long long)ticket);
        return CHOL_ERR_HANDLE;
    }
    if (!it->second->done) return CHOL_ERR_BUSY;
    *res = it->second->res;
    delete it->second;
    s->tickets.erase(it);
    return CHOL_OK;
}

int chol_server_wait(chol_server_h s, uint64_t ticket, chol_result *res, double timeout_s) {
    if (!s || !res) {
        chol::set_error("invalid server handle or result pointer");
        return CHOL_ERR_HANDLE;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        chol::set_error("unknown ticket %llu", (unsigned long long)ticket);
        return CHOL_ERR_HANDLE;
    }
    Request *r = it->second;
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9);
    if (!s->cv_done.wait_until(lk, deadline, [&] { return r->done; })) return CHOL_ERR_BUSY;
    *res = r->res;
    s->tickets.erase(ticket);
    delete r;
    return CHOL_OK;
}

int chol_server_release(chol_server_h s, uint64_t factor_id) {
    if (!s) {
        chol::set_error("invalid server handle");
        return CHOL_ERR_HANDLE;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->resident.find(factor_id);
    if (it == s->resident.end()) {
        chol::set_error("factor %llu is not resident", (unsigned long long)factor_id);
        return CHOL_ERR_HANDLE;
    }
    if (it->second.refs > 0) return CHOL_ERR_BUSY;
    if (it->second.store) cudaFreeAsync(it->second.store, it->second.stream);
    if (it->second.mixed) chol_factor_free(it->second.mixed);
    s->in_use -= it->second.bytes;
    s->resident.erase(it);
    s->admit_locked();
    return CHOL_OK;
}

int chol_server_stats(chol_server_h s, chol_server_stats_t *st) {
    if (!s || !st) {
        chol::set_error("invalid server handle or stats pointer");
        return CHOL_ERR_HANDLE;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof(*st));
    st->completed = s->completed;
    st->failed = s->failed;
    st->rejected = s->rejected;
    st->resident_factors = (int64_t)s->resident.size();
    st->bytes_in_use = s->in_use;
    st->budget = s->budget;
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const size_t k = (size_t)std::min<double>(v.size() - 1, std::max(0.0, std::ceil(p * v.size()) - 1));
            return v[k];
        };
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        st->mean_ms = sum / v.size();
    }
    if (s->any_submit && s->completed > 0) {
        st->elapsed_s = std::chrono::duration<double>(s->last_done - s->first_submit).count();
        st->solves_per_s = st->elapsed_s > 0 ? s->completed / st->elapsed_s : 0;
    }
    return CHOL_OK;
}

void chol_server_destroy(chol_server_h s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // requests not yet admitted are dropped
        for (Request *r : s->pending) {
            r->t_admit = Clock::now();
            s->finish_locked(r, CHOL_ERR_HANDLE);
        }
        s->pending.clear();
        s->cv_work.notify_all();
    }
    for (auto &t : s->workers) t.join();
    for (auto &kv : s->resident) {
        if (kv.second.store) cudaFreeAsync(kv.second.store, kv.second.stream);
        if (kv.second.mixed) chol_factor_free(kv.second.mixed);
    }
    for (auto st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto &kv : s->tickets) delete kv.second;
    delete s;
}

}  // extern "C"
