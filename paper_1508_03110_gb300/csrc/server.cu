// Serving scheduler: continuous batching of fold-in requests (Eq. (3) for new
// users against a fixed M) and admission of small factorisation jobs by
// device-memory budget.  One worker thread drives everything on its own CUDA
// streams; no device code waits on the host (no spinning kernels):
//   * fold-in: pending requests are packed into pinned staging slots, copied
//     to the device, solved by the same per-row sweep kernels as a half
//     sweep (one CTA per request row), and copied back; `slots` batches can
//     be in flight, so requests arriving while batches run join the next one;
//   * jobs: admitted in arrival order while they fit the budget and the job
//     limit; each has its own context and stream and advances one ALS-NCG
//     iteration (a CUDA graph replay) whenever its previous one completed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    std::vector<int32_t> items;
    std::vector<float> vals;
    clk::time_point t0, t1;
    std::vector<float> result;
    bool done = false;
    als_status status = ALS_OK;
};

struct Job {
    int64_t ticket = 0;
    als_config cfg;
    int64_t n_u = 0, n_m = 0;
    std::vector<int32_t> rows, cols;
    std::vector<float> vals;
    std::vector<double> x0;
    int32_t iters = 0, done_iters = 0;
    size_t bytes = 0;
    als_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    clk::time_point t0, t1;
    std::vector<double> result;
    bool done = false, running = false;
    als_status status = ALS_OK;
    std::string error;
};

struct Slot {
    int *dflag = nullptr, *hflag = nullptr;  // [0] rows not SPD, [1] bounded wait expired
    int64_t *hptr = nullptr, *dptr = nullptr;
    int32_t *hidx = nullptr, *didx = nullptr;
    float *hval = nullptr, *dval = nullptr;
    void *hout = nullptr, *dout = nullptr;
    int32_t *horder = nullptr, *dorder = nullptr;  // the batch's requests by descending degree
    cudaEvent_t ev = nullptr;
    std::vector<Request *> reqs;
    bool busy = false;
};

size_t estimate_job_bytes(const als_config &cfg, int64_t n_u, int64_t n_m, int64_t nnz) {
    const int ld = (cfg.n_f + 3) & ~3;
    const size_t esz = cfg.precision == ALS_FP64 ? 8 : 4;
    const size_t rows = (size_t)(n_u + n_m);
    size_t b = (size_t)nnz * (24 + 24);        // both orders + builder scratch
    b += rows * ld * esz * 7 + rows * ld * 8;  // x, xbar, gbar, g0, g1, p, staging
    b += rows * 5 * 8 + rows * 4 * 2;          // row terms, degree orders
    if (cfg.precision == ALS_MIXED && cfg.n_f > 32) b += (size_t)std::max(n_u, n_m) * 2 * ALS_TC_LD * 2;
    return b + (4u << 20);
}

}  // namespace

struct als_server {
    als_ctx *model = nullptr;
    als_server_config cfg;
    cudaStream_t stream = nullptr;
    int *dflags = nullptr;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;    // worker wake-up
    std::condition_variable done;  // completion notifications
    std::thread worker;
    bool stop = false;
    int64_t next_ticket = 1;
    std::deque<Request *> pending;
    std::map<int64_t, Request *> reqs;
    std::deque<Job *> pending_jobs;
    std::vector<Job *> running;
    std::map<int64_t, Job *> jobs;
    size_t budget_used = 0;
    std::vector<double> latencies;
    clk::time_point t_first, t_last;
    bool have_first = false;
    als_status fatal = ALS_OK;
};

namespace {

void complete_batch(als_server *s, Slot &sl) {
    const int nf = s->model->nf, ld = s->model->ld;
    const bool f64 = s->model->f64;
    const auto now = clk::now();
    const als_status st = sl.hflag[1] ? ALS_ETIMEOUT : ALS_OK;
    for (size_t q = 0; q < sl.reqs.size(); ++q) {
        Request *r = sl.reqs[q];
        r->status = st;
        r->result.resize(nf);
        for (int k = 0; k < nf; ++k)
            r->result[k] = f64 ? (float)((const double *)sl.hout)[q * ld + k] : ((const float *)sl.hout)[q * ld + k];
        r->t1 = now;
        r->done = true;
        s->latencies.push_back(std::chrono::duration<double>(r->t1 - r->t0).count());
        s->t_last = now;
    }
    sl.reqs.clear();
    sl.busy = false;
}

// pack pending requests into a free slot and launch its batch (lock held)
bool launch_batch(als_server *s, Slot &sl) {
    als_ctx *c = s->model;
    int64_t nreq = 0, nrat = 0;
    sl.hptr[0] = 0;
    while (!s->pending.empty() && nreq < s->cfg.max_batch) {
        Request *r = s->pending.front();
        const int64_t n = (int64_t)r->items.size();
        if (nreq > 0 && nrat + n > s->cfg.max_batch_ratings) break;
        std::memcpy(sl.hidx + nrat, r->items.data(), n * sizeof(int32_t));
        std::memcpy(sl.hval + nrat, r->vals.data(), n * sizeof(float));
        nrat += n;
        sl.hptr[++nreq] = nrat;
        sl.reqs.push_back(r);
        s->pending.pop_front();
    }
    if (nreq == 0) return false;
    cudaMemsetAsync(sl.dflag, 0, 2 * sizeof(int), s->stream);
    cudaMemcpyAsync(sl.dptr, sl.hptr, (nreq + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s->stream);
    if (nrat > 0) {
        cudaMemcpyAsync(sl.didx, sl.hidx, nrat * sizeof(int32_t), cudaMemcpyHostToDevice, s->stream);
        cudaMemcpyAsync(sl.dval, sl.hval, nrat * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    }
    // requests by descending degree (ties by arrival), as the sweep orders
    // rows: the heaviest take the prefetching tensor-core kernel, the
    // lightest (at most min(dual_max, n_f) ratings, lambda > 0, mixed form)
    // the light-row solve through their n_i x n_i matrix
    int64_t npf = 0, ndual = 0, nsmall = 0;
    const int T = std::min(c->dual_max, c->nf);
    const bool dual = c->use_tc && !c->f64 && c->cfg.lambda > 0.0 && T > 0;
    for (int64_t q = 0; q < nreq; ++q) sl.horder[q] = (int32_t)q;
    std::stable_sort(sl.horder, sl.horder + nreq, [&](int32_t x, int32_t y) {
        return sl.hptr[x + 1] - sl.hptr[x] > sl.hptr[y + 1] - sl.hptr[y];
    });
    for (int64_t q = 0; q < nreq; ++q) {
        const int64_t d = sl.hptr[sl.horder[q] + 1] - sl.hptr[sl.horder[q]];
        if (d >= ALS_TC_PF_MIN) ++npf;
        if (dual && d <= T) ++ndual;
        if (dual && d <= std::min(T, ALS_DUAL_SMALL)) ++nsmall;
    }
    cudaMemcpyAsync(sl.dorder, sl.horder, nreq * sizeof(int32_t), cudaMemcpyHostToDevice, s->stream);
    SweepArgs a;
    a.ptr = sl.dptr;
    a.idx = sl.didx;
    a.val = sl.dval;
    a.order = sl.dorder;
    a.nrows = nreq;
    a.npf = npf;
    a.ndual = ndual;
    a.ndual_small = nsmall;
    a.dual_nmax = dual ? T : 0;
    a.F = (const char *)c->X + (size_t)c->n_u * c->ld * c->esz;
    a.nF = c->n_m;
    a.Xin = nullptr;
    a.Xout = sl.dout;
    a.Gbar = nullptr;
    a.nf = c->nf;
    a.ld = c->ld;
    a.lambda = c->cfg.lambda;
    a.refine = c->cfg.refine_steps + 1;
    a.notspd = sl.dflag;
    a.timeout = sl.dflag + 1;
    a.stream = s->stream;
    if (launch_sweep(c, a, c->f64, c->use_tc) != ALS_OK) {
        for (Request *r : sl.reqs) {
            r->status = ALS_ECUDA;
            r->t1 = clk::now();
            r->done = true;
        }
        sl.reqs.clear();
        return true;  // progress: the requests are answered (with an error)
    }
    cudaMemcpyAsync(sl.hout, sl.dout, (size_t)nreq * c->ld * c->esz, cudaMemcpyDeviceToHost, s->stream);
    cudaMemcpyAsync(sl.hflag, sl.dflag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    cudaEventRecord(sl.ev, s->stream);
    sl.busy = true;
    return true;
}

void finish_job(als_server *s, Job *j, als_status st) {
    if (st == ALS_OK && j->ctx) {
        const int nf = j->cfg.n_f;
        std::vector<double> U((size_t)j->n_u * nf), M((size_t)j->n_m * nf);
        st = als_get_factors(j->ctx, U.data(), M.data(), ALS_DT_F64, 0);
        if (st == ALS_OK) {
            j->result = U;
            j->result.insert(j->result.end(), M.begin(), M.end());
        } else {
            j->error = als_last_error();
        }
    }
    if (j->ctx) als_destroy(j->ctx);
    j->ctx = nullptr;
    if (j->ev) cudaEventDestroy(j->ev);
    if (j->stream) cudaStreamDestroy(j->stream);
    j->ev = nullptr;
    j->stream = nullptr;
    j->t1 = clk::now();
    j->status = st;
    j->done = true;
    j->running = false;
    s->budget_used -= j->bytes;
}

void start_job(als_server *s, Job *j) {
    j->running = true;
    s->budget_used += j->bytes;
    als_status st = ALS_OK;
    if (cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        finish_job(s, j, ALS_ECUDA);
        return;
    }
    j->cfg.alloc = nullptr;   // jobs allocate with cudaMalloc on the worker thread
    j->cfg.free = nullptr;
    st = als_create(&j->cfg, j->n_u, j->n_m, (int64_t)j->vals.size(), j->rows.data(), nullptr, j->cols.data(),
                    j->vals.data(), 0, j->stream, &j->ctx);
    if (st == ALS_OK) {
        const size_t nf = j->cfg.n_f;
        st = als_set_factors(j->ctx, j->x0.data(), j->x0.data() + (size_t)j->n_u * nf, ALS_DT_F64, 0);
    }
    if (st == ALS_OK && j->iters > 0) st = alsncg_step(j->ctx, nullptr);
    if (st != ALS_OK) {
        j->error = als_last_error();
        finish_job(s, j, st);
        return;
    }
    if (j->iters == 0) {
        finish_job(s, j, ALS_OK);
        return;
    }
    cudaEventRecord(j->ev, j->stream);
}

void worker_main(als_server *s) {
    cudaSetDevice(s->model->dev);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool progress = false;
        // fold-in batches: harvest finished ones, launch new ones
        for (Slot &sl : s->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaSuccess) {
                complete_batch(s, sl);
                progress = true;
            } else if (q != cudaErrorNotReady) {  // a failed batch: report, never poll forever
                cudaGetLastError();
                for (Request *r : sl.reqs) {
                    r->status = ALS_ECUDA;
                    r->t1 = clk::now();
                    r->done = true;
                }
                sl.reqs.clear();
                sl.busy = false;
                progress = true;
            }
        }
        for (Slot &sl : s->slots) {
            if (!sl.busy && !s->pending.empty()) progress |= launch_batch(s, sl);
        }
        // jobs: advance running ones, admit pending ones
        for (size_t i = 0; i < s->running.size();) {
            Job *j = s->running[i];
            const cudaError_t q = cudaEventQuery(j->ev);
            if (q != cudaSuccess && q != cudaErrorNotReady) {
                cudaGetLastError();
                j->error = cudaGetErrorString(q);
                finish_job(s, j, ALS_ECUDA);
                s->running.erase(s->running.begin() + (long)i);
                progress = true;
                continue;
            }
            if (q == cudaSuccess) {
                progress = true;
                if (++j->done_iters >= j->iters) {
                    finish_job(s, j, ALS_OK);
                    s->running.erase(s->running.begin() + (long)i);
                    continue;
                }
                const als_status st = alsncg_step(j->ctx, nullptr);
                if (st != ALS_OK) {
                    j->error = als_last_error();
                    finish_job(s, j, st);
                    s->running.erase(s->running.begin() + (long)i);
                    continue;
                }
                cudaEventRecord(j->ev, j->stream);
            }
            ++i;
        }
        while (!s->pending_jobs.empty() && (int)s->running.size() < s->cfg.max_jobs) {
            Job *j = s->pending_jobs.front();
            if (s->cfg.hbm_budget_bytes && s->budget_used + j->bytes > s->cfg.hbm_budget_bytes) break;
            s->pending_jobs.pop_front();
            start_job(s, j);
            if (j->running) s->running.push_back(j);
            progress = true;
        }
        if (progress) s->done.notify_all();
        bool busy = !s->pending.empty() || !s->running.empty() || !s->pending_jobs.empty();
        for (Slot &sl : s->slots) busy |= sl.busy;
        if (s->stop && !busy) break;
        if (!progress) {
            // poll in-flight work every 50 us; sleep until woken when idle
            if (busy) s->cv.wait_for(lk, std::chrono::microseconds(50));
            else s->cv.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
}

}  // namespace

extern "C" void als_server_config_default(als_server_config *cfg) {
    if (!cfg) return;
    cfg->max_batch = 256;
    cfg->max_batch_ratings = 1 << 20;
    cfg->slots = 4;
    cfg->max_jobs = 4;
    cfg->hbm_budget_bytes = 0;
}

extern "C" als_status als_server_create(als_ctx *model, const als_server_config *cfg_in, als_server **out) {
    if (!model || !out) { als_set_error("als_server_create: bad argument"); return ALS_EINVAL; }
    *out = nullptr;
    als_server_config cfg;
    als_server_config_default(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if (cfg.max_batch < 1 || cfg.max_batch_ratings < 1 || cfg.slots < 1 || cfg.slots > 64 || cfg.max_jobs < 0) {
        als_set_error("als_server_create: bad configuration");
        return ALS_EINVAL;
    }
    als_server *s = new als_server();
    s->model = model;
    s->cfg = cfg;
    auto fail = [&](als_status st, const char *msg) {
        als_set_error(std::string("als_server_create: ") + msg);
        als_server_destroy(s);
        return st;
    };
    if (cudaSetDevice(model->dev) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(ALS_ECUDA, "stream creation failed");
    }
    const size_t ob = (size_t)cfg.max_batch * model->ld * model->esz;
    // the model's pending work (its factors) must be finished before the
    // server's stream reads M
    if (cudaStreamSynchronize(model->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(ALS_ECUDA, "model stream failed");
    }
    if (cudaMalloc(&s->dflags, 2 * (size_t)cfg.slots * sizeof(int)) != cudaSuccess ||
        cudaMemsetAsync(s->dflags, 0, 2 * (size_t)cfg.slots * sizeof(int), s->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(ALS_ENOMEM, "device allocation failed");
    }
    s->slots.resize(cfg.slots);
    for (size_t i = 0; i < s->slots.size(); ++i) {
        Slot &sl = s->slots[i];
        sl.dflag = s->dflags + 2 * i;
        if (cudaMallocHost(&sl.hflag, 2 * sizeof(int)) != cudaSuccess || cudaMallocHost(&sl.hptr, (cfg.max_batch + 1) * sizeof(int64_t)) != cudaSuccess ||
            cudaMallocHost(&sl.hidx, cfg.max_batch_ratings * sizeof(int32_t)) != cudaSuccess ||
            cudaMallocHost(&sl.hval, cfg.max_batch_ratings * sizeof(float)) != cudaSuccess ||
            cudaMallocHost(&sl.hout, ob) != cudaSuccess || cudaMallocHost(&sl.horder, cfg.max_batch * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&sl.dorder, cfg.max_batch * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&sl.dptr, (cfg.max_batch + 1) * sizeof(int64_t)) != cudaSuccess ||
            cudaMalloc(&sl.didx, cfg.max_batch_ratings * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&sl.dval, cfg.max_batch_ratings * sizeof(float)) != cudaSuccess || cudaMalloc(&sl.dout, ob) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return fail(ALS_ENOMEM, "batch buffer allocation failed");
        }
    }
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(ALS_ECUDA, "set-up failed");
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return ALS_OK;
}

namespace {
// enqueue one fold-in request whose arrival time is t0
als_status submit_foldin_at(als_server *s, int64_t n, const int32_t *items, const float *vals, int64_t *ticket,
                            clk::time_point t0);
}  // namespace

extern "C" als_status als_server_submit_foldin(als_server *s, int64_t n, const int32_t *items, const float *vals,
                                               int64_t *ticket) {
    if (!s || n < 0 || (n > 0 && (!items || !vals)) || !ticket) {
        als_set_error("als_server_submit_foldin: bad argument");
        return ALS_EINVAL;
    }
    return submit_foldin_at(s, n, items, vals, ticket, clk::now());
}

extern "C" als_status als_server_replay(als_server *s, int64_t n_req, const double *t_arrival,
                                        const int64_t *req_ptr, const int32_t *items, const float *vals,
                                        int64_t *tickets, double *max_lag_s) {
    if (!s || n_req < 0 || (n_req > 0 && (!t_arrival || !req_ptr || !tickets))) {
        als_set_error("als_server_replay: bad argument");
        return ALS_EINVAL;
    }
    for (int64_t q = 0; q < n_req; ++q) {
        if (!(t_arrival[q] >= 0.0) || (q > 0 && t_arrival[q] < t_arrival[q - 1]) || req_ptr[q + 1] < req_ptr[q] ||
            req_ptr[0] != 0) {
            als_set_error("als_server_replay: arrival times must be >= 0 and non-decreasing, req_ptr non-decreasing from 0");
            return ALS_EINVAL;
        }
    }
    const clk::time_point start = clk::now();
    double lag = 0.0;
    for (int64_t q = 0; q < n_req; ++q) {
        const clk::time_point due = start + std::chrono::duration_cast<clk::duration>(
                                                std::chrono::duration<double>(t_arrival[q]));
        clk::time_point now = clk::now();
        while (now < due) now = clk::now();   // open loop: arrivals do not wait for answers
        lag = std::max(lag, std::chrono::duration<double>(now - due).count());
        const int64_t b = req_ptr[q], n = req_ptr[q + 1] - b;
        // latency counts from the scheduled arrival, even when the generator runs late
        const als_status st = submit_foldin_at(s, n, items ? items + b : nullptr, vals ? vals + b : nullptr,
                                               tickets + q, due);
        if (st != ALS_OK) return st;
    }
    if (max_lag_s) *max_lag_s = lag;
    return ALS_OK;
}

namespace {
als_status submit_foldin_at(als_server *s, int64_t n, const int32_t *items, const float *vals, int64_t *ticket,
                            clk::time_point t0) {
    if (n < 0 || (n > 0 && (!items || !vals))) {
        als_set_error("als_server_submit_foldin: bad argument");
        return ALS_EINVAL;
    }
    if (n > s->cfg.max_batch_ratings) {
        als_set_error("als_server_submit_foldin: request larger than max_batch_ratings");
        return ALS_EINVAL;
    }
    for (int64_t e = 0; e < n; ++e) {
        if (items[e] < 0 || items[e] >= s->model->n_m || !std::isfinite(vals[e])) {
            als_set_error("als_server_submit_foldin: item id out of range or non-finite rating");
            return ALS_EINVAL;
        }
    }
    Request *r = new Request();
    r->items.assign(items, items + n);
    r->vals.assign(vals, vals + n);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        r->t0 = t0;
        if (!s->have_first) {
            s->t_first = r->t0;
            s->have_first = true;
        }
        s->reqs[r->ticket] = r;
        s->pending.push_back(r);
        *ticket = r->ticket;
    }
    s->cv.notify_one();
    return ALS_OK;
}
}  // namespace

extern "C" als_status als_server_submit_job(als_server *s, const als_config *cfg, int64_t n_u, int64_t n_m, int64_t nnz,
                                            const int32_t *rows, const int32_t *cols, const float *vals, const double *x0,
                                            int32_t iters, int64_t *ticket) {
    if (!s || !cfg || n_u < 1 || n_m < 1 || nnz < 0 || (nnz > 0 && (!rows || !cols || !vals)) || !x0 || iters < 0 ||
        !ticket || cfg->n_f < 1 || cfg->n_f > ALS_MAX_NF) {
        als_set_error("als_server_submit_job: bad argument");
        return ALS_EINVAL;
    }
    Job *j = new Job();
    j->cfg = *cfg;
    j->n_u = n_u;
    j->n_m = n_m;
    j->rows.assign(rows, rows + nnz);
    j->cols.assign(cols, cols + nnz);
    j->vals.assign(vals, vals + nnz);
    j->x0.assign(x0, x0 + (size_t)(n_u + n_m) * cfg->n_f);
    j->iters = iters;
    j->bytes = estimate_job_bytes(*cfg, n_u, n_m, nnz);
    if (s->cfg.hbm_budget_bytes && j->bytes > s->cfg.hbm_budget_bytes) {
        delete j;
        als_set_error("als_server_submit_job: the job alone exceeds the server's device-memory budget");
        return ALS_EBUDGET;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        j->ticket = s->next_ticket++;
        j->t0 = clk::now();
        s->jobs[j->ticket] = j;
        s->pending_jobs.push_back(j);
        *ticket = j->ticket;
    }
    s->cv.notify_one();
    return ALS_OK;
}

extern "C" als_status als_server_wait(als_server *s, int64_t ticket, double timeout_s, void *result,
                                      double *latency_s) {
    if (!s) { als_set_error("als_server_wait: server is NULL"); return ALS_EINVAL; }
    std::unique_lock<std::mutex> lk(s->mu);
    auto rit = s->reqs.find(ticket);
    auto jit = s->jobs.find(ticket);
    if (rit == s->reqs.end() && jit == s->jobs.end()) {
        als_set_error("als_server_wait: unknown ticket");
        return ALS_EINVAL;
    }
    const auto deadline = clk::now() + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(timeout_s));
    auto is_done = [&]() { return rit != s->reqs.end() ? rit->second->done : jit->second->done; };
    while (!is_done()) {
        if (s->done.wait_until(lk, deadline) == std::cv_status::timeout && !is_done()) {
            als_set_error("als_server_wait: not finished yet");
            return ALS_ETIMEOUT;
        }
    }
    if (rit != s->reqs.end()) {
        Request *r = rit->second;
        const als_status st = r->status;
        if (st == ALS_OK && result) std::memcpy(result, r->result.data(), r->result.size() * sizeof(float));
        if (latency_s) *latency_s = std::chrono::duration<double>(r->t1 - r->t0).count();
        s->reqs.erase(rit);
        delete r;
        if (st != ALS_OK) als_set_error("als_server_wait: the fold-in batch failed");
        return st;
    }
    Job *j = jit->second;
    const als_status st = j->status;
    if (st == ALS_OK && result) std::memcpy(result, j->result.data(), j->result.size() * sizeof(double));
    if (latency_s) *latency_s = std::chrono::duration<double>(j->t1 - j->t0).count();
    if (st != ALS_OK) als_set_error("als_server_wait: job failed: " + j->error);
    s->jobs.erase(jit);
    delete j;
    return st;
}

extern "C" als_status als_server_stats(als_server *s, double *p50, double *p99, int64_t *completed, double *rps) {
    if (!s) { als_set_error("als_server_stats: server is NULL"); return ALS_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        if (v.empty()) return 0.0;
        const size_t i = (size_t)std::min<double>((double)v.size() - 1, std::ceil(q * (double)v.size()) - 1);
        return v[i];
    };
    if (p50) *p50 = pct(0.50);
    if (p99) *p99 = pct(0.99);
    if (completed) *completed = (int64_t)v.size();
    if (rps) {
        const double span = s->have_first && !v.empty() ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
        *rps = span > 0 ? (double)v.size() / span : 0.0;
    }
    return ALS_OK;
}

extern "C" void als_server_destroy(als_server *s) {
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv.notify_all();
        s->worker.join();
    }
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (Slot &sl : s->slots) {
        cudaFreeHost(sl.hflag); cudaFreeHost(sl.hptr); cudaFreeHost(sl.hidx); cudaFreeHost(sl.hval); cudaFreeHost(sl.hout);
        cudaFreeHost(sl.horder);
        cudaFree(sl.dptr); cudaFree(sl.didx); cudaFree(sl.dval); cudaFree(sl.dout); cudaFree(sl.dorder);
        if (sl.ev) cudaEventDestroy(sl.ev);
    }
    for (auto &kv : s->reqs) delete kv.second;
    for (auto &kv : s->jobs) {
        if (kv.second->ctx) als_destroy(kv.second->ctx);
        delete kv.second;
    }
    if (s->dflags) cudaFree(s->dflags);
    if (s->stream) cudaStreamDestroy(s->stream);
    cudaGetLastError();
    delete s;
}
