// Continuous-batching request server for contour-integral solves.
//
// Requests (operator, region, N, L, M, options, probe block) are queued on submission. A
// request is admitted as soon as a worker is free and its device footprint -- the exact
// allocation list of its plan -- fits the remaining budget; admission keeps arrival order
// (a large request at the head waits for memory rather than being overtaken). Each worker
// owns a non-blocking CUDA stream and runs the whole pass of its request there, so kernels of
// different requests overlap on the device while each request's computation is exactly the
// one nep_ciss_solve performs on the same inputs. Factors and moments stay in the request's
// device-resident plan until its result is copied out.
//
// With max_batch > 1 (nep_server_create_batched) a free worker takes up to max_batch requests from the
// head of the queue at once (in arrival order, while they fit the budget and share a precision) and
// runs them as one batch (nep_plan_execute_batch): the LU and the sweeps of all their quadrature
// points in shared launches, each request's results bitwise those it gets alone.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "nep_common.cuh"

namespace nep {
size_t plan_footprint(nep_split_t h, int N, int L, int M, int precision, int symmetric);
int plan_create_internal(nep_split_t h, const nep_region* r, int32_t N, int32_t L, int32_t M, const nep_opts* o,
                         cudaStream_t alloc_stream, nep_plan_t* out);
void result_set_times(nep_result_t r, double queued_ms, double latency_ms);
}  // namespace nep

using namespace nep;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    uint64_t ticket = 0;
    nep_split_t h = nullptr;
    nep_region region{};
    int N = 0, L = 0, M = 0;
    nep_opts opts{};
    std::vector<double> V;  // empty: drawn from opts.seed
    size_t bytes = 0;
    Clock::time_point submitted, started, finished;
    int status = NEP_PENDING;
    nep_result_t result = nullptr;
    std::string error;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct nep_server {
    int device = 0;
    int max_batch = 1;
    size_t budget = 0, in_use = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::map<uint64_t, Request*> all;
    uint64_t next_ticket = 1;
    bool stopping = false;
    int running = 0;
    std::vector<std::thread> workers;

    void worker_loop() {
        cudaSetDevice(device);
        cudaStream_t st = nullptr;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        for (;;) {
            std::vector<Request*> batch;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] {
                    return (stopping && queue.empty()) ||
                           (!queue.empty() && in_use + queue.front()->bytes <= budget);
                });
                if (queue.empty()) break;
                // the head, then its successors in order while they fit and can share launches
                do {
                    Request* rq = queue.front();
                    if (!batch.empty() && (rq->opts.precision != batch[0]->opts.precision ||
                                           split_has_host_terms(rq->h) || split_has_host_terms(batch[0]->h)))
                        break;
                    queue.pop_front();
                    in_use += rq->bytes;
                    batch.push_back(rq);
                } while ((int)batch.size() < max_batch && !queue.empty() && in_use + queue.front()->bytes <= budget);
                running += (int)batch.size();
            }
            const Clock::time_point t0 = Clock::now();
            for (Request* rq : batch) rq->started = t0;
            const int rc = batch.size() == 1 ? run(batch[0], st) : run_batch(batch, st);
            {
                std::lock_guard<std::mutex> lk(mu);
                const Clock::time_point t1 = Clock::now();
                for (Request* rq : batch) {
                    rq->finished = t1;
                    rq->status = rc;
                    if (rc != NEP_OK) {
                        rq->error = nep_last_error();
                        if (rq->result) {
                            nep_result_free(rq->result);
                            rq->result = nullptr;
                        }
                    } else {
                        result_set_times(rq->result, ms_between(rq->submitted, rq->started),
                                         ms_between(rq->submitted, rq->finished));
                    }
                    in_use -= rq->bytes;
                }
                running -= (int)batch.size();
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }

    // the request's probe block on the device (its own, or the one nep_ciss_solve draws for its seed)
    static int upload_V(Request* rq, void** dV, cudaStream_t st) {
        int n = 0;
        nep_split_info(rq->h, &n, nullptr, nullptr, nullptr, nullptr);
        const size_t nl = (size_t)n * rq->L;
        std::vector<double> Vh;
        const double* src = rq->V.data();
        if (rq->V.empty()) {
            Vh.resize(2 * nl);
            draw_probe_block(rq->opts.seed, nl, rq->opts.symmetric != 0, Vh.data());
            src = Vh.data();
        }
        *dV = nullptr;
        if (cudaMallocAsync(dV, sizeof(double) * 2 * nl, st) != cudaSuccess) return NEP_ERR_NOMEM;
        if (cudaMemcpyAsync(*dV, src, sizeof(double) * 2 * nl, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return NEP_ERR_CUDA;
        return NEP_OK;
    }

    static int run_batch(std::vector<Request*>& rqs, cudaStream_t st) {
        const int k = (int)rqs.size();
        std::vector<nep_plan_t> plans(k, nullptr);
        std::vector<void*> dV(k, nullptr);
        int rc = NEP_OK;
        for (int i = 0; i < k && !rc; ++i) {
            rc = plan_create_internal(rqs[i]->h, &rqs[i]->region, rqs[i]->N, rqs[i]->L, rqs[i]->M, &rqs[i]->opts, st,
                                      &plans[i]);
            if (!rc) rc = upload_V(rqs[i], &dV[i], st);
        }
        if (!rc) rc = nep_plan_execute_batch(k, plans.data(), const_cast<const void* const*>(dV.data()), st);
        for (int i = 0; i < k && !rc; ++i) rc = nep_plan_result(plans[i], &rqs[i]->result);
        for (int i = 0; i < k; ++i) {
            if (dV[i]) cudaFreeAsync(dV[i], st);
            if (plans[i]) nep_plan_destroy(plans[i]);
        }
        return rc;
    }

    static int run(Request* rq, cudaStream_t st) {
        nep_plan_t plan = nullptr;
        NEP_TRY(plan_create_internal(rq->h, &rq->region, rq->N, rq->L, rq->M, &rq->opts, st, &plan));
        int n = 0;
        nep_split_info(rq->h, &n, nullptr, nullptr, nullptr, nullptr);
        const size_t nl = (size_t)n * rq->L;
        std::vector<double> Vh;
        const double* src = rq->V.data();
        if (rq->V.empty()) {
            // the probe block nep_ciss_solve draws for the same seed
            Vh.resize(2 * nl);
            draw_probe_block(rq->opts.seed, nl, rq->opts.symmetric != 0, Vh.data());
            src = Vh.data();
        }
        void* dV = nullptr;
        int rc = NEP_OK;
        if (cudaMallocAsync(&dV, sizeof(double) * 2 * nl, st) != cudaSuccess) rc = NEP_ERR_NOMEM;
        if (!rc && cudaMemcpyAsync(dV, src, sizeof(double) * 2 * nl, cudaMemcpyHostToDevice, st) != cudaSuccess)
            rc = NEP_ERR_CUDA;
        if (!rc) rc = nep_plan_execute(plan, dV, st);
        if (!rc) rc = nep_plan_result(plan, &rq->result);
        if (dV) cudaFreeAsync(dV, st);
        nep_plan_destroy(plan);
        return rc;
    }
};

extern "C" int nep_server_create(int32_t workers, uint64_t hbm_budget_bytes, nep_server_t* out) {
    return nep_server_create_batched(workers, 1, hbm_budget_bytes, out);
}

extern "C" int nep_server_create_batched(int32_t workers, int32_t max_batch, uint64_t hbm_budget_bytes,
                                         nep_server_t* out) {
    if (!out || workers < 1 || max_batch < 1) {
        set_error("nep_server_create: need workers >= 1 and max_batch >= 1");
        return NEP_ERR_ARG;
    }
    *out = nullptr;
    nep_server* s = new nep_server();
    s->max_batch = max_batch;
    cudaGetDevice(&s->device);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { delete s; set_error("cudaMemGetInfo failed"); return NEP_ERR_CUDA; }
    s->budget = hbm_budget_bytes ? (size_t)hbm_budget_bytes : (size_t)(0.8 * (double)free_b);
    for (int i = 0; i < workers; ++i) s->workers.emplace_back([s] { s->worker_loop(); });
    *out = s;
    return NEP_OK;
}

extern "C" uint64_t nep_plan_bytes(nep_split_t h, int32_t N, int32_t L, int32_t M, int32_t precision) {
    if (!h || N < 1 || L < 1 || M < 1) return 0;
    int n = 0;
    nep_split_info(h, &n, nullptr, nullptr, nullptr, nullptr);
    return plan_footprint(h, N, L, M, precision, 0) + sizeof(double) * 2 * (size_t)n * L;
}

extern "C" int nep_submit(nep_server_t s, nep_split_t h, const nep_region* r, int32_t N, int32_t L, int32_t M,
                          const nep_opts* o, const double* V_host, uint64_t* ticket) {
    if (!s || !h || !r || !ticket) { set_error("nep_submit: bad arguments"); return NEP_ERR_ARG; }
    int n = 0;
    nep_split_info(h, &n, nullptr, nullptr, nullptr, nullptr);
    if (N < 2 || L < 1 || M < 1 || L > n) { set_error("nep_submit: need N >= 2, 1 <= L <= n, M >= 1"); return NEP_ERR_ARG; }
    Request* rq = new Request();
    rq->h = h;
    rq->region = *r;
    rq->N = N;
    rq->L = L;
    rq->M = M;
    if (o) rq->opts = *o;
    else nep_opts_default(&rq->opts);
    if (V_host) rq->V.assign(V_host, V_host + 2 * (size_t)n * L);
    rq->bytes = plan_footprint(h, N, L, M, rq->opts.precision, rq->opts.symmetric) + sizeof(double) * 2 * (size_t)n * L;
    rq->submitted = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (rq->bytes > s->budget) {
            const size_t need = rq->bytes;
            delete rq;
            set_error("nep_submit: the request needs %zu device bytes, more than the server budget of %zu", need,
                      s->budget);
            return NEP_ERR_NOMEM;
        }
        rq->ticket = s->next_ticket++;
        s->queue.push_back(rq);
        s->all[rq->ticket] = rq;
        *ticket = rq->ticket;
    }
    s->cv_work.notify_all();
    return NEP_OK;
}

static int take(nep_server_t s, uint64_t ticket, nep_result_t* out, bool block) {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) { set_error("unknown or already collected ticket %llu", (unsigned long long)ticket); return NEP_ERR_ARG; }
    Request* rq = it->second;
    if (block) s->cv_done.wait(lk, [&] { return rq->status != NEP_PENDING; });
    if (rq->status == NEP_PENDING) return NEP_PENDING;
    const int rc = rq->status;
    if (rc == NEP_OK) *out = rq->result;
    else set_error("%s", rq->error.c_str());
    s->all.erase(it);
    delete rq;
    return rc;
}

extern "C" int nep_poll(nep_server_t s, uint64_t ticket, nep_result_t* out) {
    if (!s || !out) { set_error("nep_poll: bad arguments"); return NEP_ERR_ARG; }
    *out = nullptr;
    return take(s, ticket, out, false);
}

extern "C" int nep_server_wait(nep_server_t s, uint64_t ticket, nep_result_t* out) {
    if (!s || !out) { set_error("nep_server_wait: bad arguments"); return NEP_ERR_ARG; }
    *out = nullptr;
    return take(s, ticket, out, true);
}

extern "C" int nep_server_destroy(nep_server_t s) {
    if (!s) return NEP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->all) {
        if (kv.second->result) nep_result_free(kv.second->result);
        delete kv.second;
    }
    delete s;
    return NEP_OK;
}
