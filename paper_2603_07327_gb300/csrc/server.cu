// server.cu -- serving loop with continuous batching.
//
// Requests (scanner design + source + digitizer + decay count + seed) arrive
// through gpet_server_submit from any host thread.  Worker threads, each with
// its own CUDA stream, repeatedly take the queued requests that fit the HBM
// budget (first come, first served), run them together as one batched launch
// (one persistent transport kernel over all their histories, one segmented
// time sort, one coincidence pass) and publish one result per request.  While
// one worker's batch is on the GPU the other admits the requests that arrived
// meanwhile and launches them, so their work overlaps on the device.  A
// request's device memory counts against the budget from admission until its
// result is freed.  Because every random number is addressed by (seed,
// history), a request's result is the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "host.h"

using namespace gpet;


namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t id = 0;
    gpet_scanner *sc = nullptr;
    gpet_source src{};
    gpet_digitizer dg{};
    uint64_t n = 0, seed = 0;
    size_t est = 0;
    uint64_t span_ps = 0;             // acquisition span (decay times lie in [0, span_ps))
    bool done = false;
    int status = GPET_OK;
    std::string error;
    gpet_result *result = nullptr;
    Clock::time_point t_submit;
};

// budget accounting shared with the release callbacks of the runs
struct Core {
    std::mutex mu;
    std::condition_variable cv;       // queue changes and memory releases
    std::condition_variable done_cv;  // request completions
    size_t budget = 0, in_use = 0, peak = 0;
};

}  // namespace

struct gpet_server {
    std::shared_ptr<Core> core;
    gpet_options opt{};
    int max_jobs = 256;
    std::deque<Req *> queue;
    std::map<uint64_t, Req *> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> workers;
    gpet_server_stats stats{};
    int device = 0;
};

static void worker_main(gpet_server *S, int widx) {
    cudaSetDevice(S->device);
    cudaStream_t stream = nullptr;
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    Core &C = *S->core;
    for (;;) {
        std::vector<Req *> batch;
        size_t taken = 0;
        uint64_t max_span = 0;
        {
            std::unique_lock<std::mutex> lk(C.mu);
            for (;;) {
                if (S->stop && S->queue.empty()) break;
                // first come, first served: take from the front while the budget allows
                while (!S->queue.empty() && (int)batch.size() < S->max_jobs) {
                    Req *r = S->queue.front();
                    if (C.in_use + r->est > C.budget && !(batch.empty() && C.in_use == 0)) break;
                    // the time stamps of every job must fit beside the job bits of the sort key
                    const uint64_t span = std::max(max_span, r->span_ps);
                    if (!batch.empty() &&
                        span > sort_time_limit(sort_job_shift((int)batch.size() + 1)) - 0xFFFFFFFFull)
                        break;
                    max_span = span;
                    S->queue.pop_front();
                    C.in_use += r->est;
                    taken += r->est;
                    batch.push_back(r);
                }
                C.peak = std::max(C.peak, C.in_use);
                if (!batch.empty()) break;
                C.cv.wait(lk);
            }
            if (batch.empty()) break;  // stopping and drained
        }
        // one batched launch over the admitted requests
        std::vector<gpet_scanner *> scs;
        std::vector<gpet_source> srcs;
        std::vector<gpet_digitizer> dgs;
        std::vector<uint64_t> ns, seeds;
        for (Req *r : batch) {
            scs.push_back(r->sc);
            srcs.push_back(r->src);
            dgs.push_back(r->dg);
            ns.push_back(r->n);
            seeds.push_back(r->seed);
        }
        auto R = std::make_shared<Run>();
        gpet_options o = S->opt;
        o.stream = stream;
        int st = gpet_batch_build_run(*R, (int32_t)batch.size(), scs.data(), srcs.data(), dgs.data(), ns.data(),
                                      seeds.data(), &o);
        if (st == GPET_OK) st = run_with_retry(*R);
        const std::string err = st == GPET_OK ? std::string() : std::string(gpet_last_error());
        const auto t_done = Clock::now();
        {
            std::lock_guard<std::mutex> lk(C.mu);
            C.in_use -= taken;
            if (st == GPET_OK) {
                // the run's real arena stays charged until its last result is freed
                const size_t bytes = R->arena_bytes;
                C.in_use += bytes;
                C.peak = std::max(C.peak, C.in_use);
                std::weak_ptr<Core> wc = S->core;
                R->on_release = [wc, bytes]() {
                    if (auto c = wc.lock()) {
                        std::lock_guard<std::mutex> l2(c->mu);
                        c->in_use -= bytes;
                        c->cv.notify_all();
                    }
                };
                S->stats.launches++;
                S->stats.max_jobs_per_launch = std::max<uint64_t>(S->stats.max_jobs_per_launch, batch.size());
            }
            for (size_t j = 0; j < batch.size(); ++j) {
                Req *r = batch[j];
                r->status = st;
                if (st == GPET_OK) {
                    gpet_result *res = new (std::nothrow) gpet_result();
                    if (res) {
                        res->run = R;
                        res->job = (int)j;
                        fill_counts(*R, (int)j, r->n, r->sc->n_crystals, &res->counts);
                        res->counts.latency_ms =
                            std::chrono::duration<double, std::milli>(t_done - r->t_submit).count();
                        r->result = res;
                    } else {
                        r->status = GPET_ERR_OOM;
                        r->error = "host allocation of a result failed";
                    }
                } else {
                    r->error = err;
                }
                r->done = true;
                S->stats.completed++;
                S->stats.pairs_completed += r->n;
            }
            C.cv.notify_all();
            C.done_cv.notify_all();
        }
        R.reset();  // views keep the run alive; the worker does not
    }
    cudaStreamSynchronize(stream);
    cudaStreamDestroy(stream);
    (void)widx;
}

extern "C" int gpet_server_create(const gpet_server_config *cfg, gpet_server **out) {
    if (!cfg || !out) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    if (cfg->hbm_budget_bytes == 0) return gpet_fail(GPET_ERR_INVALID_ARG, "hbm_budget_bytes must be > 0");
    if (cfg->workers < 0 || cfg->workers > 8) return gpet_fail(GPET_ERR_INVALID_ARG, "workers must be in [0, 8]");
    if (cfg->max_jobs_per_launch < 0 || cfg->max_jobs_per_launch > 4095)
        return gpet_fail(GPET_ERR_INVALID_ARG, "max_jobs_per_launch must be in [0, 4095]");
    gpet_server *S = new (std::nothrow) gpet_server();
    if (!S) return gpet_fail(GPET_ERR_OOM, "host allocation of the server failed");
    S->core = std::make_shared<Core>();
    S->core->budget = cfg->hbm_budget_bytes;
    S->opt = cfg->launch;
    S->opt.stream = nullptr;
    S->opt.keep_hits = 0;
    S->max_jobs = cfg->max_jobs_per_launch > 0 ? cfg->max_jobs_per_launch : 256;
    cudaError_t e = cudaGetDevice(&S->device);
    if (e != cudaSuccess) { delete S; return gpet_cuda_fail(e, "cudaGetDevice"); }
    const int nw = cfg->workers > 0 ? cfg->workers : 2;
    for (int w = 0; w < nw; ++w) S->workers.emplace_back(worker_main, S, w);
    *out = S;
    return GPET_OK;
}

extern "C" int gpet_server_submit(gpet_server *S, gpet_scanner *sc, const gpet_source *src, const gpet_digitizer *dg,
                                  uint64_t n_decays, uint64_t seed, int32_t block, uint64_t *req_id) {
    if (!S || !sc || !src || !dg || !req_id) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    JobDev J;
    int st = gpet_make_job(sc, src, dg, n_decays, seed, J);  // validate now, not in the worker
    if (st != GPET_OK) return st;
    Req *r = new (std::nothrow) Req();
    if (!r) return gpet_fail(GPET_ERR_OOM, "host allocation of a request failed");
    r->sc = sc;
    r->src = *src;
    r->dg = *dg;
    r->n = n_decays;
    r->seed = seed;
    r->est = run_footprint(n_decays, sc->n_crystals, 1, 1, false);
    r->span_ps = J.t_span_ps;
    Core &C = *S->core;
    std::unique_lock<std::mutex> lk(C.mu);
    if (r->est > C.budget) {
        const size_t est = r->est;
        delete r;
        return gpet_fail(GPET_ERR_OOM, "request needs ~%zu device bytes, more than the whole budget", est);
    }
    if (S->stop) {
        delete r;
        return gpet_fail(GPET_ERR_INVALID_ARG, "server is shutting down");
    }
    if (!block) {
        size_t queued = 0;
        for (Req *q : S->queue) queued += q->est;
        if (C.in_use + queued + r->est > C.budget) {
            delete r;
            S->stats.rejected++;
            return gpet_fail(GPET_ERR_BUSY, "HBM budget full (in use %zu + queued %zu of %zu bytes)", C.in_use, queued,
                             C.budget);
        }
    }
    r->id = S->next_id++;
    r->t_submit = Clock::now();
    S->reqs[r->id] = r;
    S->queue.push_back(r);
    S->stats.submitted++;
    *req_id = r->id;
    C.cv.notify_all();
    return GPET_OK;
}

static int take_result(gpet_server *S, std::map<uint64_t, Req *>::iterator it, gpet_result **out) {
    Req *r = it->second;
    S->reqs.erase(it);
    const int st = r->status;
    if (st == GPET_OK) *out = r->result;
    else gpet_fail(st, "%s", r->error.c_str());
    delete r;
    return st;
}

extern "C" int gpet_server_poll(gpet_server *S, uint64_t req_id, gpet_result **out) {
    if (!S || !out) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    std::lock_guard<std::mutex> lk(S->core->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return gpet_fail(GPET_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)req_id);
    if (!it->second->done) return GPET_OK;
    return take_result(S, it, out);
}

extern "C" int gpet_server_wait(gpet_server *S, uint64_t req_id, gpet_result **out) {
    if (!S || !out) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(S->core->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return gpet_fail(GPET_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)req_id);
    // Re-find the request after every wake-up: another caller polling or
    // waiting on the same id may have taken (and freed) it meanwhile.
    S->core->done_cv.wait(lk, [&] {
        it = S->reqs.find(req_id);
        return it == S->reqs.end() || it->second->done;
    });
    if (it == S->reqs.end())
        return gpet_fail(GPET_ERR_INVALID_ARG, "request %llu was taken by another caller", (unsigned long long)req_id);
    return take_result(S, it, out);
}

extern "C" int gpet_server_stats_get(gpet_server *S, gpet_server_stats *out) {
    if (!S || !out) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->core->mu);
    *out = S->stats;
    out->bytes_in_use = S->core->in_use;
    out->peak_bytes = S->core->peak;
    out->queued = S->queue.size();
    return GPET_OK;
}

extern "C" void gpet_server_destroy(gpet_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->core->mu);
        S->stop = true;
        S->core->cv.notify_all();
    }
    for (auto &t : S->workers) t.join();
    for (auto &kv : S->reqs) {
        if (kv.second->result) gpet_result_free(kv.second->result);
        delete kv.second;
    }
    delete S;
}
