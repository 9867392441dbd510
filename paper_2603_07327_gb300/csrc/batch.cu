// batch.cu -- batched form: many (scanner, source, digitizer, n, seed) jobs in
// one persistent transport launch, one segmented time sort and one
// coincidence pass; the whole enqueue is captured once into a CUDA graph and
// replayed by gpet_batch_run.  Every job keeps its own Philox key and history
// ids, so a job's results are the same alone and inside a batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>

#include "host.h"

using namespace gpet;

gpet_batch::~gpet_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
}

int gpet_batch_build_run(Run &R, int32_t n_jobs, gpet_scanner *const *scanners, const gpet_source *sources,
                         const gpet_digitizer *digitizers, const uint64_t *n_decays, const uint64_t *seeds,
                         const gpet_options *opt) {
    if (n_jobs < 1 || !scanners || !sources || !digitizers || !n_decays || !seeds)
        return gpet_fail(GPET_ERR_INVALID_ARG, "batch needs n_jobs >= 1 and non-NULL arrays");
    int st = run_default_cfg(R, opt, scanners[0]);
    if (st != GPET_OK) return st;
    std::map<std::string, int> geom_index;  // deduplicated geometry table
    uint64_t total = 0;
    for (int32_t j = 0; j < n_jobs; ++j) {
        if (!scanners[j]) return gpet_fail(GPET_ERR_INVALID_ARG, "scanner %d is NULL", j);
        JobDev J;
        st = gpet_make_job(scanners[j], &sources[j], &digitizers[j], n_decays[j], seeds[j], J);
        if (st != GPET_OK) return gpet_fail(st, "job %d: %s", j, gpet_last_error());
        const std::string key = gpet_geometry_key(scanners[j]);
        auto it = geom_index.find(key);
        if (it == geom_index.end()) {
            it = geom_index.emplace(key, (int)R.geoms.size()).first;
            R.geoms.push_back(scanners[j]->g);
            R.geom_pose.push_back(scanners[j]->pose_dev);
            R.geom_keys.push_back(key);
        }
        J.geom = it->second;
        R.jobs.push_back(J);
        R.job_crystals.push_back(scanners[j]->n_crystals);
        R.windows.push_back((uint64_t)std::llround(digitizers[j].coinc_window_ns * 1000.0));
        total += n_decays[j];
    }
    R.caps.singles = std::max<uint64_t>(65536, total * 6 / 10);
    R.caps.hits = R.keep_hits ? std::max<uint64_t>(65536, total * 5 / 2) : 0;
    R.caps.ovf = std::max<uint64_t>(4096, total / 256);
    return GPET_OK;
}

extern "C" int gpet_batch_create(int32_t n_jobs, gpet_scanner *const *scanners, const gpet_source *sources,
                                 const gpet_digitizer *digitizers, const uint64_t *n_decays, const uint64_t *seeds,
                                 const gpet_options *opt, gpet_batch **out) {
    if (!out) return gpet_fail(GPET_ERR_INVALID_ARG, "out is NULL");
    gpet_batch *b = new (std::nothrow) gpet_batch();
    if (!b) return gpet_fail(GPET_ERR_OOM, "host allocation of the batch failed");
    b->run = std::make_shared<Run>();
    Run &R = *b->run;
    int st = gpet_batch_build_run(R, n_jobs, scanners, sources, digitizers, n_decays, seeds, opt);
    if (st != GPET_OK) { delete b; return st; }
    if (!R.stream) {  // capture needs a stream other than the legacy default one
        cudaError_t e = cudaStreamCreateWithFlags(&R.stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete b; return gpet_cuda_fail(e, "cudaStreamCreate"); }
        R.own_stream = true;
    }
    for (int32_t j = 0; j < n_jobs; ++j) {
        b->n_decays.push_back(n_decays[j]);
        b->n_crystals.push_back(scanners[j]->n_crystals);
    }
    // first run sizes the buffers (exact re-run on overflow) and gives results
    st = run_with_retry(R);
    if (st != GPET_OK) { delete b; return st; }
    // capture the whole hot path once; replays reuse the same arena
    cudaError_t e = cudaStreamBeginCapture(R.stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { delete b; return gpet_cuda_fail(e, "cudaStreamBeginCapture"); }
    st = run_enqueue(R);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(R.stream, &g);
    if (st != GPET_OK) { if (g) cudaGraphDestroy(g); delete b; return st; }
    if (e != cudaSuccess) { delete b; return gpet_cuda_fail(e, "cudaStreamEndCapture"); }
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) { delete b; return gpet_cuda_fail(e, "cudaGraphInstantiate"); }
    *out = b;
    return GPET_OK;
}

extern "C" int gpet_batch_run(gpet_batch *b) {
    if (!b || !b->exec) return gpet_fail(GPET_ERR_INVALID_ARG, "batch is NULL");
    Run &R = *b->run;
    cudaError_t e = cudaGraphLaunch(b->exec, R.stream);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaGraphLaunch");
    return run_collect(R);
}

extern "C" int gpet_batch_jobs(const gpet_batch *b, int32_t *n_jobs) {
    if (!b || !n_jobs) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    *n_jobs = (int32_t)b->run->jobs.size();
    return GPET_OK;
}

extern "C" int gpet_batch_result(const gpet_batch *b, int32_t job, gpet_result **out) {
    if (!b || !out) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    if (job < 0 || job >= (int32_t)b->run->jobs.size())
        return gpet_fail(GPET_ERR_INVALID_ARG, "job %d outside [0, %zu)", job, b->run->jobs.size());
    gpet_result *r = new (std::nothrow) gpet_result();
    if (!r) return gpet_fail(GPET_ERR_OOM, "host allocation of the result failed");
    r->run = b->run;
    r->job = job;
    fill_counts(*b->run, job, b->n_decays[job], b->n_crystals[job], &r->counts);
    *out = r;
    return GPET_OK;
}

extern "C" int gpet_batch_counts(const gpet_batch *b, gpet_counts *total) {
    if (!b || !total) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    const Run &R = *b->run;
    uint64_t n = 0;
    int64_t nc = 0;
    for (size_t j = 0; j < R.jobs.size(); ++j) { n += b->n_decays[j]; nc += b->n_crystals[j]; }
    fill_counts(R, 0, n, nc, total);
    total->hits = R.h_hdr.counters[5];
    total->singles = R.h_hdr.n_sorted;
    total->coincidences = R.h_hdr.n_coinc;
    return GPET_OK;
}

extern "C" void gpet_batch_destroy(gpet_batch *b) { delete b; }

extern "C" int gpet_simulate_batch(int32_t n_jobs, gpet_scanner *const *scanners, const gpet_source *sources,
                                   const gpet_digitizer *digitizers, const uint64_t *n_decays, const uint64_t *seeds,
                                   const gpet_options *opt, gpet_result **outs) {
    if (!outs) return gpet_fail(GPET_ERR_INVALID_ARG, "outs is NULL");
    auto R = std::make_shared<Run>();
    int st = gpet_batch_build_run(*R, n_jobs, scanners, sources, digitizers, n_decays, seeds, opt);
    if (st == GPET_OK) st = run_with_retry(*R);
    if (st != GPET_OK) return st;
    for (int32_t j = 0; j < n_jobs; ++j) {
        outs[j] = new (std::nothrow) gpet_result();
        if (!outs[j]) {
            for (int32_t k = 0; k < j; ++k) { delete outs[k]; outs[k] = nullptr; }
            return gpet_fail(GPET_ERR_OOM, "host allocation of the results failed");
        }
        outs[j]->run = R;
        outs[j]->job = j;
        fill_counts(*R, j, n_decays[j], scanners[j]->n_crystals, &outs[j]->counts);
    }
    return GPET_OK;
}
