// run.cu -- run machinery: one device arena per launch, enqueue of the whole
// hot path (transport -> singles -> time sort -> coincidences) without host
// round trips, header read-back with overflow retry, and the plain
// gpet_simulate entry point with its result accessors.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "host.h"

namespace gpet {

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Carver {
    size_t off = 0;
    template <typename T>
    size_t take(T *&p, size_t count) {
        off = align_up(off, 256);
        const size_t at = off;
        p = reinterpret_cast<T *>(at);  // offset for now, rebased later
        off += sizeof(T) * std::max<size_t>(count, 1);
        return at;
    }
};

template <typename T>
static void rebase(T *&p, char *base) {
    p = reinterpret_cast<T *>(base + reinterpret_cast<size_t>(p));
}

// Keep freed arenas in the device's stream-ordered pool instead of returning
// them to the driver at every synchronisation (once per device).
static void keep_pool_memory(int dev) {
    static std::mutex mu;
    static bool done[64] = {false};
    if (dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[dev] = true;
}

int run_default_cfg(Run &R, const gpet_options *opt_in, const gpet_scanner *sc) {
    // kernel 0: the autotuner's choice for this design class when one was made
    gpet_options tuned;
    const gpet_options *opt = opt_in;
    gpet_options merged;
    int sms0 = 0, dev0 = 0;
    if (sc && (!opt_in || opt_in->kernel == 0) && cudaGetDevice(&dev0) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms0, cudaDevAttrMultiProcessorCount, dev0) == cudaSuccess &&
        ::gpet_tuned_options(sc, sms0, &tuned)) {
        if (opt_in) merged = *opt_in; else std::memset(&merged, 0, sizeof(merged));
        merged.kernel = tuned.kernel;
        if (merged.blocks_per_sm == 0) merged.blocks_per_sm = tuned.blocks_per_sm;
        if (merged.compact_every == 0) merged.compact_every = tuned.compact_every;
        if (merged.pool_depth == 0) merged.pool_depth = tuned.pool_depth;
        if (merged.block_size == 0) merged.block_size = tuned.block_size;
        opt = &merged;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaGetDevice");
    R.device = dev;
    keep_pool_memory(dev);
    e = preload_kernels();  // all of them, once per device: no lazy load while a live launch runs
    if (e != cudaSuccess) return gpet_cuda_fail(e, "kernel preload");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaDeviceGetAttribute");
    R.cfg.sm_count = sms;
    R.cfg.kernel = (opt && opt->kernel > 0) ? opt->kernel : kKernelCta;
    if (R.cfg.kernel != kKernelLoop && R.cfg.kernel != kKernelWave && R.cfg.kernel != kKernelCta)
        return gpet_fail(GPET_ERR_INVALID_ARG, "kernel %d not in {1, 2, 3}", R.cfg.kernel);
    // CTA-synchronous kernel: CTAs of 128, 256 or 512 threads; others <= 256
    R.cfg.block_size = (opt && opt->block_size > 0) ? opt->block_size : 256;
    if (R.cfg.kernel == kKernelCta
            ? (R.cfg.block_size != 128 && R.cfg.block_size != 256 && R.cfg.block_size != 512)
            : (R.cfg.block_size % 32 || R.cfg.block_size > 256))
        return gpet_fail(GPET_ERR_INVALID_ARG, "block_size %d not valid for kernel %d", R.cfg.block_size,
                         R.cfg.kernel);
    const int bps = (opt && opt->blocks_per_sm > 0) ? opt->blocks_per_sm : 4;
    R.cfg.grid = sms * bps;
    R.cfg.compact_every = (opt && opt->compact_every > 0) ? opt->compact_every : 1;
    R.cfg.pool_depth = (opt && opt->pool_depth > 0) ? opt->pool_depth : 2;
    if (R.cfg.pool_depth > 4) return gpet_fail(GPET_ERR_INVALID_ARG, "pool_depth must be in [1, 4]");
    if (R.cfg.compact_every > 64) return gpet_fail(GPET_ERR_INVALID_ARG, "compact_every must be <= 64");
    R.cfg.max_smem_geoms = kMaxStagedGeoms;
    R.keep_hits = opt && opt->keep_hits;
    R.stream = opt ? reinterpret_cast<cudaStream_t>(opt->stream) : nullptr;
    return GPET_OK;
}

int run_plan(Run &R) {
    const int nj = (int)R.jobs.size();
    // table sizes: the jobs themselves, or a live launch's capacities
    const int njc = R.live ? std::max(nj, R.live_cap.jobs) : nj;
    const size_t ngc = R.live ? std::max<size_t>(R.geoms.size(), (size_t)R.live_cap.geoms) : R.geoms.size();
    if (nj < 1) return gpet_fail(GPET_ERR_INVALID_ARG, "no jobs");
    if (njc > 4095) return gpet_fail(GPET_ERR_INVALID_ARG, "at most 4095 jobs per launch");
    // sort keys: the job index above the time stamps; every job's latest time
    // (its span plus the longest flight a uint32 ps offset holds) must fit below it
    R.S.job_shift = sort_job_shift(njc);
    for (int j = 0; j < nj; ++j)
        if (R.jobs[j].t_span_ps > sort_time_limit(R.S.job_shift) - 0xFFFFFFFFull)
            return gpet_fail(GPET_ERR_INVALID_ARG,
                             "job %d: acquisition of %.0f s does not fit beside %d job bits of the time key "
                             "(at most %.0f s in a launch of %d jobs): use fewer jobs per launch",
                             j, R.jobs[j].t_span_ps * 1e-12, 64 - R.S.job_shift,
                             (sort_time_limit(R.S.job_shift) - 0xFFFFFFFFull) * 1e-12, njc);
    // tallies per job
    R.tally_off.resize(nj);
    int64_t tc = 0;
    for (int j = 0; j < nj; ++j) { R.tally_off[j] = tc; tc += R.job_crystals[j]; }
    R.total_crystals = tc;
    const int64_t tcc = R.live ? std::max<int64_t>(tc, R.live_cap.crystals) : tc;
    R.live_tally_used = tc;
    uint64_t total = 0;
    for (auto &J : R.jobs) total += J.n_hist;
    uint64_t cs = R.live_cap.chunk;
    if (!R.live && !R.digitize_only) {
        // chunks: about 48 per resident warp, so that warps run out of work
        // within a small fraction of the launch of one another (32..4096)
        long long warps = 0;
        cudaError_t we = transport_resident_warps((int)R.geoms.size(), R.cfg, &warps);
        if (we != cudaSuccess) return gpet_cuda_fail(we, "transport occupancy query");
        cs = total / std::max<uint64_t>((uint64_t)warps * 48, 1);
        cs = std::max<uint64_t>(32, std::min<uint64_t>(4096, cs / 32 * 32));
    }
    R.chunk_size = (unsigned)cs;
    // a live launch's unpublished entries hold ~0: no chunk index reaches them
    R.chunk_start.assign(njc + 1, ~0ull);
    R.chunk_start[0] = 0;
    for (int j = 0; j < nj; ++j)
        R.chunk_start[j + 1] = R.chunk_start[j] + (R.jobs[j].n_hist + cs - 1) / cs;
    R.live_tail = R.chunk_start[nj];

    // The first guess of the singles capacity (0.6 per history) may exceed what
    // a long run needs by far (a narrow energy window keeps few singles): it
    // takes at most a quarter of the free device memory.  The device counts
    // past the capacity, so a run with more singles is detected and re-run once
    // with its exact count; so is a run with more than the launch limit.
    if (R.caps.guess) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            // arena bytes per single of capacity: raw record, two key and index
            // buffers, the time-ordered arrays, coincidence flag and pair slots
            const uint64_t per_single = sizeof(RawSingle) + 2 * 8 + 2 * 4 + 8 + 8 + 6 * 4 + 1 + 4;
            R.caps.singles = std::min<uint64_t>(R.caps.singles, std::max<uint64_t>(65536, free_b / 4 / per_single));
        } else {
            cudaGetLastError();
        }
    }
    const uint64_t cap = std::min<uint64_t>(std::max<uint64_t>(R.caps.singles, 1), kMaxSinglesPerLaunch);
    const uint64_t hcap = R.keep_hits ? std::max<uint64_t>(R.caps.hits, 1) : 0;
    const uint64_t ocap = std::max<uint64_t>(R.caps.ovf, 1);
    const uint64_t tiles = (cap + 4095) / 4096;

    Carver cv;
    // zeroed before every launch
    cv.take(R.d_hdr, 1);
    cv.take(R.S.ghist, 8 * 256);
    cv.take(R.d_tally_count, (size_t)tcc);
    cv.take(R.d_tally_efx, (size_t)tcc);
    const size_t nwin = R.win_lo.size();
    if (nwin) cv.take(R.d_win_counts, (size_t)njc * nwin);
    R.zero_bytes = align_up(cv.off, 256);
    cv.take(R.d_live, 3);
    cv.take(R.d_jobs, njc);
    cv.take(R.d_geoms, ngc);
    // posed-panel tables of the geometries in non-repetition mode, each on
    // 128-byte lines of its own (a live launch appends them)
    std::vector<size_t> pose_off(R.geoms.size(), 0);
    size_t pose_floats = 0;
    for (size_t i = 0; i < R.geoms.size(); ++i) {
        pose_off[i] = pose_floats;
        if (i < R.geom_pose.size()) pose_floats += align_up(R.geom_pose[i].size(), 32);
    }
    R.live_pose_used = pose_floats;
    const size_t pfc = R.live ? std::max(pose_floats, R.live_cap.pose_floats) : pose_floats;
    R.d_pose = nullptr;
    if (pfc) cv.take(R.d_pose, pfc);
    cv.take(R.d_chunk_start, njc + 1);
    cv.take(R.d_window, njc);
    // raw singles
    OutDev &O = R.O;
    cv.take(O.s_raw, cap);
    // hits
    if (hcap) {
        cv.take(O.hit_h, hcap); cv.take(O.hit_t, hcap);
        cv.take(O.hit_gstep, hcap); cv.take(O.hit_crystal, hcap); cv.take(O.hit_layer, hcap);
        cv.take(O.hit_job, hcap); cv.take(O.hit_wuv, 3 * hcap); cv.take(O.hit_e, hcap);
    }
    cv.take(O.ovf_h, ocap); cv.take(O.ovf_job, ocap);
    // sort
    SortDev &S = R.S;
    cv.take(S.keys[0], cap); cv.take(S.keys[1], cap);
    cv.take(S.vals[0], cap); cv.take(S.vals[1], cap);
    cv.take(S.plan, 32);
    cv.take(S.lb[0], 256 * tiles); cv.take(S.lb[1], 256 * tiles);
    cv.take(S.tile_ctr, 8);
    // sorted singles
    SinglesDev &SD = R.SD;
    cv.take(SD.t, cap); cv.take(SD.h, cap);
    cv.take(SD.unit, cap); cv.take(SD.panel, cap); cv.take(SD.job, cap);
    cv.take(SD.e, cap); cv.take(SD.eraw, cap); cv.take(SD.doi, cap);
    // coincidences
    CoincDev &C = R.C;
    cv.take(C.flag, cap);
    cv.take(C.tile_cnt, tiles);
    cv.take(C.a, cap / 2 + 1); cv.take(C.b, cap / 2 + 1);
    // per-job statistics
    JobStatsDev &JS = R.JS;
    cv.take(JS.s_off, njc + 1); cv.take(JS.c_off, njc + 1); cv.take(JS.hits, njc);
    cv.take(R.d_toff, njc); cv.take(R.d_tn, njc);
    R.arena_bytes = align_up(cv.off, 256);

    // a live launch uploads (now and while it runs) on its own stream, which
    // the running kernel does not block
    cudaStream_t up = R.upload_stream ? R.upload_stream : R.stream;
    cudaError_t e = cudaMallocAsync(&R.arena, R.arena_bytes, up);
    if (e != cudaSuccess) {
        R.arena = nullptr;
        return e == cudaErrorMemoryAllocation ? gpet_fail(GPET_ERR_OOM, "device arena of %zu bytes", R.arena_bytes)
                                              : gpet_cuda_fail(e, "cudaMallocAsync");
    }
    char *base = static_cast<char *>(R.arena);
    rebase(R.d_hdr, base);
    rebase(S.ghist, base);
    rebase(R.d_tally_count, base);
    rebase(R.d_tally_efx, base);
    if (nwin) rebase(R.d_win_counts, base); else R.d_win_counts = nullptr;
    rebase(R.d_live, base);
    rebase(R.d_jobs, base); rebase(R.d_geoms, base); rebase(R.d_chunk_start, base); rebase(R.d_window, base);
    if (pfc) rebase(R.d_pose, base);
    for (size_t i = 0; i < R.geoms.size(); ++i)
        R.geoms[i].pose = (i < R.geom_pose.size() && !R.geom_pose[i].empty())
                              ? reinterpret_cast<const float4 *>(R.d_pose + pose_off[i]) : nullptr;
    rebase(O.s_raw, base);
    if (hcap) {
        rebase(O.hit_h, base); rebase(O.hit_t, base); rebase(O.hit_gstep, base); rebase(O.hit_crystal, base);
        rebase(O.hit_layer, base); rebase(O.hit_job, base); rebase(O.hit_wuv, base); rebase(O.hit_e, base);
    } else {
        O.hit_h = nullptr; O.hit_t = nullptr; O.hit_gstep = O.hit_crystal = O.hit_layer = O.hit_job = nullptr;
        O.hit_wuv = O.hit_e = nullptr;
    }
    rebase(O.ovf_h, base); rebase(O.ovf_job, base);
    rebase(S.keys[0], base); rebase(S.keys[1], base); rebase(S.vals[0], base); rebase(S.vals[1], base);
    rebase(S.plan, base); rebase(S.lb[0], base); rebase(S.lb[1], base); rebase(S.tile_ctr, base);
    rebase(SD.t, base); rebase(SD.h, base); rebase(SD.unit, base); rebase(SD.panel, base); rebase(SD.job, base);
    rebase(SD.e, base); rebase(SD.eraw, base); rebase(SD.doi, base);
    rebase(C.flag, base); rebase(C.tile_cnt, base); rebase(C.a, base); rebase(C.b, base);
    rebase(JS.s_off, base); rebase(JS.c_off, base); rebase(JS.hits, base); rebase(R.d_toff, base);
    rebase(R.d_tn, base);
    JS.n_jobs = nj;
    JS.tally_count = R.d_tally_count;
    JS.tally_off = R.d_toff;
    JS.tally_n = R.d_tn;

    // wire the structs
    for (int j = 0; j < nj; ++j) {
        if (R.jobs[j].s_raw) continue;  // a job with its own singles buffer brings its own tallies
        R.jobs[j].tally_count = R.d_tally_count + R.tally_off[j];
        R.jobs[j].tally_efx = R.d_tally_efx + R.tally_off[j];
    }
    RunHeader *H = R.d_hdr;
    O.n_singles = &H->n_singles;
    O.s_cap = cap;
    O.n_hits = &H->n_hits;
    O.hit_cap = hcap;
    O.n_ovf = &H->n_ovf;
    O.ovf_cap = ocap;
    O.counters = H->counters;
    O.status = &H->status;
    WorkDev &W = R.W;
    W.jobs = R.d_jobs;
    W.n_jobs = njc;
    W.geoms = R.d_geoms;
    W.n_geoms = (int)R.geoms.size();
    W.chunk_start = R.d_chunk_start;
    W.total_chunks = R.live ? 0 : R.chunk_start[nj];
    W.next_chunk = &H->next_chunk;
    W.chunk_size = R.chunk_size;
    W.live_tail = R.live ? R.d_live : nullptr;
    W.live_closed = R.live ? reinterpret_cast<const int *>(R.d_live + 1) : nullptr;
    W.live_taken = R.live ? R.d_live + 2 : nullptr;
    int st = gpet_xs_table(&W.gtab, &W.ln_emin, &W.inv_h);
    if (st != GPET_OK) return st;
    S.max_tiles = tiles;
    S.cap = cap;
    S.n_in = &H->n_singles;
    S.status = &H->status;
    S.in_raw = O.s_raw;
    // the transport writes each single's sort key into the sort's first key buffer
    O.s_keys = S.keys[0];
    O.key_shift = S.job_shift;
    SD.n = &H->n_sorted;
    C.n = &H->n_coinc;
    C.window_ps = R.d_window;

    // upload descriptors (small; stream-ordered after the allocation)
    e = cudaMemcpyAsync(R.d_jobs, R.jobs.data(), sizeof(JobDev) * nj, cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(R.d_geoms, R.geoms.data(), sizeof(GeomDev) * R.geoms.size(), cudaMemcpyHostToDevice, up);
    for (size_t i = 0; i < R.geoms.size() && e == cudaSuccess; ++i)
        if (i < R.geom_pose.size() && !R.geom_pose[i].empty())
            e = cudaMemcpyAsync(R.d_pose + pose_off[i], R.geom_pose[i].data(), sizeof(float) * R.geom_pose[i].size(),
                                cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(R.d_chunk_start, R.chunk_start.data(), sizeof(unsigned long long) * (njc + 1),
                            cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(R.d_window, R.windows.data(), sizeof(uint64_t) * nj, cudaMemcpyHostToDevice, up);
    std::vector<long long> toff(R.tally_off.begin(), R.tally_off.end()), tn(R.job_crystals.begin(), R.job_crystals.end());
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.d_toff, toff.data(), sizeof(long long) * nj, cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.d_tn, tn.data(), sizeof(long long) * nj, cudaMemcpyHostToDevice, up);
    const unsigned long long live0[3] = {R.live_tail, 0ull, 0ull};  // published chunks, closed, claimed
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.d_live, live0, sizeof(live0), cudaMemcpyHostToDevice, up);
    // a digitize-only run's singles and tallies are written by other launches'
    // kernels, possibly running now: the copy engine clears its zeroed region
    for (size_t off = 0; R.digitize_only && off < R.zero_bytes && e == cudaSuccess; off += R.zeros_bytes) {
        if (!R.zeros || !R.zeros_bytes) return gpet_fail(GPET_ERR_INVALID_ARG, "digitize-only run without zeros");
        e = cudaMemcpyAsync(base + off, R.zeros, std::min(R.zeros_bytes, R.zero_bytes - off), cudaMemcpyHostToDevice,
                            up);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(up);  // host vectors may change after return
    R.h2d_bytes = sizeof(JobDev) * nj + sizeof(GeomDev) * R.geoms.size() + sizeof(float) * pose_floats +
                  sizeof(unsigned long long) * (njc + 1) +
                  sizeof(uint64_t) * nj + 2 * sizeof(long long) * nj;
    if (e != cudaSuccess) return gpet_cuda_fail(e, "upload of the job descriptors");
    if (R.live) R.geom_keys.resize(R.geoms.size());
    return GPET_OK;
}

static int stage_events(Run &R, unsigned *rec_flags) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        if (!R.ev[i]) e = cudaEventCreate(&R.ev[i]);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaEventCreate");
    // under stream capture the stage events must be external records, which
    // the replayed graph really records (a plain record there only orders
    // work); outside capture the external flag is refused, so record plainly
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(R.stream, &cap);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaStreamIsCapturing");
    *rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    return GPET_OK;
}

int run_enqueue_transport(Run &R) {
    unsigned rec_flags = 0;
    int st = stage_events(R, &rec_flags);
    if (st != GPET_OK) return st;
    cudaError_t e = cudaMemsetAsync(R.arena, 0, R.zero_bytes, R.stream);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaMemsetAsync");
    e = cudaEventRecordWithFlags(R.ev[0], R.stream, rec_flags);
    // A live launch's kernel waits on the host: nothing else is launched while
    // it runs (the re-simulation of overflowed histories follows at its close).
    if (e == cudaSuccess) e = launch_transport(R.W, R.O, R.cfg, R.stream, !R.live);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "transport launch");
    if (!R.live) {
        e = cudaEventRecordWithFlags(R.ev[1], R.stream, rec_flags);
        if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaEventRecord");
    }
    return GPET_OK;
}

int run_enqueue(Run &R) {
    int st = run_enqueue_transport(R);
    return st == GPET_OK ? run_enqueue_digitizer(R) : st;
}

int run_enqueue_digitizer(Run &R) {
    unsigned rec_flags = 0;
    int st = stage_events(R, &rec_flags);
    if (st != GPET_OK) return st;
    cudaError_t e = cudaSuccess;
    if (R.digitize_only) {  // no transport: both transport marks here
        e = cudaEventRecordWithFlags(R.ev[0], R.stream, rec_flags);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(R.ev[1], R.stream, rec_flags);
        if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaEventRecord");
    } else if (R.live) {    // closed: the re-simulation of overflowed histories, then the transport's end
        e = launch_transport_redo(R.W, R.O, R.cfg, R.stream);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(R.ev[1], R.stream, rec_flags);
        if (e != cudaSuccess) return gpet_cuda_fail(e, "re-simulation launch");
    }
    R.JS.n_jobs = (int)R.jobs.size();
    e = launch_sort_coinc(R.S, R.SD, R.C, R.cfg.sm_count, R.stream);
    if (e == cudaSuccess) e = launch_job_stats(R.SD, R.C, R.JS, R.stream);
    if (e == cudaSuccess && R.d_win_counts) {
        WinDev win{};
        win.n = (int)R.win_lo.size();
        for (int w = 0; w < win.n; ++w) { win.lo[w] = R.win_lo[w]; win.hi[w] = R.win_hi[w]; }
        e = launch_coinc_windows(R.SD, R.C, win, R.d_win_counts, R.S.cap, R.stream);
    }
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(R.ev[2], R.stream, rec_flags);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "sort / coincidence launch");
    return GPET_OK;
}

int run_collect(Run &R) {
    const size_t nj = R.jobs.size();
    R.s_off.resize(nj + 1);
    R.c_off.resize(nj + 1);
    R.job_hits.resize(nj);
    // A run with an upload stream (the serving loop's) is read back on that
    // stream, once the caller has seen its work complete: its own stream may
    // already hold the next launch.
    cudaStream_t rs = R.upload_stream ? R.upload_stream : R.stream;
    cudaError_t e = cudaMemcpyAsync(&R.h_hdr, R.d_hdr, sizeof(RunHeader), cudaMemcpyDeviceToHost, rs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(R.s_off.data(), R.JS.s_off, 8 * (nj + 1), cudaMemcpyDeviceToHost, rs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(R.c_off.data(), R.JS.c_off, 8 * (nj + 1), cudaMemcpyDeviceToHost, rs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.job_hits.data(), R.JS.hits, 8 * nj, cudaMemcpyDeviceToHost, rs);
    if (e == cudaSuccess && R.d_win_counts) {
        R.win_counts.resize(nj * R.win_lo.size());
        e = cudaMemcpyAsync(R.win_counts.data(), R.d_win_counts, 8 * R.win_counts.size(), cudaMemcpyDeviceToHost,
                            rs);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(rs);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "run read-back");
    if (R.ev[0] && cudaEventElapsedTime(&R.transport_ms, R.ev[0], R.ev[1]) != cudaSuccess) {
        R.transport_ms = -1.f;
        cudaGetLastError();  // a missing stage time is not an error of the run: clear it
    }
    if (R.ev[1] && cudaEventElapsedTime(&R.digitizer_ms, R.ev[1], R.ev[2]) != cudaSuccess) {
        R.digitizer_ms = -1.f;
        cudaGetLastError();
    }
    const RunHeader &H = R.h_hdr;
    if (H.status & kStatusTimeout)
        return gpet_fail(GPET_ERR_TIMEOUT, "a photon exceeded %d steps or %d Compton trials", kMaxSteps, kMaxTrials);
    if (H.n_singles > R.O.s_cap || (R.keep_hits && H.n_hits > R.O.hit_cap) || H.n_ovf > R.O.ovf_cap)
        return gpet_fail(GPET_ERR_OVERFLOW, "output capacity exceeded (singles %llu/%llu, hits %llu/%llu, ovf %llu/%llu)",
                         H.n_singles, R.O.s_cap, H.n_hits, R.O.hit_cap, H.n_ovf, R.O.ovf_cap);
    if (H.status & kStatusBadPhase)
        return gpet_fail(GPET_ERR_CUDA, "internal error: a history reached a phase no event handles");
    if (H.status & kStatusLiveStall)
        return gpet_fail(GPET_ERR_CUDA,
                         "internal error: a live launch waited %.3f s for work or its end (it last saw %llu "
                         "chunks published, closed flag %llu; the host had published %llu)",
                         H.counters[17] * 1e-9, H.counters[18], H.counters[19],
                         (unsigned long long)R.live_tail);
    if (H.status & kStatusSortStall)
        return gpet_fail(GPET_ERR_CUDA, "internal error: a time-sort pass did not complete (a tile copy or look-back wait ran out, or an offset was out of range)");
    if (H.status & kStatusOverflow)
        return gpet_fail(GPET_ERR_OVERFLOW, "a history touched more than 64 readout units");
    return GPET_OK;
}

void run_release(Run &R) {
    // Every run's work has been synchronised before its memory is released,
    // and a run may outlive the stream it ran on (a server worker's, a
    // caller's): free in the order of the legacy stream, never the run's own.
    if (R.arena) cudaFreeAsync(R.arena, cudaStreamLegacy);
    R.arena = nullptr;
    for (auto &e : R.ev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
}

Run::~Run() {
    run_release(*this);
    if (own_stream && stream) {
        cudaStreamSynchronize(stream);
        cudaStreamDestroy(stream);
    }
    if (on_release) on_release();
}

size_t run_footprint(uint64_t total_decays, int64_t total_crystals, int n_jobs, size_t n_geoms, bool keep_hits) {
    const uint64_t cap = std::min<uint64_t>(std::max<uint64_t>(65536, total_decays * 6 / 10), kMaxSinglesPerLaunch);
    const uint64_t hcap = keep_hits ? std::max<uint64_t>(65536, total_decays * 5 / 2) : 0;
    const uint64_t ocap = std::max<uint64_t>(4096, total_decays / 256);
    const uint64_t tiles = (cap + 4095) / 4096;
    size_t b = 0;
    b += sizeof(RunHeader) + 8 * 256 * 4 + 16 * (size_t)total_crystals;
    b += sizeof(JobDev) * n_jobs + (sizeof(GeomDev) + 16 * 4 * kMaxPanels) * n_geoms + 8 * (n_jobs + 1) + 8 * n_jobs;
    b += cap * sizeof(RawSingle);                // raw singles
    b += hcap * (8 + 8 + 4 * 4 + 12 + 4);        // hits
    b += ocap * 12;                              // overflow list
    b += cap * (2 * 8 + 2 * 4) + 2 * 256 * 8 * tiles + 8 * 4 + 128;  // sort (look-back words, tile counters)
    b += cap * (8 + 8 + 4 * 6);                  // sorted singles
    b += cap + 4 * tiles + 2 * 4 * (cap / 2 + 1); // coincidences
    b += 8 * (n_jobs + 1) * 2 + 8 * n_jobs * 3;  // per-job statistics
    return b + 64 * 256;                         // alignment slack
}

int run_with_retry(Run &R) {
    int st = GPET_OK;
    for (int attempt = 0; attempt < 2; ++attempt) {
        st = run_plan(R);
        if (st == GPET_OK) st = run_enqueue(R);
        if (st == GPET_OK) st = run_collect(R);
        if (st == GPET_ERR_OVERFLOW && R.h_hdr.n_singles > kMaxSinglesPerLaunch) {
            st = gpet_fail(GPET_ERR_OVERFLOW, "%llu singles in one launch, more than %llu: split the run",
                           R.h_hdr.n_singles, (unsigned long long)kMaxSinglesPerLaunch);
            break;
        }
        if (st == GPET_ERR_OVERFLOW && attempt == 0 && !(R.h_hdr.status & kStatusOverflow)) {
            // the device counters kept counting past the capacities: re-run with exact sizes
            R.caps.guess = false;
            R.caps.singles = std::max<uint64_t>(R.caps.singles, R.h_hdr.n_singles + 1024);
            R.caps.hits = std::max<uint64_t>(R.caps.hits, R.h_hdr.n_hits + 1024);
            R.caps.ovf = std::max<uint64_t>(R.caps.ovf, R.h_hdr.n_ovf + 1024);
            run_release(R);
            continue;
        }
        break;
    }
    if (st != GPET_OK) run_release(R);
    return st;
}

void fill_counts(const Run &R, int job, uint64_t n_decays, int64_t n_crystals, gpet_counts *c) {
    const RunHeader &H = R.h_hdr;
    std::memset(c, 0, sizeof(*c));
    c->n_decays = n_decays;
    c->hits = R.job_hits.empty() ? H.counters[5] : R.job_hits[job];
    c->singles = R.s_off.empty() ? H.n_sorted : R.s_off[job + 1] - R.s_off[job];
    c->coincidences = R.c_off.empty() ? H.n_coinc : R.c_off[job + 1] - R.c_off[job];
    c->n_crystals = n_crystals;
    c->det_steps = H.counters[0];
    c->flights = H.counters[1];
    c->compton_trials = H.counters[2];
    c->entered = H.counters[3];
    c->phantom_steps = H.counters[4];
    c->status = GPET_OK;
    c->transport_ms = R.transport_ms;
    c->digitizer_ms = R.digitizer_ms;
    c->h2d_bytes = R.h2d_bytes;
    c->wave_iterations = H.counters[6];
    c->wave_lanes = H.counters[7];
    c->screened_flights = H.counters[8];
    c->singles_formed = H.counters[9];
    for (int p = 0; p < 7; ++p) c->phase_events[p] = H.counters[10 + p];
}

// ---------------------------------------------------------------------------
// live launch: jobs appended while the transport kernel runs
// ---------------------------------------------------------------------------

// Staged host bytes of one append, copied in this order on the upload stream:
// the table entries first, the published chunk count last.
struct LiveStage {
    JobDev job;
    GeomDev geom;
    unsigned long long chunk_end, window, tail;
    long long toff, tn;
};

int run_live_append(Run &R, const JobDev &J_in, const gpet_scanner *sc, uint64_t window_ps) {
    if (!R.live || !R.arena || !sc) return gpet_fail(GPET_ERR_INVALID_ARG, "not a live launch");
    const size_t pose_need = sc->pose_dev.empty() ? 0 : align_up(sc->pose_dev.size(), 32);
    if (!R.stage || R.stage_bytes < sizeof(LiveStage) + sizeof(float) * pose_need)
        return gpet_fail(GPET_ERR_INVALID_ARG, "live launch without a large enough staging buffer");
    const int j = (int)R.jobs.size();
    if (j >= R.live_cap.jobs) return gpet_fail(GPET_ERR_BUSY, "live launch: job table full");
    if (J_in.t_span_ps > sort_time_limit(R.S.job_shift) - 0xFFFFFFFFull)
        return gpet_fail(GPET_ERR_BUSY, "live launch: acquisition too long for its time key");
    const std::string key = gpet_geometry_key(sc);
    int gi = -1;
    for (size_t i = 0; i < R.geom_keys.size(); ++i)
        if (R.geom_keys[i] == key) { gi = (int)i; break; }
    const bool new_geom = gi < 0;
    if (new_geom && ((int)R.geoms.size() >= R.live_cap.geoms ||
                     R.live_pose_used + pose_need > std::max(R.live_cap.pose_floats, R.live_pose_used)))
        return gpet_fail(GPET_ERR_BUSY, "live launch: geometry table full");
    // a job with its own singles buffer brings its own tallies
    const int64_t crystals = J_in.s_raw ? 0 : sc->n_crystals;
    if (R.live_tally_used + crystals > R.live_cap.crystals)
        return gpet_fail(GPET_ERR_BUSY, "live launch: tally space full");
    LiveStage *S = static_cast<LiveStage *>(R.stage);
    float *pose_stage = reinterpret_cast<float *>(S + 1);
    if (new_geom) {
        gi = (int)R.geoms.size();
        S->geom = sc->g;
        S->geom.pose = pose_need ? reinterpret_cast<const float4 *>(R.d_pose + R.live_pose_used) : nullptr;
        if (pose_need) std::memcpy(pose_stage, sc->pose_dev.data(), sizeof(float) * sc->pose_dev.size());
    }
    S->job = J_in;
    S->job.geom = gi;
    if (!J_in.s_raw) {
        S->job.tally_count = R.d_tally_count + R.live_tally_used;
        S->job.tally_efx = R.d_tally_efx + R.live_tally_used;
    }
    const uint64_t chunks = (J_in.n_hist + R.chunk_size - 1) / R.chunk_size;
    S->chunk_end = R.live_tail + chunks;
    S->window = window_ps;
    S->tail = S->chunk_end;
    S->toff = R.live_tally_used;
    S->tn = crystals;
    cudaStream_t up = R.upload_stream;
    cudaError_t e = cudaSuccess;
    if (new_geom) {
        e = cudaMemcpyAsync(R.d_geoms + gi, &S->geom, sizeof(GeomDev), cudaMemcpyHostToDevice, up);
        if (e == cudaSuccess && pose_need)
            e = cudaMemcpyAsync(R.d_pose + R.live_pose_used, pose_stage, sizeof(float) * sc->pose_dev.size(),
                                cudaMemcpyHostToDevice, up);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.d_jobs + j, &S->job, sizeof(JobDev), cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.d_window + j, &S->window, 8, cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.d_toff + j, &S->toff, 8, cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.d_tn + j, &S->tn, 8, cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.d_chunk_start + j + 1, &S->chunk_end, 8, cudaMemcpyHostToDevice, up);
    // copies of one stream complete in order: the tail lands after the entries
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.d_live, &S->tail, 8, cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaStreamSynchronize(up);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "live launch append");
    if (new_geom) {
        R.geoms.push_back(S->geom);
        R.geom_pose.push_back(sc->pose_dev);
        R.geom_keys.push_back(key);
        R.live_pose_used += pose_need;
        R.h2d_bytes += sizeof(GeomDev) + sizeof(float) * sc->pose_dev.size();
    }
    R.jobs.push_back(S->job);
    R.job_crystals.push_back(crystals);
    R.windows.push_back(window_ps);
    R.tally_off.push_back(R.live_tally_used);
    R.live_tally_used += crystals;
    R.total_crystals = R.live_tally_used;
    R.chunk_start[j + 1] = S->chunk_end;
    R.live_tail = S->chunk_end;
    R.h2d_bytes += sizeof(JobDev) + 5 * 8;
    return GPET_OK;
}

int run_live_close(Run &R) {
    if (!R.live || !R.arena || !R.stage) return gpet_fail(GPET_ERR_INVALID_ARG, "not a live launch");
    unsigned long long *one = static_cast<unsigned long long *>(R.stage);
    *one = 1ull;  // the closed flag is the low int of its word (little-endian)
    cudaError_t e = cudaMemcpyAsync(R.d_live + 1, one, 8, cudaMemcpyHostToDevice, R.upload_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(R.upload_stream);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "live launch close");
    return GPET_OK;
}

// A copy of a collected run's results -- time-ordered singles, coincidences,
// tallies and the per-job segments -- in device memory of exactly their size,
// made by the copy engine on `st`.  The serving loop hands out views of the
// copy, so that results a client keeps do not hold a launch's buffers.
std::shared_ptr<Run> run_compact(const Run &R, cudaStream_t st, int *status) {
    auto C = std::make_shared<Run>();
    const size_t nj = R.jobs.size();
    if (R.s_off.size() != nj + 1 || R.c_off.size() != nj + 1) {
        *status = gpet_fail(GPET_ERR_INVALID_ARG, "compact copy of a run without collected results");
        return nullptr;
    }
    const uint64_t ns = R.s_off[nj], nc = R.c_off[nj];
    const size_t tc = (size_t)R.total_crystals;
    Carver cv;
    SinglesDev &SD = C->SD;
    cv.take(SD.t, ns); cv.take(SD.h, ns); cv.take(SD.unit, ns); cv.take(SD.panel, ns); cv.take(SD.job, ns);
    cv.take(SD.e, ns); cv.take(SD.eraw, ns); cv.take(SD.doi, ns);
    cv.take(C->C.a, nc); cv.take(C->C.b, nc);
    cv.take(C->d_tally_count, tc); cv.take(C->d_tally_efx, tc);
    C->arena_bytes = align_up(cv.off, 256);
    cudaError_t e = cudaMallocAsync(&C->arena, C->arena_bytes, st);
    if (e != cudaSuccess) {
        C->arena = nullptr;
        *status = e == cudaErrorMemoryAllocation ? gpet_fail(GPET_ERR_OOM, "compact copy of %zu bytes", C->arena_bytes)
                                                 : gpet_cuda_fail(e, "cudaMallocAsync");
        return nullptr;
    }
    char *base = static_cast<char *>(C->arena);
    rebase(SD.t, base); rebase(SD.h, base); rebase(SD.unit, base); rebase(SD.panel, base); rebase(SD.job, base);
    rebase(SD.e, base); rebase(SD.eraw, base); rebase(SD.doi, base);
    rebase(C->C.a, base); rebase(C->C.b, base);
    rebase(C->d_tally_count, base); rebase(C->d_tally_efx, base);
    struct Part { void *dst; const void *src; size_t bytes; };
    const Part parts[] = {{SD.t, R.SD.t, 8 * ns}, {SD.h, R.SD.h, 8 * ns}, {SD.unit, R.SD.unit, 4 * ns},
                          {SD.panel, R.SD.panel, 4 * ns}, {SD.job, R.SD.job, 4 * ns}, {SD.e, R.SD.e, 4 * ns},
                          {SD.eraw, R.SD.eraw, 4 * ns}, {SD.doi, R.SD.doi, 4 * ns}, {C->C.a, R.C.a, 4 * nc},
                          {C->C.b, R.C.b, 4 * nc}, {C->d_tally_count, R.d_tally_count, 8 * tc},
                          {C->d_tally_efx, R.d_tally_efx, 8 * tc}};
    for (const Part &p : parts)
        if (e == cudaSuccess && p.bytes) e = cudaMemcpyAsync(p.dst, p.src, p.bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *status = gpet_cuda_fail(e, "compact copy of a run's results");
        return nullptr;
    }
    C->device = R.device;
    C->jobs = R.jobs;
    C->job_crystals = R.job_crystals;
    C->tally_off = R.tally_off;
    C->total_crystals = R.total_crystals;
    C->s_off = R.s_off;
    C->c_off = R.c_off;
    C->job_hits = R.job_hits;
    C->h_hdr = R.h_hdr;
    C->transport_ms = R.transport_ms;
    C->digitizer_ms = R.digitizer_ms;
    C->h2d_bytes = R.h2d_bytes;
    C->keep_hits = false;
    *status = GPET_OK;
    return C;
}

int run_live_taken(Run &R, uint64_t *taken) {
    if (!R.live || !R.arena || !R.stage) return gpet_fail(GPET_ERR_INVALID_ARG, "not a live launch");
    unsigned long long *v = static_cast<unsigned long long *>(R.stage);
    cudaError_t e = cudaMemcpyAsync(v, R.d_live + 2, 8, cudaMemcpyDeviceToHost, R.upload_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(R.upload_stream);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "live launch progress read");
    *taken = *v;
    return GPET_OK;
}

}  // namespace gpet

using namespace gpet;

extern "C" int gpet_simulate(gpet_scanner *sc, const gpet_source *src, const gpet_digitizer *dg, uint64_t n_decays,
                             uint64_t seed, const gpet_options *opt, gpet_result **out) {
    if (!out) return gpet_fail(GPET_ERR_INVALID_ARG, "out is NULL");
    JobDev J;
    int st = gpet_make_job(sc, src, dg, n_decays, seed, J, opt ? opt->h_begin : 0, opt ? opt->h_end : 0);
    if (st != GPET_OK) return st;
    gpet_result *res = new (std::nothrow) gpet_result();
    if (!res) return gpet_fail(GPET_ERR_OOM, "host allocation of the result failed");
    res->run = std::make_shared<Run>();
    Run &R = *res->run;
    st = run_default_cfg(R, opt, sc);
    if (st != GPET_OK) { delete res; return st; }
    R.jobs = {J};
    R.geoms = {sc->g};
    R.geom_pose = {sc->pose_dev};
    R.job_crystals = {sc->n_crystals};
    R.windows = {(uint64_t)std::llround(dg->coinc_window_ns * 1000.0)};
    R.caps.singles = std::max<uint64_t>(65536, J.n_hist * 6 / 10);
    R.caps.hits = R.keep_hits ? std::max<uint64_t>(65536, J.n_hist * 5 / 2) : 0;
    R.caps.ovf = std::max<uint64_t>(4096, J.n_hist / 256);
    st = run_with_retry(R);
    if (st != GPET_OK) {
        delete res;
        return st;
    }
    fill_counts(R, 0, n_decays, sc->n_crystals, &res->counts);
    *out = res;
    return GPET_OK;
}

extern "C" int gpet_result_counts(const gpet_result *r, gpet_counts *out) {
    if (!r || !out) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    *out = r->counts;
    return GPET_OK;
}

struct ArrayView {
    const void *ptr;
    size_t bytes;
};

static int result_array(const gpet_result *r, int32_t which, ArrayView &v) {
    const Run &R = *r->run;
    const int j = r->job;
    const uint64_t s0 = R.s_off[j], ns = R.s_off[j + 1] - s0, c0 = R.c_off[j], nc = R.c_off[j + 1] - c0;
    const uint64_t nh = std::min<uint64_t>(R.h_hdr.n_hits, R.O.hit_cap);
    switch (which) {
        case GPET_SINGLES_T_PS: v = {R.SD.t + s0, ns * 8}; break;
        case GPET_SINGLES_H: v = {R.SD.h + s0, ns * 8}; break;
        case GPET_SINGLES_UNIT: v = {R.SD.unit + s0, ns * 4}; break;
        case GPET_SINGLES_PANEL: v = {R.SD.panel + s0, ns * 4}; break;
        case GPET_SINGLES_E: v = {R.SD.e + s0, ns * 4}; break;
        case GPET_SINGLES_E_RAW: v = {R.SD.eraw + s0, ns * 4}; break;
        case GPET_SINGLES_DOI: v = {R.SD.doi + s0, ns * 4}; break;
        case GPET_COINC_A: v = {R.C.a + c0, nc * 4}; break;
        case GPET_COINC_B: v = {R.C.b + c0, nc * 4}; break;
        case GPET_TALLY_COUNT: v = {R.d_tally_count + R.tally_off[j], (size_t)R.job_crystals[j] * 8}; break;
        case GPET_TALLY_EFX: v = {R.d_tally_efx + R.tally_off[j], (size_t)R.job_crystals[j] * 8}; break;
        case GPET_HITS_H: v = {R.O.hit_h, nh * 8}; break;
        case GPET_HITS_GSTEP: v = {R.O.hit_gstep, nh * 4}; break;
        case GPET_HITS_CRYSTAL: v = {R.O.hit_crystal, nh * 4}; break;
        case GPET_HITS_LAYER: v = {R.O.hit_layer, nh * 4}; break;
        case GPET_HITS_WUV: v = {R.O.hit_wuv, nh * 12}; break;
        case GPET_HITS_E: v = {R.O.hit_e, nh * 4}; break;
        case GPET_HITS_T_PS: v = {R.O.hit_t, nh * 8}; break;
        default: return gpet_fail(GPET_ERR_INVALID_ARG, "unknown result array %d", which);
    }
    if (which >= GPET_HITS_H && which <= GPET_HITS_T_PS && !R.keep_hits)
        return gpet_fail(GPET_ERR_INVALID_ARG, "hits were not kept (gpet_options.keep_hits = 0)");
    if (which >= GPET_HITS_H && which <= GPET_HITS_T_PS && R.jobs.size() > 1)
        return gpet_fail(GPET_ERR_INVALID_ARG, "hit lists are kept for single-job runs only");
    return GPET_OK;
}

extern "C" int gpet_result_copy(const gpet_result *r, int32_t which, void *dst, size_t cap_bytes) {
    if (!r || (!dst && cap_bytes)) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    ArrayView v{nullptr, 0};
    int st = result_array(r, which, v);
    if (st != GPET_OK) return st;
    if (cap_bytes < v.bytes)
        return gpet_fail(GPET_ERR_TOO_SMALL, "array %d needs %zu bytes, got %zu", which, v.bytes, cap_bytes);
    if (v.bytes == 0) return GPET_OK;
    cudaError_t e = cudaMemcpy(dst, v.ptr, v.bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "result copy");
    if (which == GPET_COINC_A || which == GPET_COINC_B) {
        // device indices count from the run's first single; renumber from the view's
        const int32_t s0 = (int32_t)r->run->s_off[r->job];
        if (s0) {
            int32_t *p = static_cast<int32_t *>(dst);
            for (size_t i = 0; i < v.bytes / 4; ++i) p[i] -= s0;
        }
    }
    return GPET_OK;
}

static int copy_run(const gpet_result *r, int32_t which, void *dst, size_t cap_bytes, size_t *bytes, bool async,
                    cudaStream_t stream);

// Device-to-host copy made by the SMs: each thread loads 16-byte words of the
// device array and stores them into page-locked host memory through its device
// mapping; the n4 (< 4) trailing 4-byte words go to the first block.  The copy
// engines' reads of device memory that had been freed and allocated again were
// measured at a fifth of the host link's rate once other GPU work had run on the
// device, where these stores kept the link's rate.
__global__ void k_store_to_host(const uint4 *__restrict__ src, uint4 *dst, size_t n16,
                                const uint32_t *__restrict__ src4, uint32_t *dst4, unsigned n4) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = __ldcs(src + i);
    if (blockIdx.x == 0 && threadIdx.x < n4) dst4[threadIdx.x] = src4[threadIdx.x];
}

// The device's address of dst when it is page-locked host memory that the
// device can store to, and both ends suit the 16-byte copy; else NULL.
static void *store_target(void *dst, const void *src, size_t bytes) {
    if ((reinterpret_cast<uintptr_t>(src) & 15) || (bytes & 3)) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, dst) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    if (reinterpret_cast<uintptr_t>(a.devicePointer) & 15) return nullptr;
    return a.devicePointer;
}

// load the copy kernel with the others (internal.h)
cudaError_t gpet::preload_copy_kernels() {
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(k_store_to_host));
}

static cudaError_t store_to_host(void *dst_dev, const void *src, size_t bytes, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t n16 = bytes / 16;
    const unsigned n4 = (unsigned)((bytes - 16 * n16) / 4);
    const size_t want = (n16 + 511) / 512;
    const int grid = (int)std::max<size_t>(1, std::min<size_t>(want, (size_t)sms * 4));
    k_store_to_host<<<grid, 512, 0, st>>>(static_cast<const uint4 *>(src), static_cast<uint4 *>(dst_dev), n16,
                                          reinterpret_cast<const uint32_t *>(static_cast<const char *>(src) + 16 * n16),
                                          reinterpret_cast<uint32_t *>(static_cast<char *>(dst_dev) + 16 * n16), n4);
    return cudaGetLastError();
}

extern "C" int gpet_result_copy_run(const gpet_result *r, int32_t which, void *dst, size_t cap_bytes,
                                    size_t *bytes) {
    return copy_run(r, which, dst, cap_bytes, bytes, false, nullptr);
}

extern "C" int gpet_result_copy_run_async(const gpet_result *r, int32_t which, void *dst, size_t cap_bytes,
                                          size_t *bytes, void *stream) {
    return copy_run(r, which, dst, cap_bytes, bytes, true, static_cast<cudaStream_t>(stream));
}

static int copy_run(const gpet_result *r, int32_t which, void *dst, size_t cap_bytes, size_t *bytes, bool async,
                    cudaStream_t stream) {
    if (!r || (!dst && cap_bytes)) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    const Run &R = *r->run;
    const size_t nj = R.jobs.size();
    if (R.s_off.size() != nj + 1 || R.c_off.size() != nj + 1)
        return gpet_fail(GPET_ERR_INVALID_ARG, "the run has no collected results");
    const uint64_t ns = R.s_off[nj], nc = R.c_off[nj];
    ArrayView v{nullptr, 0};
    switch (which) {
        case GPET_SINGLES_T_PS: v = {R.SD.t, ns * 8}; break;
        case GPET_SINGLES_H: v = {R.SD.h, ns * 8}; break;
        case GPET_SINGLES_UNIT: v = {R.SD.unit, ns * 4}; break;
        case GPET_SINGLES_PANEL: v = {R.SD.panel, ns * 4}; break;
        case GPET_SINGLES_E: v = {R.SD.e, ns * 4}; break;
        case GPET_SINGLES_E_RAW: v = {R.SD.eraw, ns * 4}; break;
        case GPET_SINGLES_DOI: v = {R.SD.doi, ns * 4}; break;
        case GPET_COINC_A: v = {R.C.a, nc * 4}; break;
        case GPET_COINC_B: v = {R.C.b, nc * 4}; break;
        case GPET_TALLY_COUNT: v = {R.d_tally_count, (size_t)R.total_crystals * 8}; break;
        case GPET_TALLY_EFX: v = {R.d_tally_efx, (size_t)R.total_crystals * 8}; break;
        default: {
            const int st = result_array(r, which, v);  // hit lists: single-job runs only
            if (st != GPET_OK) return st;
        }
    }
    if (bytes) *bytes = v.bytes;
    if (!dst) return GPET_OK;
    if (cap_bytes < v.bytes)
        return gpet_fail(GPET_ERR_TOO_SMALL, "array %d needs %zu bytes, got %zu", which, v.bytes, cap_bytes);
    if (v.bytes == 0) return GPET_OK;
    cudaError_t e;
    if (void *dd = store_target(dst, v.ptr, v.bytes)) {
        // the blocking form orders itself like cudaMemcpy: on the legacy stream
        e = store_to_host(dd, v.ptr, v.bytes, async ? stream : cudaStreamLegacy);
        if (e == cudaSuccess && !async) e = cudaStreamSynchronize(cudaStreamLegacy);
    } else {
        e = async ? cudaMemcpyAsync(dst, v.ptr, v.bytes, cudaMemcpyDeviceToHost, stream)
                  : cudaMemcpy(dst, v.ptr, v.bytes, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return gpet_cuda_fail(e, "result copy");
    return GPET_OK;
}

extern "C" const void *gpet_result_device_ptr(const gpet_result *r, int32_t which) {
    if (!r) return nullptr;
    ArrayView v{nullptr, 0};
    if (result_array(r, which, v) != GPET_OK) return nullptr;
    return v.ptr;
}

extern "C" void gpet_result_free(gpet_result *r) { delete r; }
