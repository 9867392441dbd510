// event_costs.cu -- per-event cost of the transport, measured on micro-kernels.
//
// The transport kernels advance many histories at once through the events of
// Sec. 2.1 and 2.3 (decay, phantom step, flight, detector step, finish).  This
// file times each event type alone.  A capture pass runs histories of the
// caller's own workload through the events, one lane per history, and keeps a
// pool of the states that entered each phase; then, for each phase, a kernel in
// which every lane of every warp runs that phase's event on pool states, over
// and over, is timed with CUDA events.  Its time per event is what the event
// costs when the whole GPU runs nothing else at full SIMT width -- without the
// regrouping, barriers and refills of a wavefront kernel.  The sum over a
// launch's events of these costs, over the launch's transport time, is the
// transport's event-isolated roofline fraction.
#include <algorithm>
#include <cstring>
#include <vector>

#include "host.h"

namespace gpet {

namespace {

constexpr int kPhases = 7;       // phases 1..6 (0 = idle)
constexpr int kListS = 6;        // singles-list entries kept per captured state
constexpr int kCostThreads = 256;

struct SlEntry {
    uint32_t unit;
    float e;
    uint32_t dt;
    float ew;
};

struct PoolDev {
    PState *st[kPhases];          // states captured on entry to each phase
    SlEntry *sl[kPhases];         // their singles lists, kListS entries each
    unsigned long long *n;        // [kPhases] states taken per phase
    unsigned long long cap;       // pool size per phase
};

// Capture: histories 0.. of job 0, one per thread, run event by event with no
// regrouping; the state entering each phase is copied into that phase's pool
// while it has room.  A finished history is not digitized here (the finish
// pool keeps its singles list).
__global__ void __launch_bounds__(128) k_capture(WorkDev W, OutDev O, PoolDev P) {
    uint32_t l_unit[kListS];
    float l_e[kListS];
    uint32_t l_dt[kListS];
    float l_ew[kListS];
    const SinglesList SL{l_unit, l_e, l_dt, l_ew, 1};
    const JobDev &J = W.jobs[0];
    const GeomDev &g = W.geoms[J.geom];
    Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
    int status = kStatusOk;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < J.n_hist; i += stride) {
        PState s;
        s.h = J.h_base + i;
        s.job = 0;
        s.phase = kPhSource;
        s.nsing = 0;
        s.ovf = 0;
        while (s.phase != kPhIdle) {
            const uint32_t p = s.phase;
            if (p < kPhases && *reinterpret_cast<volatile unsigned long long *>(P.n + p) < P.cap) {
                const unsigned long long k = atomicAdd(P.n + p, 1ull);
                if (k < P.cap) {
                    P.st[p][k] = s;
                    for (int j = 0; j < kListS; ++j)
                        P.sl[p][k * kListS + j] = j < (int)s.nsing ? SlEntry{l_unit[j], l_e[j], l_dt[j], l_ew[j]}
                                                                   : SlEntry{0u, 0.f, 0u, 0.f};
                }
            }
            int st = kStatusOk;
            switch (p) {
                case kPhSource: ev_source(J, g, s, cnt); break;
                case kPhPhantom: st = ev_phantom(J, g, W, s, cnt); break;
                case kPhFlight: case kPhFlightOut: ev_flight(J, g, s, cnt); break;
                case kPhPanel: st = ev_panel<true>(J, g, W, O, s, SL, kListS, cnt); break;
                case kPhFinish: s.phase = kPhIdle; break;
                default: st = kStatusBadPhase; break;
            }
            if (st != kStatusOk) { status |= st; s.phase = kPhIdle; }
        }
    }
    if (status) atomicOr(O.status, status);
}

// One event type alone: every lane takes a pool state of phase PH and runs
// its event `reps` times (a decay on a fresh history each time), so that every
// warp executes that event's code with all lanes busy.
template <int PH>
__global__ void __launch_bounds__(kCostThreads) k_event_alone(WorkDev W, OutDev O, PoolDev P, int reps,
                                                             unsigned long long *sink) {
    __shared__ uint32_t s_unit[kListS * kCostThreads];
    __shared__ float s_e[kListS * kCostThreads];
    __shared__ uint32_t s_dt[kListS * kCostThreads];
    __shared__ float s_ew[kListS * kCostThreads];
    const unsigned long long n = min(P.n[PH], P.cap);
    const unsigned long long gid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long i = gid % n;
    const PState s0 = P.st[PH][i];
    for (int j = 0; j < kListS; ++j) {
        const SlEntry e = P.sl[PH][i * kListS + j];
        s_unit[j * kCostThreads + threadIdx.x] = e.unit;
        s_e[j * kCostThreads + threadIdx.x] = e.e;
        s_dt[j * kCostThreads + threadIdx.x] = e.dt;
        s_ew[j * kCostThreads + threadIdx.x] = e.ew;
    }
    const SinglesList SL{s_unit + threadIdx.x, s_e + threadIdx.x, s_dt + threadIdx.x, s_ew + threadIdx.x,
                         kCostThreads};
    const JobDev &J = W.jobs[s0.job];
    const GeomDev &g = W.geoms[J.geom];
    Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t acc = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        PState s = s0;
        if (PH == kPhSource) s.h = s0.h + (unsigned long long)r * stride;
        if (PH == kPhSource) ev_source(J, g, s, cnt);
        else if (PH == kPhPhantom) ev_phantom(J, g, W, s, cnt);
        else if (PH == kPhFlight || PH == kPhFlightOut) ev_flight(J, g, s, cnt);
        else if (PH == kPhPanel) ev_panel<true>(J, g, W, O, s, SL, kListS, cnt);
        else if (PH == kPhFinish) ev_finish<false>(W.jobs, W.geoms, O, s, true, SL, kFullMask, cnt);
        acc ^= __float_as_uint(s.x) ^ __float_as_uint(s.E) ^ s.phase ^ cnt.singles ^ cnt.hits;
    }
    if (acc == 0x9E3779B9u) *sink = acc;  // never true in practice; keeps the work
}

template <int PH>
cudaError_t time_event(const Run &R, const PoolDev &P, int sms, cudaStream_t st, unsigned long long *sink,
                       double *ns_per_event) {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_event_alone<PH>, kCostThreads, 0);
    if (e != cudaSuccess) return e;
    const int grid = sms * std::max(occ, 1);
    const int reps = 16;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 1e30f;
    for (int it = 0; it < 4 && e == cudaSuccess; ++it) {  // the first launch warms caches and tables
        // every launch appends its singles from the start of the buffer
        if (e == cudaSuccess) e = cudaMemsetAsync(R.O.n_singles, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(R.O.n_ovf, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = cudaEventRecord(a, st);
        if (e == cudaSuccess) {
            k_event_alone<PH><<<grid, kCostThreads, 0, st>>>(R.W, R.O, P, reps, sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && it > 0) best = std::min(best, ms);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e == cudaSuccess) *ns_per_event = best * 1e6 / ((double)grid * kCostThreads * reps);
    return e;
}

}  // namespace

}  // namespace gpet

using namespace gpet;

extern "C" int gpet_event_costs(gpet_scanner *sc, const gpet_source *src, const gpet_digitizer *dg,
                                uint64_t n_sample, uint64_t seed, double *ns_per_event, uint64_t *states) {
    if (!sc || !src || !dg || !ns_per_event) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    if (n_sample < 1000 || n_sample > (1ull << 32))
        return gpet_fail(GPET_ERR_INVALID_ARG, "n_sample must be in [1000, 2^32]");
    for (int p = 0; p < kPhases; ++p) ns_per_event[p] = 0.0;
    JobDev J;
    int st = gpet_make_job(sc, src, dg, n_sample, seed, J);
    if (st != GPET_OK) return st;
    Run R;
    st = run_default_cfg(R, nullptr, sc);
    if (st != GPET_OK) return st;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaStreamCreate");
    R.stream = cs;
    R.own_stream = true;
    R.jobs = {J};
    R.geoms = {sc->g};
    R.geom_pose = {sc->pose_dev};
    R.job_crystals = {sc->n_crystals};
    R.windows = {(uint64_t)std::llround(dg->coinc_window_ns * 1000.0)};
    // the finish micro-kernel appends singles: room for every lane of every rep
    R.caps.singles = 1ull << 23;
    R.caps.guess = false;
    R.caps.ovf = 4096;
    st = run_plan(R);
    if (st != GPET_OK) return st;
    e = cudaMemsetAsync(R.arena, 0, R.zero_bytes, cs);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaMemsetAsync");
    // state pools
    PoolDev P{};
    P.cap = 1ull << 16;
    const size_t st_bytes = sizeof(PState) * P.cap, sl_bytes = sizeof(SlEntry) * kListS * P.cap;
    void *pool = nullptr;
    const size_t pool_bytes = kPhases * (st_bytes + sl_bytes) + 256;
    e = cudaMallocAsync(&pool, pool_bytes, cs);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "pool allocation");
    char *b = static_cast<char *>(pool);
    P.n = reinterpret_cast<unsigned long long *>(b);
    for (int p = 0; p < kPhases; ++p) {
        P.st[p] = reinterpret_cast<PState *>(b + 256 + p * (st_bytes + sl_bytes));
        P.sl[p] = reinterpret_cast<SlEntry *>(b + 256 + p * (st_bytes + sl_bytes) + st_bytes);
    }
    unsigned long long *sink = reinterpret_cast<unsigned long long *>(b + 128);
    e = cudaMemsetAsync(pool, 0, 256, cs);
    if (e == cudaSuccess) {
        k_capture<<<R.cfg.sm_count * 8, 128, 0, cs>>>(R.W, R.O, P);
        e = cudaGetLastError();
    }
    unsigned long long taken[kPhases] = {0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(taken, P.n, sizeof(taken), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        cudaFreeAsync(pool, cs);
        return gpet_cuda_fail(e, "state capture");
    }
    double ns[kPhases] = {0};
    if (e == cudaSuccess && taken[kPhSource]) e = time_event<kPhSource>(R, P, R.cfg.sm_count, cs, sink, &ns[kPhSource]);
    if (e == cudaSuccess && taken[kPhPhantom]) e = time_event<kPhPhantom>(R, P, R.cfg.sm_count, cs, sink, &ns[kPhPhantom]);
    if (e == cudaSuccess && taken[kPhFlight]) e = time_event<kPhFlight>(R, P, R.cfg.sm_count, cs, sink, &ns[kPhFlight]);
    if (e == cudaSuccess && taken[kPhPanel]) e = time_event<kPhPanel>(R, P, R.cfg.sm_count, cs, sink, &ns[kPhPanel]);
    if (e == cudaSuccess && taken[kPhFinish]) e = time_event<kPhFinish>(R, P, R.cfg.sm_count, cs, sink, &ns[kPhFinish]);
    if (e == cudaSuccess && taken[kPhFlightOut])
        e = time_event<kPhFlightOut>(R, P, R.cfg.sm_count, cs, sink, &ns[kPhFlightOut]);
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &R.d_hdr->status, sizeof(int), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    cudaFreeAsync(pool, cs);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "event micro-kernels");
    if (status & (kStatusTimeout | kStatusBadPhase))
        return gpet_fail(GPET_ERR_TIMEOUT, "a sampled history hit an iteration cap");
    for (int p = 0; p < kPhases; ++p) {
        ns_per_event[p] = ns[p];
        if (states) states[p] = std::min<unsigned long long>(taken[p], P.cap);
    }
    return GPET_OK;
}
