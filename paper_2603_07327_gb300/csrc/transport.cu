// transport.cu -- photon-pair transport kernels.
//
//   k_transport_loop  : persistent CTAs; every lane owns one history and runs
//                       one event per loop iteration; idle lanes are refilled
//                       warp-wide (one atomic per chunk of histories).
//   k_transport_wave  : wavefront form with warp-ballot regrouping (transport_wave.cu).
//   k_transport_cta   : wavefront form with one event per CTA and iteration, the
//                       default launch form (transport_cta.cu).
//   k_transport_redo  : exact fallback for the rare history whose on-chip
//                       singles list overflowed: re-simulated alone with a
//                       long list (the RNG is addressed by history id, so the
//                       replay is bit for bit the same history).
#include "internal.h"
#include "transport.cuh"

namespace gpet {

__device__ __forceinline__ void flush_counters(const OutDev &O, const Counters &c) {
    const uint32_t v[8] = {c.det_steps, c.flights, c.trials, c.entered, c.ph_steps, c.hits, c.screened, c.singles};
    const int slot[8] = {0, 1, 2, 3, 4, 5, 8, 9};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t x = __reduce_add_sync(kFullMask, v[i]);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(O.counters + slot[i], (unsigned long long)x);
    }
}

template <int S>
__global__ void __launch_bounds__(256) k_transport_loop(WorkDev W, OutDev O, int ng_smem) {
    extern __shared__ __align__(16) uint8_t smem[];
    GeomDev *sgeom = reinterpret_cast<GeomDev *>(smem);
    uint32_t *sl_unit = reinterpret_cast<uint32_t *>(sgeom + ng_smem);
    float *sl_e = reinterpret_cast<float *>(sl_unit + S * blockDim.x);
    uint32_t *sl_dt = reinterpret_cast<uint32_t *>(sl_e + S * blockDim.x);
    float *sl_ew = reinterpret_cast<float *>(sl_dt + S * blockDim.x);
    stage_geometry(W, sgeom, ng_smem);
    __syncthreads();

    const SinglesList SL{sl_unit + threadIdx.x, sl_e + threadIdx.x, sl_dt + threadIdx.x, sl_ew + threadIdx.x,
                         (int)blockDim.x};
    PState s;
    s.phase = kPhIdle;
    s.job = 0;
    Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
    Refill rf;
    refill_init(rf);
    int status = kStatusOk;
    LiveIdle idle;
    live_idle_reset(idle);

    for (;;) {
        const uint32_t need = __ballot_sync(kFullMask, s.phase == kPhIdle);
        if (need) {
            bool got;
            uint64_t h = 0;
            int job = 0;
            warp_refill(W, need, rf, got, h, job);
            if (got) {
                s.h = h;
                s.job = job;
                s.phase = kPhSource;
            }
        }
        if (__all_sync(kFullMask, s.phase == kPhIdle)) {
            // the queue is exhausted, or a live launch has nothing published yet
            if (!rf.waiting || __any_sync(kFullMask, live_idle_wait(idle, status, W, O))) break;
            continue;
        }
        live_idle_reset(idle);

        const JobDev &J = W.jobs[s.job];
        const GeomDev &g = J.geom < ng_smem ? sgeom[J.geom] : W.geoms[J.geom];
        int st = kStatusOk;
        switch (s.phase) {
            case kPhSource: ev_source(J, g, s, cnt); break;
            case kPhPhantom: st = ev_phantom(J, g, W, s, cnt); break;
            case kPhFlight: case kPhFlightOut: ev_flight(J, g, s, cnt); break;
            case kPhPanel: st = ev_panel<true>(J, g, W, O, s, SL, S, cnt); break;
            case kPhIdle: case kPhFinish: break;
            default: st = kStatusBadPhase; break;
        }
        if (st != kStatusOk) {          // iteration cap hit: abandon the history, flag the run
            status |= st;
            s.phase = kPhIdle;
        }
        const bool fin = s.phase == kPhFinish;
        if (__any_sync(kFullMask, fin)) {
            ev_finish(W.jobs, W.geoms, O, s, fin, SL, kFullMask, cnt);
            if (fin) s.phase = kPhIdle;
        }
    }
    flush_counters(O, cnt);
    if (status) atomicOr(O.status, status);
}

// Re-simulate the histories listed in O.ovf_* with a 64-entry singles list in
// local memory.  Tallies and hits were already counted by the main kernel, so
// only the singles are emitted here.
__global__ void __launch_bounds__(128) k_transport_redo(WorkDev W, OutDev O) {
    constexpr int S = 64;
    uint32_t l_unit[S];
    float l_e[S];
    uint32_t l_dt[S];
    float l_ew[S];
    const SinglesList SL{l_unit, l_e, l_dt, l_ew, 1};
    const unsigned long long n = min(*O.n_ovf, O.ovf_cap);
    Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
    int status = kStatusOk;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long base0 = (unsigned long long)blockIdx.x * blockDim.x;
    for (unsigned long long base = base0; base < n; base += stride) {
        const unsigned long long i = base + threadIdx.x;
        PState s;
        s.phase = kPhIdle;
        s.job = 0;
        if (i < n) {
            s.h = O.ovf_h[i];
            s.job = O.ovf_job[i];
            s.phase = kPhSource;
            const JobDev &J = W.jobs[s.job];
            const GeomDev &g = W.geoms[J.geom];
            while (s.phase != kPhFinish && s.phase != kPhIdle) {
                int st = kStatusOk;
                switch (s.phase) {
                    case kPhSource: ev_source(J, g, s, cnt); break;
                    case kPhPhantom: st = ev_phantom(J, g, W, s, cnt); break;
                    case kPhFlight: case kPhFlightOut: ev_flight(J, g, s, cnt); break;
                    case kPhPanel: st = ev_panel<false>(J, g, W, O, s, SL, S, cnt); break;
                    default: st = kStatusBadPhase; break;
                }
                if (st != kStatusOk) { status |= st; s.phase = kPhIdle; }
            }
            if (s.ovf) { status |= kStatusOverflow; s.phase = kPhIdle; }
        }
        __syncwarp();
        const bool fin = s.phase == kPhFinish;
        ev_finish(W.jobs, W.geoms, O, s, fin, SL, kFullMask, cnt);
    }
    // the singles of re-simulated histories are formed here (the rest was counted before)
    const uint32_t ns = __reduce_add_sync(kFullMask, cnt.singles);
    if ((threadIdx.x & 31) == 0 && ns) atomicAdd(O.counters + 9, (unsigned long long)ns);
    if (status) atomicOr(O.status, status);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static size_t loop_smem(int ng_smem, int block, int S) {
    return (size_t)ng_smem * sizeof(GeomDev) + (size_t)S * block * 16;
}

// dynamic shared memory and resident CTAs of the per-lane loop kernel
static cudaError_t loop_shape(int n_geoms, const LaunchCfg &cfg, size_t *smem, int *ctas, int *ng) {
    constexpr int S = 8;
    int occ = 0;
    cudaError_t e = staged_geometry(k_transport_loop<S>, cfg.block_size, loop_smem(0, cfg.block_size, S), n_geoms,
                                    cfg.max_smem_geoms, ng, smem, &occ);
    if (e != cudaSuccess) return e;
    // persistent grid: never more CTAs than can be resident at once
    *ctas = cfg.sm_count * max(1, min(occ, cfg.grid / max(cfg.sm_count, 1)));
    return cudaSuccess;
}

cudaError_t transport_resident_warps(int n_geoms, const LaunchCfg &cfg, long long *warps) {
    if (cfg.kernel == kKernelWave) return wave_resident_warps(n_geoms, cfg, warps);
    if (cfg.kernel == kKernelCta) return cta_resident_warps(n_geoms, cfg, warps);
    size_t smem = 0;
    int ctas = 0, ng = 0;
    cudaError_t e = loop_shape(n_geoms, cfg, &smem, &ctas, &ng);
    *warps = (long long)ctas * (cfg.block_size / 32);
    return e;
}

cudaError_t launch_transport_redo(const WorkDev &W, const OutDev &O, const LaunchCfg &cfg, cudaStream_t st) {
    k_transport_redo<<<cfg.sm_count, 128, 0, st>>>(W, O);
    return cudaGetLastError();
}

cudaError_t launch_transport(const WorkDev &W, const OutDev &O, const LaunchCfg &cfg, cudaStream_t st,
                             bool with_redo) {
    constexpr int S = 8;
    if (cfg.kernel == kKernelWave) {
        cudaError_t e = launch_transport_wave(W, O, cfg, st);
        if (e != cudaSuccess) return e;
    } else if (cfg.kernel == kKernelCta) {
        cudaError_t e = launch_transport_cta(W, O, cfg, st);
        if (e != cudaSuccess) return e;
    } else {
        size_t smem = 0;
        int ctas = 0, ng = 0;
        cudaError_t e = loop_shape(W.n_geoms, cfg, &smem, &ctas, &ng);
        if (e != cudaSuccess) return e;
        k_transport_loop<S><<<ctas, cfg.block_size, smem, st>>>(W, O, ng);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return with_redo ? launch_transport_redo(W, O, cfg, st) : cudaSuccess;
}

// Load the transport kernels and set their shared-memory limits (internal.h).
// The re-simulation kernel keeps its long singles list in local memory: the
// per-thread stack limit is raised to hold it now, since growing the device's
// local-memory reservation at a later launch waits for every running kernel.
cudaError_t preload_transport_kernels() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_transport_redo);
    size_t stack = 0;
    if (e == cudaSuccess) e = cudaDeviceGetLimit(&stack, cudaLimitStackSize);
    if (e == cudaSuccess && stack < fa.localSizeBytes) e = cudaDeviceSetLimit(cudaLimitStackSize, fa.localSizeBytes);
    if (e == cudaSuccess)
        e = ensure_dynamic_smem(reinterpret_cast<const void *>(k_transport_loop<8>),
                                loop_smem(kMaxStagedGeoms, 256, 8));
    if (e == cudaSuccess) e = preload_wave_kernels();
    if (e == cudaSuccess) e = preload_cta_kernels();
    return e;
}

}  // namespace gpet
