// transport_wave.cu -- wavefront transport kernel with warp-ballot regrouping.
//
// Each warp keeps a pool of 32 x depth history slots in shared memory (structure of
// arrays, one 32-bit word per field and slot).  Every iteration the warp
//   1. refills idle slots with new history ids from the chunked work queue,
//   2. ballots the phase of all slots (decay, phantom step, flight, panel
//      step, flight after a panel exit, finish) and picks the most populated,
//   3. maps its 32 lanes onto the slots in that phase (__fns over the ballot
//      masks), so every lane runs the same event code,
//   4. runs up to `compact_every` events of that phase per lane and stores
//      the state back; finished histories wait in their slot until the
//      finish phase (blur, window, append of their singles) is chosen.
// The events are the ones of the per-lane kernel (transport.cuh), so the two
// kernels produce the same histories bit for bit.
#include "internal.h"
#include "transport.cuh"

namespace gpet {

constexpr int kWaveWarps = 4;           // warps per CTA
constexpr int kWaveS = 6;               // singles-list entries per history (overflow -> redo kernel)
constexpr int kWords = 23;              // 32-bit words of state per slot

// shared-memory footprint of one warp's pool of 32 * SPL slots
template <int SPL>
struct WarpPool {
    static constexpr int kPool = 32 * SPL;
    uint32_t st[kWords][kPool];
    uint32_t sl_unit[kWaveS * kPool];
    float sl_e[kWaveS * kPool];
    uint32_t sl_dt[kWaveS * kPool];
    float sl_ew[kWaveS * kPool];
};

enum : int {
    kWh0 = 0, kWh1, kWt0, kWt1, kWx, kWy, kWz, kWdx, kWdy, kWdz, kWx0, kWy0, kWz0, kWox, kWoy, kWoz, kWE, kWpath,
    kWtrem, kWjob, kWpack, kWsteps
};

template <class Pool>
__device__ __forceinline__ uint32_t pool_phase(const Pool &P, int q) { return (P.st[kWpack][q] >> 16) & 7u; }

// packed word: [0:7) panel+1, [7:14) last+1, [14] gamma, [16:19) phase, [19:24) nsing, [24] ovf
template <class Pool>
__device__ __forceinline__ void pool_load(const Pool &P, int q, PState &s) {
    s.h = ((uint64_t)P.st[kWh1][q] << 32) | P.st[kWh0][q];
    s.t0 = ((uint64_t)P.st[kWt1][q] << 32) | P.st[kWt0][q];
    s.x = __uint_as_float(P.st[kWx][q]);
    s.y = __uint_as_float(P.st[kWy][q]);
    s.z = __uint_as_float(P.st[kWz][q]);
    s.dx = __uint_as_float(P.st[kWdx][q]);
    s.dy = __uint_as_float(P.st[kWdy][q]);
    s.dz = __uint_as_float(P.st[kWdz][q]);
    s.x0 = __uint_as_float(P.st[kWx0][q]);
    s.y0 = __uint_as_float(P.st[kWy0][q]);
    s.z0 = __uint_as_float(P.st[kWz0][q]);
    s.ox = __uint_as_float(P.st[kWox][q]);
    s.oy = __uint_as_float(P.st[kWoy][q]);
    s.oz = __uint_as_float(P.st[kWoz][q]);
    s.E = __uint_as_float(P.st[kWE][q]);
    s.path = __uint_as_float(P.st[kWpath][q]);
    s.trem = __uint_as_float(P.st[kWtrem][q]);
    s.job = (int32_t)P.st[kWjob][q];
    const uint32_t pk = P.st[kWpack][q];
    s.panel = (int32_t)(pk & 0x7Fu) - 1;
    s.last = (int32_t)((pk >> 7) & 0x7Fu) - 1;
    s.gamma = (pk >> 14) & 1u;
    s.phase = (pk >> 16) & 7u;
    s.nsing = (pk >> 19) & 31u;
    s.ovf = (pk >> 24) & 1u;
    const uint32_t sw = P.st[kWsteps][q];
    s.sph = sw & 0xFFFFu;
    s.sdet = sw >> 16;
}

// `all`: also the words only the decay event changes (history, decay time,
// job, decay point and direction); the other events leave them as loaded
template <class Pool>
__device__ __forceinline__ void pool_store(Pool &P, int q, const PState &s, bool all) {
    if (all) {
        P.st[kWh0][q] = (uint32_t)s.h;
        P.st[kWh1][q] = (uint32_t)(s.h >> 32);
        P.st[kWt0][q] = (uint32_t)s.t0;
        P.st[kWt1][q] = (uint32_t)(s.t0 >> 32);
        P.st[kWx0][q] = __float_as_uint(s.x0);
        P.st[kWy0][q] = __float_as_uint(s.y0);
        P.st[kWz0][q] = __float_as_uint(s.z0);
        P.st[kWox][q] = __float_as_uint(s.ox);
        P.st[kWoy][q] = __float_as_uint(s.oy);
        P.st[kWoz][q] = __float_as_uint(s.oz);
        P.st[kWjob][q] = (uint32_t)s.job;
    }
    P.st[kWx][q] = __float_as_uint(s.x);
    P.st[kWy][q] = __float_as_uint(s.y);
    P.st[kWz][q] = __float_as_uint(s.z);
    P.st[kWdx][q] = __float_as_uint(s.dx);
    P.st[kWdy][q] = __float_as_uint(s.dy);
    P.st[kWdz][q] = __float_as_uint(s.dz);
    P.st[kWE][q] = __float_as_uint(s.E);
    P.st[kWpath][q] = __float_as_uint(s.path);
    P.st[kWtrem][q] = __float_as_uint(s.trem);
    P.st[kWpack][q] = (uint32_t)(s.panel + 1) | ((uint32_t)(s.last + 1) << 7) | (s.gamma << 14) | (s.phase << 16) |
                      (s.nsing << 19) | (s.ovf << 24);
    P.st[kWsteps][q] = (s.sph & 0xFFFFu) | (s.sdet << 16);
}

template <int SPL>
__global__ void __launch_bounds__(kWaveWarps * 32) k_transport_wave(WorkDev W, OutDev O, int ng_smem, int repeat) {
    using Pool = WarpPool<SPL>;
    constexpr int kPool = Pool::kPool;
    extern __shared__ __align__(16) uint8_t smem[];
    GeomDev *sgeom = reinterpret_cast<GeomDev *>(smem);
    Pool *pools = reinterpret_cast<Pool *>(sgeom + ng_smem);
    stage_geometry(W, sgeom, ng_smem);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    Pool &P = pools[wid];
#pragma unroll
    for (int g = 0; g < SPL; ++g) P.st[kWpack][g * 32 + lane] = 0;  // every slot idle
    __syncthreads();

    Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
    Refill rf;
    refill_init(rf);
    int status = kStatusOk;
    LiveIdle idle;
    live_idle_reset(idle);
    unsigned long long iters = 0, lanes_used = 0;   // wavefront fill diagnostics

    for (;;) {
        // 1. refill idle slots, 32 at a time
#pragma unroll
        for (int g = 0; g < SPL; ++g) {
            const int q = g * 32 + lane;
            const uint32_t need = __ballot_sync(kFullMask, pool_phase(P, q) == kPhIdle);
            if (need && !rf.exhausted) {
                bool got;
                uint64_t h = 0;
                int job = 0;
                warp_refill(W, need, rf, got, h, job);
                if (got) {
                    P.st[kWh0][q] = (uint32_t)h;
                    P.st[kWh1][q] = (uint32_t)(h >> 32);
                    P.st[kWjob][q] = (uint32_t)job;
                    P.st[kWpack][q] = (uint32_t)kPhSource << 16;
                }
            }
        }
        __syncwarp();
        // 2. phase census over the pool
        uint32_t ph[SPL];
#pragma unroll
        for (int g = 0; g < SPL; ++g) ph[g] = pool_phase(P, g * 32 + lane);
        uint32_t best_b[SPL];
#pragma unroll
        for (int g = 0; g < SPL; ++g) best_b[g] = 0;
        int best_n = 0;
        uint32_t best_p = kPhIdle;
#pragma unroll
        for (uint32_t p = kPhSource; p <= kPhFlightOut; ++p) {
            uint32_t b[SPL];
            int n = 0;
#pragma unroll
            for (int g = 0; g < SPL; ++g) { b[g] = __ballot_sync(kFullMask, ph[g] == p); n += __popc(b[g]); }
            if (n > best_n) {
                best_n = n;
                best_p = p;
#pragma unroll
                for (int g = 0; g < SPL; ++g) best_b[g] = b[g];
            }
        }
        if (best_n == 0) {
            // every slot idle after a refill: the queue is exhausted, or a live
            // launch has nothing published yet
            if (!rf.waiting || __any_sync(kFullMask, live_idle_wait(idle, status, W, O))) break;
            continue;
        }
        live_idle_reset(idle);
        // 3. lane i takes the i-th slot of that phase
        const bool active = lane < best_n;
        int q = 0;
        if (active) {
            int rank = lane;
#pragma unroll
            for (int g = 0; g < SPL; ++g) {
                const int c = __popc(best_b[g]);
                if (rank >= 0 && rank < c) q = g * 32 + (int)__fns(best_b[g], 0, rank + 1);
                rank -= c;
            }
        }
        ++iters;
        lanes_used += (unsigned long long)min(best_n, 32);
        // 4. events
        PState s;
        s.phase = kPhIdle;
        s.job = 0;
        const SinglesList SL{P.sl_unit + q, P.sl_e + q, P.sl_dt + q, P.sl_ew + q, kPool};
        if (best_p == kPhFinish) {
            // finished histories as one wavefront: blur, window, append
            if (active) pool_load(P, q, s);
            __syncwarp();
            ev_finish(W.jobs, W.geoms, O, s, active, SL, kFullMask, cnt);
            if (active) P.st[kWpack][q] = 0;   // slot idle
            __syncwarp();
            continue;
        }
        if (active) {
            pool_load(P, q, s);
            const JobDev &J = W.jobs[s.job];
            const GeomDev &g = J.geom < ng_smem ? sgeom[J.geom] : W.geoms[J.geom];
            for (int r = 0; r < repeat && s.phase == best_p; ++r) {
                int st = kStatusOk;
                switch (best_p) {
                    case kPhSource: ev_source(J, g, s, cnt); break;
                    case kPhPhantom: st = ev_phantom(J, g, W, s, cnt); break;
                    case kPhFlight: case kPhFlightOut: ev_flight(J, g, s, cnt); break;
                    case kPhPanel: st = ev_panel<true>(J, g, W, O, s, SL, kWaveS, cnt); break;
                    default: st = kStatusBadPhase; break;
                }
                if (st != kStatusOk) {
                    status |= st;
                    s.phase = kPhIdle;
                }
            }
            pool_store(P, q, s, best_p == kPhSource);
        }
        __syncwarp();
    }
    // flush counters (all lanes converged here)
    const uint32_t v[8] = {cnt.det_steps, cnt.flights, cnt.trials, cnt.entered, cnt.ph_steps, cnt.hits,
                           cnt.screened, cnt.singles};
    const int slot[8] = {0, 1, 2, 3, 4, 5, 8, 9};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t x = __reduce_add_sync(kFullMask, v[i]);
        if (lane == 0 && x) atomicAdd(O.counters + slot[i], (unsigned long long)x);
    }
    if (lane == 0) {
        atomicAdd(O.counters + 6, iters);
        atomicAdd(O.counters + 7, lanes_used);
    }
    if (status) atomicOr(O.status, status);
}

template <int SPL>
static cudaError_t wave_shape(int n_geoms, const LaunchCfg &cfg, size_t *smem, int *ctas, int *ng) {
    int occ = 0;
    cudaError_t e = staged_geometry(k_transport_wave<SPL>, kWaveWarps * 32, sizeof(WarpPool<SPL>) * kWaveWarps,
                                    n_geoms, cfg.max_smem_geoms, ng, smem, &occ);
    if (e != cudaSuccess) return e;
    const int per_sm = max(1, cfg.grid >= cfg.sm_count && cfg.grid / cfg.sm_count < occ ? cfg.grid / cfg.sm_count : occ);
    *ctas = cfg.sm_count * per_sm;
    return cudaSuccess;
}

template <int SPL>
static cudaError_t launch_wave_spl(const WorkDev &W, const OutDev &O, const LaunchCfg &cfg, cudaStream_t st) {
    size_t smem = 0;
    int ctas = 0, ng = 0;
    cudaError_t e = wave_shape<SPL>(W.n_geoms, cfg, &smem, &ctas, &ng);
    if (e != cudaSuccess) return e;
    k_transport_wave<SPL><<<ctas, kWaveWarps * 32, smem, st>>>(W, O, ng,
                                                              max(1, cfg.compact_every));
    return cudaGetLastError();
}

cudaError_t launch_transport_wave(const WorkDev &W, const OutDev &O, const LaunchCfg &cfg, cudaStream_t st) {
    switch (cfg.pool_depth) {
        case 3: return launch_wave_spl<3>(W, O, cfg, st);
        case 4: return launch_wave_spl<4>(W, O, cfg, st);
        default: return launch_wave_spl<2>(W, O, cfg, st);
    }
}

// resident warps of the launch that launch_transport_wave makes
cudaError_t wave_resident_warps(int n_geoms, const LaunchCfg &cfg, long long *warps) {
    size_t smem = 0;
    int ctas = 0, ng = 0;
    cudaError_t e;
    switch (cfg.pool_depth) {
        case 3: e = wave_shape<3>(n_geoms, cfg, &smem, &ctas, &ng); break;
        case 4: e = wave_shape<4>(n_geoms, cfg, &smem, &ctas, &ng); break;
        default: e = wave_shape<2>(n_geoms, cfg, &smem, &ctas, &ng); break;
    }
    *warps = (long long)ctas * kWaveWarps;
    return e;
}

template <int SPL>
static cudaError_t preload_wave() {
    return ensure_dynamic_smem(reinterpret_cast<const void *>(k_transport_wave<SPL>),
                               sizeof(WarpPool<SPL>) * kWaveWarps + (size_t)kMaxStagedGeoms * sizeof(GeomDev));
}

// load every instantiation and set its shared-memory limit (internal.h)
cudaError_t preload_wave_kernels() {
    cudaError_t e = preload_wave<2>();
    if (e == cudaSuccess) e = preload_wave<3>();
    if (e == cudaSuccess) e = preload_wave<4>();
    return e;
}

}  // namespace gpet
