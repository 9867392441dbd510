// transport_cta.cu -- CTA-synchronous wavefront transport kernel.
//
// Same per-warp pools of history slots as the wavefront kernel, but the phase
// is chosen for the whole CTA: every iteration each warp posts the phase
// census of its pool to shared memory, one barrier later all warps read the
// CTA totals and agree on the most populated phase, and every warp of the CTA
// runs that same event.  All of a CTA's warps then execute one event's code
// at a time, which keeps the instruction cache warm (an SM holds one or two
// such CTAs); warps with no slot in the chosen phase wait for the next
// iteration.  The events are those of transport.cuh, so the results equal the
// other kernels' bit for bit.
#include "internal.h"
#include "transport.cuh"

namespace gpet {

namespace {

constexpr int kCtaS = 6;     // singles-list entries per history (overflow -> redo kernel)
constexpr int kCtaWords = 23;
constexpr int kNumPh = 7;    // phases 0..6

enum : int {
    kCh0 = 0, kCh1, kCt0, kCt1, kCx, kCy, kCz, kCdx, kCdy, kCdz, kCx0, kCy0, kCz0, kCox, kCoy, kCoz, kCE, kCpath,
    kCtrem, kCjob, kCpack, kCsteps
};

template <int SPL>
struct CtaPool {
    static constexpr int kPool = 32 * SPL;
    uint32_t st[kCtaWords][kPool];
    uint32_t sl_unit[kCtaS * kPool];
    float sl_e[kCtaS * kPool];
    uint32_t sl_dt[kCtaS * kPool];
    float sl_ew[kCtaS * kPool];
};

template <class Pool>
__device__ __forceinline__ uint32_t cphase(const Pool &P, int q) { return (P.st[kCpack][q] >> 16) & 7u; }

template <class Pool>
__device__ __forceinline__ void cload(const Pool &P, int q, PState &s) {
    s.h = ((uint64_t)P.st[kCh1][q] << 32) | P.st[kCh0][q];
    s.t0 = ((uint64_t)P.st[kCt1][q] << 32) | P.st[kCt0][q];
    s.x = __uint_as_float(P.st[kCx][q]);
    s.y = __uint_as_float(P.st[kCy][q]);
    s.z = __uint_as_float(P.st[kCz][q]);
    s.dx = __uint_as_float(P.st[kCdx][q]);
    s.dy = __uint_as_float(P.st[kCdy][q]);
    s.dz = __uint_as_float(P.st[kCdz][q]);
    s.x0 = __uint_as_float(P.st[kCx0][q]);
    s.y0 = __uint_as_float(P.st[kCy0][q]);
    s.z0 = __uint_as_float(P.st[kCz0][q]);
    s.ox = __uint_as_float(P.st[kCox][q]);
    s.oy = __uint_as_float(P.st[kCoy][q]);
    s.oz = __uint_as_float(P.st[kCoz][q]);
    s.E = __uint_as_float(P.st[kCE][q]);
    s.path = __uint_as_float(P.st[kCpath][q]);
    s.trem = __uint_as_float(P.st[kCtrem][q]);
    s.job = (int32_t)P.st[kCjob][q];
    const uint32_t pk = P.st[kCpack][q];
    s.panel = (int32_t)(pk & 0x7Fu) - 1;
    s.last = (int32_t)((pk >> 7) & 0x7Fu) - 1;
    s.gamma = (pk >> 14) & 1u;
    s.phase = (pk >> 16) & 7u;
    s.nsing = (pk >> 19) & 31u;
    s.ovf = (pk >> 24) & 1u;
    const uint32_t sw = P.st[kCsteps][q];
    s.sph = sw & 0xFFFFu;
    s.sdet = sw >> 16;
}

template <class Pool>
__device__ __forceinline__ void cstore(Pool &P, int q, const PState &s, bool all) {
    if (all) {
        P.st[kCh0][q] = (uint32_t)s.h;
        P.st[kCh1][q] = (uint32_t)(s.h >> 32);
        P.st[kCt0][q] = (uint32_t)s.t0;
        P.st[kCt1][q] = (uint32_t)(s.t0 >> 32);
        P.st[kCx0][q] = __float_as_uint(s.x0);
        P.st[kCy0][q] = __float_as_uint(s.y0);
        P.st[kCz0][q] = __float_as_uint(s.z0);
        P.st[kCox][q] = __float_as_uint(s.ox);
        P.st[kCoy][q] = __float_as_uint(s.oy);
        P.st[kCoz][q] = __float_as_uint(s.oz);
        P.st[kCjob][q] = (uint32_t)s.job;
    }
    P.st[kCx][q] = __float_as_uint(s.x);
    P.st[kCy][q] = __float_as_uint(s.y);
    P.st[kCz][q] = __float_as_uint(s.z);
    P.st[kCdx][q] = __float_as_uint(s.dx);
    P.st[kCdy][q] = __float_as_uint(s.dy);
    P.st[kCdz][q] = __float_as_uint(s.dz);
    P.st[kCE][q] = __float_as_uint(s.E);
    P.st[kCpath][q] = __float_as_uint(s.path);
    P.st[kCtrem][q] = __float_as_uint(s.trem);
    P.st[kCpack][q] = (uint32_t)(s.panel + 1) | ((uint32_t)(s.last + 1) << 7) | (s.gamma << 14) | (s.phase << 16) |
                      (s.nsing << 19) | (s.ovf << 24);
    P.st[kCsteps][q] = (s.sph & 0xFFFFu) | (s.sdet << 16);
}

// one event of phase p for a lane's history
__device__ __forceinline__ int run_event(int p, const JobDev &J, const GeomDev &g, const WorkDev &W, const OutDev &O,
                                         PState &s, const SinglesList &SL, Counters &cnt) {
    int st = kStatusOk;
    switch (p) {
        case kPhSource: ev_source(J, g, s, cnt); break;
        case kPhPhantom: st = ev_phantom(J, g, W, s, cnt); break;
        case kPhFlight: case kPhFlightOut:
            cnt.fl_out += p == kPhFlightOut ? 1u : 0u;
            ev_flight(J, g, s, cnt);
            break;
        case kPhPanel: st = ev_panel<true>(J, g, W, O, s, SL, kCtaS, cnt); break;
        default: st = kStatusBadPhase; break;
    }
    return st;
}

// Launch modes, one instantiation each, so that a fixed launch carries none
// of the other modes' instructions:
//   kModeFixed  : a fixed work table, one event per slot and phase choice;
//   kModeRepeat : the compaction interval -- a slot repeats its event up to
//                 `repeat` times while it stays in the chosen phase (steps of
//                 the phantom and of the detector repeat);
//   kModeLive   : a live launch (chunks the host appends while the kernel
//                 runs, bounded idle waits, per-job singles buffers).
enum : int { kModeFixed = 0, kModeRepeat = 1, kModeLive = 2 };

}  // namespace

// at most 128 registers a thread: 16 warps of the kernel stay resident per SM
template <int SPL, int WARPS, int MODE>
__global__ void __launch_bounds__(WARPS * 32, (16 / WARPS > 1 ? 16 / WARPS : 1)) k_transport_cta(WorkDev W, OutDev O, int ng_smem,
                                                                                                 int repeat) {
    constexpr bool kLive = MODE == kModeLive;
    using Pool = CtaPool<SPL>;
    constexpr int kPool = Pool::kPool;
    extern __shared__ __align__(16) uint8_t smem[];
    GeomDev *sgeom = reinterpret_cast<GeomDev *>(smem);
    Pool *pools = reinterpret_cast<Pool *>(sgeom + ng_smem);
    // CTA-wide phase totals, triple-buffered: iteration i adds into buffer
    // i % 3 before its barrier and reads it after; the buffer of iteration
    // i - 1 is cleared after the barrier of iteration i, which every read of
    // it precedes and every add of iteration i + 2 follows.
    __shared__ int census[3][8];
    __shared__ uint8_t assign[WARPS][32];  // slot of each lane in the chosen phase
    stage_geometry(W, sgeom, ng_smem);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    Pool &P = pools[wid];
#pragma unroll
    for (int g = 0; g < SPL; ++g) P.st[kCpack][g * 32 + lane] = 0;
    if (threadIdx.x < 24) (&census[0][0])[threadIdx.x] = 0;
    __syncthreads();

    Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
    Refill rf;
    refill_init(rf);
    int status = kStatusOk;
    LiveIdle idle;
    live_idle_reset(idle);
    unsigned long long iters = 0, lanes_used = 0;
    int buf = 0;
    // slots turn idle only in the finish event (or on an error); a warp whose
    // next chunk a live launch has not published yet retries every iteration
    bool may_idle = true;

    for (;;) {
        // 1. refill the warp's idle slots
#pragma unroll
        for (int g = 0; g < SPL; ++g) {
            if (!may_idle || rf.exhausted) break;
            const int q = g * 32 + lane;
            const uint32_t need = __ballot_sync(kFullMask, cphase(P, q) == kPhIdle);
            if (need) {
                bool got;
                uint64_t h = 0;
                int job = 0;
                warp_refill<kLive>(W, need, rf, got, h, job);
                if (got) {
                    P.st[kCh0][q] = (uint32_t)h;
                    P.st[kCh1][q] = (uint32_t)(h >> 32);
                    P.st[kCjob][q] = (uint32_t)job;
                    P.st[kCpack][q] = (uint32_t)kPhSource << 16;
                }
                if (kLive && rf.waiting) break;
            }
        }
        may_idle = kLive && rf.waiting && !rf.exhausted;
        __syncwarp();
        // 2. the warp's census: lane p adds the warp's count of phase p
        uint32_t ph[SPL];
#pragma unroll
        for (int g = 0; g < SPL; ++g) ph[g] = cphase(P, g * 32 + lane);
        uint32_t mask_p[kNumPh][SPL];
        int my_n = 0;
#pragma unroll
        for (int p = 1; p < kNumPh; ++p) {
            int n = 0;
#pragma unroll
            for (int g = 0; g < SPL; ++g) {
                mask_p[p][g] = __ballot_sync(kFullMask, ph[g] == (uint32_t)p);
                n += __popc(mask_p[p][g]);
            }
            if (lane == p) my_n = n;
        }
        if (my_n) atomicAdd(&census[buf][lane], my_n);
        int any_waiting = 0;
        if constexpr (kLive) any_waiting = __syncthreads_or(rf.waiting && !rf.exhausted);
        else __syncthreads();
        // 3. every warp reads the same totals: the most populated phase wins
        //    (ties to the later phase, which finishes histories sooner)
        const uint32_t key = (lane >= 1 && lane < kNumPh) ? ((uint32_t)census[buf][lane] << 3) | (uint32_t)lane : 0u;
        const uint32_t best = __reduce_max_sync(kFullMask, key);
        if (threadIdx.x < 8) census[buf == 0 ? 2 : buf - 1][threadIdx.x] = 0;
        buf = buf == 2 ? 0 : buf + 1;
        const int best_p = (int)(best & 7u);
        if ((best >> 3) == 0) {
            // every slot of every warp idle after refills: done, unless a warp
            // of a live launch waits for a chunk the host has not published yet
            if (!kLive || !any_waiting) break;
            // one decision for the whole CTA: its threads leave the loop together
            if (__syncthreads_or(live_idle_wait(idle, status, W, O))) {
                status |= kStatusLiveStall;
                break;
            }
            continue;
        }
        if (kLive) live_idle_reset(idle);
        // 4. lanes onto this warp's slots of the chosen phase: the slot of
        //    rank r (in slot order) goes to lane r
        int mine = 0;
#pragma unroll
        for (int g = 0; g < SPL; ++g) {
            uint32_t m = 0;
#pragma unroll
            for (int p = 1; p < kNumPh; ++p) m = p == best_p ? mask_p[p][g] : m;
            const int r = mine + __popc(m & lanemask_lt());
            if (ph[g] == (uint32_t)best_p && r < 32) assign[wid][r] = (uint8_t)(g * 32 + lane);
            mine += __popc(m);
        }
        __syncwarp();
        const bool active = lane < mine;
        const int q = active ? assign[wid][lane] : 0;
        if (mine == 0) continue;  // nothing of this phase here: wait for the next choice
        ++iters;
        lanes_used += (unsigned long long)min(mine, 32);
        PState s;
        s.phase = kPhIdle;
        s.job = 0;
        const SinglesList SL{P.sl_unit + q, P.sl_e + q, P.sl_dt + q, P.sl_ew + q, kPool};
        if (best_p == kPhFinish) {
            if (active) cload(P, q, s);
            __syncwarp();
            cnt.fin += active ? 1u : 0u;
            ev_finish<kLive>(W.jobs, W.geoms, O, s, active, SL, kFullMask, cnt);
            if (active) P.st[kCpack][q] = 0;
            may_idle = true;
            __syncwarp();
            continue;
        }
        int n_ev = 0;
        if (active) {
            cload(P, q, s);
            const JobDev &J = W.jobs[s.job];
            const GeomDev &g = J.geom < ng_smem ? sgeom[J.geom] : W.geoms[J.geom];
            int st = kStatusOk;
            if constexpr (MODE == kModeRepeat) {
                // the chosen event, then again while the slot stays in its
                // phase, up to `repeat` events in all
                do {
                    ++n_ev;
                    st = run_event(best_p, J, g, W, O, s, SL, cnt);
                } while (st == kStatusOk && n_ev < repeat && s.phase == (uint32_t)best_p);
            } else {
                st = run_event(best_p, J, g, W, O, s, SL, cnt);
            }
            if (st != kStatusOk) {
                status |= st;
                s.phase = kPhIdle;
            }
            cstore(P, q, s, best_p == kPhSource);
        }
        may_idle = may_idle || __any_sync(kFullMask, active && s.phase == kPhIdle);
        __syncwarp();
    }
    // totals, then the events per phase (slots 10 + phase: decay, phantom
    // step, flight, detector step, finish, flight after a panel exit)
    const uint32_t v[14] = {cnt.det_steps, cnt.flights, cnt.trials, cnt.entered, cnt.ph_steps, cnt.hits,
                            cnt.screened, cnt.singles, cnt.src, cnt.ph_steps, cnt.fl_ev - cnt.fl_out,
                            cnt.det_steps, cnt.fin, cnt.fl_out};
    const int slot[14] = {0, 1, 2, 3, 4, 5, 8, 9, 11, 12, 13, 14, 15, 16};
#pragma unroll
    for (int i = 0; i < 14; ++i) {
        const uint32_t x = __reduce_add_sync(kFullMask, v[i]);
        if (lane == 0 && x) atomicAdd(O.counters + slot[i], (unsigned long long)x);
    }
    if (lane == 0) {
        atomicAdd(O.counters + 6, iters);
        atomicAdd(O.counters + 7, lanes_used);
    }
    if (status) atomicOr(O.status, status);
}

// dynamic shared memory and resident CTAs of one shape (the same in every
// mode: the launch bounds cap each mode's registers alike)
template <int SPL, int WARPS>
static cudaError_t cta_shape(int n_geoms, const LaunchCfg &cfg, size_t *smem, int *ctas, int *ng) {
    int occ = 0;
    cudaError_t e = staged_geometry(k_transport_cta<SPL, WARPS, kModeFixed>, WARPS * 32, sizeof(CtaPool<SPL>) * WARPS,
                                    n_geoms, cfg.max_smem_geoms, ng, smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    *ctas = cfg.sm_count * occ;
    return cudaSuccess;
}

template <int SPL, int WARPS>
static cudaError_t launch_cta(const WorkDev &W, const OutDev &O, const LaunchCfg &cfg, cudaStream_t st) {
    size_t smem = 0;
    int ctas = 0, ng = 0;
    cudaError_t e = cta_shape<SPL, WARPS>(W.n_geoms, cfg, &smem, &ctas, &ng);
    if (e != cudaSuccess) return e;
    // a live launch runs one event per choice (its compaction interval is 1)
    const int repeat = max(1, cfg.compact_every);
    if (W.live_tail) k_transport_cta<SPL, WARPS, kModeLive><<<ctas, WARPS * 32, smem, st>>>(W, O, ng, 1);
    else if (repeat > 1) k_transport_cta<SPL, WARPS, kModeRepeat><<<ctas, WARPS * 32, smem, st>>>(W, O, ng, repeat);
    else k_transport_cta<SPL, WARPS, kModeFixed><<<ctas, WARPS * 32, smem, st>>>(W, O, ng, 1);
    return cudaGetLastError();
}

template <int SPL, int WARPS>
static cudaError_t warps_cta(int n_geoms, const LaunchCfg &cfg, long long *warps) {
    size_t smem = 0;
    int ctas = 0, ng = 0;
    cudaError_t e = cta_shape<SPL, WARPS>(n_geoms, cfg, &smem, &ctas, &ng);
    *warps = (long long)ctas * WARPS;
    return e;
}

// resident warps of the launch that launch_transport_cta makes
cudaError_t cta_resident_warps(int n_geoms, const LaunchCfg &cfg, long long *warps) {
    if (cfg.pool_depth == 3) {
        switch (cfg.block_size) {
            case 128: return warps_cta<3, 4>(n_geoms, cfg, warps);
            case 512: return warps_cta<3, 16>(n_geoms, cfg, warps);
            default: return warps_cta<3, 8>(n_geoms, cfg, warps);
        }
    }
    switch (cfg.block_size) {
        case 128: return warps_cta<2, 4>(n_geoms, cfg, warps);
        case 512: return warps_cta<2, 16>(n_geoms, cfg, warps);
        default: return warps_cta<2, 8>(n_geoms, cfg, warps);
    }
}

cudaError_t launch_transport_cta(const WorkDev &W, const OutDev &O, const LaunchCfg &cfg, cudaStream_t st) {
    // block_size selects the CTA width; pool_depth 3 deepens the per-warp pools
    if (cfg.pool_depth == 3) {
        switch (cfg.block_size) {
            case 128: return launch_cta<3, 4>(W, O, cfg, st);
            case 512: return launch_cta<3, 16>(W, O, cfg, st);
            default: return launch_cta<3, 8>(W, O, cfg, st);
        }
    }
    switch (cfg.block_size) {
        case 128: return launch_cta<2, 4>(W, O, cfg, st);
        case 512: return launch_cta<2, 16>(W, O, cfg, st);
        default: return launch_cta<2, 8>(W, O, cfg, st);
    }
}

template <int SPL, int WARPS>
static cudaError_t preload_cta() {
    const size_t bytes = sizeof(CtaPool<SPL>) * WARPS + (size_t)kMaxStagedGeoms * sizeof(GeomDev);
    cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void *>(k_transport_cta<SPL, WARPS, kModeFixed>), bytes);
    if (e == cudaSuccess)
        e = ensure_dynamic_smem(reinterpret_cast<const void *>(k_transport_cta<SPL, WARPS, kModeRepeat>), bytes);
    if (e == cudaSuccess)
        e = ensure_dynamic_smem(reinterpret_cast<const void *>(k_transport_cta<SPL, WARPS, kModeLive>), bytes);
    return e;
}

// load every instantiation and set its shared-memory limit (internal.h)
cudaError_t preload_cta_kernels() {
    cudaError_t e = preload_cta<2, 4>();
    if (e == cudaSuccess) e = preload_cta<2, 8>();
    if (e == cudaSuccess) e = preload_cta<2, 16>();
    if (e == cudaSuccess) e = preload_cta<3, 4>();
    if (e == cudaSuccess) e = preload_cta<3, 8>();
    if (e == cudaSuccess) e = preload_cta<3, 16>();
    return e;
}

}  // namespace gpet
