// transport.cuh -- per-history photon-pair transport as a set of events that
// advance one history by one step.  Every transport kernel (the per-lane event
// loop, the per-warp wavefront, the CTA-synchronous wavefront and the overflow
// re-simulation) runs these same events, so they produce identical histories.
//
// Paper anchors (arxiv 2603.07327): Sec. 2.1 (flight by line-plane
// intersection, panel-local frame, Woodcock stepping until the photon leaves
// the panel or drops below the cutoff, layer selection, crystal / layer /
// module / panel labels, singles readout level), Sec. 2.3 (back-to-back pairs,
// no positron range, energy blur and window), abstract (transport across
// layers and panels).
#pragma once

#include "device.cuh"

namespace gpet {

// history phases.  A flight after a panel exit has its own phase: it starts
// in the annulus of the panels, not inside the ring, and takes the other
// branch of the flight code, so a wavefront of one kind does not diverge.
enum : uint32_t { kPhIdle = 0, kPhSource = 1, kPhPhantom = 2, kPhFlight = 3, kPhPanel = 4, kPhFinish = 5,
                  kPhFlightOut = 6 };

// per-history singles list: unit ids, energy sums, earliest time offset
// (t - t0 in ps); `stride` separates consecutive entries of one history
struct SinglesList {
    uint32_t *unit;
    float *e;
    uint32_t *dt;
    float *ew;      // sum of energy x depth (for the single's depth of interaction)
    int stride;
};

// outputs shared by all jobs of a launch
struct OutDev {
    // kept singles (SoA); count in *n_singles (may exceed cap -> overflow, host re-runs)
    RawSingle *s_raw;
    unsigned long long *n_singles;
    unsigned long long s_cap;
    // each kept single's 64-bit time-sort key, at its record's slot: (job <<
    // key_shift) | t_ps, the time alone when key_shift is 64 (the digitizer's
    // sort starts from these keys instead of reading the records)
    uint64_t *s_keys;
    int key_shift;
    // optional crystal interactions
    uint64_t *hit_h, *hit_t;
    int32_t *hit_gstep, *hit_crystal, *hit_layer, *hit_job;
    float *hit_wuv, *hit_e;
    unsigned long long *n_hits;   // slots taken when storing hits
    unsigned long long hit_cap;   // 0 = do not store
    // histories whose singles list overflowed: re-simulated by the fallback kernel
    uint64_t *ovf_h;
    int32_t *ovf_job;
    unsigned long long *n_ovf;
    unsigned long long ovf_cap;
    // event counters: det_steps, flights, compton_trials, entered, phantom_steps, hits
    unsigned long long *counters;
    int *status;
};

struct WorkDev {
    const JobDev *jobs;
    int n_jobs;
    const GeomDev *geoms;                   // deduplicated geometry table
    int n_geoms;
    const unsigned long long *chunk_start;  // n_jobs + 1 prefix sums of chunks per job
    unsigned long long total_chunks;
    unsigned long long *next_chunk;        // global work counter
    unsigned int chunk_size;
    const float *gtab;                      // Compton ratio table, kXsIntervals + 1 nodes
    float ln_emin, inv_h;
    // A live launch (the serving loop's) takes jobs that the host appends while
    // the kernel runs.  The host writes, with the copy engine and in this order,
    // the new jobs, their geometry and chunk_start entries, then *live_tail
    // (chunks published so far); *live_closed = 1 once it appends no more, after
    // the last tail.  chunk_start then spans n_jobs = the table's capacity, its
    // unpublished entries ~0.  NULL live_tail: a fixed launch of total_chunks.
    const unsigned long long *live_tail;
    const int *live_closed;
    unsigned long long *live_taken;         // chunks claimed so far (a progress hint for the host)
};

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

constexpr unsigned long long kNoChunk = ~0ull;
// idle waits of a live launch: sleeps that double up to 16 us, for at most
// this long in a row by the GPU's global timer before the kernel gives up with
// kStatusLiveStall (a sleep's length is only approximate, the timer is not)
constexpr unsigned long long kLiveIdleNs = 10ull * 1000 * 1000 * 1000;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Where a warp takes its next histories from: the current chunk [next, end) of
// job `job`, whose chunks are [jc0, jend) and histories h_base + [0, nh); a
// chunk index claimed while a live launch had not yet published it (pend,
// lane 0 only); and whether the queue is exhausted.
struct Refill {
    uint64_t next, end;
    unsigned long long pend;
    unsigned long long jc0, jend;
    uint64_t base, nh;
    int job;
    bool exhausted, waiting;
};

__device__ __forceinline__ void refill_init(Refill &r) {
    r.next = r.end = 0;
    r.pend = kNoChunk;
    r.jc0 = r.jend = 0;
    r.base = r.nh = 0;
    r.job = 0;
    r.exhausted = r.waiting = false;
}

// Claim of the next chunk by a warp (lanes converged).  Lane 0 takes the next
// index of the work counter, or re-checks the one it took before while that
// chunk was not yet published.  Returns 1 (chunk c ready), 0 (a live launch
// has not published it yet) or -1 (no more work).  kLive = false: the caller
// runs fixed launches only (live_tail is NULL), and the live branch is left out.
template <bool kLive>
__device__ __forceinline__ int claim_chunk(const WorkDev &W, unsigned long long &pend, unsigned long long &c) {
    int r = 0;
    unsigned long long cc = 0;
    if ((threadIdx.x & 31) == 0) {
        if (pend == kNoChunk) pend = atomicAdd(W.next_chunk, 1ull);
        cc = pend;
        if (!kLive || !W.live_tail) {
            r = cc < W.total_chunks ? 1 : -1;
        } else {
            // closed first: once it reads 1, the tail read after it is final
            const int closed = *reinterpret_cast<const volatile int *>(W.live_closed);
            __threadfence();
            const unsigned long long tail = *reinterpret_cast<const volatile unsigned long long *>(W.live_tail);
            r = cc < tail ? 1 : (closed ? -1 : 0);
            if (r == 1) atomicMax(W.live_taken, cc + 1);
        }
        if (r != 0) pend = kNoChunk;
    }
    r = __shfl_sync(kFullMask, r, 0);
    c = __shfl_sync(kFullMask, cc, 0);
    if (kLive && r == 1 && W.live_tail) __threadfence();  // the chunk's table entries were written before its tail
    return r;
}

// a work-table entry: through L2 where a live launch may append to the table,
// else through the read-only cache
template <bool kLive, class T>
__device__ __forceinline__ T table_load(const T *p) {
    return kLive ? __ldcg(p) : __ldg(p);
}

// Warp-wide refill: lanes in `need` receive consecutive history ids from the
// warp's current chunk, fetching new chunks (one atomic each) as needed.
// kLive: table reads go to L2 (ld.cg), since a live launch appends to these
// tables.
template <bool kLive = true>
__device__ __forceinline__ void warp_refill(const WorkDev &W, uint32_t need, Refill &R, bool &got, uint64_t &h,
                                            int &job) {
    const int lane = threadIdx.x & 31;
    got = false;
    R.waiting = false;
    while (need && !R.exhausted) {
        const uint64_t avail = R.end - R.next;
        if (avail == 0) {
            unsigned long long c = 0;
            const int cl = claim_chunk<kLive>(W, R.pend, c);
            if (cl < 0) {
                R.exhausted = true;
                break;
            }
            if (cl == 0) {
                R.waiting = true;  // try again at the next refill
                break;
            }
            if (!kLive || c >= R.jend) {
                // The job: the last chunk_start entry <= c.  A live launch's
                // warp searches from its current job (its claims increase, so
                // chunk_start[job] <= c), galloping forward, then bisects; a
                // fixed launch bisects the whole table (cached in L1; measured
                // faster there).
                int lo = kLive ? R.job : 0, hi = W.n_jobs - 1, step = 1;
                while (kLive && lo < hi) {
                    const int probe = min(lo + step, hi);
                    if (table_load<kLive>(W.chunk_start + probe) <= c) {
                        lo = probe;
                        step <<= 1;
                    } else {
                        hi = probe - 1;
                        break;
                    }
                }
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (table_load<kLive>(W.chunk_start + mid) <= c) lo = mid; else hi = mid - 1;
                }
                // a published job's entries are final (its end is written with it)
                R.job = lo;
                R.jc0 = table_load<kLive>(W.chunk_start + lo);
                R.jend = table_load<kLive>(W.chunk_start + lo + 1);
                R.base = table_load<kLive>(reinterpret_cast<const unsigned long long *>(&W.jobs[lo].h_base));
                R.nh = table_load<kLive>(reinterpret_cast<const unsigned long long *>(&W.jobs[lo].n_hist));
            }
            const uint64_t h0 = (uint64_t)(c - R.jc0) * W.chunk_size;
            R.next = R.base + h0;
            R.end = R.base + min(h0 + (uint64_t)W.chunk_size, R.nh);
            continue;
        }
        const uint32_t cnt = (uint32_t)__popc(need);
        const uint32_t take = avail < cnt ? (uint32_t)avail : cnt;
        const uint32_t rank = (uint32_t)__popc(need & lanemask_lt());
        if (((need >> lane) & 1u) && rank < take) {
            got = true;
            h = R.next + rank;
            job = R.job;
        }
        R.next += take;
        need &= ~__ballot_sync(kFullMask, ((need >> lane) & 1u) && rank < take);  // drop the served lanes
    }
}

// Idle state of a live launch's warp or CTA: when its idle stretch began (by
// the global timer, 0 = not idle) and how many sleeps it took.
struct LiveIdle {
    unsigned long long t0;
    uint32_t polls;
};

__device__ __forceinline__ void live_idle_reset(LiveIdle &w) {
    w.t0 = 0;
    w.polls = 0;
}

// One idle wait of a live launch whose slots are all idle while work may still
// be published: sleeps (doubling up to 16 us) and returns false, or, once the
// idle stretch has lasted kLiveIdleNs, records it (counters 17..19: the
// stretch in ns, the published chunk count and the closed flag it last saw),
// sets kStatusLiveStall and returns true.
__device__ __forceinline__ bool live_idle_wait(LiveIdle &w, int &status, const WorkDev &W, const OutDev &O) {
    const unsigned long long now = global_ns();
    if (w.t0 == 0) w.t0 = now;
    if (now - w.t0 > kLiveIdleNs) {
        status |= kStatusLiveStall;
        if ((threadIdx.x & 31) == 0) {
            atomicMax(O.counters + 17, now - w.t0);
            atomicMax(O.counters + 18, *reinterpret_cast<const volatile unsigned long long *>(W.live_tail));
            atomicMax(O.counters + 19, (unsigned long long)*reinterpret_cast<const volatile int *>(W.live_closed));
        }
        return true;
    }
    ++w.polls;
    __nanosleep(w.polls < 14u ? (1u << w.polls) : 16384u);
    return false;
}

// copy the first ng geometry descriptors into shared memory
__device__ __forceinline__ void stage_geometry(const WorkDev &W, GeomDev *sg, int ng) {
    constexpr int words = (int)(sizeof(GeomDev) / 4);
    const uint32_t *src = reinterpret_cast<const uint32_t *>(W.geoms);
    uint32_t *dst = reinterpret_cast<uint32_t *>(sg);
    for (int i = threadIdx.x; i < ng * words; i += blockDim.x) dst[i] = src[i];
}

struct PState {
    uint64_t h, t0;
    float x, y, z, dx, dy, dz;      // global frame, or panel frame (w, u, v) when panel >= 0
    float x0, y0, z0, ox, oy, oz;   // decay point and photon-0 direction
    float E, path, trem;
    int32_t job, panel, last;
    uint32_t sph, sdet, gamma, phase, nsing, ovf;
};

struct Counters {
    uint32_t det_steps, flights, trials, entered, ph_steps, hits, screened, singles;
    // events per phase beyond ph_steps and det_steps (the CTA kernel reports
    // them): decays, flight events (flights less the photon starts that the
    // axial screen ends), flights after a panel exit, finish events
    uint32_t src, fl_ev, fl_out, fin;
};

__device__ __forceinline__ void to_global(const GeomDev &g, PState &s) {
    if (g.posed) {
        const float4 aw = __ldg(g.pose + 4 * s.panel), au = __ldg(g.pose + 4 * s.panel + 1);
        const float4 av = __ldg(g.pose + 4 * s.panel + 2), o = __ldg(g.pose + 4 * s.panel + 3);
        const float w = s.x, u = s.y, v = s.z, dw = s.dx, du = s.dy, dv = s.dz;
        s.x = fmaf(w, aw.x, fmaf(u, au.x, fmaf(v, av.x, o.x)));
        s.y = fmaf(w, aw.y, fmaf(u, au.y, fmaf(v, av.y, o.y)));
        s.z = fmaf(w, aw.z, fmaf(u, au.z, fmaf(v, av.z, o.z)));
        s.dx = fmaf(dw, aw.x, fmaf(du, au.x, dv * av.x));
        s.dy = fmaf(dw, aw.y, fmaf(du, au.y, dv * av.y));
        s.dz = fmaf(dw, aw.z, fmaf(du, au.z, dv * av.z));
        return;
    }
    const float c = g.pc[s.panel], sn = g.ps[s.panel];
    const float rw = g.R + s.x;
    const float gx = rw * c - s.y * sn, gy = rw * sn + s.y * c;
    const float gdx = s.dx * c - s.dy * sn, gdy = s.dx * sn + s.dy * c;
    s.x = gx; s.y = gy;
    s.dx = gdx; s.dy = gdy;
}

__device__ __forceinline__ bool in_phantom(const JobDev &J, float x, float y, float z) {
    return x >= J.ph_origin[0] && x < J.ph_hi[0] && y >= J.ph_origin[1] && y < J.ph_hi[1] && z >= J.ph_origin[2] &&
           z < J.ph_hi[2];
}

// Start photon s.gamma of the pair at the decay point.  A photon whose first
// flight would be screened at once (flight() applies the same test first) is
// finished here as a screened flight, without a flight event: photon 0 hands
// over to photon 1, photon 1 ends the history.
__device__ __forceinline__ void start_photon(const JobDev &J, const GeomDev &g, PState &s, Counters &cnt) {
    for (;;) {
        const float sg = s.gamma == 0 ? 1.0f : -1.0f;
        s.x = s.x0; s.y = s.y0; s.z = s.z0;
        s.dx = sg * s.ox; s.dy = sg * s.oy; s.dz = sg * s.oz;
        s.E = kE0;
        s.path = 0.0f;
        s.sph = 0; s.sdet = 0;
        s.panel = -1; s.last = -1;
        s.phase = (J.has_phantom && in_phantom(J, s.x, s.y, s.z)) ? kPhPhantom : kPhFlight;
        if (s.phase != kPhFlight || !start_screened(g, s.x, s.y, s.z, s.dx, s.dy, s.dz)) return;
        cnt.flights++;
        cnt.screened++;
        if (s.gamma == 0) {
            s.gamma = 1;
            continue;
        }
        s.phase = (s.nsing == 0 && !s.ovf) ? kPhIdle : kPhFinish;
        return;
    }
}

__device__ __forceinline__ void photon_done(const JobDev &J, const GeomDev &g, PState &s, Counters &cnt) {
    if (s.gamma == 0) {
        s.gamma = 1;
        start_photon(J, g, s, cnt);
    } else {
        // a history without singles has nothing to digitize: its slot is free
        s.phase = (s.nsing == 0 && !s.ovf) ? kPhIdle : kPhFinish;
    }
}

// Smallest voxel with cdf > target.  A guide table (Chen & Asau) narrows the
// search: guide[k] is the first voxel whose prefix sum falls in bucket k or
// later, the bucket of a value x being floor(x * gscale) computed exactly as
// when the table was built, so the answer lies in [guide[b], guide[b + 1]].
__device__ __forceinline__ int64_t pick_voxel(const JobDev &J, double target) {
    if (target >= J.ph_total) return J.ph_last_active;
    int64_t lo = 0, hi = J.ph_n - 1;
    if (J.ph_guide) {
        const int b = min((int)(target * J.ph_gscale), J.ph_buckets - 1);
        lo = __ldg(J.ph_guide + b);
        if (b + 1 < J.ph_buckets) hi = min(hi, (int64_t)__ldg(J.ph_guide + b + 1));
    }
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(J.ph_cdf + mid) > target) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// decay of history h (Sec. 2.3): time, annihilation point, photon-0 direction
__device__ __forceinline__ void ev_source(const JobDev &J, const GeomDev &g, PState &s, Counters &cnt) {
    cnt.src++;
    const uint4 r = draw(J.seed, s.h, kTagSource, 0u, 0u, 0u);
    const uint64_t r64 = ((uint64_t)r.x << 32) | r.y;
    s.t0 = __umul64hi(J.t_span_ps, r64);
    if (J.src_kind == 1) {
        const uint4 q = draw(J.seed, s.h, kTagSource, 0u, 0u, 1u);
        const uint4 zq = draw(J.seed, s.h, kTagSource, 0u, 0u, 2u);
        const uint64_t r53 = ((uint64_t)q.x << 21) | (q.y >> 11);
        const double target = (double)r53 * 0x1p-53 * J.ph_total;
        const int64_t vi = pick_voxel(J, target);
        int64_t ix, iy, iz;
        if (J.ph_n <= 0x7FFFFFFFll) {   // 32-bit index arithmetic: a 64-bit division is ~5x dearer
            const uint32_t v = (uint32_t)vi, nx = (uint32_t)J.ph_nx, nxy = nx * (uint32_t)J.ph_ny;
            const uint32_t vz = v / nxy, r = v - vz * nxy, vy = r / nx;
            ix = r - vy * nx; iy = vy; iz = vz;
        } else {
            ix = vi % J.ph_nx; iy = (vi / J.ph_nx) % J.ph_ny; iz = vi / ((int64_t)J.ph_nx * J.ph_ny);
        }
        s.x0 = fmaf((float)ix + u01(q.z), J.ph_voxel[0], J.ph_origin[0]);
        s.y0 = fmaf((float)iy + u01(q.w), J.ph_voxel[1], J.ph_origin[1]);
        s.z0 = fmaf((float)iz + u01(zq.x), J.ph_voxel[2], J.ph_origin[2]);
    } else {
        s.x0 = J.src_pos[0]; s.y0 = J.src_pos[1]; s.z0 = J.src_pos[2];
    }
    if (J.src_kind == 2) {
        s.ox = J.src_dir[0]; s.oy = J.src_dir[1]; s.oz = J.src_dir[2];
    } else {
        const float ct = 2.0f * u01(r.z) - 1.0f;
        const float st = sqrtf((1.0f - ct) * (1.0f + ct));
        float sp, cp;
        sincospif(2.0f * u01(r.w), &sp, &cp);
        s.ox = st * cp; s.oy = st * sp; s.oz = ct;
    }
    s.gamma = 0;
    s.nsing = 0;
    s.ovf = 0;
    start_photon(J, g, s, cnt);
}

// one Woodcock step in the voxel phantom
__device__ __forceinline__ int ev_phantom(const JobDev &J, const GeomDev &g, const WorkDev &W, PState &s,
                                          Counters &cnt) {
    if (s.sph >= (uint32_t)kMaxSteps) return kStatusTimeout;
    const uint4 r = draw(J.seed, s.h, kTagPhantom, s.gamma, s.sph, 0u);
    const uint32_t step_id = s.sph++;
    cnt.ph_steps++;
    // distance to the grid box exit
    float t_out = 3.0e38f;
    if (s.dx > 0.f) t_out = fminf(t_out, (J.ph_hi[0] - s.x) / s.dx); else if (s.dx < 0.f) t_out = fminf(t_out, (J.ph_origin[0] - s.x) / s.dx);
    if (s.dy > 0.f) t_out = fminf(t_out, (J.ph_hi[1] - s.y) / s.dy); else if (s.dy < 0.f) t_out = fminf(t_out, (J.ph_origin[1] - s.y) / s.dy);
    if (s.dz > 0.f) t_out = fminf(t_out, (J.ph_hi[2] - s.z) / s.dz); else if (s.dz < 0.f) t_out = fminf(t_out, (J.ph_origin[2] - s.z) / s.dz);
    t_out = fmaxf(t_out, 0.0f);
    const Xs xs = xs_at(s.E, W.gtab, W.ln_emin, W.inv_h);
    float mu_maj = 0.0f;
    for (int m = 0; m < J.ph_nmat; ++m) mu_maj = fmaxf(mu_maj, mu_total(J.ph_mu_c511[m], J.ph_mu_pe511[m], xs));
    // free path -ln(u) / mu: the fast log's absolute error (< 4e-7) moves a
    // step by < 5e-5 mm even in water, far below the position tolerance
    const float step = mu_maj > 0.0f ? -__logf(u01(r.x)) * (10.0f / mu_maj) : 3.0e38f;
    if (step >= t_out) {
        s.x = fmaf(t_out, s.dx, s.x); s.y = fmaf(t_out, s.dy, s.y); s.z = fmaf(t_out, s.dz, s.z);
        s.path += t_out;
        s.phase = kPhFlight;
        return kStatusOk;
    }
    s.x = fmaf(step, s.dx, s.x); s.y = fmaf(step, s.dy, s.y); s.z = fmaf(step, s.dz, s.z);
    s.path += step;
    int ix = (int)floorf((s.x - J.ph_origin[0]) * J.ph_inv_voxel[0]);
    int iy = (int)floorf((s.y - J.ph_origin[1]) * J.ph_inv_voxel[1]);
    int iz = (int)floorf((s.z - J.ph_origin[2]) * J.ph_inv_voxel[2]);
    ix = min(max(ix, 0), J.ph_nx - 1); iy = min(max(iy, 0), J.ph_ny - 1); iz = min(max(iz, 0), J.ph_nz - 1);
    const int m = __ldg(J.ph_mat + ((int64_t)iz * J.ph_ny + iy) * J.ph_nx + ix);
    const float pe = J.ph_mu_pe511[m] * xs.r3;
    const float mu_m = fmaf(J.ph_mu_c511[m], xs.g, pe);
    if (u01(r.y) * mu_maj >= mu_m) return kStatusOk;          // virtual
    if (u01(r.z) * mu_m < pe) { photon_done(J, g, s, cnt); return kStatusOk; }   // photoelectric
    float xm1;                                                   // Compton (Klein-Nishina)
    const int nt = kahn_sample(J.seed, s.h, kTagPhantom, s.gamma, step_id, s.E, xm1);
    if (nt < 0) return kStatusTimeout;
    cnt.trials += (uint32_t)nt;
    const float omc = xm1 / (s.E * kInvMec2);
    rotate_dir(s.dx, s.dy, s.dz, omc, u01(r.w));
    const float Ep = s.E / (1.0f + xm1);
    if (Ep < J.e_cut) { photon_done(J, g, s, cnt); return kStatusOk; }
    s.E = Ep;
    return kStatusOk;
}

// flight to the next panel by line-plane intersection
__device__ __forceinline__ void ev_flight(const JobDev &J, const GeomDev &g, PState &s, Counters &cnt) {
    cnt.flights++;
    cnt.fl_ev++;
    float t_in, t_out;
    const int k = flight(g, s.x, s.y, s.z, s.dx, s.dy, s.dz, s.last, t_in, t_out);
    if (k < 0) {
        if (k == kFlightScreened) cnt.screened++;
        photon_done(J, g, s, cnt);
        return;
    }
    cnt.entered++;
    // entry point, then the panel-local frame (w, u, v)
    const float ex = fmaf(t_in, s.dx, s.x), ey = fmaf(t_in, s.dy, s.y), ez = fmaf(t_in, s.dz, s.z);
    s.path += t_in;
    if (g.posed) {
        const float4 aw = __ldg(g.pose + 4 * k), au = __ldg(g.pose + 4 * k + 1), av = __ldg(g.pose + 4 * k + 2);
        const float dw = fmaf(s.dx, aw.x, fmaf(s.dy, aw.y, s.dz * aw.z));
        const float du = fmaf(s.dx, au.x, fmaf(s.dy, au.y, s.dz * au.z));
        const float dv = fmaf(s.dx, av.x, fmaf(s.dy, av.y, s.dz * av.z));
        s.x = fmaf(ex, aw.x, fmaf(ey, aw.y, fmaf(ez, aw.z, -aw.w)));
        s.y = fmaf(ex, au.x, fmaf(ey, au.y, fmaf(ez, au.z, -au.w)));
        s.z = fmaf(ex, av.x, fmaf(ey, av.y, fmaf(ez, av.z, -av.w)));
        s.dx = dw; s.dy = du; s.dz = dv;
    } else {
        const float c = g.pc[k], sn = g.ps[k];
        const float w = fmaf(ex, c, ey * sn) - g.R;
        const float u = fmaf(-ex, sn, ey * c);
        const float dw = fmaf(s.dx, c, s.dy * sn), du = fmaf(-s.dx, sn, s.dy * c);
        s.x = w; s.y = u; s.z = ez;
        s.dx = dw; s.dy = du;
    }
    s.trem = t_out - t_in;
    s.panel = k;
    s.phase = kPhPanel;
}

// record energy `dep` deposited in crystal L.crystal into the history's singles list
__device__ __forceinline__ void add_single(const GeomDev &g, PState &s, const SinglesList &SL, int max_entries,
                                           int crystal, int module, float dep, uint32_t dtp, float w) {
    uint32_t unit;
    if (g.readout_level == 0) unit = (uint32_t)s.panel;
    else if (g.readout_level == 1) unit = (uint32_t)(s.panel * g.modules_u * g.modules_v + module);
    else unit = (uint32_t)crystal;
    for (uint32_t j = 0; j < s.nsing; ++j) {
        if (SL.unit[j * SL.stride] == unit) {
            SL.e[j * SL.stride] += dep;
            SL.ew[j * SL.stride] += dep * w;
            SL.dt[j * SL.stride] = min(SL.dt[j * SL.stride], dtp);
            return;
        }
    }
    if ((int)s.nsing < max_entries) {
        SL.unit[s.nsing * SL.stride] = unit;
        SL.e[s.nsing * SL.stride] = dep;
        SL.ew[s.nsing * SL.stride] = dep * w;
        SL.dt[s.nsing * SL.stride] = dtp;
        s.nsing++;
    } else {
        s.ovf = 1;
    }
}

// a crystal interaction: tallies, optional hit list, singles list of the history
template <bool kTallies>
__device__ __forceinline__ void record_hit(const JobDev &J, const GeomDev &g, const OutDev &O, PState &s,
                                           const SinglesList &SL, int max_entries, Counters &cnt, int crystal,
                                           int module, int layer, uint32_t step_id, float dep) {
    cnt.hits++;
    const uint32_t dtp = (uint32_t)floorf(s.path * kInvCmmPerPs);
    if (kTallies) {
        atomicAdd(J.tally_count + crystal, 1ull);
        atomicAdd(J.tally_efx + crystal, (unsigned long long)__float2ull_rn(dep * kEfxScale));
        if (O.hit_cap) {
            const unsigned long long slot = atomicAdd(O.n_hits, 1ull);
            if (slot < O.hit_cap) {
                O.hit_h[slot] = s.h;
                O.hit_t[slot] = s.t0 + dtp;
                O.hit_gstep[slot] = (int32_t)((s.gamma << 24) | step_id);
                O.hit_crystal[slot] = crystal;
                O.hit_layer[slot] = layer;
                O.hit_job[slot] = s.job;
                O.hit_wuv[3 * slot] = s.x;
                O.hit_wuv[3 * slot + 1] = s.y;
                O.hit_wuv[3 * slot + 2] = s.z;
                O.hit_e[slot] = dep;
            }
        }
    }
    add_single(g, s, SL, max_entries, crystal, module, dep, dtp, s.x);
}

// one Woodcock step inside the current panel (layer selection, interaction, hit)
template <bool kTallies>
__device__ __forceinline__ int ev_panel(const JobDev &J, const GeomDev &g, const WorkDev &W, const OutDev &O,
                                        PState &s, const SinglesList &SL, int max_entries, Counters &cnt) {
    if (s.sdet >= (uint32_t)kMaxSteps) return kStatusTimeout;
    const uint4 r = draw(J.seed, s.h, kTagDetector, s.gamma, s.sdet, 0u);
    const uint32_t step_id = s.sdet++;
    cnt.det_steps++;
    const Xs xs = xs_at(s.E, W.gtab, W.ln_emin, W.inv_h);
    float mu_maj = 0.0f;
    for (int m = 0; m < g.n_materials; ++m) mu_maj = fmaxf(mu_maj, mu_total(g.mu_c511[m], g.mu_pe511[m], xs));
    // free path -ln(u) / mu: the fast log's absolute error (< 4e-7) moves a
    // step by < 5e-5 mm even in water, far below the position tolerance
    const float step = mu_maj > 0.0f ? -__logf(u01(r.x)) * (10.0f / mu_maj) : 3.0e38f;
    if (step >= s.trem) {                      // leaves the panel: back to flight
        s.x = fmaf(s.trem, s.dx, s.x); s.y = fmaf(s.trem, s.dy, s.y); s.z = fmaf(s.trem, s.dz, s.z);
        s.path += s.trem;
        to_global(g, s);
        s.last = s.panel;
        s.panel = -1;
        s.phase = kPhFlightOut;
        return kStatusOk;
    }
    s.x = fmaf(step, s.dx, s.x); s.y = fmaf(step, s.dy, s.y); s.z = fmaf(step, s.dz, s.z);
    s.path += step;
    s.trem -= step;
    const Loc L = locate(g, s.panel, s.x, s.y, s.z);
    const float pe = g.mu_pe511[L.mat] * xs.r3;
    const float mu_m = fmaf(g.mu_c511[L.mat], xs.g, pe);
    if (u01(r.y) * mu_maj >= mu_m) return kStatusOk;   // virtual
    float dep;
    bool dead = false;
    if (u01(r.z) * mu_m < pe) {                        // photoelectric
        dep = s.E;
        dead = true;
    } else {                                           // Compton (Klein-Nishina)
        float xm1;
        const int nt = kahn_sample(J.seed, s.h, kTagDetector, s.gamma, step_id, s.E, xm1);
        if (nt < 0) return kStatusTimeout;
        cnt.trials += (uint32_t)nt;
        const float omc = xm1 / (s.E * kInvMec2);
        // rotation in the panel frame with v as polar reference: for the ring
        // (w, u, v) is a rotation of (x, y, z) about the axis, so this equals the
        // global rotation; a posed panel takes its own v axis
        rotate_dir(s.dx, s.dy, s.dz, omc, u01(r.w));
        const float Ep = s.E / (1.0f + xm1);
        if (Ep < J.e_cut) {
            dep = s.E;
            dead = true;
        } else {
            dep = s.E * xm1 / (1.0f + xm1);
            s.E = Ep;
        }
    }
    if (L.crystal >= 0)
        record_hit<kTallies>(J, g, O, s, SL, max_entries, cnt, L.crystal, L.module, L.layer, step_id, dep);
    if (dead) { photon_done(J, g, s, cnt); return kStatusOk; }
    s.trem = panel_exit(g, s.x, s.y, s.z, s.dx, s.dy, s.dz);
    return kStatusOk;
}

// digitizer for one finished history: blur, window, warp-aggregated append
// (call with the lanes of `mask` converged; `active` lanes own a history).
// kJobDest = false: no job of the launch has a singles buffer of its own
// (every fixed launch), and the singles go to the launch's buffer alone.
template <bool kJobDest = true>
__device__ __forceinline__ void ev_finish(const JobDev *__restrict__ jobs, const GeomDev *__restrict__ geoms,
                                          const OutDev &O, const PState &s, bool active, const SinglesList &SL,
                                          uint32_t mask, Counters &cnt) {
    const int lane = threadIdx.x & 31;
    const JobDev *J = active ? &jobs[s.job] : nullptr;
    const bool ovf = active && s.ovf;
    const uint32_t n = (active && !ovf) ? s.nsing : 0u;
    cnt.singles += n;
    // histories whose list overflowed go to the fallback list instead
    {
        const uint32_t b = __ballot_sync(mask, ovf);
        if (b) {
            unsigned long long base = 0;
            const int leader = __ffs(b) - 1;
            if (lane == leader) base = atomicAdd(O.n_ovf, (unsigned long long)__popc(b));
            base = __shfl_sync(mask, base, leader);
            if (ovf) {
                const unsigned long long slot = base + __popc(b & lanemask_lt());
                if (slot < O.ovf_cap) { O.ovf_h[slot] = s.h; O.ovf_job[slot] = s.job; }
            }
        }
    }
    const uint32_t nmax = __reduce_max_sync(mask, n);
    for (uint32_t j = 0; j < nmax; ++j) {
        bool keep = false;
        float e = 0.f, eb = 0.f, db = 0.f;
        uint32_t unit = 0, dt = 0;
        if (j < n) {
            unit = SL.unit[j * SL.stride];
            e = SL.e[j * SL.stride];
            dt = SL.dt[j * SL.stride];
            const uint4 q = philox4x32_10(make_uint4((uint32_t)s.h, (uint32_t)(s.h >> 32), kTagDigi << 28, unit),
                                          make_uint2((uint32_t)J->seed, (uint32_t)(J->seed >> 32)));
            // one Box-Muller pair: the cosine normal blurs the energy, the sine one the depth
            float sp, cp;
            sincospif(2.0f * u01(q.y), &sp, &cp);
            // the accurate log here: near u = 1 the radius is small and an
            // absolute log error would become a large relative error of the blur
            const float rad = sqrtf(-2.0f * logf(u01(q.x)));
            const float sigma = J->sig_k * sqrtf(kE0 * e);
            eb = fmaf(sigma, rad * cp, e);
            db = fmaf(J->sig_doi, rad * sp, SL.ew[j * SL.stride] / e);
            keep = eb >= J->e_lo && eb <= J->e_hi;
        }
        const uint32_t b = __ballot_sync(mask, keep);
        if (!b) continue;
        // destination: the launch's singles buffer, or the job's own
        RawSingle *dst = O.s_raw;
        unsigned long long *dst_n = O.n_singles, dst_cap = O.s_cap;
        if (kJobDest && keep && J->s_raw) {
            dst = J->s_raw;
            dst_n = J->n_singles;
            dst_cap = J->s_cap;
        }
        unsigned long long slot = 0;
        if (!kJobDest || __all_sync(mask, dst_n == O.n_singles)) {
            // one counter for the warp (every fixed launch)
            unsigned long long base = 0;
            const int leader = __ffs(b) - 1;
            if (lane == leader) base = atomicAdd(O.n_singles, (unsigned long long)__popc(b));
            base = __shfl_sync(mask, base, leader);
            slot = base + __popc(b & lanemask_lt());
        } else if (keep) {
            // lanes grouped by destination, one atomic per group
            const uint32_t grp = __match_any_sync(b, reinterpret_cast<unsigned long long>(dst_n));
            const int leader = __ffs(grp) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(dst_n, (unsigned long long)__popc(grp));
            base = __shfl_sync(grp, base, leader);
            slot = base + __popc(grp & lanemask_lt());
        }
        if (keep) {
            if (slot < dst_cap) {
                const GeomDev &g = geoms[J->geom];
                int panel;
                if (g.readout_level == 0) panel = (int)unit;
                else if (g.readout_level == 1) panel = (int)(unit / (uint32_t)(g.modules_u * g.modules_v));
                else panel = (int)(unit / (uint32_t)(g.crystals_per_module * g.modules_u * g.modules_v));
                const uint64_t t = s.t0 + dt;
                // the sort key: a job with its own buffer is the one job of its run
                if (kJobDest && J->s_raw) J->s_keys[slot] = t;
                else O.s_keys[slot] = O.key_shift < 64 ? ((uint64_t)s.job << O.key_shift) | t : t;
                uint4 *r = reinterpret_cast<uint4 *>(dst + slot);
                r[0] = make_uint4((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)s.h, (uint32_t)(s.h >> 32));
                // a job with its own buffer is job 0 of the run that buffer belongs to
                r[1] = make_uint4(unit, (uint32_t)panel, kJobDest && J->s_raw ? 0u : (uint32_t)s.job,
                                  __float_as_uint(eb));
                r[2] = make_uint4(__float_as_uint(e), __float_as_uint(db), 0u, 0u);
            }
        }
    }
}

}  // namespace gpet
