// internal.h -- declarations shared by the library's translation units
// (device structs of the sort / coincidence stage and the host launchers).
#pragma once

#include <cuda_runtime.h>

#include "transport.cuh"

namespace gpet {

enum { kKernelDefault = 0, kKernelLoop = 1, kKernelWave = 2, kKernelCta = 3 };

struct LaunchCfg {
    int grid;            // CTAs of the transport kernel
    int block_size;      // threads per CTA
    int sm_count;
    int kernel;          // kKernelLoop / kKernelWave
    int max_smem_geoms;  // geometry descriptors staged in shared memory
    int compact_every;   // wavefront regrouping interval (events)
    int pool_depth;      // wavefront slots per lane (pool = 32 x depth histories per warp)
};

// radix sort working set (keys ping-pong between two buffers)
struct SortDev {
    uint64_t *keys[2];
    uint32_t *vals[2];
    uint32_t *ghist;                 // [8][256]
    int *plan;                       // [8] active, [8] source buffer, [1] final buffer
    uint32_t *tile_hist;             // [256][max_tiles]
    unsigned long long max_tiles;
    unsigned long long cap;
    const unsigned long long *n_in;  // device count of unsorted singles
    const RawSingle *in_raw;         // unsorted singles
    int *status;                     // run status word (kStatusSortStall), or NULL: unstaged passes
    int job_shift;                   // sort key = (job << job_shift) | t_ps; 64: the key is t_ps alone
    // one-sweep passes (the simulation path): decoupled look-back words, two
    // buffers of [tiles][256] that alternate between active passes, and a
    // tile counter per pass; NULL where the passes run through tile_hist
    unsigned long long *lb[2] = {nullptr, nullptr};
    unsigned int *tile_ctr = nullptr;
};

// Bit position of the job index in the 64-bit sort keys of a launch of n_jobs
// jobs: the job takes the fewest high bits that number the jobs, the time stamp
// the rest (64 for one job: the key is the time alone).
inline int sort_job_shift(int n_jobs) {
    int bits = 0;
    while ((1ll << bits) < (long long)n_jobs) ++bits;
    return 64 - bits;
}
// Largest time stamp a key with this shift holds (2^64 - 1 without job bits).
inline unsigned long long sort_time_limit(int job_shift) {
    return job_shift >= 64 ? ~0ull : (1ull << job_shift) - 1ull;
}

// time-ordered singles
struct SinglesDev {
    uint64_t *t, *h;
    int32_t *unit, *panel, *job;
    float *e, *eraw, *doi;
    unsigned long long *n;
};

struct CoincDev {
    uint8_t *flag;
    uint32_t *tile_cnt;
    int32_t *a, *b;
    unsigned long long *n;
    const uint64_t *window_ps;       // per job
};

struct JobStatsDev {
    int n_jobs;
    unsigned long long *s_off, *c_off;   // [n_jobs + 1]
    unsigned long long *hits;            // [n_jobs]
    const unsigned long long *tally_count;
    const long long *tally_off, *tally_n; // [n_jobs]
};

// most geometry descriptors a transport CTA stages in shared memory
constexpr int kMaxStagedGeoms = 16;

// Raise kernel fn's dynamic shared-memory limit on the current device to at
// least `bytes` (capped at the device's opt-in maximum).  The attribute is set
// only when it grows, so a launch never changes it while a live launch of the
// same kernel may be running (a change can wait for running launches).
cudaError_t ensure_dynamic_smem(const void *fn, size_t bytes);

// Load every kernel the transport and digitizer can launch (and set their
// shared-memory limits), once per device.  CUDA loads kernels lazily, and a
// load can wait for running kernels: a live launch's kernel waits on the host,
// so nothing may be loaded while it runs.
cudaError_t preload_kernels();
cudaError_t preload_transport_kernels();
cudaError_t preload_wave_kernels();
cudaError_t preload_cta_kernels();
cudaError_t preload_sort_kernels();
cudaError_t preload_window_kernels();
cudaError_t preload_copy_kernels();

// Geometry descriptors a transport launch stages in shared memory: as many of
// the first min(n_geoms, max_geoms) as fit without fewer resident CTAs than a
// launch that stages none (the rest are read through L1).  The kernel's
// dynamic shared-memory limit covers the largest staging.
template <class Kernel>
cudaError_t staged_geometry(Kernel k, int block, size_t pool_smem, int n_geoms, int max_geoms, int *ng_out,
                            size_t *smem_out, int *occ_out) {
    int ng = n_geoms < max_geoms ? n_geoms : max_geoms;
    if (ng < 0) ng = 0;
    cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void *>(k),
                                        pool_smem + (size_t)(max_geoms > 0 ? max_geoms : 0) * sizeof(GeomDev));
    if (e != cudaSuccess) return e;
    int occ0 = 0, occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, k, block, pool_smem);
    if (e != cudaSuccess) return e;
    for (;; --ng) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, block, pool_smem + (size_t)ng * sizeof(GeomDev));
        if (e != cudaSuccess) return e;
        if (occ >= occ0 || ng == 0) break;
    }
    *ng_out = ng;
    *smem_out = pool_smem + (size_t)ng * sizeof(GeomDev);
    *occ_out = occ;
    return cudaSuccess;
}

cudaError_t launch_job_stats(const SinglesDev &s, const CoincDev &C, const JobStatsDev &J, cudaStream_t st);
// the transport kernel cfg selects, then (with_redo) the re-simulation of
// histories whose singles list overflowed
cudaError_t launch_transport(const WorkDev &W, const OutDev &O, const LaunchCfg &cfg, cudaStream_t st,
                             bool with_redo = true);
cudaError_t launch_transport_redo(const WorkDev &W, const OutDev &O, const LaunchCfg &cfg, cudaStream_t st);
cudaError_t launch_transport_wave(const WorkDev &W, const OutDev &O, const LaunchCfg &cfg, cudaStream_t st);
cudaError_t launch_transport_cta(const WorkDev &W, const OutDev &O, const LaunchCfg &cfg, cudaStream_t st);
// warps resident at once in the transport launch that cfg selects (sizes the work chunks)
cudaError_t transport_resident_warps(int n_geoms, const LaunchCfg &cfg, long long *warps);
cudaError_t wave_resident_warps(int n_geoms, const LaunchCfg &cfg, long long *warps);
cudaError_t cta_resident_warps(int n_geoms, const LaunchCfg &cfg, long long *warps);
cudaError_t launch_sort_coinc(const SortDev &S, const SinglesDev &out, const CoincDev &C, int sm_count,
                              cudaStream_t st);
cudaError_t launch_radix_passes(const SortDev &S, int sm_count, cudaStream_t st);

// energy windows of one pass over the time-sorted singles
constexpr int kMaxWindows = 16;
struct WinDev {
    float lo[kMaxWindows], hi[kMaxWindows];
    int n;
};
// counts[job * n + w] += coincidences of window w (cap = capacity of the singles)
cudaError_t launch_coinc_windows(const SinglesDev &s, const CoincDev &C, const WinDev &win,
                                 unsigned long long *counts, unsigned long long cap, cudaStream_t st);

}  // namespace gpet
