// host.h -- host-side objects behind the opaque handles of include/gpet.h and
// the run machinery shared by the plain, batched and served entry points.
#pragma once

#include <cstdint>
#include <functional>
#include <memory>
#include <string>
#include <vector>

#include "gpet.h"
#include "internal.h"

struct gpet_scanner {
    gpet_scanner_desc desc;
    std::vector<gpet_layer> layers;
    std::vector<gpet_material> materials;
    gpet::GeomDev g;
    std::vector<double> poses;   // non-repetition mode: n_panels x 12 (copy of desc.panel_poses)
    std::vector<float> pose_dev; // its device form: n_panels x 16 (see GeomDev::pose)
    int64_t n_crystals = 0;
    // phantom
    bool has_phantom = false;
    int32_t ph_n[3] = {0, 0, 0};
    double ph_voxel[3] = {0, 0, 0}, ph_origin[3] = {0, 0, 0};
    std::vector<gpet_material> ph_materials;
    uint8_t *ph_mat = nullptr;
    double *ph_cdf = nullptr;
    int32_t *ph_guide = nullptr;
    int32_t ph_buckets = 0;
    double ph_gscale = 0.0;
    double ph_total = 0.0;
    int64_t ph_last_active = -1;
};

int gpet_fail(int code, const char *fmt, ...);
// tuned launch form for this scanner's design class on a device with `sms` SMs
bool gpet_tuned_options(const gpet_scanner *sc, int sms, gpet_options *out);
int gpet_cuda_fail(cudaError_t e, const char *where);
int gpet_xs_table(const float **out, float *ln_emin, float *inv_h);
int gpet_build_geometry(const gpet_scanner_desc *d, gpet::GeomDev &g, int64_t &n_crystals,
                        std::vector<float> *pose_dev = nullptr);
// bytes that identify a scanner's geometry (descriptor and panel poses), for deduplication
std::string gpet_geometry_key(const gpet_scanner *sc);
int gpet_make_job(const gpet_scanner *sc, const gpet_source *src, const gpet_digitizer *dg, uint64_t n_decays,
                  uint64_t seed, gpet::JobDev &J, uint64_t h_begin = 0, uint64_t h_end = 0);

namespace gpet {

// Most singles one launch holds: coincidences index the time-ordered singles
// with int32 (GPET_COINC_A/B), and the sort's indices and scatter positions
// are 32-bit.  Larger runs are split by history range or into fewer jobs.
constexpr uint64_t kMaxSinglesPerLaunch = 0x7FFFFFFFull;

// capacities of one run's output buffers
struct RunCaps {
    uint64_t singles = 0, hits = 0, ovf = 0;
    bool guess = true;   // first guesses (clamped to the free device memory), not exact counts
};

// device header read back after a run (all zeroed before launch)
struct RunHeader {
    // det_steps, flights, trials, entered, phantom_steps, hits, wavefront iterations,
    // wavefront lanes, screened flights, singles formed
    // ... singles formed, then (CTA-synchronous kernel) the events run per phase in slots 10 + phase
    unsigned long long counters[20];
    unsigned long long n_singles, n_hits, n_ovf, n_sorted, n_coinc, next_chunk;
    int status;
    int pad[3];
};

// One launch of one or more jobs: all device memory lives in a single arena.
struct Run {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<JobDev> jobs;            // host copies (tally pointers filled by plan)
    std::vector<GeomDev> geoms;
    std::vector<std::vector<float>> geom_pose;  // per geometry: posed-panel table (empty for the ring)
    std::vector<int64_t> tally_off;      // per job, in crystals
    std::vector<int64_t> job_crystals;
    std::vector<uint64_t> windows;       // coincidence window per job (ps)
    std::vector<unsigned long long> chunk_start;
    unsigned int chunk_size = 2048;
    RunCaps caps;
    bool keep_hits = false;
    LaunchCfg cfg{};
    // arena
    void *arena = nullptr;
    size_t arena_bytes = 0;
    size_t zero_bytes = 0;               // leading bytes cleared before every launch
    RunHeader *d_hdr = nullptr;
    RunHeader h_hdr{};
    WorkDev W{};
    OutDev O{};
    SortDev S{};
    SinglesDev SD{};
    CoincDev C{};
    unsigned long long *d_tally_count = nullptr, *d_tally_efx = nullptr;
    uint64_t *d_window = nullptr;
    int64_t total_crystals = 0;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // before transport, after transport, after digitizer
    float transport_ms = 0.f, digitizer_ms = 0.f;
    uint64_t h2d_bytes = 0;
    // per-job segments of the outputs (device, then host copies after collect)
    JobStatsDev JS{};
    std::vector<unsigned long long> s_off, c_off, job_hits;
    // energy windows counted in one pass over the sorted singles (sensitivity map)
    std::vector<float> win_lo, win_hi;
    unsigned long long *d_win_counts = nullptr;  // [job][window], cleared before every launch
    std::vector<unsigned long long> win_counts;
    bool own_stream = false;
    std::function<void()> on_release;    // called once when the run's memory is gone
    // Live launch (serving loop): the tables have room for `live_cap` jobs,
    // geometries, tally crystals and posed-panel floats; the host appends jobs
    // while the transport kernel runs (run_live_append) and closes the launch
    // (run_live_close) before enqueuing the digitizer.
    bool live = false;
    struct LiveCap {
        int jobs = 0, geoms = 0;
        int64_t crystals = 0;
        size_t pose_floats = 0;
        unsigned chunk = 512;            // histories per chunk
    } live_cap;
    cudaStream_t upload_stream = nullptr;  // descriptor uploads and live appends (NULL: the run's stream)
    void *stage = nullptr;               // pinned host staging of live appends (caller-owned)
    size_t stage_bytes = 0;
    unsigned long long *d_live = nullptr;   // [0] published chunks, [1] closed flag, [2] chunks claimed
    uint64_t live_tail = 0;
    int64_t live_tally_used = 0;
    size_t live_pose_used = 0;
    std::vector<std::string> geom_keys;  // live: descriptor bytes of each geometry (deduplication)
    // device tables (kept for live appends)
    JobDev *d_jobs = nullptr;
    GeomDev *d_geoms = nullptr;
    unsigned long long *d_chunk_start = nullptr;
    float *d_pose = nullptr;
    long long *d_toff = nullptr, *d_tn = nullptr;
    // digitize-only run: its singles were appended by other launches' kernels
    // (a served request split over several launches); no transport, and its
    // zeroed region is cleared by the copy engine when planned
    bool digitize_only = false;
    const void *zeros = nullptr;         // pinned host block of zeros (caller-owned) for that clear
    size_t zeros_bytes = 0;
    ~Run();
};

int run_plan(Run &R);                  // allocate the arena, upload jobs and geometry
int run_enqueue(Run &R);               // memset + transport + sort + coincidences (capturable)
int run_enqueue_transport(Run &R);     // memset + transport
int run_enqueue_digitizer(Run &R);     // sort + coincidences + per-job statistics
int run_collect(Run &R);               // synchronise, read the header, map device status
// live launch: append one job (its scanner's geometry is added when new) and
// publish it to the running kernel; GPET_ERR_BUSY when a table is full
int run_live_append(Run &R, const JobDev &J, const gpet_scanner *sc, uint64_t window_ps);
int run_live_close(Run &R);            // publish the end of the work queue
int run_live_taken(Run &R, uint64_t *taken);  // chunks the kernel has claimed so far
// results of a collected run copied into device memory of exactly their size
std::shared_ptr<Run> run_compact(const Run &R, cudaStream_t st, int *status);
void run_release(Run &R);
int run_default_cfg(Run &R, const gpet_options *opt, const gpet_scanner *sc_for_tuning = nullptr);

}  // namespace gpet

// A result views one job of a run: the whole run for gpet_simulate, one job
// of a batch for gpet_batch_result.  Runs are shared by their views.
struct gpet_result {
    std::shared_ptr<gpet::Run> run;
    gpet_counts counts{};
    int job = 0;
};

namespace gpet {
// device bytes a run of these totals will take (the arena layout of run_plan)
size_t run_footprint(uint64_t total_decays, int64_t total_crystals, int n_jobs, size_t n_geoms, bool keep_hits);
}

struct gpet_batch {
    std::shared_ptr<gpet::Run> run;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<uint64_t> n_decays;
    std::vector<int64_t> n_crystals;
    ~gpet_batch();
};

int gpet_batch_build_run(gpet::Run &R, int32_t n_jobs, gpet_scanner *const *scanners, const gpet_source *sources,
                         const gpet_digitizer *digitizers, const uint64_t *n_decays, const uint64_t *seeds,
                         const gpet_options *opt);

namespace gpet {
void fill_counts(const Run &R, int job, uint64_t n_decays, int64_t n_crystals, gpet_counts *c);
int run_with_retry(Run &R);            // plan + enqueue + collect, one exact-size re-run on overflow
}
