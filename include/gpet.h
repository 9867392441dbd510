/*
 * gpet.h -- C ABI of the GB300 library for multi-layer PET photon-pair
 * transport (arxiv 2603.07327, "Extending gPET for Multi-Layer PET
 * Simulation").
 *
 * The library simulates back-to-back 511 keV annihilation photon pairs: decay
 * sampling (Sec. 2.3: point source, no positron range, annihilation at the
 * emission site; or a voxel activity map), Woodcock tracking through a
 * voxelised phantom (Sec. 2.1), straight flight to the first panel by
 * line-plane intersection (Sec. 2.1), step-by-step Woodcock transport inside
 * the panel-local frame with the layer-selection step and crystal
 * identification from the repetitive structure (Sec. 2.1, Fig. 1), transport
 * across several layers and panels (abstract), per-crystal hit tallies, and a
 * digitizer: per-readout-unit singles (crystal, module or panel level, Sec.
 * 2.1), energy blur, energy window, coincidence sorting (Sec. 2.3).
 *
 * Conventions for every call:
 *   - units are mm, keV, ns and 1/cm; times in the outputs are integer
 *     picoseconds;
 *   - every function returns an int status: 0 = GPET_OK, < 0 = an error code
 *     below; the thread-local message of the last error is gpet_last_error();
 *     no exception crosses the ABI;
 *   - pointer arguments marked "host" are read (or written) during the call
 *     only and are copied where kept; arguments marked "device" are CUDA
 *     device pointers owned by the caller;
 *   - opaque objects (gpet_scanner, gpet_result, gpet_batch, gpet_server) are
 *     owned by the library and released with their destroy/free call;
 *   - a `stream` argument is a cudaStream_t passed as void*; NULL selects the
 *     legacy default stream.  Calls that return results to the host
 *     synchronise that stream before returning.
 */
#ifndef GPET_H
#define GPET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* status codes                                                              */
/* ------------------------------------------------------------------------ */
#define GPET_OK 0
#define GPET_ERR_INVALID_ARG (-1) /* a NULL pointer, a negative size, an out-of-range field */
#define GPET_ERR_GEOMETRY (-2)    /* panels overlap, a layer leaves its module, zero pitch  */
#define GPET_ERR_OOM (-3)         /* a device or host allocation failed                    */
#define GPET_ERR_CUDA (-4)        /* a CUDA runtime call failed (message has the CUDA text),  */
                                  /* or a kernel reported an internal error: a history in   */
                                  /* a phase no event handles, or a time-sort tile copy     */
                                  /* that did not land within its bounded wait             */
#define GPET_ERR_TIMEOUT (-5)     /* a device loop hit its iteration cap (steps, trials)     */
#define GPET_ERR_OVERFLOW (-6)    /* an output buffer was too small; the run is flagged      */
#define GPET_ERR_BUSY (-7)        /* server admission denied (non-blocking submit)          */
#define GPET_ERR_TOO_SMALL (-8)   /* destination capacity too small; see gpet_result_counts  */

/* readout levels of singles (Sec. 2.1: crystal-, module- or panel-level) */
#define GPET_READOUT_PANEL 0
#define GPET_READOUT_MODULE 1
#define GPET_READOUT_CRYSTAL 3

/* source kinds */
#define GPET_SOURCE_POINT 0    /* isotropic pairs from pos_mm                              */
#define GPET_SOURCE_PHANTOM 1  /* isotropic pairs from the loaded phantom's activity map   */
#define GPET_SOURCE_PENCIL 2   /* collimated pair: photon 0 along dir, photon 1 along -dir */

/* ------------------------------------------------------------------------ */
/* descriptions (plain structs, host memory, copied by the calls)           */
/* ------------------------------------------------------------------------ */

/* Material of the synthetic physics model: linear attenuation at 511 keV and
 * its photoelectric share.  Photoelectric scales as (511/E)^3; Compton follows
 * the Klein-Nishina total cross section.  electron_density_cm3 = 0 anchors the
 * Compton coefficient at mu_total*(1-photo_frac) at 511 keV; > 0 uses
 * n_e * sigma_KN(E) as given. */
typedef struct {
    double mu_total_511_cm;
    double photo_frac_511;
    double electron_density_cm3;
} gpet_material;

/* One crystal layer inside a module (Sec. 2.1: each layer carries its own
 * crystal size, spacing and offset, and its own crystal and inter-crystal
 * materials, listed layer by layer).  A crystal occupies
 * [gap/2, pitch - gap/2) of its cell in u and v.  offset_u/v place the
 * crystal grid's low edge inside the module; gap_before is a radial gap
 * (e.g. a reflector) in front of the layer, filled with interval_mat. */
typedef struct {
    int32_t n_u, n_v;
    double pitch_u, pitch_v;
    double gap_u, gap_v;
    double depth;
    double gap_before;
    double offset_u, offset_v;
    int32_t crystal_mat, interval_mat; /* indices into gpet_scanner_desc.materials */
} gpet_layer;

/* Repetition-mode ring (Sec. 2.1): one panel definition, n_panels copies at
 * angles first_angle + 2 pi k / n_panels about the z axis, inner face at
 * inner_radius_mm.  Panel-local frame: w = depth from the inner face, u =
 * tangential (z x normal), v = axial.  Modules tile the panel face
 * (modules_u x modules_v of module_size, separated by module_gap); layers
 * stack along w in order.
 *
 * Non-repetition mode (Sec. 2.1: panels placed one by one): panel_poses != NULL
 * gives each of the n_panels copies of the same panel definition its own pose,
 * 12 doubles per panel in host memory, row k at panel_poses + 12 k: the global
 * unit vectors of the panel's w (depth, pointing away from the inner face), u
 * and v axes, then the global position (mm) of the centre of its inner face.
 * The axes must be orthonormal and right-handed (v = w x u) to 1e-6, and no two
 * panel boxes may overlap (GPET_ERR_GEOMETRY otherwise).  inner_radius_mm and
 * first_angle_rad are then ignored.  A Compton scatter inside a posed panel
 * takes the panel's own v axis as the polar reference of its direction
 * rotation (in the ring v = z, so both modes agree on a ring written as poses).
 * The array is copied by gpet_create_scanner. */
typedef struct {
    int32_t n_panels;
    double inner_radius_mm;
    double first_angle_rad;
    int32_t modules_u, modules_v;
    double module_size_u, module_size_v;
    double module_gap_u, module_gap_v;
    int32_t n_layers;
    const gpet_layer *layers;       /* host, n_layers entries */
    int32_t n_materials;
    const gpet_material *materials; /* host, n_materials entries */
    int32_t readout_level;          /* GPET_READOUT_* */
    const double *panel_poses;      /* host, n_panels x 12, or NULL for the ring */
} gpet_scanner_desc;

typedef struct {
    int32_t kind;         /* GPET_SOURCE_* */
    double pos_mm[3];     /* point and pencil sources */
    double dir[3];        /* pencil source axis (unit vector) */
    double activity_bq;   /* decay times are iid uniform on [0, n_decays / activity) */
} gpet_source;

/* Digitizer (Sec. 2.3: energy resolution, energy window, coincidence window).
 * Blur: FWHM(E) = fwhm_at_511 * sqrt(511 keV * E).  Window inclusive.
 * e_cut_kev is the transport cutoff: a photon below it deposits the rest. */
typedef struct {
    double fwhm_at_511;
    double e_lo_kev, e_hi_kev;
    double coinc_window_ns;
    double e_cut_kev;
    double doi_fwhm_mm;   /* analytic depth-of-interaction blur of each single (0 = none); the
                             single's depth is the energy-weighted depth of its hits (Sec. 4
                             favours analytic light-sharing / DOI blurring over optical transport) */
} gpet_digitizer;

/* Launch options; pass NULL for defaults. */
typedef struct {
    int32_t keep_hits;       /* 1: also store every crystal interaction (tests, DOI studies) */
    int32_t block_size;      /* threads per CTA of the transport kernel (0 = 256; kernel 3: 128, 256 or 512) */
    int32_t blocks_per_sm;   /* resident CTAs per SM (0 = tuned default)                   */
    int32_t kernel;          /* 0 = tuned, else 3; 1 = per-lane event loop, 2 = per-warp
                                wavefront, 3 = wavefront with one phase per CTA            */
    int32_t compact_every;   /* wavefront regrouping interval in events (0 = default)      */
    int32_t pool_depth;      /* wavefront histories per lane in shared memory, 2..4 (0 = 2)  */
    void *stream;            /* cudaStream_t */
    uint64_t h_begin, h_end; /* run only histories [h_begin, h_end) of the n_decays run (a shard);
                                h_end = 0 means n_decays.  Decay times keep the whole run's span,
                                so shards of one run merge exactly (tallies add, singles concatenate) */
} gpet_options;

typedef struct gpet_scanner gpet_scanner;
typedef struct gpet_result gpet_result;

/* ------------------------------------------------------------------------ */
/* scanner and phantom                                                      */
/* ------------------------------------------------------------------------ */

/* Build a scanner from its hierarchical description (Sec. 2.1, Fig. 1).
 * desc: host, copied.  Validates: counts >= 1, n_panels <= 64, n_layers <= 8,
 * n_materials <= 8, pitches > gaps >= 0, every layer inside its module,
 * panels not overlapping.  Returns GPET_ERR_GEOMETRY or GPET_ERR_INVALID_ARG
 * on a bad description; *out is set only on success. */
int gpet_create_scanner(const gpet_scanner_desc *desc, gpet_scanner **out);
void gpet_destroy_scanner(gpet_scanner *sc);

/* Number of crystals of the scanner (crystal identification from the
 * repetitive structure, Sec. 2.1; global crystal ids are 0 .. n-1):
 * id = (((panel * modules_v + m_v) * modules_u + m_u) * C + layer_offset + i_v * n_u + i_u)
 * with C the crystal count of one module summed over layers. */
int gpet_scanner_crystals(const gpet_scanner *sc, int64_t *n_crystals);

/* Load (or replace) the voxelised phantom used by the next simulations
 * (Sec. 2.3: the phantom attenuates and, with an activity map, is the source).
 * Grid: nx x ny x nz voxels of voxel_mm, low corner at origin_mm (global mm).
 * material_ids: host, nx*ny*nz bytes, x fastest, indices into materials.
 * activity: host, nx*ny*nz floats (>= 0) or NULL when the phantom only
 * attenuates.  Photons never re-enter the phantom after reaching a panel, so
 * the grid must clear the detector: inside the ring's inner radius, or, for a
 * scanner with panel poses, overlapping no panel box (GPET_ERR_GEOMETRY
 * otherwise).  All arrays are copied; the device copies are the scanner's. */
int gpet_load_phantom(gpet_scanner *sc, int32_t nx, int32_t ny, int32_t nz, const double voxel_mm[3],
                      const double origin_mm[3], const uint8_t *material_ids, const float *activity,
                      int32_t n_materials, const gpet_material *materials);

/* ------------------------------------------------------------------------ */
/* simulation (plain form: one scanner, one source)                          */
/* ------------------------------------------------------------------------ */

/* Simulate histories 0 .. n_decays-1 of one source with RNG key `seed`: the
 * decays of Sec. 2.3, the transport of Sec. 2.1, and the digitizer and
 * coincidence sorting of Sec. 2.3.
 * Random numbers come from Philox4x32-10 addressed by (history, region,
 * photon, step, sub-draw), so any history is reproducible on its own.
 * Enqueues transport, digitizer, time sort and coincidence sorting on
 * opt->stream and synchronises it.  On success *out holds the result.
 * n_decays must be >= 1, and the acquisition n_decays / activity_bq below
 * 2^62 ps (53 days): GPET_ERR_INVALID_ARG otherwise.  One launch holds at most
 * 2^31 - 1 singles (coincidences index them with int32): GPET_ERR_OVERFLOW
 * beyond, and the run is to be split by history range.  GPET_ERR_TIMEOUT when a photon
 * exceeded 1000 Woodcock steps in one region or 1000 Klein-Nishina trials
 * (the photon is dropped, nothing waits); the run's other outputs are not
 * returned. */
int gpet_simulate(gpet_scanner *sc, const gpet_source *src, const gpet_digitizer *dg, uint64_t n_decays,
                  uint64_t seed, const gpet_options *opt, gpet_result **out);

/* Counts of a finished result. */
typedef struct {
    uint64_t n_decays;
    uint64_t hits;          /* crystal interactions (all, whether stored or not) */
    uint64_t singles;       /* singles inside the energy window */
    uint64_t coincidences;
    int64_t n_crystals;
    uint64_t det_steps, flights, compton_trials, entered, phantom_steps; /* event counters */
    int32_t status;         /* GPET_OK or the device error that flagged the run */
    float transport_ms;     /* CUDA-event time of the transport kernels on the run's stream */
    float digitizer_ms;     /* CUDA-event time of time sort + coincidence sorting */
    uint64_t h2d_bytes;     /* descriptor bytes uploaded for the run (jobs, geometry, work table) */
    uint64_t wave_iterations, wave_lanes; /* wavefront kernel: regrouping steps and lanes they fed */
    uint64_t screened_flights;            /* flights decided by the axial screen (no panel test) */
    uint64_t singles_formed;              /* singles before the energy window */
    double latency_ms;      /* served requests: submission to result ready (0 otherwise) */
    /* events run per history phase by the CTA-synchronous kernel (kernel 3; zero for the others):
       [1] decay, [2] phantom step, [3] flight from the decay or phantom, [4] detector step,
       [5] finish (digitizer of a history), [6] flight after a panel exit; [0] unused */
    uint64_t phase_events[7];
} gpet_counts;
int gpet_result_counts(const gpet_result *r, gpet_counts *out);

/* Result arrays: the hits and tallies of Sec. 2.1 and the singles and
 * coincidences of Sec. 2.3.  (The accessors themselves are library
 * infrastructure; the paper defines no interface.)  Singles are sorted by
 * time (ties in any order).
 * Coincidence indices copied by gpet_result_copy number the result's own
 * singles; through gpet_result_device_ptr of a batch view they count from the
 * first single of the whole batch. */
enum {
    GPET_SINGLES_T_PS = 0,      /* uint64 [singles]   time of the earliest hit */
    GPET_SINGLES_H = 1,         /* uint64 [singles]   history id               */
    GPET_SINGLES_UNIT = 2,      /* int32  [singles]   readout unit id          */
    GPET_SINGLES_PANEL = 3,     /* int32  [singles]                            */
    GPET_SINGLES_E = 4,         /* float  [singles]   blurred energy (keV)     */
    GPET_SINGLES_E_RAW = 5,     /* float  [singles]   deposited energy (keV)   */
    GPET_COINC_A = 6,           /* int32  [coincidences] index into singles    */
    GPET_COINC_B = 7,           /* int32  [coincidences]                       */
    GPET_TALLY_COUNT = 8,       /* uint64 [n_crystals] interactions per crystal */
    GPET_TALLY_EFX = 9,         /* uint64 [n_crystals] sum of round(E * 2^20) */
    GPET_HITS_H = 10,           /* uint64 [hits] (keep_hits only)              */
    GPET_HITS_GSTEP = 11,       /* int32  [hits] photon << 24 | step           */
    GPET_HITS_CRYSTAL = 12,     /* int32  [hits] global crystal id             */
    GPET_HITS_LAYER = 13,       /* int32  [hits]                               */
    GPET_HITS_WUV = 14,         /* float  [hits][3] panel-local position (mm)  */
    GPET_HITS_E = 15,           /* float  [hits] deposit (keV)                 */
    GPET_HITS_T_PS = 16,        /* uint64 [hits]                               */
    GPET_SINGLES_DOI = 17,      /* float  [singles]   blurred depth of interaction (mm from the inner face) */
    GPET_RESULT_ARRAYS = 18
};

/* Copy one result array to host memory dst (cap_bytes long).  Returns
 * GPET_ERR_TOO_SMALL when cap_bytes is below the array's size, and
 * GPET_ERR_INVALID_ARG for an array the run did not keep. */
int gpet_result_copy(const gpet_result *r, int32_t which, void *dst, size_t cap_bytes);

/* Copy one array of the whole launch that result r belongs to -- every job of
 * its batch, in job order (for a plain run, the same as gpet_result_copy):
 * singles of all jobs, coincidences with indices into those singles, the
 * tallies of all jobs one after the other.  One large copy instead of one per
 * job.  *bytes (may be NULL) receives the array's size; dst = NULL with
 * cap_bytes = 0 only queries it.  GPET_ERR_TOO_SMALL when cap_bytes is below
 * the size. */
int gpet_result_copy_run(const gpet_result *r, int32_t which, void *dst, size_t cap_bytes, size_t *bytes);
/* The same copy enqueued on `stream` (a cudaStream_t) and returned at once.
 * The caller keeps r (and with it the device arrays) alive and dst untouched
 * until the stream has passed the copy.
 * How both run copies move the bytes: into page-locked host memory
 * (cudaHostAlloc, cudaHostRegister) whose address is 16-byte aligned, a
 * kernel whose threads load the device array and store into dst through its
 * device mapping; anywhere else, cudaMemcpy / cudaMemcpyAsync.  The copy
 * engines' reads of device memory that had been freed and allocated again
 * fell to a fifth of the host link's rate once other GPU work had run on the
 * device, where the stores kept the link's rate (193 GB/s on GB300).  The
 * kernel needs free SMs: enqueued beside a running persistent launch, it runs
 * once that launch ends.  Into pageable memory the async copy is not
 * asynchronous. */
int gpet_result_copy_run_async(const gpet_result *r, int32_t which, void *dst, size_t cap_bytes, size_t *bytes,
                               void *stream);

/* Device pointer of one result array (valid until gpet_result_free), or NULL. */
const void *gpet_result_device_ptr(const gpet_result *r, int32_t which);
void gpet_result_free(gpet_result *r);

/* ------------------------------------------------------------------------ */
/* batched form: many designs and sources in one persistent launch           */
/* ------------------------------------------------------------------------ */

/* The paper runs one simulation per design (Sec. 3); a batch, which it does
 * not define, runs several in one launch.
 * A batch runs n_jobs independent simulations -- job j is (scanners[j],
 * sources[j], digitizers[j], n_decays[j], seeds[j]) exactly as gpet_simulate
 * would run it -- in one persistent transport launch over a shared work
 * queue, one time sort segmented by job and one coincidence pass.  The
 * enqueue is captured into a CUDA graph at creation and replayed by
 * gpet_batch_run.  A job's results are identical to gpet_simulate's for the
 * same inputs (every random number is addressed by seed and history id).
 * All arrays: host, n_jobs entries, copied.  Scanners must outlive the batch.
 * n_jobs <= 4095.  opt->stream NULL: the batch creates its own stream.
 * The time sort orders (job, time) keys of 64 bits whose job field takes the
 * fewest bits that number the jobs (7 for 65..128 jobs, 12 for 4095): every
 * job's acquisition must fit in the rest, 2^(64 - bits) ps minus 2^32 ps of
 * flight time (about 20 h for 256 jobs, 75 min for 4095);
 * GPET_ERR_INVALID_ARG otherwise, before any device work. */
typedef struct gpet_batch gpet_batch;
int gpet_batch_create(int32_t n_jobs, gpet_scanner *const *scanners, const gpet_source *sources,
                      const gpet_digitizer *digitizers, const uint64_t *n_decays, const uint64_t *seeds,
                      const gpet_options *opt, gpet_batch **out);
/* Replay the captured graph (the same simulations again) and synchronise. */
int gpet_batch_run(gpet_batch *b);
int gpet_batch_jobs(const gpet_batch *b, int32_t *n_jobs);
/* Counts over the whole batch (event counters and stage times are batch-wide). */
int gpet_batch_counts(const gpet_batch *b, gpet_counts *total);
/* A view of job `job` of the last run: its singles, coincidences (indices
 * into its own singles) and tallies.  Free with gpet_result_free; the view
 * keeps the batch's device memory alive, and a later gpet_batch_run
 * overwrites it with identical values. */
int gpet_batch_result(const gpet_batch *b, int32_t job, gpet_result **out);
void gpet_batch_destroy(gpet_batch *b);
/* One-shot batch without a graph: outs[j] receives job j's result. */
int gpet_simulate_batch(int32_t n_jobs, gpet_scanner *const *scanners, const gpet_source *sources,
                        const gpet_digitizer *digitizers, const uint64_t *n_decays, const uint64_t *seeds,
                        const gpet_options *opt, gpet_result **outs);

/* ------------------------------------------------------------------------ */
/* sensitivity map (Sec. 2.4)                                                */
/* ------------------------------------------------------------------------ */

#define GPET_MAX_WINDOWS 16

/* NEMA NU4-style sensitivity S(r, E) (Sec. 2.4: sensitivity as a function of
 * source position and energy window): the coincidences a point source at r
 * gives in energy window E, per decay.  One batched launch runs every
 * (scanner, position) pair as a job: job j = s * n_positions + p is an
 * isotropic point source at positions_mm[3p .. 3p + 2] (mm) with n_decays
 * decays at activity_bq, under Philox key seed + p -- the same decays for
 * every scanner, so designs are compared on common random numbers.  The
 * digitizer's blur, coincidence window, cutoff and DOI blur apply; its
 * e_lo_kev / e_hi_kev are ignored.  Transport and singles run once with the
 * union of the energy windows, and one pass over the time-sorted singles
 * counts, for every window, the coincidences that a run with that window alone
 * counts (dropping singles outside a window can split a cluster of singles
 * close in time, never join two).
 *   scanners     host, n_scanners handles (>= 1)
 *   positions_mm host, n_positions x 3 doubles (>= 1 position)
 *   windows_kev  host, n_windows x (lo, hi) doubles, 0 <= lo <= hi, inclusive;
 *                1 <= n_windows <= GPET_MAX_WINDOWS
 *   counts       host, n_scanners x n_positions x n_windows uint64 (row-major):
 *                coincidences
 *   sens         host, the same shape in double: counts / n_decays, or NULL
 *   total        host or NULL: counts of the whole launch (event counters,
 *                stage times; singles and coincidences of the union window)
 * n_scanners x n_positions <= 4095 jobs.  Returns GPET_ERR_INVALID_ARG for bad
 * sizes or windows; other codes as gpet_simulate. */
int gpet_sensitivity_map(int32_t n_scanners, gpet_scanner *const *scanners, int32_t n_positions,
                         const double *positions_mm, double activity_bq, const gpet_digitizer *digitizer,
                         int32_t n_windows, const double *windows_kev, uint64_t n_decays, uint64_t seed,
                         const gpet_options *opt, uint64_t *counts, double *sens, gpet_counts *total);

/* Symmetric percent difference of two sensitivities (Sec. 2.4):
 * out[i] = 200 (s_a[i] - s_b[i]) / (s_a[i] + s_b[i]), NaN where both are zero.
 * Host arrays of n doubles (out may alias either input). */
int gpet_delta_sym(int64_t n, const double *s_a, const double *s_b, double *out);

/* ------------------------------------------------------------------------ */
/* time sort that allocates no device memory                                 */
/* ------------------------------------------------------------------------ */

/* The paper has no counterpart of this call.  It exists for callers that
 * cannot call cudaMalloc -- a process whose device memory is all handed out
 * up front by another allocator (for example a caching allocator that has
 * reserved the pool, or a server with a fixed memory budget), or a
 * latency-critical loop that cannot take an allocation's implicit device
 * synchronisation.  It runs the digitizer's radix time sort on n 64-bit keys
 * (the singles' time stamps in ps) with its whole working set in a fixed
 * 24.3 MiB array that is part of the library image, held on every GPU that
 * loads the library until the process exits; it calls no cudaMalloc, no
 * cudaFree and no allocating library routine.
 *   d_t_in     device, n uint64 keys (read only)
 *   d_t_out    device, n uint64: the keys in ascending order
 *   d_perm_out device, n uint32 or NULL: d_t_out[i] = d_t_in[d_perm_out[i]];
 *              the sort is stable (equal keys keep their input order)
 *   n          <= 1048576 (2^20); larger n returns GPET_ERR_INVALID_ARG
 *   stream     cudaStream_t; the call is asynchronous on it
 * The first call on a device, made with that device current, is its set-up:
 * CUDA loads a library's kernels and device arrays lazily, so that call loads
 * the code it runs and the 24.3 MiB array, which takes device memory then.
 * Make that first call before the process hands its device memory to another
 * allocator, and before any stream capture; later calls allocate nothing.
 * Every call looks up the array's device address afresh (a host-side lookup),
 * so a cudaDeviceReset, which reloads the array, leaves no stale address.
 * Every call shares the one array and overwrites its previous contents, so
 * calls that overlap on the GPU (other streams, other host threads) race:
 * serialise them. */
int gpet_sort_times_noalloc(const uint64_t *d_t_in, uint64_t n, uint64_t *d_t_out, uint32_t *d_perm_out,
                            void *stream);

/* ------------------------------------------------------------------------ */
/* autotuner                                                                 */
/* ------------------------------------------------------------------------ */

/* Library infrastructure with no counterpart in the paper: a launch-form
 * choice for the transport of Sec. 2.1.
 * Time the candidate launch forms of the transport kernel -- the per-lane
 * event loop, the per-warp wavefront, the CTA-synchronous wavefront at 128,
 * 256 or 512 threads, pool depth 2 or 3 and compaction interval 1, 2 or 4
 * (gpet_options.compact_every: detector or phantom steps a lane runs between
 * regroupings) -- on a pilot run (pilot_decays >= 1000, seed)
 * of the caller's workload, and return the fastest in *best (its transport
 * time in *best_ms, may be NULL).  The choice is remembered for the scanner's
 * design class (panels, layers, phantom) on this device's SM count; later
 * launches with gpet_options.kernel = 0 use it.  Runs the pilot on the
 * legacy default stream. */
int gpet_autotune(gpet_scanner *sc, const gpet_source *src, const gpet_digitizer *dg, uint64_t pilot_decays,
                  uint64_t seed, gpet_options *best, float *best_ms);

/* ------------------------------------------------------------------------ */
/* per-event costs (measurement)                                             */
/* ------------------------------------------------------------------------ */

/* Library infrastructure with no counterpart in the paper: the cost of each
 * event of the transport of Sec. 2.1 / 2.3 when it runs alone.  Histories
 * 0 .. n_sample - 1 of the caller's workload (scanner, source, digitizer,
 * seed) are run once, one GPU lane per history, keeping up to 65536 states
 * that entered each history phase; then, per phase, a kernel in which every
 * lane of the GPU runs that phase's event on those states is timed with CUDA
 * events (best of three after a warm-up launch).
 *   ns_per_event  host, 7 doubles: [p] = GPU time per event of phase p when
 *                 the whole GPU runs only that event (phases as in
 *                 gpet_counts.phase_events; 0 where no state of the phase
 *                 occurred; [0] unused)
 *   states        host, 7 uint64 or NULL: states kept per phase
 * n_sample in [1000, 2^32].  Runs on a stream of its own and synchronises it;
 * allocates device memory for the sample run and the state pools. */
int gpet_event_costs(gpet_scanner *sc, const gpet_source *src, const gpet_digitizer *dg, uint64_t n_sample,
                     uint64_t seed, double *ns_per_event, uint64_t *states);

/* ------------------------------------------------------------------------ */
/* serving loop: continuous batching of simulation requests                  */
/* ------------------------------------------------------------------------ */

/* Library infrastructure with no counterpart in the paper: simulations of
 * Sec. 2.1-2.3 served as requests, with continuous batching.
 * A server accepts simulation requests from any host thread while earlier
 * ones run.  One pipeline thread keeps a transport launch running and appends
 * arriving requests to the work table of that launch while its kernel runs;
 * the persistent kernel takes them up as slots free.  A request of more than
 * piece_decays decays is split into history ranges that join successive
 * launches (one range per request at a time, so small requests do not queue
 * behind large ones); the kernel writes those ranges' singles and tallies into
 * the request's own device buffers, which stay on the device until its last
 * range has run, and its time sort and coincidence sorting then run once.  A
 * launch takes new requests until it is max_launch_ms old or full, or until
 * the queue is empty and its published work is all taken; its digitizer then
 * runs, and the next launch starts.  Device memory counts against the budget
 * per launch (a quarter of the budget at most) and per split request, until
 * the results that view it are freed, so a client that keeps results while it
 * waits for later requests can stall admission: free results once read.  A
 * launch's results then move to memory of their own size, and its buffers go
 * back: during that copy the server holds both, so its peak can pass the
 * budget by the size of the results being copied.  A request whose singles
 * overflowed its launch's buffer runs again alone, at its exact size, once no
 * launch is running; that run is not held to the budget either.  A request's
 * result equals gpet_simulate's for the same inputs. */
typedef struct gpet_server gpet_server;
typedef struct {
    size_t hbm_budget_bytes;      /* device memory the server may hold */
    int32_t workers;              /* 0..8, accepted for compatibility: one pipeline serves all requests */
    int32_t max_jobs_per_launch;  /* jobs one launch takes (0 = 256, at most 4095) */
    gpet_options launch;          /* kernel options of every launch (stream, keep_hits ignored) */
    double max_launch_ms;         /* a launch takes new requests for at most this long (0 = 20 ms) */
    uint64_t piece_decays;        /* larger requests run in ranges of this many decays (0 = 4e6; at
                                     most half of what one launch's singles buffer is sized for) */
} gpet_server_config;
typedef struct {
    uint64_t submitted, completed, rejected, launches, max_jobs_per_launch, pairs_completed;
    uint64_t bytes_in_use, peak_bytes, queued;
    uint64_t live_appends;        /* jobs appended to a launch whose kernel was already running */
    uint64_t pieces;              /* history ranges of split requests handed to launches */
    double transport_ms;          /* GPU time of the launches' transport kernels, open to close (a live
                                   * kernel's waits for appended work included) */
    double digitizer_ms;          /* GPU time of the launches' and split requests' time sorts and
                                   * coincidence sorting */
} gpet_server_stats;
int gpet_server_create(const gpet_server_config *cfg, gpet_server **out);
/* Queue one request.  The scanner (and its phantom) must stay alive until the
 * request's result has been taken.  block = 0: GPET_ERR_BUSY when the budget
 * cannot take it now; block = 1: it waits in the queue.  GPET_ERR_OOM when it
 * alone exceeds the budget, or when a request above piece_decays does not fit
 * beside one launch arena (its own buffers and the launch that runs its pieces
 * are held together).  *req_id identifies it for poll / wait. */
int gpet_server_submit(gpet_server *s, gpet_scanner *sc, const gpet_source *src, const gpet_digitizer *dg,
                       uint64_t n_decays, uint64_t seed, int32_t block, uint64_t *req_id);
/* *out = NULL while the request runs; its result (ownership passes to the
 * caller, latency in gpet_counts.latency_ms) once done; the request's error
 * code if it failed.  A taken request id is forgotten.  wait blocks until the
 * request is done; if another caller takes the same id meanwhile, wait
 * returns GPET_ERR_INVALID_ARG. */
int gpet_server_poll(gpet_server *s, uint64_t req_id, gpet_result **out);
int gpet_server_wait(gpet_server *s, uint64_t req_id, gpet_result **out);
int gpet_server_stats_get(gpet_server *s, gpet_server_stats *out);
/* Finish the queued requests, stop the pipeline, free untaken results. */
void gpet_server_destroy(gpet_server *s);

/* Thread-local text of the last error (never NULL). */
const char *gpet_last_error(void);

/* Library version string. */
const char *gpet_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GPET_H */
