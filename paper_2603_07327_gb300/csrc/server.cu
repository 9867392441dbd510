// server.cu -- serving loop with continuous batching into live launches.
//
// Requests (scanner design + source + digitizer + decay count + seed) arrive
// through gpet_server_submit from any host thread.  One pipeline thread keeps
// a transport launch open on the GPU and appends the requests that arrive to
// its work table while its kernel runs (a live launch: the persistent warps
// take the new jobs' chunks as they are published, see WorkDev).  A request of
// more than piece_decays histories is split into history ranges that join
// successive launches, one range per request and pass so that small requests
// are not queued behind large ones; the kernel writes the singles and tallies
// of those pieces straight into the request's own device buffers, so the
// request's state stays on the device between pieces, and its time sort and
// coincidence sorting run once, after its last piece.  A launch takes new work
// until it is max_launch_ms old or a table is full, or until the queue is empty
// and every published chunk has been claimed; it is then closed, its time sort,
// coincidence sorting and per-job statistics are enqueued behind its transport
// on the same stream, and the next launch opens once those have run and the
// results have been collected (while a live kernel holds every SM, the loop
// makes no device-to-device copy: such a copy may need the SMs).  Device memory
// counts against the budget per launch arena and per split request, from
// allocation until the results that view it are freed.  Every random number is
// addressed by (seed, history), so a request's result is the same alone and in
// any mix, whole or in pieces.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "host.h"

using namespace gpet;

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t id = 0;
    gpet_scanner *sc = nullptr;
    uint64_t n = 0;
    size_t est = 0;
    JobDev J{};                       // the whole request as one job (validated at submission)
    uint64_t window_ps = 0;
    uint64_t next_h = 0;              // first history not yet handed to a launch
    bool split = false;               // runs in pieces through its own buffers
    std::shared_ptr<Run> own;         // split request: singles buffer, tallies and digitizer
    int piece_status = GPET_OK;       // error of a launch that carried one of its pieces
    std::string piece_error;
    bool done = false;
    int status = GPET_OK;
    std::string error;
    gpet_result *result = nullptr;
    Clock::time_point t_submit;
};

// budget accounting shared with the release callbacks of the runs
struct Core {
    std::mutex mu;
    std::condition_variable cv;       // submissions, memory releases, stop
    std::condition_variable done_cv;  // request completions
    size_t budget = 0, in_use = 0, peak = 0;
};

// one live launch
struct Launch {
    std::shared_ptr<Run> R;
    std::vector<std::pair<Req *, int>> whole;   // requests run whole here: (request, job)
    std::vector<Req *> pieces;                  // split requests with a piece here
    std::vector<Req *> finishing;               // split requests whose last piece is here
    Clock::time_point t_open;
    uint64_t singles_guess = 0;                 // expected singles of the whole requests
    bool full = false;
    cudaEvent_t done = nullptr;
    ~Launch() {
        if (done) cudaEventDestroy(done);
    }
};

// the pipeline's streams and pinned host blocks
struct Pipe {
    cudaStream_t gpu = nullptr;       // transport launches and every digitizer, in order
    cudaStream_t up = nullptr;        // uploads, appends and read-backs (never blocked by a kernel)
    cudaStream_t fb = nullptr;        // whole-request re-runs after an overflow
    void *stage = nullptr;
    size_t stage_bytes = 64 << 10;
    void *zeros = nullptr;
    size_t zeros_bytes = 8 << 20;
};

constexpr double kGuessPerDecay = 0.6;   // first guess of singles per history (as the plain runs)

}  // namespace

struct gpet_server {
    std::shared_ptr<Core> core;
    gpet_options opt{};
    int max_jobs = 256;
    double max_launch_ms = 20.0;
    uint64_t piece = 4000000;
    uint64_t launch_singles = 0;      // singles one launch's buffer holds
    int64_t launch_crystals = 0;      // tally crystals one launch holds
    std::deque<Req *> queue;         // requests with histories not yet handed to a launch
    std::map<uint64_t, Req *> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread pipeline;
    gpet_server_stats stats{};
    int device = 0;
};

namespace {

// charge `bytes` of the budget to run R until its memory is released
void charge(gpet_server *S, Run &R, size_t bytes) {
    Core &C = *S->core;
    {
        std::lock_guard<std::mutex> lk(C.mu);
        C.in_use += bytes;
        C.peak = std::max(C.peak, C.in_use);
    }
    std::weak_ptr<Core> wc = S->core;
    R.on_release = [wc, bytes]() {
        if (auto c = wc.lock()) {
            std::lock_guard<std::mutex> l2(c->mu);
            c->in_use -= bytes;
            c->cv.notify_all();
        }
    };
}

bool budget_allows(gpet_server *S, size_t bytes) {
    Core &C = *S->core;
    std::lock_guard<std::mutex> lk(C.mu);
    return C.in_use + bytes <= C.budget || C.in_use == 0;
}

// hand a finished request its result (or error); caller does not hold the lock
void publish(gpet_server *S, Req *r, int st, const std::string &err, std::shared_ptr<Run> run, int job) {
    Core &C = *S->core;
    // the request's own run is let go outside the lock: its release callback takes it
    std::shared_ptr<Run> drop = std::move(r->own);
    gpet_result *res = nullptr;
    if (st == GPET_OK) {
        res = new (std::nothrow) gpet_result();
        if (res) {
            res->run = std::move(run);
            res->job = job;
            fill_counts(*res->run, job, r->n, r->sc->n_crystals, &res->counts);
            res->counts.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
        }
    }
    std::lock_guard<std::mutex> lk(C.mu);
    r->status = st;
    if (st == GPET_OK && !res) {
        r->status = GPET_ERR_OOM;
        r->error = "host allocation of a result failed";
    } else if (st != GPET_OK) {
        r->error = err;
    }
    r->result = res;
    r->done = true;
    S->stats.completed++;
    S->stats.pairs_completed += r->n;
    C.done_cv.notify_all();
}

// the whole request in a fixed launch of its own (after an overflow of a live one)
int run_whole(gpet_server *S, Pipe &P, Req *r, std::shared_ptr<Run> &out) {
    auto R = std::make_shared<Run>();
    gpet_options o = S->opt;
    o.stream = P.fb;
    int st = run_default_cfg(*R, &o, r->sc);
    if (st != GPET_OK) return st;
    R->jobs = {r->J};
    R->geoms = {r->sc->g};
    R->geom_pose = {r->sc->pose_dev};
    R->job_crystals = {r->sc->n_crystals};
    R->windows = {r->window_ps};
    R->caps.singles = std::max<uint64_t>(65536, (uint64_t)(r->n * kGuessPerDecay));
    R->caps.ovf = std::max<uint64_t>(4096, r->n / 256);
    st = run_with_retry(*R);
    if (st != GPET_OK) return st;
    charge(S, *R, R->arena_bytes);
    out = R;
    return GPET_OK;
}

// a split request's own run: singles buffer and tallies that its pieces fill
int make_own(gpet_server *S, Pipe &P, Req *r) {
    auto M = std::make_shared<Run>();
    gpet_options o = S->opt;
    o.stream = P.gpu;
    int st = run_default_cfg(*M, &o, r->sc);
    if (st != GPET_OK) return st;
    M->jobs = {r->J};
    M->geoms = {r->sc->g};
    M->geom_pose = {r->sc->pose_dev};
    M->job_crystals = {r->sc->n_crystals};
    M->windows = {r->window_ps};
    M->caps.singles = std::max<uint64_t>(65536, (uint64_t)(r->n * kGuessPerDecay));
    M->caps.ovf = 1;
    M->digitize_only = true;
    M->upload_stream = P.up;
    M->zeros = P.zeros;
    M->zeros_bytes = P.zeros_bytes;
    st = run_plan(*M);
    if (st != GPET_OK) return st;
    charge(S, *M, M->arena_bytes);
    r->own = M;
    return GPET_OK;
}

// arena bytes of one live launch of this server
size_t launch_bytes(gpet_server *S) {
    return run_footprint((uint64_t)(S->launch_singles / kGuessPerDecay), S->launch_crystals, S->max_jobs, 64, false);
}

// Start a live launch with `J` as its first job; returns null on an error
// (reported to the request by the caller).
std::unique_ptr<Launch> open_launch(gpet_server *S, Pipe &P, const JobDev &J, const gpet_scanner *sc,
                                    uint64_t window_ps, int64_t crystals, int &st) {
    auto L = std::make_unique<Launch>();
    L->R = std::make_shared<Run>();
    Run &R = *L->R;
    gpet_options o = S->opt;
    o.stream = P.gpu;
    st = run_default_cfg(R, &o, sc);
    if (st != GPET_OK) return nullptr;
    R.live = true;
    R.live_cap.jobs = S->max_jobs;
    R.live_cap.geoms = 64;
    R.live_cap.crystals = S->launch_crystals;
    R.live_cap.pose_floats = 64 * 16 * kMaxPanels;
    R.upload_stream = P.up;
    R.stage = P.stage;
    R.stage_bytes = P.stage_bytes;
    R.jobs = {J};
    R.geoms = {sc->g};
    R.geom_pose = {sc->pose_dev};
    R.geom_keys = {gpet_geometry_key(sc)};
    R.job_crystals = {crystals};
    R.windows = {window_ps};
    R.caps.singles = S->launch_singles;
    R.caps.guess = false;
    R.caps.ovf = std::max<uint64_t>(4096, S->launch_singles / 64);
    st = run_plan(R);
    if (st == GPET_OK) st = run_enqueue_transport(R);
    if (st != GPET_OK) return nullptr;
    charge(S, R, R.arena_bytes);
    L->t_open = Clock::now();
    return L;
}

// Hand one pass of queued work to the open launch (opening one when none is):
// a whole request, or the next piece of a split one.  Returns false when the
// request must wait (budget, a full launch).
bool admit(gpet_server *S, Pipe &P, std::unique_ptr<Launch> &L, Req *r, bool pieces_ok) {
    JobDev J = r->J;
    int64_t crystals = r->sc->n_crystals;
    uint64_t guess = 0;
    if (!r->split) {
        guess = std::max<uint64_t>(64, (uint64_t)(r->n * kGuessPerDecay));
        if (L && L->singles_guess + guess > S->launch_singles) {
            L->full = true;
            return false;
        }
    } else {
        if (!pieces_ok) return false;
        if (!r->own) {
            // Its own buffers leave room for one launch arena (charged already
            // when a launch is open): pieces progress only through launches,
            // so buffers that took the whole budget would wait forever.
            const size_t need = run_footprint(r->n, r->sc->n_crystals, 1, 1, false);
            const size_t arena = launch_bytes(S);
            const size_t open_arena = L ? std::min(L->R->arena_bytes, arena) : 0;
            if (!budget_allows(S, need + arena - open_arena)) return false;
            const int st = make_own(S, P, r);
            if (st != GPET_OK) {
                std::lock_guard<std::mutex> lk(S->core->mu);
                r->next_h = r->n;  // nothing more of it runs
                r->piece_status = st;
                r->piece_error = gpet_last_error();
                return true;
            }
        }
        const uint64_t h1 = std::min(r->n, r->next_h + S->piece);
        J.h_base = r->next_h;
        J.n_hist = h1 - r->next_h;
        Run &M = *r->own;
        J.s_raw = M.O.s_raw;
        J.n_singles = &M.d_hdr->n_singles;
        J.s_cap = M.O.s_cap;
        J.s_keys = M.O.s_keys;
        J.tally_count = M.d_tally_count;
        J.tally_efx = M.d_tally_efx;
        crystals = 0;
    }
    int job = 0;
    if (!L) {
        if (!budget_allows(S, launch_bytes(S))) return false;
        int st = GPET_OK;
        L = open_launch(S, P, J, r->sc, r->window_ps, crystals, st);
        if (!L) {
            std::lock_guard<std::mutex> lk(S->core->mu);
            r->piece_status = st;
            r->piece_error = gpet_last_error();
            r->next_h = r->n;
            return true;
        }
    } else {
        const int st = run_live_append(*L->R, J, r->sc, r->window_ps);
        if (st == GPET_ERR_BUSY) {
            L->full = true;
            return false;
        }
        if (st != GPET_OK) {
            std::lock_guard<std::mutex> lk(S->core->mu);
            r->piece_status = st;
            r->piece_error = gpet_last_error();
            r->next_h = r->n;
            return true;
        }
        job = (int)L->R->jobs.size() - 1;
        std::lock_guard<std::mutex> lk(S->core->mu);
        S->stats.live_appends++;
    }
    if (!r->split) {
        L->whole.push_back({r, job});
        L->singles_guess += guess;
        r->next_h = r->n;
    } else {
        r->next_h += J.n_hist;
        L->pieces.push_back(r);
        if (r->next_h == r->n) L->finishing.push_back(r);
        std::lock_guard<std::mutex> lk(S->core->mu);
        S->stats.pieces++;
    }
    return true;
}

// no more appends: digitizers of the launch and of the split requests it
// finishes go behind its transport, then an event marks the end
int close_launch(gpet_server *S, Launch &L) {
    Run &R = *L.R;
    int st = run_live_close(R);
    if (st == GPET_OK) st = run_enqueue_digitizer(R);
    for (Req *r : L.finishing)
        if (r->own && r->piece_status == GPET_OK && run_enqueue_digitizer(*r->own) != GPET_OK) {
            r->piece_status = GPET_ERR_CUDA;
            r->piece_error = gpet_last_error();
        }
    cudaError_t e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(L.done, R.stream);
    if (e != cudaSuccess) {
        // no end marker: wait for the launch here, so that its results are not read early
        if (L.done) { cudaEventDestroy(L.done); L.done = nullptr; }
        cudaStreamSynchronize(R.stream);
        if (st == GPET_OK) st = gpet_cuda_fail(e, "launch end event");
    }
    std::lock_guard<std::mutex> lk(S->core->mu);
    S->stats.launches++;
    S->stats.max_jobs_per_launch = std::max<uint64_t>(S->stats.max_jobs_per_launch, R.jobs.size());
    return st;
}

// Results of a launch whose work (and that of the digitizers behind it) is
// done.  Requests that met a full buffer go to `rerun`: they run again, whole
// and with exact sizes, once no launch is on the GPU.  The compact copies of
// the results go on st_copy, called with no live launch on the GPU.
void finish_launch(gpet_server *S, Launch &L, int close_status, const std::string &close_error,
                   std::vector<Req *> &rerun, cudaStream_t st_copy) {
    int st = close_status;
    std::string err = close_error;
    if (st == GPET_OK) {
        st = run_collect(*L.R);
        if (st != GPET_OK) err = gpet_last_error();
    }
    {
        std::lock_guard<std::mutex> lk(S->core->mu);
        S->stats.transport_ms += std::max(0.f, L.R->transport_ms);
        S->stats.digitizer_ms += std::max(0.f, L.R->digitizer_ms);
    }
    // the results move to memory of their own size, and the launch's buffers
    // go back at once (results a client keeps then hold only what they are).
    // The copy is made whatever the budget's state: results left viewing the
    // launch's buffers would keep the whole arena charged, and a client that
    // holds them could then keep every later launch from opening.
    std::shared_ptr<Run> views = L.R;
    if (st == GPET_OK && !L.whole.empty()) {
        int cst = GPET_OK;
        std::shared_ptr<Run> compact = run_compact(*L.R, st_copy, &cst);
        if (compact) {
            charge(S, *compact, compact->arena_bytes);
            views = compact;
        }
    }
    // only the launch's own singles buffer was too small: pieces (which write
    // to their requests' buffers) are complete
    const RunHeader &H = L.R->h_hdr;
    const bool shared_only = st == GPET_ERR_OVERFLOW && H.n_ovf <= L.R->O.ovf_cap && !(H.status & kStatusOverflow);
    for (auto &w : L.whole) {
        Req *r = w.first;
        if (st == GPET_OK) publish(S, r, GPET_OK, "", views, w.second);
        else if (st == GPET_ERR_OVERFLOW) rerun.push_back(r);
        else publish(S, r, st, err, nullptr, 0);
    }
    if (st != GPET_OK && !shared_only)
        for (Req *r : L.pieces)
            if (r->piece_status == GPET_OK) {
                r->piece_status = st;
                r->piece_error = err;
            }
    for (Req *r : L.finishing) {
        int s2 = r->piece_status;
        std::string e2 = r->piece_error;
        if (s2 == GPET_OK && r->own) {
            s2 = run_collect(*r->own);
            if (s2 != GPET_OK) e2 = gpet_last_error();
            std::lock_guard<std::mutex> lk(S->core->mu);
            S->stats.digitizer_ms += std::max(0.f, r->own->digitizer_ms);
        }
        if (s2 == GPET_OK) {
            int cst = GPET_OK;
            std::shared_ptr<Run> own = run_compact(*r->own, st_copy, &cst);
            if (own) charge(S, *own, own->arena_bytes);
            else own = r->own;
            publish(S, r, GPET_OK, "", own, 0);
        } else if (s2 == GPET_ERR_OVERFLOW) {
            r->own.reset();
            rerun.push_back(r);
        } else {
            publish(S, r, s2, e2, nullptr, 0);
        }
    }
    views.reset();
    L.R.reset();  // views of the launch itself (no compact copy) keep its memory; the pipeline does not
}

void pipeline_main(gpet_server *S) {
    cudaSetDevice(S->device);
    Pipe P;
    cudaStreamCreateWithFlags(&P.gpu, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&P.up, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&P.fb, cudaStreamNonBlocking);
    if (cudaMallocHost(&P.stage, P.stage_bytes) != cudaSuccess) P.stage = nullptr;
    if (cudaMallocHost(&P.zeros, P.zeros_bytes) != cudaSuccess) P.zeros = nullptr;
    if (P.zeros) std::memset(P.zeros, 0, P.zeros_bytes);
    Core &C = *S->core;
    std::unique_ptr<Launch> open;
    std::deque<std::pair<std::unique_ptr<Launch>, std::pair<int, std::string>>> inflight;
    // histories published to the open launch and not yet claimed by its kernel
    const uint64_t backlog_target = 4 * S->piece;
    std::vector<Req *> rerun;
    for (;;) {
        // 1. launches whose work is done, in order
        while (!inflight.empty() && cudaEventQuery(inflight.front().first->done) != cudaErrorNotReady) {
            cudaGetLastError();
            finish_launch(S, *inflight.front().first, inflight.front().second.first, inflight.front().second.second,
                          rerun, P.gpu);
            inflight.pop_front();
        }
        // requests that met a full buffer run again alone, with exact sizes, on
        // an idle GPU (a live launch would hold every SM while they wait)
        if (!rerun.empty()) {
            if (open) {
                const int st = close_launch(S, *open);
                std::string err = st == GPET_OK ? std::string() : std::string(gpet_last_error());
                inflight.emplace_back(std::move(open), std::make_pair(st, std::move(err)));
                open.reset();
            }
            if (inflight.empty()) {
                for (Req *r : rerun) {
                    std::shared_ptr<Run> R;
                    const int s2 = run_whole(S, P, r, R);
                    publish(S, r, s2, s2 == GPET_OK ? "" : std::string(gpet_last_error()), R, 0);
                }
                rerun.clear();
            } else {
                std::unique_lock<std::mutex> lk(C.mu);
                C.cv.wait_for(lk, std::chrono::microseconds(100));
            }
            continue;
        }
        std::vector<Req *> work;
        {
            std::unique_lock<std::mutex> lk(C.mu);
            if (S->stop && S->queue.empty() && !open && inflight.empty()) break;
            if (S->queue.empty() && !open && inflight.empty()) {
                C.cv.wait(lk);
                continue;
            }
            if (!S->queue.empty() && !open && !inflight.empty()) {
                // The next live launch opens only once the last one has been
                // collected: its results are compacted by device-to-device
                // copies, which may run on the SMs, and a live kernel holds
                // every SM while it waits on this thread.
                lk.unlock();
                cudaEventSynchronize(inflight.front().first->done);
                continue;
            }
            work.assign(S->queue.begin(), S->queue.end());
            S->queue.clear();
        }
        // 2. one pass over the queue: whole requests, and one piece of each split one.
        //    Requests without a phantom go first, those with one after (each in
        //    arrival order): a CTA runs one event type at a time, and its warps
        //    then hold histories of one kind, not phantom steps beside flights.
        //    Only while two more launch arenas fit the budget: a client that
        //    takes results in submission order holds the later ones, and once
        //    the budget runs short the request it waits for must come first.
        //    The results of the launch still finishing take at most one arena,
        //    so the next launch can still open, and takes the oldest request.
        const size_t arena = launch_bytes(S);
        bool reorder = false;
        {
            std::lock_guard<std::mutex> lk(C.mu);
            reorder = C.in_use + 2 * arena <= C.budget;
        }
        if (reorder)
            std::stable_partition(work.begin(), work.end(), [](const Req *r) { return !r->J.has_phantom; });
        else  // arrival order again: ids rise with submission
            std::sort(work.begin(), work.end(), [](const Req *a, const Req *b) { return a->id < b->id; });
        bool pieces_ok = true;
        if (open && std::any_of(work.begin(), work.end(), [](Req *r) { return r->split; })) {
            uint64_t taken = 0;
            if (run_live_taken(*open->R, &taken) == GPET_OK)
                pieces_ok = (open->R->live_tail - std::min(taken, open->R->live_tail)) * open->R->chunk_size <
                            backlog_target;
        }
        std::vector<Req *> keep;
        const Launch *opened_before = open.get();
        const size_t jobs_before = open ? open->R->jobs.size() : 0;
        for (Req *r : work) {
            if (!P.stage || !P.zeros) {
                std::lock_guard<std::mutex> lk(C.mu);
                r->piece_status = GPET_ERR_OOM;
                r->piece_error = "pinned host staging of the serving loop could not be allocated";
                r->next_h = r->n;
            } else if (!(open && open->full)) {
                admit(S, P, open, r, pieces_ok);
            }
            if (r->next_h < r->n) {
                keep.push_back(r);
            } else if (r->piece_status != GPET_OK) {
                // A failed request is answered once every launch holding a
                // piece of it has finished (kernels may still write its
                // buffers): with the latest launch, as launches end in order.
                if (r->split && r->own && open) open->finishing.push_back(r);
                else if (r->split && r->own && !inflight.empty()) inflight.back().first->finishing.push_back(r);
                else publish(S, r, r->piece_status, r->piece_error, nullptr, 0);
            }
        }
        {
            std::lock_guard<std::mutex> lk(C.mu);
            S->queue.insert(S->queue.begin(), keep.begin(), keep.end());  // ahead of later arrivals
        }
        // 3. close the open launch: old enough, full, or out of published work
        //    with nothing more to take now (an empty queue, or requests that
        //    wait for memory)
        const bool appended = open && (open.get() != opened_before || open->R->jobs.size() > jobs_before);
        if (open) {
            bool close = open->full ||
                         std::chrono::duration<double, std::milli>(Clock::now() - open->t_open).count() >=
                             S->max_launch_ms;
            if (!close && (keep.empty() || !appended)) {
                uint64_t taken = 0;
                close = run_live_taken(*open->R, &taken) != GPET_OK || taken >= open->R->live_tail;
            }
            if (close) {
                const int st = close_launch(S, *open);
                std::string err = st == GPET_OK ? std::string() : std::string(gpet_last_error());
                inflight.emplace_back(std::move(open), std::make_pair(st, std::move(err)));
                open.reset();
            }
        }
        // 4. a short wait: arrivals wake it; launch progress and ends are polled
        std::unique_lock<std::mutex> lk(C.mu);
        C.cv.wait_for(lk, std::chrono::microseconds(100));
    }
    cudaStreamSynchronize(P.gpu);
    cudaStreamSynchronize(P.fb);
    cudaStreamDestroy(P.gpu);
    cudaStreamDestroy(P.up);
    cudaStreamDestroy(P.fb);
    if (P.stage) cudaFreeHost(P.stage);
    if (P.zeros) cudaFreeHost(P.zeros);
}

}  // namespace

extern "C" int gpet_server_create(const gpet_server_config *cfg, gpet_server **out) {
    if (!cfg || !out) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    if (cfg->hbm_budget_bytes == 0) return gpet_fail(GPET_ERR_INVALID_ARG, "hbm_budget_bytes must be > 0");
    if (cfg->workers < 0 || cfg->workers > 8) return gpet_fail(GPET_ERR_INVALID_ARG, "workers must be in [0, 8]");
    if (cfg->max_jobs_per_launch < 0 || cfg->max_jobs_per_launch > 4095)
        return gpet_fail(GPET_ERR_INVALID_ARG, "max_jobs_per_launch must be in [0, 4095]");
    if (!(cfg->max_launch_ms >= 0.0) || !(cfg->max_launch_ms <= 1.0e4))
        return gpet_fail(GPET_ERR_INVALID_ARG, "max_launch_ms must be in [0, 1e4]");
    gpet_server *S = new (std::nothrow) gpet_server();
    if (!S) return gpet_fail(GPET_ERR_OOM, "host allocation of the server failed");
    S->core = std::make_shared<Core>();
    S->core->budget = cfg->hbm_budget_bytes;
    S->opt = cfg->launch;
    S->opt.stream = nullptr;
    S->opt.keep_hits = 0;
    S->opt.h_begin = S->opt.h_end = 0;
    S->max_jobs = cfg->max_jobs_per_launch > 0 ? cfg->max_jobs_per_launch : 256;
    S->max_launch_ms = cfg->max_launch_ms > 0.0 ? cfg->max_launch_ms : 20.0;
    // One launch's arena takes at most a quarter of the budget (the open launch,
    // the one finishing and split requests' buffers share it), and at most
    // 2^26 singles (7.9 GB); a piece's first guess of singles fits half of it.
    const size_t per_single = sizeof(RawSingle) + 2 * 8 + 2 * 4 + 8 + 8 + 6 * 4 + 1 + 4;
    S->launch_crystals = (int64_t)std::min<size_t>(1 << 22, std::max<size_t>(1 << 18, cfg->hbm_budget_bytes / 400));
    const size_t fixed = run_footprint(0, S->launch_crystals, S->max_jobs, 64, false);
    const size_t quarter = cfg->hbm_budget_bytes / 4;
    S->launch_singles = std::min<uint64_t>(1ull << 26, quarter > fixed ? (quarter - fixed) / per_single : 0);
    S->launch_singles = std::max<uint64_t>(S->launch_singles, 65536);
    const uint64_t piece_cap = std::max<uint64_t>(1024, (uint64_t)(S->launch_singles / kGuessPerDecay / 2));
    S->piece = std::min<uint64_t>(cfg->piece_decays > 0 ? cfg->piece_decays : 4000000, piece_cap);
    cudaError_t e = cudaGetDevice(&S->device);
    // every kernel a launch may run is loaded now: loading one later could wait
    // for a live launch, whose kernel waits for the pipeline
    if (e == cudaSuccess) e = preload_kernels();
    if (e != cudaSuccess) { delete S; return gpet_cuda_fail(e, "server set-up"); }
    S->pipeline = std::thread(pipeline_main, S);
    *out = S;
    return GPET_OK;
}

extern "C" int gpet_server_submit(gpet_server *S, gpet_scanner *sc, const gpet_source *src, const gpet_digitizer *dg,
                                  uint64_t n_decays, uint64_t seed, int32_t block, uint64_t *req_id) {
    if (!S || !sc || !src || !dg || !req_id) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    JobDev J;
    int st = gpet_make_job(sc, src, dg, n_decays, seed, J);  // validate now, not in the pipeline
    if (st != GPET_OK) return st;
    Req *r = new (std::nothrow) Req();
    if (!r) return gpet_fail(GPET_ERR_OOM, "host allocation of a request failed");
    r->sc = sc;
    r->n = n_decays;
    r->J = J;
    r->window_ps = (uint64_t)std::llround(dg->coinc_window_ns * 1000.0);
    r->split = n_decays > S->piece;
    r->est = run_footprint(n_decays, sc->n_crystals, 1, 1, false);
    Core &C = *S->core;
    std::unique_lock<std::mutex> lk(C.mu);
    if (r->est > C.budget) {
        const size_t est = r->est;
        delete r;
        return gpet_fail(GPET_ERR_OOM, "request needs ~%zu device bytes, more than the whole budget", est);
    }
    if (r->split && r->est + launch_bytes(S) > C.budget) {
        // its buffers and one launch arena, which runs its pieces, must fit together
        const size_t est = r->est, arena = launch_bytes(S);
        delete r;
        return gpet_fail(GPET_ERR_OOM, "request needs ~%zu device bytes and a launch arena of %zu, more than the budget",
                         est, arena);
    }
    if (S->stop) {
        delete r;
        return gpet_fail(GPET_ERR_INVALID_ARG, "server is shutting down");
    }
    if (!block) {
        size_t queued = 0;
        for (Req *q : S->queue) queued += q->est;
        if (C.in_use + queued + r->est > C.budget) {
            delete r;
            S->stats.rejected++;
            return gpet_fail(GPET_ERR_BUSY, "HBM budget full (in use %zu + queued %zu of %zu bytes)", C.in_use, queued,
                             C.budget);
        }
    }
    r->id = S->next_id++;
    r->t_submit = Clock::now();
    S->reqs[r->id] = r;
    S->queue.push_back(r);
    S->stats.submitted++;
    *req_id = r->id;
    C.cv.notify_all();
    return GPET_OK;
}

static int take_result(gpet_server *S, std::map<uint64_t, Req *>::iterator it, gpet_result **out) {
    Req *r = it->second;
    S->reqs.erase(it);
    const int st = r->status;
    if (st == GPET_OK) *out = r->result;
    else gpet_fail(st, "%s", r->error.c_str());
    delete r;
    return st;
}

extern "C" int gpet_server_poll(gpet_server *S, uint64_t req_id, gpet_result **out) {
    if (!S || !out) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    std::lock_guard<std::mutex> lk(S->core->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return gpet_fail(GPET_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)req_id);
    if (!it->second->done) return GPET_OK;
    return take_result(S, it, out);
}

extern "C" int gpet_server_wait(gpet_server *S, uint64_t req_id, gpet_result **out) {
    if (!S || !out) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(S->core->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return gpet_fail(GPET_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)req_id);
    // Re-find the request after every wake-up: another caller polling or
    // waiting on the same id may have taken (and freed) it meanwhile.
    S->core->done_cv.wait(lk, [&] {
        it = S->reqs.find(req_id);
        return it == S->reqs.end() || it->second->done;
    });
    if (it == S->reqs.end())
        return gpet_fail(GPET_ERR_INVALID_ARG, "request %llu was taken by another caller", (unsigned long long)req_id);
    return take_result(S, it, out);
}

extern "C" int gpet_server_stats_get(gpet_server *S, gpet_server_stats *out) {
    if (!S || !out) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->core->mu);
    *out = S->stats;
    out->bytes_in_use = S->core->in_use;
    out->peak_bytes = S->core->peak;
    out->queued = S->queue.size();
    return GPET_OK;
}

extern "C" void gpet_server_destroy(gpet_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->core->mu);
        S->stop = true;
        S->core->cv.notify_all();
    }
    if (S->pipeline.joinable()) S->pipeline.join();
    for (auto &kv : S->reqs) {
        if (kv.second->result) gpet_result_free(kv.second->result);
        delete kv.second;
    }
    delete S;
}
