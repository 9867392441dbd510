// sensitivity.cu -- NEMA NU4-style sensitivity map S(r, E) (Sec. 2.4): point
// sources at many positions, for one or more scanner designs, in one batched
// launch, with the coincidences of several energy windows counted in one pass
// over the time-sorted singles; and the symmetric percent difference of two
// designs' sensitivities.
//
// Why one pass suffices: a window only removes singles.  A cluster -- a
// maximal run of one job's time-sorted singles whose consecutive gaps are at
// most the coincidence window -- can therefore only split when singles are
// removed, never grow into its neighbour (the gap to the neighbour is already
// wider than the window and removing singles only widens it).  The thread at
// the start of each cluster of the widest window replays the coincidence
// policy (earliest unconsumed single opens [t, t + window]; exactly two
// singles in different panels count; everything in the window is consumed)
// on the cluster's singles inside each energy window in turn.  The blurred
// energies and the window edges are the same FP32 values a run with that
// window alone compares, so the counts equal those runs' counts exactly.
#include <cmath>
#include <vector>

#include "host.h"

namespace gpet {

namespace {

constexpr int kWinThreads = 256;
constexpr int kWinTile = kWinThreads * 8;  // singles per block
constexpr int kWinLocalJobs = 32;          // jobs a block counts in shared memory

__global__ void __launch_bounds__(kWinThreads) k_coinc_windows(SinglesDev s, const uint64_t *__restrict__ window_ps,
                                                               WinDev win, unsigned long long *counts) {
    __shared__ unsigned int cnt[kWinLocalJobs * kMaxWindows];
    const unsigned long long n = *s.n;
    const unsigned long long first = (unsigned long long)blockIdx.x * kWinTile;
    if (first >= n) return;
    const unsigned long long last = (first + kWinTile < n ? first + kWinTile : n) - 1;
    const int nw = win.n;
    // singles are ordered by job: the block's jobs are [j0, j1]
    const int j0 = s.job[first], j1 = s.job[last];
    const bool local = j1 - j0 < kWinLocalJobs;
    for (int i = threadIdx.x; i < kWinLocalJobs * nw; i += kWinThreads) cnt[i] = 0u;
    __syncthreads();
    for (unsigned long long i = first + threadIdx.x; i <= last; i += kWinThreads) {
        const int ji = s.job[i];
        const uint64_t ti = s.t[i];
        const uint64_t W = window_ps[ji];
        if (!(i == 0 || s.job[i - 1] != ji || ti - s.t[i - 1] > W)) continue;
        // end of this cluster of the widest window
        unsigned long long e = i;
        while (e + 1 < n && s.job[e + 1] == ji && s.t[e + 1] - s.t[e] <= W) ++e;
        for (int w = 0; w < nw; ++w) {
            const float lo = win.lo[w], hi = win.hi[w];
            unsigned int c = 0;
            unsigned long long k = i;
            while (k <= e && !(s.e[k] >= lo && s.e[k] <= hi)) ++k;
            while (k <= e) {
                const unsigned long long a = k;
                const uint64_t ta = s.t[a];
                unsigned long long second = a;
                int in_window = 1;
                for (k = a + 1; k <= e && s.t[k] - ta <= W; ++k) {
                    if (s.e[k] >= lo && s.e[k] <= hi) {
                        if (++in_window == 2) second = k;
                    }
                }
                if (in_window == 2 && s.panel[a] != s.panel[second]) ++c;
                while (k <= e && !(s.e[k] >= lo && s.e[k] <= hi)) ++k;
            }
            if (c) {
                if (local) atomicAdd(&cnt[(ji - j0) * nw + w], c);
                else atomicAdd(counts + (unsigned long long)ji * nw + w, (unsigned long long)c);
            }
        }
    }
    if (!local) return;
    __syncthreads();
    const int m = (j1 - j0 + 1) * nw;
    for (int i = threadIdx.x; i < m; i += kWinThreads)
        if (cnt[i]) atomicAdd(counts + (unsigned long long)j0 * nw + i, (unsigned long long)cnt[i]);
}

}  // namespace

cudaError_t launch_coinc_windows(const SinglesDev &s, const CoincDev &C, const WinDev &win,
                                 unsigned long long *counts, unsigned long long cap, cudaStream_t st) {
    const unsigned long long blocks = (cap + kWinTile - 1) / kWinTile;
    k_coinc_windows<<<(unsigned int)(blocks ? blocks : 1), kWinThreads, 0, st>>>(s, C.window_ps, win, counts);
    return cudaGetLastError();
}

// load the window-count kernel (internal.h)
cudaError_t preload_window_kernels() {
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, k_coinc_windows);
}

}  // namespace gpet

using namespace gpet;

extern "C" int gpet_sensitivity_map(int32_t n_scanners, gpet_scanner *const *scanners, int32_t n_positions,
                                    const double *positions_mm, double activity_bq, const gpet_digitizer *digitizer,
                                    int32_t n_windows, const double *windows_kev, uint64_t n_decays, uint64_t seed,
                                    const gpet_options *opt, uint64_t *counts, double *sens, gpet_counts *total) {
    if (n_scanners < 1 || !scanners || n_positions < 1 || !positions_mm || !digitizer || !windows_kev || !counts)
        return gpet_fail(GPET_ERR_INVALID_ARG, "sensitivity map needs scanners, positions, windows and counts");
    if (n_windows < 1 || n_windows > kMaxWindows)
        return gpet_fail(GPET_ERR_INVALID_ARG, "n_windows=%d outside [1, %d]", n_windows, kMaxWindows);
    if ((int64_t)n_scanners * n_positions > 4095)
        return gpet_fail(GPET_ERR_INVALID_ARG, "%d scanners x %d positions exceed 4095 jobs", n_scanners,
                         n_positions);
    double lo_u = 0.0, hi_u = 0.0;
    for (int w = 0; w < n_windows; ++w) {
        const double lo = windows_kev[2 * w], hi = windows_kev[2 * w + 1];
        if (!(lo >= 0.0) || !(hi >= lo) || !std::isfinite(hi))
            return gpet_fail(GPET_ERR_INVALID_ARG, "window %d = [%g, %g] keV: need 0 <= lo <= hi", w, lo, hi);
        lo_u = w == 0 ? lo : std::min(lo_u, lo);
        hi_u = w == 0 ? hi : std::max(hi_u, hi);
    }
    for (int p = 0; p < 3 * n_positions; ++p)
        if (!std::isfinite(positions_mm[p])) return gpet_fail(GPET_ERR_INVALID_ARG, "position %d not finite", p / 3);
    const int nj = n_scanners * n_positions;
    std::vector<gpet_scanner *> scs((size_t)nj);
    std::vector<gpet_source> srcs((size_t)nj);
    std::vector<gpet_digitizer> dgs((size_t)nj, *digitizer);
    std::vector<uint64_t> nds((size_t)nj, n_decays), seeds((size_t)nj);
    for (int i = 0; i < n_scanners; ++i)
        for (int p = 0; p < n_positions; ++p) {
            const int j = i * n_positions + p;
            scs[j] = scanners[i];
            gpet_source &S = srcs[j];
            S = gpet_source{};
            S.kind = GPET_SOURCE_POINT;
            for (int a = 0; a < 3; ++a) S.pos_mm[a] = positions_mm[3 * p + a];
            S.dir[2] = 1.0;
            S.activity_bq = activity_bq;
            dgs[j].e_lo_kev = lo_u;
            dgs[j].e_hi_kev = hi_u;
            seeds[j] = seed + (uint64_t)p;
        }
    Run R;
    int st = gpet_batch_build_run(R, nj, scs.data(), srcs.data(), dgs.data(), nds.data(), seeds.data(), opt);
    if (st != GPET_OK) return st;
    // a wide union window keeps more singles than the default guess of 0.6 per
    // pair: size for one per pair so that the first run fits
    R.caps.singles = std::max<uint64_t>(R.caps.singles, n_decays * (uint64_t)nj + 65536);
    for (int w = 0; w < n_windows; ++w) {
        // the same FP32 edges a run with this window alone compares against
        R.win_lo.push_back((float)windows_kev[2 * w]);
        R.win_hi.push_back((float)windows_kev[2 * w + 1]);
    }
    st = run_with_retry(R);
    if (st != GPET_OK) return st;
    const size_t m = (size_t)nj * n_windows;
    if (R.win_counts.size() != m) return gpet_fail(GPET_ERR_CUDA, "window counts missing after the run");
    for (size_t i = 0; i < m; ++i) {
        counts[i] = R.win_counts[i];
        if (sens) sens[i] = n_decays ? (double)R.win_counts[i] / (double)n_decays : 0.0;
    }
    if (total) {
        int64_t crystals = 0;
        for (int64_t c : R.job_crystals) crystals += c;
        fill_counts(R, 0, n_decays * (uint64_t)nj, crystals, total);
        total->singles = R.h_hdr.n_sorted;
        total->coincidences = R.h_hdr.n_coinc;
        total->hits = R.h_hdr.counters[5];
    }
    return GPET_OK;
}

extern "C" int gpet_delta_sym(int64_t n, const double *s_a, const double *s_b, double *out) {
    if (n < 0 || (n > 0 && (!s_a || !s_b || !out))) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL array or n < 0");
    for (int64_t i = 0; i < n; ++i) {
        const double a = s_a[i], b = s_b[i], t = a + b;
        out[i] = t != 0.0 ? 200.0 * (a - b) / t : NAN;
    }
    return GPET_OK;
}
