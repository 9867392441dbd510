// sort.cu -- digitizer back end: LSD radix sort of singles by 64-bit time key,
// gather into time order, coincidence sorting (Sec. 2.3 timing window).
//
// Keys are (job << shift) | t_ps, with the job in the fewest high bits that
// number the launch's jobs (none for one job), so a batch of jobs sorts as
// independent segments and a single run sorts on the whole 64-bit time.  The
// transport writes them beside the records.  The
// sort is a least-significant-digit radix sort with 8-bit
// digits: one fused pass builds the eight digit histograms, a plan kernel
// drops the passes whose digit is the same for every key (high time bytes,
// unused job bits), and in the simulation path every remaining pass is one
// kernel (k_onesweep: tiles claimed in order, each tile's digit offsets from
// the global histogram and a decoupled look-back over the tiles before it).
// The allocation-free sort runs each pass as tile histogram -> per-digit scan
// -> stable scatter.  Stable ranks inside a tile come from the lanes of
// a warp with the same digit (the intersection of bit-plane ballots), in input
// order.  In the simulation path the scatter's input tiles are streamed into
// shared memory by the bulk-copy engine (cp.async.bulk completing on an
// mbarrier), one tile ahead of the tile being ranked.  The element count is
// read on the device, so the whole chain is enqueued without a host round
// trip.
#include "internal.h"

namespace gpet {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kTile = kSortThreads * kSortItems;  // 4096 keys per tile
constexpr int kPasses = 8;
static_assert(kSortThreads == 256, "one thread per 8-bit digit in the scatter's prefix step");

__device__ __forceinline__ uint32_t lane_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long sort_n(const SortDev &S) {
    const unsigned long long n = *S.n_in;
    return n < S.cap ? n : S.cap;
}

// Values (the identity permutation) and the eight digit histograms of the
// keys (smem, then global atomics).  The keys themselves were written by the
// transport's finish event, next to each single's record.
__global__ void __launch_bounds__(kSortThreads) k_make_keys(SortDev S) {
    __shared__ uint32_t h[kPasses][256];
    for (int i = threadIdx.x; i < kPasses * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const unsigned long long n = sort_n(S);
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint64_t key = __ldg(S.keys[0] + i);
        S.vals[0][i] = (uint32_t)i;
#pragma unroll
        for (int p = 0; p < kPasses; ++p) atomicAdd(&h[p][(key >> (8 * p)) & 0xFF], 1u);
    }
    // the first active pass's look-back words (each pass clears the next one's)
    if (S.lb[0]) {
        const unsigned long long words = (n + kTile - 1) / kTile * 256;
        for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < words;
             i += (unsigned long long)gridDim.x * blockDim.x)
            S.lb[0][i] = 0ull;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kPasses * 256; i += blockDim.x) {
        const uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(S.ghist + i, v);
    }
}

// which passes run, and which buffer each one reads (one warp per pass)
__global__ void __launch_bounds__(kPasses * 32) k_plan(SortDev S) {
    __shared__ int active[kPasses];
    const int p = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long n = sort_n(S);
    uint32_t mx = 0;
    for (int d = lane; d < 256; d += 32) mx = max(mx, S.ghist[p * 256 + d]);
    mx = __reduce_max_sync(kFullMask, mx);
    if (lane == 0) active[p] = (n > 1 && (unsigned long long)mx < n) ? 1 : 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        int cur = 0;
        for (int q = 0; q < kPasses; ++q) {
            S.plan[q] = active[q];
            S.plan[kPasses + q] = cur;
            if (active[q]) cur ^= 1;
        }
        S.plan[2 * kPasses] = cur;  // buffer holding the sorted result
    }
}

__global__ void __launch_bounds__(kSortThreads) k_tile_hist(SortDev S, int p) {
    if (!S.plan[p]) return;
    const int src = S.plan[kPasses + p];
    const unsigned long long n = sort_n(S);
    const unsigned long long tiles = (n + kTile - 1) / kTile;
    __shared__ uint32_t h[256];
    const uint64_t *keys = src ? S.keys[1] : S.keys[0];
    for (unsigned long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
        __syncthreads();
        const unsigned long long b = t * kTile;
        // all of the tile's loads are issued before the first shared atomic
        uint64_t k[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const unsigned long long i = b + (unsigned long long)j * kSortThreads + threadIdx.x;
            k[j] = i < n ? __ldg(keys + i) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const unsigned long long i = b + (unsigned long long)j * kSortThreads + threadIdx.x;
            if (i < n) atomicAdd(&h[(k[j] >> (8 * p)) & 0xFF], 1u);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < 256; d += blockDim.x) S.tile_hist[(size_t)d * S.max_tiles + t] = h[d];
        __syncthreads();
    }
}

// block-wide exclusive scan of one value per thread (blockDim a multiple of 32, at most 1024)
__device__ __forceinline__ uint32_t block_exscan(uint32_t v, uint32_t &total, uint32_t *sw) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFullMask, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? sw[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullMask, w, o);
            if (lane >= o) w += y;
        }
        sw[lane] = w;  // inclusive warp prefix
    }
    __syncthreads();
    const uint32_t warp_base = wid ? sw[wid - 1] : 0;
    total = sw[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_base + x - v;
}

// per digit: base of the digit + exclusive scan over tiles -> scatter offsets
__global__ void __launch_bounds__(1024) k_digit_scan(SortDev S, int p) {
    if (!S.plan[p]) return;
    __shared__ uint32_t sw[32];
    const int d = blockIdx.x;
    const unsigned long long n = sort_n(S);
    const unsigned long long tiles = (n + kTile - 1) / kTile;
    uint32_t base = 0;
    for (int e = 0; e < d; ++e) base += S.ghist[p * 256 + e];
    uint32_t *row = S.tile_hist + (size_t)d * S.max_tiles;
    for (unsigned long long c = 0; c < tiles; c += blockDim.x) {
        const unsigned long long t = c + threadIdx.x;
        const uint32_t v = t < tiles ? row[t] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exscan(v, tot, sw);
        if (t < tiles) row[t] = base + ex;
        base += tot;
    }
}

// Stable scatter of one tile.  Ranks come in (warp, round, lane) order, which
// is input order.  The tile is first rebuilt in shared memory in digit order,
// then written out from there: consecutive threads write consecutive slots of
// one digit's run, so the global stores coalesce (a direct store from the
// ranking registers would send each of a warp's 32 keys to its own sector).
struct ScatterSmem {
    uint64_t keys[kTile];
    uint32_t vals[kTile];
    uint32_t wh[kSortThreads / 32][256];
    uint32_t gdelta[256];   // global run start - local run start (mod 2^32)
    uint32_t sw[32];
};
// Staged form: while a tile is ranked and written, the bulk-copy engine
// streams the CTA's next tile (keys and indices) into shared memory, so each
// CTA keeps 48 KB of reads in flight through all of its tile's work instead
// of waiting for its loads at the start of every tile.
struct ScatterStage {
    uint64_t keys[kTile];
    uint32_t vals[kTile];
    unsigned long long bar;  // mbarrier: the copy of the staged tile has landed
};
constexpr size_t kScatterSmem = sizeof(ScatterSmem);
constexpr size_t kScatterSmemStaged = sizeof(ScatterSmem) + sizeof(ScatterStage);
constexpr uint32_t kStageBytes = kTile * (sizeof(uint64_t) + sizeof(uint32_t));
static_assert(sizeof(ScatterSmem) % 16 == 0, "staging buffer must start on a 16-byte boundary");
static_assert((kTile * sizeof(uint32_t)) % 16 == 0 && (kTile * sizeof(uint64_t)) % 16 == 0,
              "bulk copies move multiples of 16 bytes");
// mbarrier waits give up after this many polls (each poll may suspend the
// thread for a bounded time); a tile copy that never lands is reported, not
// waited for forever
constexpr int kStageWaitPolls = 1 << 22;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool stage_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < kStageWaitPolls; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// one thread: expect the tile's bytes on the barrier, start both copies
__device__ __forceinline__ void stage_issue(ScatterStage &sg, const uint64_t *kin, const uint32_t *vin,
                                            unsigned long long t) {
    const uint32_t bar = smem_addr(&sg.bar);
    // the staging buffer was last read by ordinary loads; order them before
    // the copy engine's writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kStageBytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(sg.keys)), "l"(kin + t * kTile), "r"((uint32_t)(kTile * sizeof(uint64_t))), "r"(bar)
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(sg.vals)), "l"(vin + t * kTile), "r"((uint32_t)(kTile * sizeof(uint32_t))), "r"(bar)
        : "memory");
}

template <bool kStaged>
__global__ void __launch_bounds__(kSortThreads, 2) k_scatter(SortDev S, int p) {
    if (!S.plan[p]) return;
    extern __shared__ __align__(16) unsigned char scatter_raw[];
    ScatterSmem &sm = *reinterpret_cast<ScatterSmem *>(scatter_raw);
    ScatterStage &sg = *reinterpret_cast<ScatterStage *>(scatter_raw + sizeof(ScatterSmem));
    const int src = S.plan[kPasses + p];
    const unsigned long long n = sort_n(S);
    const unsigned long long tiles = (n + kTile - 1) / kTile;
    const unsigned long long full_tiles = n / kTile;  // tiles the copy engine stages
    constexpr int kWarps = kSortThreads / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // selects, not an index: a dynamic index would copy the argument to the stack
    const uint64_t *kin = src ? S.keys[1] : S.keys[0];
    const uint32_t *vin = src ? S.vals[1] : S.vals[0];
    uint64_t *kout = src ? S.keys[0] : S.keys[1];
    uint32_t *vout = src ? S.vals[0] : S.vals[1];
    uint32_t parity = 0;
    if (kStaged) {
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sg.bar)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            if (blockIdx.x < full_tiles) stage_issue(sg, kin, vin, blockIdx.x);
        }
        __syncthreads();
    }
    for (unsigned long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        for (int i = threadIdx.x; i < kWarps * 256; i += blockDim.x) (&sm.wh[0][0])[i] = 0;
        const unsigned long long wb = t * kTile + (unsigned long long)w * (32 * kSortItems);
        // this tile's global start of digit threadIdx.x, fetched with the keys
        const uint32_t gstart = S.tile_hist[(size_t)threadIdx.x * S.max_tiles + t];
        uint64_t k[kSortItems];
        uint32_t v[kSortItems];
        uint32_t rank[kSortItems];
        const bool staged = kStaged && t < full_tiles;
        if (staged) {
            // every thread sees the copy land; the CTA gives up together
            const bool ok = stage_wait(smem_addr(&sg.bar), parity);
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0) {
                    atomicOr(S.status, kStatusSortStall);
                    stage_wait(smem_addr(&sg.bar), parity);  // let the copy in flight land
                }
                return;
            }
            parity ^= 1u;
            const int lb = w * (32 * kSortItems) + lane;
#pragma unroll
            for (int j = 0; j < kSortItems; ++j) {
                k[j] = sg.keys[lb + j * 32];
                v[j] = sg.vals[lb + j * 32];
            }
            __syncthreads();  // the staging buffer is free: stream in the next tile
            const unsigned long long nt = t + gridDim.x;
            if (threadIdx.x == 0 && nt < full_tiles) stage_issue(sg, kin, vin, nt);
        } else {
            // Every load of the tile is in flight before the ranking starts:
            // the ranking's shared-memory stores would otherwise order each
            // item's load after the previous item's ranking.
#pragma unroll
            for (int j = 0; j < kSortItems; ++j) {
                const unsigned long long i = wb + (unsigned long long)j * 32 + lane;
                k[j] = i < n ? __ldg(kin + i) : 0ull;
                v[j] = i < n ? __ldg(vin + i) : 0u;
            }
            __syncthreads();  // the warp histograms are cleared
        }
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const unsigned long long i = wb + (unsigned long long)j * 32 + lane;
            const bool ok = i < n;
            const uint32_t d = ok ? (uint32_t)((k[j] >> (8 * p)) & 0xFF) : 256u;
            // lanes with the same digit: intersect the eight bit-plane ballots
            // (and the ninth bit that marks lanes past the end)
            uint32_t peers = kFullMask;
#pragma unroll
            for (int bit = 0; bit < 9; ++bit) {
                const uint32_t m = __ballot_sync(kFullMask, (d >> bit) & 1u);
                peers &= ((d >> bit) & 1u) ? m : ~m;
            }
            const uint32_t before = (d < 256u) ? sm.wh[w][d] : 0u;
            rank[j] = before + __popc(peers & lane_lt());
            __syncwarp();
            if (d < 256u && (peers & lane_lt()) == 0) sm.wh[w][d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // thread d owns digit d: warp prefixes, local run start, global delta
        {
            const int d = threadIdx.x;  // kSortThreads == 256 digits
            uint32_t c = 0;
#pragma unroll
            for (int ww = 0; ww < kWarps; ++ww) {
                const uint32_t x = sm.wh[ww][d];
                sm.wh[ww][d] = c;
                c += x;
            }
            uint32_t tot;
            const uint32_t lstart = block_exscan(c, tot, sm.sw);
#pragma unroll
            for (int ww = 0; ww < kWarps; ++ww) sm.wh[ww][d] += lstart;
            sm.gdelta[d] = gstart - lstart;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const unsigned long long i = wb + (unsigned long long)j * 32 + lane;
            if (i < n) {
                const uint32_t lp = sm.wh[w][(uint32_t)((k[j] >> (8 * p)) & 0xFF)] + rank[j];
                sm.keys[lp] = k[j];
                sm.vals[lp] = v[j];
            }
        }
        __syncthreads();
        const unsigned long long rem = n - t * kTile;
        const int tn = rem < (unsigned long long)kTile ? (int)rem : kTile;
        for (int i = threadIdx.x; i < tn; i += kSortThreads) {
            const uint64_t key = sm.keys[i];
            const uint32_t pos = sm.gdelta[(uint32_t)((key >> (8 * p)) & 0xFF)] + (uint32_t)i;
            kout[pos] = key;
            vout[pos] = sm.vals[i];
        }
        __syncthreads();
    }
}

// Decoupled look-back words of the one-sweep passes: the kind in the top two
// bits (a tile's own count of a digit, or the count of that digit over all
// tiles up to and including it), the count below.  A word is written whole
// (one aligned 64-bit store), so a reader sees 0 or a complete word.
constexpr unsigned long long kLbAgg = 1ull << 62, kLbIncl = 2ull << 62, kLbCount = (1ull << 62) - 1ull;
// polls of a look-back word before the pass gives up (with 64 ns sleeps after
// the first 64 polls: about a second); a tile whose owner never publishes is
// reported, not waited for forever
constexpr int kLookbackPolls = 1 << 24;

__device__ __forceinline__ void lb_store(unsigned long long *p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long *>(p) = v;
}
__device__ __forceinline__ unsigned long long lb_load(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// One radix pass in one kernel (the simulation path): tiles are claimed in
// order from a counter; a tile's digit counts come from its own ranking, and
// its global run starts from the digits' bases (the global histogram) plus
// the counts of the tiles before it, found by looking back over their
// published words until an inclusive count.  Every tile a CTA waits on was
// claimed earlier by a running CTA, and waits only on tiles before it, so the
// waits end.  The tile histogram and digit scan passes are not needed.  Tiles
// are staged into shared memory one ahead by the bulk-copy engine, as in
// k_scatter; the ranking and the write-out are those of k_scatter.
__global__ void __launch_bounds__(kSortThreads, 2) k_onesweep(SortDev S, int p) {
    if (!S.plan[p]) return;
    extern __shared__ __align__(16) unsigned char scatter_raw[];
    ScatterSmem &sm = *reinterpret_cast<ScatterSmem *>(scatter_raw);
    ScatterStage &sg = *reinterpret_cast<ScatterStage *>(scatter_raw + sizeof(ScatterSmem));
    __shared__ uint32_t dbase[256];
    __shared__ uint32_t thist[256];  // the tile's own digit counts
    __shared__ unsigned long long tile_sh[2];  // the tile being sorted, the one claimed next
    const int src = S.plan[kPasses + p];
    const unsigned long long n = sort_n(S);
    const unsigned long long tiles = (n + kTile - 1) / kTile;
    const unsigned long long full_tiles = n / kTile;
    constexpr int kWarps = kSortThreads / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint64_t *kin = src ? S.keys[1] : S.keys[0];
    const uint32_t *vin = src ? S.vals[1] : S.vals[0];
    uint64_t *kout = src ? S.keys[0] : S.keys[1];
    uint32_t *vout = src ? S.vals[0] : S.vals[1];
    unsigned long long *lbc = src ? S.lb[1] : S.lb[0];  // this pass's words
    unsigned long long *lbn = src ? S.lb[0] : S.lb[1];  // the next active pass's, cleared here
    {
        // the digits' bases: exclusive scan of this pass's global histogram
        uint32_t tot;
        dbase[threadIdx.x] = block_exscan(S.ghist[p * 256 + threadIdx.x], tot, sm.sw);
    }
    uint32_t parity = 0;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sg.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const unsigned long long t0 = atomicAdd(S.tile_ctr + p, 1u);
        tile_sh[0] = t0;
        tile_sh[1] = tiles;
        if (t0 < full_tiles) stage_issue(sg, kin, vin, t0);
    }
    __syncthreads();
    for (;;) {
        const unsigned long long t = tile_sh[0];
        if (t >= tiles) break;
        for (int i = threadIdx.x; i < kWarps * 256; i += blockDim.x) (&sm.wh[0][0])[i] = 0;
        thist[threadIdx.x] = 0;
        const unsigned long long wb = t * kTile + (unsigned long long)w * (32 * kSortItems);
        uint64_t k[kSortItems];
        uint32_t v[kSortItems];
        uint32_t rank[kSortItems];
        if (t < full_tiles) {
            const bool ok = stage_wait(smem_addr(&sg.bar), parity);
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0) {
                    atomicOr(S.status, kStatusSortStall);
                    stage_wait(smem_addr(&sg.bar), parity);  // let the copy in flight land
                }
                return;
            }
            parity ^= 1u;
            const int lb = w * (32 * kSortItems) + lane;
#pragma unroll
            for (int j = 0; j < kSortItems; ++j) {
                k[j] = sg.keys[lb + j * 32];
                v[j] = sg.vals[lb + j * 32];
            }
        } else {
#pragma unroll
            for (int j = 0; j < kSortItems; ++j) {
                const unsigned long long i = wb + (unsigned long long)j * 32 + lane;
                k[j] = i < n ? __ldg(kin + i) : 0ull;
                v[j] = i < n ? __ldg(vin + i) : 0u;
            }
        }
        __syncthreads();  // the staging buffer is free and the histograms are cleared
        if (threadIdx.x == 0) {
            // claim the next tile and stream it in while this one is sorted
            const unsigned long long nt = atomicAdd(S.tile_ctr + p, 1u);
            tile_sh[1] = nt;
            if (nt < full_tiles) stage_issue(sg, kin, vin, nt);
        }
        // The tile's digit counts first, published before the ranking, so that
        // the tiles after it rarely find its word missing.
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const unsigned long long i = wb + (unsigned long long)j * 32 + lane;
            if (i < n) atomicAdd(&thist[(uint32_t)((k[j] >> (8 * p)) & 0xFF)], 1u);
        }
        __syncthreads();
        unsigned long long *row = lbc + t * 256;
        const uint32_t cnt = thist[threadIdx.x];
        lb_store(row + threadIdx.x, (t == 0 ? kLbIncl : kLbAgg) | cnt);
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const unsigned long long i = wb + (unsigned long long)j * 32 + lane;
            const bool ok = i < n;
            const uint32_t d = ok ? (uint32_t)((k[j] >> (8 * p)) & 0xFF) : 256u;
            uint32_t peers = kFullMask;
#pragma unroll
            for (int bit = 0; bit < 8; ++bit) {
                const uint32_t m = __ballot_sync(kFullMask, (d >> bit) & 1u);
                peers &= ((d >> bit) & 1u) ? m : ~m;
            }
            if (t >= full_tiles) {  // the last, partial tile: separate the lanes past the end
                const uint32_t m = __ballot_sync(kFullMask, d >> 8);
                peers &= (d >> 8) ? m : ~m;
            }
            const uint32_t before = (d < 256u) ? sm.wh[w][d] : 0u;
            rank[j] = before + __popc(peers & lane_lt());
            __syncwarp();
            if (d < 256u && (peers & lane_lt()) == 0) sm.wh[w][d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint32_t lstart;
        {
            const int d = threadIdx.x;  // kSortThreads == 256 digits
            uint32_t c = 0;
#pragma unroll
            for (int ww = 0; ww < kWarps; ++ww) {
                const uint32_t x = sm.wh[ww][d];
                sm.wh[ww][d] = c;
                c += x;
            }
            uint32_t tot;
            lstart = block_exscan(c, tot, sm.sw);
#pragma unroll
            for (int ww = 0; ww < kWarps; ++ww) sm.wh[ww][d] += lstart;
        }
        __syncthreads();
        // the tile in digit order in shared memory; its global offsets follow
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const unsigned long long i = wb + (unsigned long long)j * 32 + lane;
            if (i < n) {
                const uint32_t lp = sm.wh[w][(uint32_t)((k[j] >> (8 * p)) & 0xFF)] + rank[j];
                sm.keys[lp] = k[j];
                sm.vals[lp] = v[j];
            }
        }
        // Look back: add the counts of the tiles before this one, eight words
        // per round trip, newest first, until an inclusive count.
        int fail = 0;
        {
            const int d = threadIdx.x;
            unsigned long long excl = 0;
            if (t > 0) {
                constexpr int kWin = 8;
                unsigned long long j = t;  // tiles [0, j) not yet added
                bool found = false;
                int polls = 0;
                while (!found && !fail) {
                    unsigned long long wv[kWin];
#pragma unroll
                    for (int q = 0; q < kWin; ++q)
                        wv[q] = (unsigned long long)q < j ? lb_load(lbc + (j - 1 - q) * 256 + d) : kLbIncl;
#pragma unroll
                    for (int q = 0; q < kWin; ++q) {
                        if (found || fail || (unsigned long long)q >= j) break;
                        unsigned long long x = wv[q];
                        while ((x >> 62) == 0) {
                            if (++polls > kLookbackPolls) { fail = 1; break; }
                            if (polls > 64) __nanosleep(64);
                            x = lb_load(lbc + (j - 1 - q) * 256 + d);
                        }
                        if (fail) break;
                        excl += x & kLbCount;
                        if ((x >> 62) == 2) found = true;
                    }
                    j = j > (unsigned long long)kWin ? j - kWin : 0;
                    if (j == 0 && !found) fail = 1;  // tile 0 always publishes an inclusive count
                }
                if (!fail) lb_store(row + d, kLbIncl | (excl + cnt));
            }
            sm.gdelta[d] = dbase[d] + (uint32_t)excl - lstart;
            lbn[t * 256 + d] = 0ull;
        }
        if (__syncthreads_or(fail)) {
            if (threadIdx.x == 0) {
                atomicOr(S.status, kStatusSortStall);
                if (tile_sh[1] < full_tiles) stage_wait(smem_addr(&sg.bar), parity);  // the copy in flight
            }
            return;
        }
        const unsigned long long rem = n - t * kTile;
        const int tn = rem < (unsigned long long)kTile ? (int)rem : kTile;
        bool stray = false;
        for (int i = threadIdx.x; i < tn; i += kSortThreads) {
            const uint64_t key = sm.keys[i];
            const uint32_t pos = sm.gdelta[(uint32_t)((key >> (8 * p)) & 0xFF)] + (uint32_t)i;
            if (pos < n) {
                kout[pos] = key;
                vout[pos] = sm.vals[i];
            } else {
                stray = true;  // an offset past the keys: reported, never written
            }
        }
        if (stray) atomicOr(S.status, kStatusSortStall);
        __syncthreads();
        if (threadIdx.x == 0) tile_sh[0] = tile_sh[1];
        __syncthreads();
    }
}

static cudaError_t scatter_smem_attr() {
    cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void *>(k_scatter<false>), kScatterSmem);
    if (e == cudaSuccess) e = ensure_dynamic_smem(reinterpret_cast<const void *>(k_scatter<true>), kScatterSmemStaged);
    if (e != cudaSuccess) return e;
    return ensure_dynamic_smem(reinterpret_cast<const void *>(k_onesweep), kScatterSmemStaged);
}

// singles into time order
__global__ void k_gather(SortDev S, SinglesDev out) {
    const unsigned long long n = sort_n(S);
    const int fin = S.plan[2 * kPasses];
    const uint32_t *perm = fin ? S.vals[1] : S.vals[0];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint4 *r = reinterpret_cast<const uint4 *>(S.in_raw + perm[i]);
        const uint4 a = __ldg(r), b = __ldg(r + 1), c = __ldg(r + 2);
        out.t[i] = ((uint64_t)a.y << 32) | a.x;
        out.h[i] = ((uint64_t)a.w << 32) | a.z;
        out.unit[i] = (int32_t)b.x;
        out.panel[i] = (int32_t)b.y;
        out.job[i] = (int32_t)b.z;
        out.e[i] = __uint_as_float(b.w);
        out.eraw[i] = __uint_as_float(c.x);
        out.doi[i] = __uint_as_float(c.y);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *out.n = n;
}

// Coincidence sorting.  A cluster is a maximal run of time-sorted singles of
// one job whose consecutive gaps are <= window; windows never cross cluster
// ends, so each cluster is processed alone by the thread at its start: the
// earliest unconsumed single opens [t0, t0 + window]; exactly two singles in
// different panels make a coincidence; all singles in the window are consumed.
__global__ void k_coinc_flags(SinglesDev s, CoincDev C) {
    const unsigned long long n = *s.n;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint64_t ti = s.t[i];
        const int ji = s.job[i];
        const uint64_t W = C.window_ps[ji];
        const bool start = i == 0 || s.job[i - 1] != ji || ti - s.t[i - 1] > W;
        if (!start) continue;
        unsigned long long a = i;
        for (;;) {
            unsigned long long b = a;
            const uint64_t ta = s.t[a];
            while (b + 1 < n && s.job[b + 1] == ji && s.t[b + 1] - ta <= W) ++b;
            if (b == a + 1 && s.panel[a] != s.panel[b]) C.flag[a] = 1;
            // the cluster ends where the next gap exceeds the window
            if (b + 1 >= n || s.job[b + 1] != ji || s.t[b + 1] - s.t[b] > W) break;
            a = b + 1;
        }
    }
}

// compaction of flagged indices, in index order: counts per tile, one
// scan block, writes
__global__ void __launch_bounds__(1024) k_coinc_count(SinglesDev s, CoincDev C) {
    __shared__ uint32_t sw[32];
    const unsigned long long n = *s.n;
    const unsigned long long tiles = (n + 4095) / 4096;
    for (unsigned long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        uint32_t c = 0;
        for (int j = 0; j < 4; ++j) {
            const unsigned long long i = t * 4096 + (unsigned long long)j * 1024 + threadIdx.x;
            if (i < n) c += C.flag[i];
        }
        uint32_t tot;
        block_exscan(c, tot, sw);
        if (threadIdx.x == 0) C.tile_cnt[t] = tot;
    }
}

__global__ void __launch_bounds__(1024) k_coinc_scan(SinglesDev s, CoincDev C) {
    __shared__ uint32_t sw[32];
    const unsigned long long n = *s.n;
    const unsigned long long tiles = (n + 4095) / 4096;
    uint32_t base = 0;
    for (unsigned long long c = 0; c < tiles; c += blockDim.x) {
        const unsigned long long t = c + threadIdx.x;
        const uint32_t v = t < tiles ? C.tile_cnt[t] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exscan(v, tot, sw);
        if (t < tiles) C.tile_cnt[t] = base + ex;
        base += tot;
    }
    if (threadIdx.x == 0) *C.n = base;
}

__global__ void __launch_bounds__(1024) k_coinc_write(SinglesDev s, CoincDev C) {
    __shared__ uint32_t sw[32];
    const unsigned long long n = *s.n;
    const unsigned long long tiles = (n + 4095) / 4096;
    for (unsigned long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        uint32_t base = C.tile_cnt[t];
        for (int j = 0; j < 4; ++j) {
            const unsigned long long i = t * 4096 + (unsigned long long)j * 1024 + threadIdx.x;
            const uint32_t f = i < n ? C.flag[i] : 0u;
            uint32_t tot;
            const uint32_t ex = block_exscan(f, tot, sw);
            if (f) {
                C.a[base + ex] = (int32_t)i;
                C.b[base + ex] = (int32_t)(i + 1);
            }
            base += tot;
        }
    }
}

// Per-job statistics of a (batched) run: start of each job's segment in the
// time-sorted singles and in the coincidences (both are ordered by job, the
// high bits of the sort key), and the job's hit count from its tallies.
__global__ void __launch_bounds__(256) k_job_stats(SinglesDev s, CoincDev C, JobStatsDev J) {
    const int j = blockIdx.x;
    const unsigned long long ns = *s.n, nc = *C.n;
    if (threadIdx.x == 0) {
        unsigned long long lo = 0, hi = ns;  // first single with job >= j
        while (lo < hi) {
            const unsigned long long mid = (lo + hi) >> 1;
            if (s.job[mid] < j) lo = mid + 1; else hi = mid;
        }
        J.s_off[j] = lo;
        lo = 0;
        hi = nc;                             // first coincidence whose first single has job >= j
        while (lo < hi) {
            const unsigned long long mid = (lo + hi) >> 1;
            if (s.job[C.a[mid]] < j) lo = mid + 1; else hi = mid;
        }
        J.c_off[j] = lo;
        if (j == J.n_jobs - 1) {
            J.s_off[J.n_jobs] = ns;
            J.c_off[J.n_jobs] = nc;
        }
    }
    // hits of job j = sum of its per-crystal counts
    unsigned long long acc = 0;
    const unsigned long long *t = J.tally_count + J.tally_off[j];
    const long long nt = J.tally_n[j];
    for (long long i = threadIdx.x; i < nt; i += blockDim.x) acc += t[i];
    __shared__ unsigned long long red[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFullMask, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        J.hits[j] = tot;
    }
}

cudaError_t launch_job_stats(const SinglesDev &s, const CoincDev &C, const JobStatsDev &J, cudaStream_t st) {
    k_job_stats<<<J.n_jobs, 256, 0, st>>>(s, C, J);
    return cudaGetLastError();
}

// Plan plus the eight radix passes over an already keyed working set (used by
// the allocation-free sort entry point; the simulation path keeps its own
// launcher below).
cudaError_t launch_radix_passes(const SortDev &S, int sm_count, cudaStream_t st) {
    cudaError_t e = scatter_smem_attr();
    if (e != cudaSuccess) return e;
    k_plan<<<1, kPasses * 32, 0, st>>>(S);
    for (int p = 0; p < kPasses; ++p) {
        const int tg = (int)(S.max_tiles < (unsigned long long)sm_count * 8 ? S.max_tiles
                                                                              : (unsigned long long)sm_count * 8);
        k_tile_hist<<<tg, kSortThreads, 0, st>>>(S, p);
        k_digit_scan<<<256, 1024, 0, st>>>(S, p);
        k_scatter<false><<<tg, kSortThreads, kScatterSmem, st>>>(S, p);
    }
    return cudaGetLastError();
}

cudaError_t launch_sort_coinc(const SortDev &S, const SinglesDev &out, const CoincDev &C, int sm_count,
                              cudaStream_t st) {
    // the staged passes report a stalled copy or look-back in the status word
    if (!S.status || !S.lb[0] || !S.lb[1] || !S.tile_ctr) return cudaErrorInvalidValue;
    cudaError_t e = scatter_smem_attr();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(S.ghist, 0, sizeof(uint32_t) * kPasses * 256, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.tile_ctr, 0, sizeof(unsigned int) * kPasses, st);
    if (e != cudaSuccess) return e;
    k_make_keys<<<sm_count * 4, kSortThreads, 0, st>>>(S);
    k_plan<<<1, kPasses * 32, 0, st>>>(S);
    // two CTAs per SM are resident; more would only claim tiles later
    const int tg = (int)(S.max_tiles < (unsigned long long)sm_count * 2 ? (S.max_tiles ? S.max_tiles : 1)
                                                                        : (unsigned long long)sm_count * 2);
    for (int p = 0; p < kPasses; ++p) k_onesweep<<<tg, kSortThreads, kScatterSmemStaged, st>>>(S, p);
    const int grid = sm_count * 4;
    k_gather<<<grid, 256, 0, st>>>(S, out);
    // a cluster's flags are written by the thread at its start, possibly past
    // its own grid-stride range: clear them all before the flag kernel
    e = cudaMemsetAsync(C.flag, 0, S.cap ? S.cap : 1, st);
    if (e != cudaSuccess) return e;
    k_coinc_flags<<<grid, 256, 0, st>>>(out, C);
    const int cg = (int)(S.max_tiles < (unsigned long long)sm_count * 4 ? S.max_tiles : (unsigned long long)sm_count * 4);
    k_coinc_count<<<cg, 1024, 0, st>>>(out, C);
    k_coinc_scan<<<1, 1024, 0, st>>>(out, C);
    k_coinc_write<<<cg, 1024, 0, st>>>(out, C);
    return cudaGetLastError();
}

// load the digitizer's kernels and set their shared-memory limits (internal.h)
cudaError_t preload_sort_kernels() {
    const void *fns[] = {reinterpret_cast<const void *>(k_make_keys), reinterpret_cast<const void *>(k_plan),
                         reinterpret_cast<const void *>(k_tile_hist), reinterpret_cast<const void *>(k_digit_scan),
                         reinterpret_cast<const void *>(k_onesweep),
                         reinterpret_cast<const void *>(k_gather), reinterpret_cast<const void *>(k_coinc_flags),
                         reinterpret_cast<const void *>(k_coinc_count), reinterpret_cast<const void *>(k_coinc_scan),
                         reinterpret_cast<const void *>(k_coinc_write), reinterpret_cast<const void *>(k_job_stats)};
    cudaFuncAttributes fa;
    for (const void *f : fns) {
        const cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return e;
    }
    return scatter_smem_attr();
}

}  // namespace gpet
