// sort_noalloc.cu -- time sort that allocates no device memory.
//
// Some callers cannot call cudaMalloc: processes whose device memory is all
// handed out up front by another allocator (a caching allocator that has
// already reserved the pool, a serving process with a fixed memory budget),
// or latency-critical loops where an allocation's implicit device
// synchronisation is not acceptable.  For them this file provides one entry
// point, gpet_sort_times_noalloc, a variant of the radix time sort of the
// digitizer whose whole working set (ping-pong key and index buffers, digit
// histograms, pass plan, element count) lives in the file-scope array below.
// The array is part of the library image: every GPU that loads the library
// holds it until the process exits.  The caller still passes its inputs and
// outputs.
#include "gpet.h"
#include "host.h"

namespace gpet {

constexpr unsigned long long kNoallocMaxKeys = 1ull << 20;            // largest n accepted
constexpr unsigned long long kNoallocTiles = (kNoallocMaxKeys + 4095) / 4096;
// layout of the scratch array (all offsets multiples of 256 bytes)
constexpr size_t kOffN = 0;                                           // element count (8 bytes)
constexpr size_t kOffHist = 256;                                      // [8][256] uint32 digit histograms
constexpr size_t kOffPlan = kOffHist + 8 * 256 * 4;                   // 32 int plan words
constexpr size_t kOffKeys0 = kOffPlan + 256;
constexpr size_t kOffKeys1 = kOffKeys0 + 8 * kNoallocMaxKeys;
constexpr size_t kOffVals0 = kOffKeys1 + 8 * kNoallocMaxKeys;
constexpr size_t kOffVals1 = kOffVals0 + 4 * kNoallocMaxKeys;
constexpr size_t kOffTiles = kOffVals1 + 4 * kNoallocMaxKeys;
constexpr size_t kScratchBytes = kOffTiles + 256 * 4 * kNoallocTiles;  // 24.26 MiB

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

// keys[0] = t, vals[0] = index, eight digit histograms
__global__ void __launch_bounds__(256) k_noalloc_keys(const uint64_t *__restrict__ t_in, SortDev S) {
    __shared__ uint32_t h[8][256];
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const unsigned long long n = *S.n_in;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint64_t key = t_in[i];
        S.keys[0][i] = key;
        S.vals[0][i] = (uint32_t)i;
#pragma unroll
        for (int p = 0; p < 8; ++p) atomicAdd(&h[p][(key >> (8 * p)) & 0xFF], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) {
        const uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(S.ghist + i, v);
    }
}

__global__ void k_noalloc_set_n(unsigned long long *n_slot, unsigned long long n) { *n_slot = n; }

__global__ void k_noalloc_out(SortDev S, uint64_t *__restrict__ t_out, uint32_t *__restrict__ perm_out) {
    const unsigned long long n = *S.n_in;
    const int fin = S.plan[16];
    const uint64_t *k = fin ? S.keys[1] : S.keys[0];
    const uint32_t *v = fin ? S.vals[1] : S.vals[0];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        t_out[i] = k[i];
        if (perm_out) perm_out[i] = v[i];
    }
}

}  // namespace gpet

using namespace gpet;

extern "C" int gpet_sort_times_noalloc(const uint64_t *d_t_in, uint64_t n, uint64_t *d_t_out, uint32_t *d_perm_out,
                                       void *stream) {
    if (n > kNoallocMaxKeys)
        return gpet_fail(GPET_ERR_INVALID_ARG, "gpet_sort_times_noalloc: n = %llu exceeds its maximum of %llu keys",
                         (unsigned long long)n, kNoallocMaxKeys);
    if (n == 0) return GPET_OK;
    if (!d_t_in || !d_t_out) return gpet_fail(GPET_ERR_INVALID_ARG, "gpet_sort_times_noalloc: NULL input or output");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaGetDevice");
    // The host-side name of the array is not a device address: ask the runtime
    // for the address of the current device's copy.  The first lookup on a
    // device loads the module that holds the array (modules load lazily), which
    // is when its device memory is taken; later lookups read the loaded
    // module's symbol table.  Looking it up on every call, rather than caching
    // it, keeps the address right after a cudaDeviceReset reloads the module.
    void *sym = nullptr;
    e = cudaGetSymbolAddress(&sym, g_sort_scratch);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaGetSymbolAddress(sort scratch)");
    unsigned char *base = static_cast<unsigned char *>(sym);
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaDeviceGetAttribute");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SortDev S{};
    S.n_in = reinterpret_cast<const unsigned long long *>(base + kOffN);
    S.ghist = reinterpret_cast<uint32_t *>(base + kOffHist);
    S.plan = reinterpret_cast<int *>(base + kOffPlan);
    S.keys[0] = reinterpret_cast<uint64_t *>(base + kOffKeys0);
    S.keys[1] = reinterpret_cast<uint64_t *>(base + kOffKeys1);
    S.vals[0] = reinterpret_cast<uint32_t *>(base + kOffVals0);
    S.vals[1] = reinterpret_cast<uint32_t *>(base + kOffVals1);
    S.tile_hist = reinterpret_cast<uint32_t *>(base + kOffTiles);
    S.max_tiles = kNoallocTiles;
    S.cap = kNoallocMaxKeys;
    S.job_shift = 64;  // the keys are the caller's time stamps alone
    // the histograms keep the previous call's contents: clear them
    e = cudaMemsetAsync(S.ghist, 0, 8 * 256 * 4, st);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaMemsetAsync(sort scratch)");
    k_noalloc_set_n<<<1, 1, 0, st>>>(reinterpret_cast<unsigned long long *>(base + kOffN), n);
    k_noalloc_keys<<<sms * 4, 256, 0, st>>>(d_t_in, S);
    e = launch_radix_passes(S, sms, st);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "radix passes");
    k_noalloc_out<<<sms * 4, 256, 0, st>>>(S, d_t_out, d_perm_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return gpet_cuda_fail(e, "gpet_sort_times_noalloc launch");
    return GPET_OK;
}
