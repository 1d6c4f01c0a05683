// vrs_sort_pairs_noalloc: the library's stable LSD radix sort of (key, value)
// pairs, for callers that must not allocate device memory.  Its scratch (one
// ping-pong pair buffer, the per-CTA digit counts and a status block) is a
// file-scope static device array, so the entry point calls no cudaMalloc,
// cudaFree or allocating library routine.
//
// The array exists once per GPU that loads this library and is held until the
// process exits.  Host code cannot use the array's name as a device address
// (on the host it names a stand-in object), so the first call on each device
// looks the address up with cudaGetSymbolAddress, with that device current,
// and caches it.  Every call shares the array and it keeps the previous
// call's contents: each call rewrites the status block before its passes, and
// every pass rewrites the counts it reads.  Two calls whose work overlaps on
// the GPU (different streams, no ordering between them) race on the array.
#include <mutex>

#include "vrs_sort.cuh"

namespace vrs {

constexpr int64_t kNoAllocMaxPairs = VRS_NOALLOC_MAX_PAIRS;
constexpr int kNoAllocMaxCtas = 1024;
constexpr int kNoAllocMaxDevices = 64;

struct NoAllocScratch {
    unsigned long long keys[kNoAllocMaxPairs];
    uint32_t vals[kNoAllocMaxPairs];
    uint32_t counts[kRadix * kNoAllocMaxCtas];
    uint32_t totals[kRadix];
    DevStatus st;
};

// ~13.6 MB per device: 12 bytes per pair for 2^20 pairs, 1 MB of digit counts.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// The sort kernels take the pair count from a status block: set it for this call.
__global__ void k_noalloc_begin(DevStatus *st, unsigned long long n)
{
    st->flags = 0u;
    st->reserved = 0u;
    st->instances = n;
    st->pair_evals = 0ull;
    st->pair_blends = 0ull;
    st->block_evals = 0ull;
}

namespace {
std::mutex g_mu;
NoAllocScratch *g_addr[kNoAllocMaxDevices];
int g_ctas[kNoAllocMaxDevices];
}  // namespace

}  // namespace vrs

using namespace vrs;

extern "C" vrs_status vrs_sort_pairs_noalloc(const uint64_t *keys_in, const uint32_t *vals_in,
                                              uint64_t *keys_out, uint32_t *vals_out, int64_t n,
                                              int32_t key_bits, void *stream)
{
    if (n < 0 || key_bits < 1 || key_bits > 64) return VRS_ERR_INVALID;
    if (n > kNoAllocMaxPairs) return VRS_ERR_CAPACITY;   // more pairs than the static scratch holds
    if (n == 0) return VRS_OK;
    if (!keys_in || !vals_in || !keys_out || !vals_out) return VRS_ERR_INVALID;
    if ((const void *)keys_in == (const void *)keys_out || (const void *)vals_in == (const void *)vals_out)
        return VRS_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return VRS_ERR_CUDA;
    NoAllocScratch *S;
    int G;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return VRS_ERR_CUDA;
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
                return VRS_ERR_CUDA;
            g_ctas[dev] = 2 * sms > kNoAllocMaxCtas ? kNoAllocMaxCtas : 2 * sms;
            g_addr[dev] = static_cast<NoAllocScratch *>(p);
        }
        S = g_addr[dev];
        G = g_ctas[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaFuncSetAttribute(k_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(DownSmem)) != cudaSuccess)
        return VRS_ERR_CUDA;
    k_noalloc_begin<<<1, 1, 0, s>>>(&S->st, (unsigned long long)n);
    const int passes = (key_bits + 7) / 8;
    const int scan_threads = ((G + 31) / 32) * 32;
    const unsigned long long *src_k = reinterpret_cast<const unsigned long long *>(keys_in);
    const uint32_t *src_v = vals_in;
    for (int p = 0; p < passes; ++p) {
        // the last pass writes the caller's output; earlier passes alternate so that it does
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        unsigned long long *dst_k = to_out ? reinterpret_cast<unsigned long long *>(keys_out) : S->keys;
        uint32_t *dst_v = to_out ? vals_out : S->vals;
        // the last pass sorts only the bits left below key_bits, so that bits above it
        // (which the caller may leave nonzero) do not reorder pairs with equal sort bits
        const int left = key_bits - 8 * p;
        const uint32_t mask = left >= 8 ? 255u : ((1u << left) - 1u);
        SortArgs a{src_k, src_v, dst_k, dst_v, S->counts, S->totals, &S->st,
                   (unsigned long long)n, 8 * p, G, mask};
        k_upsweep<<<G, kSortThreads, 0, s>>>(a);
        k_scan_digits<<<kRadix, scan_threads, 0, s>>>(a);
        k_downsweep<<<G, kSortThreads, sizeof(DownSmem), s>>>(a);
        src_k = dst_k;
        src_v = dst_v;
    }
    return cudaGetLastError() == cudaSuccess ? VRS_OK : VRS_ERR_CUDA;
}
