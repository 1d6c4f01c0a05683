// Step 2: sort the (tile, depth) instance keys (Sec. 1: tiling and sorting all
// primitives).  An LSD radix sort with 8-bit digits over the key's significant
// bits, each pass a reduce-then-scan triple of kernels with fixed grids:
//   upsweep   per-CTA digit counts of a contiguous chunk of whole 4096-key tiles
//   scan      per digit, exclusive scan of the counts over CTAs (digit-major)
//   downsweep stable local ranking (warp match_any), reorder through shared
//             memory, coalesced scatter
// followed by one pass that writes each tile's [start, end) range and orders
// every run of equal keys by record index (the atomic emission order of the
// instances is not deterministic; after this pass the list is).
// The instance count is read on the device, so the launch sequence is fixed
// by the plan and can be captured in a CUDA graph.
#include "vrs_sort.cuh"

namespace vrs {

__device__ __forceinline__ uint32_t live_count(const DevStatus *st, unsigned long long cap)
{
    if (st->flags & ST_CAPACITY) return 0u;   // after an overflow every later step is skipped
    unsigned long long n = st->instances;
    return (uint32_t)(n < cap ? n : cap);
}

__device__ __forceinline__ void chunk_of(uint32_t M, int c, int G, uint32_t &b, uint32_t &e)
{
    const uint64_t tiles = (M + (uint64_t)kSortTile - 1) / kSortTile;
    const uint64_t per = (tiles + G - 1) / G;
    const uint64_t b64 = (uint64_t)c * per * kSortTile;
    b = (uint32_t)(b64 < M ? b64 : M);
    const uint64_t e64 = b64 + per * kSortTile;
    e = (uint32_t)(e64 < M ? e64 : M);
}

// Exclusive scan of one value per thread over a 256-thread block; returns the
// block total through `total`.
__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t v, uint32_t *warp_tot, uint32_t &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    uint32_t off = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < kSortWarps; ++i) {
        uint32_t t = warp_tot[i];
        off += (i < w) ? t : 0u;
        tot += t;
    }
    total = tot;
    __syncthreads();
    return off + x - v;
}

__global__ void __launch_bounds__(kSortThreads) k_upsweep(const SortArgs a)
{
    __shared__ uint32_t h[kSortWarps][kRadix];
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&h[0][0])[i] = 0u;
    __syncthreads();
    const uint32_t M = live_count(a.st, a.cap);
    uint32_t b, e;
    chunk_of(M, blockIdx.x, a.G, b, e);
    const int w = threadIdx.x >> 5;
    for (uint32_t i = b + threadIdx.x; i < e; i += kSortThreads) {
        const uint32_t d = (uint32_t)(a.keys_in[i] >> a.shift) & a.digit_mask;
        atomicAdd(&h[w][d], 1u);
    }
    __syncthreads();
    const int d = threadIdx.x;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kSortWarps; ++i) s += h[i][d];
    a.counts[(size_t)d * a.G + blockIdx.x] = s;
}

// One CTA per digit, blockDim >= G: exclusive scan of that digit's counts over CTAs.
__global__ void __launch_bounds__(1024) k_scan_digits(const SortArgs a)
{
    __shared__ uint32_t wt[32];
    const int d = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t v = t < a.G ? a.counts[(size_t)d * a.G + t] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wt[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t y = lane < nw ? wt[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        if (lane < nw) wt[lane] = y;   // inclusive warp totals
    }
    __syncthreads();
    const uint32_t incl = x + (w > 0 ? wt[w - 1] : 0u);
    if (t < a.G) a.counts[(size_t)d * a.G + t] = incl - v;
    if (t == (int)blockDim.x - 1) a.totals[d] = incl;
}


__global__ void __launch_bounds__(kSortThreads) k_downsweep(const SortArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DownSmem &S = *reinterpret_cast<DownSmem *>(smem_raw);
    const unsigned FULL = 0xffffffffu;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t M = live_count(a.st, a.cap);
    uint32_t b, e;
    chunk_of(M, blockIdx.x, a.G, b, e);
    if (b >= e) return;   // uniform across the block
    // global base of each digit for this CTA: exclusive scan of the digit totals
    {
        uint32_t tot;
        const uint32_t db = block_excl_scan256(a.totals[t], S.wtot, tot);
        S.gbase[t] = db + a.counts[(size_t)t * a.G + blockIdx.x];
    }
    __syncthreads();
    const uint32_t lmask = lanemask_lt();
    for (uint32_t ts = b; ts < e; ts += kSortTile) {
        const uint32_t n = min((uint32_t)kSortTile, e - ts);
        for (int i = t; i < kSortWarps * (kRadix + 1); i += kSortThreads) (&S.whist[0][0])[i] = 0u;
        __syncthreads();
        unsigned long long kk[kSortItems];
        uint32_t vv[kSortItems], rk[kSortItems], dg[kSortItems];
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const uint32_t idx = (uint32_t)w * (kSortItems * 32) + i * 32 + lane;
            const bool valid = idx < n;
            kk[i] = valid ? a.keys_in[ts + idx] : 0ull;
            vv[i] = valid ? a.vals_in[ts + idx] : 0u;
            dg[i] = valid ? ((uint32_t)(kk[i] >> a.shift) & a.digit_mask) : (uint32_t)kRadix;
        }
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const uint32_t peers = __match_any_sync(FULL, dg[i]);
            const uint32_t r = __popc(peers & lmask);
            const uint32_t base = S.whist[w][dg[i]];
            __syncwarp();
            if (r == 0) S.whist[w][dg[i]] = base + __popc(peers);
            __syncwarp();
            rk[i] = base + r;
        }
        __syncthreads();
        {   // per digit: offsets of the warps, digit count of the tile
            uint32_t acc = 0;
#pragma unroll
            for (int ww = 0; ww < kSortWarps; ++ww) {
                const uint32_t x = S.whist[ww][t];
                S.whist[ww][t] = acc;
                acc += x;
            }
            S.tcnt[t] = acc;
            uint32_t tot;
            S.dstart[t] = block_excl_scan256(acc, S.wtot, tot);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            if (dg[i] < (uint32_t)kRadix) {
                const uint32_t pos = S.dstart[dg[i]] + S.whist[w][dg[i]] + rk[i];
                S.keys[pos] = kk[i];
                S.vals[pos] = vv[i];
            }
        }
        __syncthreads();
        for (uint32_t j = t; j < n; j += kSortThreads) {
            const unsigned long long key = S.keys[j];
            const uint32_t d = (uint32_t)(key >> a.shift) & a.digit_mask;
            const uint32_t dst = S.gbase[d] + (j - S.dstart[d]);
            a.keys_out[dst] = key;
            a.vals_out[dst] = S.vals[j];
        }
        __syncthreads();
        S.gbase[t] += S.tcnt[t];
        __syncthreads();
    }
}

// Tile ranges and the equal-key fix-up over the sorted list.
__global__ void k_ranges(const unsigned long long *keys, uint32_t *vals, uint2 *ranges,
                         int64_t n_tiles, const DevStatus *st, unsigned long long cap)
{
    const uint32_t M = live_count(st, cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        const unsigned long long key = keys[i];
        const uint32_t tile = (uint32_t)(key >> 32);
        if ((int64_t)tile >= n_tiles) continue;   // cannot happen for keys from vrs_preprocess
        const unsigned long long prev = i > 0 ? keys[i - 1] : 0ull;
        const unsigned long long next = i + 1 < M ? keys[i + 1] : 0ull;
        if (i == 0 || (uint32_t)(prev >> 32) != tile) ranges[tile].x = i;
        if (i + 1 == M || (uint32_t)(next >> 32) != tile) ranges[tile].y = i + 1;
        if ((i == 0 || prev != key) && i + 1 < M && next == key) {
            uint32_t j = i + 1;
            while (j < M && keys[j] == key) ++j;
            for (uint32_t a = i + 1; a < j; ++a) {      // insertion sort of the run by record index
                const uint32_t v = vals[a];
                uint32_t b = a;
                while (b > i && vals[b - 1] > v) {
                    vals[b] = vals[b - 1];
                    --b;
                }
                vals[b] = v;
            }
        }
    }
}

cudaError_t launch_sort(unsigned long long *keys0, uint32_t *vals0, unsigned long long *keys1,
                        uint32_t *vals1, uint32_t *counts, uint32_t *totals, uint2 *ranges,
                        int64_t n_tiles, const DevStatus *st, unsigned long long cap, int passes,
                        int G, int n_sms, cudaStream_t stream)
{
    {
        cudaError_t e = cudaFuncSetAttribute(k_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(DownSmem));
        if (e != cudaSuccess) return e;
    }
    unsigned long long *kin = keys0, *kout = keys1;
    uint32_t *vin = vals0, *vout = vals1;
    const int scan_threads = ((G + 31) / 32) * 32;
    for (int p = 0; p < passes; ++p) {
        SortArgs a{kin, vin, kout, vout, counts, totals, st, cap, 8 * p, G, 255u};
        k_upsweep<<<G, kSortThreads, 0, stream>>>(a);
        k_scan_digits<<<kRadix, scan_threads, 0, stream>>>(a);
        k_downsweep<<<G, kSortThreads, sizeof(DownSmem), stream>>>(a);
        unsigned long long *tk = kin; kin = kout; kout = tk;
        uint32_t *tv = vin; vin = vout; vout = tv;
    }
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)(n_tiles > 0 ? n_tiles : 1), stream);
    if (e != cudaSuccess) return e;
    k_ranges<<<n_sms * 8, 256, 0, stream>>>(kin, vin, ranges, n_tiles, st, cap);
    return cudaGetLastError();
}

}  // namespace vrs
