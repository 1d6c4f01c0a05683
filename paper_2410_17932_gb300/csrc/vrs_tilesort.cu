// Step 2, bucketed form (the default): the (tile, depth) instances are grouped
// by tile and each tile's bucket is sorted on its own (Sec. 1: tiling and
// sorting all primitives).  vrs_preprocess already counted every tile's
// instances while emitting them; here
//   k_tile_blocksum, k_tile_scan   exclusive scan of the counts -> tile ranges (up
//                                  to 64 Ki tiles, k_tile_scan alone: each CTA
//                                  sums the counts before its block itself)
//   k_tile_scatter                 each instance into its tile's bucket as the
//                                  composite (depth bits << 32 | record index)
//   k_tile_sort                    one launch for both sizes: one warp per tile
//                                  of <= 256 instances (a bitonic network in
//                                  registers and shuffles, on 32-bit keys of the
//                                  depth and the bucket slot), and larger tiles one
//                                  CTA each (runs of 128 sorted by its warps in
//                                  registers and merged in shared memory up to
//                                  1024, beyond that sorted 1024-runs merged in
//                                  global memory)
// Sorting the composite orders equal depths by record index, so the result is
// the unique (tile, depth, record) order and matches the radix path bit for bit.
#include "vrs_internal.cuh"

namespace vrs {

constexpr int kScanBlock = 1024;
constexpr int kSmallMax = 256;
constexpr int kBigChunk = 1024;       // shared-memory run of the big-tile path (8 KB)
constexpr int kBigThreads = 256;

struct TileSortArgs {
    const unsigned long long *keys_in;   // emitted keys (tile << 32 | depth bits)
    const uint32_t *vals_in;             // emitted record indices
    unsigned long long *bucket;          // [cap] composites
    unsigned long long *keys_out;        // sorted keys (may alias keys_in)
    uint32_t *vals_out;                  // sorted record indices (may alias vals_in)
    const uint32_t *cnt;                 // [n_tiles] instances per tile
    uint32_t *cursor;                    // [n_tiles]
    uint32_t *blocksum;                  // [ceil(n_tiles / kScanBlock)]
    uint32_t *big_list;                  // [n_tiles]
    uint2 *ranges;                       // [n_tiles]
    DevStatus *st;
    unsigned long long cap;
    int64_t n_tiles;
    uint32_t blend_max;                  // sort mode 2: tiles of <= blend_max instances are left
                                         // unsorted in the bucket for the blend to order (0: none)
};

__device__ __forceinline__ uint32_t live_instances(const DevStatus *st, unsigned long long cap)
{
    if (st->flags & ST_CAPACITY) return 0u;
    const unsigned long long n = st->instances;
    return (uint32_t)(n < cap ? n : cap);
}

__device__ __forceinline__ uint32_t block_sum1024(uint32_t v, uint32_t *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = __reduce_add_sync(0xffffffffu, v);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    uint32_t s = 0;
    if (w == 0) {
        s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
        s = __reduce_add_sync(0xffffffffu, s);
    }
    __syncthreads();
    return s;   // valid in warp 0
}

__global__ void __launch_bounds__(kScanBlock) k_tile_blocksum(const TileSortArgs a)
{
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t sh[32];
    if (a.st->flags & ST_CAPACITY) return;    // every tile range is written, even with no instances
    const int64_t t = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const uint32_t v = t < a.n_tiles ? a.cnt[t] : 0u;
    const uint32_t s = block_sum1024(v, sh);
    if (threadIdx.x == 0) a.blocksum[blockIdx.x] = s;
}

// direct = 1: each CTA sums the counts of all tiles before its block itself (one
// launch; for grids of up to kDirectBlocks blocks), else it sums the block sums
// k_tile_blocksum wrote.
constexpr unsigned kDirectBlocks = 64;

__global__ void __launch_bounds__(kScanBlock) k_tile_scan(const TileSortArgs a, int direct)
{
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t sh[32];
    __shared__ uint32_t base_s;
    if (a.st->flags & ST_CAPACITY) return;    // every tile range is written, even with no instances
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // prefix of the counts of the blocks before this one
    uint32_t p = 0;
    if (!direct) {
        for (uint32_t b = threadIdx.x; b < blockIdx.x; b += kScanBlock) p += a.blocksum[b];
    } else if ((reinterpret_cast<uintptr_t>(a.cnt) & 15u) == 0) {
        const uint4 *c4 = reinterpret_cast<const uint4 *>(a.cnt);
        for (uint32_t i = threadIdx.x; i < blockIdx.x * (kScanBlock / 4); i += kScanBlock) {
            const uint4 v = c4[i];
            p += (v.x + v.y) + (v.z + v.w);
        }
    } else {
        for (uint32_t i = threadIdx.x; i < blockIdx.x * kScanBlock; i += kScanBlock) p += a.cnt[i];
    }
    p = block_sum1024(p, sh);
    if (threadIdx.x == 0) base_s = p;
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const uint32_t v = t < a.n_tiles ? a.cnt[t] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    uint32_t wo = 0;
    for (int i = 0; i < w; ++i) wo += sh[i];
    const uint32_t off = base_s + wo + x - v;
    if (t < a.n_tiles) {
        a.ranges[t] = v ? make_uint2(off, off + v) : make_uint2(0u, 0u);
        a.cursor[t] = off;
        if (v > (uint32_t)kSmallMax && v > a.blend_max) {
            const uint32_t slot = atomicAdd(&a.st->work[1], 1u);
            // the counter starts at zero, so the slot is in range; the test keeps a sort
            // that did not run to its end from sending the next one past the list
            if (slot < (uint32_t)a.n_tiles) a.big_list[slot] = (uint32_t)t;
        }
    }
}

// Each thread keeps four instances in flight (loads, then the four atomics,
// then the four stores): the scatter is bound by the latency of the position
// atomics, not by bandwidth.
__global__ void __launch_bounds__(256) k_tile_scatter(const TileSortArgs a)
{
    pdl_wait();
    pdl_trigger();
    const uint32_t M = live_instances(a.st, a.cap);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < M; i0 += 4 * stride) {
        unsigned long long key[4];
        uint32_t val[4], pos[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t i = i0 + u * stride;
            key[u] = i < M ? a.keys_in[i] : ~0ull;
            val[u] = i < M ? a.vals_in[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t t = (uint32_t)(key[u] >> 32);
            pos[u] = (int64_t)t < a.n_tiles ? atomicAdd(&a.cursor[t], 1u) : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (pos[u] != 0xffffffffu) a.bucket[pos[u]] = (key[u] << 32) | (unsigned long long)val[u];
    }
}

// Bitonic sort of 32*E keys held by one warp, element e = i*32 + lane in v[i],
// in the form whose comparators all put the minimum at the lower element: each
// merge of width k starts by comparing e with its mirror e ^ (k - 1), then
// half-cleans with partners e ^ j.  No comparator needs a direction bit.
// The per-element bodies are unrolled; the stage loops are not, which keeps the
// instantiations small enough for the instruction cache.  T: the 64-bit
// composites, or 32-bit keys.
template <int E, typename T>
__device__ __forceinline__ void shfl_stage(T (&v)[E], int mask, int lowbit, int lane)
{
    const bool lower = (lane & lowbit) == 0;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const T o = __shfl_xor_sync(0xffffffffu, v[i], mask);
        v[i] = (lower == (v[i] < o)) ? v[i] : o;
    }
}

// Mirror step of a merge wider than a warp: partner register i ^ M, lane ^ 31.
template <int E, int M, typename T>
__device__ __forceinline__ void flip_regs(T (&v)[E])
{
    if constexpr (M < E) {
        T o[E];
#pragma unroll
        for (int i = 0; i < E; ++i) o[i] = __shfl_xor_sync(0xffffffffu, v[i ^ M], 31);
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = ((i < (i ^ M)) == (v[i] < o[i])) ? v[i] : o[i];
    }
}

// Half-cleaner step across registers: partners i and i ^ JI in the same lane.
template <int E, int JI, typename T>
__device__ __forceinline__ void reg_half(T (&v)[E])
{
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int p = i ^ JI;
        if (p > i && p < E) {
            const T x = v[i], y = v[p];
            v[i] = x < y ? x : y;
            v[p] = x < y ? y : x;
        }
    }
}

template <int E, typename T>
__device__ __forceinline__ void warp_bitonic(T (&v)[E], int lane)
{
    constexpr int P = 32 * E;
#pragma unroll 1
    for (int k = 2; k <= P; k <<= 1) {
        if (k <= 32) shfl_stage<E>(v, k - 1, k >> 1, lane);
        else if (k == 64) flip_regs<E, 1>(v);
        else if (k == 128) flip_regs<E, 3>(v);
        else flip_regs<E, 7>(v);
#pragma unroll 1
        for (int j = k >> 2; j > 0; j >>= 1) {
            if (j >= 32) {
                if (j == 32) reg_half<E, 1>(v);
                else if (j == 64) reg_half<E, 2>(v);
                else reg_half<E, 4>(v);
            } else {
                shfl_stage<E>(v, j, j, lane);
            }
        }
    }
}

// One warp sorts a tile of n <= 32 E instances.  The network runs on 32-bit keys: the
// depth bits' offset from the tile's least (depth is non-negative, so its bits order as
// its value), shifted right just enough to fit 23 bits, above the instance's 8-bit
// slot in the bucket; the sorted slots then gather the composites.  Keys order the
// depths exactly except where two shifted offsets are equal (equal depths, or depths
// within 2^shift units in the last place): the warp finds any such neighbours after
// the sort and then sorts the full 64-bit composites instead, which also order equal
// depths by record index.
template <int E>
__device__ __forceinline__ void warp_sort_tile(const TileSortArgs &a, uint32_t t, uint32_t start, uint32_t n,
                                               int lane)
{
    static_assert(32 * E <= 256, "8-bit slots");
    const unsigned FULL = 0xffffffffu;
    uint32_t d[E];
    uint32_t dmin = 0xffffffffu, dmax = 0u;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const uint32_t e = i * 32 + lane;
        d[i] = e < n ? (uint32_t)(a.bucket[start + e] >> 32) : 0xffffffffu;
        if (e < n) {
            dmin = min(dmin, d[i]);
            dmax = max(dmax, d[i]);
        }
    }
    dmin = __reduce_min_sync(FULL, dmin);
    dmax = __reduce_max_sync(FULL, dmax);
    const uint32_t range = dmax - dmin;
    const int shift = max(0, (32 - __clz(range)) - 23);
    uint32_t k[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const uint32_t e = i * 32 + lane;
        k[i] = e < n ? (((d[i] - dmin) >> shift) << 8) | e : 0xffffffffu;
    }
    warp_bitonic<E>(k, lane);
    // equal shifted offsets between sorted neighbours (padding keys excluded)
    bool tie = false;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const uint32_t down = __shfl_down_sync(FULL, k[i], 1);
        const uint32_t wrap = __shfl_sync(FULL, k[i + 1 < E ? i + 1 : i], 0);
        const uint32_t nxt = lane < 31 ? down : (i + 1 < E ? wrap : 0xffffffffu);
        tie |= k[i] != 0xffffffffu && nxt != 0xffffffffu && (k[i] >> 8) == (nxt >> 8);
    }
    const unsigned long long th = (unsigned long long)t << 32;
    if (__any_sync(FULL, tie)) {
        unsigned long long v[E];
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const uint32_t e = i * 32 + lane;
            v[i] = e < n ? a.bucket[start + e] : ~0ull;
        }
        warp_bitonic<E>(v, lane);
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const uint32_t e = i * 32 + lane;
            if (e < n) {
                a.keys_out[start + e] = th | (v[i] >> 32);
                a.vals_out[start + e] = (uint32_t)v[i];
            }
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const uint32_t e = i * 32 + lane;
        if (e < n) {
            const unsigned long long c = a.bucket[start + (k[i] & 0xffu)];
            a.keys_out[start + e] = th | (c >> 32);
            a.vals_out[start + e] = (uint32_t)c;
        }
    }
}

// One warp sorts tile t if it holds 1..256 instances (larger tiles go to the CTA path).
__device__ __forceinline__ void sort_small_tile(const TileSortArgs &a, int64_t t, int lane)
{
    if (t >= a.n_tiles) return;
    const uint2 r = a.ranges[t];          // {start, end}, {0, 0} when empty: one load, no chain
    const uint32_t n = r.y - r.x;
    if (n == 0 || n > (uint32_t)kSmallMax || n <= a.blend_max) return;
    const uint32_t start = r.x;
    if (n <= 32) warp_sort_tile<1>(a, (uint32_t)t, start, n, lane);
    else if (n <= 64) warp_sort_tile<2>(a, (uint32_t)t, start, n, lane);
    else if (n <= 128) warp_sort_tile<4>(a, (uint32_t)t, start, n, lane);
    else warp_sort_tile<8>(a, (uint32_t)t, start, n, lane);
}

// Sorts the P composites of s (P a power of two, 256 <= P <= kBigChunk; the
// caller pads with ~0): each warp sorts a run of 128 in registers (the warp
// bitonic network), then log2(P / 128) merge-path passes in shared memory, each
// thread writing P / kBigThreads consecutive outputs of its pair of runs.
// Returns the buffer that holds the result (s or t).
__device__ unsigned long long *chunk_sort(unsigned long long *s, unsigned long long *t, uint32_t P)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if ((uint32_t)(128 * w) < P) {
        unsigned long long v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = s[128 * w + 32 * i + lane];
        warp_bitonic<4>(v, lane);
#pragma unroll
        for (int i = 0; i < 4; ++i) s[128 * w + 32 * i + lane] = v[i];
    }
    __syncthreads();
    unsigned long long *src = s, *dst = t;
    const uint32_t ipt = P / kBigThreads;
    for (uint32_t L = 128; L < P; L <<= 1) {
        const uint32_t o0 = threadIdx.x * ipt;
        const uint32_t pr = o0 / (2 * L), d = o0 - pr * 2 * L;
        const unsigned long long *A = src + pr * 2 * L, *B = A + L;
        // split of diagonal d: the number of elements taken from A
        uint32_t lo = d > L ? d - L : 0u, hi = d < L ? d : L;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (A[mid] <= B[d - 1 - mid]) lo = mid + 1; else hi = mid;
        }
        uint32_t i = lo, j = d - lo;
        for (uint32_t k = 0; k < ipt; ++k) {
            const bool takeA = j >= L || (i < L && A[i] <= B[j]);
            dst[o0 + k] = takeA ? A[i++] : B[j++];
        }
        __syncthreads();
        unsigned long long *x = src;
        src = dst;
        dst = x;
    }
    return src;
}

// Merges sorted src[0, la) and src[la, la + lb) into dst (merge path; one CTA).
__device__ void block_merge(const unsigned long long *src, uint32_t la, uint32_t lb, unsigned long long *dst)
{
    const unsigned long long *A = src, *B = src + la;
    const uint32_t total = la + lb;
    const uint32_t per = (total + blockDim.x - 1) / blockDim.x;
    const uint32_t d0 = min(total, threadIdx.x * per), d1 = min(total, d0 + per);
    if (d0 >= d1) return;
    // split point of diagonal d0: number of elements taken from A
    uint32_t lo = d0 > lb ? d0 - lb : 0u, hi = min(d0, la);
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (A[mid] <= B[d0 - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    uint32_t i = lo, j = d0 - lo;
    for (uint32_t d = d0; d < d1; ++d) {
        const bool takeA = j >= lb || (i < la && A[i] <= B[j]);
        dst[d] = takeA ? A[i++] : B[j++];
    }
}

// One CTA pulls tiles of more than 256 instances from the big-tile list until it
// is empty: sorted runs of kBigChunk in shared memory, merged in global memory.
__device__ __forceinline__ void sort_big_tiles(const TileSortArgs &a, unsigned long long *s, unsigned long long *s2,
                                               uint32_t &s_idx)
{
    const uint32_t n_big = min(a.st->work[1], (uint32_t)a.n_tiles);
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(&a.st->work[2], 1u);
        __syncthreads();
        const uint32_t idx = s_idx;
        __syncthreads();
        if (idx >= n_big) break;
        const uint32_t t = a.big_list[idx];
        const uint32_t start = a.ranges[t].x, n = a.cnt[t];
        unsigned long long *bk = a.bucket + start;
        unsigned long long *tmp = a.keys_out + start;   // scratch until the final write
        // sorted runs of kBigChunk in the bucket
        for (uint32_t c0 = 0; c0 < n; c0 += kBigChunk) {
            const uint32_t m = min((uint32_t)kBigChunk, n - c0);
            uint32_t P = 256;
            while (P < m) P <<= 1;
            for (uint32_t e = threadIdx.x; e < P; e += blockDim.x) s[e] = e < m ? bk[c0 + e] : ~0ull;
            __syncthreads();
            const unsigned long long *r = chunk_sort(s, s2, P);
            for (uint32_t e = threadIdx.x; e < m; e += blockDim.x) bk[c0 + e] = r[e];
            __syncthreads();
        }
        // pairwise merges, bucket <-> scratch
        unsigned long long *src = bk, *dst = tmp;
        for (uint32_t width = kBigChunk; width < n; width <<= 1) {
            for (uint32_t r0 = 0; r0 < n; r0 += 2 * width) {
                const uint32_t la = min(width, n - r0);
                const uint32_t lb = min(width, n - r0 - la);
                block_merge(src + r0, la, lb, dst + r0);
            }
            __syncthreads();
            unsigned long long *x = src;
            src = dst;
            dst = x;
        }
        // split the composites into the sorted key and record-index lists (in place
        // when the result is already in the key list: every thread reads, then writes,
        // the same element)
        const unsigned long long th = (unsigned long long)t << 32;
        for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
            const unsigned long long c = src[e];
            a.keys_out[start + e] = th | (c >> 32);
            a.vals_out[start + e] = (uint32_t)c;
        }
        __syncthreads();
    }
}

// Both sorts in one launch, so that the few long big-tile CTAs overlap the many
// short warp sorts: CTAs below n_big work through the big-tile list, the others
// give each of their warps one tile.
__global__ void __launch_bounds__(kBigThreads, 6) k_tile_sort(const TileSortArgs a, unsigned n_big)
{
    __shared__ unsigned long long s[kBigChunk], s2[kBigChunk];
    __shared__ uint32_t s_idx;
    pdl_wait();
    pdl_trigger();
    if (live_instances(a.st, a.cap) != 0) {
        if (blockIdx.x < n_big) {
            sort_big_tiles(a, s, s2, s_idx);
        } else {
            const int64_t t = (int64_t)(blockIdx.x - n_big) * (kBigThreads / 32) + (threadIdx.x >> 5);
            sort_small_tile(a, t, threadIdx.x & 31);
        }
    }
    // the last CTA to finish clears the big-tile counters for the next sort (the
    // scan appends to work[1]; no CTA reads them after its own ticket)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&a.st->work[3], 1u) == gridDim.x - 1) {
            a.st->work[1] = 0u;
            a.st->work[2] = 0u;
            a.st->work[3] = 0u;
        }
    }
}

cudaError_t launch_tile_sort(const unsigned long long *keys_in, const uint32_t *vals_in,
                             unsigned long long *bucket, unsigned long long *keys_out, uint32_t *vals_out,
                             const uint32_t *cnt, uint32_t *cursor, uint32_t *blocksum, uint32_t *big_list,
                             uint2 *ranges, DevStatus *st, unsigned long long cap, int64_t n_tiles,
                             uint32_t blend_max, int n_sms, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    TileSortArgs a{keys_in, vals_in, bucket, keys_out, vals_out, cnt, cursor, blocksum, big_list,
                   ranges, st, cap, n_tiles, blend_max};
    // the big-tile counters (work[1], work[2]) are zero here: cleared with the status
    // block by the preprocess, and again by the last CTA of every tile sort
    const unsigned nb = (unsigned)((n_tiles + kScanBlock - 1) / kScanBlock);
    const int direct = nb <= kDirectBlocks ? 1 : 0;
    cudaError_t e;
    if (!direct) {
        e = launch_pdl(k_tile_blocksum, dim3(nb), dim3(kScanBlock), 0, s, a);
        if (e != cudaSuccess) return e;
    }
    e = launch_pdl(k_tile_scan, dim3(nb), dim3(kScanBlock), 0, s, a, direct);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_tile_scatter, dim3(n_sms * 8), dim3(256), 0, s, a);
    if (e != cudaSuccess) return e;
    const unsigned n_big = (unsigned)n_sms * 2u;
    const int64_t per = kBigThreads / 32;
    k_tile_sort<<<(unsigned)(n_big + (n_tiles + per - 1) / per), kBigThreads, 0, s>>>(a, n_big);
    return cudaGetLastError();
}

}  // namespace vrs
