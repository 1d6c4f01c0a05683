// Step 3: per-tile front-to-back alpha compositing of colour, the approximate
// depth of Eq. 1 (Sec. 3.2) and the final transmittance.
//
// One CTA owns one tile (TS x TS pixels); every warp owns an 8x8 block and
// every lane two horizontally adjacent pixels.  The tile's sorted instances
// are staged in shared memory in batches of one per thread: the staging lane
// gathers the 48-byte record, moves its 2D mean into the tile-local frame in
// double-float (2016-pixel-wide views keep sub-1e-5 px positions), and tests
// the splat against every warp's block (a bounding-box screen, then the exact
// minimum of the quadratic form over the block).  Each warp compacts the
// batch to the splats that can reach its block (ballot + popc, list order
// kept) and evaluates only those, two at a time, without branches: a pixel's
// update is a select on its skip / stop / blend decision.  The culling only
// drops pairs with alpha < 1/255 for certain, so the image is the same as
// without it.  The CTA leaves a tile when all of its pixels have stopped.
#include "vrs_internal.cuh"

namespace vrs {

struct FwdArgs {
    const float4 *viewtab;      // per view (cx, cy, -, -)
    const float4 *rec;
    const uint32_t *vals;
    const uint2 *ranges;
    DevStatus *st;
    float *rgb;
    float *depth;
    float *Tf;
    uint32_t *ncontrib;
    const uint32_t *order;      // persistent: tile work order (heaviest first), or null: tile order
    uint32_t *tile_work;        // LAST, nullable: per tile and warp, its block's largest last blended position
    int64_t n_tiles;
    int64_t n_records;
    unsigned long long cap;
    int persistent;
    int half_out;               // write the outputs as IEEE binary16
    int tiles_per_pull;         // persistent: work-order items claimed per atomic
    // sort mode 2: a tile of <= blend_max instances is still an unsorted bucket of composites
    // (depth bits << 32 | record index); the blend orders it while staging and writes the
    // sorted key and record-index lists back
    const unsigned long long *bucket;
    unsigned long long *keys_w;
    uint32_t *vals_w;
    uint32_t blend_max;
};

// The state of a thread's two pixels, packed in pairs so that the blend's
// multiplies and fused multiply-adds issue as FP32x2 instructions.  Each
// component of a packed operation is the correctly rounded scalar operation,
// so the result is bit for bit that of the scalar code.
struct PixAcc2 {
    float2 T, R, G, B, D;
    uint32_t last0, last1, stop0, stop1;
    bool done0, done1;
};

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// One splat at a thread's two pixels, front to back: skip below 1/255, stop
// before T would drop under 1e-4, otherwise blend.  Written as selects (no
// branches).  u holds the two pixels' q' - lo (pair_u2); B = (-l2, lo, lt,
// depth), C = (r, g, b, list position).  LAST tracks each pixel's last
// blended position, the reverse pass's starting point (plans made for the
// backward); COUNT also tracks the stop position and the blend count for the
// work counters.
template <bool COUNT, bool LAST>
__device__ __forceinline__ void pix_update2(PixAcc2 &P, float2 u, const float4 &B, const float4 &C,
                                            uint32_t &n_blend)
{
    const bool h0 = !P.done0 && u.x <= kLog2_255, h1 = !P.done1 && u.y <= kLog2_255;
    const float2 al = make_float2(fminf(ex2_approx(-u.x), 0.99f), fminf(ex2_approx(-u.y), 0.99f));
    const float2 m = __fmul2_rn(al, P.T);                       // alpha T, the weight if it blends
    const float2 Tn = __ffma2_rn(m, f2(-1.f), P.T);             // T - alpha T = T (1 - alpha)
    const bool s0 = h0 && Tn.x < 1e-4f, s1 = h1 && Tn.y < 1e-4f;
    const bool b0 = h0 && !s0, b1 = h1 && !s1;
    // the weight where the pixel blends, 0 elsewhere (alpha T times a 0/1 factor, a
    // multiply rather than a select): then T - weight is T' or T exactly, without a
    // select on T
    const float2 wt = __fmul2_rn(m, make_float2(b0 ? 1.f : 0.f, b1 ? 1.f : 0.f));
    P.R = __ffma2_rn(f2(C.x), wt, P.R);
    P.G = __ffma2_rn(f2(C.y), wt, P.G);
    P.B = __ffma2_rn(f2(C.z), wt, P.B);
    P.D = __ffma2_rn(f2(B.w), wt, P.D);
    P.T = __ffma2_rn(wt, f2(-1.f), P.T);
    const uint32_t pos = (uint32_t)__float_as_int(C.w);
    if (LAST) {
        P.last0 = b0 ? pos : P.last0;
        P.last1 = b1 ? pos : P.last1;
    }
    P.done0 = P.done0 || s0;
    P.done1 = P.done1 || s1;
    if (COUNT) {
        P.stop0 = s0 ? pos : P.stop0;
        P.stop1 = s1 ? pos : P.stop1;
        n_blend += (b0 ? 1u : 0u) + (b1 ? 1u : 0u);
    }
}

// pair_u2 for a splat staged as A = (K, L, -l0, -l1), B.x = -l2, B.y = lo: the
// same operations (negation is exact), the per-pixel ones packed; pxc2 =
// (pxc, pxc + 1).
__device__ __forceinline__ float2 pair_u2v(const float4 &A, const float4 &B, float2 pxc2, float pyc)
{
    const float s = __fmaf_rn(B.x, pyc, A.y);
    const float w = __fmaf_rn(s, s, -B.y);
    const float r = __fmaf_rn(A.w, pyc, A.x);
    const float2 t = __ffma2_rn(f2(A.z), pxc2, f2(r));
    return __ffma2_rn(t, t, f2(w));
}

template <int TS, bool COUNT, bool LAST, bool PERSIST, bool HALF = false>
__global__ void __launch_bounds__(BlendCfg<TS>::THREADS, BlendCfg<TS>::MIN_BLOCKS)
    k_render_fwd(const __grid_constant__ ViewTable vt, const FwdArgs a)
{
    using Cfg = BlendCfg<TS>;
    __shared__ float4 sR[Cfg::BATCH][3];   // staged splats: A, B, C of one instance together
    __shared__ uint32_t smask[Cfg::BATCH];
    __shared__ uint16_t slist[Cfg::WARPS][Cfg::BATCH];
    __shared__ int64_t s_tile;
    __shared__ uint32_t s_k, s_left;      // persistent: the CTA's claimed run of the work order
    __shared__ unsigned long long s_comp[Cfg::BATCH];   // sort mode 2: the tile's composites
    __shared__ unsigned long long s_cnt[3];

    pdl_wait();
    pdl_trigger();
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int bx = (w % Cfg::WGX) * 8, by = (w / Cfg::WGX) * 8;
    const float pxc = (float)(bx + 2 * (lane & 3)) + 0.5f, pyc = (float)(by + (lane >> 2)) + 0.5f;
    const float2 pxc2 = make_float2(pxc, pxc + 1.0f);
    const uint32_t lmask = lanemask_lt();
    if (tid == 0) {
        s_cnt[0] = s_cnt[1] = s_cnt[2] = 0ull;
        s_left = 0u;
    }
    __syncthreads();
    const bool skip_all = (a.st->flags & ST_CAPACITY) != 0;
    uint32_t n_eval = 0, n_blend = 0, n_blk = 0;

    for (int64_t iter = 0; !skip_all; ++iter) {
        int64_t t;
        if (PERSIST) {
            if (tid == 0) {
                // one atomic claims the next tiles_per_pull items of the order
                if (s_left == 0u) {
                    s_k = atomicAdd(&a.st->work[0], (uint32_t)a.tiles_per_pull);
                    s_left = (uint32_t)a.tiles_per_pull;
                }
                const uint32_t k = s_k + ((uint32_t)a.tiles_per_pull - s_left);
                --s_left;
                s_tile = (int64_t)k < a.n_tiles ? (a.order ? (int64_t)a.order[k] : (int64_t)k) : -1;
            }
            __syncthreads();
            t = s_tile;
            __syncthreads();
            if (t < 0) break;
        } else {
            if (iter > 0) break;
            t = blockIdx.x;
        }
        const int vi = view_of_tile(vt, t);
        const DevView &V = vt.v[vi];
        const float4 pp = a.viewtab[vi];
        const int64_t lt_ = t - V.tile_base;
        int tx, ty;
        tile_xy(lt_, V.gw, tx, ty);
        const int px = tx * TS + bx + 2 * (lane & 3), py = ty * TS + by + (lane >> 2);
        const bool in0 = px < V.w && py < V.h, in1 = px + 1 < V.w && py < V.h;
        float oxh, oxl, oyh, oyl;
        tile_origin((float)(tx * TS), pp.x, oxh, oxl);
        tile_origin((float)(ty * TS), pp.y, oyh, oyl);
        const uint2 range = live_range(a.ranges, t, a.st, a.cap);
        // sort mode 2, a tile of one batch at most: order it here (CTA-uniform)
        const bool rank_sort = a.blend_max != 0u && range.y - range.x <= a.blend_max;

        PixAcc2 P;
        P.T = f2(1.f);
        P.R = P.G = P.B = P.D = f2(0.f);
        P.last0 = P.last1 = 0u;
        P.stop0 = in0 ? range.y - range.x : 0u;
        P.stop1 = in1 ? range.y - range.x : 0u;
        P.done0 = !in0;
        P.done1 = !in1;

        for (uint32_t bs = range.x; bs < range.y; bs += Cfg::BATCH) {
            // before a later batch: the previous one is no longer read, and the CTA leaves
            // when all of its pixels have stopped (the first batch needs neither)
            if (bs != range.x && __syncthreads_and(P.done0 && P.done1)) break;
            const uint32_t j = bs + tid;
            uint32_t rid, slot = tid;
            if (rank_sort) {
                // the composites are unique (record indices differ): a splat's place is the
                // number of smaller composites in the tile
                const unsigned long long comp = j < range.y ? a.bucket[j] : ~0ull;
                s_comp[tid] = comp;
                __syncthreads();
                const uint32_t n = range.y - range.x;
                uint32_t r = 0;
                for (uint32_t i = 0; i < n; ++i) r += s_comp[i] < comp ? 1u : 0u;
                rid = 0xffffffffu;
                if (j < range.y) {
                    slot = r;
                    rid = (uint32_t)comp;
                    a.keys_w[range.x + r] = ((unsigned long long)t << 32) | (comp >> 32);
                    a.vals_w[range.x + r] = rid;
                }
            } else {
                rid = j < range.y ? __ldg(a.vals + j) : 0xffffffffu;
            }
            uint32_t mask = 0u;
            if ((int64_t)rid < a.n_records) {
                float4 r0, r1, r2, A, B, C;
                load_record(a.rec, rid, r0, r1, r2);
                stage_record(r0, r1, r2, oxh, oxl, oyh, oyl, A, B, C);
                C.w = __int_as_float((int)(bs - range.x + slot + 1));
                mask = cull_blocks<Cfg::WGX, Cfg::WARPS / Cfg::WGX>(cull_setup(A.x, A.y, A.z, A.w, B.x, B.z));
                float K, L;
                splat_KL(A.x, A.y, A.z, A.w, B.x, K, L);
                sR[slot][0] = make_float4(K, L, -A.z, -A.w);   // the mean enters only through K and L
                B.x = -B.x;
                sR[slot][1] = B;
                sR[slot][2] = C;
            }
            smask[slot] = mask;
            __syncthreads();
            int cnt = 0;
#pragma unroll
            for (int c = 0; c < Cfg::BATCH / 32; ++c) {
                const uint32_t bit = (smask[c * 32 + lane] >> w) & 1u;
                const uint32_t bal = __ballot_sync(FULL, bit);
                if (bit) slist[w][cnt + __popc(bal & lmask)] = (uint16_t)(c * 32 + lane);
                cnt += __popc(bal);
            }
            __syncwarp();
            if (!__all_sync(FULL, P.done0 && P.done1)) {
                if (COUNT) n_blk += cnt;
                int k = 0;
                // two splats per iteration, four iterations unrolled (fewer loop instructions)
#pragma unroll 4
                for (; k + 1 < cnt; k += 2) {
                    const int j0 = slist[w][k], j1 = slist[w][k + 1];
                    const float4 A0 = sR[j0][0], B0 = sR[j0][1], C0 = sR[j0][2];
                    const float4 A1 = sR[j1][0], B1 = sR[j1][1], C1 = sR[j1][2];
                    const float2 u0 = pair_u2v(A0, B0, pxc2, pyc);
                    const float2 u1 = pair_u2v(A1, B1, pxc2, pyc);
                    pix_update2<COUNT, LAST>(P, u0, B0, C0, n_blend);
                    pix_update2<COUNT, LAST>(P, u1, B1, C1, n_blend);
                }
                if (k < cnt) {
                    const int j0 = slist[w][k];
                    const float4 A0 = sR[j0][0], B0 = sR[j0][1], C0 = sR[j0][2];
                    pix_update2<COUNT, LAST>(P, pair_u2v(A0, B0, pxc2, pyc), B0, C0, n_blend);
                }
            }
        }
        if (LAST && a.tile_work) {
            // the reverse pass walks each block from its largest last position: its work estimate
            const uint32_t m = __reduce_max_sync(FULL, max(P.last0, P.last1));
            if (lane == 0) a.tile_work[t * Cfg::WARPS + w] = m;
        }
        n_eval += (in0 ? P.stop0 : 0u) + (in1 ? P.stop1 : 0u);
        const int64_t HW = (int64_t)V.w * V.h;
        const int64_t lp = (int64_t)py * V.w + px;
        const int64_t pix = V.pix_base + lp;
        float *rgb = a.rgb + 3 * V.pix_base;
        // both pixels at once when every plane's pair is 8-byte aligned
        const bool bases8 = ((reinterpret_cast<uintptr_t>(a.rgb) | reinterpret_cast<uintptr_t>(a.depth) |
                              reinterpret_cast<uintptr_t>(a.Tf) | reinterpret_cast<uintptr_t>(a.ncontrib)) & 7u) == 0;
        const bool pair = bases8 && in1 && ((3 * V.pix_base + lp) & 1) == 0 && (HW & 1) == 0 && (pix & 1) == 0;
        // (half-output plans address the same planes as binary16 arrays; rgb is then
        // a half pointer in float's clothing, offset by element counts below)
        using O = OutStore<HALF>;
        float *rgbv = HALF ? reinterpret_cast<float *>(reinterpret_cast<__half *>(a.rgb) + 3 * V.pix_base) : rgb;
        if (pair) {
            O::two(rgbv, lp, P.R);
            O::two(rgbv, HW + lp, P.G);
            O::two(rgbv, 2 * HW + lp, P.B);
            O::two(a.depth, pix, P.D);
            O::two(a.Tf, pix, P.T);
            if (LAST) *reinterpret_cast<uint2 *>(a.ncontrib + pix) = make_uint2(P.last0, P.last1);
        } else if (in0) {
            O::one(rgbv, lp, P.R.x);
            O::one(rgbv, HW + lp, P.G.x);
            O::one(rgbv, 2 * HW + lp, P.B.x);
            O::one(a.depth, pix, P.D.x);
            O::one(a.Tf, pix, P.T.x);
            if (LAST) a.ncontrib[pix] = P.last0;
        }
        if (in1 && !pair) {
            O::one(rgbv, lp + 1, P.R.y);
            O::one(rgbv, HW + lp + 1, P.G.y);
            O::one(rgbv, 2 * HW + lp + 1, P.B.y);
            O::one(a.depth, pix + 1, P.D.y);
            O::one(a.Tf, pix + 1, P.T.y);
            if (LAST) a.ncontrib[pix + 1] = P.last1;
        }
    }
    if (!COUNT) return;
    // algorithmic work counters: warp sums, one shared add per warp, one RED per CTA
    const uint32_t ev = __reduce_add_sync(FULL, n_eval), bl = __reduce_add_sync(FULL, n_blend);
    if (lane == 0 && (ev | bl | n_blk)) {
        atomicAdd(&s_cnt[0], (unsigned long long)ev);
        atomicAdd(&s_cnt[1], (unsigned long long)bl);
        atomicAdd(&s_cnt[2], (unsigned long long)n_blk);   // warp-uniform
    }
    __syncthreads();
    if (tid == 0 && (s_cnt[0] | s_cnt[1] | s_cnt[2])) {
        atomicAdd(&a.st->pair_evals, s_cnt[0]);
        atomicAdd(&a.st->pair_blends, s_cnt[1]);
        atomicAdd(&a.st->block_evals, s_cnt[2]);
    }
}

// ---------------------------------------------------------------------------
// Tile work order, heaviest first (a longest-processing-time-first schedule):
// tiles bucketed by a work estimate, four buckets per octave.  The estimate is
// the largest of a tile's wpt entries of work (the reverse pass: each warp's
// largest last blended position), else the tile's instance count.

__device__ __forceinline__ uint32_t tile_estimate(const uint2 *ranges, const uint32_t *work, int wpt, int64_t t)
{
    if (!work) return ranges[t].y - ranges[t].x;
    uint32_t m = 0;
    for (int i = 0; i < wpt; ++i) m = max(m, work[t * wpt + i]);
    return m;
}

__global__ void k_order_hist(const uint2 *ranges, const uint32_t *work, int wpt, int64_t n_tiles, uint32_t *hist,
                             const DevStatus *st)
{
    pdl_wait();
    pdl_trigger();
    if (st->flags & ST_CAPACITY) return;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tiles;
         t += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[order_bucket(tile_estimate(ranges, work, wpt, t))], 1u);
}

__global__ void k_order_scatter(const uint2 *ranges, const uint32_t *work, int wpt, int64_t n_tiles,
                                const uint32_t *hist, uint32_t *cursor, uint32_t *order, const DevStatus *st)
{
    pdl_wait();
    pdl_trigger();
    if (st->flags & ST_CAPACITY) return;
    // bucket b starts after every heavier bucket's tiles: the histogram is read once into
    // shared memory, then each bucket's start is summed by its own thread
    __shared__ uint32_t h[kOrderBuckets], start[kOrderBuckets];
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) h[b] = hist[b];
    __syncthreads();
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) {
        uint32_t acc = 0;
        for (int q = b + 1; q < kOrderBuckets; ++q) acc += h[q];
        start[b] = acc;
    }
    __syncthreads();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = order_bucket(tile_estimate(ranges, work, wpt, t));
        order[start[b] + atomicAdd(&cursor[b], 1u)] = (uint32_t)t;
    }
}

// order_tmp: [kOrderBuckets] histogram + [kOrderBuckets] cursors, cleared here unless
// the caller has (clear_tmp = false: cleared earlier in the stream).
cudaError_t launch_tile_order(const uint2 *ranges, const uint32_t *work, int wpt, int64_t n_tiles,
                              const DevStatus *st, uint32_t *order, uint32_t *order_tmp, int n_sms, bool clear_tmp,
                              cudaStream_t s)
{
    cudaError_t e;
    if (clear_tmp) {
        e = cudaMemsetAsync(order_tmp, 0, sizeof(uint32_t) * 2 * kOrderBuckets, s);
        if (e != cudaSuccess) return e;
    }
    const dim3 g(n_sms * 4), b(256);
    e = launch_pdl(k_order_hist, g, b, 0, s, ranges, work, wpt, n_tiles, order_tmp, st);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_order_scatter, g, b, 0, s, ranges, work, wpt, n_tiles, (const uint32_t *)order_tmp,
                      order_tmp + kOrderBuckets, order, st);
}

template <int TS, bool PERSIST>
static cudaError_t launch_fwd_tsp(const ViewTable &vt, const FwdArgs &a, int grid, bool count, cudaStream_t s)
{
    // the last-blended-position plane is written only when the caller keeps it
    constexpr int T = BlendCfg<TS>::THREADS;
    if (a.half_out) k_render_fwd<TS, false, false, PERSIST, true><<<grid, T, 0, s>>>(vt, a);
    else if (count && a.ncontrib) k_render_fwd<TS, true, true, PERSIST><<<grid, T, 0, s>>>(vt, a);
    else if (count) k_render_fwd<TS, true, false, PERSIST><<<grid, T, 0, s>>>(vt, a);
    else if (a.ncontrib) k_render_fwd<TS, false, true, PERSIST><<<grid, T, 0, s>>>(vt, a);
    else k_render_fwd<TS, false, false, PERSIST><<<grid, T, 0, s>>>(vt, a);
    return cudaGetLastError();
}

// The persistent schedule is a separate instantiation, so that the per-tile
// grid carries none of its work-queue code.
template <int TS>
static cudaError_t launch_fwd_ts(const ViewTable &vt, const FwdArgs &a, int grid, bool count, cudaStream_t s)
{
    return a.persistent ? launch_fwd_tsp<TS, true>(vt, a, grid, count, s)
                        : launch_fwd_tsp<TS, false>(vt, a, grid, count, s);
}

// CTAs of the persistent instantiation that fit on one SM at once.
template <int TS>
static int resident_ctas_ts(bool count, bool last, bool half)
{
    int n = 0;
    cudaError_t e;
    constexpr int T = BlendCfg<TS>::THREADS;
    if (half) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_render_fwd<TS, false, false, true, true>, T, 0);
    else if (count && last) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_render_fwd<TS, true, true, true>, T, 0);
    else if (count) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_render_fwd<TS, true, false, true>, T, 0);
    else if (last) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_render_fwd<TS, false, true, true>, T, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_render_fwd<TS, false, false, true>, T, 0);
    if (e != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

static int resident_ctas(int tile, bool count, bool last, bool half)
{
    switch (tile) {
        case 8: return resident_ctas_ts<8>(count, last, half);
        case 32: return resident_ctas_ts<32>(count, last, half);
        default: return resident_ctas_ts<16>(count, last, half);
    }
}

cudaError_t launch_render_fwd(const ViewTable &vt, const float4 *viewtab, const float4 *rec,
                              const uint32_t *vals, const uint2 *ranges, DevStatus *st, float *rgb,
                              float *depth, float *Tf, uint32_t *ncontrib, uint32_t *tile_work, uint32_t *order,
                              uint32_t *order_tmp, int64_t n_tiles, int64_t n_records,
                              unsigned long long cap, int persistent, int count, int half_out,
                              int tiles_per_pull, const unsigned long long *bucket,
                              unsigned long long *keys_w, uint32_t *vals_w, uint32_t blend_max, int n_sms,
                              cudaStream_t s)
{
    FwdArgs a;
    a.bucket = bucket;
    a.keys_w = keys_w;
    a.vals_w = vals_w;
    a.blend_max = blend_max;
    a.half_out = half_out;
    a.tiles_per_pull = tiles_per_pull < 1 ? 1 : tiles_per_pull;
    a.cap = cap;
    a.viewtab = viewtab;
    a.rec = rec;
    a.vals = vals;
    a.ranges = ranges;
    a.st = st;
    a.rgb = rgb;
    a.depth = depth;
    a.Tf = Tf;
    a.ncontrib = ncontrib;
    a.tile_work = ncontrib ? tile_work : nullptr;
    a.order = order;
    a.n_tiles = n_tiles;
    a.n_records = n_records;
    a.persistent = persistent;
    int grid = (int)n_tiles;
    cudaError_t e;
    if (persistent) {
        e = cudaMemsetAsync(&st->work[0], 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
        if (persistent == 1) {
            e = launch_tile_order(ranges, nullptr, 0, n_tiles, st, order, order_tmp, n_sms, true, s);
            if (e != cudaSuccess) return e;
        } else {
            a.order = nullptr;           // tile order: neighbouring tiles run together
        }
        // one resident wave of CTAs pulling tiles
        const int per_sm = resident_ctas(vt.tile, count != 0, ncontrib != nullptr, half_out != 0);
        const int64_t ctas = (int64_t)n_sms * per_sm;
        grid = (int)(ctas < n_tiles ? ctas : n_tiles);
    }
    if (grid <= 0) return cudaSuccess;
    switch (vt.tile) {
        case 8: return launch_fwd_ts<8>(vt, a, grid, count != 0, s);
        case 16: return launch_fwd_ts<16>(vt, a, grid, count != 0, s);
        case 32: return launch_fwd_ts<32>(vt, a, grid, count != 0, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vrs
