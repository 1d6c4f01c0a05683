// Step 3: per-tile front-to-back alpha compositing of colour, the approximate
// depth of Eq. 1 (Sec. 3.2) and the final transmittance.
//
// One CTA owns one tile (TS x TS pixels); every thread owns two horizontally
// adjacent pixels and every warp an 8x8 block.  The tile's sorted instances are
// staged in batches of one per thread: the staging thread gathers the 48-byte
// record, moves the 2D mean into the tile-local frame (double-float, so that a
// 2016-pixel-wide view keeps sub-1e-5 px positions), and tests the splat's
// alpha >= 1/255 ellipse against each warp's 8x8 block.  Each warp then
// compacts the batch to the splats that can reach its block (ballot + popc,
// order preserved) and evaluates only those.  A warp that has finished all its
// pixels skips the evaluation; the CTA leaves when every pixel has stopped.
// The culling is conservative (only pairs with alpha < 1/255 for certain are
// skipped), so the image is the same as without it.
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
    const uint32_t *order;      // persistent: tile work order (heaviest first)
    int64_t n_tiles;
    int64_t n_records;
    int persistent;
};

template <int TS>
__global__ void __launch_bounds__(BlendCfg<TS>::THREADS)
    k_render_fwd(const __grid_constant__ ViewTable vt, const FwdArgs a)
{
    using Cfg = BlendCfg<TS>;
    __shared__ float4 sA[Cfg::BATCH], sB[Cfg::BATCH], sC[Cfg::BATCH];
    __shared__ uint32_t smask[Cfg::BATCH];
    __shared__ uint16_t slist[Cfg::WARPS][Cfg::BATCH];
    __shared__ int64_t s_tile;
    __shared__ unsigned long long s_cnt[2];

    if (a.st->flags & ST_CAPACITY) return;
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int px_l = (w % Cfg::WGX) * 8 + 2 * (lane & 3);
    const int py_l = (w / Cfg::WGX) * 8 + (lane >> 2);
    const float pxc = (float)px_l + 0.5f, pyc = (float)py_l + 0.5f;
    const uint32_t lmask = lanemask_lt();
    if (tid == 0) s_cnt[0] = s_cnt[1] = 0ull;
    uint32_t n_eval = 0, n_blend = 0;

    for (int64_t iter = 0;; ++iter) {
        int64_t t;
        if (a.persistent) {
            if (tid == 0) {
                const uint32_t k = atomicAdd(&a.st->work[0], 1u);
                s_tile = (int64_t)k < a.n_tiles ? (int64_t)a.order[k] : -1;
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
        const int tx = (int)(lt_ % V.gw), ty = (int)(lt_ / V.gw);
        const int px = tx * TS + px_l, py = ty * TS + py_l;
        const bool in0 = px < V.w && py < V.h, in1 = px + 1 < V.w && py < V.h;
        float oxh, oxl, oyh, oyl;
        tile_origin((float)(tx * TS), pp.x, oxh, oxl);
        tile_origin((float)(ty * TS), pp.y, oyh, oyl);
        const uint2 range = a.ranges[t];

        float T0 = 1.f, T1 = 1.f, D0 = 0.f, D1 = 0.f;
        float c0r = 0.f, c0g = 0.f, c0b = 0.f, c1r = 0.f, c1g = 0.f, c1b = 0.f;
        uint32_t last0 = 0, last1 = 0;
        uint32_t stop0 = range.y - range.x, stop1 = range.y - range.x;
        bool done0 = !in0, done1 = !in1;
        if (!in0) stop0 = 0;
        if (!in1) stop1 = 0;

        for (uint32_t bs = range.x; bs < range.y; bs += Cfg::BATCH) {
            if (__syncthreads_and(done0 && done1)) break;
            const uint32_t j = bs + tid;
            const uint32_t rid = j < range.y ? __ldg(a.vals + j) : 0xffffffffu;
            if ((int64_t)rid < a.n_records) {
                float4 A, B, C;
                smask[tid] = stage_instance<TS>(a.rec, rid, oxh, oxl, oyh, oyl, A, B, C);
                sA[tid] = A;
                sB[tid] = B;
                sC[tid] = C;
            } else {
                smask[tid] = 0u;
            }
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
            if (!__all_sync(FULL, done0 && done1)) {
                for (int k = 0; k < cnt; ++k) {
                    const int jj = slist[w][k];
                    const float4 A = sA[jj];
                    const float4 B = sB[jj];
                    float q0, q1;
                    pair_q2(A.x, A.y, A.z, A.w, B.x, pxc, pyc, q0, q1);
                    const bool h0 = !done0 && q0 <= B.z;
                    const bool h1 = !done1 && q1 <= B.z;
                    if (h0 || h1) {
                        const float4 C = sC[jj];
                        const uint32_t pos = bs + jj + 1 - range.x;
                        if (h0) {
                            const float al = pair_alpha(B.y, q0);
                            const float Tn = T0 * (1.f - al);
                            if (Tn < 1e-4f) {
                                done0 = true;
                                stop0 = pos;
                            } else {
                                ++n_blend;
                                const float wt = al * T0;
                                c0r = fmaf(C.x, wt, c0r);
                                c0g = fmaf(C.y, wt, c0g);
                                c0b = fmaf(C.z, wt, c0b);
                                D0 = fmaf(B.w, wt, D0);
                                T0 = Tn;
                                last0 = pos;
                            }
                        }
                        if (h1) {
                            const float al = pair_alpha(B.y, q1);
                            const float Tn = T1 * (1.f - al);
                            if (Tn < 1e-4f) {
                                done1 = true;
                                stop1 = pos;
                            } else {
                                ++n_blend;
                                const float wt = al * T1;
                                c1r = fmaf(C.x, wt, c1r);
                                c1g = fmaf(C.y, wt, c1g);
                                c1b = fmaf(C.z, wt, c1b);
                                D1 = fmaf(B.w, wt, D1);
                                T1 = Tn;
                                last1 = pos;
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
        n_eval += stop0 + stop1;
        const int64_t HW = (int64_t)V.w * V.h;
        const int64_t pix = V.pix_base + (int64_t)py * V.w + px;
        float *rgb = a.rgb + 3 * V.pix_base;
        const int64_t lp = (int64_t)py * V.w + px;
        if (in0) {
            rgb[lp] = c0r;
            rgb[HW + lp] = c0g;
            rgb[2 * HW + lp] = c0b;
            a.depth[pix] = D0;
            a.Tf[pix] = T0;
            a.ncontrib[pix] = last0;
        }
        if (in1) {
            rgb[lp + 1] = c1r;
            rgb[HW + lp + 1] = c1g;
            rgb[2 * HW + lp + 1] = c1b;
            a.depth[pix + 1] = D1;
            a.Tf[pix + 1] = T1;
            a.ncontrib[pix + 1] = last1;
        }
    }
    // algorithmic work counters: one reduction and one RED per CTA
    const uint32_t ev = __reduce_add_sync(FULL, n_eval), bl = __reduce_add_sync(FULL, n_blend);
    __syncthreads();
    if (lane == 0) {
        atomicAdd(&s_cnt[0], (unsigned long long)ev);
        atomicAdd(&s_cnt[1], (unsigned long long)bl);
    }
    __syncthreads();
    if (tid == 0) {
        atomicAdd(&a.st->pair_evals, s_cnt[0]);
        atomicAdd(&a.st->pair_blends, s_cnt[1]);
    }
}

// ---------------------------------------------------------------------------
// Work order for the persistent launch: tiles bucketed by floor(log2(count)),
// heaviest bucket first (a longest-processing-time-first schedule).

constexpr int kBuckets = 34;

__global__ void k_order_hist(const uint2 *ranges, int64_t n_tiles, uint32_t *hist, const DevStatus *st)
{
    if (st->flags & ST_CAPACITY) return;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = ranges[t].y - ranges[t].x;
        const int b = c == 0 ? 0 : 33 - __clz(c);
        atomicAdd(&hist[b], 1u);
    }
}

__global__ void k_order_scatter(const uint2 *ranges, int64_t n_tiles, const uint32_t *hist,
                                uint32_t *cursor, uint32_t *order, const DevStatus *st)
{
    if (st->flags & ST_CAPACITY) return;
    __shared__ uint32_t start[kBuckets];
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int b = kBuckets - 1; b >= 0; --b) {
            start[b] = acc;
            acc += hist[b];
        }
    }
    __syncthreads();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = ranges[t].y - ranges[t].x;
        const int b = c == 0 ? 0 : 33 - __clz(c);
        order[start[b] + atomicAdd(&cursor[b], 1u)] = (uint32_t)t;
    }
}

template <int TS>
static cudaError_t launch_fwd_ts(const ViewTable &vt, const FwdArgs &a, int grid, cudaStream_t s)
{
    k_render_fwd<TS><<<grid, BlendCfg<TS>::THREADS, 0, s>>>(vt, a);
    return cudaGetLastError();
}

cudaError_t launch_render_fwd(const ViewTable &vt, const float4 *viewtab, const float4 *rec,
                              const uint32_t *vals, const uint2 *ranges, DevStatus *st, float *rgb,
                              float *depth, float *Tf, uint32_t *ncontrib, uint32_t *order,
                              uint32_t *order_tmp, int64_t n_tiles, int64_t n_records,
                              int persistent, int n_sms, cudaStream_t s)
{
    FwdArgs a;
    a.n_records = n_records;
    a.viewtab = viewtab;
    a.rec = rec;
    a.vals = vals;
    a.ranges = ranges;
    a.st = st;
    a.rgb = rgb;
    a.depth = depth;
    a.Tf = Tf;
    a.ncontrib = ncontrib;
    a.order = order;
    a.n_tiles = n_tiles;
    a.persistent = persistent;
    int grid = (int)n_tiles;
    cudaError_t e;
    if (persistent) {
        // order_tmp: [kBuckets] histogram + [kBuckets] cursors
        e = cudaMemsetAsync(order_tmp, 0, sizeof(uint32_t) * 2 * kBuckets, s);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(&st->work[0], 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
        const int g = n_sms * 4;
        k_order_hist<<<g, 256, 0, s>>>(ranges, n_tiles, order_tmp, st);
        k_order_scatter<<<g, 256, 0, s>>>(ranges, n_tiles, order_tmp, order_tmp + kBuckets, order, st);
        const int per_sm = vt.tile == 8 ? 16 : (vt.tile == 16 ? 8 : 2);
        grid = (int)((int64_t)n_sms * per_sm < n_tiles ? (int64_t)n_sms * per_sm : n_tiles);
    }
    if (grid <= 0) return cudaSuccess;
    switch (vt.tile) {
        case 8: return launch_fwd_ts<8>(vt, a, grid, s);
        case 16: return launch_fwd_ts<16>(vt, a, grid, s);
        case 32: return launch_fwd_ts<32>(vt, a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vrs
