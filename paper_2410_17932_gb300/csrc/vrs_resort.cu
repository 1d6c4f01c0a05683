// Step 3 with the per-pixel depth order: the popping fix of Sec. 3.2, which
// sorts the Gaussian contributions per pixel instead of per primitive.
//
// Each pixel orders the splats it blends by t*, the camera-space depth of the
// 3D Gaussian's density maximum along the pixel's ray, and accumulates Eq. 1
// with d_i = t*.  The tile's list arrives sorted by t* at the tile's centre
// (clamped into each splat's footprint), which is close to each pixel's order;
// the pixel holds the K nearest splats it has not blended yet in a window in
// shared memory (a sorted ring of t* keys with premultiplied colours) and
// blends the nearest one whenever a new splat would overfill it.  A splat that
// arrives nearer than one the pixel has already blended, or than the one it
// stopped at, cannot be put back in order: the pixel is flagged.  An unflagged pixel has blended exactly the prefix of its
// per-pixel order that the stop rule admits.  Pixels keep checking arrivals
// after they stop, so the per-tile early exit is not taken.
//
// CTA and warp layout, staging and block culling are the per-tile blend's: one
// CTA per tile, each warp an 8x8 block, each lane two horizontally adjacent
// pixels; staged splats also carry the four terms per axis of t*.
#include "vrs_internal.cuh"

namespace vrs {

struct ResortArgs {
    const float4 *viewtab;
    const float4 *rec;
    const float4 *raydepth;     // 3 float4 per record: (e_kx/(fx s_k), e_ky/(fy s_k), e_kz/s_k, b_k)
    const uint32_t *vals;
    const uint2 *ranges;
    DevStatus *st;
    float *rgb;
    float *depth;
    float *Tf;
    uint8_t *flags;
    int64_t n_records;
    unsigned long long cap;
    int half_out;
};

// Order-preserving map of a float to an unsigned integer, and back.
__device__ __forceinline__ uint32_t fkey(float t)
{
    const uint32_t b = __float_as_uint(t);
    return b ^ ((b & 0x80000000u) ? 0xffffffffu : 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k)
{
    return __uint_as_float(k ^ ((k & 0x80000000u) ? 0x80000000u : 0xffffffffu));
}

// One pixel's compositing state and its window, a sorted ring in shared memory
// of (key, premultiplied colour and alpha) entries: key = fkey(t*), the colour
// alpha (r, g, b) and alpha.  The head (nearest) and tail (farthest) keys are
// kept in registers, so that an arrival in order touches shared memory only to
// store itself and to read the entry it pushes out.  Exact ties of t* keep
// their arrival order.
struct RsPix {
    float T, R, G, B, D;
    uint32_t last;             // key of the last blended splat, or of the one the pixel stopped at
    uint32_t hk, tk;           // keys at the head and the tail of the ring
    int head, n;
    bool done, flag;
};

template <int K>
struct RsWin {
    uint32_t *key;             // [K][stride]
    float4 *col;               // [K][stride]: (alpha r, alpha g, alpha b, alpha)
    int stride;
};

__device__ __forceinline__ void rs_blend(RsPix &P, uint32_t key, float4 c)
{
    const float Tn = P.T * (1.0f - c.w);
    P.last = key;
    if (Tn < 1e-4f) {
        P.done = true;
        return;
    }
    P.R = fmaf(c.x, P.T, P.R);
    P.G = fmaf(c.y, P.T, P.G);
    P.B = fmaf(c.z, P.T, P.B);
    P.D = fmaf(fkey_inv(key) * c.w, P.T, P.D);
    P.T = Tn;
}

// A splat reaches the pixel with alpha >= 1/255: order check, then window.
template <int K>
__device__ __forceinline__ void rs_push(RsPix &P, const RsWin<K> &W, int col, uint32_t key, float4 c)
{
    if (key < P.last) P.flag = true;
    if (P.done) return;
    if (P.n == K) {
        if (key < P.hk) {               // nearer than everything held: it goes first
            rs_blend(P, key, c);
            return;
        }
        rs_blend(P, P.hk, W.col[P.head * W.stride + col]);
        P.head = (P.head + 1) & (K - 1);
        P.n = K - 1;
        if (P.done) return;
        P.hk = W.key[P.head * W.stride + col];
    }
    if (P.n == 0 || key >= P.tk) {      // in order: append at the tail
        const int dst = ((P.head + P.n) & (K - 1)) * W.stride + col;
        W.key[dst] = key;
        W.col[dst] = c;
        if (P.n == 0) P.hk = key;
        P.tk = key;
        ++P.n;
        return;
    }
    // insertion from the far end of the ring
    int i = P.n;
    while (i > 0) {
        const int src = ((P.head + i - 1) & (K - 1)) * W.stride + col;
        const uint32_t kp = W.key[src];
        if (kp <= key) break;
        const int dst = ((P.head + i) & (K - 1)) * W.stride + col;
        W.key[dst] = kp;
        W.col[dst] = W.col[src];
        --i;
    }
    const int dst = ((P.head + i) & (K - 1)) * W.stride + col;
    W.key[dst] = key;
    W.col[dst] = c;
    if (i == 0) P.hk = key;
    ++P.n;
}

template <int K>
__device__ __forceinline__ void rs_drain(RsPix &P, const RsWin<K> &W, int col)
{
    while (P.n > 0 && !P.done) {
        const int h = P.head * W.stride + col;
        rs_blend(P, W.key[h], W.col[h]);
        P.head = (P.head + 1) & (K - 1);
        --P.n;
    }
}

__device__ __forceinline__ float2 f2r(float a) { return make_float2(a, a); }

template <int TS, int K, bool HALF>
__global__ void __launch_bounds__(BlendCfg<TS>::THREADS)
    k_render_resort(const __grid_constant__ ViewTable vt, const ResortArgs a)
{
    using Cfg = BlendCfg<TS>;
    constexpr int STRIDE = 2 * Cfg::THREADS;
    __shared__ float4 sR[Cfg::BATCH][3];   // staged splats: A, B, C as in the per-tile blend
    __shared__ float4 sD[Cfg::BATCH][3];   // per axis: (c0, c1, c2 in the tile frame, b)
    __shared__ uint32_t smask[Cfg::BATCH];
    __shared__ uint16_t slist[Cfg::WARPS][Cfg::BATCH];
    __shared__ unsigned long long s_flagged;
    extern __shared__ __align__(16) unsigned char s_win[];

    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int bx = (w % Cfg::WGX) * 8, by = (w / Cfg::WGX) * 8;
    const float pxc = (float)(bx + 2 * (lane & 3)) + 0.5f, pyc = (float)(by + (lane >> 2)) + 0.5f;
    const float2 pxc2 = make_float2(pxc, pxc + 1.0f);
    const uint32_t lmask = lanemask_lt();
    RsWin<K> Wn;
    Wn.col = reinterpret_cast<float4 *>(s_win);
    Wn.key = reinterpret_cast<uint32_t *>(s_win + sizeof(float4) * K * STRIDE);
    Wn.stride = STRIDE;
    if (tid == 0) s_flagged = 0ull;
    if (a.st->flags & ST_CAPACITY) return;

    const int64_t t = blockIdx.x;
    const int vi = view_of_tile(vt, t);
    const DevView &V = vt.v[vi];
    const float4 pp = a.viewtab[vi];
    int tx, ty;
    tile_xy(t - V.tile_base, V.gw, tx, ty);
    const int px = tx * TS + bx + 2 * (lane & 3), py = ty * TS + by + (lane >> 2);
    const bool in0 = px < V.w && py < V.h, in1 = px + 1 < V.w && py < V.h;
    float oxh, oxl, oyh, oyl;
    tile_origin((float)(tx * TS), pp.x, oxh, oxl);
    tile_origin((float)(ty * TS), pp.y, oyh, oyl);
    const float ox = oxh + oxl, oy = oyh + oyl;     // tile origin minus the principal point
    const uint2 range = live_range(a.ranges, t, a.st, a.cap);

    RsPix P0, P1;
    P0.T = P1.T = 1.f;
    P0.R = P0.G = P0.B = P0.D = P1.R = P1.G = P1.B = P1.D = 0.f;
    P0.last = P1.last = 0u;
    P0.hk = P0.tk = P1.hk = P1.tk = 0u;
    P0.head = P0.n = P1.head = P1.n = 0;
    P0.done = !in0;
    P1.done = !in1;
    P0.flag = P1.flag = false;

    for (uint32_t bs = range.x; bs < range.y; bs += Cfg::BATCH) {
        if (bs != range.x) __syncthreads();            // the previous batch is no longer read
        const uint32_t j = bs + tid;
        const uint32_t rid = j < range.y ? __ldg(a.vals + j) : 0xffffffffu;
        uint32_t mask = 0u;
        if ((int64_t)rid < a.n_records) {
            float4 r0, r1, r2, A, B, C;
            load_record(a.rec, rid, r0, r1, r2);
            stage_record(r0, r1, r2, oxh, oxl, oyh, oyl, A, B, C);
            mask = cull_blocks<Cfg::WGX, Cfg::WARPS / Cfg::WGX>(cull_setup(A.x, A.y, A.z, A.w, B.x, B.z));
            float Kc, Lc;
            splat_KL(A.x, A.y, A.z, A.w, B.x, Kc, Lc);
            sR[tid][0] = make_float4(Kc, Lc, -A.z, -A.w);
            B.x = -B.x;
            sR[tid][1] = B;
            sR[tid][2] = C;
            const float4 *rd = a.raydepth + (size_t)rid * 3;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float4 c = __ldg(rd + k);
                sD[tid][k] = make_float4(c.x, c.y, fmaf(c.x, ox, fmaf(c.y, oy, c.z)), c.w);
            }
        }
        smask[tid] = mask;
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
        for (int k = 0; k < cnt; ++k) {
            const int js = slist[w][k];
            const float4 A = sR[js][0], B = sR[js][1];
            // q' - lo at the two pixels, as the per-tile blend evaluates it
            const float s = __fmaf_rn(B.x, pyc, A.y);
            const float ww = __fmaf_rn(s, s, -B.y);
            const float r = __fmaf_rn(A.w, pyc, A.x);
            const float t0 = __fmaf_rn(A.z, pxc, r), t1 = __fmaf_rn(A.z, pxc + 1.0f, r);
            const float u0 = __fmaf_rn(t0, t0, ww), u1 = __fmaf_rn(t1, t1, ww);
            const bool h0 = in0 && u0 <= kLog2_255, h1 = in1 && u1 <= kLog2_255;
            if (!(h0 || h1)) continue;
            // t* at both pixels (packed): a_k = c0 x + c1 y + c2, t* = sum a_k b_k / sum a_k^2
            float2 nn = f2r(0.f), dd = f2r(0.f);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float4 c = sD[js][q];
                const float2 ak = __ffma2_rn(f2r(c.x), pxc2, f2r(fmaf(c.y, pyc, c.z)));
                nn = __ffma2_rn(ak, f2r(c.w), nn);
                dd = __ffma2_rn(ak, ak, dd);
            }
            const float2 tt = __fmul2_rn(nn, make_float2(rcp_approx(dd.x), rcp_approx(dd.y)));
            const float4 C = sR[js][2];
            if (h0) {
                const float al = fminf(ex2_approx(-u0), 0.99f);
                rs_push<K>(P0, Wn, tid, fkey(tt.x), make_float4(C.x * al, C.y * al, C.z * al, al));
            }
            if (h1) {
                const float al = fminf(ex2_approx(-u1), 0.99f);
                rs_push<K>(P1, Wn, Cfg::THREADS + tid, fkey(tt.y), make_float4(C.x * al, C.y * al, C.z * al, al));
            }
        }
    }
    rs_drain<K>(P0, Wn, tid);
    rs_drain<K>(P1, Wn, Cfg::THREADS + tid);

    const int64_t HW = (int64_t)V.w * V.h;
    const int64_t lp = (int64_t)py * V.w + px;
    const int64_t pix = V.pix_base + lp;
    using O = OutStore<HALF>;
    float *rgb = HALF ? reinterpret_cast<float *>(reinterpret_cast<__half *>(a.rgb) + 3 * V.pix_base)
                      : a.rgb + 3 * V.pix_base;
    if (in0) {
        O::one(rgb, lp, P0.R);
        O::one(rgb, HW + lp, P0.G);
        O::one(rgb, 2 * HW + lp, P0.B);
        O::one(a.depth, pix, P0.D);
        O::one(a.Tf, pix, P0.T);
        a.flags[pix] = P0.flag ? 1 : 0;
    }
    if (in1) {
        O::one(rgb, lp + 1, P1.R);
        O::one(rgb, HW + lp + 1, P1.G);
        O::one(rgb, 2 * HW + lp + 1, P1.B);
        O::one(a.depth, pix + 1, P1.D);
        O::one(a.Tf, pix + 1, P1.T);
        a.flags[pix + 1] = P1.flag ? 1 : 0;
    }
    const uint32_t nf = __reduce_add_sync(FULL, (in0 && P0.flag ? 1u : 0u) + (in1 && P1.flag ? 1u : 0u));
    if (lane == 0 && nf) atomicAdd(&s_flagged, (unsigned long long)nf);
    __syncthreads();
    if (tid == 0 && s_flagged) atomicAdd(&a.st->resort_flagged, s_flagged);
}

template <int TS, int K, bool HALF>
static cudaError_t launch_resort_tkh(const ViewTable &vt, const ResortArgs &a, int64_t n_tiles, cudaStream_t s)
{
    constexpr int T = BlendCfg<TS>::THREADS;
    const size_t smem = (size_t)K * 2 * T * (sizeof(float4) + sizeof(uint32_t));
    cudaError_t e = cudaFuncSetAttribute(k_render_resort<TS, K, HALF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_render_resort<TS, K, HALF><<<(unsigned)n_tiles, T, smem, s>>>(vt, a);
    return cudaGetLastError();
}

template <int TS, int K>
static cudaError_t launch_resort_tk(const ViewTable &vt, const ResortArgs &a, int64_t n_tiles, cudaStream_t s)
{
    return a.half_out ? launch_resort_tkh<TS, K, true>(vt, a, n_tiles, s)
                      : launch_resort_tkh<TS, K, false>(vt, a, n_tiles, s);
}

template <int TS>
static cudaError_t launch_resort_t(const ViewTable &vt, const ResortArgs &a, int64_t n_tiles, int window,
                                   cudaStream_t s)
{
    switch (window) {
        case 4: return launch_resort_tk<TS, 4>(vt, a, n_tiles, s);
        case 8: return launch_resort_tk<TS, 8>(vt, a, n_tiles, s);
        case 16:
            if (TS == 32) return cudaErrorInvalidValue;
            return launch_resort_tk<TS, (TS == 32 ? 8 : 16)>(vt, a, n_tiles, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_render_resort(const ViewTable &vt, const float4 *viewtab, const float4 *rec,
                                 const float4 *raydepth, const uint32_t *vals, const uint2 *ranges,
                                 DevStatus *st, float *rgb, float *depth, float *Tf, uint8_t *flags,
                                 int64_t n_tiles, int64_t n_records, unsigned long long cap, int window,
                                 int half_out, cudaStream_t s)
{
    ResortArgs a;
    a.half_out = half_out;
    a.viewtab = viewtab;
    a.rec = rec;
    a.raydepth = raydepth;
    a.vals = vals;
    a.ranges = ranges;
    a.st = st;
    a.rgb = rgb;
    a.depth = depth;
    a.Tf = Tf;
    a.flags = flags;
    a.n_records = n_records;
    a.cap = cap;
    cudaError_t e = cudaMemsetAsync(&st->resort_flagged, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n_tiles <= 0) return e;
    switch (vt.tile) {
        case 8: return launch_resort_t<8>(vt, a, n_tiles, window, s);
        case 16: return launch_resort_t<16>(vt, a, n_tiles, window, s);
        case 32: return launch_resort_t<32>(vt, a, n_tiles, window, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vrs
