// Step 1 of the periphery rasterizer: per Gaussian and per view of its scene,
// EWA projection with the 0.3 px dilation, 3-sigma screen radius,
// view-dependent SH colour (Sec. 3.1 "Naive Method": splats with opacity,
// colour and a covariance from scale and rotation, projected to screen), and
// emission of one (tile, depth) key per touched 16x16 tile (Sec. 1: tiling
// and sorting all primitives is the cost that grows with their number).
#include "vrs_internal.cuh"

namespace vrs {

struct PreParams {
    DevScene S;
    int32_t n_views;                 // views of this scene
    int8_t views[VRS_MAX_VIEWS];     // their indices in the view table
    float4 *rec;
    unsigned long long *keys;
    uint32_t *vals;
    uint32_t *tile_cnt;              // nullable: instances per tile (bucketed sort)
    DevStatus *st;
    unsigned long long cap;
};

// Per CTA of 128 Gaussians: (1) the coefficient rows are staged in shared
// memory, by one bulk copy (TMA, cp.async.bulk) per row when a row is a whole
// number of 16-byte chunks (SH degree 1 and 3) and by plain loads otherwise,
// so the copies overlap the FP32 decision path; (2) per view, every lane takes
// its Gaussian's integer decisions and the warp emits the tile keys; the
// visible (Gaussian, view) pairs are queued in shared memory; (3) the queue is
// drained densely, one pair per thread, to write the projected records.
// Only about a quarter of the pairs of a VR view are visible, so draining a
// compacted queue instead of running the record math in every warp with a
// visible lane cuts the issued instructions several-fold.
template <int K>
struct ShStage {
    static constexpr bool kBulk = (12 * K) % 16 == 0;
    static constexpr int kRow = kBulk ? 3 * K + 4 : 3 * K + 1;   // padded row (floats): 52 for SH-3
};

constexpr uint32_t kBulkWaitIters = 1u << 20;
constexpr int kPreThreads = 128;
constexpr int kViewChunk = 4;                       // views per queue round
constexpr int kPreWarps = kPreThreads / 32;
constexpr int kQueue = 32 * kViewChunk;             // per warp

struct PreItem {
    float n1, b, det, tz;
};

template <int K>
__global__ void __launch_bounds__(kPreThreads) k_preprocess(const __grid_constant__ ViewTable vt,
                                                            const __grid_constant__ PreParams p)
{
    using SS = ShStage<K>;
    __shared__ __align__(16) float sh_s[kPreThreads * SS::kRow];
    __shared__ float m_s[kPreThreads][3];
    __shared__ float lo_s[kPreThreads];
    __shared__ PreItem items[kPreWarps][kQueue];
    __shared__ uint8_t item_g[kPreWarps][kQueue];
    __shared__ uint8_t item_v[kPreWarps][kQueue];
    __shared__ __align__(8) uint64_t bar;
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x;
    const int g = blockIdx.x * kPreThreads + tid;
    const int lane = tid & 31, wp = tid >> 5;
    const bool in = g < p.S.n;
    const bool use_bulk = SS::kBulk && (reinterpret_cast<uintptr_t>(p.S.sh) & 15u) == 0;
    float *row = &sh_s[tid * SS::kRow];

    if (use_bulk) {
        if (tid == 0) {
            const int n_here = min(kPreThreads, p.S.n - (int)(blockIdx.x * kPreThreads));
            mbar_init(&bar, 1);
            mbar_arrive_expect_tx(&bar, (uint32_t)n_here * 12u * K);
        }
        __syncthreads();
        if (in) bulk_g2s(row, p.S.sh + (size_t)g * 3 * K, 12u * K, &bar);
    } else if (in) {
        const float *src = p.S.sh + (size_t)g * 3 * K;
        for (int i = 0; i < 3 * K; ++i) row[i] = __ldg(src + i);
    }

    float m[3] = {0.f, 0.f, 0.f}, ls[3] = {0.f, 0.f, 0.f}, q[4] = {1.f, 0.f, 0.f, 0.f};
    float logit = 0.f;
    bool ok = in;
    if (in) {
        m[0] = __ldg(p.S.means + 3 * g);
        m[1] = __ldg(p.S.means + 3 * g + 1);
        m[2] = __ldg(p.S.means + 3 * g + 2);
        ls[0] = __ldg(p.S.log_scales + 3 * g);
        ls[1] = __ldg(p.S.log_scales + 3 * g + 1);
        ls[2] = __ldg(p.S.log_scales + 3 * g + 2);
        if ((reinterpret_cast<uintptr_t>(p.S.quats) & 15u) == 0) {
            float4 qv = __ldg(reinterpret_cast<const float4 *>(p.S.quats) + g);
            q[0] = qv.x; q[1] = qv.y; q[2] = qv.z; q[3] = qv.w;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) q[i] = __ldg(p.S.quats + 4 * g + i);
        }
        logit = __ldg(p.S.logits + g);
        const float chk = m[0] + m[1] + m[2] + ls[0] + ls[1] + ls[2] + q[0] + q[1] + q[2] + q[3] + logit;
        if (!isfinite(chk)) ok = false;
    }
    GaussPre pre;
    bool zero_quat = false;
    if (ok && !gauss_pre(ls, q, pre)) {
        ok = false;
        zero_quat = true;
    }
    const bool nonfinite_params = in && !ok && !zero_quat;
    m_s[tid][0] = m[0];
    m_s[tid][1] = m[1];
    m_s[tid][2] = m[2];
    // log2(sigmoid(x)) = -log2(1 + e^-x)
    lo_s[tid] = logit >= 0.f ? -__log2f(1.0f + __expf(-logit)) : logit * 1.4426950408889634f - __log2f(1.0f + __expf(logit));
    bool sh_checked = false, nonfinite_sh = false, timed_out = false;

    __syncwarp();   // this warp's m_s, lo_s (and plainly loaded rows) are visible to its lanes
    for (int vc = 0; vc < p.n_views; vc += kViewChunk) {
        uint32_t qn = 0;   // this warp's queue of visible (Gaussian, view) pairs
        const int vend = min(p.n_views, vc + kViewChunk);
        for (int vi = vc; vi < vend; ++vi) {
            const DevView &V = vt.v[p.views[vi]];
            Decision d;
            d.visible = false;
            d.x0 = d.x1 = d.y0 = d.y1 = 0;
            d.tz = 0.f;
            if (ok) decide(V, pre, m[0], m[1], m[2], vt.tile, d);
            if (d.visible && !sh_checked) {
                // the coefficients are needed from here on: wait for them, check them
                if (use_bulk && !mbar_wait(&bar, 0, kBulkWaitIters)) {
                    timed_out = true;
                    ok = false;
                } else {
                    float shs = 0.f;
                    for (int i = 0; i < 3 * K; ++i) shs += row[i];
                    if (!isfinite(shs)) {
                        ok = false;
                        nonfinite_sh = true;
                    }
                }
                sh_checked = true;
                if (!ok) d.visible = false;
            }
            // queue the visible pair
            const uint32_t vb = __ballot_sync(FULL, d.visible);
            if (d.visible) {
                const uint32_t slot = qn + __popc(vb & lanemask_lt());
                items[wp][slot] = PreItem{d.n1, d.b, d.det, d.tz};
                item_g[wp][slot] = (uint8_t)lane;
                item_v[wp][slot] = (uint8_t)(vi - vc);
            }
            qn += __popc(vb);
            // warp-cooperative emission: one atomic per warp, coalesced key writes
            const uint32_t cnt = d.visible ? (uint32_t)((d.x1 - d.x0) * (d.y1 - d.y0)) : 0u;
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t total = __shfl_sync(FULL, incl, 31);
            if (total == 0) continue;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&p.st->instances, (unsigned long long)total);
            base = __shfl_sync(FULL, base, 0);
            const uint32_t excl = incl - cnt;
            const int nx = d.visible ? d.x1 - d.x0 : 1;
            const uint32_t dbits = __float_as_uint(d.tz);
            const uint32_t rid = (uint32_t)(V.rec_base + g);
            for (uint32_t k0 = 0; k0 < total; k0 += 32) {
                const uint32_t k = k0 + lane;
                int j = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    uint32_t v = __shfl_sync(FULL, incl, j + step - 1);
                    if (v <= k) j += step;
                }
                const uint32_t oex = __shfl_sync(FULL, excl, j);
                const int ox0 = __shfl_sync(FULL, d.x0, j);
                const int oy0 = __shfl_sync(FULL, d.y0, j);
                const int onx = __shfl_sync(FULL, nx, j);
                const uint32_t odb = __shfl_sync(FULL, dbits, j);
                const uint32_t orid = __shfl_sync(FULL, rid, j);
                if (k < total) {
                    const uint32_t local = k - oex;
                    const int ty = oy0 + (int)(local / (uint32_t)onx);
                    const int tx = ox0 + (int)(local % (uint32_t)onx);
                    const unsigned long long tid64 =
                        (unsigned long long)(V.tile_base + (int64_t)ty * V.gw + tx);
                    const unsigned long long pos = base + k;
                    if (pos < p.cap) {
                        p.keys[pos] = (tid64 << 32) | odb;
                        p.vals[pos] = orid;
                        if (p.tile_cnt) atomicAdd(p.tile_cnt + tid64, 1u);
                    }
                }
            }
            if (lane == 0 && base + total > p.cap) atomicOr(&p.st->flags, ST_CAPACITY);
        }
        __syncwarp();
        // the rows read below belong to this warp's Gaussians; their bulk copies are
        // complete once any lane of the CTA has seen the barrier's phase
        if (qn && use_bulk && !mbar_wait(&bar, 0, kBulkWaitIters)) timed_out = true;
        sh_checked = sh_checked || qn != 0;
        // drain the warp's queue: one visible (Gaussian, view) pair per lane
        for (uint32_t it = lane; it < qn && !timed_out; it += 32) {
            const PreItem I_ = items[wp][it];
            const int gl = wp * 32 + item_g[wp][it];
            const DevView &V = vt.v[p.views[vc + item_v[wp][it]]];
            const float mx = m_s[gl][0], my = m_s[gl][1], mz = m_s[gl][2];
            // 2D mean relative to the principal point, as an unevaluated double-float sum
            float xh, xl, yh, yl, zh, zl, uh, ul, vh, vl;
            dot3_plus(V.R[0], V.R[1], V.R[2], mx, my, mz, V.t[0], xh, xl);
            dot3_plus(V.R[3], V.R[4], V.R[5], mx, my, mz, V.t[1], yh, yl);
            dot3_plus(V.R[6], V.R[7], V.R[8], mx, my, mz, V.t[2], zh, zl);
            proj_ratio(V.fx, xh, xl, zh, zl, uh, ul);
            proj_ratio(V.fy, yh, yl, zh, zl, vh, vl);
            // Cholesky factors of the conic of [[n0+.3, b], [b, n1+.3]] with the
            // cancellation-free determinant of the decision path
            const float c = I_.n1 + 0.3f;
            const float rc = rsqrtf(c), rd = rsqrtf(I_.det);
            const float l0 = c * rc * rd * kCholScale;       // sqrt(c / det)
            const float l1 = -I_.b * rc * rd * kCholScale;   // -b / sqrt(c det)
            const float l2 = rc * kCholScale;                // 1 / sqrt(c)
            // colour from the view direction (camera centre = -R^T t)
            const float cc0 = -(V.R[0] * V.t[0] + V.R[3] * V.t[1] + V.R[6] * V.t[2]);
            const float cc1 = -(V.R[1] * V.t[0] + V.R[4] * V.t[1] + V.R[7] * V.t[2]);
            const float cc2 = -(V.R[2] * V.t[0] + V.R[5] * V.t[1] + V.R[8] * V.t[2]);
            float dx = mx - cc0, dy = my - cc1, dz = mz - cc2;
            const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
            dx *= inv; dy *= inv; dz *= inv;
            float Y[16];
            sh_basis(dx, dy, dz, K, Y);
            float col[3] = {0.5f, 0.5f, 0.5f};
            const float *sr = &sh_s[gl * SS::kRow];
            if constexpr (SS::kBulk) {
                const float4 *s4 = reinterpret_cast<const float4 *>(sr);
#pragma unroll
                for (int i = 0; i < 3 * K / 4; ++i) {
                    const float4 v4 = s4[i];
                    const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) col[(4 * i + e) % 3] += Y[(4 * i + e) / 3] * vv[e];
                }
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) col[ch] += Y[k] * sr[3 * k + ch];
            }
            float4 *r = p.rec + (size_t)(V.rec_base + blockIdx.x * kPreThreads + gl) * kRecF4;
            r[0] = make_float4(uh, vh, ul, vl);
            r[1] = make_float4(l0, l1, l2, lo_s[gl]);
            r[2] = make_float4(fmaxf(col[0], 0.f), fmaxf(col[1], 0.f), fmaxf(col[2], 0.f), I_.tz);
        }
        __syncwarp();
    }
    if (nonfinite_params || nonfinite_sh) atomicOr(&p.st->flags, ST_NONFINITE);
    if (zero_quat) atomicOr(&p.st->flags, ST_ZERO_QUAT);
    // the CTA's shared memory must outlive its bulk copies
    if (use_bulk && in && !sh_checked && !mbar_wait(&bar, 0, kBulkWaitIters)) timed_out = true;
    if (timed_out) atomicOr(&p.st->flags, ST_TIMEOUT);
}

// Principal points of the views, read by the blend kernels to build each
// tile's local frame (the plan holds sizes only).
__global__ void k_write_viewtab(const __grid_constant__ ViewTable vt, float4 *viewtab)
{
    const int v = threadIdx.x;
    if (v < vt.n_views) viewtab[v] = make_float4(vt.v[v].cx, vt.v[v].cy, 0.f, 0.f);
}

cudaError_t launch_write_viewtab(const ViewTable &vt, float4 *viewtab, cudaStream_t stream)
{
    k_write_viewtab<<<1, VRS_MAX_VIEWS, 0, stream>>>(vt, viewtab);
    return cudaGetLastError();
}

// Host launcher: one launch per scene (the SH degree is a template argument so
// that a Gaussian's coefficients stay in registers across its views).
cudaError_t launch_preprocess(const ViewTable &vt, const DevScene &S, const int8_t *views,
                              int n_views, float4 *rec, unsigned long long *keys, uint32_t *vals,
                              uint32_t *tile_cnt, DevStatus *st, unsigned long long cap,
                              cudaStream_t stream)
{
    if (S.n <= 0 || n_views <= 0) return cudaSuccess;
    PreParams p;
    p.S = S;
    p.n_views = n_views;
    for (int i = 0; i < VRS_MAX_VIEWS; ++i) p.views[i] = i < n_views ? views[i] : 0;
    p.rec = rec;
    p.keys = keys;
    p.vals = vals;
    p.tile_cnt = tile_cnt;
    p.st = st;
    p.cap = cap;
    const int block = kPreThreads;
    const unsigned grid = grid_for(S.n, block);
    switch (S.K) {
        case 1: k_preprocess<1><<<grid, block, 0, stream>>>(vt, p); break;
        case 4: k_preprocess<4><<<grid, block, 0, stream>>>(vt, p); break;
        case 9: k_preprocess<9><<<grid, block, 0, stream>>>(vt, p); break;
        case 16: k_preprocess<16><<<grid, block, 0, stream>>>(vt, p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace vrs
