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
    int32_t scene;                   // index of S in the plan
    int32_t n_views;                 // views of this scene
    int8_t views[VRS_MAX_VIEWS];     // their indices in the view table
    uint4 *pairs;                    // this scene's visible-pair list (2 uint4 per pair)
    unsigned long long pair_cap;     // entries the list holds (n x n_views)
    float4 *rec;
    unsigned long long *keys;
    uint32_t *vals;
    uint32_t *tile_cnt;              // nullable: instances per tile (bucketed sort)
    DevStatus *st;
    unsigned long long cap;
    float4 *viewtab;                 // [VRS_MAX_VIEWS] principal points, written by the decision kernel's first CTA
    int64_t zero_tiles;              // > 0: the decision kernel clears tile_cnt[0, zero_tiles) (the frame's first
                                     // scene, before any pair kernel counts into it)
    float4 *raydepth;                // nullable (per-pixel order plans): 3 float4 per record
};

// The step runs as two kernels per scene.
//
// k_decide_listed reads only the 44 bytes of geometry per Gaussian (mean,
// log-scales, quaternion, opacity logit), applies the parameter rules, screens
// every (Gaussian, view) pair with a cheap conservative bound of the splat's
// extent, and the CTA's threads take the exact FP32 integer decisions of the
// pairs the bound keeps densely, from a candidate list in shared memory; each
// visible pair is appended to a list with the decision values the record needs
// (one slot atomic per CTA and round).  Only a fraction of a view's pairs is
// visible (a quarter in a VR eye, 6 % in the training view) and the scene's
// Gaussians are not ordered in space, so deciding every pair in place would run
// the exact path on nearly every warp; the list also makes the second kernel
// walk the visible pairs, not the scene.
//
// k_pairs walks the list, one pair per thread: it reads the pair's SH row
// (only visible Gaussians' colour coefficients are ever read), checks it,
// evaluates the view-dependent colour, writes the projected record and emits
// the pair's tile keys cooperatively across the warp (prefix sum of the
// per-lane counts, one atomic per CTA for the slots, coalesced key writes).
constexpr int kDecideThreads = 256;
constexpr int kPairThreads = 128;

// The conservative bound of a splat's screen extent that screens the (Gaussian,
// view) pairs before the exact path: Sigma' = V V^T + 0.3 I with V = (J W)(R S),
// so the eigenvalue the radius takes (at most the trace plus sqrt(0.1), as the
// discriminant is floored at 0.1) is below (|J_0|^2 + |J_1|^2) s_max^2 + 0.92,
// with |J_0|^2 = (fx/z)^2 (1 + x'^2) for the clamped x' = x/z; the radius
// ceil(3 sqrt(lambda)) is then below 3 sqrt(trace bound) + 1.  The bound adds 1 %
// and 1 px more than FP32 rounding needs, and the rectangle clipped to the alpha
// box only shrinks.  The camera-space depth is the exact path's own sequence, so
// the near-plane test is the same.  True: the exact path could find the pair
// visible; false: its rectangle would be empty.
__device__ __forceinline__ bool may_touch_grid(const DevView &V, int tile, float mx, float my, float mz,
                                               float s2)
{
    float tc[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float a_ = __fmul_rn(V.R[3 * r], mx);
        a_ = __fadd_rn(a_, __fmul_rn(V.R[3 * r + 1], my));
        a_ = __fadd_rn(a_, __fmul_rn(V.R[3 * r + 2], mz));
        tc[r] = __fadd_rn(a_, V.t[r]);
    }
    if (!(tc[2] > V.znear)) return false;
    const float iz = rcp_approx(tc[2]);           // approximations: the bound has 1 % margins
    const float rx = tc[0] * iz, ry = tc[1] * iz;
    const float limx = 1.3f * V.tanx, limy = 1.3f * V.tany;
    const float cx_ = fminf(limx, fmaxf(-limx, rx)), cy_ = fminf(limy, fmaxf(-limy, ry));
    const float jx = V.fx * iz, jy = V.fy * iz;
    const float tr = (jx * jx * (1.f + cx_ * cx_) + jy * jy * (1.f + cy_ * cy_)) * s2 + 1.0f;
    const float R = 3.03f * sqrt_approx(tr) + 2.0f;
    const float u = V.fx * rx + V.cx, v = V.fy * ry + V.cy;
    const float gx = (float)(V.gw * tile), gy = (float)(V.gh * tile);
    // written so that a NaN (from an overflowing mean) keeps the pair for the exact path
    return !(u + R < 0.f || u - R >= gx || v + R < 0.f || v - R >= gy);
}

// The exact FP32 decisions of pair (Gaussian cg, view vi of the scene), from the
// parameters or their baked form (decide_op: the only definition of visibility,
// radius and rectangle).  The caller has applied the parameter rules.
__device__ __forceinline__ void decide_pair(const ViewTable &vt, const PreParams &p, int cg, int vi, Decision &d)
{
    const float mx = __ldg(p.S.means + 3 * cg), my = __ldg(p.S.means + 3 * cg + 1);
    const float mz = __ldg(p.S.means + 3 * cg + 2);
    GaussPre pre;
    float op;
    if (p.S.baked) {
        // the scales, rotation and opacity gauss_pre and decision_opacity compute, bit for bit
        const float4 b0 = __ldg(p.S.baked + 4 * cg), b1 = __ldg(p.S.baked + 4 * cg + 1);
        const float4 b2 = __ldg(p.S.baked + 4 * cg + 2), b3 = __ldg(p.S.baked + 4 * cg + 3);
        pre.s[0] = b0.x; pre.s[1] = b0.y; pre.s[2] = b0.z;
        pre.Rq[0] = b0.w; pre.Rq[1] = b1.x; pre.Rq[2] = b1.y; pre.Rq[3] = b1.z; pre.Rq[4] = b1.w;
        pre.Rq[5] = b2.x; pre.Rq[6] = b2.y; pre.Rq[7] = b2.z; pre.Rq[8] = b2.w;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) pre.M[3 * k + j] = __fmul_rn(pre.Rq[3 * k + j], pre.s[j]);
        op = b3.x;
    } else {
        float ls[3], q[4];
#pragma unroll
        for (int k = 0; k < 3; ++k) ls[k] = __ldg(p.S.log_scales + 3 * cg + k);
        if ((reinterpret_cast<uintptr_t>(p.S.quats) & 15u) == 0) {
            const float4 qv = __ldg(reinterpret_cast<const float4 *>(p.S.quats) + cg);
            q[0] = qv.x; q[1] = qv.y; q[2] = qv.z; q[3] = qv.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = __ldg(p.S.quats + 4 * cg + k);
        }
        gauss_pre(ls, q, pre);                    // the rules have excluded a zero quaternion
        op = decision_opacity(__ldg(p.S.logits + cg));
    }
    decide_op(vt.v[p.views[vi]], pre, mx, my, mz, op, vt.tile, d);
}

// Appends the visible pairs of one round (every thread of the CTA calls it, with
// d.visible false where it has none): one slot atomic per CTA and round.
__device__ __forceinline__ void append_visible(const PreParams &p, const Decision &d, int cg, int vi,
                                               uint32_t *s_cnt, unsigned long long *s_base)
{
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const uint32_t vb = __ballot_sync(0xffffffffu, d.visible);
    if (lane == 0) s_cnt[wp] = __popc(vb);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long sum = 0;
        for (int w = 0; w < kDecideThreads / 32; ++w) sum += s_cnt[w];
        unsigned long long b = sum ? atomicAdd(&p.st->scene_pairs[p.scene], sum) : 0ull;
        for (int w = 0; w < kDecideThreads / 32; ++w) {
            s_base[w] = b;
            b += s_cnt[w];
        }
    }
    __syncthreads();
    if (d.visible) {
        const unsigned long long slot = s_base[wp] + __popc(vb & lanemask_lt());
        if (slot < p.pair_cap) {
            uint4 *e = p.pairs + 2 * slot;
            e[0] = make_uint4((uint32_t)cg, (uint32_t)vi, (uint32_t)d.x0 | ((uint32_t)d.x1 << 16),
                              (uint32_t)d.y0 | ((uint32_t)d.y1 << 16));
            e[1] = make_uint4(__float_as_uint(d.n1), __float_as_uint(d.b), __float_as_uint(d.det),
                              __float_as_uint(d.tz));
        }
    }
    // (a later round's counts are written only after every thread has passed the
    // second barrier above, so no third one is needed)
}

constexpr int kViewChunk = 4;       // views screened per candidate list

// The parameter rules of Gaussian g (non-finite values, the all-zero
// quaternion; flagged in the status block when `flag`) and what the screening
// bound needs: the mean and 1.01 x the largest scale squared.  False when the
// rules exclude the Gaussian.
__device__ __forceinline__ bool gauss_rules(const PreParams &p, int g, bool flag, float (&m)[3], float &s2)
{
    m[0] = __ldg(p.S.means + 3 * g);
    m[1] = __ldg(p.S.means + 3 * g + 1);
    m[2] = __ldg(p.S.means + 3 * g + 2);
    // x * 0 is 0 for every finite x and NaN for an infinity or a NaN, so the sum of
    // those products is finite exactly when every parameter is (a plain sum of the
    // values could overflow on large finite ones)
    float chk = __fmaf_rn(m[0], 0.f, __fmaf_rn(m[1], 0.f, __fmaf_rn(m[2], 0.f, 0.f)));
    bool ok, zero_quat = false;
    float smax;
    if (p.S.baked) {
        // baked attributes (vrs_bake) carry the rules' outcome in their status word
        const float4 b0 = __ldg(p.S.baked + 4 * g), b3 = __ldg(p.S.baked + 4 * g + 3);
        const uint32_t bst = __float_as_uint(b3.z);
        smax = fmaxf(b0.x, fmaxf(b0.y, b0.z));
        zero_quat = (bst & 1u) != 0;
        ok = isfinite(chk) && bst == 0u;
    } else {
        float ls[3], q[4];
#pragma unroll
        for (int i = 0; i < 3; ++i) ls[i] = __ldg(p.S.log_scales + 3 * g + i);
        if ((reinterpret_cast<uintptr_t>(p.S.quats) & 15u) == 0) {
            const float4 qv = __ldg(reinterpret_cast<const float4 *>(p.S.quats) + g);
            q[0] = qv.x; q[1] = qv.y; q[2] = qv.z; q[3] = qv.w;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) q[i] = __ldg(p.S.quats + 4 * g + i);
        }
        const float logit = __ldg(p.S.logits + g);
#pragma unroll
        for (int i = 0; i < 3; ++i) chk = __fmaf_rn(ls[i], 0.f, chk);
#pragma unroll
        for (int i = 0; i < 4; ++i) chk = __fmaf_rn(q[i], 0.f, chk);
        chk = __fmaf_rn(logit, 0.f, chk);
        ok = isfinite(chk);
        if (ok) {
            // the zero-quaternion rule, with gauss_pre's own |q|^2
            float qq = __fmul_rn(q[0], q[0]);
            qq = __fadd_rn(qq, __fmul_rn(q[1], q[1]));
            qq = __fadd_rn(qq, __fmul_rn(q[2], q[2]));
            qq = __fadd_rn(qq, __fmul_rn(q[3], q[3]));
            zero_quat = !(qq > 0.0f);
            ok = !zero_quat;
        }
        smax = __expf(fmaxf(ls[0], fmaxf(ls[1], ls[2])));
    }
    if (flag && !ok && !zero_quat) atomicOr(&p.st->flags, ST_NONFINITE);
    if (flag && zero_quat) atomicOr(&p.st->flags, ST_ZERO_QUAT);
    s2 = smax * smax * 1.01f;
    return ok;
}

// Gaussians per thread of the listed decision kernel: one CTA screens
// kDecideThreads x PER Gaussians into one candidate list, so the latency of the
// exact path is paid once for all of them.
template <int PER>
__global__ void __launch_bounds__(kDecideThreads) k_decide_listed(const __grid_constant__ ViewTable vt,
                                                                  const __grid_constant__ PreParams p)
{
    pdl_wait();
    pdl_trigger();
    // the views' principal points, read by the blend kernels to build each
    // tile's local frame (the plan holds sizes only); every scene's launch
    // writes the same values
    if (blockIdx.x == 0 && threadIdx.x < vt.n_views)
        p.viewtab[threadIdx.x] = make_float4(vt.v[threadIdx.x].cx, vt.v[threadIdx.x].cy, 0.f, 0.f);
    for (int64_t t = (int64_t)blockIdx.x * kDecideThreads + threadIdx.x; t < p.zero_tiles;
         t += (int64_t)gridDim.x * kDecideThreads)
        p.tile_cnt[t] = 0u;
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31;
    const int g0 = blockIdx.x * kDecideThreads * PER;

    __shared__ uint32_t s_cnt[kDecideThreads / 32];
    __shared__ unsigned long long s_base[kDecideThreads / 32];
    // Per chunk of views, the pairs the bound keeps form a list in shared memory and
    // the CTA's threads take their exact decisions densely, one candidate each:
    // only a fraction of a view's pairs is visible (a quarter in a VR eye, 6 % in
    // the training view) and the scene's Gaussians are not ordered in space, so
    // deciding every pair in place would run the exact path on nearly every warp.
    __shared__ uint32_t s_list[kViewChunk * kDecideThreads * PER];   // view in chunk << 16 | Gaussian in CTA
    __shared__ uint32_t s_ncand;
    for (int vc = 0; vc < p.n_views; vc += kViewChunk) {
        const int nvc = min(kViewChunk, p.n_views - vc);
        if (tid == 0) s_ncand = 0u;
        __syncthreads();                          // (and the previous chunk's list is read)
#pragma unroll 1
        for (int r = 0; r < PER; ++r) {
            const int lg = r * kDecideThreads + tid;
            const int g = g0 + lg;
            float m[3] = {0.f, 0.f, 0.f}, s2 = 0.f;
            const bool ok = g < p.S.n && gauss_rules(p, g, vc == 0, m, s2);
            for (int c = 0; c < nvc; ++c) {
                const bool cand = ok && may_touch_grid(vt.v[p.views[vc + c]], vt.tile, m[0], m[1], m[2], s2);
                const uint32_t vb = __ballot_sync(FULL, cand);
                uint32_t base = 0u;
                if (lane == 0 && vb) base = atomicAdd(&s_ncand, (uint32_t)__popc(vb));
                base = __shfl_sync(FULL, base, 0);
                if (cand) s_list[base + __popc(vb & lanemask_lt())] = ((uint32_t)c << 16) | (uint32_t)lg;
            }
        }
        __syncthreads();
        const uint32_t nc = s_ncand;
        for (uint32_t r0 = 0; r0 < nc; r0 += kDecideThreads) {
            const uint32_t i = r0 + tid;
            Decision d;
            d.visible = false;
            int cg = 0, vi = 0;
            if (i < nc) {
                const uint32_t e = s_list[i];
                cg = g0 + (int)(e & 0xffffu);
                vi = vc + (int)(e >> 16);
                decide_pair(vt, p, cg, vi, d);
            }
            append_visible(p, d, cg, vi, s_cnt, s_base);
        }
    }
}

// SH coefficient rows in FP32 or, for scenes stored in half precision, IEEE binary16.
template <bool HALF>
struct ShRow;

template <>
struct ShRow<false> {
    // visits the 3K coefficients of row g in order: f(index, value)
    template <int K, typename F>
    __device__ __forceinline__ static void visit(const float *sh, int g, F f)
    {
        const float *src = sh + (size_t)g * 3 * K;
        if ((12 * K) % 16 == 0 && (reinterpret_cast<uintptr_t>(sh) & 15u) == 0) {
            const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
            for (int c = 0; c < 3 * K / 4; ++c) {
                const float4 v4 = __ldg(s4 + c);
                f(4 * c, v4.x);
                f(4 * c + 1, v4.y);
                f(4 * c + 2, v4.z);
                f(4 * c + 3, v4.w);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 3 * K; ++i) f(i, __ldg(src + i));
        }
    }
};

template <>
struct ShRow<true> {
    template <int K, typename F>
    __device__ __forceinline__ static void visit(const float *sh, int g, F f)
    {
        const __half *src = reinterpret_cast<const __half *>(sh) + (size_t)g * 3 * K;
        if ((6 * K) % 16 == 0 && (reinterpret_cast<uintptr_t>(sh) & 15u) == 0) {
            const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
#pragma unroll
            for (int c = 0; c < 3 * K / 8; ++c) {
                const uint4 v = __ldg(s4 + c);
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 h = __half22float2(*reinterpret_cast<const __half2 *>(&w[e]));
                    f(8 * c + 2 * e, h.x);
                    f(8 * c + 2 * e + 1, h.y);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < 3 * K; ++i) f(i, __half2float(src[i]));
        }
    }
};

template <int K, bool HALF>
__global__ void __launch_bounds__(kPairThreads, 8) k_pairs(const __grid_constant__ ViewTable vt,
                                                        const __grid_constant__ PreParams p)
{
    pdl_wait();
    pdl_trigger();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned long long n_pairs_raw = p.st->scene_pairs[p.scene];
    const unsigned long long n_pairs = n_pairs_raw < p.pair_cap ? n_pairs_raw : p.pair_cap;
    bool nonfinite_sh = false;
    __shared__ uint32_t s_wtot[kPairThreads / 32];
    __shared__ unsigned long long s_wbase[kPairThreads / 32];
    // per-pixel-order plans: each lane's terms of t* in tile units and its 2D mean in tile
    // units, for the keys (see below)
    __shared__ float4 s_rd[kPairThreads / 32][32][3];
    __shared__ float4 s_rdm[kPairThreads / 32][32];
    const int wp = threadIdx.x >> 5;
    const unsigned long long stride = (unsigned long long)gridDim.x * kPairThreads;
    for (unsigned long long c0 = (unsigned long long)blockIdx.x * kPairThreads; c0 < n_pairs; c0 += stride) {
        const unsigned long long w0 = c0 + (threadIdx.x & ~31);
        const unsigned long long i = w0 + lane;
        const bool act = i < n_pairs;
        uint4 e0 = make_uint4(0u, 0u, 0u, 0u), e1 = e0;
        if (act) {
            e0 = __ldg(p.pairs + 2 * i);
            e1 = __ldg(p.pairs + 2 * i + 1);
        }
        const int g = (int)e0.x;
        const DevView &V = vt.v[p.views[act ? (int)e0.y : 0]];
        // the pair's colour coefficients: checked, then evaluated
        float col[3] = {0.5f, 0.5f, 0.5f};
        bool vis = act;
        float mx = 0.f, my = 0.f, mz = 0.f, lo = 0.f;
        if (act) {
            mx = __ldg(p.S.means + 3 * g);
            my = __ldg(p.S.means + 3 * g + 1);
            mz = __ldg(p.S.means + 3 * g + 2);
            lo = p.S.baked ? __ldg(p.S.baked + 4 * g + 3).y : record_log2_opacity(__ldg(p.S.logits + g));
            // colour from the view direction (camera centre = -R^T t)
            const float cc0 = -(V.R[0] * V.t[0] + V.R[3] * V.t[1] + V.R[6] * V.t[2]);
            const float cc1 = -(V.R[1] * V.t[0] + V.R[4] * V.t[1] + V.R[7] * V.t[2]);
            const float cc2 = -(V.R[2] * V.t[0] + V.R[5] * V.t[1] + V.R[8] * V.t[2]);
            float dx = mx - cc0, dy = my - cc1, dz = mz - cc2;
            const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
            dx *= inv; dy *= inv; dz *= inv;
            float Y[16];
            sh_basis(dx, dy, dz, K, Y);
            float shs = 0.f;
            ShRow<HALF>::template visit<K>(p.S.sh, g, [&](int i, float v) {
                shs = __fmaf_rn(v, 0.f, shs);       // NaN iff some value is not finite
                col[i % 3] += Y[i / 3] * v;
            });
            if (!isfinite(shs)) {
                vis = false;
                nonfinite_sh = true;
            }
        }
        if (vis) {
            const float n1 = __uint_as_float(e1.x), bb = __uint_as_float(e1.y), det = __uint_as_float(e1.z);
            // 2D mean relative to the principal point, as an unevaluated double-float sum
            float xh, xl, yh, yl, zh, zl, uh, ul, vh, vl;
            dot3_plus(V.R[0], V.R[1], V.R[2], mx, my, mz, V.t[0], xh, xl);
            dot3_plus(V.R[3], V.R[4], V.R[5], mx, my, mz, V.t[1], yh, yl);
            dot3_plus(V.R[6], V.R[7], V.R[8], mx, my, mz, V.t[2], zh, zl);
            proj_ratio(V.fx, xh, xl, zh, zl, uh, ul);
            proj_ratio(V.fy, yh, yl, zh, zl, vh, vl);
            // Cholesky factors of the conic of [[n0+.3, b], [b, n1+.3]] with the
            // cancellation-free determinant of the decision path
            const float c = n1 + 0.3f;
            const float rc = rsqrtf(c), rd = rsqrtf(det);
            const float l0 = c * rc * rd * kCholScale;       // sqrt(c / det)
            const float l1 = -bb * rc * rd * kCholScale;     // -b / sqrt(c det)
            const float l2 = rc * kCholScale;                // 1 / sqrt(c)
            float4 *r = p.rec + (size_t)(V.rec_base + g) * kRecF4;
            r[0] = make_float4(uh, vh, ul, vl);
            r[1] = make_float4(l0, l1, l2, lo);
            r[2] = make_float4(fmaxf(col[0], 0.f), fmaxf(col[1], 0.f), fmaxf(col[2], 0.f), __uint_as_float(e1.w));
            if (p.raydepth) {
                // terms of the per-pixel depth t* = sum_k a_k b_k / sum_k a_k^2 (the depth of
                // the density maximum along the pixel's ray): with the camera-space axes
                // e_k = W R_k of the Gaussian and u, v the pixel centre minus the principal
                // point, a_k = (e_k . (u/fx, v/fy, 1)) / s_k and b_k = (e_k . mu_cam) / s_k;
                // the record holds (e_kx / (fx s_k), e_ky / (fy s_k), e_kz / s_k, b_k)
                // scales and rotation as the decision path has them (or baked), so that baked
                // and parameter scenes key and order alike
                float sk[3], Rq[9];
                if (p.S.baked) {
                    const float4 b0 = __ldg(p.S.baked + 4 * g), b1 = __ldg(p.S.baked + 4 * g + 1);
                    const float4 b2 = __ldg(p.S.baked + 4 * g + 2);
                    sk[0] = b0.x; sk[1] = b0.y; sk[2] = b0.z;
                    Rq[0] = b0.w; Rq[1] = b1.x; Rq[2] = b1.y; Rq[3] = b1.z; Rq[4] = b1.w;
                    Rq[5] = b2.x; Rq[6] = b2.y; Rq[7] = b2.z; Rq[8] = b2.w;
                } else {
                    float lsv[3], q[4];
#pragma unroll
                    for (int i = 0; i < 3; ++i) lsv[i] = __ldg(p.S.log_scales + 3 * g + i);
#pragma unroll
                    for (int i = 0; i < 4; ++i) q[i] = __ldg(p.S.quats + 4 * g + i);
                    GaussPre gp;
                    gauss_pre(lsv, q, gp);          // visible, so the quaternion is not zero
#pragma unroll
                    for (int i = 0; i < 3; ++i) sk[i] = gp.s[i];
#pragma unroll
                    for (int i = 0; i < 9; ++i) Rq[i] = gp.Rq[i];
                }
                const float mc0 = xh + xl, mc1 = yh + yl, mc2 = zh + zl;
                float4 *rdp = p.raydepth + (size_t)(V.rec_base + g) * 3;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float is = 1.0f / sk[k];
                    const float e0 = V.R[0] * Rq[k] + V.R[1] * Rq[3 + k] + V.R[2] * Rq[6 + k];
                    const float e1_ = V.R[3] * Rq[k] + V.R[4] * Rq[3 + k] + V.R[5] * Rq[6 + k];
                    const float e2 = V.R[6] * Rq[k] + V.R[7] * Rq[3 + k] + V.R[8] * Rq[6 + k];
                    const float4 c = make_float4(e0 * is / V.fx, e1_ * is / V.fy, e2 * is,
                                                 (e0 * mc0 + e1_ * mc1 + e2 * mc2) * is);
                    rdp[k] = c;
                    // the same terms over tile coordinates
                    const float ts = (float)vt.tile;
                    s_rd[wp][lane][k] = make_float4(c.x * ts, c.y * ts, c.z - c.x * V.cx - c.y * V.cy, c.w);
                }
                // the 2D mean and the half extents of the alpha >= 1/255 box, sqrt(thr Sigma'_xx)
                // and sqrt(thr c) with thr = 2 ln(255 o) and Sigma'_xx = (det + b^2) / c, in tile units
                const float thr = fmaxf(2.0f * 0.69314718f * (lo + kLog2_255), 0.f);
                const float its = 1.0f / (float)vt.tile;
                s_rdm[wp][lane] = make_float4((uh + ul + V.cx) * its, (vh + vl + V.cy) * its,
                                              sqrtf(thr * (det + bb * bb) / c) * its, sqrtf(thr * c) * its);
            }
        }
        // warp-cooperative emission: one atomic per warp, coalesced key writes
        const int x0 = (int)(e0.z & 0xffffu), x1 = (int)(e0.z >> 16);
        const int y0 = (int)(e0.w & 0xffffu), y1 = (int)(e0.w >> 16);
        const uint32_t cnt = vis ? (uint32_t)((x1 - x0) * (y1 - y0)) : 0u;
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(FULL, incl, 31);
        // one atomic per CTA: the warps' totals are summed and the CTA's slots split
        if (lane == 0) s_wtot[wp] = total;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long sum = 0;
            for (int q = 0; q < kPairThreads / 32; ++q) sum += s_wtot[q];
            unsigned long long b = sum ? atomicAdd(&p.st->instances, sum) : 0ull;
            for (int q = 0; q < kPairThreads / 32; ++q) {
                s_wbase[q] = b;
                b += s_wtot[q];
            }
        }
        __syncthreads();
        const unsigned long long base = s_wbase[wp];
        __syncthreads();
        if (total == 0) continue;
        const uint32_t excl = incl - cnt;
        const int nx = vis ? x1 - x0 : 1;
        const uint32_t dbits = e1.w;
        const uint32_t rid = (uint32_t)(V.rec_base + g);
        const long long first = V.tile_base + (long long)y0 * V.gw + x0;   // tile id of (x0, y0)
        const int gw = V.gw;
        // two keys per lane per round: independent shuffle chains overlap
        for (uint32_t k0 = 0; k0 < total; k0 += 64) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const uint32_t k = k0 + 32 * u + lane;
            int j = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t v = __shfl_sync(FULL, incl, j + step - 1);
                if (v <= k) j += step;
            }
            const uint32_t oex = __shfl_sync(FULL, excl, j);
            const long long ofirst = __shfl_sync(FULL, first, j);
            const int onx = __shfl_sync(FULL, nx, j);
            const int ogw = __shfl_sync(FULL, gw, j);
            uint32_t odb = __shfl_sync(FULL, dbits, j);
            const uint32_t orid = __shfl_sync(FULL, rid, j);
            int ox0 = 0, oy0 = 0;
            if (p.raydepth) {
                ox0 = __shfl_sync(FULL, x0, j);
                oy0 = __shfl_sync(FULL, y0, j);
            }
            if (k < total) {
                // (row, column) of the pair's local tile index: a reciprocal estimate
                // (the hardware reciprocal is within 1 ulp, so the quotient is off by
                // at most 0.75 below 2^22, and a rectangle holds at most 2^22 tiles)
                // and one correction step
                const int local = (int)(k - oex);
                int ty = (int)__fmul_rn((float)local, rcp_approx((float)onx));
                int tx = local - ty * onx;
                if (tx < 0) {
                    --ty;
                    tx += onx;
                } else if (tx >= onx) {
                    ++ty;
                    tx -= onx;
                }
                if (p.raydepth) {
                    // per-pixel-order plans sort each tile's list by t* at the tile's centre, moved
                    // into the splat's alpha >= 1/255 box where it lies outside (t* stays where the
                    // splat is seen): for splats on a common surface their order there is the order
                    // at most of the tile's pixels (non-negative, so its bits sort as its value)
                    const float4 mt = s_rdm[wp][j];
                    const float cx_ = fminf(fmaxf((float)(ox0 + tx) + 0.5f, mt.x - mt.z), mt.x + mt.z);
                    const float cy_ = fminf(fmaxf((float)(oy0 + ty) + 0.5f, mt.y - mt.w), mt.y + mt.w);
                    float num = 0.f, den = 0.f;
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const float4 c = s_rd[wp][j][q];
                        const float a_ = fmaf(c.x, cx_, fmaf(c.y, cy_, c.z));
                        num = fmaf(a_, c.w, num);
                        den = fmaf(a_, a_, den);
                    }
                    odb = __float_as_uint(fmaxf(__fdividef(num, den), 0.f));
                }
                const unsigned long long tid64 = (unsigned long long)(ofirst + (long long)ty * ogw + tx);
                const unsigned long long pos = base + k;
                if (pos < p.cap) {
                    p.keys[pos] = (tid64 << 32) | odb;
                    p.vals[pos] = orid;
                    if (p.tile_cnt) atomicAdd(p.tile_cnt + tid64, 1u);
                }
            }
          }
        }
        if (lane == 0 && base + total > p.cap) atomicOr(&p.st->flags, ST_CAPACITY);
    }
    if (nonfinite_sh) atomicOr(&p.st->flags, ST_NONFINITE);
}

template <int K, bool HALF>
static cudaError_t launch_pairs(const ViewTable &vt, const PreParams &p, int64_t want, int n_sms, cudaStream_t s)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs<K, HALF>, kPairThreads, 0) != cudaSuccess ||
        per_sm <= 0) {
        cudaGetLastError();
        per_sm = 4;
    }
    const int64_t wave = (int64_t)(n_sms > 0 ? n_sms : 152) * per_sm;
    const unsigned grid = (unsigned)(want < wave ? want : wave);
    return launch_pdl(k_pairs<K, HALF>, dim3(grid > 0 ? grid : 1), dim3(kPairThreads), 0, s, vt, p);
}

// Host launcher: two launches per scene (the SH degree is a template argument
// of the pair kernel so that a row's coefficients stay in registers).
cudaError_t launch_preprocess(const ViewTable &vt, const DevScene &S, int scene, const int8_t *views,
                              int n_views, uint4 *pairs, float4 *rec, unsigned long long *keys,
                              uint32_t *vals, uint32_t *tile_cnt, DevStatus *st, unsigned long long cap,
                              float4 *viewtab, int64_t zero_tiles, float4 *raydepth, int n_sms,
                              cudaStream_t stream)
{
    if (S.n <= 0 || n_views <= 0) return cudaSuccess;
    PreParams p;
    p.raydepth = raydepth;
    p.S = S;
    p.scene = scene;
    p.n_views = n_views;
    for (int i = 0; i < VRS_MAX_VIEWS; ++i) p.views[i] = i < n_views ? views[i] : 0;
    p.pairs = pairs;
    p.pair_cap = (unsigned long long)S.n * (unsigned long long)n_views;
    p.rec = rec;
    p.keys = keys;
    p.vals = vals;
    p.tile_cnt = tile_cnt;
    p.st = st;
    p.cap = cap;
    p.viewtab = viewtab;
    p.zero_tiles = tile_cnt ? zero_tiles : 0;
    // one view: 8 Gaussians per thread (about 6 % of a training view's pairs survive
    // the screen, so a CTA gathers enough candidates to keep its threads busy);
    // several views: 2 per thread (a quarter of an eye's pairs survive, and more
    // CTAs keep more of the exact path's latency in flight)
    cudaError_t e =
        n_views == 1
            ? launch_pdl(k_decide_listed<8>, dim3(grid_for(S.n, 8 * kDecideThreads)), dim3(kDecideThreads), 0, stream,
                         vt, p)
            : launch_pdl(k_decide_listed<2>, dim3(grid_for(S.n, 2 * kDecideThreads)), dim3(kDecideThreads), 0, stream,
                         vt, p);
    if (e != cudaSuccess) return e;
    // one pair per thread, CTAs looping over the list: the grid is sized for the list's
    // capacity but capped at one resident wave, since the list holds only the visible pairs
    // (a quarter of an eye's) and launching thousands of CTAs that exit at once costs time
    const int64_t want = grid_for((int64_t)S.n * n_views, kPairThreads);
    switch (S.K + (S.sh_half ? 100 : 0)) {
        case 1: return launch_pairs<1, false>(vt, p, want, n_sms, stream);
        case 4: return launch_pairs<4, false>(vt, p, want, n_sms, stream);
        case 9: return launch_pairs<9, false>(vt, p, want, n_sms, stream);
        case 16: return launch_pairs<16, false>(vt, p, want, n_sms, stream);
        case 101: return launch_pairs<1, true>(vt, p, want, n_sms, stream);
        case 104: return launch_pairs<4, true>(vt, p, want, n_sms, stream);
        case 109: return launch_pairs<9, true>(vt, p, want, n_sms, stream);
        case 116: return launch_pairs<16, true>(vt, p, want, n_sms, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vrs
