// Adjoint of the rasterizer.  The method is trained end to end by gradient
// descent with torch as the automatic-gradient framework over hand-written
// renderers (Sec. 3.5, Sec. 4 "Training"); this file is that renderer's
// reverse pass.
//
// k_render_bwd: per tile, the reverse of the forward blend.  Each pixel starts
// from its final transmittance and walks its tile list backwards from the last
// blended splat, recovering T_i = T_{i+1} / (1 - alpha_i), with running suffix
// sums S_C = sum_{j>i} rgb_j w_j and S_D = sum_{j>i} d_j w_j (w_j = alpha_j T_j):
//   dL/dalpha_i = T_i (g_C . rgb_i + g_D d_i) - (g_C . S_C + g_D S_D + g_T T_final) / (1 - alpha_i).
// The staging, culling and alpha of every pair are the forward's, bit for bit
// (shared device functions), so the same pairs are blended.  Each warp owns an
// 8x8 block; per splat its lanes write their 10 gradient terms to a per-warp
// shared-memory buffer, and every three splats lane p sums row p and adds it to
// the splat's record gradient with one atomic.  CTA i takes the i-th tile of a
// work order, heaviest first by the forward's per-block estimates.
//
// k_clear_pair_rows: for a scene with one view, clears the record gradients of
// its visible pairs, the only ones the pass reads, before it runs.
//
// k_touched / k_touched_pairs: the list of Gaussians with a nonzero record
// gradient in some view.
//
// k_backward_params: per listed Gaussian, the chain rule from the record
// gradients of each view to means, log-scales, quaternion, opacity logit and SH
// coefficients, accumulated into the caller's arrays.
#include "vrs_internal.cuh"

namespace vrs {

struct BwdArgs {
    const float4 *viewtab;
    const float4 *rec;
    const uint32_t *vals;
    const uint2 *ranges;
    const DevStatus *st;
    const uint32_t *ncontrib;
    const float *Tf;
    const float *g_rgb;
    const float *g_depth;
    const float *g_T;        // nullable
    float *grad2d;
    const uint32_t *order;   // tile of each CTA (heaviest first), or null: tile order
    int64_t n_records;
    unsigned long long cap;
};

constexpr float kInvChol2 = 1.0f / (kCholScale * kCholScale);   // 2 / log2(e)

// A lane's two pixels (x and x + 1 of one row) as packed pairs.
struct PixState2 {
    float2 T, SC0, SC1, SC2, SD, gC0, gC1, gC2, gD, gT, Tfin;
    uint32_t last0, last1;
};

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// The two pixels' contributions to the 10 record gradients of a splat, as FP32x2
// pairs (each component rounded as the scalar operation); u = q' - lo per pixel
// (pair_u2).  A pixel the splat does
// not reach (c false) contributes zero and keeps its state: its weight and
// dL/dalpha are multiplied by 0, its T is selected.  g[i].x + g[i].y is the
// lane's value i.
__device__ __forceinline__ void pixel_adjoint2(PixState2 &p, float2 u, bool c0, bool c1, float2 dx, float dy,
                                               const float4 A, const float4 B, const float4 C, float2 *g)
{
    const float2 e = make_float2(ex2_approx(-u.x), ex2_approx(-u.y));
    const float2 al = make_float2(fminf(e.x, 0.99f), fminf(e.y, 0.99f));
    const float2 om = __ffma2_rn(al, f2(-1.f), f2(1.f));
    // 1 / (1 - alpha) by the hardware reciprocal (a few ulp, against the 0.5 ulp of the
    // correctly rounded one, whose slow path cost 8 % of the training step's backward);
    // 1 - alpha >= 0.01, and T recovered over hundreds of splats drifts by < 1e-4 relative
    const float2 rom = make_float2(rcp_approx(om.x), rcp_approx(om.y));
    const float2 Tb = __fmul2_rn(p.T, rom);
    const float2 m = make_float2(c0 ? 1.f : 0.f, c1 ? 1.f : 0.f);
    const float2 w = __fmul2_rn(__fmul2_rn(al, Tb), m);
    g[6] = __ffma2_rn(p.gC0, w, g[6]);
    g[7] = __ffma2_rn(p.gC1, w, g[7]);
    g[8] = __ffma2_rn(p.gC2, w, g[8]);
    g[9] = __ffma2_rn(p.gD, w, g[9]);
    float2 s1 = __fmul2_rn(p.gC0, f2(C.x));
    s1 = __ffma2_rn(p.gC1, f2(C.y), s1);
    s1 = __ffma2_rn(p.gC2, f2(C.z), s1);
    s1 = __ffma2_rn(p.gD, f2(B.w), s1);
    float2 s2 = __fmul2_rn(p.gC0, p.SC0);
    s2 = __ffma2_rn(p.gC1, p.SC1, s2);
    s2 = __ffma2_rn(p.gC2, p.SC2, s2);
    s2 = __ffma2_rn(p.gD, p.SD, s2);
    s2 = __ffma2_rn(p.gT, p.Tfin, s2);
    // dL/dalpha, zero where the pixel is not reached or alpha was clamped
    const float2 mc = make_float2(c0 && e.x < 0.99f ? 1.f : 0.f, c1 && e.y < 0.99f ? 1.f : 0.f);
    const float2 dLda = __fmul2_rn(__ffma2_rn(Tb, s1, __fmul2_rn(s2, make_float2(-rom.x, -rom.y))), mc);
    p.SC0 = __ffma2_rn(f2(C.x), w, p.SC0);
    p.SC1 = __ffma2_rn(f2(C.y), w, p.SC1);
    p.SC2 = __ffma2_rn(f2(C.z), w, p.SC2);
    p.SD = __ffma2_rn(f2(B.w), w, p.SD);
    p.T = make_float2(c0 ? Tb.x : p.T.x, c1 ? Tb.y : p.T.y);
    const float2 dLdp = __fmul2_rn(dLda, al);                  // d alpha / d power = alpha (natural units)
    g[5] = __ffma2_rn(dLda, make_float2(ex2_approx(-(u.x + B.y)), ex2_approx(-(u.y + B.y))), g[5]);   // d alpha / d opacity = 2^-q'
    const float l0 = A.z, l1 = A.w, l2 = B.x;
    const float2 t = __ffma2_rn(f2(l0), dx, f2(l1 * dy));
    // w = Sigma'^-1 d = (l0 t, l1 t + l2^2 dy) / kCholScale^2, the conic applied to the offset
    const float2 wx = __fmul2_rn(f2(l0), t), wy = __ffma2_rn(f2(l1), t, f2(l2 * l2 * dy));
    const float2 ndp = __fmul2_rn(dLdp, f2(-kInvChol2));
    g[0] = __ffma2_rn(ndp, wx, g[0]);                                   // -(a dx + b dy)
    g[1] = __ffma2_rn(ndp, wy, g[1]);                                   // -(c dy + b dx)
    // d power / d Sigma' = w w^T / 2: the gradient of the 2D covariance [[A, B], [B, C]]
    // itself (B one variable), a sum of bounded terms; the gradient of the conic would
    // cancel by orders of magnitude on the way back to Sigma' for elongated splats
    const float2 hdp = __fmul2_rn(dLdp, f2(0.5f * kInvChol2 * kInvChol2));
    g[2] = __ffma2_rn(hdp, __fmul2_rn(wx, wx), g[2]);
    g[3] = __ffma2_rn(__fmul2_rn(hdp, f2(2.f)), __fmul2_rn(wx, wy), g[3]);
    g[4] = __ffma2_rn(hdp, __fmul2_rn(wy, wy), g[4]);
}

constexpr int kGroup = 3;     // splats whose gradients are reduced together (3 x 10 rows <= 32 lanes)
constexpr int kGStride = 36;  // row pitch in floats: lane-column writes and float4 row reads are conflict-free

// Sums the 32 lanes' contributions of each (splat, value) of a group and adds
// them to the splats' record gradients: lane p reduces row p.
__device__ __forceinline__ void flush_group(float (*G)[kGStride], const uint32_t *R, int ng, int lane, float *grad2d)
{
    __syncwarp();
    for (int p = lane; p < ng * kGrad2D; p += 32) {
        // the row's 32 values as 16 FP32x2 pairs: two packed accumulators
        const float4 *row = reinterpret_cast<const float4 *>(G[p]);
        const float4 r0 = row[0];
        float2 a01 = make_float2(r0.x, r0.y), a23 = make_float2(r0.z, r0.w);
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            const float4 q = row[j];
            a01 = __fadd2_rn(a01, make_float2(q.x, q.y));
            a23 = __fadd2_rn(a23, make_float2(q.z, q.w));
        }
        const int sp = p / kGrad2D, v = p - sp * kGrad2D;
        atomicAdd(grad2d + (size_t)R[sp] * kGrad2D + v, (a01.x + a01.y) + (a23.x + a23.y));
    }
    __syncwarp();
}

template <int TS>
__global__ void __launch_bounds__(BlendCfg<TS>::THREADS)
    k_render_bwd(const __grid_constant__ ViewTable vt, const BwdArgs a)
{
    using Cfg = BlendCfg<TS>;
    __shared__ float4 wA[Cfg::WARPS][32], wB[Cfg::WARPS][32], wC[Cfg::WARPS][32];
    __shared__ uint32_t wR[Cfg::WARPS][32];
    __shared__ float2 wKL[Cfg::WARPS][32];     // the staged splats' K, L (splat_KL)
    // per-lane gradient contributions of up to kGroup splats, reduced together
    __shared__ __align__(16) float wG[Cfg::WARPS][kGroup * kGrad2D][kGStride];
    __shared__ uint32_t wGR[Cfg::WARPS][kGroup];
    int ng = 0;

    pdl_wait();
    pdl_trigger();
    if (a.st->flags & ST_CAPACITY) return;
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t lmask = lanemask_lt();
    const int bx = (w % Cfg::WGX) * 8, by = (w / Cfg::WGX) * 8;
    const float pxc = (float)(bx + 2 * (lane & 3)) + 0.5f, pyc = (float)(by + (lane >> 2)) + 0.5f;
    const float2 pxc2 = make_float2(pxc, pxc + 1.0f);

    const int64_t t = a.order ? (int64_t)__ldg(a.order + blockIdx.x) : (int64_t)blockIdx.x;
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

    const int64_t HW = (int64_t)V.w * V.h;
    const int64_t lp = (int64_t)py * V.w + px;
    const int64_t pix = V.pix_base + lp;
    const float *grgb = a.g_rgb + 3 * V.pix_base;
    PixState2 P;
    P.SC0 = P.SC1 = P.SC2 = P.SD = f2(0.f);
    P.last0 = P.last1 = 0;
    P.T = P.Tfin = f2(1.f);
    P.gC0 = P.gC1 = P.gC2 = P.gD = P.gT = f2(0.f);
    if (in0) {
        P.last0 = a.ncontrib[pix];
        P.T.x = P.Tfin.x = a.Tf[pix];
        P.gC0.x = grgb[lp];
        P.gC1.x = grgb[HW + lp];
        P.gC2.x = grgb[2 * HW + lp];
        P.gD.x = a.g_depth[pix];
        P.gT.x = a.g_T ? a.g_T[pix] : 0.f;
    }
    if (in1) {
        P.last1 = a.ncontrib[pix + 1];
        P.T.y = P.Tfin.y = a.Tf[pix + 1];
        P.gC0.y = grgb[lp + 1];
        P.gC1.y = grgb[HW + lp + 1];
        P.gC2.y = grgb[2 * HW + lp + 1];
        P.gD.y = a.g_depth[pix + 1];
        P.gT.y = a.g_T ? a.g_T[pix + 1] : 0.f;
    }
    // this warp's blended positions end at its largest last contributor
    const uint32_t maxlast = __reduce_max_sync(FULL, max(P.last0, P.last1));
    if (maxlast == 0) return;
    const int nb = (int)((maxlast + 31) / 32);

    for (int bi = nb - 1; bi >= 0; --bi) {
        const uint32_t bs = range.x + (uint32_t)bi * 32;
        const uint32_t j = bs + lane;
        const uint32_t rid = (j < range.x + maxlast) ? __ldg(a.vals + j) : 0xffffffffu;
        bool hit = false;
        float4 A, B, C;
        if ((int64_t)rid < a.n_records) {
            float4 r0, r1, r2;
            load_record(a.rec, rid, r0, r1, r2);
            stage_record(r0, r1, r2, oxh, oxl, oyh, oyl, A, B, C);
            hit = cull_blocks<1, 1>(cull_setup(A.x, A.y, A.z, A.w, B.x, B.z), (float)bx + 0.5f, (float)by + 0.5f) != 0u;
        }
        const uint32_t bal = __ballot_sync(FULL, hit);
        if (hit) {
            const int slot = __popc(bal & lmask);
            C.w = __int_as_float(lane);
            wA[w][slot] = A;
            wB[w][slot] = B;
            wC[w][slot] = C;
            wR[w][slot] = rid;
            float K, L;
            splat_KL(A.x, A.y, A.z, A.w, B.x, K, L);
            wKL[w][slot] = make_float2(K, L);
        }
        __syncwarp();
        for (int k = __popc(bal) - 1; k >= 0; --k) {
            const float4 Ak = wA[w][k];
            const float4 Bk = wB[w][k];
            const float4 Ck = wC[w][k];
            const uint32_t pos = (uint32_t)bi * 32 + (uint32_t)__float_as_int(Ck.w) + 1;
            // pair_u2 with the per-pixel steps packed (each component the same rounded FMA)
            const float2 KL = wKL[w][k];
            const float s_ = __fmaf_rn(-Bk.x, pyc, KL.y);
            const float w_ = __fmaf_rn(s_, s_, -Bk.y);
            const float r_ = __fmaf_rn(-Ak.w, pyc, KL.x);
            const float2 t_ = __ffma2_rn(f2(-Ak.z), pxc2, f2(r_));
            const float2 u_ = __ffma2_rn(t_, t_, f2(w_));
            const float u0 = u_.x, u1 = u_.y;
            const bool c0 = pos <= P.last0 && u0 <= kLog2_255;
            const bool c1 = pos <= P.last1 && u1 <= kLog2_255;
            if (!__any_sync(FULL, c0 || c1)) continue;
            float2 g2[kGrad2D];
#pragma unroll
            for (int i = 0; i < kGrad2D; ++i) g2[i] = f2(0.f);
            const float dx = Ak.x - pxc, dy = Ak.y - pyc;
            pixel_adjoint2(P, make_float2(u0, u1), c0, c1, make_float2(dx, dx - 1.0f), dy, Ak, Bk, Ck, g2);
            float g[kGrad2D];
#pragma unroll
            for (int i = 0; i < kGrad2D; ++i) g[i] = g2[i].x + g2[i].y;
            // the lane's contributions go to the group buffer; the group is reduced
            // when full: each lane sums whole 32-lane rows, one (splat, value) at a time
#pragma unroll
            for (int i = 0; i < kGrad2D; ++i) wG[w][ng * kGrad2D + i][lane] = g[i];
            if (lane == 0) wGR[w][ng] = wR[w][k];
            if (++ng == kGroup) {
                flush_group(wG[w], wGR[w], ng, lane, a.grad2d);
                ng = 0;
            }
        }
        __syncwarp();
    }
    if (ng) flush_group(wG[w], wGR[w], ng, lane, a.grad2d);
}

template <int TS>
static cudaError_t launch_bwd_ts(const ViewTable &vt, const BwdArgs &a, int64_t n_tiles, cudaStream_t s)
{
    return launch_pdl(k_render_bwd<TS>, dim3((unsigned)n_tiles), dim3(BlendCfg<TS>::THREADS), 0, s, vt, a);
}

cudaError_t launch_render_bwd(const ViewTable &vt, const float4 *viewtab, const float4 *rec,
                              const uint32_t *vals, const uint2 *ranges, const DevStatus *st,
                              const uint32_t *ncontrib, const float *Tf, const float *dL_drgb,
                              const float *dL_ddepth, const float *dL_dT, float *grad2d, const uint32_t *order,
                              int64_t n_tiles, int64_t n_records, unsigned long long cap, cudaStream_t s)
{
    BwdArgs a{viewtab, rec, vals, ranges, st, ncontrib, Tf, dL_drgb, dL_ddepth, dL_dT, grad2d, order, n_records, cap};
    if (n_tiles <= 0) return cudaSuccess;
    switch (vt.tile) {
        case 8: return launch_bwd_ts<8>(vt, a, n_tiles, s);
        case 16: return launch_bwd_ts<16>(vt, a, n_tiles, s);
        case 32: return launch_bwd_ts<32>(vt, a, n_tiles, s);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Per-Gaussian chain rule.

// Partial derivatives of the 16 SH basis polynomials w.r.t. x, y, z.
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, int K, float *gx, float *gy,
                                              float *gz)
{
    const float C1 = 0.48860251190291992f;
    const float C2a = 1.0925484305920792f, C2b = 0.31539156525252005f, C2c = 0.54627421529603959f;
    const float C3a = 0.59004358992664352f, C3b = 2.8906114426405538f, C3c = 0.45704579946446572f;
    const float C3d = 0.3731763325901154f, C3e = 1.4453057213202769f;
#pragma unroll
    for (int k = 0; k < 16; ++k) gx[k] = gy[k] = gz[k] = 0.f;
    if (K > 1) {
        gy[1] = -C1;
        gz[2] = C1;
        gx[3] = -C1;
    }
    if (K > 4) {
        gx[4] = C2a * y;            gy[4] = C2a * x;
        gy[5] = -C2a * z;           gz[5] = -C2a * y;
        gx[6] = -2.f * C2b * x;     gy[6] = -2.f * C2b * y;     gz[6] = 4.f * C2b * z;
        gx[7] = -C2a * z;           gz[7] = -C2a * x;
        gx[8] = 2.f * C2c * x;      gy[8] = -2.f * C2c * y;
    }
    if (K > 9) {
        const float xx = x * x, yy = y * y, zz = z * z;
        gx[9] = -C3a * 6.f * x * y;                   gy[9] = -C3a * (3.f * xx - 3.f * yy);
        gx[10] = C3b * y * z;  gy[10] = C3b * x * z;  gz[10] = C3b * x * y;
        gx[11] = C3c * 2.f * x * y;
        gy[11] = -C3c * (4.f * zz - xx - 3.f * yy);
        gz[11] = -C3c * 8.f * y * z;
        gx[12] = -C3d * 6.f * x * z;                  gy[12] = -C3d * 6.f * y * z;
        gz[12] = C3d * (6.f * zz - 3.f * xx - 3.f * yy);
        gx[13] = -C3c * (4.f * zz - 3.f * xx - yy);
        gy[13] = C3c * 2.f * x * y;
        gz[13] = -C3c * 8.f * x * z;
        gx[14] = C3e * 2.f * x * z;  gy[14] = -C3e * 2.f * y * z;  gz[14] = C3e * (xx - yy);
        gx[15] = -C3a * (3.f * xx - 3.f * yy);        gy[15] = C3a * 6.f * x * y;
    }
}

struct ParamArgs {
    DevScene S;            // parameters
    DevScene G;            // gradient arrays (written through a cast)
    int32_t n_views;
    int8_t views[VRS_MAX_VIEWS];
    const float *grad2d;
    const DevStatus *st;
    uint32_t *list;            // Gaussians with a nonzero record gradient (scratch)
    uint32_t *list_count;
    const uint4 *pairs;        // the scene's visible-pair list of the forward (2 uint4 per pair)
    int32_t scene;             // index of the scene in the plan
    unsigned long long pair_cap;
};

// The 3K values of an SH row in order, f(index, value), as 16-byte loads where
// the row's length and start allow (vec: the array base is 16-byte aligned).
template <int K, typename F>
__device__ __forceinline__ void sh_row_read(const float *row, bool vec, F f)
{
    if constexpr ((12 * K) % 16 == 0) {
        if (vec) {
            const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
            for (int c = 0; c < 3 * K / 4; ++c) {
                const float4 v = __ldg(r4 + c);
                f(4 * c, v.x);
                f(4 * c + 1, v.y);
                f(4 * c + 2, v.z);
                f(4 * c + 3, v.w);
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < 3 * K; ++i) f(i, __ldg(row + i));
}

// row[i] += val(i) over an SH gradient row, as 16-byte loads and stores where allowed.
template <int K, typename F>
__device__ __forceinline__ void sh_row_add(float *row, bool vec, F val)
{
    if constexpr ((12 * K) % 16 == 0) {
        if (vec) {
            float4 *r4 = reinterpret_cast<float4 *>(row);
#pragma unroll
            for (int c = 0; c < 3 * K / 4; ++c) {
                float4 v = r4[c];
                v.x += val(4 * c);
                v.y += val(4 * c + 1);
                v.z += val(4 * c + 2);
                v.w += val(4 * c + 3);
                r4[c] = v;
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < 3 * K; ++i) row[i] += val(i);
}

template <int K>
__device__ __forceinline__ void param_grads_one(const ViewTable &vt, const ParamArgs &p, int g)
{
    const float m[3] = {p.S.means[3 * g], p.S.means[3 * g + 1], p.S.means[3 * g + 2]};
    const float ls[3] = {p.S.log_scales[3 * g], p.S.log_scales[3 * g + 1], p.S.log_scales[3 * g + 2]};
    const float q[4] = {p.S.quats[4 * g], p.S.quats[4 * g + 1], p.S.quats[4 * g + 2], p.S.quats[4 * g + 3]};
    const float logit = p.S.logits[g];
    const float *shg = p.S.sh + (size_t)g * 3 * K;
    GaussPre pre;
    if (!gauss_pre(ls, q, pre)) return;
    float *gs_out = const_cast<float *>(p.G.sh) + (size_t)g * 3 * K;
    float gm[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gqh[4] = {0.f, 0.f, 0.f, 0.f}, glogit = 0.f;
    const float o = 1.0f / (1.0f + expf(-logit));
    const bool vec_in = (reinterpret_cast<uintptr_t>(p.S.sh) & 15u) == 0;
    const bool vec_out = (reinterpret_cast<uintptr_t>(p.G.sh) & 15u) == 0;
    bool any = false;

    for (int vi = 0; vi < p.n_views; ++vi) {
        const DevView &V = vt.v[p.views[vi]];
        // a record's 10 gradients are 5 float2 (40-byte records in an aligned array)
        const float2 *G2 = reinterpret_cast<const float2 *>(p.grad2d + (size_t)(V.rec_base + g) * kGrad2D);
        float G[kGrad2D];
        bool nz = false;
#pragma unroll
        for (int i = 0; i < kGrad2D / 2; ++i) {
            const float2 v = G2[i];
            G[2 * i] = v.x;
            G[2 * i + 1] = v.y;
            nz |= v.x != 0.f || v.y != 0.f;
        }
        if (!nz) continue;
        Decision d;
        decide(V, pre, m[0], m[1], m[2], logit, vt.tile, d);
        if (!d.visible) continue;
        any = true;
        // opacity
        glogit += G[5] * o * (1.0f - o);
        // colour through the SH basis and the view direction
        const float cc0 = -(V.R[0] * V.t[0] + V.R[3] * V.t[1] + V.R[6] * V.t[2]);
        const float cc1 = -(V.R[1] * V.t[0] + V.R[4] * V.t[1] + V.R[7] * V.t[2]);
        const float cc2 = -(V.R[2] * V.t[0] + V.R[5] * V.t[1] + V.R[8] * V.t[2]);
        const float v0_ = m[0] - cc0, v1_ = m[1] - cc1, v2_ = m[2] - cc2;
        const float vn = sqrtf(v0_ * v0_ + v1_ * v1_ + v2_ * v2_);
        const float dx = v0_ / vn, dy = v1_ / vn, dz = v2_ / vn;
        // (the SH row is streamed from L1 twice and the SH gradient is added to
        // memory per view, so that neither row is held in registers)
        float Y[16];
        sh_basis(dx, dy, dz, K, Y);
        float col[3] = {0.5f, 0.5f, 0.5f};
        sh_row_read<K>(shg, vec_in, [&](int i, float v) { col[i % 3] += Y[i / 3] * v; });
        // max(0, .) clamped channels pass no gradient
        const float gc[3] = {col[0] < 0.f ? 0.f : G[6], col[1] < 0.f ? 0.f : G[7], col[2] < 0.f ? 0.f : G[8]};
        float wY[16];                                 // dL/dY_k
#pragma unroll
        for (int k = 0; k < 16; ++k) wY[k] = 0.f;
        sh_row_read<K>(shg, vec_in, [&](int i, float v) { wY[i / 3] += gc[i % 3] * v; });
        sh_row_add<K>(gs_out, vec_out, [&](int i) { return gc[i % 3] * Y[i / 3]; });
        float Yx[16], Yy[16], Yz[16];
        sh_basis_grad(dx, dy, dz, K, Yx, Yy, Yz);
        float gd0 = 0.f, gd1 = 0.f, gd2 = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            gd0 += wY[k] * Yx[k];
            gd1 += wY[k] * Yy[k];
            gd2 += wY[k] * Yz[k];
        }
        const float dd = dx * gd0 + dy * gd1 + dz * gd2;
        gm[0] += (gd0 - dx * dd) / vn;
        gm[1] += (gd1 - dy * dd) / vn;
        gm[2] += (gd2 - dz * dd) / vn;
        // projection of the mean and the depth
        const float tx = d.tx, ty = d.ty, tz = d.tz;
        const float iz = 1.0f / tz, iz2 = iz * iz;
        float dtx = G[0] * V.fx * iz;
        float dty = G[1] * V.fy * iz;
        float dtz = G[9] - (G[0] * V.fx * tx + G[1] * V.fy * ty) * iz2;
        // the record holds dL/d of Sigma' = [[A, B], [B, C]] = V V^T + 0.3 I directly:
        // A = v0.v0 + .3, B = v0.v1, C = v1.v1 + .3 with V = T M
        const float gA = G[2], gB = G[3], gC = G[4];
        float gV0[3], gV1[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            gV0[j] = 2.f * gA * d.v0[j] + gB * d.v1[j];
            gV1[j] = gB * d.v0[j] + 2.f * gC * d.v1[j];
        }
        float gT0[3], gT1[3], gM[9];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            gT0[k] = gV0[0] * pre.M[3 * k] + gV0[1] * pre.M[3 * k + 1] + gV0[2] * pre.M[3 * k + 2];
            gT1[k] = gV1[0] * pre.M[3 * k] + gV1[1] * pre.M[3 * k + 1] + gV1[2] * pre.M[3 * k + 2];
#pragma unroll
            for (int j = 0; j < 3; ++j) gM[3 * k + j] = d.T0[k] * gV0[j] + d.T1[k] * gV1[j];
        }
        // T0 = J00 W0 + J02 W2, T1 = J11 W1 + J12 W2
        const float *W = V.R;
        const float gJ00 = gT0[0] * W[0] + gT0[1] * W[1] + gT0[2] * W[2];
        const float gJ02 = gT0[0] * W[6] + gT0[1] * W[7] + gT0[2] * W[8];
        const float gJ11 = gT1[0] * W[3] + gT1[1] * W[4] + gT1[2] * W[5];
        const float gJ12 = gT1[0] * W[6] + gT1[1] * W[7] + gT1[2] * W[8];
        dtz -= (gJ00 * V.fx + gJ11 * V.fy) * iz2;
        if (!d.clampx) {
            dtx -= gJ02 * V.fx * iz2;
            dtz += gJ02 * 2.f * V.fx * tx * iz2 * iz;
        } else {
            const float L = fminf(1.3f * V.tanx, fmaxf(-1.3f * V.tanx, d.txtz));
            dtz += gJ02 * V.fx * L * iz2;
        }
        if (!d.clampy) {
            dty -= gJ12 * V.fy * iz2;
            dtz += gJ12 * 2.f * V.fy * ty * iz2 * iz;
        } else {
            const float L = fminf(1.3f * V.tany, fmaxf(-1.3f * V.tany, d.tytz));
            dtz += gJ12 * V.fy * L * iz2;
        }
        gm[0] += W[0] * dtx + W[3] * dty + W[6] * dtz;
        gm[1] += W[1] * dtx + W[4] * dty + W[7] * dtz;
        gm[2] += W[2] * dtx + W[5] * dty + W[8] * dtz;
        // M = Rq S
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float gs = gM[j] * pre.Rq[j] + gM[3 + j] * pre.Rq[3 + j] + gM[6 + j] * pre.Rq[6 + j];
            gls[j] += gs * pre.s[j];
        }
        float gR[9];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) gR[3 * k + j] = gM[3 * k + j] * pre.s[j];
        // Rq(w, x, y, z) of the normalised quaternion
        const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const float w_ = q[0] / qn, x_ = q[1] / qn, y_ = q[2] / qn, z_ = q[3] / qn;
        gqh[0] += 2.f * (-z_ * gR[1] + y_ * gR[2] + z_ * gR[3] - x_ * gR[5] - y_ * gR[6] + x_ * gR[7]);
        gqh[1] += 2.f * (y_ * gR[1] + z_ * gR[2] + y_ * gR[3] - 2.f * x_ * gR[4] - w_ * gR[5] +
                         z_ * gR[6] + w_ * gR[7] - 2.f * x_ * gR[8]);
        gqh[2] += 2.f * (-2.f * y_ * gR[0] + x_ * gR[1] + w_ * gR[2] + x_ * gR[3] + z_ * gR[5] -
                         w_ * gR[6] + z_ * gR[7] - 2.f * y_ * gR[8]);
        gqh[3] += 2.f * (-2.f * z_ * gR[0] - w_ * gR[1] + x_ * gR[2] + w_ * gR[3] - 2.f * z_ * gR[4] +
                         y_ * gR[5] + x_ * gR[6] + y_ * gR[7]);
    }
    if (!any) return;
    float *Gm = const_cast<float *>(p.G.means), *Gl = const_cast<float *>(p.G.log_scales);
    float *Gq = const_cast<float *>(p.G.quats), *Go = const_cast<float *>(p.G.logits);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Gm[3 * g + i] += gm[i];
        Gl[3 * g + i] += gls[i];
    }
    const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float qh[4] = {q[0] / qn, q[1] / qn, q[2] / qn, q[3] / qn};
    const float dot = gqh[0] * qh[0] + gqh[1] * qh[1] + gqh[2] * qh[2] + gqh[3] * qh[3];
#pragma unroll
    for (int i = 0; i < 4; ++i) Gq[4 * g + i] += (gqh[i] - qh[i] * dot) / qn;
    Go[g] += glogit;
}

// Whether the warp's Gaussian g0 + lane has a nonzero record gradient in some
// view of the scene.  The 32 records of a view are 160 contiguous float2: the
// warp reads them coalesced (five loads per lane), one ballot per load marks the
// nonzero float2, and the lane takes the five bits of its own record.
__device__ __forceinline__ bool touched_warp(const ViewTable &vt, const ParamArgs &p, int g0, int lane)
{
    static_assert(kGrad2D == 10, "five float2 per record");
    const int n2 = min(32, p.S.n - g0) * 5;   // float2 of the warp's valid records
    uint32_t m0 = 0u, m1 = 0u, m2 = 0u, m3 = 0u, m4 = 0u;
    for (int vi = 0; vi < p.n_views; ++vi) {
        const float2 *G2 = reinterpret_cast<const float2 *>(p.grad2d + (size_t)(vt.v[p.views[vi]].rec_base + g0) * kGrad2D);
        float2 v[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) v[i] = 32 * i + lane < n2 ? __ldg(G2 + 32 * i + lane) : make_float2(0.f, 0.f);
        m0 |= __ballot_sync(0xffffffffu, v[0].x != 0.f || v[0].y != 0.f);
        m1 |= __ballot_sync(0xffffffffu, v[1].x != 0.f || v[1].y != 0.f);
        m2 |= __ballot_sync(0xffffffffu, v[2].x != 0.f || v[2].y != 0.f);
        m3 |= __ballot_sync(0xffffffffu, v[3].x != 0.f || v[3].y != 0.f);
        m4 |= __ballot_sync(0xffffffffu, v[4].x != 0.f || v[4].y != 0.f);
    }
    const int bit = 5 * lane, w = bit >> 5, off = bit & 31;
    const uint32_t lo = w == 0 ? m0 : w == 1 ? m1 : w == 2 ? m2 : w == 3 ? m3 : m4;
    const uint32_t hi = w == 0 ? m1 : w == 1 ? m2 : w == 2 ? m3 : w == 3 ? m4 : 0u;
    return ((((uint64_t)hi << 32) | lo) >> off & 31u) != 0u;
}

// A scene with one view: its reverse pass and chain rule read only the 2D-gradient rows
// of the forward's visible pairs, so only those are cleared (the pair list's records,
// a few percent of the scene's) instead of every record's.
__global__ void __launch_bounds__(256) k_clear_pair_rows(const uint4 *pairs, const DevStatus *st, int scene,
                                                         unsigned long long pair_cap, int64_t rec_base,
                                                         float *grad2d)
{
    pdl_wait();
    pdl_trigger();
    if (st->flags & ST_CAPACITY) return;
    const unsigned long long n_raw = st->scene_pairs[scene];
    const unsigned long long n = n_raw < pair_cap ? n_raw : pair_cap;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        float2 *r = reinterpret_cast<float2 *>(grad2d + (size_t)(rec_base + __ldg(&pairs[2 * i].x)) * kGrad2D);
#pragma unroll
        for (int k = 0; k < kGrad2D / 2; ++k) r[k] = make_float2(0.f, 0.f);
    }
}

cudaError_t launch_clear_pair_rows(const uint4 *pairs, const DevStatus *st, int scene, int64_t n_gauss,
                                   int64_t rec_base, float *grad2d, int n_sms, cudaStream_t s)
{
    if (n_gauss <= 0) return cudaSuccess;
    k_clear_pair_rows<<<(n_sms > 0 ? n_sms : 152) * 4, 256, 0, s>>>(pairs, st, scene, (unsigned long long)n_gauss,
                                                                     rec_base, grad2d);
    return cudaGetLastError();
}

// Most Gaussians touch no pixel of any view: a light pass lists those that do
// (one warp-aggregated atomic per warp), and the chain rule, heavy in registers,
// then walks that list densely.
constexpr int kTouchedThreads = 256;
constexpr int kTouchedWarps = kTouchedThreads / 32;

__global__ void __launch_bounds__(kTouchedThreads) k_touched(const __grid_constant__ ViewTable vt,
                                                 const __grid_constant__ ParamArgs p)
{
    // one list atomic per CTA: the warps' counts meet in shared memory
    __shared__ uint32_t s_cnt[kTouchedWarps], s_base[kTouchedWarps];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int g0 = (blockIdx.x * blockDim.x + threadIdx.x) - lane;
    pdl_wait();
    pdl_trigger();
    if (p.st->flags & ST_CAPACITY) return;     // uniform over the grid
    const int g = g0 + lane;
    const bool t = g0 < p.S.n && touched_warp(vt, p, g0, lane) && g < p.S.n;
    const uint32_t b = __ballot_sync(0xffffffffu, t);
    if (lane == 0) s_cnt[wp] = (uint32_t)__popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t sum = 0;
        for (int q = 0; q < kTouchedWarps; ++q) sum += s_cnt[q];
        uint32_t base = sum ? atomicAdd(p.list_count, sum) : 0u;
        for (int q = 0; q < kTouchedWarps; ++q) {
            s_base[q] = base;
            base += s_cnt[q];
        }
    }
    __syncthreads();
    if (t) p.list[s_base[wp] + __popc(b & lanemask_lt())] = (uint32_t)g;
}

// One view: every Gaussian with a nonzero record gradient is a visible pair of the
// forward's pair list, once, so the list is walked instead of every record (6 % of a
// training view's pairs are visible).  One atomic per CTA and round.
__global__ void __launch_bounds__(kTouchedThreads) k_touched_pairs(const __grid_constant__ ViewTable vt,
                                                                   const __grid_constant__ ParamArgs p)
{
    __shared__ uint32_t s_cnt[kTouchedWarps], s_base[kTouchedWarps];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    pdl_wait();
    pdl_trigger();
    if (p.st->flags & ST_CAPACITY) return;     // uniform over the grid
    const unsigned long long n_raw = p.st->scene_pairs[p.scene];
    const unsigned long long n = n_raw < p.pair_cap ? n_raw : p.pair_cap;
    const int64_t rec_base = vt.v[p.views[0]].rec_base;
    const unsigned long long stride = (unsigned long long)gridDim.x * kTouchedThreads;
    for (unsigned long long i0 = (unsigned long long)blockIdx.x * kTouchedThreads; i0 < n; i0 += stride) {
        const unsigned long long i = i0 + threadIdx.x;
        bool t = false;
        uint32_t g = 0u;
        if (i < n) {
            g = __ldg(p.pairs + 2 * i).x;
            const float2 *G2 = reinterpret_cast<const float2 *>(p.grad2d + (size_t)(rec_base + g) * kGrad2D);
#pragma unroll
            for (int k = 0; k < kGrad2D / 2; ++k) {
                const float2 v = G2[k];
                t |= v.x != 0.f || v.y != 0.f;
            }
        }
        const uint32_t b = __ballot_sync(0xffffffffu, t);
        if (lane == 0) s_cnt[wp] = (uint32_t)__popc(b);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t sum = 0;
            for (int q = 0; q < kTouchedWarps; ++q) sum += s_cnt[q];
            uint32_t base = sum ? atomicAdd(p.list_count, sum) : 0u;
            for (int q = 0; q < kTouchedWarps; ++q) {
                s_base[q] = base;
                base += s_cnt[q];
            }
        }
        __syncthreads();
        if (t) p.list[s_base[wp] + __popc(b & lanemask_lt())] = g;
        __syncthreads();                      // s_cnt and s_base are rewritten next round
    }
}

template <int K>
__global__ void __launch_bounds__(128) k_backward_params(const __grid_constant__ ViewTable vt,
                                                         const __grid_constant__ ParamArgs p)
{
    pdl_wait();
    pdl_trigger();
    if (p.st->flags & ST_CAPACITY) return;
    const uint32_t n = *p.list_count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        param_grads_one<K>(vt, p, (int)p.list[i]);
}

template <int K>
static cudaError_t launch_params_k(const ViewTable &vt, const ParamArgs &p, int n_sms, cudaStream_t s)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward_params<K>, 128, 0) != cudaSuccess ||
        per_sm <= 0) {
        cudaGetLastError();
        per_sm = 2;
    }
    return launch_pdl(k_backward_params<K>, dim3((unsigned)(n_sms * per_sm)), dim3(128), 0, s, vt, p);
}

cudaError_t launch_backward_params(const ViewTable &vt, const DevScene &S, const DevScene &G,
                                   const int8_t *views, int n_views, const float *grad2d, DevStatus *st,
                                   uint32_t *list, const uint4 *pairs, int scene, int n_sms, cudaStream_t s)
{
    if (S.n <= 0 || n_views <= 0) return cudaSuccess;
    ParamArgs p;
    p.S = S;
    p.G = G;
    p.n_views = n_views;
    for (int i = 0; i < VRS_MAX_VIEWS; ++i) p.views[i] = i < n_views ? views[i] : 0;
    p.grad2d = grad2d;
    p.st = st;
    p.list = list;
    p.list_count = &st->work[4];
    p.pairs = pairs;
    p.scene = scene;
    p.pair_cap = (unsigned long long)S.n * (unsigned long long)n_views;
    cudaError_t e = cudaMemsetAsync(&st->work[4], 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if (n_sms <= 0) n_sms = 152;
    // one view: the forward's pair list holds each touched Gaussian once; several (or no
    // pair list): a Gaussian has a pair per view, so every record of the scene is read
    if (n_views == 1 && pairs) k_touched_pairs<<<n_sms * 8, kTouchedThreads, 0, s>>>(vt, p);
    else k_touched<<<grid_for(S.n, kTouchedThreads), kTouchedThreads, 0, s>>>(vt, p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (S.K) {
        case 1: return launch_params_k<1>(vt, p, n_sms, s);
        case 4: return launch_params_k<4>(vt, p, n_sms, s);
        case 9: return launch_params_k<9>(vt, p, n_sms, s);
        case 16: return launch_params_k<16>(vt, p, n_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vrs
