// Internal definitions of libvrs (sm_103a).  Not part of the C-ABI.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "vrs.h"

namespace vrs {

// ---------------------------------------------------------------------------
// Device-side views of the plan, passed to kernels by value.

struct DevView {
    float R[9];
    float t[3];
    float fx, fy, cx, cy, znear, tanx, tany;
    int32_t w, h, gw, gh, scene, pad;
    int64_t rec_base, tile_base, pix_base;
};

struct DevScene {
    const float *means, *log_scales, *quats, *logits, *sh;
    const float4 *baked;       // nullable: 4 float4 per Gaussian (vrs_bake)
    int32_t n, K;
    int32_t sh_half;           // sh holds IEEE binary16 values
};

struct ViewTable {
    DevView v[VRS_MAX_VIEWS];
    int32_t n_views;
    int32_t tile;
};

// Status block at the head of the workspace.
struct DevStatus {
    uint32_t flags;
    uint32_t reserved;
    unsigned long long instances;
    unsigned long long pair_evals;
    unsigned long long pair_blends;
    unsigned long long block_evals;
    unsigned long long scene_pairs[VRS_MAX_SCENES];   // visible (Gaussian, view) pairs per scene
    unsigned long long resort_flagged;                  // per-pixel order: pixels whose window overflowed
    uint32_t work[8];          // counters: [0] persistent blend, [1..3] tile sort, [4] backward list
};
static_assert(sizeof(DevStatus) <= 256, "the status block is 256 bytes");

enum : uint32_t {
    ST_ZERO_QUAT = 1u,
    ST_NONFINITE = 2u,
    ST_CAPACITY = 4u,
    ST_TIMEOUT = 8u,
};

constexpr int kRecF4 = 3;                               // float4s per projected-splat record
constexpr float kLog2_255 = 7.99435343685885793f;       // log2(255)
constexpr float kCholScale = 0.849321800288019f;        // sqrt(log2(e) / 2)
constexpr int kGrad2D = 10;                             // 2D gradient floats per record

// Record layout (3 x float4 per (view, Gaussian)):
//   r0 = (ubar_hi, vbar_hi, ubar_lo, vbar_lo)   2D mean minus the principal point, double-float
//   r1 = (l0, l1, l2, lo)  conic = L^T L / kCholScale^2 with L = [[l0, l1], [0, l2]];
//                          lo = log2(opacity); alpha = min(0.99, 2^(lo - q')),
//                          q' = (l0 dx + l1 dy)^2 + (l2 dy)^2
//   r2 = (r, g, b, depth)

__device__ __forceinline__ int view_of_tile(const ViewTable &vt, int64_t tile)
{
    int lo = 0, hi = vt.n_views - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (vt.v[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Column and row of tile lt in a view gw tiles wide.  Below 2^22 tiles: a
// reciprocal estimate (relative error below 2^-21, so the quotient is off by
// at most one for gw >= 2; exact for gw = 1) and one correction step, instead
// of a 64-bit division.
__device__ __forceinline__ void tile_xy(int64_t lt, int gw, int &tx, int &ty)
{
    if (lt < ((int64_t)1 << 22)) {
        int q = (int)((float)(int)lt * rcp_approx((float)gw));
        int r = (int)lt - q * gw;
        if (r < 0) {
            --q;
            r += gw;
        } else if (r >= gw) {
            ++q;
            r -= gw;
        }
        tx = r;
        ty = q;
    } else {
        tx = (int)(lt % gw);
        ty = (int)(lt / gw);
    }
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Programmatic dependent launch.  A kernel started by launch_pdl may be
// scheduled while the kernel before it in the stream is still draining; its
// threads call pdl_wait() first, which returns once that kernel has completed
// and its writes are visible, so the body runs in stream order and only the
// launch and the CTAs' scheduling overlap.  pdl_trigger() lets the next kernel
// be scheduled once every CTA of this one has started.  Both are no-ops under
// an ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              const Args &...args)
{
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// The integer decisions in FP32.  Every operation is an explicitly rounded
// intrinsic (no contraction into fused multiply-adds, no reassociation), in a
// fixed order, so that the visibility, screen radius, tile rectangle and
// depth key are defined to the bit.

#define FMUL __fmul_rn
#define FADD __fadd_rn
#define FSUB __fsub_rn
#define FDIV __fdiv_rn

// e^x: Cody-Waite reduction x = k ln2 + r (ln2 split in a short high part and
// a low correction), degree-7 Taylor polynomial of e^r by Horner's rule with
// fused multiply-adds, exact scaling by 2^k.
__device__ __forceinline__ float exp32_cw(float x)
{
    x = fminf(fmaxf(x, -80.0f), 80.0f);
    float kf = rintf(FMUL(x, 1.44269502f));
    float r = __fmaf_rn(-kf, 0.693145751953125f, x);
    r = __fmaf_rn(-kf, 1.42860677e-06f, r);
    float p = 1.98412698e-04f;
    p = __fmaf_rn(p, r, 1.38888889e-03f);
    p = __fmaf_rn(p, r, 8.33333377e-03f);
    p = __fmaf_rn(p, r, 4.16666679e-02f);
    p = __fmaf_rn(p, r, 1.66666672e-01f);
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    int k = (int)kf;
    return FMUL(p, __int_as_float((k + 127) << 23));
}

// FP32 natural logarithm of the decision path, for finite normal x > 0:
// x = 2^e m with m in [sqrt(1/2), sqrt(2)) split off the bit pattern (exact),
// ln x = e ln2 + 2 atanh(s), s = (m - 1)/(m + 1), |s| < 0.172, and
// 2 atanh(s) = 2 s (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9) by Horner's rule.
// Each step is one correctly rounded operation, in this order.
__device__ __forceinline__ float log32_cw(float x)
{
    uint32_t bits = __float_as_uint(x);
    int e = (int)((bits >> 23) & 0xffu) - 126;
    float m = __uint_as_float((bits & 0x807fffffu) | 0x3f000000u);
    if (m < 0.70710678f) {
        m = FMUL(m, 2.0f);
        e = e - 1;
    }
    const float s = FDIV(FSUB(m, 1.0f), FADD(m, 1.0f));
    const float z = FMUL(s, s);
    float p = 0.111111111f;
    p = FADD(FMUL(p, z), 0.142857143f);
    p = FADD(FMUL(p, z), 0.2f);
    p = FADD(FMUL(p, z), 0.333333333f);
    p = FADD(FMUL(p, z), 1.0f);
    const float r = FMUL(FMUL(2.0f, s), p);
    return FADD(FMUL((float)e, 0.693147182f), r);
}

// Per-Gaussian part: scales, rotation of the normalised quaternion, M = Rq S.
struct GaussPre {
    float s[3];
    float Rq[9];
    float M[9];
};

// Returns false for an all-zero quaternion.
__device__ __forceinline__ bool gauss_pre(const float ls[3], const float q[4], GaussPre &g)
{
    g.s[0] = exp32_cw(ls[0]);
    g.s[1] = exp32_cw(ls[1]);
    g.s[2] = exp32_cw(ls[2]);
    float qq = FMUL(q[0], q[0]);
    qq = FADD(qq, FMUL(q[1], q[1]));
    qq = FADD(qq, FMUL(q[2], q[2]));
    qq = FADD(qq, FMUL(q[3], q[3]));
    if (!(qq > 0.0f)) return false;
    float iq = FDIV(1.0f, __fsqrt_rn(qq));
    float w = FMUL(q[0], iq), x = FMUL(q[1], iq), y = FMUL(q[2], iq), z = FMUL(q[3], iq);
    float xx = FMUL(x, x), yy = FMUL(y, y), zz = FMUL(z, z);
    float xy = FMUL(x, y), xz = FMUL(x, z), yz = FMUL(y, z);
    float wx = FMUL(w, x), wy = FMUL(w, y), wz = FMUL(w, z);
    g.Rq[0] = FSUB(1.0f, FMUL(2.0f, FADD(yy, zz)));
    g.Rq[1] = FMUL(2.0f, FSUB(xy, wz));
    g.Rq[2] = FMUL(2.0f, FADD(xz, wy));
    g.Rq[3] = FMUL(2.0f, FADD(xy, wz));
    g.Rq[4] = FSUB(1.0f, FMUL(2.0f, FADD(xx, zz)));
    g.Rq[5] = FMUL(2.0f, FSUB(yz, wx));
    g.Rq[6] = FMUL(2.0f, FSUB(xz, wy));
    g.Rq[7] = FMUL(2.0f, FADD(yz, wx));
    g.Rq[8] = FSUB(1.0f, FMUL(2.0f, FADD(xx, yy)));
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) g.M[3 * k + j] = FMUL(g.Rq[3 * k + j], g.s[j]);
    return true;
}

// floor((a + b) * inv_tile) of the exact real sum of two floats, inv_tile a
// power of two: the rounded sum s and its exact error e (Knuth's two-sum), then
// one step down when s is a multiple of the tile and e < 0.  Exact for
// |a + b| < 2^24; larger values lie far outside any tile grid and are clamped.
__device__ __forceinline__ int floor_sum_div(float a, float b, float inv_tile)
{
    const float s = FADD(a, b);
    const float bb = FSUB(s, a);
    const float e = FADD(FSUB(a, FSUB(s, bb)), FSUB(b, bb));
    const float q = FMUL(s, inv_tile);
    float k = floorf(q);
    if (q == k && e < 0.0f) k = FSUB(k, 1.0f);
    k = fminf(fmaxf(k, -1.0e9f), 1.0e9f);
    return (int)k;
}

struct Decision {
    float tx, ty, tz;          // camera-space mean (FP32 decision values)
    float txtz, tytz;
    float T0[3], T1[3];        // rows of J W
    float v0[3], v1[3];        // rows of V = (J W) M
    float n0, n1, b;           // |v0|^2, |v1|^2, v0.v1
    float det;                 // det of the dilated 2D covariance
    float ub, vb, rad;
    int x0, x1, y0, y1;
    bool visible;
    bool clampx, clampy;
};

// Opacity of the decision path: o = 1 / (1 + e^-logit), each operation rounded.
__device__ __forceinline__ float decision_opacity(float logit)
{
    return FDIV(1.0f, FADD(1.0f, exp32_cw(-logit)));
}

// Per view.  `tile` is the tile edge; gw, gh the view's tile grid; op the
// opacity (decision_opacity of the logit, or its baked value).
__device__ __forceinline__ void decide_op(const DevView &V, const GaussPre &g, float mx, float my,
                                          float mz, float op, int tile, Decision &d)
{
    d.visible = false;
    const float *W = V.R;
    float tc[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float a = FMUL(W[3 * r], mx);
        a = FADD(a, FMUL(W[3 * r + 1], my));
        a = FADD(a, FMUL(W[3 * r + 2], mz));
        tc[r] = FADD(a, V.t[r]);
    }
    d.tx = tc[0];
    d.ty = tc[1];
    d.tz = tc[2];
    const float tz = tc[2];
    if (!(tz > V.znear)) return;
    const float limx = FMUL(1.3f, V.tanx), limy = FMUL(1.3f, V.tany);
    const float iz = FDIV(1.0f, tz);
    d.txtz = FMUL(tc[0], iz);
    d.tytz = FMUL(tc[1], iz);
    d.clampx = (d.txtz > limx) || (d.txtz < -limx);
    d.clampy = (d.tytz > limy) || (d.tytz < -limy);
    const float cxz = fminf(limx, fmaxf(-limx, d.txtz));     // clamped x/z
    const float cyz = fminf(limy, fmaxf(-limy, d.tytz));
    const float j00 = FMUL(V.fx, iz), j11 = FMUL(V.fy, iz);
    const float j02 = -FMUL(j00, cxz);                        // -fx (x/z) / z
    const float j12 = -FMUL(j11, cyz);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        d.T0[k] = FADD(FMUL(j00, W[k]), FMUL(j02, W[6 + k]));
        d.T1[k] = FADD(FMUL(j11, W[3 + k]), FMUL(j12, W[6 + k]));
    }
    float *v0 = d.v0, *v1 = d.v1;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float a = FMUL(d.T0[0], g.M[j]);
        a = FADD(a, FMUL(d.T0[1], g.M[3 + j]));
        v0[j] = FADD(a, FMUL(d.T0[2], g.M[6 + j]));
        float b = FMUL(d.T1[0], g.M[j]);
        b = FADD(b, FMUL(d.T1[1], g.M[3 + j]));
        v1[j] = FADD(b, FMUL(d.T1[2], g.M[6 + j]));
    }
    float n0 = FMUL(v0[0], v0[0]);
    n0 = FADD(n0, FMUL(v0[1], v0[1]));
    n0 = FADD(n0, FMUL(v0[2], v0[2]));
    float n1 = FMUL(v1[0], v1[0]);
    n1 = FADD(n1, FMUL(v1[1], v1[1]));
    n1 = FADD(n1, FMUL(v1[2], v1[2]));
    float bb = FMUL(v0[0], v1[0]);
    bb = FADD(bb, FMUL(v0[1], v1[1]));
    bb = FADD(bb, FMUL(v0[2], v1[2]));
    // det(V V^T) = |v0 x v1|^2 with v0 x v1 = diag(s1 s2, s0 s2, s0 s1) Rq^T (T0 x T1)
    float c0 = FSUB(FMUL(d.T0[1], d.T1[2]), FMUL(d.T0[2], d.T1[1]));
    float c1 = FSUB(FMUL(d.T0[2], d.T1[0]), FMUL(d.T0[0], d.T1[2]));
    float c2 = FSUB(FMUL(d.T0[0], d.T1[1]), FMUL(d.T0[1], d.T1[0]));
    float e[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float a = FMUL(g.Rq[j], c0);
        a = FADD(a, FMUL(g.Rq[3 + j], c1));
        e[j] = FADD(a, FMUL(g.Rq[6 + j], c2));
    }
    float g0 = FMUL(FMUL(g.s[1], g.s[2]), e[0]);
    float g1 = FMUL(FMUL(g.s[0], g.s[2]), e[1]);
    float g2 = FMUL(FMUL(g.s[0], g.s[1]), e[2]);
    float dvv = FMUL(g0, g0);
    dvv = FADD(dvv, FMUL(g1, g1));
    dvv = FADD(dvv, FMUL(g2, g2));
    float a_ = FADD(n0, 0.3f), c_ = FADD(n1, 0.3f);
    float det = FADD(FADD(dvv, FMUL(0.3f, FADD(n0, n1))), 0.09f);
    d.n0 = n0;
    d.n1 = n1;
    d.b = bb;
    d.det = det;
    if (!(det > 0.0f)) return;
    float mid = FMUL(0.5f, FADD(a_, c_));
    float disc = fmaxf(0.1f, FSUB(FMUL(mid, mid), det));
    float lam = FADD(mid, __fsqrt_rn(disc));
    float rad = ceilf(FMUL(3.0f, __fsqrt_rn(lam)));
    d.rad = rad;
    d.ub = FMUL(V.fx, d.txtz);
    d.vb = FMUL(V.fy, d.tytz);
    // The 3-sigma rectangle clipped to the bounding box of the ellipse where
    // alpha >= 1/255: x^T Sigma'^-1 x <= thr = 2 ln(255 o), o = sigmoid(logit),
    // half extents sqrt(thr Sigma'_xx) and sqrt(thr Sigma'_yy); thr carries a
    // margin far above the rounding of any FP32 evaluation of alpha, so no tile
    // that can hold a pixel with alpha >= 1/255 is dropped.  Each bound is the
    // floor of the exact value of (edge + principal point) / tile.  Rounding and
    // that floor are monotone, so the tighter of the two rectangles' bounds is
    // the bound of the nearer edge: max(floor(u - r), floor(u - h)) =
    // floor(u - min(r, h)), one exact floor per side instead of two.
    float thr = FMUL(2.0f, log32_cw(FMUL(255.0f, op)));
    thr = FADD(FMUL(thr, 1.001f), 0.001f);
    if (!(thr > 0.0f)) return;
    const float hx = fminf(rad, __fsqrt_rn(FMUL(thr, a_))), hy = fminf(rad, __fsqrt_rn(FMUL(thr, c_)));
    const float inv = 1.0f / (float)tile;    // a power of two: exact
    int x0 = floor_sum_div(FSUB(d.ub, hx), V.cx, inv), x1 = floor_sum_div(FADD(d.ub, hx), V.cx, inv) + 1;
    int y0 = floor_sum_div(FSUB(d.vb, hy), V.cy, inv), y1 = floor_sum_div(FADD(d.vb, hy), V.cy, inv) + 1;
    x0 = min(max(x0, 0), V.gw);
    x1 = min(max(x1, 0), V.gw);
    y0 = min(max(y0, 0), V.gh);
    y1 = min(max(y1, 0), V.gh);
    d.x0 = x0;
    d.x1 = x1;
    d.y0 = y0;
    d.y1 = y1;
    d.visible = x1 > x0 && y1 > y0;
}

__device__ __forceinline__ void decide(const DevView &V, const GaussPre &g, float mx, float my,
                                       float mz, float logit, int tile, Decision &d)
{
    decide_op(V, g, mx, my, mz, decision_opacity(logit), tile, d);
}

// log2 of the opacity as the records hold it: log2(sigmoid(x)) = -log2(1 + e^-x).
__device__ __forceinline__ float record_log2_opacity(float logit)
{
    return logit >= 0.f ? -__log2f(1.0f + __expf(-logit))
                        : logit * 1.4426950408889634f - __log2f(1.0f + __expf(logit));
}

#undef FMUL
#undef FADD
#undef FSUB
#undef FDIV

// ---------------------------------------------------------------------------
// Error-free transformations for the double-float 2D mean.

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// w0 x + w1 y + w2 z + t as an unevaluated sum hi + lo (compensated dot
// product, Ogita, Rump and Oishi 2005, "Accurate sum and dot product").
__device__ __forceinline__ void dot3_plus(float w0, float w1, float w2, float x, float y, float z,
                                          float t, float &hi, float &lo)
{
    float p, s, h, r, q;
    two_prod(w0, x, p, s);
    two_prod(w1, y, h, r);
    two_sum(p, h, p, q);
    s = __fadd_rn(s, __fadd_rn(q, r));
    two_prod(w2, z, h, r);
    two_sum(p, h, p, q);
    s = __fadd_rn(s, __fadd_rn(q, r));
    two_sum(p, t, p, q);
    s = __fadd_rn(s, q);
    two_sum(p, s, hi, lo);
}

// f * (xh + xl) / (zh + zl) as hi + lo, accurate to a few units of 2^-46.
__device__ __forceinline__ void proj_ratio(float f, float xh, float xl, float zh, float zl,
                                           float &hi, float &lo)
{
    float q1 = __fdiv_rn(xh, zh);
    float rem = __fmaf_rn(-q1, zh, xh);
    rem = __fadd_rn(rem, __fsub_rn(xl, __fmul_rn(q1, zl)));
    float q2 = __fdiv_rn(rem, zh);
    float p, pe;
    two_prod(f, q1, p, pe);
    float l = __fmaf_rn(f, q2, pe);
    hi = __fadd_rn(p, l);
    lo = __fsub_rn(l, __fsub_rn(hi, p));
}

// ---------------------------------------------------------------------------
// Real spherical harmonics, degree <= 3, (l, m = -l..l) order; constants are
// the closed-form normalisations sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times
// each polynomial's own factor.

__device__ __forceinline__ void sh_basis(float x, float y, float z, int K, float *Y)
{
    Y[0] = 0.28209479177387814f;
    if (K > 1) {
        Y[1] = -0.48860251190291992f * y;
        Y[2] = 0.48860251190291992f * z;
        Y[3] = -0.48860251190291992f * x;
    }
    if (K > 4) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = 1.0925484305920792f * x * y;
        Y[5] = -1.0925484305920792f * y * z;
        Y[6] = 0.31539156525252005f * (2.0f * zz - xx - yy);
        Y[7] = -1.0925484305920792f * x * z;
        Y[8] = 0.54627421529603959f * (xx - yy);
        if (K > 9) {
            Y[9] = -0.59004358992664352f * y * (3.0f * xx - yy);
            Y[10] = 2.8906114426405538f * x * y * z;
            Y[11] = -0.45704579946446572f * y * (4.0f * zz - xx - yy);
            Y[12] = 0.3731763325901154f * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
            Y[13] = -0.45704579946446572f * x * (4.0f * zz - xx - yy);
            Y[14] = 1.4453057213202769f * z * (xx - yy);
            Y[15] = -0.59004358992664352f * x * (xx - 3.0f * yy);
        }
    }
}

// ---------------------------------------------------------------------------
// Per-pair evaluation shared by the forward and backward blend kernels, so that
// both take the same skip / stop decisions bit for bit.  A thread owns two
// horizontally adjacent pixels at tile-local centres (pxc, pyc), (pxc+1, pyc);
// (su, sv) is the splat's 2D mean in the same tile-local frame.
//   q' = (l0 dx + l1 dy)^2 + (l2 dy)^2,  dx = su - pxc, dy = sv - pyc,
// the quadratic form of the conic in the log2 domain; the splat contributes to
// a pixel iff q' <= lt = lo + log2(255) (alpha >= 1/255), with
// alpha = min(0.99, 2^(lo - q')).  Evaluated as u = q' - lo, expanded so that
// the per-pixel part is fused multiply-adds: l0 dx + l1 dy = K - l0 pxc - l1 pyc
// with K = l0 su + l1 sv, and l2 dy = L - l2 pyc with L = l2 sv (per splat,
// splat_KL); then u = t^2 + (s^2 - lo), alpha = min(0.99, 2^-u), and the splat
// contributes iff u <= log2(255).  In the tile-local frame |K| stays below ~50
// where alpha >= 1/255; an FP32 emulation over the periphery frame's instances
// put the error of 2^-u at <= 4.7e-6 relative there (the unexpanded form: ~6e-6).
__device__ __forceinline__ void splat_KL(float su, float sv, float l0, float l1, float l2, float &K, float &L)
{
    K = __fmaf_rn(l0, su, __fmul_rn(l1, sv));
    L = __fmul_rn(l2, sv);
}

__device__ __forceinline__ void pair_u2(float K, float L, float l0, float l1, float l2, float lo, float pxc,
                                        float pyc, float &u0, float &u1)
{
    const float s = __fmaf_rn(-l2, pyc, L);
    const float w = __fmaf_rn(s, s, -lo);
    const float r = __fmaf_rn(-l1, pyc, K);
    const float t0 = __fmaf_rn(-l0, pxc, r);
    const float t1 = __fmaf_rn(-l0, pxc + 1.0f, r);
    u0 = __fmaf_rn(t0, t0, w);
    u1 = __fmaf_rn(t1, t1, w);
}

// ---------------------------------------------------------------------------
// Blend-kernel geometry and the staging of one instance into a tile's local
// frame, shared by the forward and backward blend kernels.

// Buckets of the tile work order: zero, then four per octave of the work estimate
// (see order_bucket); the order's scratch holds a histogram and cursors of them.
constexpr int kOrderBuckets = 129;

__device__ __forceinline__ int order_bucket(uint32_t c)
{
    if (c == 0) return 0;
    const int lz = 31 - __clz(c);                                  // floor(log2 c)
    const int sub = lz >= 2 ? (int)((c >> (lz - 2)) & 3u) : (lz == 1 ? (int)((c & 1u) << 1) : 0);
    return 1 + 4 * lz + sub;
}

template <int TS>
struct BlendCfg {
    static constexpr int THREADS = TS * TS / 2;
    static constexpr int WARPS = THREADS / 32;
    static constexpr int WGX = TS / 8;       // warps per tile row
    static constexpr int BATCH = THREADS;
    // forward blend: 36 warps per SM (<= 56 registers), at most 32 CTAs
    static constexpr int MIN_BLOCKS = (1024 / THREADS) * 9 / 8 < 32 ? (1024 / THREADS) * 9 / 8 : 32;
};


// Tile-local frame of a tile: origin (tx*TS - cx, ty*TS - cy) as an exact
// double-float pair (hi, lo).
__device__ __forceinline__ void tile_origin(float tile_px, float c, float &hi, float &lo)
{
    hi = __fsub_rn(tile_px, c);
    const float bb = __fsub_rn(hi, tile_px);
    lo = __fadd_rn(__fsub_rn(tile_px, __fsub_rn(hi, bb)), __fsub_rn(-c, bb));
}

// Culling of one staged splat against the 8x8 pixel blocks of a tile.
// q'(p) = (l0 (su - px) + l1 (sv - py))^2 + (l2 (sv - py))^2 is convex, so
// unless its minimiser (su, sv) lies in a block's rectangle of pixel centres,
// its minimum over the rectangle lies on an edge, where it is a 1D quadratic
// minimised at a clamped vertex.  A block is kept when that minimum is within
// lt plus a margin far above the rounding of either evaluation, so only pairs
// with alpha < 1/255 for certain are dropped.  A bounding-box test of the
// ellipse q' <= lt screens the blocks first.
struct CullSplat {
    float su, sv, l0, l1, l2, thr, il0, ic, hx, hy;
};

__device__ __forceinline__ CullSplat cull_setup(float su, float sv, float l0, float l1, float l2, float lt)
{
    CullSplat c;
    c.su = su;
    c.sv = sv;
    c.l0 = l0;
    c.l1 = l1;
    c.l2 = l2;
    c.thr = lt + 1e-3f * (1.0f + fabsf(lt));
    // hardware reciprocal and square root (a few ulp): the minimiser they place
    // sits within ~1e-6 px of the exact one, where q' is flat to second order, and
    // the half extents carry a 1e-3 relative margin
    c.il0 = rcp_approx(l0);
    const float s2 = l1 * l1 + l2 * l2;
    c.ic = rcp_approx(s2);
    const float rl2 = rcp_approx(l2);
    const float lp = fmaxf(c.thr, 0.f);
    // half extents of q' <= thr: sqrt(thr * Sigma''_xx), sqrt(thr * Sigma''_yy), plus the half block
    c.hx = sqrt_approx(lp * s2) * c.il0 * rl2 * 1.001f + 3.5f + 1e-3f;
    c.hy = sqrt_approx(lp) * rl2 * 1.001f + 3.5f + 1e-3f;
    return c;
}

// WGX x WGY adjacent 8x8 blocks at once, the first one's pixel centres
// [x0, x0 + 7] x [y0, y0 + 7] (tile-local).  A block is kept when it passes the
// bounding-box screen and holds the minimiser or has an edge minimum within thr.
// Branch-free; the minimiser along each edge line is computed once for the
// blocks that share the line.  Bit w of the result is block (w % WGX, w / WGX).
template <int WGX, int WGY>
__device__ __forceinline__ uint32_t cull_blocks(const CullSplat &c, float x0 = 0.5f, float y0 = 0.5f)
{
    const float ku = -c.l1 * c.il0;           // on a horizontal line v: u = ku v minimises q'
    const float kv = -c.l0 * c.l1 * c.ic;     // on a vertical line u: v = kv u
    float u0[WGX], u1[WGX], v0[WGY], v1[WGY];
    bool inx[WGX], iny[WGY], bbx[WGX], bby[WGY];
#pragma unroll
    for (int b = 0; b < WGX; ++b) {
        u1[b] = c.su - (x0 + 8.0f * b);
        u0[b] = u1[b] - 7.0f;
        inx[b] = u0[b] <= 0.f && u1[b] >= 0.f;
        bbx[b] = fabsf(u1[b] - 3.5f) <= c.hx;
    }
#pragma unroll
    for (int b = 0; b < WGY; ++b) {
        v1[b] = c.sv - (y0 + 8.0f * b);
        v0[b] = v1[b] - 7.0f;
        iny[b] = v0[b] <= 0.f && v1[b] >= 0.f;
        bby[b] = fabsf(v1[b] - 3.5f) <= c.hy;
    }
    float best[WGY][WGX];
#pragma unroll
    for (int by = 0; by < WGY; ++by)
#pragma unroll
        for (int bx = 0; bx < WGX; ++bx) best[by][bx] = 3.0e38f;
#pragma unroll
    for (int by = 0; by < WGY; ++by)
#pragma unroll
        for (int e = 0; e < 2; ++e) {                      // horizontal edges
            const float v = e ? v1[by] : v0[by];
            const float uh = ku * v, l1v = c.l1 * v, sy = c.l2 * v, sy2 = sy * sy;
#pragma unroll
            for (int bx = 0; bx < WGX; ++bx) {
                const float t = fmaf(c.l0, fminf(fmaxf(uh, u0[bx]), u1[bx]), l1v);
                best[by][bx] = fminf(best[by][bx], fmaf(t, t, sy2));
            }
        }
#pragma unroll
    for (int bx = 0; bx < WGX; ++bx)
#pragma unroll
        for (int e = 0; e < 2; ++e) {                      // vertical edges
            const float u = e ? u1[bx] : u0[bx];
            const float vu = kv * u, l0u = c.l0 * u;
#pragma unroll
            for (int by = 0; by < WGY; ++by) {
                const float v = fminf(fmaxf(vu, v0[by]), v1[by]);
                const float t = fmaf(c.l1, v, l0u), sy = c.l2 * v;
                best[by][bx] = fminf(best[by][bx], fmaf(t, t, sy * sy));
            }
        }
    uint32_t m = 0u;
#pragma unroll
    for (int by = 0; by < WGY; ++by)
#pragma unroll
        for (int bx = 0; bx < WGX; ++bx) {
            const bool hit = bbx[bx] && bby[by] && ((inx[bx] && iny[by]) || best[by][bx] <= c.thr);
            m |= (hit ? 1u : 0u) << (by * WGX + bx);
        }
    return c.thr > 0.f ? m : 0u;
}

// Gathers one instance's record and moves it into the tile-local frame:
// A = (su, sv, l0, l1), B = (l2, lo, lt, depth), C = (r, g, b, -).
__device__ __forceinline__ void load_record(const float4 *rec, uint32_t rid, float4 &r0, float4 &r1,
                                            float4 &r2)
{
    const float4 *rp = rec + (size_t)rid * kRecF4;
    r0 = __ldg(rp);
    r1 = __ldg(rp + 1);
    r2 = __ldg(rp + 2);
}

__device__ __forceinline__ void stage_record(const float4 r0, const float4 r1, const float4 r2,
                                             float oxh, float oxl, float oyh, float oyl, float4 &A,
                                             float4 &B, float4 &C)
{
    const float su = __fadd_rn(__fsub_rn(r0.x, oxh), __fsub_rn(r0.z, oxl));
    const float sv = __fadd_rn(__fsub_rn(r0.y, oyh), __fsub_rn(r0.w, oyl));
    A = make_float4(su, sv, r1.x, r1.y);
    B = make_float4(r1.z, r1.w, r1.w + kLog2_255, r2.w);
    C = make_float4(r2.x, r2.y, r2.z, 0.f);
}

// A tile's [start, end) clamped to the live instance list, so that no range
// value can send a gather outside the list.
__device__ __forceinline__ uint2 live_range(const uint2 *ranges, int64_t t, const DevStatus *st,
                                            unsigned long long cap)
{
    const unsigned long long n = st->instances;
    const uint32_t m = (uint32_t)(n < cap ? n : cap);
    uint2 r = ranges[t];
    r.y = min(r.y, m);
    r.x = min(r.x, r.y);
    return r;
}

// Output stores of the blend kernels: FP32, or IEEE binary16 for half-output plans.
template <bool HALF>
struct OutStore {
    __device__ __forceinline__ static void one(float *base, int64_t i, float v) { base[i] = v; }
    __device__ __forceinline__ static void two(float *base, int64_t i, float2 v)
    {
        *reinterpret_cast<float2 *>(base + i) = v;
    }
};

template <>
struct OutStore<true> {
    __device__ __forceinline__ static void one(float *base, int64_t i, float v)
    {
        reinterpret_cast<__half *>(base)[i] = __float2half_rn(v);
    }
    __device__ __forceinline__ static void two(float *base, int64_t i, float2 v)
    {
        *reinterpret_cast<__half2 *>(reinterpret_cast<__half *>(base) + i) = __float22half2_rn(v);
    }
};

// Launch helpers (host).
inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace vrs
