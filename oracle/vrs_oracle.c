/*
 * CPU oracle for the tile-based 3D Gaussian Splatting rasterizer that draws
 * VR-Splatting's peripheral image P and its approximate depth buffer
 * (Sec. 3.2, Eq. 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant table with the CUDA path; it is written from the method's
 * definition, step by step, so that it can be checked by eye.
 *
 * Two precisions, on purpose:
 *  - The integer decisions of the method (visibility, screen radius, tile
 *    rectangle, depth sort key) are taken in FP32, the kernel's precision,
 *    following a fixed sequence of individually rounded operations
 *    (orc_decide).  Build with -ffp-contract=off so that no multiply-add is
 *    fused behind our back.
 *  - Every floating output (2D mean, conic, opacity, colour, the composited
 *    image, depth and transmittance, and all gradients) is computed in FP64
 *    from the same FP32 inputs (orc_project, orc_render, orc_render_bwd,
 *    orc_param_grads).
 *
 * Projection follows the EWA splatting / 3DGS formulation that the paper's
 * periphery renderer builds on (Sec. 3.1 "Naive Method": splats with opacity,
 * colour and a covariance built from scale and rotation, projected and blended
 * to screen).  Compositing is front-to-back alpha blending with the 1/255 skip,
 * the 0.99 clamp and the T < 1e-4 stop; the depth channel is Eq. 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    float R[9];          /* world -> camera rotation, row-major */
    float t[3];          /* x_cam = R x_world + t */
    float fx, fy, cx, cy;
    float znear;
    float tan_fovx, tan_fovy;   /* half-FOV tangents bounding the Jacobian clamp */
    int32_t width, height;
} orc_camera;

/* Output record of the FP64 projection, one per Gaussian. */
typedef struct {
    double ubar, vbar;        /* fx*x/z, fy*y/z: pixel offset from the principal point */
    double depth;             /* view-space z of the mean (d_i of Eq. 1) */
    double conic[3];          /* inverse of the dilated 2D covariance: a, b, c */
    double opacity;
    double rgb[3];
    int32_t clamp_rgb[3];     /* 1 where max(0, .) clamped the colour channel */
    int32_t clamp_x, clamp_y; /* 1 where the Jacobian clamp was active */
} orc_proj;

/* ------------------------------------------------------------------------- */
/* Real spherical harmonics up to degree 3, in the (l, m = -l..l) order used by
 * 3DGS, with the orthonormalisation constants written from their closed form
 * (sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the polynomial's own factor). */

static double sh_c0(void) { return 0.5 / sqrt(M_PI); }              /* 1/(2 sqrt(pi)) */
static double sh_c1(void) { return sqrt(3.0 / (4.0 * M_PI)); }
static double sh_c2a(void) { return 0.5 * sqrt(15.0 / M_PI); }
static double sh_c2b(void) { return 0.25 * sqrt(5.0 / M_PI); }
static double sh_c2c(void) { return 0.25 * sqrt(15.0 / M_PI); }
static double sh_c3a(void) { return 0.25 * sqrt(35.0 / (2.0 * M_PI)); }
static double sh_c3b(void) { return 0.5 * sqrt(105.0 / M_PI); }
static double sh_c3c(void) { return 0.25 * sqrt(21.0 / (2.0 * M_PI)); }
static double sh_c3d(void) { return 0.25 * sqrt(7.0 / M_PI); }
static double sh_c3e(void) { return 0.25 * sqrt(105.0 / M_PI); }

/* Basis polynomials at (x, y, z); the renderer passes a unit direction. */
void orc_sh_basis_xyz(double x, double y, double z, double *Y)
{
    double xx = x * x, yy = y * y, zz = z * z;
    Y[0] = sh_c0();
    Y[1] = -sh_c1() * y;
    Y[2] = sh_c1() * z;
    Y[3] = -sh_c1() * x;
    Y[4] = sh_c2a() * x * y;
    Y[5] = -sh_c2a() * y * z;
    Y[6] = sh_c2b() * (2.0 * zz - xx - yy);
    Y[7] = -sh_c2a() * x * z;
    Y[8] = sh_c2c() * (xx - yy);
    Y[9] = -sh_c3a() * y * (3.0 * xx - yy);
    Y[10] = sh_c3b() * x * y * z;
    Y[11] = -sh_c3c() * y * (4.0 * zz - xx - yy);
    Y[12] = sh_c3d() * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    Y[13] = -sh_c3c() * x * (4.0 * zz - xx - yy);
    Y[14] = sh_c3e() * z * (xx - yy);
    Y[15] = -sh_c3a() * x * (xx - 3.0 * yy);
}

/* Partial derivatives of the 16 basis polynomials w.r.t. x, y, z. */
static void sh_basis_grad(double x, double y, double z, double *dx, double *dy, double *dz)
{
    double xx = x * x, yy = y * y, zz = z * z;
    for (int k = 0; k < 16; ++k) dx[k] = dy[k] = dz[k] = 0.0;
    dy[1] = -sh_c1();
    dz[2] = sh_c1();
    dx[3] = -sh_c1();
    dx[4] = sh_c2a() * y;            dy[4] = sh_c2a() * x;
    dy[5] = -sh_c2a() * z;           dz[5] = -sh_c2a() * y;
    dx[6] = -2.0 * sh_c2b() * x;     dy[6] = -2.0 * sh_c2b() * y;   dz[6] = 4.0 * sh_c2b() * z;
    dx[7] = -sh_c2a() * z;           dz[7] = -sh_c2a() * x;
    dx[8] = 2.0 * sh_c2c() * x;      dy[8] = -2.0 * sh_c2c() * y;
    dx[9] = -sh_c3a() * 6.0 * x * y;                 dy[9] = -sh_c3a() * (3.0 * xx - 3.0 * yy);
    dx[10] = sh_c3b() * y * z;  dy[10] = sh_c3b() * x * z;  dz[10] = sh_c3b() * x * y;
    dx[11] = sh_c3c() * 2.0 * x * y;
    dy[11] = -sh_c3c() * (4.0 * zz - xx - 3.0 * yy);
    dz[11] = -sh_c3c() * 8.0 * y * z;
    dx[12] = -sh_c3d() * 6.0 * x * z;   dy[12] = -sh_c3d() * 6.0 * y * z;
    dz[12] = sh_c3d() * (6.0 * zz - 3.0 * xx - 3.0 * yy);
    dx[13] = -sh_c3c() * (4.0 * zz - 3.0 * xx - yy);
    dy[13] = sh_c3c() * 2.0 * x * y;
    dz[13] = -sh_c3c() * 8.0 * x * z;
    dx[14] = sh_c3e() * 2.0 * x * z;  dy[14] = -sh_c3e() * 2.0 * y * z;  dz[14] = sh_c3e() * (xx - yy);
    dx[15] = -sh_c3a() * (3.0 * xx - 3.0 * yy);     dy[15] = sh_c3a() * 6.0 * x * y;
}

/* ------------------------------------------------------------------------- */
/* FP32 exponential used by the decision path: Cody & Waite's range reduction
 * (x = k ln2 + r with ln2 split into a short high part and a low correction)
 * followed by the degree-7 Taylor polynomial of e^r on |r| <= ln2/2, evaluated
 * by Horner's rule with fused multiply-adds, and an exact scaling by 2^k. */
float orc_exp32(float x)
{
    if (x > 80.0f) x = 80.0f;
    if (x < -80.0f) x = -80.0f;
    const float log2e = 1.44269502f;
    const float ln2_hi = 0.693145751953125f;       /* 22713 / 32768 */
    const float ln2_lo = 1.42860677e-06f;          /* ln 2 - ln2_hi */
    float kf = rintf(x * log2e);
    float r = fmaf(-kf, ln2_hi, x);
    r = fmaf(-kf, ln2_lo, r);
    float p = 1.98412698e-04f;                     /* 1/7! */
    p = fmaf(p, r, 1.38888889e-03f);               /* 1/6! */
    p = fmaf(p, r, 8.33333377e-03f);               /* 1/5! */
    p = fmaf(p, r, 4.16666679e-02f);               /* 1/4! */
    p = fmaf(p, r, 1.66666672e-01f);               /* 1/3! */
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int k = (int)kf;
    uint32_t bits = (uint32_t)(k + 127) << 23;     /* 2^k, normal for |k| <= 116 */
    float scale;
    memcpy(&scale, &bits, 4);
    return p * scale;
}

/* FP32 natural logarithm used by the decision path, for finite normal x > 0:
 * x = 2^e m with m in [sqrt(1/2), sqrt(2)) (exponent and mantissa split off
 * the bit pattern, exact), ln x = e ln2 + 2 atanh(s) with s = (m - 1)/(m + 1),
 * |s| < 0.172, and 2 atanh(s) = 2 s (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9) by
 * Horner's rule (truncation below 2e-9 relative).  Every step is one correctly
 * rounded FP32 operation in the order written. */
float orc_log32(float x)
{
    uint32_t bits;
    memcpy(&bits, &x, 4);
    int e = (int)((bits >> 23) & 0xffu) - 126;
    bits = (bits & 0x807fffffu) | 0x3f000000u;        /* mantissa into [0.5, 1) */
    float m;
    memcpy(&m, &bits, 4);
    if (m < 0.70710678f) { m = m * 2.0f; e = e - 1; }
    const float s = (m - 1.0f) / (m + 1.0f);
    const float z = s * s;
    float p = 0.111111111f;
    p = p * z;
    p = p + 0.142857143f;
    p = p * z;
    p = p + 0.2f;
    p = p * z;
    p = p + 0.333333333f;
    p = p * z;
    p = p + 1.0f;
    const float r = (2.0f * s) * p;
    return (float)e * 0.693147182f + r;
}

static int f_isfinite(float v) { return isfinite(v) ? 1 : 0; }

/* keeps a tile index inside the int range before conversion */
static double clamp_big(double v) { return v < -1.0e9 ? -1.0e9 : (v > 1.0e9 ? 1.0e9 : v); }

/* floor((a + b) / tile) of the exact real sum of two floats: the rounded sum
 * s and its exact error e (Knuth's two-sum, in double), then one step down
 * when s is a multiple of the tile and e < 0. */
static int floor_sum_div(float a, float b, int tile)
{
    double s = (double)a + (double)b;
    double bb = s - (double)a;
    double e = ((double)a - (s - bb)) + ((double)b - bb);
    double k = floor(s / tile);
    if (s == k * tile && e < 0.0) k -= 1.0;
    return (int)clamp_big(k);
}

/* ------------------------------------------------------------------------- */
/* The integer decisions, in FP32.  Each statement below is one correctly
 * rounded IEEE operation; the order is part of the definition.
 *
 * Returns per Gaussian: visible (0/1), the FP32 depth key, the FP32 screen
 * offsets (ubar, vbar), the radius, and the tile rectangle [x0,x1) x [y0,y1).
 * status bit 1: a quaternion had zero norm; bit 2: a non-finite parameter.
 * `pre` (nullable, 8 floats per Gaussian) receives the values just before each
 * rounding to an integer, for comparison with the FP64 decisions below:
 * (tz, ubar, vbar, 3 sqrt(lambda), sqrt(thr a), sqrt(thr c), thr, det); NaN
 * where the sequence stopped earlier.  They take no part in the decisions.
 */
int orc_decide(int n, const float *means, const float *log_scales, const float *quats,
               const float *logits, const orc_camera *cam, int tile, uint8_t *visible, float *depth,
               float *ubar, float *vbar, int32_t *radius, int32_t *rect, float *pre)
{
    int status = 0;
    const float *W = cam->R;
    const int gw = (cam->width + tile - 1) / tile;
    const int gh = (cam->height + tile - 1) / tile;
    const float limx = 1.3f * cam->tan_fovx;
    const float limy = 1.3f * cam->tan_fovy;
    for (int g = 0; g < n; ++g) {
        visible[g] = 0; depth[g] = 0.f; ubar[g] = 0.f; vbar[g] = 0.f; radius[g] = 0;
        rect[4 * g + 0] = rect[4 * g + 1] = rect[4 * g + 2] = rect[4 * g + 3] = 0;
        float *pv = pre ? pre + 8 * (size_t)g : NULL;
        if (pv) for (int k = 0; k < 8; ++k) pv[k] = NAN;
        const float mx = means[3 * g], my = means[3 * g + 1], mz = means[3 * g + 2];
        const float *ls = log_scales + 3 * g;
        const float *q = quats + 4 * g;
        int finite = f_isfinite(mx) & f_isfinite(my) & f_isfinite(mz) & f_isfinite(ls[0]) &
                     f_isfinite(ls[1]) & f_isfinite(ls[2]) & f_isfinite(q[0]) & f_isfinite(q[1]) &
                     f_isfinite(q[2]) & f_isfinite(q[3]);
        if (!finite) { status |= 2; continue; }
        /* scales */
        float s0 = orc_exp32(ls[0]), s1 = orc_exp32(ls[1]), s2 = orc_exp32(ls[2]);
        /* normalised quaternion (w, x, y, z) */
        float qq = q[0] * q[0];
        qq = qq + q[1] * q[1];
        qq = qq + q[2] * q[2];
        qq = qq + q[3] * q[3];
        if (!(qq > 0.0f)) { status |= 1; continue; }
        float iq = 1.0f / sqrtf(qq);
        float w = q[0] * iq, x = q[1] * iq, y = q[2] * iq, z = q[3] * iq;
        float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
        float wx = w * x, wy = w * y, wz = w * z;
        float Rq[9];
        Rq[0] = 1.0f - 2.0f * (yy + zz); Rq[1] = 2.0f * (xy - wz);        Rq[2] = 2.0f * (xz + wy);
        Rq[3] = 2.0f * (xy + wz);        Rq[4] = 1.0f - 2.0f * (xx + zz); Rq[5] = 2.0f * (yz - wx);
        Rq[6] = 2.0f * (xz - wy);        Rq[7] = 2.0f * (yz + wx);        Rq[8] = 1.0f - 2.0f * (xx + yy);
        float s[3] = {s0, s1, s2};
        float M[9];
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) M[3 * k + j] = Rq[3 * k + j] * s[j];
        /* camera-space mean */
        float tc[3];
        for (int r = 0; r < 3; ++r) {
            float a = W[3 * r] * mx;
            a = a + W[3 * r + 1] * my;
            a = a + W[3 * r + 2] * mz;
            tc[r] = a + cam->t[r];
        }
        const float tx = tc[0], ty = tc[1], tz = tc[2];
        if (pv) pv[0] = tz;
        if (!(tz > cam->znear)) continue;
        /* clamped projection Jacobian, rows of T = J W */
        float iz = 1.0f / tz;
        float txtz = tx * iz, tytz = ty * iz;
        float cxz = fminf(limx, fmaxf(-limx, txtz));      /* clamped x/z */
        float cyz = fminf(limy, fmaxf(-limy, tytz));
        float j00 = cam->fx * iz, j11 = cam->fy * iz;
        float j02 = -(j00 * cxz);                          /* -fx (x/z) / z */
        float j12 = -(j11 * cyz);
        float T0[3], T1[3];
        for (int k = 0; k < 3; ++k) {
            T0[k] = j00 * W[k] + j02 * W[6 + k];
            T1[k] = j11 * W[3 + k] + j12 * W[6 + k];
        }
        /* V = T M (2x3); projected covariance = V V^T + 0.3 I */
        float v0[3], v1[3];
        for (int j = 0; j < 3; ++j) {
            float a = T0[0] * M[j];
            a = a + T0[1] * M[3 + j];
            v0[j] = a + T0[2] * M[6 + j];
            float b = T1[0] * M[j];
            b = b + T1[1] * M[3 + j];
            v1[j] = b + T1[2] * M[6 + j];
        }
        float n0 = v0[0] * v0[0]; n0 = n0 + v0[1] * v0[1]; n0 = n0 + v0[2] * v0[2];
        float n1 = v1[0] * v1[0]; n1 = n1 + v1[1] * v1[1]; n1 = n1 + v1[2] * v1[2];
        /* det(V V^T) = |v0 x v1|^2, with v0 x v1 = diag(s1 s2, s0 s2, s0 s1) Rq^T (T0 x T1) */
        float c0 = T0[1] * T1[2] - T0[2] * T1[1];
        float c1 = T0[2] * T1[0] - T0[0] * T1[2];
        float c2 = T0[0] * T1[1] - T0[1] * T1[0];
        float e[3];
        for (int j = 0; j < 3; ++j) {
            float a = Rq[j] * c0;
            a = a + Rq[3 + j] * c1;
            e[j] = a + Rq[6 + j] * c2;
        }
        float g0 = (s1 * s2) * e[0], g1 = (s0 * s2) * e[1], g2 = (s0 * s1) * e[2];
        float dvv = g0 * g0; dvv = dvv + g1 * g1; dvv = dvv + g2 * g2;
        float a_ = n0 + 0.3f, c_ = n1 + 0.3f;
        float det = (dvv + 0.3f * (n0 + n1)) + 0.09f;
        if (pv) pv[7] = det;
        if (!(det > 0.0f)) continue;
        float mid = 0.5f * (a_ + c_);
        float disc = fmaxf(0.1f, mid * mid - det);
        float lam = mid + sqrtf(disc);
        float rad = ceilf(3.0f * sqrtf(lam));
        float ub = cam->fx * txtz, vb = cam->fy * tytz;
        if (pv) { pv[1] = ub; pv[2] = vb; pv[3] = 3.0f * sqrtf(lam); }
        float xlo = ub - rad, xhi = ub + rad, ylo = vb - rad, yhi = vb + rad;
        /* tile rectangle: floor of the exact value of (edge + principal point) / tile */
        int x0 = floor_sum_div(xlo, cam->cx, tile);
        int x1 = floor_sum_div(xhi, cam->cx, tile) + 1;
        int y0 = floor_sum_div(ylo, cam->cy, tile);
        int y1 = floor_sum_div(yhi, cam->cy, tile) + 1;
        /* clipped to the bounding box of the ellipse where alpha >= 1/255:
         * x^T Sigma'^-1 x <= thr = 2 ln(255 o), o = sigmoid(logit), its half extents
         * sqrt(thr Sigma'_xx) and sqrt(thr Sigma'_yy); thr carries a margin far above
         * the rounding of any FP32 evaluation of alpha */
        float eo = orc_exp32(-logits[g]);
        float op = 1.0f / (1.0f + eo);
        float thr = 2.0f * orc_log32(255.0f * op);
        thr = thr * 1.001f;
        thr = thr + 0.001f;
        if (pv) pv[6] = thr;
        if (!(thr > 0.0f)) continue;
        float hx = sqrtf(thr * a_), hy = sqrtf(thr * c_);
        if (pv) { pv[4] = hx; pv[5] = hy; }
        int bx0 = floor_sum_div(ub - hx, cam->cx, tile);
        int bx1 = floor_sum_div(ub + hx, cam->cx, tile) + 1;
        int by0 = floor_sum_div(vb - hy, cam->cy, tile);
        int by1 = floor_sum_div(vb + hy, cam->cy, tile) + 1;
        x0 = x0 > bx0 ? x0 : bx0;
        x1 = x1 < bx1 ? x1 : bx1;
        y0 = y0 > by0 ? y0 : by0;
        y1 = y1 < by1 ? y1 : by1;
        x0 = x0 < 0 ? 0 : (x0 > gw ? gw : x0);
        x1 = x1 < 0 ? 0 : (x1 > gw ? gw : x1);
        y0 = y0 < 0 ? 0 : (y0 > gh ? gh : y0);
        y1 = y1 < 0 ? 0 : (y1 > gh ? gh : y1);
        if (x1 <= x0 || y1 <= y0) continue;
        visible[g] = 1;
        depth[g] = tz;
        ubar[g] = ub; vbar[g] = vb;
        radius[g] = (int32_t)rad;
        rect[4 * g + 0] = x0; rect[4 * g + 1] = x1; rect[4 * g + 2] = y0; rect[4 * g + 3] = y1;
    }
    return status;
}

/* ------------------------------------------------------------------------- */
/* FP64 projection of one Gaussian (the floating outputs of the preprocess). */

static void quat_to_rot(const double *q, double *R)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void project_one(const float *m, const float *ls, const float *qf, float logit,
                        const float *sh, int K, const orc_camera *cam, orc_proj *o)
{
    double W[9], t[3];
    for (int i = 0; i < 9; ++i) W[i] = cam->R[i];
    for (int i = 0; i < 3; ++i) t[i] = cam->t[i];
    double mu[3] = {m[0], m[1], m[2]};
    /* 3D covariance  Sigma = R S S^T R^T */
    double s[3] = {exp((double)ls[0]), exp((double)ls[1]), exp((double)ls[2])};
    double q[4] = {qf[0], qf[1], qf[2], qf[3]};
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) q[i] /= qn;
    double Rq[9];
    quat_to_rot(q, Rq);
    double M[9];
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) M[3 * k + j] = Rq[3 * k + j] * s[j];
    double Sig[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double a = 0;
            for (int k = 0; k < 3; ++k) a += M[3 * i + k] * M[3 * j + k];
            Sig[3 * i + j] = a;
        }
    /* camera-space mean */
    double tc[3];
    for (int r = 0; r < 3; ++r) tc[r] = W[3 * r] * mu[0] + W[3 * r + 1] * mu[1] + W[3 * r + 2] * mu[2] + t[r];
    double tx = tc[0], ty = tc[1], tz = tc[2];
    /* Jacobian of the perspective projection, with the 1.3 x half-FOV guard */
    double limx = 1.3 * cam->tan_fovx, limy = 1.3 * cam->tan_fovy;
    double rx = tx / tz, ry = ty / tz;
    o->clamp_x = (rx > limx || rx < -limx);
    o->clamp_y = (ry > limy || ry < -limy);
    double cxz = (rx > limx ? limx : (rx < -limx ? -limx : rx)) * tz;
    double cyz = (ry > limy ? limy : (ry < -limy ? -limy : ry)) * tz;
    double J[6] = {cam->fx / tz, 0.0, -cam->fx * cxz / (tz * tz),
                   0.0, cam->fy / tz, -cam->fy * cyz / (tz * tz)};
    /* T = J W ; Sigma' = T Sigma T^T + 0.3 I */
    double T[6];
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j) {
            double v = 0;
            for (int k = 0; k < 3; ++k) v += J[3 * a + k] * W[3 * k + j];
            T[3 * a + j] = v;
        }
    double S2[4];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double v = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) v += T[3 * a + i] * Sig[3 * i + j] * T[3 * b + j];
            S2[2 * a + b] = v;
        }
    double A = S2[0] + 0.3, B = S2[1], C = S2[3] + 0.3;
    double det = A * C - B * B;
    o->conic[0] = C / det;
    o->conic[1] = -B / det;
    o->conic[2] = A / det;
    o->ubar = cam->fx * tx / tz;
    o->vbar = cam->fy * ty / tz;
    o->depth = tz;
    o->opacity = 1.0 / (1.0 + exp(-(double)logit));
    /* view-dependent colour: dir from the camera centre (-W^T t) to the mean */
    double cc[3];
    for (int i = 0; i < 3; ++i) cc[i] = -(W[i] * t[0] + W[3 + i] * t[1] + W[6 + i] * t[2]);
    double d[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 3; ++i) d[i] /= dn;
    double Y[16];
    orc_sh_basis_xyz(d[0], d[1], d[2], Y);
    for (int ch = 0; ch < 3; ++ch) {
        double v = 0;
        for (int k = 0; k < K; ++k) v += Y[k] * sh[3 * k + ch];
        v += 0.5;
        o->clamp_rgb[ch] = v < 0.0;
        o->rgb[ch] = v < 0.0 ? 0.0 : v;
    }
}

void orc_project(int n, const float *means, const float *log_scales, const float *quats,
                 const float *opacity_logits, const float *sh, int K, const orc_camera *cam,
                 orc_proj *out)
{
#pragma omp parallel for schedule(static)
    for (int g = 0; g < n; ++g)
        project_one(means + 3 * g, log_scales + 3 * g, quats + 4 * g, opacity_logits[g],
                    sh + (size_t)3 * K * g, K, cam, out + g);
}

/* ------------------------------------------------------------------------- */
/* The integer decisions from their plain definition, in FP64, written
 * independently of the FP32 sequence of orc_decide (Sec. 3.1: splats with a
 * covariance built from scale and rotation, projected to screen; the 3-sigma
 * radius and tile rectangle of the 3DGS rasterizer the paper builds on):
 *   Sigma  = R S S^T R^T with S = diag(exp(log_s)), R from the normalised quaternion
 *   t      = W mu + t_c; not visible when t_z <= znear
 *   J      = [[fx/z, 0, -fx x'/z^2], [0, fy/z, -fy y'/z^2]], x' and y' clamped to
 *            +-1.3 tan(half-FOV) z
 *   Sigma' = J W Sigma W^T J^T + 0.3 I = [[a, b], [b, c]]; det = a c - b^2
 *   lambda = mid + sqrt(max(0.1, mid^2 - det)), mid = (a + c) / 2
 *   r      = ceil(3 sqrt(lambda))
 *   x0 = floor((ubar - r + cx) / T), x1 = floor((ubar + r + cx) / T) + 1 (same in y),
 *   and, when `clip` is set, clipped to the bounding box of the ellipse where
 *   alpha >= 1/255: thr = 2 ln(255 o) 1.001 + 0.001 with o = sigmoid(logit) (not
 *   visible when thr <= 0), half extents hx = sqrt(thr a), hy = sqrt(thr c),
 *   x0 = max(x0, floor((ubar - hx + cx) / T)), x1 = min(x1, floor((ubar + hx + cx) / T) + 1);
 *   clamped to the tile grid; an empty rectangle is not visible.
 *
 * Knife edges.  Beside each value that is rounded to an integer or compared
 * with a threshold, a first-order bound e on how far an FP32 evaluation of
 * these steps can land from the exact value (Wilkinson's running error
 * analysis: every operation carries its operands' bounds forward and adds half
 * an ulp of its own FP32 result; the FP32 exp and log add their ulp bounds;
 * FP32 constants such as 0.3f carry their own rounding).  An integer output is
 * returned with the range of values that value +- ORC_KNIFE e can round to, and
 * vis_amb says whether visibility itself lies within such a window.  A
 * different FP32 decision outside these ranges is an error, not rounding. */

#define ORC_U32 5.9604644775390625e-08      /* 2^-24: unit roundoff of FP32 */
#define ORC_KNIFE 2.0                       /* windows are twice the first-order bound */

typedef struct { double v, e; } rb_t;

static rb_t rb_exact(double v) { rb_t r = {v, 0.0}; return r; }
static rb_t rb_const32(double v) { rb_t r = {v, ORC_U32 * fabs(v)}; return r; }
static rb_t rb_round(double v, double e) { rb_t r = {v, e + ORC_U32 * fabs(v)}; return r; }
static rb_t rb_add(rb_t a, rb_t b) { return rb_round(a.v + b.v, a.e + b.e); }
static rb_t rb_sub(rb_t a, rb_t b) { return rb_round(a.v - b.v, a.e + b.e); }
static rb_t rb_neg(rb_t a) { rb_t r = {-a.v, a.e}; return r; }
static rb_t rb_mul(rb_t a, rb_t b)
{
    return rb_round(a.v * b.v, fabs(a.v) * b.e + fabs(b.v) * a.e + a.e * b.e);
}
static rb_t rb_div(rb_t a, rb_t b)
{
    double q = a.v / b.v, den = fabs(b.v) - b.e;
    return rb_round(q, den > 0.0 ? (a.e + fabs(q) * b.e) / den : INFINITY);
}
static rb_t rb_sqrt(rb_t a)
{
    double r = a.v > 0.0 ? sqrt(a.v) : 0.0;
    double lo = a.v - a.e > 0.0 ? sqrt(a.v - a.e) : 0.0;
    return rb_round(r, r - lo);          /* concave: the downward step is the larger */
}
static rb_t rb_maxc(rb_t a, double c)
{
    if (a.v - a.e >= c) return a;
    rb_t r = {a.v > c ? a.v : c, a.v + a.e <= c ? 0.0 : a.e};
    return r;
}
static rb_t rb_clamp(rb_t a, double lim)
{
    rb_t r = a;
    if (a.v > lim) r.v = lim;
    if (a.v < -lim) r.v = -lim;
    if (fabs(a.v) - a.e > lim) r.e = 0.0;
    return r;
}
/* exp and log of the decision path: within 2 and 4 ulp of the exact result */
static rb_t rb_exp(rb_t a)
{
    double v = exp(a.v);
    rb_t r = {v, v * expm1(a.e) + 4.0 * ORC_U32 * v};
    return r;
}
static rb_t rb_log(rb_t a)
{
    double v = log(a.v), den = a.v - a.e;
    rb_t r = {v, (den > 0.0 ? -log1p(-a.e / a.v) : INFINITY) + 8.0 * ORC_U32 * fabs(v) + 1e-12};
    return r;
}

typedef struct {
    int32_t visible, vis_amb;                 /* FP64 decision; 1 = visibility is a knife edge */
    int32_t radius, r_lo, r_hi;               /* ceil(3 sqrt(lambda)) and its reachable range */
    int32_t rect[4], rect_lo[4], rect_hi[4];  /* [x0, x1, y0, y1], clamped; reachable ranges */
    double tz, e_tz, ubar, e_u, vbar, e_v, rho, e_rho, hx, e_hx, hy, e_hy, thr, e_thr, det, e_det;
} orc_dec64;

static int clampi(double v, int hi) { return v < 0.0 ? 0 : (v > hi ? hi : (int)v); }

static void decide64_one(const float *m, const float *ls, const float *qf, float logit,
                         const orc_camera *cam, int tile, int clip, orc_dec64 *o, int *status)
{
    memset(o, 0, sizeof(*o));
    int finite = f_isfinite(m[0]) & f_isfinite(m[1]) & f_isfinite(m[2]) & f_isfinite(ls[0]) &
                 f_isfinite(ls[1]) & f_isfinite(ls[2]) & f_isfinite(qf[0]) & f_isfinite(qf[1]) &
                 f_isfinite(qf[2]) & f_isfinite(qf[3]) & f_isfinite(logit);
    if (!finite) { *status |= 2; return; }
    const int gw = (cam->width + tile - 1) / tile, gh = (cam->height + tile - 1) / tile;
    /* 3D covariance */
    rb_t s[3];
    for (int j = 0; j < 3; ++j) s[j] = rb_exp(rb_exact(ls[j]));
    rb_t qq = rb_mul(rb_exact(qf[0]), rb_exact(qf[0]));
    for (int i = 1; i < 4; ++i) qq = rb_add(qq, rb_mul(rb_exact(qf[i]), rb_exact(qf[i])));
    if (!(qq.v > 0.0)) { *status |= 1; return; }
    rb_t iq = rb_div(rb_exact(1.0), rb_sqrt(qq));
    rb_t w = rb_mul(rb_exact(qf[0]), iq), x = rb_mul(rb_exact(qf[1]), iq);
    rb_t y = rb_mul(rb_exact(qf[2]), iq), z = rb_mul(rb_exact(qf[3]), iq);
    rb_t one = rb_exact(1.0), two = rb_exact(2.0);
    rb_t R[9];
    R[0] = rb_sub(one, rb_mul(two, rb_add(rb_mul(y, y), rb_mul(z, z))));
    R[1] = rb_mul(two, rb_sub(rb_mul(x, y), rb_mul(w, z)));
    R[2] = rb_mul(two, rb_add(rb_mul(x, z), rb_mul(w, y)));
    R[3] = rb_mul(two, rb_add(rb_mul(x, y), rb_mul(w, z)));
    R[4] = rb_sub(one, rb_mul(two, rb_add(rb_mul(x, x), rb_mul(z, z))));
    R[5] = rb_mul(two, rb_sub(rb_mul(y, z), rb_mul(w, x)));
    R[6] = rb_mul(two, rb_sub(rb_mul(x, z), rb_mul(w, y)));
    R[7] = rb_mul(two, rb_add(rb_mul(y, z), rb_mul(w, x)));
    R[8] = rb_sub(one, rb_mul(two, rb_add(rb_mul(x, x), rb_mul(y, y))));
    rb_t M[9], Sig[9];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) M[3 * i + k] = rb_mul(R[3 * i + k], s[k]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            rb_t a = rb_mul(M[3 * i], M[3 * j]);
            for (int k = 1; k < 3; ++k) a = rb_add(a, rb_mul(M[3 * i + k], M[3 * j + k]));
            Sig[3 * i + j] = a;
        }
    /* camera-space mean */
    rb_t tc[3];
    for (int r = 0; r < 3; ++r) {
        rb_t a = rb_mul(rb_exact(cam->R[3 * r]), rb_exact(m[0]));
        a = rb_add(a, rb_mul(rb_exact(cam->R[3 * r + 1]), rb_exact(m[1])));
        a = rb_add(a, rb_mul(rb_exact(cam->R[3 * r + 2]), rb_exact(m[2])));
        tc[r] = rb_add(a, rb_exact(cam->t[r]));
    }
    o->tz = tc[2].v;
    o->e_tz = tc[2].e;
    const double zn = cam->znear, wz = ORC_KNIFE * tc[2].e;
    if (tc[2].v + wz <= zn) return;                         /* certainly behind the near plane */
    int amb = !(tc[2].v - wz > zn);
    int vis = tc[2].v > zn;
    /* Jacobian with the 1.3 x half-FOV guard, T = J W */
    rb_t iz = rb_div(one, tc[2]);
    rb_t rx = rb_mul(tc[0], iz), ry = rb_mul(tc[1], iz);
    rb_t limx = rb_mul(rb_exact(1.3f), rb_exact(cam->tan_fovx));
    rb_t limy = rb_mul(rb_exact(1.3f), rb_exact(cam->tan_fovy));
    rb_t cx_ = rb_clamp(rx, limx.v), cy_ = rb_clamp(ry, limy.v);
    rb_t j00 = rb_mul(rb_exact(cam->fx), iz), j11 = rb_mul(rb_exact(cam->fy), iz);
    rb_t j02 = rb_neg(rb_mul(j00, cx_)), j12 = rb_neg(rb_mul(j11, cy_));
    rb_t T[6];
    for (int k = 0; k < 3; ++k) {
        T[k] = rb_add(rb_mul(j00, rb_exact(cam->R[k])), rb_mul(j02, rb_exact(cam->R[6 + k])));
        T[3 + k] = rb_add(rb_mul(j11, rb_exact(cam->R[3 + k])), rb_mul(j12, rb_exact(cam->R[6 + k])));
    }
    /* Sigma' = T Sigma T^T + 0.3 I */
    rb_t TS[6], S2[4];
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j) {
            rb_t v = rb_mul(T[3 * a], Sig[j]);
            for (int i = 1; i < 3; ++i) v = rb_add(v, rb_mul(T[3 * a + i], Sig[3 * i + j]));
            TS[3 * a + j] = v;
        }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            rb_t v = rb_mul(TS[3 * a], T[3 * b]);
            for (int j = 1; j < 3; ++j) v = rb_add(v, rb_mul(TS[3 * a + j], T[3 * b + j]));
            S2[2 * a + b] = v;
        }
    rb_t dil = rb_const32(0.3);
    rb_t A = rb_add(S2[0], dil), B = S2[1], C = rb_add(S2[3], dil);
    rb_t det = rb_sub(rb_mul(A, C), rb_mul(B, B));
    o->det = det.v;
    o->e_det = det.e;
    if (det.v + ORC_KNIFE * det.e <= 0.0) return;
    amb |= !(det.v - ORC_KNIFE * det.e > 0.0);
    vis &= det.v > 0.0;
    rb_t mid = rb_mul(rb_exact(0.5), rb_add(A, C));
    rb_t disc = rb_maxc(rb_sub(rb_mul(mid, mid), det), 0.1);
    disc.e += ORC_U32 * 0.1;
    rb_t lam = rb_add(mid, rb_sqrt(disc));
    rb_t rho = rb_mul(rb_exact(3.0), rb_sqrt(lam));
    o->rho = rho.v;
    o->e_rho = rho.e;
    const double wr = ORC_KNIFE * rho.e;
    const double r = ceil(rho.v), r_lo = ceil(rho.v - wr), r_hi = ceil(rho.v + wr);
    o->radius = (int32_t)r;
    o->r_lo = (int32_t)r_lo;
    o->r_hi = (int32_t)r_hi;
    rb_t ub = rb_mul(rb_exact(cam->fx), rx), vb = rb_mul(rb_exact(cam->fy), ry);
    o->ubar = ub.v; o->e_u = ub.e;
    o->vbar = vb.v; o->e_v = vb.e;
    /* half extents: the 3-sigma radius, or the alpha >= 1/255 box when it is nearer */
    double hx = INFINITY, hy = INFINITY, whx = 0.0, why = 0.0;
    if (clip) {
        rb_t eo = rb_exp(rb_exact(-(double)logit));
        rb_t op = rb_div(one, rb_add(one, eo));
        rb_t thr = rb_mul(two, rb_log(rb_mul(rb_exact(255.0), op)));
        thr = rb_add(rb_mul(thr, rb_const32(1.001)), rb_const32(0.001));
        o->thr = thr.v;
        o->e_thr = thr.e;
        if (thr.v + ORC_KNIFE * thr.e <= 0.0) return;
        amb |= !(thr.v - ORC_KNIFE * thr.e > 0.0);
        vis &= thr.v > 0.0;
        rb_t bx = rb_sqrt(rb_mul(rb_maxc(thr, 0.0), A)), by = rb_sqrt(rb_mul(rb_maxc(thr, 0.0), C));
        hx = bx.v; whx = ORC_KNIFE * bx.e;
        hy = by.v; why = ORC_KNIFE * by.e;
        o->hx = hx; o->e_hx = bx.e;
        o->hy = hy; o->e_hy = by.e;
    }
    /* each bound: floor((centre -+ min(r, h) + principal point) / T); the FP32 edge
     * is one more rounded subtraction, then an exact floor */
    const double ctr[2] = {ub.v, vb.v}, wc[2] = {ORC_KNIFE * ub.e, ORC_KNIFE * vb.e};
    const double h[2] = {hx, hy}, wh[2] = {whx, why}, pp[2] = {cam->cx, cam->cy};
    const int gsz[2] = {gw, gh};
    for (int ax = 0; ax < 2; ++ax) {
        const double e0 = h[ax] < r ? h[ax] : r;                                 /* point */
        const double e_lo = fmin(r_lo, h[ax] - wh[ax]), e_hi = fmin(r_hi, h[ax] + wh[ax]);
        const double wround = ORC_KNIFE * ORC_U32 * (fabs(ctr[ax]) + e_hi);
        const double lo_lo = ctr[ax] - wc[ax] - e_hi - wround, lo_hi = ctr[ax] + wc[ax] - e_lo + wround;
        const double hi_lo = ctr[ax] - wc[ax] + e_lo - wround, hi_hi = ctr[ax] + wc[ax] + e_hi + wround;
        const int g = gsz[ax];
        o->rect[2 * ax] = clampi(floor((ctr[ax] - e0 + pp[ax]) / tile), g);
        o->rect[2 * ax + 1] = clampi(floor((ctr[ax] + e0 + pp[ax]) / tile) + 1.0, g);
        o->rect_lo[2 * ax] = clampi(floor((lo_lo + pp[ax]) / tile), g);
        o->rect_hi[2 * ax] = clampi(floor((lo_hi + pp[ax]) / tile), g);
        o->rect_lo[2 * ax + 1] = clampi(floor((hi_lo + pp[ax]) / tile) + 1.0, g);
        o->rect_hi[2 * ax + 1] = clampi(floor((hi_hi + pp[ax]) / tile) + 1.0, g);
    }
    const int *rc = o->rect, *lo = o->rect_lo, *hi = o->rect_hi;
    const int nonempty = rc[1] > rc[0] && rc[3] > rc[2];
    const int surely = lo[1] > hi[0] && lo[3] > hi[2];
    const int surely_not = hi[1] <= lo[0] || hi[3] <= lo[2];
    if (surely_not) vis = 0, amb = 0;
    else amb |= !surely;
    vis &= nonempty;
    if (!vis) memset(o->rect, 0, sizeof(o->rect));
    o->visible = vis;
    o->vis_amb = amb;
}

int orc_decide64(int n, const float *means, const float *log_scales, const float *quats,
                 const float *logits, const orc_camera *cam, int tile, int clip, orc_dec64 *out)
{
    int status = 0;
#pragma omp parallel for schedule(static) reduction(| : status)
    for (int g = 0; g < n; ++g) {
        int st = 0;
        decide64_one(means + 3 * g, log_scales + 3 * g, quats + 4 * g, logits[g], cam, tile, clip,
                     out + g, &st);
        status |= st;
    }
    return status;
}

/* ------------------------------------------------------------------------- */
/* Compositing.  The candidate list of a pixel is every visible Gaussian whose
 * tile rectangle holds the pixel's tile, ordered by (FP32 depth key, index):
 * the tile's sorted instance list.  Front to back, each candidate gets
 *   power = -1/2 (a dx^2 + c dy^2) - b dx dy ,  d = 2D mean - pixel centre,
 *   alpha = min(0.99, opacity * exp(power)), skipped if power > 0 or alpha < 1/255;
 *   T' = T (1 - alpha); if T' < 1e-4 the pixel stops without this candidate;
 *   otherwise C += rgb alpha T, D += depth alpha T (Eq. 1), T = T'.
 * n_contrib is the 1-based position of the last blended candidate.
 * flags: bit 1 = some alpha within the relative window of 1/255,
 *        bit 2 = some T' within the relative window of 1e-4.             */

typedef struct { float key; int32_t idx; } cand_t;

static int cand_cmp(const void *pa, const void *pb)
{
    const cand_t *a = (const cand_t *)pa, *b = (const cand_t *)pb;
    uint32_t ka, kb;
    memcpy(&ka, &a->key, 4);
    memcpy(&kb, &b->key, 4);
    if (ka != kb) return ka < kb ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

typedef struct {
    double alpha_win;   /* relative window around 1/255 that flags a pixel */
    double t_win;       /* relative window around 1e-4 that flags a pixel */
} orc_flag_opts;

static void composite_pixel(const cand_t *cands, int nc, const orc_proj *P, double pxc, double pyc,
                            const orc_flag_opts *fo, double *rgb, double *dep, double *Tout,
                            int32_t *last_out, uint8_t *flag_out, int32_t *sig_out)
{
    double T = 1.0, C[3] = {0, 0, 0}, D = 0.0;
    int last = 0, nblend = 0, nclamp = 0;
    uint8_t flag = 0;
    for (int p = 0; p < nc; ++p) {
        const orc_proj *g = P + cands[p].idx;
        double dx = g->ubar - pxc, dy = g->vbar - pyc;
        double power = -0.5 * (g->conic[0] * dx * dx + g->conic[2] * dy * dy) - g->conic[1] * dx * dy;
        if (power > 0.0) continue;
        double raw = g->opacity * exp(power);
        if (fabs(raw * 255.0 - 1.0) < fo->alpha_win) flag |= 1;
        double alpha = raw < 0.99 ? raw : 0.99;
        if (alpha < 1.0 / 255.0) continue;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn * 1e4 - 1.0) < fo->t_win) flag |= 2;
        if (Tn < 1e-4) break;
        double w = alpha * T;
        for (int ch = 0; ch < 3; ++ch) C[ch] += g->rgb[ch] * w;
        D += g->depth * w;
        T = Tn;
        last = p + 1;
        ++nblend;
        if (raw >= 0.99) ++nclamp;
    }
    rgb[0] = C[0]; rgb[1] = C[1]; rgb[2] = C[2];
    *dep = D;
    *Tout = T;
    *last_out = last;
    *flag_out = flag;
    /* signature of the blended set: changes when any discrete choice changes */
    *sig_out = nblend + 65536 * nclamp;
}

/* Brute force: every pixel scans all n Gaussians.  Outputs are CHW. */
void orc_render_brute(int n, const uint8_t *visible, const float *depth_key, const int32_t *rect,
                      const orc_proj *P, const orc_camera *cam, int tile, const orc_flag_opts *fo,
                      double *rgb, double *depth, double *Tfin, int32_t *n_contrib, uint8_t *flags,
                      int32_t *sig)
{
    const int W = cam->width, H = cam->height;
    const size_t HW = (size_t)W * H;
#pragma omp parallel
    {
        cand_t *cands = (cand_t *)malloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 4)
        for (int j = 0; j < H; ++j) {
            for (int i = 0; i < W; ++i) {
                int tx = i / tile, ty = j / tile, nc = 0;
                for (int g = 0; g < n; ++g) {
                    if (!visible[g]) continue;
                    const int32_t *r = rect + 4 * g;
                    if (tx < r[0] || tx >= r[1] || ty < r[2] || ty >= r[3]) continue;
                    cands[nc].key = depth_key[g];
                    cands[nc].idx = g;
                    ++nc;
                }
                qsort(cands, nc, sizeof(cand_t), cand_cmp);
                double c3[3], d, T;
                int32_t last, sg;
                uint8_t fl;
                composite_pixel(cands, nc, P, i + 0.5 - cam->cx, j + 0.5 - cam->cy, fo, c3, &d, &T,
                                &last, &fl, &sg);
                size_t pix = (size_t)j * W + i;
                rgb[pix] = c3[0]; rgb[HW + pix] = c3[1]; rgb[2 * HW + pix] = c3[2];
                depth[pix] = d; Tfin[pix] = T; n_contrib[pix] = last; flags[pix] = fl; sig[pix] = sg;
            }
        }
        free(cands);
    }
}

/* Per-tile candidate lists, built by scanning each Gaussian's rectangle. */
typedef struct { int32_t *start; int32_t *count; cand_t *items; int ntiles; } tile_lists;

static void build_tile_lists(int n, const uint8_t *visible, const float *depth_key,
                             const int32_t *rect, int gw, int gh, tile_lists *L)
{
    int nt = gw * gh;
    L->ntiles = nt;
    L->start = (int32_t *)calloc((size_t)nt + 1, sizeof(int32_t));
    L->count = (int32_t *)calloc((size_t)nt, sizeof(int32_t));
    int64_t total = 0;
    for (int g = 0; g < n; ++g) {
        if (!visible[g]) continue;
        const int32_t *r = rect + 4 * g;
        for (int y = r[2]; y < r[3]; ++y)
            for (int x = r[0]; x < r[1]; ++x) { L->count[y * gw + x]++; ++total; }
    }
    int64_t acc = 0;
    for (int t = 0; t < nt; ++t) { L->start[t] = (int32_t)acc; acc += L->count[t]; }
    L->start[nt] = (int32_t)acc;
    L->items = (cand_t *)malloc(sizeof(cand_t) * (size_t)(total > 0 ? total : 1));
    int32_t *fill = (int32_t *)calloc((size_t)nt, sizeof(int32_t));
    for (int g = 0; g < n; ++g) {
        if (!visible[g]) continue;
        const int32_t *r = rect + 4 * g;
        for (int y = r[2]; y < r[3]; ++y)
            for (int x = r[0]; x < r[1]; ++x) {
                int t = y * gw + x;
                cand_t *c = L->items + L->start[t] + fill[t]++;
                c->key = depth_key[g];
                c->idx = g;
            }
    }
    free(fill);
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < nt; ++t)
        qsort(L->items + L->start[t], L->count[t], sizeof(cand_t), cand_cmp);
}

static void free_tile_lists(tile_lists *L) { free(L->start); free(L->count); free(L->items); }

/* Bucketed: each pixel iterates its tile's list only; the same result as the
 * brute force.  `tile_mask` (nullable, gw*gh bytes) restricts the work to the
 * tiles marked 1; other pixels are left untouched (used for bounded timing). */
void orc_render_bucketed(int n, const uint8_t *visible, const float *depth_key, const int32_t *rect,
                         const orc_proj *P, const orc_camera *cam, int tile, const orc_flag_opts *fo,
                         const uint8_t *tile_mask, double *rgb, double *depth, double *Tfin,
                         int32_t *n_contrib, uint8_t *flags, int32_t *sig)
{
    const int W = cam->width, H = cam->height;
    const size_t HW = (size_t)W * H;
    const int gw = (W + tile - 1) / tile, gh = (H + tile - 1) / tile;
    tile_lists L;
    build_tile_lists(n, visible, depth_key, rect, gw, gh, &L);
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < gw * gh; ++t) {
        if (tile_mask && !tile_mask[t]) continue;
        int tx = t % gw, ty = t / gw;
        for (int j = ty * tile; j < (ty + 1) * tile && j < H; ++j)
            for (int i = tx * tile; i < (tx + 1) * tile && i < W; ++i) {
                double c3[3], d, T;
                int32_t last, sg;
                uint8_t fl;
                composite_pixel(L.items + L.start[t], L.count[t], P, i + 0.5 - cam->cx,
                                j + 0.5 - cam->cy, fo, c3, &d, &T, &last, &fl, &sg);
                size_t pix = (size_t)j * W + i;
                rgb[pix] = c3[0]; rgb[HW + pix] = c3[1]; rgb[2 * HW + pix] = c3[2];
                depth[pix] = d; Tfin[pix] = T; n_contrib[pix] = last; flags[pix] = fl; sig[pix] = sg;
            }
    }
    free_tile_lists(&L);
}

/* ------------------------------------------------------------------------- */
/* Per-pixel depth order: the popping fix of Sec. 3.2, which sorts the Gaussian
 * contributions per pixel instead of per primitive.  A pixel's candidates are
 * the same as above (visible, tile rectangle holding the pixel's tile, alpha >=
 * 1/255 at the pixel); they are ordered by the depth of each Gaussian's 3D
 * density maximum along the pixel's viewing ray, ties by index, and composited
 * front to back with the same skip, clamp and stop rules.  With the camera-space
 * ray r = ((px - cx)/fx, (py - cy)/fy, 1) through the pixel centre, the camera-
 * space mean mu and covariance Sigma_c = W R S S^T R^T W^T, the density along
 * the ray, exp(-1/2 (t r - mu)^T Sigma_c^-1 (t r - mu)), is largest at
 *   t* = r^T Sigma_c^-1 mu / r^T Sigma_c^-1 r,
 * the camera-space z of that point (r has unit z).  Eq. 1 then accumulates
 * these per-pixel depths: d_i = t*_i at the pixel.
 * Near ties.  Neighbours in the order whose t* lie within tie_win relative of
 * each other form a run; an evaluation of t* in lower precision may order a
 * run differently.  Reordering a run does not change its total weight
 * T_start (1 - prod (1 - alpha)), so the colour can move by at most that
 * weight times the run's colour range (and the depth by the weight times its
 * t* range): tie_bound sums the colour bound over the runs.  flags bit 4: the
 * pixel has such a run; bit 8: a run reaches the candidate at which the pixel
 * stops, where another order may stop elsewhere. */

typedef struct { double P[6]; double Pm[3]; } orc_raydepth;   /* Sigma_c^-1 (xx xy xz yy yz zz), Sigma_c^-1 mu */

void orc_raydepth_setup(int n, const float *means, const float *log_scales, const float *quats,
                        const orc_camera *cam, orc_raydepth *out)
{
#pragma omp parallel for schedule(static)
    for (int g = 0; g < n; ++g) {
        const float *m = means + 3 * g, *ls = log_scales + 3 * g, *qf = quats + 4 * g;
        double q[4] = {qf[0], qf[1], qf[2], qf[3]};
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        orc_raydepth *o = out + g;
        memset(o, 0, sizeof(*o));
        if (!(qn > 0.0)) continue;
        for (int i = 0; i < 4; ++i) q[i] /= qn;
        double Rq[9];
        quat_to_rot(q, Rq);
        double W[9];
        for (int i = 0; i < 9; ++i) W[i] = cam->R[i];
        /* camera-space axes e_k = W R_k; Sigma_c^-1 = sum_k e_k e_k^T / s_k^2 */
        double Pm[9] = {0};
        for (int k = 0; k < 3; ++k) {
            double e[3];
            for (int i = 0; i < 3; ++i) e[i] = W[3 * i] * Rq[k] + W[3 * i + 1] * Rq[3 + k] + W[3 * i + 2] * Rq[6 + k];
            double is2 = exp(-2.0 * (double)ls[k]);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) Pm[3 * i + j] += e[i] * e[j] * is2;
        }
        double mu[3];
        for (int r = 0; r < 3; ++r)
            mu[r] = W[3 * r] * m[0] + W[3 * r + 1] * m[1] + W[3 * r + 2] * m[2] + cam->t[r];
        o->P[0] = Pm[0]; o->P[1] = Pm[1]; o->P[2] = Pm[2]; o->P[3] = Pm[4]; o->P[4] = Pm[5]; o->P[5] = Pm[8];
        for (int i = 0; i < 3; ++i) o->Pm[i] = Pm[3 * i] * mu[0] + Pm[3 * i + 1] * mu[1] + Pm[3 * i + 2] * mu[2];
    }
}

static double ray_depth(const orc_raydepth *g, double rx, double ry)
{
    const double *P = g->P;
    double num = rx * g->Pm[0] + ry * g->Pm[1] + g->Pm[2];
    double den = P[0] * rx * rx + 2.0 * P[1] * rx * ry + 2.0 * P[2] * rx + P[3] * ry * ry + 2.0 * P[4] * ry + P[5];
    return num / den;
}

typedef struct { double t; int32_t idx; double alpha; } pix_cand_t;

static int pix_cand_cmp(const void *pa, const void *pb)
{
    const pix_cand_t *a = (const pix_cand_t *)pa, *b = (const pix_cand_t *)pb;
    if (a->t != b->t) return a->t < b->t ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

static void composite_pixel_resort(const cand_t *cands, int nc, const orc_proj *P, const orc_raydepth *RD,
                                   double pxc, double pyc, double rx, double ry, const orc_flag_opts *fo,
                                   double tie_win, pix_cand_t *buf, double *rgb, double *dep, double *Tout,
                                   uint8_t *flag_out, int32_t *nblend_out, double *tie_out)
{
    uint8_t flag = 0;
    int m = 0;
    for (int p = 0; p < nc; ++p) {
        const int gi = cands[p].idx;
        const orc_proj *g = P + gi;
        double dx = g->ubar - pxc, dy = g->vbar - pyc;
        double power = -0.5 * (g->conic[0] * dx * dx + g->conic[2] * dy * dy) - g->conic[1] * dx * dy;
        if (power > 0.0) continue;
        double raw = g->opacity * exp(power);
        if (fabs(raw * 255.0 - 1.0) < fo->alpha_win) flag |= 1;
        double alpha = raw < 0.99 ? raw : 0.99;
        if (alpha < 1.0 / 255.0) continue;
        buf[m].t = ray_depth(RD + gi, rx, ry);
        buf[m].idx = gi;
        buf[m].alpha = alpha;
        ++m;
    }
    qsort(buf, m, sizeof(pix_cand_t), pix_cand_cmp);
    double T = 1.0, C[3] = {0, 0, 0}, D = 0.0;
    int nb = 0, stop = -1;
    for (int k = 0; k < m; ++k) {
        const orc_proj *g = P + buf[k].idx;
        double alpha = buf[k].alpha;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn * 1e4 - 1.0) < fo->t_win) flag |= 2;
        if (Tn < 1e-4) { stop = k; break; }
        double w = alpha * T;
        for (int ch = 0; ch < 3; ++ch) C[ch] += g->rgb[ch] * w;
        D += buf[k].t * w;
        T = Tn;
        ++nb;
    }
    /* runs of near-tied neighbours among the blended candidates and the stopping one */
    const int last = stop >= 0 ? stop : nb - 1;
    double tie = 0.0, Tr = 1.0;
    int k = 0;
    while (k <= last) {
        int e = k;
        while (e < last && fabs(buf[e + 1].t - buf[e].t) <= tie_win * fmax(fabs(buf[e + 1].t), fabs(buf[e].t)))
            ++e;
        double keep = 1.0, lo[3], hi[3];
        for (int ch = 0; ch < 3; ++ch) lo[ch] = hi[ch] = P[buf[k].idx].rgb[ch];
        for (int j = k; j <= e; ++j) {
            if (j < nb) keep *= 1.0 - buf[j].alpha;
            for (int ch = 0; ch < 3; ++ch) {
                double c = P[buf[j].idx].rgb[ch];
                lo[ch] = c < lo[ch] ? c : lo[ch];
                hi[ch] = c > hi[ch] ? c : hi[ch];
            }
        }
        if (e > k) {
            flag |= 4;
            if (e == stop) flag |= 8;
            double range = 0.0;
            for (int ch = 0; ch < 3; ++ch) range = hi[ch] - lo[ch] > range ? hi[ch] - lo[ch] : range;
            tie += Tr * (1.0 - keep) * range;
        }
        Tr *= keep;
        k = e + 1;
    }
    rgb[0] = C[0]; rgb[1] = C[1]; rgb[2] = C[2];
    *dep = D;
    *Tout = T;
    *flag_out = flag;
    *nblend_out = nb;
    *tie_out = tie;
}

void orc_render_resort(int n, const uint8_t *visible, const float *depth_key, const int32_t *rect,
                       const orc_proj *P, const orc_raydepth *RD, const orc_camera *cam, int tile,
                       const orc_flag_opts *fo, double tie_win, const uint8_t *tile_mask, double *rgb,
                       double *depth, double *Tfin, uint8_t *flags, int32_t *nblend, double *tie_bound)
{
    const int W = cam->width, H = cam->height;
    const size_t HW = (size_t)W * H;
    const int gw = (W + tile - 1) / tile, gh = (H + tile - 1) / tile;
    tile_lists L;
    build_tile_lists(n, visible, depth_key, rect, gw, gh, &L);
    int maxc = 1;
    for (int t = 0; t < gw * gh; ++t) if (L.count[t] > maxc) maxc = L.count[t];
#pragma omp parallel
    {
        pix_cand_t *buf = (pix_cand_t *)malloc(sizeof(pix_cand_t) * (size_t)maxc);
#pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < gw * gh; ++t) {
            if (tile_mask && !tile_mask[t]) continue;
            int tx = t % gw, ty = t / gw;
            for (int j = ty * tile; j < (ty + 1) * tile && j < H; ++j)
                for (int i = tx * tile; i < (tx + 1) * tile && i < W; ++i) {
                    double c3[3], d, T;
                    uint8_t fl;
                    int32_t nb;
                    double tb;
                    const double pxc = i + 0.5 - cam->cx, pyc = j + 0.5 - cam->cy;
                    composite_pixel_resort(L.items + L.start[t], L.count[t], P, RD, pxc, pyc,
                                           pxc / cam->fx, pyc / cam->fy, fo, tie_win, buf, c3, &d, &T,
                                           &fl, &nb, &tb);
                    size_t pix = (size_t)j * W + i;
                    rgb[pix] = c3[0]; rgb[HW + pix] = c3[1]; rgb[2 * HW + pix] = c3[2];
                    depth[pix] = d; Tfin[pix] = T; flags[pix] = fl; nblend[pix] = nb; tie_bound[pix] = tb;
                }
        }
        free(buf);
    }
    free_tile_lists(&L);
}

/* ------------------------------------------------------------------------- */
/* Reverse pass.  For each pixel the forward list is recomputed; with
 * w_i = alpha_i T_i, T_i = prod_{m<i} (1 - alpha_m) (a prefix product, no
 * division), and the explicit suffix sums S_C,i = sum_{j>i} rgb_j w_j,
 * S_D,i = sum_{j>i} d_j w_j over the blended candidates:
 *   dL/drgb_i   += g_C w_i ,   dL/ddepth_i += g_D w_i ,
 *   dL/dalpha_i  = T_i (g_C . rgb_i + g_D d_i) - (g_C . S_C,i + g_D S_D,i + g_T T_final) / (1 - alpha_i),
 * and, where alpha was not clamped at 0.99, through alpha = o exp(power):
 *   dL/do += dL/dalpha exp(power);  dL/dpower = dL/dalpha alpha.
 * Per-Gaussian 2D gradients (FP64), 10 per Gaussian:
 *   [d ubar, d vbar, d conic_a, d conic_b, d conic_c, d opacity, d r, d g, d b, d depth]. */

#define G2_N 10

static void reverse_pixel(const cand_t *cands, int nc, const orc_proj *P, double pxc, double pyc,
                          const double *gC, double gD, double gT, double *g2, int *blend_idx,
                          double *alpha_s, double *Tpre, double *powr)
{
    /* forward again, recording the blended candidates */
    double T = 1.0;
    int nb = 0;
    for (int p = 0; p < nc; ++p) {
        const orc_proj *g = P + cands[p].idx;
        double dx = g->ubar - pxc, dy = g->vbar - pyc;
        double power = -0.5 * (g->conic[0] * dx * dx + g->conic[2] * dy * dy) - g->conic[1] * dx * dy;
        if (power > 0.0) continue;
        double raw = g->opacity * exp(power);
        double alpha = raw < 0.99 ? raw : 0.99;
        if (alpha < 1.0 / 255.0) continue;
        double Tn = T * (1.0 - alpha);
        if (Tn < 1e-4) break;
        blend_idx[nb] = p;
        alpha_s[nb] = alpha;
        powr[nb] = power;
        Tpre[nb] = T;
        ++nb;
        T = Tn;
    }
    const double Tfinal = T;
    /* suffix sums by an explicit backward accumulation over the blended list */
    double SC[3] = {0, 0, 0}, SD = 0.0;
    for (int b = nb - 1; b >= 0; --b) {
        const int gi = cands[blend_idx[b]].idx;
        const orc_proj *g = P + gi;
        const double a = alpha_s[b], Ti = Tpre[b], w = a * Ti;
        double *o = g2 + (size_t)G2_N * gi;
        for (int ch = 0; ch < 3; ++ch) o[6 + ch] += gC[ch] * w;
        o[9] += gD * w;
        double dot_c = gC[0] * g->rgb[0] + gC[1] * g->rgb[1] + gC[2] * g->rgb[2];
        double dot_s = gC[0] * SC[0] + gC[1] * SC[1] + gC[2] * SC[2];
        double dL_da = Ti * (dot_c + gD * g->depth) - (dot_s + gD * SD + gT * Tfinal) / (1.0 - a);
        double raw = g->opacity * exp(powr[b]);
        if (raw < 0.99) {
            double ex = exp(powr[b]);
            o[5] += dL_da * ex;
            double dL_dp = dL_da * a;
            double dx = g->ubar - pxc, dy = g->vbar - pyc;
            o[0] += dL_dp * (-(g->conic[0] * dx + g->conic[1] * dy));
            o[1] += dL_dp * (-(g->conic[2] * dy + g->conic[1] * dx));
            o[2] += dL_dp * (-0.5 * dx * dx);
            o[3] += dL_dp * (-dx * dy);
            o[4] += dL_dp * (-0.5 * dy * dy);
        }
        for (int ch = 0; ch < 3; ++ch) SC[ch] += g->rgb[ch] * w;
        SD += g->depth * w;
    }
}

/* dL_drgb [3,H,W], dL_ddepth [H,W], dL_dT [H,W] (nullable); g2 is [n, 10], accumulated. */
void orc_render_bwd(int n, const uint8_t *visible, const float *depth_key, const int32_t *rect,
                    const orc_proj *P, const orc_camera *cam, int tile, const double *dL_drgb,
                    const double *dL_ddepth, const double *dL_dT, double *g2)
{
    const int W = cam->width, H = cam->height;
    const size_t HW = (size_t)W * H;
    const int gw = (W + tile - 1) / tile, gh = (H + tile - 1) / tile;
    tile_lists L;
    build_tile_lists(n, visible, depth_key, rect, gw, gh, &L);
    int maxc = 1;
    for (int t = 0; t < gw * gh; ++t) if (L.count[t] > maxc) maxc = L.count[t];
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double *acc = (double *)calloc((size_t)nthreads * G2_N * (size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = acc + (size_t)tid * G2_N * (size_t)(n > 0 ? n : 1);
        int *bi = (int *)malloc(sizeof(int) * maxc);
        double *as = (double *)malloc(sizeof(double) * maxc);
        double *tp = (double *)malloc(sizeof(double) * maxc);
        double *pw = (double *)malloc(sizeof(double) * maxc);
#pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < gw * gh; ++t) {
            int tx = t % gw, ty = t / gw;
            for (int j = ty * tile; j < (ty + 1) * tile && j < H; ++j)
                for (int i = tx * tile; i < (tx + 1) * tile && i < W; ++i) {
                    size_t pix = (size_t)j * W + i;
                    double gC[3] = {dL_drgb[pix], dL_drgb[HW + pix], dL_drgb[2 * HW + pix]};
                    reverse_pixel(L.items + L.start[t], L.count[t], P, i + 0.5 - cam->cx,
                                  j + 0.5 - cam->cy, gC, dL_ddepth[pix], dL_dT ? dL_dT[pix] : 0.0,
                                  mine, bi, as, tp, pw);
                }
        }
        free(bi); free(as); free(tp); free(pw);
    }
    for (int th = 0; th < nthreads; ++th)
        for (size_t k = 0; k < (size_t)G2_N * n; ++k) g2[k] += acc[(size_t)th * G2_N * n + k];
    free(acc);
    free_tile_lists(&L);
}

/* ------------------------------------------------------------------------- */
/* Chain rule from the 2D gradients of one view to the Gaussian parameters, in
 * FP64.  Accumulates (+=) into the parameter gradients.  Gaussians that are not
 * visible in the view get nothing. */

void orc_param_grads(int n, const float *means, const float *log_scales, const float *quats,
                     const float *opacity_logits, const float *sh, int K, const orc_camera *cam,
                     const uint8_t *visible, const double *g2, double *g_means, double *g_log_scales,
                     double *g_quats, double *g_logits, double *g_sh)
{
#pragma omp parallel for schedule(static)
    for (int gi = 0; gi < n; ++gi) {
        if (!visible[gi]) continue;
        const double *G = g2 + (size_t)G2_N * gi;
        const float *m = means + 3 * gi, *ls = log_scales + 3 * gi, *qf = quats + 4 * gi;
        const float *shg = sh + (size_t)3 * K * gi;
        orc_proj pr;
        project_one(m, ls, qf, opacity_logits[gi], shg, K, cam, &pr);
        double W[9], t[3];
        for (int i = 0; i < 9; ++i) W[i] = cam->R[i];
        for (int i = 0; i < 3; ++i) t[i] = cam->t[i];
        double mu[3] = {m[0], m[1], m[2]};
        double dmu[3] = {0, 0, 0};

        /* opacity = sigmoid(logit) */
        g_logits[gi] += G[5] * pr.opacity * (1.0 - pr.opacity);

        /* colour: rgb_ch = max(0, sum_k Y_k(dir) sh_k,ch + 0.5), dir = (mu - c)/|mu - c| */
        double cc[3];
        for (int i = 0; i < 3; ++i) cc[i] = -(W[i] * t[0] + W[3 + i] * t[1] + W[6 + i] * t[2]);
        double v[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
        double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double d[3] = {v[0] / vn, v[1] / vn, v[2] / vn};
        double Y[16], Yx[16], Yy[16], Yz[16];
        orc_sh_basis_xyz(d[0], d[1], d[2], Y);
        sh_basis_grad(d[0], d[1], d[2], Yx, Yy, Yz);
        double gdir[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            if (pr.clamp_rgb[ch]) continue;
            double gc = G[6 + ch];
            for (int k = 0; k < K; ++k) {
                g_sh[(size_t)3 * K * gi + 3 * k + ch] += gc * Y[k];
                gdir[0] += gc * shg[3 * k + ch] * Yx[k];
                gdir[1] += gc * shg[3 * k + ch] * Yy[k];
                gdir[2] += gc * shg[3 * k + ch] * Yz[k];
            }
        }
        double dd = d[0] * gdir[0] + d[1] * gdir[1] + d[2] * gdir[2];
        for (int i = 0; i < 3; ++i) dmu[i] += (gdir[i] - d[i] * dd) / vn;

        /* camera-space mean and projection */
        double tc[3];
        for (int r = 0; r < 3; ++r) tc[r] = W[3 * r] * mu[0] + W[3 * r + 1] * mu[1] + W[3 * r + 2] * mu[2] + t[r];
        double tx = tc[0], ty = tc[1], tz = tc[2];
        double dtc[3] = {0, 0, 0};
        /* ubar = fx tx / tz, vbar = fy ty / tz, depth = tz */
        dtc[0] += G[0] * cam->fx / tz;
        dtc[1] += G[1] * cam->fy / tz;
        dtc[2] += -G[0] * cam->fx * tx / (tz * tz) - G[1] * cam->fy * ty / (tz * tz);
        dtc[2] += G[9];

        /* rebuild Sigma, J, T and Sigma' */
        double s[3] = {exp((double)ls[0]), exp((double)ls[1]), exp((double)ls[2])};
        double q[4] = {qf[0], qf[1], qf[2], qf[3]};
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double qh[4] = {q[0] / qn, q[1] / qn, q[2] / qn, q[3] / qn};
        double Rq[9];
        quat_to_rot(qh, Rq);
        double M[9];
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) M[3 * k + j] = Rq[3 * k + j] * s[j];
        double Sig[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double a = 0;
                for (int k = 0; k < 3; ++k) a += M[3 * i + k] * M[3 * j + k];
                Sig[3 * i + j] = a;
            }
        double limx = 1.3 * cam->tan_fovx, limy = 1.3 * cam->tan_fovy;
        double rx = tx / tz, ry = ty / tz;
        double Lx = rx > limx ? limx : (rx < -limx ? -limx : rx);
        double Ly = ry > limy ? limy : (ry < -limy ? -limy : ry);
        double J00 = cam->fx / tz, J11 = cam->fy / tz;
        double J02 = -cam->fx * Lx * tz / (tz * tz), J12 = -cam->fy * Ly * tz / (tz * tz);
        double T0[3], T1[3];
        for (int j = 0; j < 3; ++j) {
            T0[j] = J00 * W[j] + J02 * W[6 + j];
            T1[j] = J11 * W[3 + j] + J12 * W[6 + j];
        }
        double ST0[3], ST1[3];
        for (int i = 0; i < 3; ++i) {
            ST0[i] = Sig[3 * i] * T0[0] + Sig[3 * i + 1] * T0[1] + Sig[3 * i + 2] * T0[2];
            ST1[i] = Sig[3 * i] * T1[0] + Sig[3 * i + 1] * T1[1] + Sig[3 * i + 2] * T1[2];
        }
        double A = T0[0] * ST0[0] + T0[1] * ST0[1] + T0[2] * ST0[2] + 0.3;
        double B = T0[0] * ST1[0] + T0[1] * ST1[1] + T0[2] * ST1[2];
        double C = T1[0] * ST1[0] + T1[1] * ST1[1] + T1[2] * ST1[2] + 0.3;
        double det = A * C - B * B, det2 = det * det;
        /* conic = (C/det, -B/det, A/det): partials w.r.t. (A, B, C) */
        double dca_dA = -C * C / det2, dca_dB = 2.0 * B * C / det2, dca_dC = -B * B / det2;
        double dcb_dA = B * C / det2, dcb_dB = -(A * C + B * B) / det2, dcb_dC = A * B / det2;
        double dcc_dA = -B * B / det2, dcc_dB = 2.0 * A * B / det2, dcc_dC = -A * A / det2;
        double gA = G[2] * dca_dA + G[3] * dcb_dA + G[4] * dcc_dA;
        double gB = G[2] * dca_dB + G[3] * dcb_dB + G[4] * dcc_dB;
        double gC = G[2] * dca_dC + G[3] * dcb_dC + G[4] * dcc_dC;
        /* A = T0' Sig T0 + .3, B = T0' Sig T1, C = T1' Sig T1 + .3 */
        double gSig[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                gSig[3 * i + j] = gA * T0[i] * T0[j] + gB * T0[i] * T1[j] + gC * T1[i] * T1[j];
        double gT0[3], gT1[3];
        for (int i = 0; i < 3; ++i) {
            gT0[i] = 2.0 * gA * ST0[i] + gB * ST1[i];
            gT1[i] = gB * ST0[i] + 2.0 * gC * ST1[i];
        }
        /* T0 = J00 W0 + J02 W2 ; T1 = J11 W1 + J12 W2 */
        double gJ00 = 0, gJ02 = 0, gJ11 = 0, gJ12 = 0;
        for (int j = 0; j < 3; ++j) {
            gJ00 += gT0[j] * W[j];
            gJ02 += gT0[j] * W[6 + j];
            gJ11 += gT1[j] * W[3 + j];
            gJ12 += gT1[j] * W[6 + j];
        }
        dtc[2] += gJ00 * (-cam->fx / (tz * tz)) + gJ11 * (-cam->fy / (tz * tz));
        if (!pr.clamp_x) {   /* J02 = -fx tx / tz^2 */
            dtc[0] += gJ02 * (-cam->fx / (tz * tz));
            dtc[2] += gJ02 * (2.0 * cam->fx * tx / (tz * tz * tz));
        } else {             /* J02 = -fx L / tz */
            dtc[2] += gJ02 * (cam->fx * Lx / (tz * tz));
        }
        if (!pr.clamp_y) {
            dtc[1] += gJ12 * (-cam->fy / (tz * tz));
            dtc[2] += gJ12 * (2.0 * cam->fy * ty / (tz * tz * tz));
        } else {
            dtc[2] += gJ12 * (cam->fy * Ly / (tz * tz));
        }
        /* tc = W mu + t */
        for (int i = 0; i < 3; ++i) dmu[i] += W[i] * dtc[0] + W[3 + i] * dtc[1] + W[6 + i] * dtc[2];
        for (int i = 0; i < 3; ++i) g_means[3 * gi + i] += dmu[i];

        /* Sigma = M M^T (gSig taken as the gradient w.r.t. a general matrix) */
        double gM[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double a = 0;
                for (int k = 0; k < 3; ++k) a += (gSig[3 * i + k] + gSig[3 * k + i]) * M[3 * k + j];
                gM[3 * i + j] = a;
            }
        /* M = Rq S */
        double gR[9];
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) gR[3 * k + j] = gM[3 * k + j] * s[j];
        for (int j = 0; j < 3; ++j) {
            double gs = 0;
            for (int k = 0; k < 3; ++k) gs += gM[3 * k + j] * Rq[3 * k + j];
            g_log_scales[3 * gi + j] += gs * s[j];
        }
        /* Rq(w, x, y, z): explicit partial derivatives of each entry */
        double w = qh[0], x = qh[1], y = qh[2], z = qh[3];
        double dRw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
        double dRx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
        double dRy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
        double dRz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
        double gq[4] = {0, 0, 0, 0};
        for (int i = 0; i < 9; ++i) {
            gq[0] += gR[i] * dRw[i];
            gq[1] += gR[i] * dRx[i];
            gq[2] += gR[i] * dRy[i];
            gq[3] += gR[i] * dRz[i];
        }
        /* q_hat = q / |q| */
        double dot = gq[0] * qh[0] + gq[1] * qh[1] + gq[2] * qh[2] + gq[3] * qh[3];
        for (int i = 0; i < 4; ++i) g_quats[4 * gi + i] += (gq[i] - qh[i] * dot) / qn;
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Occlusion culling of the foveal neural points against the approximate depth
 * buffer (Sec. 3.3: points are projected with the subfrustum's adapted
 * projection, those outside it are discarded, and those hidden behind the
 * Gaussians are culled with the Eq. 1 depth of Sec. 3.2).
 *
 * The paper does not spell out the occlusion test; this oracle states one
 * reading.  Eq. 1 accumulates d_i alpha_i T_i without normalisation, so the
 * surface depth of a pixel is taken as d / (1 - T_final), and a pixel occludes
 * only where its accumulated opacity 1 - T_final is at least alpha_min.  A
 * point is occluded when its view depth exceeds that surface depth scaled by
 * (1 + rel_margin) plus abs_margin.
 *
 * Every step is one correctly rounded FP32 operation in the order written, so
 * that the three-way decision is a definition the kernel can meet exactly.
 * The subfrustum camera is the eye camera with its principal point moved by
 * the crop origin (x0, y0); its pixel (i, j) is pixel (i + x0, j + y0) of the
 * depth map (map_w x map_h, row-major).
 * mask[p]: 0 outside the subfrustum (or behind znear, or non-finite), 1 occluded, 2 kept. */
typedef struct { float alpha_min, rel_margin, abs_margin; int32_t reserved; } orc_cull_opts;

void orc_cull_points(int64_t m, const float *pts, const orc_camera *cam, int32_t x0, int32_t y0,
                     const float *depth, const float *Tfin, int32_t map_w, int32_t map_h,
                     const orc_cull_opts *o, uint8_t *mask)
{
    const float *R = cam->R;
    const float scale = 1.0f + o->rel_margin;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < m; ++p) {
        const float px = pts[3 * p], py = pts[3 * p + 1], pz = pts[3 * p + 2];
        uint8_t r = 0;
        /* camera space, x_cam = R x + t */
        float x = R[0] * px;
        x = x + R[1] * py;
        x = x + R[2] * pz;
        x = x + cam->t[0];
        float y = R[3] * px;
        y = y + R[4] * py;
        y = y + R[5] * pz;
        y = y + cam->t[1];
        float z = R[6] * px;
        z = z + R[7] * py;
        z = z + R[8] * pz;
        z = z + cam->t[2];
        if (z > cam->znear && f_isfinite(x) && f_isfinite(y)) {
            const float iz = 1.0f / z;
            float u = x * iz;
            u = cam->fx * u;
            u = u + cam->cx;
            float v = y * iz;
            v = cam->fy * v;
            v = v + cam->cy;
            if (u >= 0.0f && u < (float)cam->width && v >= 0.0f && v < (float)cam->height) {
                const int32_t mi = (int32_t)u + x0, mj = (int32_t)v + y0;
                if (mi >= 0 && mi < map_w && mj >= 0 && mj < map_h) {
                    const int64_t pix = (int64_t)mj * map_w + mi;
                    const float a = 1.0f - Tfin[pix];
                    r = 2;
                    if (a >= o->alpha_min) {
                        const float dn = depth[pix] / a;
                        float thr = dn * scale;
                        thr = thr + o->abs_margin;
                        if (z > thr) r = 1;
                    }
                }
            }
        }
        mask[p] = r;
    }
}

/* ------------------------------------------------------------------------- */
/* Combination of the peripheral image P and the foveal image F (Sec. 3.4), in
 * FP64 over the foveal crop window [x0, x0 + w) x [y0, y0 + h) of P.
 *
 * For crop pixel (i, j), at P-frame position (u, v) = (x0 + i + 0.5, y0 + j + 0.5):
 *   r_norm = clamp(|(u, v) - (e_x, e_y)| / d_f, 0, 1)
 *   f_p    = (r_norm - m) / (1 - m)
 *   f_e    = S(F, i, j): the magnitude of the Sobel gradient of F's channel mean
 *            (3x3 kernels, weights 1-2-1 across and -1/0/+1 along, divided by 8 so a
 *            unit-slope ramp gives 1), the crop's border replicated
 *   c      = 1 - S2(clamp(f_p + gamma f_e, 0, 1)),  S2(x) = 6x^5 - 15x^4 + 10x^3
 *   out    = (1 - c) p + c f per channel.
 * P is [3][ph][pw], F and out are [3][h][w], c_out (nullable) is [h][w]. */
static double orc_chan_mean(const float *F, int w, int h, int i, int j)
{
    i = i < 0 ? 0 : (i >= w ? w - 1 : i);
    j = j < 0 ? 0 : (j >= h ? h - 1 : j);
    const size_t hw = (size_t)w * h, p = (size_t)j * w + i;
    return ((double)F[p] + (double)F[hw + p] + (double)F[2 * hw + p]) / 3.0;
}

void orc_combine(const float *P, int pw, int ph, const float *F, int w, int h, int x0, int y0,
                 double ex, double ey, double d_f, double m, double gamma, double *out, double *c_out)
{
    const size_t hw = (size_t)w * h, phw = (size_t)pw * ph;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < h; ++j)
        for (int i = 0; i < w; ++i) {
            double du = (x0 + i + 0.5) - ex, dv = (y0 + j + 0.5) - ey;
            double r = sqrt(du * du + dv * dv) / d_f;
            r = r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
            double fp = (r - m) / (1.0 - m);
            double L[3][3];
            for (int b = -1; b <= 1; ++b)
                for (int a = -1; a <= 1; ++a) L[b + 1][a + 1] = orc_chan_mean(F, w, h, i + a, j + b);
            double gx = ((L[0][2] + 2.0 * L[1][2] + L[2][2]) - (L[0][0] + 2.0 * L[1][0] + L[2][0])) / 8.0;
            double gy = ((L[2][0] + 2.0 * L[2][1] + L[2][2]) - (L[0][0] + 2.0 * L[0][1] + L[0][2])) / 8.0;
            double fe = sqrt(gx * gx + gy * gy);
            double x = fp + gamma * fe;
            x = x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
            double s2 = x * x * x * (x * (6.0 * x - 15.0) + 10.0);
            double c = 1.0 - s2;
            const size_t q = (size_t)j * w + i;
            const size_t pp = (size_t)(y0 + j) * pw + (x0 + i);
            for (int ch = 0; ch < 3; ++ch)
                out[ch * hw + q] = (1.0 - c) * (double)P[ch * phw + pp] + c * (double)F[ch * hw + q];
            if (c_out) c_out[q] = c;
        }
}

/* Reverse pass of the combination (Sec. 3.4, for the end-to-end training of
 * Sec. 3.5), in FP64.  With out = p + c (f - p) per channel and
 * c = 1 - S2(x), x = clamp(f_p + gamma f_e, 0, 1):
 *   dL/dp += (1 - c) g,   dL/df += c g (direct),
 *   dL/dc  = sum_ch g (f - p),   dc/dx = -S2'(x) = -30 x^2 (1 - x)^2 inside (0, 1), else 0,
 *   dx/df_e = gamma,   f_e = |(g_x, g_y)| (its gradient taken as 0 where f_e = 0),
 *   g_x, g_y: the Sobel sums over the channel mean L of F (border replicated),
 *   dL/dL at each clamped tap += dL/dg_x k_x / 8 + dL/dg_y k_y / 8,
 *   dL/df_ch += dL/dL / 3.
 * g = dL/dout [3][h][w]; dP [3][ph][pw] (the window is written by +=), dF [3][h][w] (+=). */
void orc_combine_bwd(const float *P, int pw, int ph, const float *F, int w, int h, int x0, int y0,
                     double ex, double ey, double d_f, double m, double gamma, const double *g,
                     double *dP, double *dF)
{
    const size_t hw = (size_t)w * h, phw = (size_t)pw * ph;
    double *dL = (double *)calloc(hw > 0 ? hw : 1, sizeof(double));
    static const int kx[3][3] = {{-1, 0, 1}, {-2, 0, 2}, {-1, 0, 1}};
    static const int ky[3][3] = {{-1, -2, -1}, {0, 0, 0}, {1, 2, 1}};
    for (int j = 0; j < h; ++j)
        for (int i = 0; i < w; ++i) {
            double du = (x0 + i + 0.5) - ex, dv = (y0 + j + 0.5) - ey;
            double r = sqrt(du * du + dv * dv) / d_f;
            r = r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
            double fp = (r - m) / (1.0 - m);
            double gx = 0.0, gy = 0.0;
            for (int b = -1; b <= 1; ++b)
                for (int a = -1; a <= 1; ++a) {
                    double L = orc_chan_mean(F, w, h, i + a, j + b);
                    gx += kx[b + 1][a + 1] * L;
                    gy += ky[b + 1][a + 1] * L;
                }
            gx /= 8.0;
            gy /= 8.0;
            double fe = sqrt(gx * gx + gy * gy);
            double x = fp + gamma * fe;
            double xc = x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
            double c = 1.0 - xc * xc * xc * (xc * (6.0 * xc - 15.0) + 10.0);
            const size_t q = (size_t)j * w + i;
            const size_t pp = (size_t)(y0 + j) * pw + (x0 + i);
            double dLdc = 0.0;
            for (int ch = 0; ch < 3; ++ch) {
                const double gc = g[ch * hw + q];
                dP[ch * phw + pp] += (1.0 - c) * gc;
                dF[ch * hw + q] += c * gc;
                dLdc += gc * ((double)F[ch * hw + q] - (double)P[ch * phw + pp]);
            }
            if (!(x > 0.0 && x < 1.0) || fe == 0.0) continue;
            double dLdfe = dLdc * (-30.0 * x * x * (1.0 - x) * (1.0 - x)) * gamma;
            double dgx = dLdfe * gx / fe, dgy = dLdfe * gy / fe;
            for (int b = -1; b <= 1; ++b)
                for (int a = -1; a <= 1; ++a) {
                    int ii = i + a, jj = j + b;
                    ii = ii < 0 ? 0 : (ii >= w ? w - 1 : ii);
                    jj = jj < 0 ? 0 : (jj >= h ? h - 1 : jj);
                    dL[(size_t)jj * w + ii] += (dgx * kx[b + 1][a + 1] + dgy * ky[b + 1][a + 1]) / 8.0;
                }
        }
    for (size_t q = 0; q < hw; ++q)
        for (int ch = 0; ch < 3; ++ch) dF[ch * hw + q] += dL[q] / 3.0;
    free(dL);
}

/* ------------------------------------------------------------------------- */
/* Training loss of the Gaussian branch (Sec. 3.5: the first two terms of L,
 * identical to 3DGS, with lambda = 0.2): L = (1 - lambda) L1 + lambda (1 - SSIM),
 * L1 the mean absolute difference over the C H W values and SSIM the mean over
 * channels and pixels of the structural similarity of Wang et al. (2004) with
 * an 11 x 11 Gaussian window of standard deviation 1.5 (normalised to sum 1),
 * the window zero outside the image, C1 = 0.01^2 and C2 = 0.03^2:
 *   S = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
 *   mu_x = w * x, s_x^2 = w * x^2 - mu_x^2, s_xy = w * (x y) - mu_x mu_y.
 * Every window sum is written out over the 121 taps (no separable shortcut).
 * The gradient dL/dx follows from S as a function of mu_x, A = w * x^2 and
 * B = w * (x y): dS/dx_p = sum_q w(q - p) (S_mu(q) + 2 x_p S_A(q) + y_p S_B(q)).
 * At x = y the L1 term's gradient is taken as 0 (the subgradient sign(0) = 0). */

#define SSIM_R 5

static void ssim_window(double w[2 * SSIM_R + 1][2 * SSIM_R + 1])
{
    double sum = 0.0;
    for (int i = -SSIM_R; i <= SSIM_R; ++i)
        for (int j = -SSIM_R; j <= SSIM_R; ++j) {
            double v = exp(-(double)(i * i + j * j) / (2.0 * 1.5 * 1.5));
            w[i + SSIM_R][j + SSIM_R] = v;
            sum += v;
        }
    for (int i = 0; i < 2 * SSIM_R + 1; ++i)
        for (int j = 0; j < 2 * SSIM_R + 1; ++j) w[i][j] /= sum;
}

/* image, target: [C][H][W] float32.  out: [0] L, [1] L1, [2] SSIM.  grad (nullable): [C][H][W]. */
void orc_image_loss(const float *image, const float *target, int C, int H, int W, double lambda,
                    double *out, double *grad)
{
    double w[2 * SSIM_R + 1][2 * SSIM_R + 1];
    ssim_window(w);
    const size_t HW = (size_t)H * W, N = (size_t)C * HW;
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    double *Smu = (double *)calloc(N, sizeof(double));
    double *SA = (double *)calloc(N, sizeof(double));
    double *SB = (double *)calloc(N, sizeof(double));
    double l1 = 0.0, ssim = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : l1, ssim)
    for (long long e = 0; e < (long long)N; ++e) {
        const int c = (int)(e / HW);
        const int py = (int)((e % HW) / W), px = (int)(e % W);
        const float *x = image + (size_t)c * HW, *y = target + (size_t)c * HW;
        double mx = 0, my = 0, ex2 = 0, ey2 = 0, exy = 0;
        for (int i = -SSIM_R; i <= SSIM_R; ++i)
            for (int j = -SSIM_R; j <= SSIM_R; ++j) {
                const int qy = py + i, qx = px + j;
                if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;
                const double wv = w[i + SSIM_R][j + SSIM_R];
                const double a = x[(size_t)qy * W + qx], b = y[(size_t)qy * W + qx];
                mx += wv * a;
                my += wv * b;
                ex2 += wv * a * a;
                ey2 += wv * b * b;
                exy += wv * a * b;
            }
        const double n1 = 2.0 * mx * my + C1, n2 = 2.0 * (exy - mx * my) + C2;
        const double d1 = mx * mx + my * my + C1, d2 = (ex2 - mx * mx) + (ey2 - my * my) + C2;
        const double S = n1 * n2 / (d1 * d2);
        ssim += S;
        Smu[e] = S * (2.0 * my / n1 - 2.0 * my / n2 - 2.0 * mx / d1 + 2.0 * mx / d2);
        SA[e] = -S / d2;
        SB[e] = 2.0 * S / n2;
        l1 += fabs((double)x[(size_t)py * W + px] - (double)y[(size_t)py * W + px]);
    }
    l1 /= (double)N;
    ssim /= (double)N;
    out[0] = (1.0 - lambda) * l1 + lambda * (1.0 - ssim);
    out[1] = l1;
    out[2] = ssim;
    if (grad) {
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < (long long)N; ++e) {
            const int c = (int)(e / HW);
            const int py = (int)((e % HW) / W), px = (int)(e % W);
            const size_t base = (size_t)c * HW;
            const double xp = image[base + (size_t)py * W + px], yp = target[base + (size_t)py * W + px];
            double gm = 0, ga = 0, gb = 0;
            for (int i = -SSIM_R; i <= SSIM_R; ++i)
                for (int j = -SSIM_R; j <= SSIM_R; ++j) {
                    const int qy = py + i, qx = px + j;
                    if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;
                    const double wv = w[i + SSIM_R][j + SSIM_R];
                    const size_t q = base + (size_t)qy * W + qx;
                    gm += wv * Smu[q];
                    ga += wv * SA[q];
                    gb += wv * SB[q];
                }
            const double dssim = (gm + 2.0 * xp * ga + yp * gb) / (double)N;
            const double sgn = xp > yp ? 1.0 : (xp < yp ? -1.0 : 0.0);
            grad[e] = (1.0 - lambda) * sgn / (double)N - lambda * dssim;
        }
    }
    free(Smu); free(SA); free(SB);
}

/* Opacity decay of training (Sec. 4 "Training": opacities multiplied by 0.999 at
 * intervals) and the pruning threshold (0.005): o' = factor sigmoid(logit), the
 * new logit ln(o' / (1 - o')), keep = o' >= threshold.  FP64. */
void orc_opacity_decay(int n, const float *logits, double factor, double threshold, double *new_logits,
                       double *new_opacity, uint8_t *keep)
{
#pragma omp parallel for schedule(static)
    for (int g = 0; g < n; ++g) {
        const double o = factor / (1.0 + exp(-(double)logits[g]));
        new_opacity[g] = o;
        new_logits[g] = log(o / (1.0 - o));
        keep[g] = o >= threshold;
    }
}
