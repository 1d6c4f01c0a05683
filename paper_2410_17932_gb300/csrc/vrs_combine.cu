// Sec. 3.4: the foveated combination of the peripheral image P and the foveal
// image F over the crop window: a positional factor from the distance to the
// fixation, an edge factor from the Sobel gradient of F, smootherstep, and a
// per-pixel convex mix.  A small stencil kernel: each 32x8 block stages the
// channel mean of F over its pixels and a one-pixel halo in shared memory,
// then every thread takes its pixel's 3x3 neighbourhood from there.
#include "vrs_internal.cuh"

namespace vrs {

constexpr int kCbX = 32, kCbY = 8;

struct CombineArgs {
    const float *P, *F;
    float *out, *c_out;
    int pw, ph, w, h, x0, y0;
    float ex, ey, inv_df, m, inv_1m, gamma;
};

__global__ void __launch_bounds__(kCbX * kCbY) k_foveal_combine(const __grid_constant__ CombineArgs a)
{
    __shared__ float sL[kCbY + 2][kCbX + 2];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int bx = blockIdx.x * kCbX, by = blockIdx.y * kCbY;
    const size_t hw = (size_t)a.w * a.h;
    // channel mean of F over the block and its halo, the crop's border replicated
    for (int k = ty * kCbX + tx; k < (kCbX + 2) * (kCbY + 2); k += kCbX * kCbY) {
        const int li = k % (kCbX + 2), lj = k / (kCbX + 2);
        const int i = min(max(bx + li - 1, 0), a.w - 1), j = min(max(by + lj - 1, 0), a.h - 1);
        const size_t q = (size_t)j * a.w + i;
        sL[lj][li] = (__ldg(a.F + q) + __ldg(a.F + hw + q) + __ldg(a.F + 2 * hw + q)) * (1.0f / 3.0f);
    }
    __syncthreads();
    const int i = bx + tx, j = by + ty;
    if (i >= a.w || j >= a.h) return;
    const float du = (float)(a.x0 + i) + 0.5f - a.ex, dv = (float)(a.y0 + j) + 0.5f - a.ey;
    const float r = fminf(fmaxf(sqrtf(du * du + dv * dv) * a.inv_df, 0.f), 1.f);
    const float fp = (r - a.m) * a.inv_1m;
    const int li = tx + 1, lj = ty + 1;
    const float gx = ((sL[lj - 1][li + 1] + 2.f * sL[lj][li + 1] + sL[lj + 1][li + 1]) -
                      (sL[lj - 1][li - 1] + 2.f * sL[lj][li - 1] + sL[lj + 1][li - 1])) * 0.125f;
    const float gy = ((sL[lj + 1][li - 1] + 2.f * sL[lj + 1][li] + sL[lj + 1][li + 1]) -
                      (sL[lj - 1][li - 1] + 2.f * sL[lj - 1][li] + sL[lj - 1][li + 1])) * 0.125f;
    const float fe = sqrtf(gx * gx + gy * gy);
    const float x = fminf(fmaxf(fp + a.gamma * fe, 0.f), 1.f);
    const float c = 1.f - x * x * x * (x * (6.f * x - 15.f) + 10.f);
    const size_t q = (size_t)j * a.w + i;
    const size_t pp = (size_t)(a.y0 + j) * a.pw + (a.x0 + i), phw = (size_t)a.pw * a.ph;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float p = __ldg(a.P + ch * phw + pp), f = __ldg(a.F + ch * hw + q);
        a.out[ch * hw + q] = fmaf(c, f - p, p);
    }
    if (a.c_out) a.c_out[q] = c;
}

// Reverse pass: per pixel the direct terms and, on the blending band, the edge
// factor's gradient spread over the 3x3 Sobel taps of the channel mean
// (atomics into the scratch map); a second kernel adds the mean's share to
// every channel of dL/dF.
struct CombineBwdArgs {
    CombineArgs f;
    const float *g;
    float *dP, *dF, *dLum;
};

__global__ void __launch_bounds__(kCbX * kCbY) k_foveal_combine_bwd(const __grid_constant__ CombineBwdArgs b)
{
    const CombineArgs &a = b.f;
    __shared__ float sL[kCbY + 2][kCbX + 2];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int bx = blockIdx.x * kCbX, by = blockIdx.y * kCbY;
    const size_t hw = (size_t)a.w * a.h;
    for (int k = ty * kCbX + tx; k < (kCbX + 2) * (kCbY + 2); k += kCbX * kCbY) {
        const int li = k % (kCbX + 2), lj = k / (kCbX + 2);
        const int i = min(max(bx + li - 1, 0), a.w - 1), j = min(max(by + lj - 1, 0), a.h - 1);
        const size_t q = (size_t)j * a.w + i;
        sL[lj][li] = (__ldg(a.F + q) + __ldg(a.F + hw + q) + __ldg(a.F + 2 * hw + q)) * (1.0f / 3.0f);
    }
    __syncthreads();
    const int i = bx + tx, j = by + ty;
    if (i >= a.w || j >= a.h) return;
    const float du = (float)(a.x0 + i) + 0.5f - a.ex, dv = (float)(a.y0 + j) + 0.5f - a.ey;
    const float r = fminf(fmaxf(sqrtf(du * du + dv * dv) * a.inv_df, 0.f), 1.f);
    const float fp = (r - a.m) * a.inv_1m;
    const int li = tx + 1, lj = ty + 1;
    const float gx = ((sL[lj - 1][li + 1] + 2.f * sL[lj][li + 1] + sL[lj + 1][li + 1]) -
                      (sL[lj - 1][li - 1] + 2.f * sL[lj][li - 1] + sL[lj + 1][li - 1])) * 0.125f;
    const float gy = ((sL[lj + 1][li - 1] + 2.f * sL[lj + 1][li] + sL[lj + 1][li + 1]) -
                      (sL[lj - 1][li - 1] + 2.f * sL[lj - 1][li] + sL[lj - 1][li + 1])) * 0.125f;
    const float fe = sqrtf(gx * gx + gy * gy);
    const float x = fp + a.gamma * fe;
    const float xc = fminf(fmaxf(x, 0.f), 1.f);
    const float c = 1.f - xc * xc * xc * (xc * (6.f * xc - 15.f) + 10.f);
    const size_t q = (size_t)j * a.w + i;
    const size_t pp = (size_t)(a.y0 + j) * a.pw + (a.x0 + i), phw = (size_t)a.pw * a.ph;
    float dLdc = 0.f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float gc = __ldg(b.g + ch * hw + q);
        b.dP[ch * phw + pp] += (1.f - c) * gc;
        b.dF[ch * hw + q] += c * gc;
        dLdc = fmaf(gc, __ldg(a.F + ch * hw + q) - __ldg(a.P + ch * phw + pp), dLdc);
    }
    if (!(x > 0.f && x < 1.f) || fe == 0.f) return;
    const float dfe = dLdc * (-30.f * x * x * (1.f - x) * (1.f - x)) * a.gamma;
    const float dgx = dfe * gx / fe * 0.125f, dgy = dfe * gy / fe * 0.125f;
    const float kx[3][3] = {{-1.f, 0.f, 1.f}, {-2.f, 0.f, 2.f}, {-1.f, 0.f, 1.f}};
    const float ky[3][3] = {{-1.f, -2.f, -1.f}, {0.f, 0.f, 0.f}, {1.f, 2.f, 1.f}};
#pragma unroll
    for (int bb = -1; bb <= 1; ++bb)
#pragma unroll
        for (int aa = -1; aa <= 1; ++aa) {
            const float v = dgx * kx[bb + 1][aa + 1] + dgy * ky[bb + 1][aa + 1];
            if (v == 0.f) continue;
            const int ii = min(max(i + aa, 0), a.w - 1), jj = min(max(j + bb, 0), a.h - 1);
            atomicAdd(b.dLum + (size_t)jj * a.w + ii, v);
        }
}

__global__ void k_foveal_combine_bwd_lum(float *dF, const float *dLum, size_t hw)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < hw; q += (size_t)gridDim.x * blockDim.x) {
        const float v = dLum[q] * (1.0f / 3.0f);
        dF[q] += v;
        dF[hw + q] += v;
        dF[2 * hw + q] += v;
    }
}

}  // namespace vrs

using namespace vrs;

extern "C" vrs_status vrs_foveal_combine(const float *P, int32_t pw, int32_t ph, const float *F, int32_t w,
                                         int32_t h, int32_t x0, int32_t y0, float ex, float ey,
                                         const vrs_combine_opts *opts, float *out, float *c_out, void *stream)
{
    if (!P || !F || !out || pw < 1 || ph < 1 || w < 1 || h < 1) return VRS_ERR_INVALID;
    if (x0 < 0 || y0 < 0 || (int64_t)x0 + w > pw || (int64_t)y0 + h > ph) return VRS_ERR_INVALID;
    const char *o0 = reinterpret_cast<const char *>(out), *f0 = reinterpret_cast<const char *>(F);
    const size_t bytes = sizeof(float) * 3 * (size_t)w * h;
    if (o0 < f0 + bytes && f0 < o0 + bytes) return VRS_ERR_INVALID;
    const float d_f = opts ? opts->d_f : 256.f, m = opts ? opts->m : 0.75f, gamma = opts ? opts->gamma : 0.2f;
    if (opts && opts->reserved != 0) return VRS_ERR_INVALID;
    if (!(d_f > 0.f) || !(m < 1.f)) return VRS_ERR_INVALID;
    CombineArgs a;
    a.P = P;
    a.F = F;
    a.out = out;
    a.c_out = c_out;
    a.pw = pw;
    a.ph = ph;
    a.w = w;
    a.h = h;
    a.x0 = x0;
    a.y0 = y0;
    a.ex = ex;
    a.ey = ey;
    a.inv_df = 1.f / d_f;
    a.m = m;
    a.inv_1m = 1.f / (1.f - m);
    a.gamma = gamma;
    const dim3 grid((unsigned)((w + kCbX - 1) / kCbX), (unsigned)((h + kCbY - 1) / kCbY));
    k_foveal_combine<<<grid, dim3(kCbX, kCbY), 0, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? VRS_OK : VRS_ERR_CUDA;
}

extern "C" vrs_status vrs_foveal_combine_bwd(const float *P, int32_t pw, int32_t ph, const float *F, int32_t w,
                                             int32_t h, int32_t x0, int32_t y0, float ex, float ey,
                                             const vrs_combine_opts *opts, const float *dL_dout, float *dL_dP,
                                             float *dL_dF, float *scratch, void *stream)
{
    if (!P || !F || !dL_dout || !dL_dP || !dL_dF || !scratch || pw < 1 || ph < 1 || w < 1 || h < 1)
        return VRS_ERR_INVALID;
    if (x0 < 0 || y0 < 0 || (int64_t)x0 + w > pw || (int64_t)y0 + h > ph) return VRS_ERR_INVALID;
    const float d_f = opts ? opts->d_f : 256.f, m = opts ? opts->m : 0.75f, gamma = opts ? opts->gamma : 0.2f;
    if (opts && opts->reserved != 0) return VRS_ERR_INVALID;
    if (!(d_f > 0.f) || !(m < 1.f)) return VRS_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t hw = (size_t)w * h;
    if (cudaMemsetAsync(scratch, 0, sizeof(float) * hw, s) != cudaSuccess) return VRS_ERR_CUDA;
    CombineBwdArgs b;
    CombineArgs &a = b.f;
    a.P = P;
    a.F = F;
    a.out = nullptr;
    a.c_out = nullptr;
    a.pw = pw;
    a.ph = ph;
    a.w = w;
    a.h = h;
    a.x0 = x0;
    a.y0 = y0;
    a.ex = ex;
    a.ey = ey;
    a.inv_df = 1.f / d_f;
    a.m = m;
    a.inv_1m = 1.f / (1.f - m);
    a.gamma = gamma;
    b.g = dL_dout;
    b.dP = dL_dP;
    b.dF = dL_dF;
    b.dLum = scratch;
    const dim3 grid((unsigned)((w + kCbX - 1) / kCbX), (unsigned)((h + kCbY - 1) / kCbY));
    k_foveal_combine_bwd<<<grid, dim3(kCbX, kCbY), 0, s>>>(b);
    const unsigned g2 = (unsigned)((hw + 255) / 256 < 4096 ? (hw + 255) / 256 : 4096);
    k_foveal_combine_bwd_lum<<<g2, 256, 0, s>>>(dL_dF, scratch, hw);
    return cudaGetLastError() == cudaSuccess ? VRS_OK : VRS_ERR_CUDA;
}
