// Training-loop pieces of the Gaussian branch.
//
// vrs_image_loss: L = (1 - lambda) L1 + lambda (1 - SSIM) of a rendered image
// against its target and dL/dimage, the upstream gradient of vrs_render_bwd
// (Sec. 3.5: the first two terms of the loss are those of 3DGS, lambda = 0.2).
// SSIM (Wang et al. 2004) with an 11 x 11 Gaussian window (sigma 1.5, zero
// outside the image), C1 = 0.01^2, C2 = 0.03^2, averaged over channels and
// pixels.  The window is the outer product of a 1-D Gaussian, so every window
// sum is two 11-tap passes over a shared-memory tile with a 5-pixel halo.
//   k_ssim_fwd: per pixel and channel the five window moments (means of x, y,
//     x^2, y^2, x y), S, and the three partials of S with respect to mu_x,
//     w * x^2 and w * (x y); per-CTA sums of S and |x - y|.
//   k_ssim_bwd: the window sums of the three partials (the adjoint of a
//     zero-padded symmetric window is the same window) give
//     dSSIM/dx_p = (w * S_mu + 2 x_p w * S_A + y_p w * S_B) / N.
//   the last CTA of k_ssim_fwd to finish sums the per-CTA sums in FP64, in a
//     fixed order.
//
// vrs_opacity_decay: Sec. 4 "Training" multiplies the opacities by 0.999 at
// intervals and prunes below 0.005: the new logit of factor * sigmoid(logit),
// a keep mask and the number kept.
#include "vrs_internal.cuh"

namespace vrs {

constexpr int kLW = 32, kLH = 40, kLR = 5;                // output tile, window radius
constexpr int kLThreads = 256;
constexpr int kLPW = kLW + 2 * kLR, kLPH = kLH + 2 * kLR;  // padded tile (42 x 50)
constexpr int kHSeg = 8;                                  // row-pass outputs per thread
constexpr int kVSeg = kLH / (kLThreads / kLW);            // column-pass outputs per thread (5)
static_assert((kLThreads / kLW) * kVSeg == kLH, "the column pass covers the tile");
static_assert(kLPH * (kLW / kHSeg) <= kLThreads, "the row pass is one round");
constexpr int kLoadIters = (kLPW * kLPH + kLThreads - 1) / kLThreads;   // padded-tile loads per thread

__constant__ float c_gauss[2 * kLR + 1];

struct LossArgs {
    const float *x, *y;
    float *smu, *sa, *sb;      // [C][H][W] partials of S
    float *dx;                 // nullable: dL/dimage
    float2 *block_sums;        // per CTA: (sum S, sum |x - y|)
    uint32_t *ticket;          // CTAs of k_ssim_fwd done (zeroed before the launch)
    float *loss_out;           // (L, L1, SSIM)
    int C, H, W;
    float lambda, inv_n;
    double inv_n_d;
};

// The 11-tap row pass of one padded array, in place: the thread owning row r,
// columns [c0, c0 + kHSeg) of the result reads its 18 inputs into registers
// (a sliding window: each input loaded once), and after a barrier writes the
// sums over the first kLW columns of the row.  Every thread of the CTA calls it.
__device__ __forceinline__ void row_pass(float (*t)[kLPW], bool act, int r, int c0)
{
    float out[kHSeg];
    if (act) {
        float w[kHSeg + 2 * kLR];
#pragma unroll
        for (int i = 0; i < kHSeg + 2 * kLR; ++i) w[i] = t[r][c0 + i];
#pragma unroll
        for (int j = 0; j < kHSeg; ++j) {
            float m = 0.f;
#pragma unroll
            for (int k = 0; k < 2 * kLR + 1; ++k) m = fmaf(c_gauss[k], w[j + k], m);
            out[j] = m;
        }
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int j = 0; j < kHSeg; ++j) t[r][c0 + j] = out[j];
    }
}

// The 11-tap column pass of one row-summed array: kVSeg outputs of column tx
// starting at output row ty * kVSeg, from 15 loads.
__device__ __forceinline__ void col_pass(const float (*t)[kLPW], int tx, int ty, float (&out)[kVSeg])
{
    float w[kVSeg + 2 * kLR];
#pragma unroll
    for (int i = 0; i < kVSeg + 2 * kLR; ++i) w[i] = t[ty * kVSeg + i][tx];
#pragma unroll
    for (int j = 0; j < kVSeg; ++j) {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 2 * kLR + 1; ++k) m = fmaf(c_gauss[k], w[j + k], m);
        out[j] = m;
    }
}

// The last CTA of k_ssim_fwd: the per-CTA sums in FP64, each thread over a fixed
// stride of them, then a fixed tree, so the result does not depend on which CTA
// ran last; the loss, L1 and SSIM.
__device__ void loss_sums(const LossArgs &a, uint32_t n_blocks)
{
    __shared__ double rs[kLThreads / 32], rl[kLThreads / 32];
    __threadfence();
    double s = 0.0, l = 0.0;
    for (uint32_t i = threadIdx.x; i < n_blocks; i += kLThreads) {
        const float2 v = __ldcg(a.block_sums + i);       // L2: written by other CTAs
        s += (double)v.x;
        l += (double)v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        l += __shfl_xor_sync(0xffffffffu, l, o);
    }
    if ((threadIdx.x & 31) == 0) {
        rs[threadIdx.x >> 5] = s;
        rl[threadIdx.x >> 5] = l;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kLThreads / 32; ++w) {
            s += rs[w];
            l += rl[w];
        }
        const double inv_n = a.inv_n_d;
        const double ssim = s * inv_n, l1 = l * inv_n;
        a.loss_out[0] = (float)((1.0 - a.lambda) * l1 + a.lambda * (1.0 - ssim));
        a.loss_out[1] = (float)l1;
        a.loss_out[2] = (float)ssim;
    }
}

// One CTA per 32 x 40 output tile and channel: the padded tile of x and y and
// their products in shared memory (zero outside the image), the row passes in
// place, then each thread's column of five outputs.
__global__ void __launch_bounds__(kLThreads) k_ssim_fwd(const LossArgs a)
{
    __shared__ float sm[5][kLPH][kLPW];       // x, y, x^2, y^2, x y; then their row sums
    __shared__ float2 red[kLThreads / 32];
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    const int x0 = blockIdx.x * kLW, y0 = blockIdx.y * kLH;
    const size_t base = (size_t)blockIdx.z * a.H * a.W;
    float l1_sum = 0.f;
    {
        // every load of the thread first, then the stores (the loads stay in flight together)
        float u[kLoadIters], v[kLoadIters];
#pragma unroll
        for (int it = 0; it < kLoadIters; ++it) {
            const int i = threadIdx.x + it * kLThreads;
            const int r = i / kLPW, col = i - r * kLPW;
            const int gy = y0 + r - kLR, gx = x0 + col - kLR;
            u[it] = v[it] = 0.f;
            if (i < kLPW * kLPH && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W) {
                const size_t e = base + (size_t)gy * a.W + gx;
                u[it] = __ldg(a.x + e);
                v[it] = __ldg(a.y + e);
            }
        }
#pragma unroll
        for (int it = 0; it < kLoadIters; ++it) {
            const int i = threadIdx.x + it * kLThreads;
            if (i < kLPW * kLPH) {
                const int r = i / kLPW, col = i - r * kLPW;
                // |x - y| once per pixel: over the tile's own cells (zero outside the image)
                if (r >= kLR && r < kLR + kLH && col >= kLR && col < kLR + kLW) l1_sum += fabsf(u[it] - v[it]);
                sm[0][r][col] = u[it];
                sm[1][r][col] = v[it];
                sm[2][r][col] = u[it] * u[it];
                sm[3][r][col] = v[it] * v[it];
                sm[4][r][col] = u[it] * v[it];
            }
        }
    }
    __syncthreads();
    const int hr = threadIdx.x / (kLW / kHSeg), hc = (threadIdx.x % (kLW / kHSeg)) * kHSeg;
#pragma unroll 1
    for (int m = 0; m < 5; ++m) row_pass(sm[m], hr < kLPH, hr, hc);
    __syncthreads();
    const int tx = threadIdx.x % kLW, ty = threadIdx.x / kLW;
    float mx[kVSeg], my[kVSeg], ex2[kVSeg], ey2[kVSeg], exy[kVSeg];
    col_pass(sm[0], tx, ty, mx);
    col_pass(sm[1], tx, ty, my);
    col_pass(sm[2], tx, ty, ex2);
    col_pass(sm[3], tx, ty, ey2);
    col_pass(sm[4], tx, ty, exy);
    float s_sum = 0.f;
    const int px = x0 + tx;
#pragma unroll
    for (int j = 0; j < kVSeg; ++j) {
        const int py = y0 + ty * kVSeg + j;
        if (px < a.W && py < a.H) {
            const float n1 = 2.f * mx[j] * my[j] + C1, n2 = 2.f * (exy[j] - mx[j] * my[j]) + C2;
            const float d1 = mx[j] * mx[j] + my[j] * my[j] + C1;
            const float d2 = (ex2[j] - mx[j] * mx[j]) + (ey2[j] - my[j] * my[j]) + C2;
            const float rn1 = __fdividef(1.f, n1), rn2 = __fdividef(1.f, n2);
            const float rd1 = __fdividef(1.f, d1), rd2 = __fdividef(1.f, d2);
            const float S = n1 * n2 * rd1 * rd2;
            const size_t e = base + (size_t)py * a.W + px;
            a.smu[e] = S * (2.f * my[j] * rn1 - 2.f * my[j] * rn2 - 2.f * mx[j] * rd1 + 2.f * mx[j] * rd2);
            a.sa[e] = -S * rd2;
            a.sb[e] = 2.f * S * rn2;
            s_sum += S;
        }
    }
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s_sum += __shfl_xor_sync(FULL, s_sum, o);
        l1_sum += __shfl_xor_sync(FULL, l1_sum, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_float2(s_sum, l1_sum);
    __syncthreads();
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        float2 t = red[0];
        for (int w = 1; w < kLThreads / 32; ++w) {
            t.x += red[w].x;
            t.y += red[w].y;
        }
        a.block_sums[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
        __threadfence();                      // the sum is visible before the ticket counts it
        const uint32_t n_ctas = gridDim.x * gridDim.y * gridDim.z;
        s_last = atomicAdd(a.ticket, 1u) == n_ctas - 1;
    }
    __syncthreads();
    if (s_last) loss_sums(a, gridDim.x * gridDim.y * gridDim.z);
}

// The same tiling over the three partial maps, then dL/dx per pixel.
__global__ void __launch_bounds__(kLThreads) k_ssim_bwd(const LossArgs a)
{
    __shared__ float sm[3][kLPH][kLPW];
    const int x0 = blockIdx.x * kLW, y0 = blockIdx.y * kLH;
    const size_t base = (size_t)blockIdx.z * a.H * a.W;
    {
        float m0[kLoadIters], m1[kLoadIters], m2[kLoadIters];
#pragma unroll
        for (int it = 0; it < kLoadIters; ++it) {
            const int i = threadIdx.x + it * kLThreads;
            const int r = i / kLPW, col = i - r * kLPW;
            const int gy = y0 + r - kLR, gx = x0 + col - kLR;
            m0[it] = m1[it] = m2[it] = 0.f;
            if (i < kLPW * kLPH && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W) {
                const size_t e = base + (size_t)gy * a.W + gx;
                m0[it] = __ldg(a.smu + e);
                m1[it] = __ldg(a.sa + e);
                m2[it] = __ldg(a.sb + e);
            }
        }
#pragma unroll
        for (int it = 0; it < kLoadIters; ++it) {
            const int i = threadIdx.x + it * kLThreads;
            if (i < kLPW * kLPH) {
                const int r = i / kLPW, col = i - r * kLPW;
                sm[0][r][col] = m0[it];
                sm[1][r][col] = m1[it];
                sm[2][r][col] = m2[it];
            }
        }
    }
    __syncthreads();
    const int hr = threadIdx.x / (kLW / kHSeg), hc = (threadIdx.x % (kLW / kHSeg)) * kHSeg;
#pragma unroll 1
    for (int m = 0; m < 3; ++m) row_pass(sm[m], hr < kLPH, hr, hc);
    __syncthreads();
    const int tx = threadIdx.x % kLW, ty = threadIdx.x / kLW;
    float gm[kVSeg], ga[kVSeg], gb[kVSeg];
    col_pass(sm[0], tx, ty, gm);
    col_pass(sm[1], tx, ty, ga);
    col_pass(sm[2], tx, ty, gb);
    const int px = x0 + tx;
#pragma unroll
    for (int j = 0; j < kVSeg; ++j) {
        const int py = y0 + ty * kVSeg + j;
        if (px < a.W && py < a.H) {
            const size_t e = base + (size_t)py * a.W + px;
            const float xp = __ldg(a.x + e), yp = __ldg(a.y + e);
            const float sgn = xp > yp ? 1.f : (xp < yp ? -1.f : 0.f);
            const float dssim = (gm[j] + 2.f * xp * ga[j] + yp * gb[j]) * a.inv_n;
            a.dx[e] = (1.f - a.lambda) * sgn * a.inv_n - a.lambda * dssim;
        }
    }
}

__global__ void k_opacity_decay(float *logits, int64_t n, float factor, float threshold, uint8_t *keep,
                                uint32_t *n_kept)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool k = false;
    if (i < n) {
        const float o = factor / (1.0f + expf(-logits[i]));
        logits[i] = logf(o) - log1pf(-o);
        k = o >= threshold;
        keep[i] = k ? 1 : 0;
    }
    const uint32_t b = __ballot_sync(0xffffffffu, k);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_kept, (uint32_t)__popc(b));
}

namespace {
bool g_gauss_ready[64];
}

// Scratch layout: the three partial maps (n floats each), then the per-CTA float2 sums at
// the next 16-byte boundary (3 n floats end on a 4-byte one when n is odd).
inline int64_t sums_offset(int64_t n) { return (3 * n * 4 + 15) / 16 * 16; }

}  // namespace vrs

using namespace vrs;

extern "C" {

vrs_status vrs_image_loss_scratch(int32_t C, int32_t H, int32_t W, int64_t *bytes)
{
    if (C < 1 || H < 1 || W < 1 || !bytes) return VRS_ERR_INVALID;
    const int64_t n = (int64_t)C * H * W;
    const int64_t blocks = (int64_t)((W + kLW - 1) / kLW) * ((H + kLH - 1) / kLH) * C;
    *bytes = sums_offset(n) + blocks * 8 + 16;    // the partial maps, the per-CTA sums, the ticket
    return VRS_OK;
}

vrs_status vrs_image_loss(const float *image, const float *target, int32_t C, int32_t H, int32_t W, float lambda,
                          float *loss_out, float *dL_dimage, void *scratch, int64_t scratch_bytes, void *stream)
{
    int64_t need = 0;
    if (vrs_image_loss_scratch(C, H, W, &need) != VRS_OK) return VRS_ERR_INVALID;
    if (!image || !target || !loss_out || !scratch || scratch_bytes < need) return VRS_ERR_INVALID;
    if (!(lambda >= 0.f && lambda <= 1.f)) return VRS_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(scratch) & 15u) != 0) return VRS_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return VRS_ERR_CUDA;
    if (!g_gauss_ready[dev]) {           // the normalised 1-D Gaussian of the SSIM window
        float g[2 * kLR + 1];
        double s = 0.0, v[2 * kLR + 1];
        for (int i = 0; i < 2 * kLR + 1; ++i) {
            v[i] = exp(-(double)((i - kLR) * (i - kLR)) / (2.0 * 1.5 * 1.5));
            s += v[i];
        }
        for (int i = 0; i < 2 * kLR + 1; ++i) g[i] = (float)(v[i] / s);
        if (cudaMemcpyToSymbol(c_gauss, g, sizeof(g)) != cudaSuccess) return VRS_ERR_CUDA;
        g_gauss_ready[dev] = true;
    }
    const int64_t n = (int64_t)C * H * W;
    LossArgs a;
    a.x = image;
    a.y = target;
    a.smu = static_cast<float *>(scratch);
    a.sa = a.smu + n;
    a.sb = a.sa + n;
    a.block_sums = reinterpret_cast<float2 *>(static_cast<char *>(scratch) + sums_offset(n));
    const int64_t n_ctas = (int64_t)((W + kLW - 1) / kLW) * ((H + kLH - 1) / kLH) * C;
    a.ticket = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + sums_offset(n) + n_ctas * 8);
    a.loss_out = loss_out;
    a.inv_n_d = 1.0 / (double)n;
    a.dx = dL_dimage;
    a.C = C;
    a.H = H;
    a.W = W;
    a.lambda = lambda;
    a.inv_n = (float)(1.0 / (double)n);
    const dim3 grid((W + kLW - 1) / kLW, (H + kLH - 1) / kLH, C);
    if (grid.y > 65535u || grid.z > 65535u) return VRS_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(a.ticket, 0, sizeof(uint32_t), s) != cudaSuccess) return VRS_ERR_CUDA;
    k_ssim_fwd<<<grid, kLThreads, 0, s>>>(a);
    if (dL_dimage) k_ssim_bwd<<<grid, kLThreads, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? VRS_OK : VRS_ERR_CUDA;
}

vrs_status vrs_opacity_decay(float *opacity_logits, int64_t n, float factor, float threshold, uint8_t *keep,
                             uint32_t *n_kept, void *stream)
{
    if (n < 0 || !(factor > 0.f && factor <= 1.f) || !(threshold >= 0.f && threshold < 1.f)) return VRS_ERR_INVALID;
    if (n > 0 && (!opacity_logits || !keep || !n_kept)) return VRS_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n_kept && cudaMemsetAsync(n_kept, 0, sizeof(uint32_t), s) != cudaSuccess) return VRS_ERR_CUDA;
    if (n == 0) return VRS_OK;
    k_opacity_decay<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(opacity_logits, n, factor, threshold, keep, n_kept);
    return cudaGetLastError() == cudaSuccess ? VRS_OK : VRS_ERR_CUDA;
}

}  // extern "C"
