// Sec. 3.3: occlusion culling of the foveal neural points against the Eq. 1
// depth buffer of the periphery (Sec. 3.2).  A streaming kernel: 12 bytes of
// point in, one byte of decision and a 4-byte index per kept point out; the
// depth and transmittance of the foveal window (a few MB) stay in L2.
//
// Each CTA takes chunks of 1024 points: the chunk's 12 KB are loaded with
// 16-byte vector loads into shared memory (three per thread, all issued before
// any is used), then each thread decides four points at a stride of 256 (so
// its shared reads, three consecutive words per point, are conflict-free),
// writes their mask bytes, and the kept indices are compacted with one
// atomic per CTA and chunk.
#include "vrs_internal.cuh"

namespace vrs {

struct CullArgs {
    const float *pts;
    int64_t n;
    float R[9], t[3];
    float fx, fy, cx, cy, znear;
    int32_t w, h, x0, y0, map_w, map_h;
    float alpha_min, scale, abs_margin;
    const float *depth, *Tf;
    uint8_t *mask;
    uint32_t *kept;
    unsigned long long *n_kept;
};

constexpr int kCullThreads = 256;
constexpr int kCullPer = 4;                        // points per thread and chunk
constexpr int kCullChunk = kCullThreads * kCullPer;

// The three-way decision of one point, every step a correctly rounded FP32
// operation in the order the C-ABI states.
__device__ __forceinline__ uint8_t cull_decide(const CullArgs &a, float px, float py, float pz)
{
    float x = __fmul_rn(a.R[0], px);
    x = __fadd_rn(x, __fmul_rn(a.R[1], py));
    x = __fadd_rn(x, __fmul_rn(a.R[2], pz));
    x = __fadd_rn(x, a.t[0]);
    float y = __fmul_rn(a.R[3], px);
    y = __fadd_rn(y, __fmul_rn(a.R[4], py));
    y = __fadd_rn(y, __fmul_rn(a.R[5], pz));
    y = __fadd_rn(y, a.t[1]);
    float z = __fmul_rn(a.R[6], px);
    z = __fadd_rn(z, __fmul_rn(a.R[7], py));
    z = __fadd_rn(z, __fmul_rn(a.R[8], pz));
    z = __fadd_rn(z, a.t[2]);
    if (!(z > a.znear) || !isfinite(x) || !isfinite(y)) return 0;
    const float iz = __fdiv_rn(1.0f, z);
    const float u = __fadd_rn(__fmul_rn(a.fx, __fmul_rn(x, iz)), a.cx);
    const float v = __fadd_rn(__fmul_rn(a.fy, __fmul_rn(y, iz)), a.cy);
    if (!(u >= 0.0f && u < (float)a.w && v >= 0.0f && v < (float)a.h)) return 0;
    const int mi = (int)u + a.x0, mj = (int)v + a.y0;
    if (mi < 0 || mi >= a.map_w || mj < 0 || mj >= a.map_h) return 0;
    const int64_t pix = (int64_t)mj * a.map_w + mi;
    const float al = __fsub_rn(1.0f, __ldg(a.Tf + pix));
    if (!(al >= a.alpha_min)) return 2;
    const float thr = __fadd_rn(__fmul_rn(__fdiv_rn(__ldg(a.depth + pix), al), a.scale), a.abs_margin);
    return z > thr ? 1 : 2;
}

__global__ void __launch_bounds__(kCullThreads) k_cull_points(const __grid_constant__ CullArgs a)
{
    __shared__ __align__(16) float sp[3 * kCullChunk];
    __shared__ uint32_t s_wcnt[kCullThreads / 32];
    __shared__ unsigned long long s_base[kCullThreads / 32];
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(a.pts) & 15u) == 0;
    for (int64_t c0 = (int64_t)blockIdx.x * kCullChunk; c0 < a.n; c0 += (int64_t)gridDim.x * kCullChunk) {
        const int64_t left = a.n - c0;
        const int cnt = left < kCullChunk ? (int)left : kCullChunk;
        // stage the chunk (12 bytes per point, contiguous)
        if (vec && cnt == kCullChunk) {
            const float4 *src = reinterpret_cast<const float4 *>(a.pts + 3 * c0);
            float4 *dst = reinterpret_cast<float4 *>(sp);
            float4 r[3 * kCullPer / 4];
#pragma unroll
            for (int k = 0; k < 3 * kCullPer / 4; ++k) r[k] = __ldg(src + k * kCullThreads + tid);
#pragma unroll
            for (int k = 0; k < 3 * kCullPer / 4; ++k) dst[k * kCullThreads + tid] = r[k];
        } else {
            for (int k = tid; k < 3 * cnt; k += kCullThreads) sp[k] = __ldg(a.pts + 3 * c0 + k);
        }
        __syncthreads();
        uint32_t bal[kCullPer];
        uint32_t total = 0;
#pragma unroll
        for (int k = 0; k < kCullPer; ++k) {
            const int li = k * kCullThreads + tid;
            uint8_t r = 0;
            if (li < cnt) {
                r = cull_decide(a, sp[3 * li], sp[3 * li + 1], sp[3 * li + 2]);
                a.mask[c0 + li] = r;
            }
            bal[k] = __ballot_sync(FULL, r == 2);
            total += __popc(bal[k]);
        }
        // one atomic per CTA and chunk for the kept slots
        if (lane == 0) s_wcnt[wp] = total;
        __syncthreads();
        if (tid == 0) {
            unsigned long long sum = 0;
            for (int q = 0; q < kCullThreads / 32; ++q) sum += s_wcnt[q];
            unsigned long long b = sum ? atomicAdd(a.n_kept, sum) : 0ull;
            for (int q = 0; q < kCullThreads / 32; ++q) {
                s_base[q] = b;
                b += s_wcnt[q];
            }
        }
        __syncthreads();
        if (a.kept) {
            unsigned long long base = s_base[wp];
            const uint32_t lt = lanemask_lt();
#pragma unroll
            for (int k = 0; k < kCullPer; ++k) {
                if ((bal[k] >> lane) & 1u)
                    a.kept[base + __popc(bal[k] & lt)] = (uint32_t)(c0 + k * kCullThreads + tid);
                base += __popc(bal[k]);
            }
        }
        __syncthreads();   // sp and s_base are rewritten by the next chunk
    }
}

}  // namespace vrs

using namespace vrs;

extern "C" vrs_status vrs_cull_points(const float *points, int64_t n_points, const vrs_camera *fovea,
                                      int32_t x0, int32_t y0, const float *depth, const float *T_final,
                                      int32_t map_w, int32_t map_h, const vrs_cull_opts *opts,
                                      uint8_t *mask, uint32_t *kept, uint64_t *n_kept, void *stream)
{
    if (n_points < 0 || n_points >= ((int64_t)1 << 32) || !fovea || !n_kept) return VRS_ERR_INVALID;
    if (n_points > 0 && (!points || !mask || !depth || !T_final)) return VRS_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(points) & 3u) != 0) return VRS_ERR_INVALID;
    if (fovea->width < 1 || fovea->height < 1 || map_w < 1 || map_h < 1) return VRS_ERR_INVALID;
    if (opts && opts->reserved != 0) return VRS_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(n_kept, 0, sizeof(uint64_t), s);
    if (e != cudaSuccess) return VRS_ERR_CUDA;
    if (n_points == 0) return VRS_OK;
    CullArgs a;
    a.pts = points;
    a.n = n_points;
    for (int i = 0; i < 9; ++i) a.R[i] = fovea->R[i];
    for (int i = 0; i < 3; ++i) a.t[i] = fovea->t[i];
    a.fx = fovea->fx;
    a.fy = fovea->fy;
    a.cx = fovea->cx;
    a.cy = fovea->cy;
    a.znear = fovea->znear;
    a.w = fovea->width;
    a.h = fovea->height;
    a.x0 = x0;
    a.y0 = y0;
    a.map_w = map_w;
    a.map_h = map_h;
    const float amin = opts ? opts->alpha_min : 0.5f;
    const float rel = opts ? opts->rel_margin : 0.02f;
    a.alpha_min = amin;
    a.scale = 1.0f + rel;                 // rounded once, as the definition states
    a.abs_margin = opts ? opts->abs_margin : 0.05f;
    a.depth = depth;
    a.Tf = T_final;
    a.mask = mask;
    a.kept = kept;
    a.n_kept = reinterpret_cast<unsigned long long *>(n_kept);
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 152;
    }
    const int64_t chunks = (n_points + kCullChunk - 1) / kCullChunk;
    const int64_t cap = (int64_t)sms * 8;
    const unsigned grid = (unsigned)(chunks < cap ? chunks : cap);
    k_cull_points<<<grid, kCullThreads, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? VRS_OK : VRS_ERR_CUDA;
}
