// Sec. 3.3: occlusion culling of the foveal neural points against the Eq. 1
// depth buffer of the periphery (Sec. 3.2).  A streaming kernel: 12 bytes of
// point in, one byte of decision and a 4-byte index per kept point out; the
// depth and transmittance of the foveal window (a few MB) stay in L2.
//
// Every warp streams chunks of 128 points: lane L loads the three 16-byte
// words 3L..3L+2 of the chunk, which hold its four whole points 4L..4L+3 (a
// resident wave of 56 warps per SM keeps about 90 KB of loads in flight).
// The decision runs without branches (x and y in packed FP32x2 operations,
// each component rounded as the scalar operation would be), the lane writes
// its four mask bytes as one word, and a warp with kept points takes their
// slots with one atomic.  Only the rare points inside an opaque-enough pixel
// take the divide of the depth test.
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
constexpr int kCullWarps = kCullThreads / 32;
constexpr int kCullPer = 4;                        // points per lane and chunk
constexpr int kCullChunk = 32 * kCullPer;          // points per warp chunk

__device__ __forceinline__ float2 f2c(float a) { return make_float2(a, a); }

// The three-way decision of one point, every step a correctly rounded FP32
// operation in the order the C-ABI states.
__device__ __forceinline__ uint32_t cull_decide(const CullArgs &a, float px, float py, float pz)
{
    float z = __fmul_rn(a.R[6], px);
    z = __fadd_rn(z, __fmul_rn(a.R[7], py));
    z = __fadd_rn(z, __fmul_rn(a.R[8], pz));
    z = __fadd_rn(z, a.t[2]);
    float2 xy = __fmul2_rn(make_float2(a.R[0], a.R[3]), f2c(px));
    xy = __fadd2_rn(xy, __fmul2_rn(make_float2(a.R[1], a.R[4]), f2c(py)));
    xy = __fadd2_rn(xy, __fmul2_rn(make_float2(a.R[2], a.R[5]), f2c(pz)));
    xy = __fadd2_rn(xy, make_float2(a.t[0], a.t[1]));
    const bool front = z > a.znear && isfinite(xy.x) && isfinite(xy.y);
    const float iz = __frcp_rn(z);                  // 1/z, correctly rounded
    float2 uv = __fmul2_rn(xy, f2c(iz));
    uv = __fmul2_rn(make_float2(a.fx, a.fy), uv);
    uv = __fadd2_rn(uv, make_float2(a.cx, a.cy));
    const bool in = front && uv.x >= 0.0f && uv.x < (float)a.w && uv.y >= 0.0f && uv.y < (float)a.h;
    const int mi = in ? __float2int_rz(uv.x) + a.x0 : -1, mj = in ? __float2int_rz(uv.y) + a.y0 : -1;
    const bool inmap = in && mi >= 0 && mi < a.map_w && mj >= 0 && mj < a.map_h;
    uint32_t r = inmap ? 2u : 0u;
    if (inmap) {
        const int64_t pix = (int64_t)mj * a.map_w + mi;
        const float al = __fsub_rn(1.0f, __ldg(a.Tf + pix));
        if (al >= a.alpha_min) {
            const float thr = __fadd_rn(__fmul_rn(__fdiv_rn(__ldg(a.depth + pix), al), a.scale), a.abs_margin);
            if (z > thr) r = 1u;
        }
    }
    return r;
}

__global__ void __launch_bounds__(kCullThreads) k_cull_points(const __grid_constant__ CullArgs a)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(a.pts) & 15u) == 0;
    const int64_t n_chunks = (a.n + kCullChunk - 1) / kCullChunk;
    const int64_t stride = (int64_t)gridDim.x * kCullWarps;
    for (int64_t c = (int64_t)blockIdx.x * kCullWarps + wp; c < n_chunks; c += stride) {
        // the lane's four points: 12 consecutive floats from float 12 * lane of the chunk
        const int64_t p0 = c * kCullChunk + kCullPer * lane;
        const bool whole = c * kCullChunk + kCullChunk <= a.n;
        float f[12];
        if (vec && whole) {
            const float4 *src = reinterpret_cast<const float4 *>(a.pts + 3 * p0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float4 v = __ldg(src + k);
                f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
            }
        } else {
            const int64_t lim = 3 * a.n;
#pragma unroll
            for (int e = 0; e < 12; ++e) f[e] = 3 * p0 + e < lim ? __ldg(a.pts + 3 * p0 + e) : 0.f;
        }
        uint32_t word = 0, keep = 0;
        if (whole) {                                         // a whole chunk: no per-point guard
#pragma unroll
            for (int k = 0; k < kCullPer; ++k) {
                const uint32_t r = cull_decide(a, f[3 * k], f[3 * k + 1], f[3 * k + 2]);
                word |= r << (8 * k);
                keep |= (r == 2u ? 1u : 0u) << k;
            }
        } else {
            for (int k = 0; k < kCullPer; ++k) {
                const uint32_t r = p0 + k < a.n ? cull_decide(a, f[3 * k], f[3 * k + 1], f[3 * k + 2]) : 0u;
                word |= r << (8 * k);
                keep |= (r == 2u ? 1u : 0u) << k;
            }
        }
        if (p0 + kCullPer <= a.n && (reinterpret_cast<uintptr_t>(a.mask + p0) & 3u) == 0) {
            *reinterpret_cast<uint32_t *>(a.mask + p0) = word;
        } else {
#pragma unroll
            for (int k = 0; k < kCullPer; ++k)
                if (p0 + k < a.n) a.mask[p0 + k] = (uint8_t)(word >> (8 * k));
        }
        // kept slots: one atomic per warp that has kept points
        const uint32_t nk = __popc(keep);
        if (__any_sync(FULL, nk != 0)) {
            uint32_t incl = nk;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t total = __shfl_sync(FULL, incl, 31);
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(a.n_kept, (unsigned long long)total);
            base = __shfl_sync(FULL, base, 0) + (incl - nk);
            if (a.kept) {
#pragma unroll
                for (int k = 0; k < kCullPer; ++k)
                    if ((keep >> k) & 1u) a.kept[base++] = (uint32_t)(p0 + k);
            }
        }
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
    const int64_t ctas = (n_points + (int64_t)kCullChunk * kCullWarps - 1) / ((int64_t)kCullChunk * kCullWarps);
    int per_sm = 0;                            // one resident wave; warps loop over the chunks
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cull_points, kCullThreads, 0) != cudaSuccess ||
        per_sm <= 0) {
        cudaGetLastError();
        per_sm = 4;
    }
    const int64_t cap = (int64_t)sms * per_sm;
    k_cull_points<<<(unsigned)(ctas < cap ? ctas : cap), kCullThreads, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? VRS_OK : VRS_ERR_CUDA;
}
