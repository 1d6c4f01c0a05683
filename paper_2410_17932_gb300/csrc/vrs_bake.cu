// vrs_bake: the activations of the Gaussian parameters, evaluated once for
// inference (Sec. 4 "Inference": opacities, features and covariances are baked
// into the point cloud to minimise runtime cost).  Each value is computed by the
// decision path's own device functions, so that a baked scene renders the same
// images bit for bit.
#include <string.h>

#include "vrs_internal.cuh"

namespace vrs {

__global__ void k_bake(const DevScene S, float4 *out)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= S.n) return;
    float ls[3], q[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) ls[i] = __ldg(S.log_scales + 3 * g + i);
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = __ldg(S.quats + 4 * g + i);
    const float logit = __ldg(S.logits + g);
    // x * 0 is NaN exactly for a non-finite x
    float chk = __fmaf_rn(logit, 0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 3; ++i) chk = __fmaf_rn(ls[i], 0.f, chk);
#pragma unroll
    for (int i = 0; i < 4; ++i) chk = __fmaf_rn(q[i], 0.f, chk);
    GaussPre pre;
    uint32_t st = 0u;
    if (!isfinite(chk)) st = 2u;
    else if (!gauss_pre(ls, q, pre)) st = 1u;
    if (st) {
#pragma unroll
        for (int i = 0; i < 3; ++i) pre.s[i] = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) pre.Rq[i] = 0.f;
    }
    const float op = st ? 0.f : decision_opacity(logit);
    const float lo = st ? 0.f : record_log2_opacity(logit);
    float4 *o = out + 4 * (size_t)g;
    o[0] = make_float4(pre.s[0], pre.s[1], pre.s[2], pre.Rq[0]);
    o[1] = make_float4(pre.Rq[1], pre.Rq[2], pre.Rq[3], pre.Rq[4]);
    o[2] = make_float4(pre.Rq[5], pre.Rq[6], pre.Rq[7], pre.Rq[8]);
    o[3] = make_float4(op, lo, __uint_as_float(st), 0.f);
}

}  // namespace vrs

using namespace vrs;

extern "C" vrs_status vrs_bake(const vrs_scene *scene, float *baked, void *stream)
{
    if (!scene || scene->n < 0) return VRS_ERR_INVALID;
    if (scene->n == 0) return VRS_OK;
    if (!baked || !scene->log_scales || !scene->quats || !scene->opacity_logits) return VRS_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(baked) & 15u) return VRS_ERR_INVALID;
    DevScene S;
    memset(&S, 0, sizeof(S));
    S.log_scales = scene->log_scales;
    S.quats = scene->quats;
    S.logits = scene->opacity_logits;
    S.n = scene->n;
    k_bake<<<grid_for(S.n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(S, reinterpret_cast<float4 *>(baked));
    return cudaGetLastError() == cudaSuccess ? VRS_OK : VRS_ERR_CUDA;
}
