// Adjoint of the rasterizer (placeholder until the reverse kernels land).
#include "vrs_internal.cuh"

namespace vrs {

cudaError_t launch_render_bwd(const ViewTable &, const float4 *, const float4 *, const uint32_t *,
                              const uint2 *, const DevStatus *, const uint32_t *, const float *,
                              const float *, const float *, const float *, float *, int64_t,
                              cudaStream_t)
{
    return cudaErrorNotSupported;
}

cudaError_t launch_backward_params(const ViewTable &, const DevScene &, const DevScene &,
                                   const int8_t *, int, const float *, const DevStatus *, cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace vrs
