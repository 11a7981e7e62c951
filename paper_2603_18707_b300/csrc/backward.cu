// backward.cu — reverse pass (placeholder until the reverse kernels land).
#include "gs_common.cuh"

using namespace gs;

extern "C" size_t gs_grad2d_bytes(int32_t ncam, int32_t P)
{
    if (ncam <= 0 || P < 0) return 0;
    return align256(sizeof(float) * 12 * (size_t)ncam * P);
}

extern "C" gs_status gs_render_backward(void *, const gs_camera *, int32_t, int32_t, const gs_config *,
                                        const float *, const float *, const float *, const float *,
                                        const float *, int32_t, const void *, const uint32_t *,
                                        const uint32_t *, const float *, const float *,
                                        const uint32_t *, const float *, void *, float *, float *,
                                        float *, float *, float *)
{
    return GS_ERR_UNSUPPORTED;
}
