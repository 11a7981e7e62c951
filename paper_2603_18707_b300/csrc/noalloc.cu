// noalloc.cu — gs_bin_sort for callers that cannot allocate device memory.
//
// Some hosts of this renderer cannot call cudaMalloc at all: a plugin whose
// host application owns every device allocation through its own pool, or a
// real-time frame loop whose rules forbid allocating (and the stalls that come
// with it) once it is running. gs_bin_sort needs a scratch workspace from the
// caller; this variant brings its own instead: a fixed array in static device
// memory, held until the process exits. The array is reserved when this
// file's device code is loaded on a device; under CUDA's lazy module loading
// that is the first cudaGetSymbolAddress below, i.e. the first call on the
// device, which callers make at set-up time. The caller still passes every
// input and output buffer.
#include <mutex>

#include "gs_common.cuh"

namespace {

constexpr size_t kNoAllocBytes = GS_NOALLOC_WORKSPACE_BYTES;

// The shared scratch. In host code this name is only a stand-in for the
// device symbol, never a usable address: its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per
// device (with that device current) and cached.
gs_status scratch_for_current_device(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GS_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return GS_OK;
}

} // namespace

extern "C" gs_status gs_bin_sort_noalloc(void *stream, const gs_camera *cams, int32_t ncam, int32_t P,
                                         const gs_config *cfg, const void *d_splat2d,
                                         int64_t capacity, uint32_t *d_vals, uint32_t *d_ranges,
                                         uint64_t *d_keys64, uint32_t *d_count, uint32_t *d_error)
{
    if (!cams || !cfg || ncam <= 0 || ncam > GS_MAX_CAMERAS || P < 0 || capacity < 0) return GS_ERR_ARG;
    const size_t need = gs_bin_sort_workspace_bytes(cams, ncam, P, cfg, capacity);
    if (need == 0 || need > kNoAllocBytes) return GS_ERR_ARG; // beyond the static scratch
    void *ws = nullptr;
    const gs_status st = scratch_for_current_device(&ws);
    if (st != GS_OK) return st;
    // gs_bin_sort clears the zero-initialised part of the workspace itself
    // (the error word included, so the word read below is this call's).
    const gs_status rs = gs_bin_sort(stream, cams, ncam, P, cfg, d_splat2d, capacity, ws, kNoAllocBytes,
                                     d_vals, d_ranges, d_keys64, d_count);
    if (rs != GS_OK || !d_error) return rs;
    // the error word sits at the start of the workspace; hand it out, since
    // the caller cannot name the static array
    return gs_workspace_status_async(stream, ws, d_error);
}
