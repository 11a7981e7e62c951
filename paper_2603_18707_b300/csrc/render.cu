// render.cu — front-to-back blending per tile (sm_103a).
//
// One CTA per (camera, tile); one thread per pixel. The tile's depth-sorted
// list is streamed through shared memory in batches: each thread gathers one
// 48-byte record (mean, o', conic, colour), then every thread walks the batch
// for its pixel. Per entry (Sec. 2, Eq. 1 / 2 / 6):
//   Q = A dx^2 + 2 B dx dy + C dy^2,  alpha = min(alpha_max, o' k(Q)),
//   skip if alpha < eps; stop (without adding) if T (1 - alpha) < t_min;
//   C += c alpha T; T *= 1 - alpha.
// The polynomial kernels are Horner FMAs only: no special-function unit.
// The exponential is one MUFU ex2 per entry. A CTA leaves its list as soon
// as every pixel has stopped (__syncthreads_count at each batch).
#include "gs_common.cuh"

namespace gs {
namespace {

template <int KIND>
__device__ __forceinline__ float kernel_value(const CfgDev &cfg, float Q)
{
    if (KIND == GS_K_EXP) return __expf(-0.5f * Q);
    if (KIND == GS_K_POLY1) return fmaf(cfg.c[1], Q, cfg.c[0]);
    if (KIND == GS_K_POLY2) return Q < cfg.x0 ? fmaf(fmaf(cfg.c[2], Q, cfg.c[1]), Q, cfg.c[0]) : 0.f;
    return fmaf(fmaf(fmaf(cfg.c[3], Q, cfg.c[2]), Q, cfg.c[1]), Q, cfg.c[0]);
}

constexpr int kMaxBatch = 256;

template <int KIND>
__global__ void __launch_bounds__(256)
render_kernel(const __grid_constant__ CamTable cams, const __grid_constant__ CfgDev cfg,
              const float4 *__restrict__ rec, const uint32_t *__restrict__ vals,
              const uint2 *__restrict__ ranges, uint32_t n_records, float bg0, float bg1, float bg2,
              float *__restrict__ out, float *__restrict__ final_T, uint32_t *__restrict__ last,
              uint32_t *__restrict__ n_eval)
{
    __shared__ float4 s_g[kMaxBatch];
    __shared__ float4 s_q[kMaxBatch];
    __shared__ float4 s_c[kMaxBatch];
    const int gtile = blockIdx.x;
    int c = 0;
    while (c + 1 < cams.ncam && cams.cam[c + 1].tile_base <= gtile) ++c;
    const CamDev &cm = cams.cam[c];
    const int lt = gtile - cm.tile_base;
    const int tx = lt % cm.tiles_x, ty = lt / cm.tiles_x;
    const int px = tx * cfg.tile_w + (int)threadIdx.x % cfg.tile_w;
    const int py = ty * cfg.tile_h + (int)threadIdx.x / cfg.tile_w;
    const bool inside = px < cm.W && py < cm.H;
    const float pxc = px + 0.5f, pyc = py + 0.5f;
    const uint2 rg = ranges[gtile];
    const uint32_t n = rg.y - rg.x;
    const int B = blockDim.x;

    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    bool done = !inside;
    uint32_t lastc = 0, ne = n;
    const float eps = cfg.eps, amax = cfg.alpha_max, tmin = cfg.t_min;
    for (uint32_t base = 0; base < n; base += B) {
        if (__syncthreads_count(done) == B) break;
        const uint32_t i = base + threadIdx.x;
        if (i < n) {
            uint32_t v = vals[rg.x + i];
            if (v >= n_records) v = 0; // only after a timed-out sort wait
            s_g[threadIdx.x] = rec[3 * (size_t)v + 0];
            s_q[threadIdx.x] = rec[3 * (size_t)v + 1];
            s_c[threadIdx.x] = rec[3 * (size_t)v + 2];
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)B, n - base);
        if (!done) {
            for (int j = 0; j < cnt; ++j) {
                const float4 g = s_g[j];
                const float4 q = s_q[j];
                const float dx = g.x - pxc, dy = g.y - pyc;
                const float Q = fmaf(fmaf(q.x, dx, 2.f * q.y * dy), dx, q.z * dy * dy);
                const float a = fminf(amax, g.z * kernel_value<KIND>(cfg, Q));
                if (a < eps) continue;
                const float Tn = T * (1.f - a);
                if (Tn < tmin) {
                    done = true;
                    ne = base + j + 1;
                    break;
                }
                const float4 col = s_c[j];
                const float w = a * T;
                C0 = fmaf(col.x, w, C0);
                C1 = fmaf(col.y, w, C1);
                C2 = fmaf(col.z, w, C2);
                T = Tn;
                lastc = base + j + 1;
            }
        }
    }
    if (inside) {
        const int64_t pix = cm.pix_base + (int64_t)py * cm.W + px;
        out[3 * pix + 0] = fmaf(T, bg0, C0);
        out[3 * pix + 1] = fmaf(T, bg1, C1);
        out[3 * pix + 2] = fmaf(T, bg2, C2);
        if (final_T) final_T[pix] = T;
        if (last) last[pix] = lastc;
        if (n_eval) n_eval[pix] = ne;
    }
}

} // namespace
} // namespace gs

using namespace gs;

extern "C" gs_status gs_render(void *stream, const gs_camera *cams, int32_t ncam, int32_t P,
                               const gs_config *cfg, const void *d_splat2d, const uint32_t *d_vals,
                               const uint32_t *d_ranges, const float *bg, float *d_out_rgb,
                               float *d_final_T, uint32_t *d_last, uint32_t *d_n_eval)
{
    if (!cams || !cfg || !bg || ncam <= 0 || ncam > kMaxCams || P < 0) return GS_ERR_ARG;
    if (!d_ranges || !d_out_rgb || (P > 0 && (!d_splat2d || !d_vals))) return GS_ERR_ARG;
    CamTable t;
    CfgDev c;
    if (!build_cam_table(cams, ncam, cfg, &t) || !build_cfg(cfg, &c)) return GS_ERR_ARG;
    if (cfg->fp16x2 || cfg->px_per_thread != 1) return GS_ERR_UNSUPPORTED;
    const int threads = cfg->tile_w * cfg->tile_h;
    if (threads > kMaxBatch) return GS_ERR_UNSUPPORTED;
    if (t.total_tiles == 0) return GS_OK;
    const float4 *rec = P > 0 ? splat2d_const(d_splat2d, (int64_t)ncam * P).rec : nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint2 *rg = reinterpret_cast<const uint2 *>(d_ranges);
#define GS_RENDER_LAUNCH(K)                                                                   \
    render_kernel<K><<<t.total_tiles, threads, 0, s>>>(t, c, rec, d_vals, rg, (uint32_t)((int64_t)ncam * P), bg[0], bg[1], bg[2], \
                                                      d_out_rgb, d_final_T, d_last, d_n_eval)
    switch (cfg->kind) {
    case GS_K_EXP: GS_RENDER_LAUNCH(GS_K_EXP); break;
    case GS_K_POLY1: GS_RENDER_LAUNCH(GS_K_POLY1); break;
    case GS_K_POLY2: GS_RENDER_LAUNCH(GS_K_POLY2); break;
    default: GS_RENDER_LAUNCH(GS_K_POLY3); break;
    }
#undef GS_RENDER_LAUNCH
    count_launch();
    GS_LAUNCH_CHECK();
    return GS_OK;
}
