// render.cu — front-to-back blending per tile (sm_103a).
//
// One CTA per (camera, tile). Each thread owns PPT horizontally adjacent
// pixels of one row. The tile's depth-sorted list is streamed through shared
// memory in batches: the block gathers the batch's 48-byte records and turns
// each into the per-tile coefficients of blend_math.cuh (two affine forms
// whose squares sum to the quadric, opacity folded into the kernel). Then every
// thread walks the batch. Per entry and pixel (Sec. 2, Eq. 1 / 2 / 6):
//   Q = u^2 + v^2,  alpha = min(alpha_max, o' k(Q)),
//   skip if alpha < eps; stop (without adding) if T (1 - alpha) < t_min;
//   C += c alpha T; T *= 1 - alpha.
// Cost per entry and thread: 2 LDS.128, 3 FP32 ops per row and 3 per pixel
// for alpha (f1), the blend FMAs only where alpha >= eps. The polynomial
// kernels use FMAs only; exp adds one MUFU ex2. The block leaves its list as
// soon as every pixel has stopped (__syncthreads_count at each batch). The
// kernel is bound by instruction issue on the FP32 pipes.
#include "blend_math.cuh"

namespace gs {
namespace {

constexpr int kBatch = 256;

template <int KIND, int PPT>
__global__ void __launch_bounds__(256 / PPT)
render_kernel(const __grid_constant__ CamTable cams, const __grid_constant__ CfgDev cfg,
              const float4 *__restrict__ rec, const uint32_t *__restrict__ vals,
              const uint2 *__restrict__ ranges, uint32_t n_records, float bg0, float bg1, float bg2,
              float *__restrict__ out, float *__restrict__ final_T, uint32_t *__restrict__ last,
              uint32_t *__restrict__ n_eval)
{
    __shared__ float4 s_a[kBatch];
    __shared__ float4 s_b[kBatch];
    __shared__ float4 s_c[kBatch];
    const int gtile = blockIdx.x;
    int c = 0;
    while (c + 1 < cams.ncam && cams.cam[c + 1].tile_base <= gtile) ++c;
    const CamDev &cm = cams.cam[c];
    const int lt = gtile - cm.tile_base;
    const int tx = lt % cm.tiles_x, ty = lt / cm.tiles_x;
    const int tpr = cfg.tile_w / PPT; // threads per tile row
    const int lx = ((int)threadIdx.x % tpr) * PPT, ly = (int)threadIdx.x / tpr;
    const float ox = (float)(tx * cfg.tile_w), oy = (float)(ty * cfg.tile_h);
    const int px0 = tx * cfg.tile_w + lx, py = ty * cfg.tile_h + ly;
    const float y = ly + 0.5f;
    const uint2 rg = ranges[gtile];
    const uint32_t n = rg.y - rg.x;
    const int nthreads = blockDim.x;

    float T[PPT], C0[PPT], C1[PPT], C2[PPT], xs[PPT];
    uint32_t lastc[PPT], ne[PPT];
    unsigned active = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        T[k] = 1.f;
        C0[k] = C1[k] = C2[k] = 0.f;
        xs[k] = lx + k + 0.5f;
        lastc[k] = 0;
        ne[k] = n;
        if (px0 + k < cm.W && py < cm.H) active |= 1u << k;
    }
    const float eps = cfg.eps, amax = cfg.alpha_max, tmin = cfg.t_min;
    for (uint32_t base = 0; base < n; base += kBatch) {
        if (__syncthreads_count(active != 0) == 0) break;
        for (int i = threadIdx.x; i < kBatch; i += nthreads) {
            if (base + i < n) {
                uint32_t v = vals[rg.x + base + i];
                if (v >= n_records) v = 0; // only after a timed-out sort wait
                const BlendCoef k = make_coef<KIND>(cfg, rec[3 * (size_t)v + 0], rec[3 * (size_t)v + 1],
                                                    rec[3 * (size_t)v + 2], ox, oy);
                s_a[i] = k.a;
                s_b[i] = k.b;
                s_c[i] = k.c;
            }
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)kBatch, n - base);
        for (int j = 0; j < cnt && active; ++j) {
            const float4 a = s_a[j];
            const float4 b = s_b[j];
            const float ub = fmaf(a.y, y, a.z);
            const float vv = fmaf(a.w, y, b.x);
            const float v2 = vv * vv;
            const float p3 = (KIND == GS_K_POLY3) ? s_c[j].w : 0.f; // the cubic's top coefficient
            float al[PPT];
            bool any = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const float u = fmaf(a.x, xs[k], ub);
                const float Q = fmaf(u, u, v2);
                al[k] = fminf(amax, alpha_of_q<KIND>(cfg, b, p3, Q));
                any |= (active >> k & 1u) && al[k] >= eps;
            }
            if (!any) continue;
            const float4 col = s_c[j];
            const uint32_t pos = base + j + 1;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (!(active >> k & 1u) || !(al[k] >= eps)) continue;
                const float Tn = fmaf(-al[k], T[k], T[k]);
                if (Tn < tmin) {
                    active &= ~(1u << k);
                    ne[k] = pos;
                    continue;
                }
                const float w = al[k] * T[k];
                C0[k] = fmaf(col.x, w, C0[k]);
                C1[k] = fmaf(col.y, w, C1[k]);
                C2[k] = fmaf(col.z, w, C2[k]);
                T[k] = Tn;
                lastc[k] = pos;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (px0 + k < cm.W && py < cm.H) {
            const int64_t pix = cm.pix_base + (int64_t)py * cm.W + px0 + k;
            out[3 * pix + 0] = fmaf(T[k], bg0, C0[k]);
            out[3 * pix + 1] = fmaf(T[k], bg1, C1[k]);
            out[3 * pix + 2] = fmaf(T[k], bg2, C2[k]);
            if (final_T) final_T[pix] = T[k];
            if (last) last[pix] = lastc[k];
            if (n_eval) n_eval[pix] = ne[k];
        }
    }
}

template <int KIND>
void launch_render(int ppt, int blocks, int threads, cudaStream_t s, const CamTable &t, const CfgDev &c,
                   const float4 *rec, const uint32_t *vals, const uint2 *rg, uint32_t nrec,
                   const float *bg, float *out, float *fT, uint32_t *last, uint32_t *ne)
{
    if (ppt == 4)
        render_kernel<KIND, 4><<<blocks, threads, 0, s>>>(t, c, rec, vals, rg, nrec, bg[0], bg[1], bg[2], out, fT, last, ne);
    else if (ppt == 2)
        render_kernel<KIND, 2><<<blocks, threads, 0, s>>>(t, c, rec, vals, rg, nrec, bg[0], bg[1], bg[2], out, fT, last, ne);
    else
        render_kernel<KIND, 1><<<blocks, threads, 0, s>>>(t, c, rec, vals, rg, nrec, bg[0], bg[1], bg[2], out, fT, last, ne);
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
    const int ppt = cfg->px_per_thread;
    if (ppt != 1 && ppt != 2 && ppt != 4) return GS_ERR_ARG;
    if (cfg->fp16x2) return GS_ERR_UNSUPPORTED;
    if (cfg->tile_w % ppt) return GS_ERR_ARG;
    const int threads = cfg->tile_w * cfg->tile_h / ppt;
    if (t.total_tiles == 0) return GS_OK;
    const float4 *rec = P > 0 ? splat2d_const(d_splat2d, (int64_t)ncam * P).rec : nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint2 *rg = reinterpret_cast<const uint2 *>(d_ranges);
    const uint32_t nrec = (uint32_t)((int64_t)ncam * P);
    switch (cfg->kind) {
    case GS_K_EXP: launch_render<GS_K_EXP>(ppt, t.total_tiles, threads, s, t, c, rec, d_vals, rg, nrec, bg, d_out_rgb, d_final_T, d_last, d_n_eval); break;
    case GS_K_POLY1: launch_render<GS_K_POLY1>(ppt, t.total_tiles, threads, s, t, c, rec, d_vals, rg, nrec, bg, d_out_rgb, d_final_T, d_last, d_n_eval); break;
    case GS_K_POLY2: launch_render<GS_K_POLY2>(ppt, t.total_tiles, threads, s, t, c, rec, d_vals, rg, nrec, bg, d_out_rgb, d_final_T, d_last, d_n_eval); break;
    default: launch_render<GS_K_POLY3>(ppt, t.total_tiles, threads, s, t, c, rec, d_vals, rg, nrec, bg, d_out_rgb, d_final_T, d_last, d_n_eval); break;
    }
    count_launch();
    GS_LAUNCH_CHECK();
    return GS_OK;
}
