// render.cu — front-to-back blending per tile (sm_103a).
//
// One CTA renders one (camera, tile) at a time. Each thread owns PPT
// horizontally adjacent pixels of one row. The tile's depth-sorted list is
// streamed through shared memory in batches of `batch` entries: the block
// gathers the batch's 48-byte records and turns each into the per-tile
// coefficients of blend_math.cuh (two affine forms whose squares sum to the
// quadric, opacity folded into the kernel). Then every thread walks the
// batch. Per entry and pixel (Sec. 2, Eq. 1 / 2 / 6):
//   Q = u^2 + v^2,  alpha = min(alpha_max, o' k(Q)),
//   skip if alpha < eps; stop (without adding) if T (1 - alpha) < t_min;
//   C += c alpha T; T *= 1 - alpha.
// Cost per entry and thread: 2 LDS.128, 3 FP32 ops per row and 3 per pixel
// for alpha (f1), the blend FMAs only where alpha >= eps. The polynomial
// kernels use FMAs only; exp adds one MUFU ex2. The block leaves a list as
// soon as every pixel has stopped (__syncthreads_count at each batch). The
// kernel is bound by instruction issue on the FP32 pipes.
//
// Launch modes: one CTA per tile (grid = all tiles of all cameras), or
// persistent: a grid sized to fill every SM once, each CTA taking the next
// tile from an atomic counter until all tiles of all cameras are done (one
// launch for any mix of resolutions, balanced dynamically).
#include <algorithm>

#include <cuda_fp16.h>

#include "blend_math.cuh"

namespace gs {
namespace {

constexpr int kMaxBatch = 256;
#ifndef GS_RENDER_MIN_BLOCKS
#define GS_RENDER_MIN_BLOCKS 4 // 256-thread CTAs per SM the register budget must allow (64 registers: measured fastest)
#endif
// Per-pixel update: predicated (no branch per pixel) or branching. 0: branch
// for every kernel, 1: predicate for every kernel, 2: predicate for exp only
// (measured: exp, which blends more entries per pixel, gains ~8%; f1 loses ~7%).
#ifndef GS_BLEND_BRANCHLESS
#define GS_BLEND_BRANCHLESS 2
#endif
template <int KIND>
constexpr bool blend_branchless()
{
    return GS_BLEND_BRANCHLESS == 1 || (GS_BLEND_BRANCHLESS == 2 && KIND == GS_K_EXP);
}

struct RenderArgs {
    const float4 *rec;
    const uint32_t *vals;
    const uint2 *ranges;
    uint32_t n_records;
    float bg0, bg1, bg2;
    float *out;
    float *final_T;
    uint32_t *last;
    uint32_t *n_eval;
};

// FP16x2 alpha of a pixel pair (u_a, u_b computed in FP32, sharing v^2):
// Q = u^2 + v^2 and the opacity-folded kernel in packed half2 FMAs.
// Q is clamped to the cut x0 before f'2's polynomial so that an overflowing
// Q (a far-away splat) gives 0 rather than inf * 0.
template <int KIND>
__device__ __forceinline__ float2 alpha_pair_h2(float ua, float ub, __half2 v2h, uint4 hp, __half2 x0h,
                                                __half2 amaxh)
{
    const __half2 p0 = *reinterpret_cast<__half2 *>(&hp.x), p1 = *reinterpret_cast<__half2 *>(&hp.y);
    const __half2 p2 = *reinterpret_cast<__half2 *>(&hp.z), p3 = *reinterpret_cast<__half2 *>(&hp.w);
    const __half2 u2 = __floats2half2_rn(ua, ub);
    const __half2 Q = __hfma2(u2, u2, v2h);
    __half2 al;
    if (KIND == GS_K_EXP) {
        al = h2exp2(__hfma2(p1, Q, p0));
    } else if (KIND == GS_K_POLY1) {
        al = __hfma2(p1, Q, p0);
    } else if (KIND == GS_K_POLY2) {
        const __half2 Qc = __hmin2(Q, x0h);
        al = __hmul2(__hlt2(Q, x0h), __hfma2(__hfma2(p2, Qc, p1), Qc, p0));
    } else {
        al = __hfma2(__hfma2(__hfma2(p3, Q, p2), Q, p1), Q, p0);
    }
    return __half22float2(__hmin2(al, amaxh));
}

template <int KIND, int PPT, bool HALF>
__device__ __forceinline__ void render_tile(const CamTable &cams, const CfgDev &cfg, const RenderArgs &g,
                                            int gtile, float4 *s_a, float4 *s_b, float4 *s_c, uint4 *s_h)
{
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
    const uint2 rg = g.ranges[gtile];
    const uint32_t n = rg.y - rg.x;
    const int nthreads = blockDim.x;
    const int B = cfg.batch;

    const float eps = cfg.eps, amax = cfg.alpha_max, tmin = cfg.t_min;
    float T[PPT], C0[PPT], C1[PPT], C2[PPT], xs[PPT], ek[PPT];
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
        // the alpha a pixel takes: eps while it is active, never once it
        // stopped (one compare per pixel and entry instead of a mask test)
        ek[k] = (active >> k & 1u) ? eps : INFINITY;
    }
    const __half2 x0h = __float2half2_rn(fminf(cfg.x0, 60000.f)), amaxh = __float2half2_rn(amax);
    // the FP16x2 alphas carry ~1e-3 absolute error: skip only far below eps
    const float eps_skip = HALF ? 0.5f * eps : eps * (1.f - 1.f / 1024.f);
    for (uint32_t base = 0; base < n; base += B) {
        if (__syncthreads_count(active != 0) == 0) break;
        for (int i = threadIdx.x; i < B; i += nthreads) {
            if (base + i < n) {
                uint32_t v = g.vals[rg.x + base + i];
                if (v >= g.n_records) v = 0; // only after a timed-out sort wait
                const BlendCoef k = make_coef<KIND>(cfg, g.rec[3 * (size_t)v + 0], g.rec[3 * (size_t)v + 1],
                                                    g.rec[3 * (size_t)v + 2], ox, oy);
                s_a[i] = k.a;
                s_b[i] = k.b;
                s_c[i] = k.c;
                if (HALF) {
                    const __half2 h[4] = {__float2half2_rn(k.b.y), __float2half2_rn(k.b.z),
                                          __float2half2_rn(k.b.w), __float2half2_rn(k.c.w)};
                    s_h[i] = *reinterpret_cast<const uint4 *>(h);
                }
            }
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)B, n - base);
        for (int j = 0; j < cnt && active; ++j) {
            const float4 a = s_a[j];
            const float4 b = s_b[j];
            const float ub = fmaf(a.y, y, a.z);
            const float vv = fmaf(a.w, y, b.x);
            const float v2 = vv * vv;
            const float p3 = (KIND == GS_K_POLY3) ? s_c[j].w : 0.f; // the cubic's top coefficient
            if (PPT > 1 && cfg.monotone) {
                // smallest Q over this thread's run of pixels: v^2 if u changes
                // sign along the run, else at the end with the smaller |u|.
                // With k non-increasing, alpha there bounds every pixel's; the
                // skip threshold sits below eps so that rounding can never
                // skip an entry that a pixel would take.
                const float ua = fmaf(a.x, xs[0], ub), uz = fmaf(a.x, xs[PPT - 1], ub);
                const float um = ((ua > 0.f) != (uz > 0.f)) ? 0.f : fminf(fabsf(ua), fabsf(uz));
                if (alpha_of_q<KIND>(cfg, b, p3, fmaf(um, um, v2)) < eps_skip) continue;
            }
            float al[PPT];
            if (HALF) {
                const uint4 hp = s_h[j];
                const __half2 v2h = __float2half2_rn(v2);
#pragma unroll
                for (int k = 0; k < PPT; k += 2) {
                    const float2 ap = alpha_pair_h2<KIND>(fmaf(a.x, xs[k], ub), fmaf(a.x, xs[k + 1], ub),
                                                          v2h, hp, x0h, amaxh);
                    al[k] = ap.x;
                    al[k + 1] = ap.y;
                }
            } else {
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    // min(alpha_max, x) < eps exactly when x < eps: the clamp
                    // is applied only to entries that are blended
                    const float u = fmaf(a.x, xs[k], ub);
                    const float Q = fmaf(u, u, v2);
                    al[k] = alpha_of_q<KIND>(cfg, b, p3, Q);
                }
            }
            const float4 col = s_c[j];
            const uint32_t pos = base + j + 1;
            if constexpr (blend_branchless<KIND>()) {
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const bool use = al[k] >= ek[k];
                    const float a = fminf(amax, al[k]);
                    const float Tn = fmaf(-a, T[k], T[k]);
                    const bool stop = use && Tn < tmin;
                    const bool add = use && !stop;
                    const float w = add ? a * T[k] : 0.f;
                    C0[k] = fmaf(col.x, w, C0[k]);
                    C1[k] = fmaf(col.y, w, C1[k]);
                    C2[k] = fmaf(col.z, w, C2[k]);
                    T[k] = add ? Tn : T[k];
                    lastc[k] = add ? pos : lastc[k];
                    ne[k] = stop ? pos : ne[k];
                    active &= ~((unsigned)stop << k);
                    ek[k] = stop ? INFINITY : ek[k];
                }
            } else {
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    if (!(al[k] >= ek[k])) continue;
                    al[k] = fminf(amax, al[k]);
                    const float Tn = fmaf(-al[k], T[k], T[k]);
                    if (Tn < tmin) {
                        active &= ~(1u << k);
                        ek[k] = INFINITY;
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
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (px0 + k < cm.W && py < cm.H) {
            const int64_t pix = cm.pix_base + (int64_t)py * cm.W + px0 + k;
            g.out[3 * pix + 0] = fmaf(T[k], g.bg0, C0[k]);
            g.out[3 * pix + 1] = fmaf(T[k], g.bg1, C1[k]);
            g.out[3 * pix + 2] = fmaf(T[k], g.bg2, C2[k]);
            if (g.final_T) g.final_T[pix] = T[k];
            if (g.last) g.last[pix] = lastc[k];
            if (g.n_eval) g.n_eval[pix] = ne[k];
        }
    }
}

template <int KIND, int PPT, bool HALF>
__global__ void __launch_bounds__(256, GS_RENDER_MIN_BLOCKS)
render_kernel(const __grid_constant__ CamTable cams, const __grid_constant__ CfgDev cfg,
              const __grid_constant__ RenderArgs g)
{
    __shared__ float4 s_a[kMaxBatch];
    __shared__ float4 s_b[kMaxBatch];
    __shared__ float4 s_c[kMaxBatch];
    __shared__ uint4 s_h[HALF ? kMaxBatch : 1];
    render_tile<KIND, PPT, HALF>(cams, cfg, g, blockIdx.x, s_a, s_b, s_c, s_h);
}

template <int KIND, int PPT, bool HALF>
__global__ void __launch_bounds__(256, GS_RENDER_MIN_BLOCKS)
render_persistent_kernel(const __grid_constant__ CamTable cams, const __grid_constant__ CfgDev cfg,
                         const __grid_constant__ RenderArgs g, uint32_t *work)
{
    __shared__ float4 s_a[kMaxBatch];
    __shared__ float4 s_b[kMaxBatch];
    __shared__ float4 s_c[kMaxBatch];
    __shared__ uint4 s_h[HALF ? kMaxBatch : 1];
    __shared__ uint32_t s_tile;
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(work, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        __syncthreads(); // every thread has read s_tile before it is overwritten
        if (t >= (uint32_t)cams.total_tiles) break;
        render_tile<KIND, PPT, HALF>(cams, cfg, g, (int)t, s_a, s_b, s_c, s_h);
    }
}

template <int KIND, int PPT, bool HALF>
cudaError_t launch2(int threads, cudaStream_t s, const CamTable &t, const CfgDev &c, const RenderArgs &g,
                    uint32_t *work)
{
    if (!work) {
        render_kernel<KIND, PPT, HALF><<<t.total_tiles, threads, 0, s>>>(t, c, g);
        return cudaPeekAtLastError();
    }
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_persistent_kernel<KIND, PPT, HALF>,
                                                      threads, 0) != cudaSuccess)
        return cudaGetLastError();
    const int grid = std::max(1, std::min(t.total_tiles, sms * std::max(per_sm, 1)));
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    render_persistent_kernel<KIND, PPT, HALF><<<grid, threads, 0, s>>>(t, c, g, work);
    return cudaPeekAtLastError();
}

template <int KIND>
cudaError_t launch_render(int ppt, bool half, int threads, cudaStream_t s, const CamTable &t,
                          const CfgDev &c, const RenderArgs &g, uint32_t *work)
{
    if (half) {
        if (ppt == 4) return launch2<KIND, 4, true>(threads, s, t, c, g, work);
        return launch2<KIND, 2, true>(threads, s, t, c, g, work);
    }
    if (ppt == 4) return launch2<KIND, 4, false>(threads, s, t, c, g, work);
    if (ppt == 2) return launch2<KIND, 2, false>(threads, s, t, c, g, work);
    return launch2<KIND, 1, false>(threads, s, t, c, g, work);
}

} // namespace
} // namespace gs

using namespace gs;

extern "C" size_t gs_render_work_bytes(void) { return 256; }

extern "C" gs_status gs_render(void *stream, const gs_camera *cams, int32_t ncam, int32_t P,
                               const gs_config *cfg, const void *d_splat2d, const uint32_t *d_vals,
                               const uint32_t *d_ranges, const float *bg, float *d_out_rgb,
                               float *d_final_T, uint32_t *d_last, uint32_t *d_n_eval,
                               void *d_work)
{
    if (!cams || !cfg || !bg || ncam <= 0 || ncam > kMaxCams || P < 0) return GS_ERR_ARG;
    if (!d_ranges || !d_out_rgb || (P > 0 && (!d_splat2d || !d_vals))) return GS_ERR_ARG;
    if (d_work && ((uintptr_t)d_work & 3)) return GS_ERR_ARG;
    CamTable t;
    CfgDev c;
    if (!build_cam_table(cams, ncam, cfg, &t) || !build_cfg(cfg, &c)) return GS_ERR_ARG;
    const int ppt = cfg->px_per_thread;
    if (ppt != 1 && ppt != 2 && ppt != 4) return GS_ERR_ARG;
    if (cfg->batch < 1 || cfg->batch > kMaxBatch) return GS_ERR_ARG;
    const bool half = cfg->fp16x2 != 0;
    if (half && ppt == 1) return GS_ERR_ARG; // packed pairs need 2 or 4 pixels per thread
    if (cfg->tile_w % ppt) return GS_ERR_ARG;
    const int threads = cfg->tile_w * cfg->tile_h / ppt;
    if (threads > 256) return GS_ERR_ARG; // 512-pixel tiles need 2 or 4 pixels per thread
    if (t.total_tiles == 0) return GS_OK;
    RenderArgs g;
    g.rec = P > 0 ? splat2d_const(d_splat2d, (int64_t)ncam * P).rec : nullptr;
    g.vals = d_vals;
    g.ranges = reinterpret_cast<const uint2 *>(d_ranges);
    g.n_records = (uint32_t)((int64_t)ncam * P);
    g.bg0 = bg[0]; g.bg1 = bg[1]; g.bg2 = bg[2];
    g.out = d_out_rgb;
    g.final_T = d_final_T;
    g.last = d_last;
    g.n_eval = d_n_eval;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t *work = static_cast<uint32_t *>(d_work);
    cudaError_t e;
    switch (cfg->kind) {
    case GS_K_EXP: e = launch_render<GS_K_EXP>(ppt, half, threads, s, t, c, g, work); break;
    case GS_K_POLY1: e = launch_render<GS_K_POLY1>(ppt, half, threads, s, t, c, g, work); break;
    case GS_K_POLY2: e = launch_render<GS_K_POLY2>(ppt, half, threads, s, t, c, g, work); break;
    default: e = launch_render<GS_K_POLY3>(ppt, half, threads, s, t, c, g, work); break;
    }
    count_launch();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    return GS_OK;
}
