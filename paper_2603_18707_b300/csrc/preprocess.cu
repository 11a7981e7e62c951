// preprocess.cu — projection of splats into one or more cameras (sm_103a).
//
// One thread per splat. The splat's parameters (mean, scale, rotation,
// opacity and up to 48 SH coefficients) are read from HBM once and kept in
// registers while the thread loops over every camera of the batch, writing
// one 48-byte record per (camera, splat). The kernel is bandwidth-bound:
// 4 * (3 + 3 + 4 + 1 + 3 (d+1)^2) bytes in per splat, 64 bytes out per camera.
//
// Per camera it computes, in FP32 (3DGS EWA projection, which the paper
// relies on in Sec. 2; then the paper's own steps):
//   Sigma = R S S^T R^T, t = W mu + t_cam, J (tx/tz, ty/tz clamped to
//   1.3 tan(fov/2)), Sigma' = J W Sigma W^T J^T, low-pass + v I, AA factor
//   rho = sqrt(|Sigma'| / |Sigma' + v I|) and o' = o rho (Sec. 3.4, Eq. 7-9),
//   conic (Sigma' + v I)^-1, mu', SH colour, support threshold x_cut
//   (Eq. 3-5, App. B), rectangle of tiles around the support ellipse.
#include "gs_common.cuh"

namespace gs {
namespace {

// Real SH basis (3DGS order and signs), constants from their closed forms:
// Y00 = 1/(2 sqrt(pi)); band 1: sqrt(3/(4 pi)); band 2: sqrt(15/pi)/2,
// sqrt(5/pi)/4, sqrt(15/pi)/4; band 3: sqrt(35/(2 pi))/4, sqrt(105/pi)/2,
// sqrt(21/(2 pi))/4, sqrt(7/pi)/4, sqrt(105/pi)/4.
constexpr float kY0 = 0.28209479177387814f;
constexpr float kY1 = 0.48860251190291992f;
constexpr float kY2a = 1.0925484305920792f;
constexpr float kY2b = 0.31539156525252005f;
constexpr float kY2c = 0.54627421529603959f;
constexpr float kY3a = 0.59004358992664352f;
constexpr float kY3b = 2.8906114426405538f;
constexpr float kY3c = 0.45704579946446572f;
constexpr float kY3d = 0.37317633259011546f;
constexpr float kY3e = 1.4453057213202769f;

template <int D>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y)
{
    Y[0] = kY0;
    if (D >= 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
    }
    if (D >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * x * y;
        Y[5] = -kY2a * y * z;
        Y[6] = kY2b * (2.f * zz - xx - yy);
        Y[7] = -kY2a * x * z;
        Y[8] = kY2c * (xx - yy);
        if (D >= 3) {
            Y[9] = -kY3a * y * (3.f * xx - yy);
            Y[10] = kY3b * x * y * z;
            Y[11] = -kY3c * y * (4.f * zz - xx - yy);
            Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kY3c * x * (4.f * zz - xx - yy);
            Y[14] = kY3e * z * (xx - yy);
            Y[15] = -kY3a * x * (xx - 3.f * yy);
        }
    }
}

// Support threshold in quadric units; < 0 means "no pixel reaches eps".
__device__ __forceinline__ float support_threshold(const CfgDev &cfg, float o)
{
    if (cfg.cull == GS_CULL_LEGACY3) return 9.f;
    if (cfg.cull == GS_CULL_UNIVERSAL) {
        if (cfg.kind == GS_K_EXP) return -2.f * logf(cfg.eps);
        return cfg.x0;
    }
    const int n = kind_order(cfg.kind);
    const float k0 = (cfg.kind == GS_K_EXP) ? 1.f : cfg.c[0];
    if (!(o * k0 >= cfg.eps)) return -1.f;
    if (cfg.kind == GS_K_EXP) return 2.f * (logf(o) - logf(cfg.eps)); // Eq. 3
    if (cfg.kind == GS_K_POLY1) return (cfg.eps - o * cfg.c[0]) / (o * cfg.c[1]); // Eq. 4
    float r = first_root_f32(cfg.c, n, cfg.eps / o); // App. B
    if (cfg.kind == GS_K_POLY2 && r > cfg.x0) r = cfg.x0;  // Eq. 6 cut
    return r;
}

#ifndef GS_PRE_MIN_BLOCKS
#define GS_PRE_MIN_BLOCKS 8 // 128-thread CTAs per SM the register budget must allow
#endif
template <int D>
__global__ void __launch_bounds__(128, GS_PRE_MIN_BLOCKS)
preprocess_kernel(const __grid_constant__ CamTable cams, const __grid_constant__ CfgDev cfg,
                  int P, const float *__restrict__ means, const float *__restrict__ scales,
                  const float *__restrict__ quats, const float *__restrict__ opacities,
                  const float *__restrict__ sh, Splat2DPtrs out)
{
    constexpr int K = (D + 1) * (D + 1), F = 3 * K;
    // The CTA's SH coefficients, staged once and read for every camera (kept
    // out of registers: higher occupancy). When a splat's F floats are whole
    // 16-byte chunks (degrees 1 and 3) each splat keeps a row of its own,
    // read with 16-byte loads; the row stride (in chunks) is odd, so that 8
    // lanes reading the same chunk of their rows cover all 32 banks.
    // Otherwise the layout is transposed ([coefficient][splat]).
    constexpr bool kRows = F % 4 == 0;
    constexpr int FS = kRows ? ((F / 4) % 2 ? F : F + 4) : F; // floats per staged row
    __shared__ __align__(16) float s_sh[kRows ? FS * 128 : F * 128];
    const int i0 = blockIdx.x * 128, i = i0 + (int)threadIdx.x;
    const int nb = min(128, P - i0);
    const float *src = sh + (size_t)i0 * F;
    if (kRows) {
        for (int e = threadIdx.x; e < nb * F / 4; e += 128) {
            const int sp = (4 * e) / F, j = 4 * e - sp * F; // the four floats share a splat
            *reinterpret_cast<float4 *>(&s_sh[sp * FS + j]) = reinterpret_cast<const float4 *>(src)[e];
        }
    } else {
        for (int e = threadIdx.x; e < nb * F; e += 128) {
            const int sp = e / F;
            s_sh[(e - sp * F) * 128 + sp] = src[e];
        }
    }
    __syncthreads();
    if (i >= P) return;

    const float mx = means[3 * i + 0], my = means[3 * i + 1], mz = means[3 * i + 2];
    const float sx = scales[3 * i + 0], sy = scales[3 * i + 1], sz = scales[3 * i + 2];
    const float4 q4 = reinterpret_cast<const float4 *>(quats)[i];
    const float op = opacities[i];

    // Sigma = M M^T with M = R(q) diag(s), q normalised.
    const float qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float w = q4.x * qn, x = q4.y * qn, y = q4.z * qn, z = q4.w * qn;
    const float R00 = 1.f - 2.f * (y * y + z * z), R01 = 2.f * (x * y - w * z), R02 = 2.f * (x * z + w * y);
    const float R10 = 2.f * (x * y + w * z), R11 = 1.f - 2.f * (x * x + z * z), R12 = 2.f * (y * z - w * x);
    const float R20 = 2.f * (x * z - w * y), R21 = 2.f * (y * z + w * x), R22 = 1.f - 2.f * (x * x + y * y);
    const float M00 = R00 * sx, M01 = R01 * sy, M02 = R02 * sz;
    const float M10 = R10 * sx, M11 = R11 * sy, M12 = R12 * sz;
    const float M20 = R20 * sx, M21 = R21 * sy, M22 = R22 * sz;
    const float S00 = M00 * M00 + M01 * M01 + M02 * M02;
    const float S01 = M00 * M10 + M01 * M11 + M02 * M12;
    const float S02 = M00 * M20 + M01 * M21 + M02 * M22;
    const float S11 = M10 * M10 + M11 * M11 + M12 * M12;
    const float S12 = M10 * M20 + M11 * M21 + M12 * M22;
    const float S22 = M20 * M20 + M21 * M21 + M22 * M22;

    const int sw = __ffs(cfg.tile_w) - 1, shh = __ffs(cfg.tile_h) - 1; // log2 of the tile size
    for (int c = 0; c < cams.ncam; ++c) {
        const CamDev &cm = cams.cam[c];
        const int64_t n = (int64_t)c * P + i;
        const float *W = cm.R;
        const float tx = W[0] * mx + W[1] * my + W[2] * mz + cm.T[0];
        const float ty = W[3] * mx + W[4] * my + W[5] * mz + cm.T[1];
        const float tz = W[6] * mx + W[7] * my + W[8] * mz + cm.T[2];
        bool drawn = tz > cm.znear;
        float4 r0 = make_float4(0.f, 0.f, 0.f, tz), r1 = make_float4(0.f, 0.f, 0.f, -1.f),
               r2 = make_float4(0.f, 0.f, 0.f, 0.f);
        ushort4 rect = make_ushort4(0, 0, 0, 0);
        uint32_t ntiles = 0;
        if (drawn) {
            const float iz = 1.f / tz;
            const float ux = fminf(fmaxf(tx * iz, -cm.limx), cm.limx);
            const float uy = fminf(fmaxf(ty * iz, -cm.limy), cm.limy);
            // Tm = J W: rows fx/tz (W0 - ux W2) and fy/tz (W1 - uy W2)
            const float a0 = cm.fx * iz, b0 = cm.fy * iz;
            const float T00 = a0 * (W[0] - ux * W[6]), T01 = a0 * (W[1] - ux * W[7]), T02 = a0 * (W[2] - ux * W[8]);
            const float T10 = b0 * (W[3] - uy * W[6]), T11 = b0 * (W[4] - uy * W[7]), T12 = b0 * (W[5] - uy * W[8]);
            // Sigma' = Tm Sigma Tm^T
            const float u0 = S00 * T00 + S01 * T01 + S02 * T02;
            const float u1 = S01 * T00 + S11 * T01 + S12 * T02;
            const float u2 = S02 * T00 + S12 * T01 + S22 * T02;
            const float v0 = S00 * T10 + S01 * T11 + S02 * T12;
            const float v1 = S01 * T10 + S11 * T11 + S12 * T12;
            const float v2 = S02 * T10 + S12 * T11 + S22 * T12;
            const float c00 = T00 * u0 + T01 * u1 + T02 * u2;
            const float c01 = T10 * u0 + T11 * u1 + T12 * u2;
            const float c11 = T10 * v0 + T11 * v1 + T12 * v2;
            const float a = c00 + cfg.dil, b = c01, cc = c11 + cfg.dil;
            const float det0 = c00 * c11 - c01 * c01;
            const float det1 = a * cc - b * b;
            drawn = det1 > 0.f;
            if (drawn) {
                const float idet = 1.f / det1;
                const float rho = cfg.aa ? sqrtf(fmaxf(det0, 0.f) * idet) : 1.f;
                const float o2 = op * rho;
                const float mx2 = cm.fx * tx * iz + cm.cx;
                const float my2 = cm.fy * ty * iz + cm.cy;
                float xc = support_threshold(cfg, o2);
                drawn = xc >= 0.f;
                if (drawn) {
                    // margin so that FP32 rounding never makes the rectangle too small
                    xc = xc * 1.001f + 1e-4f;
                    float hx, hy;
                    if (cfg.rect_mode == GS_RECT_CIRCLE) {
                        const float mid = 0.5f * (a + cc);
                        const float lmax = mid + sqrtf(fmaxf(mid * mid - det1, 0.f));
                        hx = hy = sqrtf(xc * lmax);
                    } else {
                        hx = sqrtf(xc * a);
                        hy = sqrtf(xc * cc);
                    }
                    const float px0 = fmaxf(ceilf(mx2 - hx - 0.5f), 0.f);
                    const float px1 = fminf(floorf(mx2 + hx - 0.5f), (float)(cm.W - 1));
                    const float py0 = fmaxf(ceilf(my2 - hy - 0.5f), 0.f);
                    const float py1 = fminf(floorf(my2 + hy - 0.5f), (float)(cm.H - 1));
                    r0 = make_float4(mx2, my2, o2, tz);
                    r1 = make_float4(cc * idet, -b * idet, a * idet, xc);
                    if (px0 <= px1 && py0 <= py1) {
                        // pixel -> tile: non-negative, power-of-two tile sizes
                        const int gx0 = (int)px0 >> sw, gx1 = (int)px1 >> sw;
                        const int gy0 = (int)py0 >> shh, gy1 = (int)py1 >> shh;
                        rect = make_ushort4(gx0, gy0, gx1, gy1);
                        if (cfg.rect_mode == GS_RECT_ELLIPSE && gx1 > gx0 && gy1 > gy0) {
                            // only the tiles of each row that the ellipse reaches (a
                            // single-row or single-column rectangle keeps all its
                            // tiles: the band covers the whole ellipse there)
                            for (int ty = gy0; ty <= gy1; ++ty) {
                                int c0, c1;
                                if (row_cols(r0.x, r0.y, r1.x, r1.y, r1.z, r1.w, ty, cfg.tile_w,
                                             cfg.tile_h, cm.W, cm.H, gx0, gx1, c0, c1))
                                    ntiles += (uint32_t)(c1 - c0 + 1);
                            }
                        } else {
                            ntiles = (uint32_t)((gx1 - gx0 + 1) * (gy1 - gy0 + 1));
                        }
                    }
                    if (ntiles) {
                        // view-dependent colour, only for records that are drawn
                        float dx = mx - cm.campos[0], dy = my - cm.campos[1], dz = mz - cm.campos[2];
                        const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
                        dx *= il; dy *= il; dz *= il;
                        float Y[K];
                        sh_basis<D>(dx, dy, dz, Y);
                        float col[3] = {0.f, 0.f, 0.f};
                        if constexpr (kRows) {
                            // coefficient m = 3 k + ch of this splat's row, 4 per load
                            const float4 *row = reinterpret_cast<const float4 *>(s_sh + threadIdx.x * FS);
#pragma unroll
                            for (int q = 0; q < F / 4; ++q) {
                                const float4 c4 = row[q];
                                const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    col[(4 * q + e) % 3] = fmaf(Y[(4 * q + e) / 3], cv[e], col[(4 * q + e) % 3]);
                            }
                        } else {
                            const float *coef = s_sh + threadIdx.x; // coefficient m at coef[128 m]
#pragma unroll
                            for (int ch = 0; ch < 3; ++ch) {
#pragma unroll
                                for (int k = 0; k < K; ++k) col[ch] = fmaf(Y[k], coef[128 * (3 * k + ch)], col[ch]);
                            }
                        }
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) col[ch] = fmaxf(col[ch] + 0.5f, 0.f);
                        r2 = make_float4(col[0], col[1], col[2], rho);
                    }
                }
            }
        }
        // a record that covers no tile is never read past its tile count:
        // only that count is written for it
        out.tiles[n] = ntiles;
        if (ntiles) {
            out.rec[3 * n + 0] = r0;
            out.rec[3 * n + 1] = r1;
            out.rec[3 * n + 2] = r2;
            out.rect[n] = rect;
            out.dkey[n] = __float_as_uint(tz);
        }
    }
}

} // namespace
} // namespace gs

using namespace gs;

extern "C" size_t gs_splat2d_bytes(int32_t ncam, int32_t P)
{
    if (ncam <= 0 || P < 0) return 0;
    return splat2d_bytes((int64_t)ncam * P);
}

extern "C" gs_status gs_preprocess(void *stream, const gs_camera *cams, int32_t ncam, int32_t P,
                                   const float *d_means, const float *d_scales,
                                   const float *d_quats, const float *d_opacities,
                                   const float *d_sh, int32_t sh_degree, const gs_config *cfg,
                                   void *d_splat2d)
{
    if (!cams || !cfg || ncam <= 0 || ncam > kMaxCams || P < 0 || sh_degree < 0 || sh_degree > 3)
        return GS_ERR_ARG;
    if (P == 0) return GS_OK;
    if (!d_means || !d_scales || !d_quats || !d_opacities || !d_sh || !d_splat2d) return GS_ERR_ARG;
    if (((uintptr_t)d_quats & 15) || ((uintptr_t)d_splat2d & 255) ||
        (sh_degree > 0 && ((uintptr_t)d_sh & 15)))
        return GS_ERR_ARG;
    if ((int64_t)ncam * P >= (int64_t)1 << 31) return GS_ERR_ARG;
    static_assert(sizeof(CamTable) < 32000, "kernel parameter space");
    CamTable t;
    CfgDev c;
    if (!build_cam_table(cams, ncam, cfg, &t) || !build_cfg(cfg, &c)) return GS_ERR_ARG;
    Splat2DPtrs o = splat2d_ptrs(d_splat2d, (int64_t)ncam * P);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int threads = 128, blocks = (P + threads - 1) / threads;
    switch (sh_degree) {
    case 0: preprocess_kernel<0><<<blocks, threads, 0, s>>>(t, c, P, d_means, d_scales, d_quats, d_opacities, d_sh, o); break;
    case 1: preprocess_kernel<1><<<blocks, threads, 0, s>>>(t, c, P, d_means, d_scales, d_quats, d_opacities, d_sh, o); break;
    case 2: preprocess_kernel<2><<<blocks, threads, 0, s>>>(t, c, P, d_means, d_scales, d_quats, d_opacities, d_sh, o); break;
    default: preprocess_kernel<3><<<blocks, threads, 0, s>>>(t, c, P, d_means, d_scales, d_quats, d_opacities, d_sh, o); break;
    }
    count_launch();
    GS_LAUNCH_CHECK();
    return GS_OK;
}
