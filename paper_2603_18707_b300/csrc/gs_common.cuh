// gs_common.cuh — shared device-side definitions of the sm_103a renderer.
//
// Camera and config tables travel as __grid_constant__ kernel parameters
// (no device allocation, capture-safe). Record layout of the per-(camera,
// splat) buffer is described in include/gs.h (gs_splat2d_bytes).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

constexpr int kMaxCams = GS_MAX_CAMERAS;

struct CamDev {
    float R[9];      // world -> camera rotation, row-major
    float T[3];      // world -> camera translation
    float campos[3]; // camera centre in world coordinates
    float fx, fy, cx, cy;
    float limx, limy; // 1.3 tan(fov/2): clamp of tx/tz, ty/tz in the EWA Jacobian
    float znear;
    int W, H;
    int tiles_x, tiles_y;
    int tile_base;    // first global tile id of this camera
    int64_t pix_base; // first pixel of this camera in the output buffers
};

struct CamTable {
    int ncam;
    int total_tiles;
    CamDev cam[kMaxCams];
};

struct CfgDev {
    int kind;
    float c[4];
    int cull;
    float eps, alpha_max, t_min;
    int aa;
    float dil;
    int tile_w, tile_h;
    int rect_mode;
    float x0;   // first positive root of the polynomial (poly kinds), +inf for exp
    int batch;
    int ppt;    // pixels per thread
    int monotone; // kernel non-increasing in Q over its support (allows skipping by Q bounds)
    // FP16x2 blend: bound on |alpha(half) - alpha(FP32)|, as a multiple of
    // p0 = o' c0 (polynomials) or of alpha (exp); and the cubic factored at
    // its support root r, c3 (Q - r)(Q^2 + f3b Q + f3g), for its half form
    float h2_band;
    float f3r, f3b, f3g;
    int f3_factored; // 1 when the cubic term is non-zero and the factors are finite
    int tail_zero;   // f3: the cubic stays <= 0 past its first root x0 (the kernel is 0 there)
};

// Pointers into the record buffer (see gs_splat2d_bytes).
struct Splat2DPtrs {
    float4 *rec;      // [N][3]
    ushort4 *rect;    // [N]
    uint32_t *tiles;  // [N]
    uint32_t *dkey;   // [N]
};

struct Splat2DConst {
    const float4 *rec;
    const ushort4 *rect;
    const uint32_t *tiles;
    const uint32_t *dkey;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline Splat2DPtrs splat2d_ptrs(void *base, int64_t N)
{
    char *p = static_cast<char *>(base);
    Splat2DPtrs s;
    s.rec = reinterpret_cast<float4 *>(p);
    p += align256(sizeof(float4) * 3 * N);
    s.rect = reinterpret_cast<ushort4 *>(p);
    p += align256(sizeof(ushort4) * N);
    s.tiles = reinterpret_cast<uint32_t *>(p);
    p += align256(sizeof(uint32_t) * N);
    s.dkey = reinterpret_cast<uint32_t *>(p);
    return s;
}

inline Splat2DConst splat2d_const(const void *base, int64_t N)
{
    Splat2DPtrs s = splat2d_ptrs(const_cast<void *>(base), N);
    return Splat2DConst{s.rec, s.rect, s.tiles, s.dkey};
}

inline size_t splat2d_bytes(int64_t N)
{
    return align256(sizeof(float4) * 3 * N) + align256(sizeof(ushort4) * N) +
           align256(sizeof(uint32_t) * N) + align256(sizeof(uint32_t) * N);
}

// ---- host helpers shared by the entry points (defined in capi.cu) ----
bool build_cam_table(const gs_camera *cams, int ncam, const gs_config *cfg, CamTable *t);
bool build_cfg(const gs_config *cfg, CfgDev *d);
void count_launch(uint64_t n = 1);
gs_status launch_status();

// ---- polynomial helpers (host + device, FP32) ----
__host__ __device__ inline int kind_order(int kind)
{
    return kind == GS_K_POLY1 ? 1 : (kind == GS_K_POLY2 ? 2 : (kind == GS_K_POLY3 ? 3 : 0));
}

__host__ __device__ inline float poly_eval(const float c[4], int order, float x)
{
    float p = c[order];
    for (int i = order - 1; i >= 0; --i) p = fmaf(p, x, c[i]);
    return p;
}

__host__ __device__ inline float poly_deriv_eval(const float c[4], int order, float x)
{
    float p = order * c[order];
    for (int i = order - 1; i >= 1; --i) p = fmaf(p, x, i * c[i]);
    return p;
}

// Smallest real root x > 0 of sum c_i x^i = rhs (App. B; Eq. 4 for order 1),
// +inf if none. FP32: quadratic formula in its cancellation-free form;
// Cardano for the cubic (real branch, the sign of the inner root chosen to
// avoid cancellation) or the trigonometric form when it has three real
// roots; then two Newton steps on sum c_i x^i - rhs.
__host__ __device__ inline float first_root_f32(const float c[4], int order, float rhs)
{
    const float INF = INFINITY;
    float c0 = c[0] - rhs;
    float x = INF;
    if (order == 1) {
        if (c[1] != 0.f) x = -c0 / c[1];
        return x > 0.f ? x : INF;
    }
    if (order == 2) {
        float a = c[2], b = c[1];
        if (a == 0.f) {
            if (b != 0.f) x = -c0 / b;
            return x > 0.f ? x : INF;
        }
        float disc = fmaf(b, b, -4.f * a * c0);
        if (disc < 0.f && -disc <= 1e-5f * (b * b + fabsf(4.f * a * c0))) disc = 0.f;
        if (disc < 0.f) return INF;
        float s = sqrtf(disc);
        // roots q / a and c0 / q with q = -(b + sign(b) s) / 2
        float q = -0.5f * (b + (b >= 0.f ? s : -s));
        float r1 = (q != 0.f) ? q / a : INF;
        float r2 = (q != 0.f) ? c0 / q : INF;
        float best = INF;
        if (r1 > 0.f && r1 < best) best = r1;
        if (r2 > 0.f && r2 < best) best = r2;
        x = best;
    } else if (order == 3) {
        float c1 = c[1], c2 = c[2], c3 = c[3];
        float D0 = c2 * c2 - 3.f * c3 * c1;
        float D1 = 2.f * c2 * c2 * c2 - 9.f * c3 * c2 * c1 + 27.f * c3 * c3 * c0;
        float disc = D1 * D1 - 4.f * D0 * D0 * D0;
        if (disc >= 0.f) {
            float s = sqrtf(disc);
            float inner = 0.5f * (D1 >= 0.f ? D1 + s : D1 - s);
            float C = cbrtf(inner);
            x = (C == 0.f) ? -c2 / (3.f * c3) : -(c2 + C + D0 / C) / (3.f * c3);
            if (!(x > 0.f)) return INF;
        } else {
            float a = c2 / c3, b = c1 / c3, d = c0 / c3;
            float p = b - a * a / 3.f;
            float qq = 2.f * a * a * a / 27.f - a * b / 3.f + d;
            if (p >= 0.f) return INF;
            float m = 2.f * sqrtf(-p / 3.f);
            float arg = fminf(fmaxf(3.f * qq / (p * m), -1.f), 1.f);
            float th = acosf(arg) / 3.f;
            float best = INF;
            for (int k = 0; k < 3; ++k) {
                float r = m * cosf(th - 2.0943951023931957f * k) - a / 3.f;
                if (r > 0.f && r < best) best = r;
            }
            x = best;
        }
    } else {
        return INF;
    }
    if (!(x < INF)) return INF;
    for (int it = 0; it < 2; ++it) {
        float f = poly_eval(c, order, x) - rhs;
        float d = poly_deriv_eval(c, order, x);
        if (d != 0.f) x -= f / d;
    }
    return x > 0.f ? x : INF;
}

// Tile columns [c0, c1] (within [cx0, cx1]) of tile row `ty` that hold a
// pixel centre inside the ellipse A dx^2 + 2 B dx dy + C dy^2 <= xc around
// (mx, my); false if none. Over the row's band of pixel-centre y values the
// ellipse's x-extent is reached either at its own extreme points (dy =
// +-Sxy sqrt(xc / Sxx), Sigma = conic^-1) or at a band edge; the pixel
// columns whose centres fall inside it are mapped to tiles. Preprocessing
// (to count) and emission (to write) call this with the same stored record
// values, so both see the same set.
__device__ __forceinline__ bool row_cols(float mx, float my, float A, float B, float C, float xc,
                                         int ty, int tile_w, int tile_h, int W, int H, int cx0,
                                         int cx1, int &c0, int &c1)
{
    const float det = A * C - B * B;
    if (!(det > 0.f) || !(A > 0.f) || !(xc >= 0.f)) return false;
    const float idet = 1.f / det;
    const float Sxx = C * idet, Syy = A * idet, Sxy = -B * idet;
    const float hy = sqrtf(xc * Syy);
    const float ya = fmaxf(ty * tile_h + 0.5f, my - hy);
    const float yb = fminf((float)min((ty + 1) * tile_h, H) - 0.5f, my + hy);
    if (!(ya <= yb)) return false;
    const float hx = sqrtf(xc * Sxx);
    const float dys = Sxy * sqrtf(xc / Sxx);
    const float dya = ya - my, dyb = yb - my;
    const float iA = 1.f / A;
    const float wa = sqrtf(fmaxf(A * xc - det * dya * dya, 0.f)) * iA;
    const float wb = sqrtf(fmaxf(A * xc - det * dyb * dyb, 0.f)) * iA;
    const float ca = -B * dya * iA, cb = -B * dyb * iA;
    const float xmax = (dys >= dya && dys <= dyb) ? mx + hx : mx + fmaxf(ca + wa, cb + wb);
    const float xmin = (-dys >= dya && -dys <= dyb) ? mx - hx : mx + fminf(ca - wa, cb - wb);
    const float p0 = fmaxf(ceilf(xmin - 0.5f), 0.f), p1 = fminf(floorf(xmax - 0.5f), (float)(W - 1));
    if (!(p0 <= p1)) return false;
    // p0, p1 >= 0 and tile sizes are powers of two: a shift divides
    c0 = max((int)p0 >> (__ffs(tile_w) - 1), cx0);
    c1 = min((int)p1 >> (__ffs(tile_w) - 1), cx1);
    return c0 <= c1;
}

} // namespace gs

#define GS_LAUNCH_CHECK()                                        \
    do {                                                         \
        if (cudaPeekAtLastError() != cudaSuccess) {              \
            cudaGetLastError();                                  \
            return GS_ERR_CUDA;                                  \
        }                                                        \
    } while (0)
