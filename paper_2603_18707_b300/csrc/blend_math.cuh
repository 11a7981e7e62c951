// blend_math.cuh — per-(splat, tile) coefficients and the alpha evaluation
// shared by the forward blend and its reverse pass, so that both take every
// skip / clamp / stop decision with bit-identical arithmetic.
//
// The quadric of Eq. 1, Q = A dx^2 + 2 B dx dy + C dy^2 (dx, dy: pixel centre
// minus mu'), is rewritten once per staged entry as a sum of two squares of
// affine functions of the tile-local pixel coordinates (x, y):
//   u = ux x + uy y + u0,  v = vy y + v0,  Q = u^2 + v^2,
//   ux = sqrt(A), uy = B / sqrt(A), vy = sqrt((A C - B^2) / A)
// (completing the square; A > 0 for the inverse of a covariance). A thread
// then needs 2 FMAs per row and 2 per pixel for Q. Opacity is folded into the
// kernel coefficients: o' f(Q) = p0 + p1 Q + p2 Q^2 + p3 Q^3 with p_i = o' c_i,
// and o' exp(-Q/2) = 2^(p0 + p1 Q) with p0 = log2 o', p1 = -log2(e)/2.
#pragma once

#include "gs_common.cuh"

namespace gs {

// Arguments of the forward blend kernels (render.cu, render_tc5.cu).
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

// The tensor-core quadric on tcgen05 (render_tc5.cu): one CTA per 16x16 tile.
cudaError_t launch_render_tc5(int kind, cudaStream_t s, const CamTable &t, const CfgDev &c, const RenderArgs &g);
// Self-test of its bounded mbarrier wait: a wait that no arrival completes
// gives up after `limit` polls and ORs GS_ERR_TIMEOUT into *err.
cudaError_t launch_tc5_wait_selftest(cudaStream_t s, uint32_t *err, int limit);

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct BlendCoef {
    float4 a; // ux, uy, u0, vy
    float4 b; // v0, p0, p1, p2 (f1, exp: x_cut)
    float4 c; // red, green, blue, p3
};

// f1 and exp in the FP32 blend: their Q coefficient p1 is negative, and
// sigma = sqrt(-p1) is folded into the two affine forms (s = sigma u,
// t = sigma v), so that p0 + p1 Q = beta - s^2 with beta = p0 - t^2 per row:
// two FMAs per pixel for the exponent / the alpha (FOLD below).
template <int KIND>
constexpr bool folds_p1()
{
    return KIND == GS_K_POLY1 || KIND == GS_K_EXP;
}

// rec0 = (mu'x, mu'y, o', depth), rec1 = (A, B, C, x_cut), rec2 = (r, g, b, rho);
// (ox, oy): pixel coordinates of the tile's corner. FOLD: a and b.x carry
// sigma (f1, exp only).
template <int KIND, bool FOLD = false>
__device__ __forceinline__ BlendCoef make_coef(const CfgDev &cfg, float4 r0, float4 r1, float4 r2,
                                               float ox, float oy)
{
    const float mx = r0.x - ox, my = r0.y - oy, o = r0.z;
    const float A = r1.x, B = r1.y, C = r1.z;
    const float sA = sqrtf(A);
    const float ux = sA, uy = B / sA;
    const float vy = sqrtf(fmaxf(C - B * uy / sA, 0.f));
    BlendCoef k;
    k.a = make_float4(ux, uy, -fmaf(ux, mx, uy * my), vy);
    float p0, p1, p2 = 0.f, p3 = 0.f;
    if (KIND == GS_K_EXP) {
        p0 = log2f(o);
        p1 = -0.72134752044448170f; // -log2(e) / 2
    } else {
        p0 = o * cfg.c[0];
        p1 = o * cfg.c[1];
        p2 = o * cfg.c[2];
        p3 = o * cfg.c[3];
    }
    // f1 and exp evaluate alpha from p0, p1 alone; their p2 slot carries
    // the record's cut x_cut instead (Eq. 3-5, with the preprocessing's
    // margin): where a lower bound of Q exceeds it, no pixel reaches eps.
    // The legacy 3-sigma cut does not bound the eps support, so it never
    // skips.
    if (KIND == GS_K_POLY1 || KIND == GS_K_EXP) p2 = (cfg.cull == GS_CULL_LEGACY3) ? INFINITY : r1.w;
    // f'2 has no cubic term: its p3 slot carries the cut instead
    if (KIND == GS_K_POLY2) p3 = (cfg.cull == GS_CULL_LEGACY3) ? INFINITY : r1.w;
    k.b = make_float4(-vy * my, p0, p1, p2);
    k.c = make_float4(r2.x, r2.y, r2.z, p3);
    if constexpr (FOLD) {
        static_assert(folds_p1<KIND>(), "only f1 and exp fold their Q coefficient");
        // sqrt(log2(e) / 2) for exp; f1's c1 < 0 (its root is finite and positive)
        const float sg = (KIND == GS_K_EXP) ? 0.84932180028801904f : sqrtf(-p1);
        k.a = make_float4(sg * k.a.x, sg * k.a.y, sg * k.a.z, sg * k.a.w);
        k.b.x *= sg;
    }
    return k;
}

// FOLD form: o' k(Q) before the alpha_max clamp, from beta = p0 - t^2 and s.
template <int KIND>
__device__ __forceinline__ float alpha_folded(float beta, float s)
{
    const float e = fmaf(-s, s, beta);
    if (KIND == GS_K_EXP) return ex2_approx(e);
    return e;
}


// o' k(Q) before the alpha_max clamp.
template <int KIND>
__device__ __forceinline__ float alpha_of_q(const CfgDev &cfg, const float4 &b, float p3, float Q)
{
    if (KIND == GS_K_EXP) return ex2_approx(fmaf(b.z, Q, b.y));
    if (KIND == GS_K_POLY1) return fmaf(b.z, Q, b.y);
    if (KIND == GS_K_POLY2) return Q < cfg.x0 ? fmaf(fmaf(b.w, Q, b.z), Q, b.y) : 0.f;
    return fmaf(fmaf(fmaf(p3, Q, b.w), Q, b.z), Q, b.y);
}

// dk/dQ of the kernel (without the opacity), for the reverse pass.
template <int KIND>
__device__ __forceinline__ float kernel_slope(const CfgDev &cfg, float Q, float alpha_raw, float o)
{
    if (KIND == GS_K_EXP) return -0.5f * alpha_raw / o;
    if (KIND == GS_K_POLY1) return cfg.c[1];
    if (KIND == GS_K_POLY2) return fmaf(2.f * cfg.c[2], Q, cfg.c[1]);
    return fmaf(fmaf(3.f * cfg.c[3], Q, 2.f * cfg.c[2]), Q, cfg.c[1]);
}

} // namespace gs
