// capi.cu — host-side helpers of the C ABI: config defaults, camera and
// config tables for the kernels, launch accounting, status strings.
#include <atomic>
#include <cmath>

#include "gs_common.cuh"

namespace gs {

static std::atomic<uint64_t> g_launches{0};

void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static bool valid_tile(const gs_config *cfg)
{
    const int w = cfg->tile_w, h = cfg->tile_h;
    return (w == 8 || w == 16 || w == 32) && (h == 8 || h == 16 || h == 32) && w * h <= 512;
}

// A-priori bound on the rounding error of the FP16x2 alpha of render.cu
// (alpha_pair_h2) against the FP32 alpha, per unit opacity and divided by c0,
// i.e. as a multiple of p0 = o' c0, over Q in [0, x0]. binary16 has unit
// roundoff u = 2^-11. The FP32 u and v^2 are rounded to half (u^2 then carries
// 2u, v^2 u) and Q = u^2 + v^2 is one fused op (u more): |dQ| <= 3.01 u Q.
// Horner (f1, f'2): each fused step s_k = s_{k+1} Q + p_k adds at most
// u (|s_{k+1} Q| + |s_k|), the half coefficients u sum |p_i| Q^i, and dQ adds
// |f'(Q)| dQ. Factored cubic: the same accounting through t1 = p3 (Q - r),
// s = Q + f3b, q2 = s Q + f3g and alpha = t1 q2. The blend widens it by 25 %.
static float half_alpha_bound(const CfgDev &d, int n)
{
    const float u = 1.f / 2048.f;
    const float *c = d.c;
    float worst = 0.f;
    for (int i = 0; i <= 256; ++i) {
        const float Q = d.x0 * (float)i / 256.f, dQ = 3.01f * u * Q;
        float e;
        if (n == 3 && d.f3_factored) {
            const float t1 = c[3] * (Q - d.f3r);
            const float dt1 = fabsf(c[3]) * dQ + u * (fabsf(c[3] * Q) + fabsf(c[3] * d.f3r) + fabsf(t1));
            const float sq = Q + d.f3b, dsq = dQ + u * (fabsf(d.f3b) + fabsf(sq));
            const float q2 = fmaf(sq, Q, d.f3g);
            const float dq2 = Q * dsq + fabsf(sq) * dQ + u * (fabsf(d.f3g) + fabsf(q2));
            e = fabsf(q2) * dt1 + fabsf(t1) * dq2 + u * fabsf(t1 * q2);
        } else {
            float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            for (int k = n; k >= 0; --k) s[k] = fmaf(Q, s[k + 1], c[k]);
            e = 0.f;
            for (int k = n - 1; k >= 0; --k) e += fabsf(s[k + 1] * Q) + fabsf(s[k]);
            float qi = 1.f;
            for (int k = 0; k <= n; ++k, qi *= Q) e += fabsf(c[k]) * qi;
            e = e * u + fabsf(poly_deriv_eval(c, n, Q)) * dQ;
        }
        worst = fmaxf(worst, e);
    }
    return 1.25f * worst / c[0];
}

bool build_cfg(const gs_config *cfg, CfgDev *d)
{
    if (!cfg) return false;
    if (cfg->kind < GS_K_EXP || cfg->kind > GS_K_POLY3) return false;
    if (cfg->cull < GS_CULL_UNIVERSAL || cfg->cull > GS_CULL_LEGACY3) return false;
    if (!(cfg->eps > 0.f && cfg->eps < 1.f)) return false;
    if (!(cfg->alpha_max > 0.f && cfg->alpha_max < 1.f)) return false;
    if (!(cfg->t_min > 0.f && cfg->t_min < 1.f)) return false;
    if (!(cfg->aa_dilation >= 0.f) || !std::isfinite(cfg->aa_dilation)) return false;
    if (!valid_tile(cfg)) return false;
    if (cfg->rect_mode != GS_RECT_AABB && cfg->rect_mode != GS_RECT_CIRCLE &&
        cfg->rect_mode != GS_RECT_ELLIPSE)
        return false;
    for (int i = 0; i < 4; ++i)
        if (!std::isfinite(cfg->c[i])) return false;
    d->kind = cfg->kind;
    for (int i = 0; i < 4; ++i) d->c[i] = cfg->c[i];
    d->cull = cfg->cull;
    d->eps = cfg->eps;
    d->alpha_max = cfg->alpha_max;
    d->t_min = cfg->t_min;
    d->aa = cfg->aa_normalize ? 1 : 0;
    d->dil = cfg->aa_dilation;
    d->tile_w = cfg->tile_w;
    d->tile_h = cfg->tile_h;
    d->rect_mode = cfg->rect_mode;
    d->batch = cfg->batch;
    d->ppt = cfg->px_per_thread;
    const int n = kind_order(cfg->kind);
    d->x0 = n ? first_root_f32(cfg->c, n, 0.f) : INFINITY;
    if (n) {
        // the polynomial must start positive and reach zero (Sec. 3.2)
        if (!(cfg->c[0] > 0.f) || !(d->x0 < INFINITY)) return false;
    }
    // Is k non-increasing on [0, x0]? (exp always; f1 iff c1 < 0; the
    // others are checked on a grid.) The blend may then skip an entry for a
    // whole pixel run from a lower bound of Q.
    d->monotone = 1;
    if (n == 1) d->monotone = cfg->c[1] < 0.f;
    if (n >= 2)
        for (int i = 0; i <= 1024; ++i)
            if (poly_deriv_eval(cfg->c, n, d->x0 * i / 1024.f) > 1e-6f) d->monotone = 0;
    // the cubic divided by (Q - x0): c3 (Q - x0)(Q^2 + f3b Q + f3g)
    d->f3r = d->f3b = d->f3g = 0.f;
    d->f3_factored = 0;
    d->tail_zero = 0;
    if (n == 3 && cfg->c[3] != 0.f) {
        d->f3r = d->x0;
        d->f3b = cfg->c[2] / cfg->c[3] + d->x0;
        d->f3g = cfg->c[1] / cfg->c[3] + d->x0 * d->f3b;
        // past x0, (Q - x0) > 0, so the cubic stays <= 0 there when c3 < 0
        // and the quadratic factor has no real root beyond x0 (in double, with
        // a margin: only then may the blend skip an entry from Q > x0 alone)
        const double b = d->f3b, g = d->f3g, disc = b * b - 4.0 * g;
        d->tail_zero = cfg->c[3] < 0.f &&
                       (disc < 0.0 || (-b + std::sqrt(disc)) / 2.0 < (double)d->x0 * (1.0 - 1e-3));
        // the half form needs the factors inside binary16 range
        d->f3_factored = std::isfinite(d->f3b) && std::isfinite(d->f3g) && fabsf(d->f3b) < 3e4f &&
                         fabsf(d->f3g) < 3e4f && fabsf(d->c[3] * d->x0) < 3e4f;
    }
    // exp: the half exponent p0 + p1 Q (|p0|, |p1 Q| <= -log2 eps ~ 8 where
    // alpha >= eps/4) has error ~48 u, 1.6 % of alpha after ex2, plus ex2's own
    // approximation and rounding; 3 % bounds both
    d->h2_band = n ? half_alpha_bound(*d, n) : 0.03f;
    return true;
}

bool build_cam_table(const gs_camera *cams, int ncam, const gs_config *cfg, CamTable *t)
{
    if (!cams || !cfg || ncam <= 0 || ncam > kMaxCams || !valid_tile(cfg)) return false;
    t->ncam = ncam;
    int64_t tiles = 0, pix = 0;
    for (int c = 0; c < ncam; ++c) {
        const gs_camera &g = cams[c];
        CamDev &d = t->cam[c];
        if (g.width <= 0 || g.height <= 0 || g.width > 16384 || g.height > 16384) return false;
        if (!(g.fx > 0.f) || !(g.fy > 0.f) || !(g.znear > 0.f)) return false;
        if (!std::isfinite(g.cx) || !std::isfinite(g.cy)) return false;
        for (int i = 0; i < 16; ++i)
            if (!std::isfinite(g.viewmat[i])) return false;
        for (int r = 0; r < 3; ++r) {
            for (int k = 0; k < 3; ++k) d.R[3 * r + k] = g.viewmat[4 * r + k];
            d.T[r] = g.viewmat[4 * r + 3];
        }
        for (int k = 0; k < 3; ++k)
            d.campos[k] = -(d.R[k] * d.T[0] + d.R[3 + k] * d.T[1] + d.R[6 + k] * d.T[2]);
        d.fx = g.fx; d.fy = g.fy; d.cx = g.cx; d.cy = g.cy;
        d.limx = 1.3f * (0.5f * g.width / g.fx);
        d.limy = 1.3f * (0.5f * g.height / g.fy);
        d.znear = g.znear;
        d.W = g.width; d.H = g.height;
        d.tiles_x = (g.width + cfg->tile_w - 1) / cfg->tile_w;
        d.tiles_y = (g.height + cfg->tile_h - 1) / cfg->tile_h;
        d.tile_base = (int)tiles;
        d.pix_base = pix;
        tiles += (int64_t)d.tiles_x * d.tiles_y;
        pix += (int64_t)g.width * g.height;
        if (tiles >= ((int64_t)1 << 30)) return false;
    }
    for (int c = ncam; c < kMaxCams; ++c) t->cam[c] = CamDev{};
    t->total_tiles = (int)tiles;
    return true;
}

} // namespace gs

using namespace gs;

// Frozen kernel coefficients. f1: Sec. 3.1 (printed c0/c1 labels swapped; c1
// set so that the root is the printed 4.386). f'2 (tangent parabola, the L1
// optimum of Eq. 6) and f3: L1 fits by the Sec. 3.1 procedure.
static const float kPoly1[4] = {0.773f, -0.17624259005927953f, 0.f, 0.f};
static const float kPoly2[4] = {0.8516280240144332f, -0.26733264653820527f, 0.020979448153971795f, 0.f};
static const float kPoly3[4] = {0.9553403177961989f, -0.40208845109000624f, 0.06272449941115653f,
                                -0.0034515811299093797f};

extern "C" gs_status gs_config_default(int32_t kind, int32_t cull, gs_config *cfg)
{
    if (!cfg || kind < GS_K_EXP || kind > GS_K_POLY3 || cull < 0 || cull > 2) return GS_ERR_ARG;
    gs_config c = {};
    c.kind = kind;
    const float *src = kind == GS_K_POLY1 ? kPoly1 : kind == GS_K_POLY2 ? kPoly2 : kind == GS_K_POLY3 ? kPoly3 : nullptr;
    for (int i = 0; i < 4; ++i) c.c[i] = src ? src[i] : 0.f;
    c.cull = cull;
    c.eps = 1.f / 255.f;
    c.alpha_max = 0.99f;
    c.t_min = 1e-4f;
    c.aa_normalize = 1;
    c.aa_dilation = 0.3f;
    c.tile_w = 16;
    c.tile_h = 16;
    c.rect_mode = GS_RECT_AABB;
    c.batch = 256;
    c.px_per_thread = 4; // fastest on B300 for f1 and exp at 16x16 (3M splats, 1080p)
    c.fp16x2 = 0;
    *cfg = c;
    return GS_OK;
}

extern "C" int64_t gs_total_tiles(const gs_camera *cams, int32_t ncam, const gs_config *cfg)
{
    CamTable t;
    if (!build_cam_table(cams, ncam, cfg, &t)) return -1;
    return t.total_tiles;
}

extern "C" uint64_t gs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" const char *gs_status_string(int32_t status)
{
    switch (status) {
    case GS_OK: return "ok";
    case GS_ERR_ARG: return "invalid argument";
    case GS_ERR_CUDA: return "CUDA error";
    case GS_ERR_CAPACITY: return "overlap capacity exceeded";
    case GS_ERR_TIMEOUT: return "bounded wait timed out";
    case GS_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "multiple errors";
    }
}
