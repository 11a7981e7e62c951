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
// Cost per entry and thread: 2 LDS.128 (f1, exp: 3 per entry pair, tested as
// a pair) and a skip test on a lower bound of Q over the run; where reached,
// pixel pairs update with packed FP32x2 FMAs (decisions scalar; exp adds one
// MUFU ex2 per pixel). Entries go in unrolled groups; a block leaves a list
// once every pixel has stopped. Bound by FP32 / ALU instruction issue.
//
// Launch modes: one CTA per tile (grid = all tiles of all cameras), or
// persistent: a grid sized to fill every SM once, each CTA taking the next
// tile from an atomic counter until all tiles of all cameras are done (one
// launch for any mix of resolutions, balanced dynamically).
#include <algorithm>
#include <type_traits>

#include <cuda_fp16.h>

#include "blend_math.cuh"

namespace gs {
namespace {

constexpr int kMaxBatch = 256;
// FP32 blend on packed FP32x2 pixel pairs (see render_tile).
#ifndef GS_BLEND_PAIRS
#define GS_BLEND_PAIRS 1 // f1 / exp: skip tests of entry pairs on FP32x2 pairs
#endif
#ifndef GS_BLEND_PACKED
#define GS_BLEND_PACKED 1
#endif
// Unroll of the per-entry loop (ILP across entries): measured fastest at 8
// for the packed blend of every kernel and for exp, 4 for the scalar
// polynomial blends (0: per kind as measured).
#ifndef GS_BLEND_UNROLL
#define GS_BLEND_UNROLL 0
#endif
template <int KIND>
constexpr int blend_unroll()
{
    return GS_BLEND_UNROLL ? GS_BLEND_UNROLL : (KIND == GS_K_EXP || GS_BLEND_PACKED ? 8 : 4);
}
#ifndef GS_SKIP_MID
#define GS_SKIP_MID 1 // per-thread skip bound from the run's centre (1) or its two ends (0)
#endif
#ifndef GS_PERSIST_CAP
#define GS_PERSIST_CAP 0 // persistent blend: CTAs per SM at most (0: as many as fit)
#endif
#ifndef GS_RENDER_MIN_BLOCKS
#define GS_RENDER_MIN_BLOCKS 4 // 256-thread CTAs per SM the register budget must allow (64 registers: measured fastest)
#endif
// Per-pixel update: predicated (no branch per pixel) or branching. 0: branch
// for every kernel, 1: predicate for every kernel, 2: predicate for exp only.
// Measured with the folded alpha (one-stream 16-camera pass): branching for
// every kernel, f1 8.07 ms / exp 10.95 ms; predicated exp 11.24 ms;
// predicated f1 8.34 ms.
#ifndef GS_BLEND_BRANCHLESS
#define GS_BLEND_BRANCHLESS 0
#endif
template <int KIND>
constexpr bool blend_branchless()
{
    return GS_BLEND_BRANCHLESS == 1 || (GS_BLEND_BRANCHLESS == 2 && KIND == GS_K_EXP);
}

// FP16x2 alpha of a pixel pair (u_a, u_b computed in FP32, sharing v^2):
// Q = u^2 + v^2 and the opacity-folded kernel in packed half2 FMAs, before
// the alpha_max clamp (which the caller applies in FP32: 0.99 is not a half).
// Q is clamped to the cut x0 before f'2's polynomial so that an overflowing
// Q (a far-away splat) gives 0 rather than inf * 0. The cubic is evaluated
// factored at its support root r, p3 (Q - r)(Q^2 + b Q + g), whose rounding
// error stays near that of f1 (Horner's intermediates reach ~1.6 and cost
// about twice as much); hp then holds (p3, -p3 r). The rounding error of the
// result is bounded on the host (CfgDev::h2_band).
template <int KIND>
__device__ __forceinline__ float2 alpha_pair_h2(float ua, float ub, __half2 v2h, uint4 hp, __half2 x0h,
                                                __half2 f3bh, __half2 f3gh, bool factored)
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
    } else if (factored) {
        al = __hmul2(__hfma2(p0, Q, p1), __hfma2(__hadd2(Q, f3bh), Q, f3gh));
    } else {
        al = __hfma2(__hfma2(__hfma2(p3, Q, p2), Q, p1), Q, p0);
    }
    return __half22float2(al);
}

// TRACK: keep each pixel's last contributor and evaluation count (only when
// the caller asks for d_last or d_n_eval: the reverse pass and the
// evaluation count need them, the image does not)
// Compaction of the still-active pixel runs between batches (GS_BLEND_COMPACT):
// per entry only about a sixth of a tile's pixels are still evaluated on the
// benchmark scene (most have stopped, T < t_min), yet a warp walks the list
// while any of its lanes holds an active run. When the active runs of a tile
// fit in fewer warps than hold runs, the runs whose pixels have all stopped
// write their pixels, the active runs move (through the batch's shared
// staging buffer, free between batches) into the lowest threads, and the
// warps left without a run skip the entries of every later batch. The
// arithmetic per pixel and its order are unchanged: images are bit-identical.
#ifndef GS_BLEND_COMPACT
#define GS_BLEND_COMPACT 1
#endif

template <int KIND, int PPT, bool HALF, bool TRACK>
__device__ __forceinline__ void render_tile(const CamTable &cams, const CfgDev &cfg, const RenderArgs &g,
                                            int gtile, float4 *s_a, float4 *s_b, float4 *s_c, uint4 *s_h,
                                            float *s_x, uint32_t *s_wc)
{
    int c = 0;
    while (c + 1 < cams.ncam && cams.cam[c + 1].tile_base <= gtile) ++c;
    const CamDev &cm = cams.cam[c];
    const int lt = gtile - cm.tile_base;
    const int tx = lt % cm.tiles_x, ty = lt / cm.tiles_x;
    const int tpr = cfg.tile_w / PPT; // threads per tile row
    // this thread's run of PPT pixels (tile-local first column and row); it
    // can change at a compaction
    int lx = ((int)threadIdx.x % tpr) * PPT, ly = (int)threadIdx.x / tpr;
    const float ox = (float)(tx * cfg.tile_w), oy = (float)(ty * cfg.tile_h);
    int px0 = tx * cfg.tile_w + lx, py = ty * cfg.tile_h + ly;
    float y = ly + 0.5f;
    float xmid = lx + 0.5f * PPT; // centre of the thread's run of pixel centres
    bool own = true;                // this thread holds a run whose pixels it writes
    const uint2 rg = g.ranges[gtile];
    // an empty or inverted range (only possible after a timed-out sort wait)
    // reads nothing: every range gs_bin_sort writes lies within its output
    const uint32_t n = rg.y > rg.x ? rg.y - rg.x : 0u;
    const int nthreads = blockDim.x;
    const int B = cfg.batch;

    const float eps = cfg.eps, amax = cfg.alpha_max, tmin = cfg.t_min;
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
        // a pixel that is off the frame or has stopped gets x = NaN: its Q
        // and alpha are NaN (in FP32 and in half) and fail every alpha
        // compare, so no per-pixel mask test is needed
        if (!(active >> k & 1u)) xs[k] = NAN;
    }
    const __half2 x0h = __float2half2_rn(fminf(cfg.x0, 60000.f));
    const __half2 f3bh = __float2half2_rn(cfg.f3b), f3gh = __float2half2_rn(cfg.f3g);
    const bool factored = KIND == GS_K_POLY3 && cfg.f3_factored;
    // FP32 f1 / exp: sigma folded into the affine forms (blend_math.cuh), so
    // the row term v2 below is beta = p0 - t^2 and the pixel's exponent /
    // alpha is beta - s^2
    constexpr bool FOLD = !HALF && folds_p1<KIND>();
    // packed pixel pairs (GS_BLEND_PACKED): the FP32 blend updates two
    // pixels per FP32x2 instruction, with the signs of the colours (and for
    // f1 / exp of beta and the exponent, NEGB) flipped so that no operand
    // needs a negation (the results are bit-identical to the scalar update)
    constexpr bool PACKED = GS_BLEND_PACKED && !HALF && PPT % 2 == 0;
    constexpr bool NEGB = PACKED && FOLD;
    // f1 / exp packed: entries staged as pairs (2m, 2m + 1), field by field,
    // so that the skip tests of both run on FP32x2 pairs too: s_a[m] = (ux,
    // uy) of both, s_a[kMaxBatch / 2 + m] = (u0, vy), s_b[m] = (v0, -p0)
    constexpr bool PAIRS = GS_BLEND_PAIRS && GS_SKIP_MID && NEGB;
    // f1's alpha never exceeds its entry's p0 = o' c0 (beta - s^2 <= beta <=
    // p0, also as rounded), so a batch whose entries all have p0 <= alpha_max
    // is walked without the clamp (for the paper's f1, c0 = 0.773: always)
    constexpr bool NOCLAMP_OK = PACKED && KIND == GS_K_POLY1;
    // skip threshold of the folded per-run test: 2^-8 below eps (exp: its
    // exponent), far more than the rounding of the run's bound on |s|
    const float fold_skip = KIND == GS_K_EXP ? log2f(eps * (1.f - 1.f / 256.f)) : eps * (1.f - 1.f / 256.f);
    // skip threshold of the per-run test: just below eps, so that rounding
    // never skips an entry a pixel takes (the FP16x2 path takes the FP32
    // path's decisions, so the same test serves both)
    const float eps_skip = eps * (1.f - 1.f / 1024.f);
    // the run's pixels to the outputs
    auto write_run = [&]() {
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            if (px0 + k < cm.W && py < cm.H) {
                const int64_t pix = cm.pix_base + (int64_t)py * cm.W + px0 + k;
                g.out[3 * pix + 0] = fmaf(T[k], g.bg0, C0[k]);
                g.out[3 * pix + 1] = fmaf(T[k], g.bg1, C1[k]);
                g.out[3 * pix + 2] = fmaf(T[k], g.bg2, C2[k]);
                if (g.final_T) g.final_T[pix] = T[k];
                if (TRACK && g.last) g.last[pix] = lastc[k];
                if (TRACK && g.n_eval) g.n_eval[pix] = ne[k];
            }
        }
    };
    // words of a run in the exchange: position, active bits, T and colour
    // per pixel (+ last contributor and evaluation count)
    constexpr int XW = 2 + 4 * PPT + (TRACK ? 2 * PPT : 0);
    const bool can_compact = GS_BLEND_COMPACT && XW * nthreads <= 3 * kMaxBatch * 4 && nthreads % 32 == 0;
    int alive = (nthreads + 31) >> 5; // warps that hold runs
    for (uint32_t base = 0; base < n; base += B) {
        const int nact = __syncthreads_count(active != 0);
        if (nact == 0) break;
        if (can_compact && ((nact + 31) >> 5) < alive) {
            // the batch's staging buffer is free: every thread has left the
            // previous batch (barrier above) and the next is not staged yet
            if (own && !active) {
                write_run();
                own = false;
            }
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            const unsigned bal = __ballot_sync(0xffffffffu, active != 0);
            if (lane == 0) s_wc[wid] = __popc(bal);
            __syncthreads();
            int rank = __popc(bal & ((1u << lane) - 1u));
            for (int w = 0; w < wid; ++w) rank += (int)s_wc[w];
            if (active) {
                float *d = s_x + rank;
                d[0] = __int_as_float(lx | (ly << 16));
                d[nthreads] = __uint_as_float(active);
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    d[(2 + 4 * k) * nthreads] = T[k];
                    d[(3 + 4 * k) * nthreads] = C0[k];
                    d[(4 + 4 * k) * nthreads] = C1[k];
                    d[(5 + 4 * k) * nthreads] = C2[k];
                    if (TRACK) {
                        d[(2 + 4 * PPT + 2 * k) * nthreads] = __uint_as_float(lastc[k]);
                        d[(3 + 4 * PPT + 2 * k) * nthreads] = __uint_as_float(ne[k]);
                    }
                }
            }
            __syncthreads();
            own = (int)threadIdx.x < nact;
            active = 0;
            if (own) {
                const float *d = s_x + threadIdx.x;
                const int pos = __float_as_int(d[0]);
                lx = pos & 0xffff;
                ly = pos >> 16;
                active = __float_as_uint(d[nthreads]);
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    T[k] = d[(2 + 4 * k) * nthreads];
                    C0[k] = d[(3 + 4 * k) * nthreads];
                    C1[k] = d[(4 + 4 * k) * nthreads];
                    C2[k] = d[(5 + 4 * k) * nthreads];
                    if (TRACK) {
                        lastc[k] = __float_as_uint(d[(2 + 4 * PPT + 2 * k) * nthreads]);
                        ne[k] = __float_as_uint(d[(3 + 4 * PPT + 2 * k) * nthreads]);
                    }
                }
                px0 = tx * cfg.tile_w + lx;
                py = ty * cfg.tile_h + ly;
                y = ly + 0.5f;
                xmid = lx + 0.5f * PPT;
            }
#pragma unroll
            for (int k = 0; k < PPT; ++k) xs[k] = (active >> k & 1u) ? lx + k + 0.5f : NAN;
            alive = (nact + 31) >> 5;
            __syncthreads(); // the exchange is read before the batch is staged over it
        }
        bool big = false; // a staged f1 entry with p0 > alpha_max
        const int cnt = (int)min((uint32_t)B, n - base);
        if (PAIRS && (cnt & 1) && threadIdx.x == 0) {
            // an odd count's last pair gets a second entry that every run skips
            float *q0 = reinterpret_cast<float *>(s_a + (cnt >> 1));
            float *q1 = reinterpret_cast<float *>(s_a + kMaxBatch / 2 + (cnt >> 1));
            float *q2 = reinterpret_cast<float *>(s_b + (cnt >> 1));
            q0[1] = q0[3] = q1[1] = q1[3] = q2[1] = 0.f;
            q2[3] = INFINITY; // -beta = +inf: the run's bound never reaches eps
        }
        for (int i = threadIdx.x; i < B; i += nthreads) {
            if (base + i < n) {
                uint32_t v = g.vals[rg.x + base + i];
                if (v >= g.n_records) v = 0; // only after a timed-out sort wait
                const BlendCoef k = make_coef<KIND, FOLD>(cfg, g.rec[3 * (size_t)v + 0],
                                                          g.rec[3 * (size_t)v + 1], g.rec[3 * (size_t)v + 2], ox, oy);
                if constexpr (PAIRS) {
                    const int h = i & 1;
                    float *q0 = reinterpret_cast<float *>(s_a + (i >> 1));
                    float *q1 = reinterpret_cast<float *>(s_a + kMaxBatch / 2 + (i >> 1));
                    float *q2 = reinterpret_cast<float *>(s_b + (i >> 1));
                    q0[h] = k.a.x;
                    q0[2 + h] = k.a.y;
                    q1[h] = k.a.z;
                    q1[2 + h] = k.a.w;
                    q2[h] = k.b.x;
                    q2[2 + h] = -k.b.y;
                } else {
                    s_a[i] = k.a;
                    s_b[i] = k.b;
                }
                s_c[i] = PACKED ? make_float4(-k.c.x, -k.c.y, -k.c.z, k.c.w) : k.c;
                if (NOCLAMP_OK) big |= k.b.y > amax;
                if (HALF) {
                    __half2 h[4] = {__float2half2_rn(k.b.y), __float2half2_rn(k.b.z),
                                    __float2half2_rn(k.b.w), __float2half2_rn(k.c.w)};
                    if (factored) {
                        h[0] = __float2half2_rn(k.c.w);
                        h[1] = __float2half2_rn(-k.c.w * cfg.f3r);
                    }
                    s_h[i] = *reinterpret_cast<const uint4 *>(h);
                }
            }
        }
        const int need_clamp = __syncthreads_or(big);
        // the walk over the batch, with or without the alpha_max clamp
        auto walk = [&](auto clamp_tag) {
        [[maybe_unused]] constexpr bool CLAMP = decltype(clamp_tag)::value;
        // the update of this thread's run by entry j (reached by its skip test)
        auto update = [&](const int j, const float4 &a, const float4 &b, const float ub, const float v2,
                          const float p3) {
            const float4 col = s_c[j];
            [[maybe_unused]] const uint32_t pos = base + j + 1;
            if constexpr (HALF) {
                // alphas in packed half, decisions in FP32: d bounds
                // |alpha(half) - alpha(FP32)| for this entry, so an alpha
                // further than d from eps is on the FP32 alpha's side of it;
                // within d (rare) the pixel's alpha is recomputed in FP32
                // (Q form, alpha_of_q), and so is it where T (1 - alpha) lies
                // within T d of t_min (the stop decision)
                const uint4 hp = s_h[j];
                const __half2 v2h = __float2half2_rn(v2);
                float al[PPT];
#pragma unroll
                for (int k = 0; k < PPT; k += 2) {
                    const float2 ap = alpha_pair_h2<KIND>(fmaf(a.x, xs[k], ub), fmaf(a.x, xs[k + 1], ub), v2h, hp,
                                                          x0h, f3bh, f3gh, factored);
                    al[k] = ap.x;
                    al[k + 1] = ap.y;
                }
                const float d = cfg.h2_band * (KIND == GS_K_EXP ? eps : b.y);
                const float lo = eps - d, hi = eps + d;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    float x = al[k];
                    if (!(x >= lo)) continue; // below eps for certain, or the pixel stopped (NaN)
                    if (x < hi) {
                        const float u = fmaf(a.x, xs[k], ub);
                        x = alpha_of_q<KIND>(cfg, b, p3, fmaf(u, u, v2));
                        if (!(x >= eps)) continue;
                    }
                    x = fminf(amax, x);
                    float Tn = fmaf(-x, T[k], T[k]);
                    if (Tn < fmaf(T[k], KIND == GS_K_EXP ? cfg.h2_band * x : d, tmin)) {
                        // (recomputing an alpha that is already FP32 gives the same value)
                        const float u = fmaf(a.x, xs[k], ub);
                        x = fminf(amax, alpha_of_q<KIND>(cfg, b, p3, fmaf(u, u, v2)));
                        Tn = fmaf(-x, T[k], T[k]);
                    }
                    if (Tn < tmin) {
                        active &= ~(1u << k);
                        xs[k] = NAN;
                        if constexpr (TRACK) ne[k] = pos;
                        continue;
                    }
                    const float w = x * T[k];
                    C0[k] = fmaf(col.x, w, C0[k]);
                    C1[k] = fmaf(col.y, w, C1[k]);
                    C2[k] = fmaf(col.z, w, C2[k]);
                    T[k] = Tn;
                    if constexpr (TRACK) lastc[k] = pos;
                }
            } else if constexpr (PACKED) {
                // per pixel pair: ne = u^2 - beta = -(exponent / alpha); na
                // = -min(alpha_max, alpha) where alpha >= eps, else 0 (a
                // skipped or stopped pixel then keeps T and its colour:
                // fma(0, T, T) = T); T' = T + na T; the colour gains
                // (-c)(na T) = c alpha T. Only a pixel that stops takes a
                // branch (T' < t_min is possible only where alpha >= eps).
                // f'2 / f3: Q = u^2 + v^2 and the polynomial's Horner steps
                // on pairs, then na = -min(alpha_max, alpha) where alpha >= eps
                const float2 ax2 = make_float2(a.x, a.x), ub2 = make_float2(ub, ub), nb2 = make_float2(v2, v2);
                float na[PPT], Tn[PPT];
                bool stop = false;
#pragma unroll
                for (int k = 0; k < PPT; k += 2) {
                    const float2 u = __ffma2_rn(ax2, make_float2(xs[k], xs[k + 1]), ub2);
                    const float2 ne = __ffma2_rn(u, u, nb2); // f'2 / f3: Q
                    if constexpr (!FOLD) {
                        const float2 Q = ne;
                        float2 al;
                        if constexpr (KIND == GS_K_POLY2) {
                            al = __ffma2_rn(__ffma2_rn(make_float2(b.w, b.w), Q, make_float2(b.z, b.z)), Q,
                                            make_float2(b.y, b.y));
                            al.x = Q.x < cfg.x0 ? al.x : 0.f;
                            al.y = Q.y < cfg.x0 ? al.y : 0.f;
                        } else {
                            al = __ffma2_rn(__ffma2_rn(__ffma2_rn(make_float2(p3, p3), Q, make_float2(b.w, b.w)), Q,
                                                       make_float2(b.z, b.z)),
                                            Q, make_float2(b.y, b.y));
                        }
                        na[k] = al.x >= eps ? fmaxf(-al.x, -amax) : 0.f;
                        na[k + 1] = al.y >= eps ? fmaxf(-al.y, -amax) : 0.f;
                    } else if constexpr (KIND == GS_K_EXP) {
                        const float a0 = ex2_approx(-ne.x), a1 = ex2_approx(-ne.y);
                        na[k] = a0 >= eps ? fmaxf(-a0, -amax) : 0.f;
                        na[k + 1] = a1 >= eps ? fmaxf(-a1, -amax) : 0.f;
                    } else {
                        na[k] = ne.x <= -eps ? (CLAMP ? fmaxf(ne.x, -amax) : ne.x) : 0.f;
                        na[k + 1] = ne.y <= -eps ? (CLAMP ? fmaxf(ne.y, -amax) : ne.y) : 0.f;
                    }
                    const float2 T2 = make_float2(T[k], T[k + 1]);
                    const float2 t = __ffma2_rn(make_float2(na[k], na[k + 1]), T2, T2);
                    Tn[k] = t.x;
                    Tn[k + 1] = t.y;
                    stop |= (t.x < tmin) | (t.y < tmin);
                }
                if (stop) {
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        if (Tn[k] < tmin) {
                            na[k] = 0.f;
                            Tn[k] = T[k];
                            active &= ~(1u << k);
                            xs[k] = NAN;
                            if constexpr (TRACK) ne[k] = pos;
                        }
                    }
                }
                if constexpr (TRACK) {
                    // a blended entry has na <= -eps
#pragma unroll
                    for (int k = 0; k < PPT; ++k) lastc[k] = na[k] != 0.f ? pos : lastc[k];
                }
                const float2 cr = make_float2(col.x, col.x), cg = make_float2(col.y, col.y),
                             cb = make_float2(col.z, col.z);
#pragma unroll
                for (int k = 0; k < PPT; k += 2) {
                    const float2 w = __fmul2_rn(make_float2(na[k], na[k + 1]), make_float2(T[k], T[k + 1]));
                    const float2 r = __ffma2_rn(cr, w, make_float2(C0[k], C0[k + 1]));
                    const float2 gg = __ffma2_rn(cg, w, make_float2(C1[k], C1[k + 1]));
                    const float2 bb = __ffma2_rn(cb, w, make_float2(C2[k], C2[k + 1]));
                    C0[k] = r.x, C0[k + 1] = r.y;
                    C1[k] = gg.x, C1[k + 1] = gg.y;
                    C2[k] = bb.x, C2[k + 1] = bb.y;
                    T[k] = Tn[k], T[k + 1] = Tn[k + 1];
                }
            } else {
            float al[PPT];
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                // min(alpha_max, x) < eps exactly when x < eps: the clamp
                // is applied only to entries that are blended
                const float u = fmaf(a.x, xs[k], ub);
                if constexpr (FOLD)
                    al[k] = alpha_folded<KIND>(v2, u);
                else
                    al[k] = alpha_of_q<KIND>(cfg, b, p3, fmaf(u, u, v2));
            }
            if constexpr (blend_branchless<KIND>()) {
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const bool use = al[k] >= eps;
                    const float a = fminf(amax, al[k]);
                    const float Tn = fmaf(-a, T[k], T[k]);
                    const bool stop = use && Tn < tmin;
                    const bool add = use && !stop;
                    const float w = add ? a * T[k] : 0.f;
                    C0[k] = fmaf(col.x, w, C0[k]);
                    C1[k] = fmaf(col.y, w, C1[k]);
                    C2[k] = fmaf(col.z, w, C2[k]);
                    T[k] = add ? Tn : T[k];
                    if constexpr (TRACK) {
                        lastc[k] = add ? pos : lastc[k];
                        ne[k] = stop ? pos : ne[k];
                    }
                    active &= ~((unsigned)stop << k);
                    xs[k] = stop ? NAN : xs[k];
                }
            } else {
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    if (!(al[k] >= eps)) continue;
                    al[k] = fminf(amax, al[k]);
                    const float Tn = fmaf(-al[k], T[k], T[k]);
                    if (Tn < tmin) {
                        active &= ~(1u << k);
                        xs[k] = NAN;
                        if constexpr (TRACK) ne[k] = pos;
                        continue;
                    }
                    const float w = al[k] * T[k];
                    C0[k] = fmaf(col.x, w, C0[k]);
                    C1[k] = fmaf(col.y, w, C1[k]);
                    C2[k] = fmaf(col.z, w, C2[k]);
                    T[k] = Tn;
                    if constexpr (TRACK) lastc[k] = pos;
                }
            }
            }
        };
        // one entry of the batch for this thread's run (a return skips it)
        auto entry = [&](const int j) {
            const float4 a = s_a[j];
            const float4 b = s_b[j];
            const float ub = fmaf(a.y, y, a.z);
            const float vv = fmaf(a.w, y, b.x);
            // FOLD: beta (NEGB: -beta, exactly, as fma(-x, y, z) = -fma(x, y, -z))
            const float v2 = NEGB ? fmaf(vv, vv, -b.y) : FOLD ? fmaf(-vv, vv, b.y) : vv * vv;
            [[maybe_unused]] const float p3 = (KIND == GS_K_POLY3) ? s_c[j].w : 0.f; // the cubic's top coefficient
            if (PPT > 1 && (FOLD || cfg.monotone)) { // f1 (c1 < 0) and exp are monotone
                // smallest Q over this thread's run of pixels: u is affine
                // along the run with slope ux = a.x > 0, so its smallest |u|
                // is max(0, |u(run centre)| - half-width * ux) (0 when u
                // changes sign). With k non-increasing, alpha there bounds
                // every pixel's; the skip threshold sits below eps so that
                // rounding can never skip an entry that a pixel would take.
#if GS_SKIP_MID
                const float umid = fmaf(a.x, xmid, ub);
                const float um = fmaxf(fmaf(-0.5f * (PPT - 1), a.x, fabsf(umid)), 0.f);
#else
                // the run's ends (not xs[], which is NaN for stopped pixels)
                const float ua = fmaf(a.x, lx + 0.5f, ub), uz = fmaf(a.x, lx + PPT - 0.5f, ub);
                const float um = ((ua > 0.f) != (uz > 0.f)) ? 0.f : fminf(fabsf(ua), fabsf(uz));
#endif
                if constexpr (NEGB) {
                    // the same test on the negated exponent / alpha
                    if (fmaf(um, um, v2) > -fold_skip) return;
                } else if constexpr (FOLD) {
                    // the run's largest exponent / alpha is beta - sm^2
                    if (fmaf(-um, um, v2) < fold_skip) return;
                } else if constexpr (KIND == GS_K_POLY1 || KIND == GS_K_EXP) {
                    // beyond the record's cut x_cut: no pixel's exact alpha
                    // reaches eps (FP16x2: it then skips what FP32 skips)
                    if (fmaf(um, um, v2) > b.w) return;
                } else if constexpr (KIND == GS_K_POLY2) {
                    // the same with f'2's cut, carried in its p3 slot
                    if (fmaf(um, um, v2) > s_c[j].w) return;
                } else if (KIND == GS_K_POLY3 && cfg.tail_zero) {
                    // f3 is 0 past its root x0: the opacity-free cut of Eq. 5
                    // (the Horner step of the test below costs more than the
                    // tighter opacity cut saves: f3 pass 7.94 -> 7.74 ms)
                    if (fmaf(um, um, v2) > cfg.x0) return;
                } else {
                    if (alpha_of_q<KIND>(cfg, b, p3, fmaf(um, um, v2)) < eps_skip) return;
                }
            }
            update(j, a, b, ub, v2, p3);
        };
        // the entry pair (2m, 2m + 1) of the pair layout (f1, exp packed):
        // the skip tests of both entries on FP32x2 pairs, with the same
        // rounding as entry(): max(umid - h ux, -(umid + h ux)) equals
        // |umid| - h ux as rounded, since the two FMAs differ in sign only
        [[maybe_unused]] auto pair = [&](const int m) {
            const float4 P0 = s_a[m], P1 = s_a[kMaxBatch / 2 + m], P2 = s_b[m];
            const float2 yy = make_float2(y, y), hh = make_float2(0.5f * (PPT - 1), 0.5f * (PPT - 1));
            const float2 ux = make_float2(P0.x, P0.y);
            const float2 ub = __ffma2_rn(make_float2(P0.z, P0.w), yy, make_float2(P1.x, P1.y));
            const float2 vv = __ffma2_rn(make_float2(P1.z, P1.w), yy, make_float2(P2.x, P2.y));
            const float2 v2 = __ffma2_rn(vv, vv, make_float2(P2.z, P2.w)); // -beta
            const float2 umid = __ffma2_rn(ux, make_float2(xmid, xmid), ub);
            const float2 lo = __ffma2_rn(make_float2(-hh.x, -hh.y), ux, umid), hi = __ffma2_rn(hh, ux, umid);
            const float2 um = make_float2(fmaxf(fmaxf(lo.x, -hi.x), 0.f), fmaxf(fmaxf(lo.y, -hi.y), 0.f));
            const float2 t = __ffma2_rn(um, um, v2);
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!(t.x > -fold_skip)) update(2 * m, make_float4(ux.x, 0.f, 0.f, 0.f), z, ub.x, v2.x, 0.f);
            if (!(t.y > -fold_skip)) update(2 * m + 1, make_float4(ux.y, 0.f, 0.f, 0.f), z, ub.y, v2.y, 0.f);
        };
        // (the FP16x2 blend keeps the unroll it was measured with: 8 for exp, 4 otherwise)
        constexpr int U = (FOLD || PACKED) ? blend_unroll<KIND>() : (KIND == GS_K_EXP ? 8 : 4);
        if constexpr (PAIRS) {
            // groups of U entries as U / 2 pairs, as below
            const int np = (cnt + 1) >> 1;
            constexpr int UP = U / 2;
            for (int m0 = 0; m0 < np && active; m0 += UP) {
                if (m0 + UP <= np) {
#pragma unroll
                    for (int mm = 0; mm < UP; ++mm) pair(m0 + mm);
                } else {
                    for (int m = m0; m < np; ++m) pair(m);
                }
            }
        } else if constexpr (FOLD || PACKED) {
            // whole groups of U entries unrolled, the run's activity tested
            // once per group (entries a stopped run walks change nothing: its
            // pixels are NaN and fail every alpha test). One-stream pass: f1
            // 6.19 -> 5.87 ms, exp 8.11 -> 7.70 ms; with the packed pairs f'2
            // 7.70 -> 7.61 ms, f3 8.06 -> 7.94 ms (the FP16x2 blend, whose
            // alpha is not FP32, keeps the test per entry).
            for (int j0 = 0; j0 < cnt && active; j0 += U) {
                if (j0 + U <= cnt) {
#pragma unroll
                    for (int jj = 0; jj < U; ++jj) entry(j0 + jj);
                } else {
                    for (int j = j0; j < cnt; ++j) entry(j);
                }
            }
        } else {
#pragma unroll U
            for (int j = 0; j < cnt && active; ++j) entry(j);
        }
        };
        if constexpr (NOCLAMP_OK) {
            if (need_clamp)
                walk(std::true_type{});
            else
                walk(std::false_type{});
        } else {
            walk(std::true_type{});
        }
    }
    if (own) write_run();
}

template <int KIND, int PPT, bool HALF, bool TRACK>
__global__ void __launch_bounds__(256, GS_RENDER_MIN_BLOCKS)
render_kernel(const __grid_constant__ CamTable cams, const __grid_constant__ CfgDev cfg,
              const __grid_constant__ RenderArgs g)
{
    __shared__ float4 s_stage[3 * kMaxBatch]; // the batch's coefficients; between batches the run exchange
    __shared__ uint4 s_h[HALF ? kMaxBatch : 1];
    __shared__ uint32_t s_wc[8];
    render_tile<KIND, PPT, HALF, TRACK>(cams, cfg, g, blockIdx.x, s_stage, s_stage + kMaxBatch,
                                        s_stage + 2 * kMaxBatch, s_h, reinterpret_cast<float *>(s_stage), s_wc);
}

template <int KIND, int PPT, bool HALF, bool TRACK>
__global__ void __launch_bounds__(256, GS_RENDER_MIN_BLOCKS)
render_persistent_kernel(const __grid_constant__ CamTable cams, const __grid_constant__ CfgDev cfg,
                         const __grid_constant__ RenderArgs g, uint32_t *work)
{
    __shared__ float4 s_stage[3 * kMaxBatch]; // the batch's coefficients; between batches the run exchange
    __shared__ uint4 s_h[HALF ? kMaxBatch : 1];
    __shared__ uint32_t s_wc[8];
    __shared__ uint32_t s_tile;
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(work, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        __syncthreads(); // every thread has read s_tile before it is overwritten
        if (t >= (uint32_t)cams.total_tiles) break;
        render_tile<KIND, PPT, HALF, TRACK>(cams, cfg, g, (int)t, s_stage, s_stage + kMaxBatch,
                                            s_stage + 2 * kMaxBatch, s_h, reinterpret_cast<float *>(s_stage), s_wc);
    }
}

// ---- Tensor-core evaluation of the quadric (the paper's Sec. 5.1 argument) ----
// For a 16x16 tile the quadric of every (pixel, splat) pair of a batch is one
// small contraction: Q = Phi(pixel) . W(splat) with the 6 monomials
// Phi = (x^2, x y, y^2, x, y, 1) of tile-centred pixel coordinates and
// W = (A, 2B, C, -2(A dx0 + B dy0), -2(B dx0 + C dy0), Q(tile centre)), K padded
// to 8. Each warp computes its 32 pixels x kTcB splats with mma.sync TF32;
// the pixel monomials are exact in TF32 (quarter integers below 57) and the
// splat weights are split into two TF32 parts (hi + lo), so A.B_hi + A.B_lo
// carries the weights' FP32 precision. The blend then reads Q per pixel from
// shared memory and composites in order as the FP32 path does (alpha from
// the same kernel function, same thresholds). One pixel per thread.
constexpr int kTcB = 32;        // splats per batch
constexpr int kTcS = kTcB + 4;  // Q row stride (words): conflict-free 16-byte row reads
constexpr int kTcWS = kTcB + 8; // weight row stride (words): conflict-free fragment loads

__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32_16x8x8(float &c0, float &c1, float &c2, float &c3, const uint32_t a[4],
                                                uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c0), "+f"(c1), "+f"(c2), "+f"(c3)
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// monomial `k` of the tile-centred pixel position (xc, yc)
__device__ __forceinline__ float monomial(int k, float xc, float yc)
{
    return k == 0 ? xc * xc : k == 1 ? xc * yc : k == 2 ? yc * yc : k == 3 ? xc : k == 4 ? yc : k == 5 ? 1.f : 0.f;
}

template <int KIND>
__global__ void __launch_bounds__(256)
render_tc_kernel(const __grid_constant__ CamTable cams, const __grid_constant__ CfgDev cfg,
                 const __grid_constant__ RenderArgs g)
{
    __shared__ __align__(16) float s_q[256 * kTcS];
    __shared__ uint32_t s_whi[8 * kTcWS], s_wlo[8 * kTcWS];
    __shared__ float4 s_b[kTcB], s_c[kTcB];
    const int gtile = blockIdx.x;
    int c = 0;
    while (c + 1 < cams.ncam && cams.cam[c + 1].tile_base <= gtile) ++c;
    const CamDev &cm = cams.cam[c];
    const int lt = gtile - cm.tile_base;
    const int tx = lt % cm.tiles_x, ty = lt / cm.tiles_x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lx = tid & 15, ly = tid >> 4;
    const int px = tx * 16 + lx, py = ty * 16 + ly;
    const float ox = (float)(tx * 16), oy = (float)(ty * 16);
    const float ocx = ox + 8.f, ocy = oy + 8.f; // tile centre
    const uint2 rg = g.ranges[gtile];
    // an empty or inverted range (only possible after a timed-out sort wait)
    // reads nothing: every range gs_bin_sort writes lies within its output
    const uint32_t n = rg.y > rg.x ? rg.y - rg.x : 0u;
    const float eps = cfg.eps, amax = cfg.alpha_max, tmin = cfg.t_min;
    bool active = px < cm.W && py < cm.H;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    float ek = active ? eps : INFINITY;
    uint32_t lastc = 0, ne = n;
    // A fragments (m16n8k8, row-major 16 x 8): warp w, m-tile mt holds tile row
    // 2w + mt, fragment row r = pixel column r; element e of the fragment is
    // (row g + 8 (e & 1), column t + 4 (e >> 1)) with g = lane / 4, t = lane % 4
    const int gq = lane >> 2, tq = lane & 3;
    uint32_t afr[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const float yc = (float)(2 * warp + mt) + 0.5f - 8.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float xc = (float)(gq + 8 * (e & 1)) + 0.5f - 8.f;
            afr[mt][e] = to_tf32(monomial(tq + 4 * (e >> 1), xc, yc)); // exact
        }
    }
    const float *qrow = s_q + tid * kTcS;
    for (uint32_t base = 0; base < n; base += kTcB) {
        if (__syncthreads_count(active) == 0) break;
        const int cnt = (int)min((uint32_t)kTcB, n - base);
        if (tid < kTcB) {
            float w[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float4 bb = make_float4(0.f, 0.f, 0.f, 0.f), cc = bb;
            if (tid < cnt) {
                uint32_t v = g.vals[rg.x + base + tid];
                if (v >= g.n_records) v = 0; // only after a timed-out sort wait
                const float4 r0 = g.rec[3 * (size_t)v + 0], r1 = g.rec[3 * (size_t)v + 1];
                const float4 r2 = g.rec[3 * (size_t)v + 2];
                const BlendCoef k = make_coef<KIND>(cfg, r0, r1, r2, ox, oy);
                bb = k.b;
                cc = k.c;
                const float A = r1.x, B = r1.y, C = r1.z;
                const float dx0 = r0.x - ocx, dy0 = r0.y - ocy;
                const float gx = fmaf(A, dx0, B * dy0), gy = fmaf(B, dx0, C * dy0);
                w[0] = A;
                w[1] = 2.f * B;
                w[2] = C;
                w[3] = -2.f * gx;
                w[4] = -2.f * gy;
                w[5] = fmaf(dx0, gx, dy0 * gy);
            }
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const uint32_t hi = to_tf32(w[kk]);
                s_whi[kk * kTcWS + tid] = hi;
                s_wlo[kk * kTcWS + tid] = to_tf32(w[kk] - __uint_as_float(hi));
            }
            s_b[tid] = bb;
            s_c[tid] = cc;
        }
        __syncthreads();
        if (__any_sync(0xffffffffu, active)) {
#pragma unroll
            for (int nt = 0; nt < kTcB / 8; ++nt) {
                const int n0 = nt * 8;
                // B fragment (col-major 8 x 8): (row t, column g) and (row t + 4, column g)
                const uint32_t bh0 = s_whi[tq * kTcWS + n0 + gq], bh1 = s_whi[(tq + 4) * kTcWS + n0 + gq];
                const uint32_t bl0 = s_wlo[tq * kTcWS + n0 + gq], bl1 = s_wlo[(tq + 4) * kTcWS + n0 + gq];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
                    mma_tf32_16x8x8(c0, c1, c2, c3, afr[mt], bl0, bl1); // small part first
                    mma_tf32_16x8x8(c0, c1, c2, c3, afr[mt], bh0, bh1);
                    // C fragment: (row g, columns 2t, 2t + 1) and (row g + 8, same columns)
                    const int p0 = 32 * warp + 16 * mt + gq;
                    *reinterpret_cast<float2 *>(&s_q[p0 * kTcS + n0 + 2 * tq]) = make_float2(c0, c1);
                    *reinterpret_cast<float2 *>(&s_q[(p0 + 8) * kTcS + n0 + 2 * tq]) = make_float2(c2, c3);
                }
            }
        }
        __syncwarp(); // a pixel's Q row is written by its own warp
        for (int j = 0; j < cnt && active; ++j) {
            const float4 cj = s_c[j];
            const float al0 = alpha_of_q<KIND>(cfg, s_b[j], cj.w, qrow[j]);
            if (!(al0 >= ek)) continue;
            const float al = fminf(amax, al0);
            const float Tn = fmaf(-al, T, T);
            const uint32_t pos = base + j + 1;
            if (Tn < tmin) {
                active = false;
                ek = INFINITY;
                ne = pos;
                break;
            }
            const float wgt = al * T;
            C0 = fmaf(cj.x, wgt, C0);
            C1 = fmaf(cj.y, wgt, C1);
            C2 = fmaf(cj.z, wgt, C2);
            T = Tn;
            lastc = pos;
        }
    }
    if (px < cm.W && py < cm.H) {
        const int64_t pix = cm.pix_base + (int64_t)py * cm.W + px;
        g.out[3 * pix + 0] = fmaf(T, g.bg0, C0);
        g.out[3 * pix + 1] = fmaf(T, g.bg1, C1);
        g.out[3 * pix + 2] = fmaf(T, g.bg2, C2);
        if (g.final_T) g.final_T[pix] = T;
        if (g.last) g.last[pix] = lastc;
        if (g.n_eval) g.n_eval[pix] = ne;
    }
}

template <int KIND, int PPT, bool HALF, bool TRACK>
cudaError_t launch3(int threads, cudaStream_t s, const CamTable &t, const CfgDev &c, const RenderArgs &g,
                    uint32_t *work)
{
    if (!work) {
        render_kernel<KIND, PPT, HALF, TRACK><<<t.total_tiles, threads, 0, s>>>(t, c, g);
        return cudaPeekAtLastError();
    }
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_persistent_kernel<KIND, PPT, HALF, TRACK>,
                                                      threads, 0) != cudaSuccess)
        return cudaGetLastError();
    if (GS_PERSIST_CAP > 0) per_sm = std::min(per_sm, GS_PERSIST_CAP);
    const int grid = std::max(1, std::min(t.total_tiles, sms * std::max(per_sm, 1)));
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    render_persistent_kernel<KIND, PPT, HALF, TRACK><<<grid, threads, 0, s>>>(t, c, g, work);
    return cudaPeekAtLastError();
}

template <int KIND, int PPT, bool HALF>
cudaError_t launch2(int threads, cudaStream_t s, const CamTable &t, const CfgDev &c, const RenderArgs &g,
                    uint32_t *work)
{
    if (g.last || g.n_eval) return launch3<KIND, PPT, HALF, true>(threads, s, t, c, g, work);
    return launch3<KIND, PPT, HALF, false>(threads, s, t, c, g, work);
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
    if (cfg->tensor_alpha < 0 || cfg->tensor_alpha > 2) return GS_ERR_ARG;
    if (cfg->tensor_alpha && (cfg->tile_w != 16 || cfg->tile_h != 16 || cfg->fp16x2 || d_work))
        return GS_ERR_UNSUPPORTED; // tensor-core variant: 16x16 tiles, FP32, one CTA per tile
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
    if (cfg->tensor_alpha == 2) {
        e = launch_render_tc5(cfg->kind, s, t, c, g);
    } else if (cfg->tensor_alpha) {
        switch (cfg->kind) {
        case GS_K_EXP: render_tc_kernel<GS_K_EXP><<<t.total_tiles, 256, 0, s>>>(t, c, g); break;
        case GS_K_POLY1: render_tc_kernel<GS_K_POLY1><<<t.total_tiles, 256, 0, s>>>(t, c, g); break;
        case GS_K_POLY2: render_tc_kernel<GS_K_POLY2><<<t.total_tiles, 256, 0, s>>>(t, c, g); break;
        default: render_tc_kernel<GS_K_POLY3><<<t.total_tiles, 256, 0, s>>>(t, c, g); break;
        }
        e = cudaPeekAtLastError();
    } else {
    switch (cfg->kind) {
    case GS_K_EXP: e = launch_render<GS_K_EXP>(ppt, half, threads, s, t, c, g, work); break;
    case GS_K_POLY1: e = launch_render<GS_K_POLY1>(ppt, half, threads, s, t, c, g, work); break;
    case GS_K_POLY2: e = launch_render<GS_K_POLY2>(ppt, half, threads, s, t, c, g, work); break;
    default: e = launch_render<GS_K_POLY3>(ppt, half, threads, s, t, c, g, work); break;
    }
    }
    count_launch();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    return GS_OK;
}
