// backward.cu — reverse pass of the blend and of the projection (sm_103a).
//
// Stage 1, per tile (one CTA, one thread per pixel): walk the tile's list
// backwards from the block's furthest last contributor. Each pixel starts
// from its saved final transmittance and recovers T before every contributor
// as T / (1 - alpha), recomputing alpha with exactly the forward arithmetic so
// that every skip / clamp decision is the forward's. Per contributor:
//   dL/dc = alpha T g,  dL/dalpha = sum_ch g (c T - S / (1 - alpha)),
//   with S the colour behind it (later contributors plus T_final bg);
//   alpha = o' k(Q) unclamped: dL/do' = k dL/dalpha, dL/dQ = o' k'(Q) dL/dalpha,
//   k' = -k/2 (exp), c1 + 2 c2 Q + 3 c3 Q^2 (polynomials; the ReLU / cut are
//   inactive wherever alpha >= eps), then dQ to the conic and the 2D mean.
// Each warp walks the list only up to its own furthest last contributor,
// sums its lanes' contributions to an entry with shuffles and adds the sums
// to shared-memory accumulators of the batch; after the batch one thread per
// entry adds the tile's sums to the record's 2D gradient with FP32 atomics.
//
// Stage 2, per splat (one thread, loop over cameras): the chain rule through
// the projection written in preprocess.cu: colour clamp and SH (and the view
// direction), o' = o rho with the AA factor (Sec. 3.4), conic = inverse of the
// low-passed covariance, Sigma' = J W Sigma W^T J^T with the clamped
// Jacobian, the pinhole mean, Sigma = R S S^T R^T, the quaternion
// normalisation. Gradients are added to the caller's buffers.
#include "blend_math.cuh"

namespace gs {
namespace {

constexpr int kG2 = 12; // floats per record in the 2D gradient buffer
// layout: dmean.x, dmean.y, dA, dB, dC, do', dr, dg, db, (unused x3)

__device__ __forceinline__ float wsum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sums of 8 values at once: at the exchanges across 16, 8 and 4 lanes
// each lane keeps half of its remaining values and sends the other half to
// its partner (4 + 2 + 1 shuffles), then two plain steps (2 shuffles) finish
// the single value left. Returns the sum of value (lane >> 2) & 7 (bit 4 of
// the lane picks the upper half first), valid in every lane; lanes with
// (lane & 3) == 0 hold the 8 different sums.
__device__ __forceinline__ float wsum8(const float (&v)[8], int lane)
{
    float a[4], b[2];
    const bool h4 = lane & 16, h2 = lane & 8, h1 = lane & 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = h4 ? v[i] : v[i + 4];
        const float keep = h4 ? v[i + 4] : v[i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = h2 ? a[i] : a[i + 2];
        const float keep = h2 ? a[i + 2] : a[i];
        b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float c;
    {
        const float send = h1 ? b[0] : b[1];
        const float keep = h1 ? b[1] : b[0];
        c = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// value index whose total wsum8 leaves in this lane
__device__ __forceinline__ int wsum8_index(int lane)
{
    return ((lane & 16) ? 4 : 0) + ((lane & 8) ? 2 : 0) + ((lane & 4) ? 1 : 0);
}

// Dynamic shared memory of the reverse blend for a batch of B entries (B =
// threads per CTA): five float4 arrays (2D mean and 1 / o', conic, three
// coefficient vectors), the record ids, and the accumulators of the
// per-entry gradient sums, [value][entry] with a row stride of B + 1 floats
// (odd), so that the 9 lanes that add one entry's 9 sums hit 9 banks.
__host__ __device__ constexpr size_t bwd_smem_bytes(int B)
{
    return (size_t)B * (5 * sizeof(float4) + sizeof(uint32_t)) + sizeof(float) * 9 * (B + 1);
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// PPT horizontally adjacent pixels per thread (1 or 2): the per-entry setup
// (shared-memory loads, the row terms of the quadric) and the warp reduction
// are shared by all of a warp's 32 PPT pixels.
template <int KIND, int PPT>
__global__ void __launch_bounds__(256)
blend_backward_kernel(const __grid_constant__ CamTable cams, const __grid_constant__ CfgDev cfg,
                      const float4 *__restrict__ rec, const uint32_t *__restrict__ vals,
                      const uint2 *__restrict__ ranges, uint32_t n_records, float bg0, float bg1,
                      float bg2, const float *__restrict__ final_T, const uint32_t *__restrict__ last,
                      const float *__restrict__ grad_out, float *__restrict__ grad2d)
{
    // the forward's FP32 alpha arithmetic (render.cu): f1 and exp fold their
    // Q coefficient into the affine forms
    constexpr bool FOLD = folds_p1<KIND>();
    extern __shared__ float4 s_dyn[];
    const int B = blockDim.x;
    float4 *s_g = s_dyn; // mu'x, mu'y, o', 1 / o'
    float4 *s_q = s_g + B;
    float4 *s_ka = s_q + B;
    float4 *s_kb = s_ka + B;
    float4 *s_kc = s_kb + B;
    uint32_t *s_id = reinterpret_cast<uint32_t *>(s_kc + B);
    float *s_acc = reinterpret_cast<float *>(s_id + B);
    const int kAccStride = B + 1;
    __shared__ uint32_t s_maxL;
    const int gtile = blockIdx.x;
    int c = 0;
    while (c + 1 < cams.ncam && cams.cam[c + 1].tile_base <= gtile) ++c;
    const CamDev &cm = cams.cam[c];
    const int lt = gtile - cm.tile_base;
    const int tx = lt % cm.tiles_x, ty = lt / cm.tiles_x;
    const int tpr = cfg.tile_w / PPT; // threads per tile row
    const int lx = ((int)threadIdx.x % tpr) * PPT, ly = (int)threadIdx.x / tpr;
    const int px0 = tx * cfg.tile_w + lx, py = ty * cfg.tile_h + ly;
    const float pyc = py + 0.5f;
    const float ox = (float)(tx * cfg.tile_w), oy = (float)(ty * cfg.tile_h);
    const float yl = (float)ly + 0.5f;
    const uint2 rg = ranges[gtile];
    const int lane = threadIdx.x & 31;

    float T[PPT], S[PPT][3], gr[PPT][3], xl[PPT];
    uint32_t L[PPT];
    uint32_t Lmax = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        T[k] = 1.f;
        L[k] = 0;
        gr[k][0] = gr[k][1] = gr[k][2] = 0.f;
        xl[k] = (float)(lx + k) + 0.5f;
        if (px0 + k < cm.W && py < cm.H) {
            const int64_t pix = cm.pix_base + (int64_t)py * cm.W + px0 + k;
            T[k] = final_T[pix];
            L[k] = last[pix];
            gr[k][0] = grad_out[3 * pix + 0];
            gr[k][1] = grad_out[3 * pix + 1];
            gr[k][2] = grad_out[3 * pix + 2];
        }
        S[k][0] = T[k] * bg0;
        S[k][1] = T[k] * bg1;
        S[k][2] = T[k] * bg2;
        Lmax = max(Lmax, L[k]);
    }
    if (threadIdx.x == 0) s_maxL = 0;
    for (int k = threadIdx.x; k < 9 * kAccStride; k += blockDim.x) s_acc[k] = 0.f;
    __syncthreads();
    if (Lmax) atomicMax(&s_maxL, Lmax);
    __syncthreads();
    // a pixel's last lies within its tile list (an inverted range, only
    // possible after a timed-out sort wait, counts as empty)
    const uint32_t n = rg.y > rg.x ? rg.y - rg.x : 0u;
    const int maxL = (int)min(s_maxL, n);
    // this warp's furthest last contributor: entries beyond it touch none of
    // its pixels
    const int wL = (int)min(__reduce_max_sync(0xffffffffu, Lmax), n);
    const float eps = cfg.eps, amax = cfg.alpha_max;
    for (int end = maxL; end > 0; end -= B) {
        const int start = max(0, end - B);
        const int i = start + (int)threadIdx.x;
        if (i < end) {
            uint32_t v = vals[rg.x + i];
            if (v >= n_records) v = 0;
            s_id[threadIdx.x] = v;
            const float4 r0 = rec[3 * (size_t)v + 0], r1 = rec[3 * (size_t)v + 1];
            const BlendCoef kc = make_coef<KIND, FOLD>(cfg, r0, r1, rec[3 * (size_t)v + 2], ox, oy);
            s_g[threadIdx.x] = make_float4(r0.x, r0.y, r0.z, 1.f / r0.z);
            s_q[threadIdx.x] = r1;
            s_ka[threadIdx.x] = kc.a;
            s_kb[threadIdx.x] = kc.b;
            s_kc[threadIdx.x] = kc.c;
        }
        __syncthreads();
        for (int j = min(end, wL) - 1; j >= start; --j) {
            const int jj = j - start;
            // alpha exactly as the forward computed it
            const float4 ka = s_ka[jj], kb = s_kb[jj];
            const float p3 = (KIND == GS_K_POLY3) ? s_kc[jj].w : 0.f;
            const float ub = fmaf(ka.y, yl, ka.z);
            const float vv = fmaf(ka.w, yl, kb.x);
            const float v2 = FOLD ? fmaf(-vv, vv, kb.y) : vv * vv; // FOLD: beta
            float Q[PPT], a0[PPT];
            bool con[PPT], anyc = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const float u = fmaf(ka.x, xl[k], ub);
                if constexpr (FOLD) {
                    Q[k] = 0.f; // f1 and exp need no Q for their slope
                    a0[k] = alpha_folded<KIND>(v2, u);
                } else {
                    Q[k] = fmaf(u, u, v2);
                    a0[k] = alpha_of_q<KIND>(cfg, kb, p3, Q[k]);
                }
                con[k] = (uint32_t)j < L[k] && fminf(amax, a0[k]) >= eps;
                anyc |= con[k];
            }
            if (!__any_sync(0xffffffffu, anyc)) continue;
            const float4 g = s_g[jj];
            const float4 q = s_q[jj];
            const float4 col = s_kc[jj];
            const float dy = g.y - pyc;
            float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (!con[k]) continue;
                const float a = fminf(amax, a0[k]);
                const float ioma = rcp_approx(1.f - a);
                T[k] *= ioma; // transmittance before this entry
                const float w = a * T[k];
                v[6] = fmaf(w, gr[k][0], v[6]);
                v[7] = fmaf(w, gr[k][1], v[7]);
                v[8] = fmaf(w, gr[k][2], v[8]);
                const float da = gr[k][0] * (col.x * T[k] - S[k][0] * ioma) +
                                 gr[k][1] * (col.y * T[k] - S[k][1] * ioma) +
                                 gr[k][2] * (col.z * T[k] - S[k][2] * ioma);
                S[k][0] = fmaf(col.x, w, S[k][0]);
                S[k][1] = fmaf(col.y, w, S[k][1]);
                S[k][2] = fmaf(col.z, w, S[k][2]);
                if (a0[k] <= amax) {
                    v[5] = fmaf(a0[k] * g.w, da, v[5]); // k(Q) = o' k(Q) / o'
                    // o' dk/dQ: -o' k / 2 for exp, o' k'(Q) for the polynomials
                    const float dQ =
                        (KIND == GS_K_EXP ? -0.5f * a0[k] : g.z * kernel_slope<KIND>(cfg, Q[k], a0[k], g.z)) * da;
                    const float dx = g.x - (float)(px0 + k) - 0.5f;
                    const float dQx = dQ * dx, dQy = dQ * dy;
                    v[2] = fmaf(dQx, dx, v[2]);
                    v[3] = fmaf(2.f * dQx, dy, v[3]);
                    v[4] = fmaf(dQy, dy, v[4]);
                    v[0] = fmaf(2.f * dQ, fmaf(q.x, dx, q.y * dy), v[0]);
                    v[1] = fmaf(2.f * dQ, fmaf(q.y, dx, q.z * dy), v[1]);
                }
            }
            const float v8[8] = {v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]};
            const float s8 = wsum8(v8, lane);
            const float s9 = wsum(v[8]);
            if ((lane & 3) == 0 && s8 != 0.f) atomicAdd(&s_acc[wsum8_index(lane) * kAccStride + jj], s8);
            if (lane == 1 && s9 != 0.f) atomicAdd(&s_acc[8 * kAccStride + jj], s9);
        }
        __syncthreads();
        // one set of global atomics per entry and tile; each thread flushes
        // (and clears) the entry it staged, so the next batch's staging by
        // the same thread needs no further barrier
        if (i < end) {
            float *dst = grad2d + (size_t)s_id[threadIdx.x] * kG2;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float sv = s_acc[k * kAccStride + threadIdx.x];
                if (sv != 0.f) {
                    atomicAdd(dst + k, sv);
                    s_acc[k * kAccStride + threadIdx.x] = 0.f;
                }
            }
        }
    }
}

// ---- stage 2: per-splat chain rule ---------------------------------------

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

// SH basis values Y[k] and their gradients with respect to the unit
// direction, G[k][0..2] (3DGS order and signs).
template <int D>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float *Y, float (*G)[3])
{
    Y[0] = kY0;
    G[0][0] = G[0][1] = G[0][2] = 0.f;
    if (D >= 1) {
        Y[1] = -kY1 * y; G[1][0] = 0.f; G[1][1] = -kY1; G[1][2] = 0.f;
        Y[2] = kY1 * z;  G[2][0] = 0.f; G[2][1] = 0.f;  G[2][2] = kY1;
        Y[3] = -kY1 * x; G[3][0] = -kY1; G[3][1] = 0.f; G[3][2] = 0.f;
    }
    if (D >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * x * y;  G[4][0] = kY2a * y; G[4][1] = kY2a * x; G[4][2] = 0.f;
        Y[5] = -kY2a * y * z; G[5][0] = 0.f; G[5][1] = -kY2a * z; G[5][2] = -kY2a * y;
        Y[6] = kY2b * (2.f * zz - xx - yy);
        G[6][0] = -2.f * kY2b * x; G[6][1] = -2.f * kY2b * y; G[6][2] = 4.f * kY2b * z;
        Y[7] = -kY2a * x * z; G[7][0] = -kY2a * z; G[7][1] = 0.f; G[7][2] = -kY2a * x;
        Y[8] = kY2c * (xx - yy); G[8][0] = 2.f * kY2c * x; G[8][1] = -2.f * kY2c * y; G[8][2] = 0.f;
        if (D >= 3) {
            Y[9] = -kY3a * y * (3.f * xx - yy);
            G[9][0] = -kY3a * 6.f * x * y; G[9][1] = -kY3a * (3.f * xx - 3.f * yy); G[9][2] = 0.f;
            Y[10] = kY3b * x * y * z;
            G[10][0] = kY3b * y * z; G[10][1] = kY3b * x * z; G[10][2] = kY3b * x * y;
            Y[11] = -kY3c * y * (4.f * zz - xx - yy);
            G[11][0] = kY3c * 2.f * x * y; G[11][1] = -kY3c * (4.f * zz - xx - 3.f * yy);
            G[11][2] = -kY3c * 8.f * y * z;
            Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            G[12][0] = -kY3d * 6.f * x * z; G[12][1] = -kY3d * 6.f * y * z;
            G[12][2] = kY3d * (6.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kY3c * x * (4.f * zz - xx - yy);
            G[13][0] = -kY3c * (4.f * zz - 3.f * xx - yy); G[13][1] = kY3c * 2.f * x * y;
            G[13][2] = -kY3c * 8.f * x * z;
            Y[14] = kY3e * z * (xx - yy);
            G[14][0] = kY3e * 2.f * x * z; G[14][1] = -kY3e * 2.f * y * z; G[14][2] = kY3e * (xx - yy);
            Y[15] = -kY3a * x * (xx - 3.f * yy);
            G[15][0] = -kY3a * (3.f * xx - 3.f * yy); G[15][1] = kY3a * 6.f * x * y; G[15][2] = 0.f;
        }
    }
}

// Chain rule of one splat through its projections (all cameras). io: the
// splat's inputs on entry (mean 3, scale 3, quaternion 4, opacity 1), its
// gradients with respect to them on return; sh_row: its 3K SH coefficients;
// dsh: its SH gradient accumulators, one every dstride floats.
constexpr int kIO = 11;
template <int D>
__device__ __forceinline__ void project_backward_splat(const CamTable &cams, const CfgDev &cfg, int P, int i,
                                                       float *io, const float *sh_row, float *dsh,
                                                       int dstride, const float *__restrict__ grad2d)
{
    constexpr int K = (D + 1) * (D + 1);
    const float mx = io[0], my = io[1], mz = io[2];
    const float sx = io[3], sy = io[4], sz = io[5];
    const float4 q4 = make_float4(io[6], io[7], io[8], io[9]);
    const float op = io[10];

    const float qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float w = q4.x * qn, x = q4.y * qn, y = q4.z * qn, z = q4.w * qn;
    float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                     {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                     {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
    const float s[3] = {sx, sy, sz};
    float M[3][3], Sg[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) M[r][k] = R[r][k] * s[k];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) Sg[r][k] = M[r][0] * M[k][0] + M[r][1] * M[k][1] + M[r][2] * M[k][2];

    float dmean[3] = {0.f, 0.f, 0.f}, dSig[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float dop = 0.f;
    bool any = false;

    for (int c = 0; c < cams.ncam; ++c) {
        const CamDev &cm = cams.cam[c];
        const int64_t n = (int64_t)c * P + i;
        const float4 ga = reinterpret_cast<const float4 *>(grad2d + n * kG2)[0];
        const float4 gb = reinterpret_cast<const float4 *>(grad2d + n * kG2)[1];
        const float4 gc = reinterpret_cast<const float4 *>(grad2d + n * kG2)[2];
        const float dmx = ga.x, dmy = ga.y, dA = ga.z, dB = ga.w, dC = gb.x, do2 = gb.y;
        const float dcol[3] = {gb.z, gb.w, gc.x};
        if (dmx == 0.f && dmy == 0.f && dA == 0.f && dB == 0.f && dC == 0.f && do2 == 0.f &&
            dcol[0] == 0.f && dcol[1] == 0.f && dcol[2] == 0.f)
            continue;
        any = true;
        const float *W = cm.R;
        const float tx = W[0] * mx + W[1] * my + W[2] * mz + cm.T[0];
        const float ty = W[3] * mx + W[4] * my + W[5] * mz + cm.T[1];
        const float tz = W[6] * mx + W[7] * my + W[8] * mz + cm.T[2];
        const float iz = 1.f / tz;
        const float rx = tx * iz, ry = ty * iz;
        const int clx = rx < -cm.limx ? -1 : (rx > cm.limx ? 1 : 0);
        const int cly = ry < -cm.limy ? -1 : (ry > cm.limy ? 1 : 0);
        const float ux = fminf(fmaxf(rx, -cm.limx), cm.limx);
        const float uy = fminf(fmaxf(ry, -cm.limy), cm.limy);
        const float a0 = cm.fx * iz, b0 = cm.fy * iz;
        float Tm[2][3] = {{a0 * (W[0] - ux * W[6]), a0 * (W[1] - ux * W[7]), a0 * (W[2] - ux * W[8])},
                          {b0 * (W[3] - uy * W[6]), b0 * (W[4] - uy * W[7]), b0 * (W[5] - uy * W[8])}};
        float TS[2][3];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                TS[r][k] = Tm[r][0] * Sg[0][k] + Tm[r][1] * Sg[1][k] + Tm[r][2] * Sg[2][k];
        const float c00 = TS[0][0] * Tm[0][0] + TS[0][1] * Tm[0][1] + TS[0][2] * Tm[0][2];
        const float c01 = TS[1][0] * Tm[0][0] + TS[1][1] * Tm[0][1] + TS[1][2] * Tm[0][2];
        const float c11 = TS[1][0] * Tm[1][0] + TS[1][1] * Tm[1][1] + TS[1][2] * Tm[1][2];
        const float a = c00 + cfg.dil, b = c01, cc = c11 + cfg.dil;
        const float det0 = c00 * c11 - c01 * c01;
        const float det1 = a * cc - b * b;
        const float rho = cfg.aa ? sqrtf(fmaxf(det0, 0.f) / det1) : 1.f;

        // colour: c = max(sum_k Y_k sh_k + 0.5, 0)
        float dvx = mx - cm.campos[0], dvy = my - cm.campos[1], dvz = mz - cm.campos[2];
        const float il = rsqrtf(dvx * dvx + dvy * dvy + dvz * dvz);
        const float ex = dvx * il, ey = dvy * il, ez = dvz * il;
        float Y[K], GY[K][3];
        sh_basis_grad<D>(ex, ey, ez, Y, GY);
        float draw[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc = fmaf(Y[k], sh_row[3 * k + ch], acc);
            draw[ch] = (acc + 0.5f > 0.f) ? dcol[ch] : 0.f;
        }
        float ddir[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float t = 0.f;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                dsh[(3 * k + ch) * dstride] = fmaf(Y[k], draw[ch], dsh[(3 * k + ch) * dstride]);
                t = fmaf(sh_row[3 * k + ch], draw[ch], t);
            }
            ddir[0] = fmaf(GY[k][0], t, ddir[0]);
            ddir[1] = fmaf(GY[k][1], t, ddir[1]);
            ddir[2] = fmaf(GY[k][2], t, ddir[2]);
        }
        const float dd = ddir[0] * ex + ddir[1] * ey + ddir[2] * ez;
        dmean[0] += (ddir[0] - ex * dd) * il;
        dmean[1] += (ddir[1] - ey * dd) * il;
        dmean[2] += (ddir[2] - ez * dd) * il;

        // o' = o rho
        dop += rho * do2;
        const float drho = cfg.aa ? op * do2 : 0.f;
        // conic = (Sigma' + vI)^-1
        const float idet = 1.f / det1;
        float ddet1 = -(dA * cc - dB * b + dC * a) * idet * idet;
        float da = dC * idet, db = -dB * idet, dc = dA * idet;
        float ddet0 = 0.f;
        if (cfg.aa && det0 > 0.f) {
            ddet0 = drho / (2.f * sqrtf(det0 * det1));
            ddet1 += -drho * rho * 0.5f * idet;
        }
        da += ddet1 * cc;
        dc += ddet1 * a;
        db += -2.f * b * ddet1;
        const float dS00 = da + ddet0 * c11, dS11 = dc + ddet0 * c00, dS01 = db - 2.f * c01 * ddet0;
        const float G[2][2] = {{dS00, 0.5f * dS01}, {0.5f * dS01, dS11}};
        // Sigma' = Tm Sigma Tm^T
        float dTm[2][3];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k) dTm[r][k] = 2.f * (G[r][0] * TS[0][k] + G[r][1] * TS[1][k]);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float acc = 0.f;
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int vv = 0; vv < 2; ++vv) acc += Tm[u][r] * G[u][vv] * Tm[vv][k];
                dSig[r][k] += acc;
            }
        // Tm = J W with J = [[a0, 0, -a0 ux], [0, b0, -b0 uy]]
        const float dJ00 = dTm[0][0] * W[0] + dTm[0][1] * W[1] + dTm[0][2] * W[2];
        const float dJ02 = dTm[0][0] * W[6] + dTm[0][1] * W[7] + dTm[0][2] * W[8];
        const float dJ11 = dTm[1][0] * W[3] + dTm[1][1] * W[4] + dTm[1][2] * W[5];
        const float dJ12 = dTm[1][0] * W[6] + dTm[1][1] * W[7] + dTm[1][2] * W[8];
        const float txc = ux * tz, tyc = uy * tz;
        const float iz2 = iz * iz, iz3 = iz2 * iz;
        float dtx = 0.f, dty = 0.f;
        float dtz = -cm.fx * iz2 * dJ00 + 2.f * cm.fx * txc * iz3 * dJ02 - cm.fy * iz2 * dJ11 +
                    2.f * cm.fy * tyc * iz3 * dJ12;
        const float dtxc = -cm.fx * iz2 * dJ02, dtyc = -cm.fy * iz2 * dJ12;
        if (clx == 0) dtx += dtxc; else dtz += clx * cm.limx * dtxc;
        if (cly == 0) dty += dtyc; else dtz += cly * cm.limy * dtyc;
        // mean2d = (fx tx / tz + cx, fy ty / tz + cy)
        dtx += cm.fx * iz * dmx;
        dty += cm.fy * iz * dmy;
        dtz += -cm.fx * tx * iz2 * dmx - cm.fy * ty * iz2 * dmy;
        // t = W mu + T
        dmean[0] += W[0] * dtx + W[3] * dty + W[6] * dtz;
        dmean[1] += W[1] * dtx + W[4] * dty + W[7] * dtz;
        dmean[2] += W[2] * dtx + W[5] * dty + W[8] * dtz;
    }
    if (!any) {
#pragma unroll
        for (int k = 0; k < kIO; ++k) io[k] = 0.f;
        return;
    }

    // Sigma = M M^T, M = R diag(s): dM = (dSig + dSig^T) M
    float ds[3] = {0.f, 0.f, 0.f}, dR[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float dM = (dSig[r][0] + dSig[0][r]) * M[0][k] + (dSig[r][1] + dSig[1][r]) * M[1][k] +
                             (dSig[r][2] + dSig[2][r]) * M[2][k];
            ds[k] += dM * R[r][k];
            dR[r][k] = dM * s[k];
        }
    float dqn[4];
    dqn[0] = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
    dqn[1] = 2.f * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] - w * dR[1][2] +
                    z * dR[2][0] + w * dR[2][1] - 2.f * x * dR[2][2]);
    dqn[2] = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] -
                    w * dR[2][0] + z * dR[2][1] - 2.f * y * dR[2][2]);
    dqn[3] = 2.f * (-2.f * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2.f * z * dR[1][1] +
                    y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
    const float dot = dqn[0] * w + dqn[1] * x + dqn[2] * y + dqn[3] * z;
    const float qv[4] = {w, x, y, z};
#pragma unroll
    for (int k = 0; k < 4; ++k) io[6 + k] = (dqn[k] - qv[k] * dot) * qn;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        io[k] = dmean[k];
        io[3 + k] = ds[k];
    }
    io[10] = dop;
}

// Splats per CTA of the per-splat pass. The CTA stages its splats' inputs
// and SH rows in shared memory with coalesced loads (row strides 11 and
// 3K + 1 floats, odd, so a warp reading one value of 32 rows hits 32 banks),
// accumulates the SH gradients there ([coefficient][splat], stride kPB + 1),
// and adds all gradients to the caller's buffers with coalesced
// read-modify-writes (none where a gradient is zero: splats no pixel saw).
constexpr int kPB = 64;

// Block-wide copy of n floats from global memory into shared memory
// (put(idx, value)), U independent loads in flight per thread.
template <int U, typename Put>
__device__ __forceinline__ void stage_in(const float *__restrict__ src, int n, Put put)
{
    for (int base = threadIdx.x; base < n; base += kPB * U) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * kPB;
            v[u] = idx < n ? __ldg(src + idx) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * kPB;
            if (idx < n) put(idx, v[u]);
        }
    }
}

// Block-wide dst[idx] += get(idx) for idx < n, skipping zero addends (no
// read or write for them), U independent loads in flight per thread.
template <int U, typename Get>
__device__ __forceinline__ void add_out(float *__restrict__ dst, int n, Get get)
{
    for (int base = threadIdx.x; base < n; base += kPB * U) {
        float v[U], o[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * kPB;
            v[u] = idx < n ? get(idx) : 0.f;
            o[u] = v[u] != 0.f ? dst[idx] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * kPB;
            if (v[u] != 0.f) dst[idx] = o[u] + v[u];
        }
    }
}

template <int D>
__global__ void __launch_bounds__(kPB, 8)
project_backward_kernel(const __grid_constant__ CamTable cams, const __grid_constant__ CfgDev cfg,
                        int P, const float *__restrict__ means, const float *__restrict__ scales,
                        const float *__restrict__ quats, const float *__restrict__ opacities,
                        const float *__restrict__ sh, const float *__restrict__ grad2d,
                        float *__restrict__ g_means, float *__restrict__ g_scales,
                        float *__restrict__ g_quats, float *__restrict__ g_opac,
                        float *__restrict__ g_sh)
{
    constexpr int K = (D + 1) * (D + 1);
    constexpr int F = 3 * K, FS = F + 1, DS = kPB + 1;
    __shared__ float s_sh[kPB * FS];
    __shared__ float s_dsh[F * DS];
    __shared__ float s_io[kPB * kIO];
    const int i0 = blockIdx.x * kPB;
    const int nb = min(kPB, P - i0);
    // (source, floats per splat, first slot in the io row)
    const float *src[4] = {means, scales, quats, opacities};
    float *gdst[4] = {g_means, g_scales, g_quats, g_opac};
    constexpr int kW[4] = {3, 3, 4, 1}, kOff[4] = {0, 3, 6, 10};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int wa = kW[a], oa = kOff[a];
        stage_in<4>(src[a] + (size_t)i0 * wa, nb * wa, [&](int idx, float v) {
            const int r = idx / wa;
            s_io[r * kIO + oa + idx - r * wa] = v;
        });
    }
    stage_in<16>(sh + (size_t)i0 * F, nb * F, [&](int idx, float v) {
        const int r = idx / F;
        s_sh[r * FS + idx - r * F] = v;
    });
    for (int k = threadIdx.x; k < F * DS; k += kPB) s_dsh[k] = 0.f;
    __syncthreads();
    const int i = i0 + (int)threadIdx.x;
    if (i < P) project_backward_splat<D>(cams, cfg, P, i, s_io + threadIdx.x * kIO, s_sh + threadIdx.x * FS,
                                         s_dsh + threadIdx.x, DS, grad2d);
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int wa = kW[a], oa = kOff[a];
        add_out<4>(gdst[a] + (size_t)i0 * wa, nb * wa, [&](int idx) {
            const int r = idx / wa;
            return s_io[r * kIO + oa + idx - r * wa];
        });
    }
    add_out<12>(g_sh + (size_t)i0 * F, nb * F, [&](int idx) {
        const int r = idx / F;
        return s_dsh[(idx - r * F) * DS + r];
    });
}

} // namespace
} // namespace gs

using namespace gs;

extern "C" size_t gs_grad2d_bytes(int32_t ncam, int32_t P)
{
    if (ncam <= 0 || P < 0) return 0;
    return align256(sizeof(float) * kG2 * (size_t)ncam * P);
}

extern "C" gs_status gs_render_backward(void *stream, const gs_camera *cams, int32_t ncam, int32_t P,
                                        const gs_config *cfg, const float *d_means,
                                        const float *d_scales, const float *d_quats,
                                        const float *d_opacities, const float *d_sh,
                                        int32_t sh_degree, const void *d_splat2d,
                                        const uint32_t *d_vals, const uint32_t *d_ranges,
                                        const float *bg, const float *d_final_T,
                                        const uint32_t *d_last, const float *d_grad_out,
                                        void *d_grad2d, float *d_grad_means, float *d_grad_scales,
                                        float *d_grad_quats, float *d_grad_opacities,
                                        float *d_grad_sh)
{
    if (!cams || !cfg || !bg || ncam <= 0 || ncam > kMaxCams || P < 0 || sh_degree < 0 || sh_degree > 3)
        return GS_ERR_ARG;
    if (P == 0) return GS_OK;
    if (!d_means || !d_scales || !d_quats || !d_opacities || !d_sh || !d_splat2d || !d_vals ||
        !d_ranges || !d_final_T || !d_last || !d_grad_out || !d_grad2d || !d_grad_means ||
        !d_grad_scales || !d_grad_quats || !d_grad_opacities || !d_grad_sh)
        return GS_ERR_ARG;
    if (((uintptr_t)d_quats & 15) || ((uintptr_t)d_splat2d & 255) || ((uintptr_t)d_grad2d & 15))
        return GS_ERR_ARG;
    CamTable t;
    CfgDev c;
    if (!build_cam_table(cams, ncam, cfg, &t) || !build_cfg(cfg, &c)) return GS_ERR_ARG;
    if (cfg->tile_w * cfg->tile_h > 512) return GS_ERR_UNSUPPORTED; // 256 threads of two pixels
    // the reverse pass recomputes alpha in FP32; an FP16x2 forward could have
    // taken different skip / stop decisions
    if (cfg->fp16x2 || cfg->tensor_alpha) return GS_ERR_UNSUPPORTED;
    const int64_t N = (int64_t)ncam * P;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_grad2d, 0, gs_grad2d_bytes(ncam, P), s) != cudaSuccess) return GS_ERR_CUDA;
    const float4 *rec = splat2d_const(d_splat2d, N).rec;
    const uint2 *rg = reinterpret_cast<const uint2 *>(d_ranges);
    float *g2 = static_cast<float *>(d_grad2d);
    // two pixels per thread (tile widths are even; one per thread otherwise)
    const int ppt = (cfg->tile_w % 2 == 0) ? 2 : 1;
    if (cfg->tile_w * cfg->tile_h / ppt > 256) return GS_ERR_UNSUPPORTED;
    const int threads = cfg->tile_w * cfg->tile_h / ppt;
    const size_t smem = bwd_smem_bytes(threads);
#define GS_BWD_LAUNCH(K, PP)                                                                         \
    blend_backward_kernel<K, PP><<<t.total_tiles, threads, smem, s>>>(t, c, rec, d_vals, rg, (uint32_t)N, \
                                                                   bg[0], bg[1], bg[2], d_final_T,   \
                                                                   d_last, d_grad_out, g2)
#define GS_BWD_KIND(PP)                                                                              \
    switch (cfg->kind) {                                                                             \
    case GS_K_EXP: GS_BWD_LAUNCH(GS_K_EXP, PP); break;                                               \
    case GS_K_POLY1: GS_BWD_LAUNCH(GS_K_POLY1, PP); break;                                           \
    case GS_K_POLY2: GS_BWD_LAUNCH(GS_K_POLY2, PP); break;                                           \
    default: GS_BWD_LAUNCH(GS_K_POLY3, PP); break;                                                   \
    }
    if (ppt == 2) {
        GS_BWD_KIND(2)
    } else {
        GS_BWD_KIND(1)
    }
#undef GS_BWD_KIND
#undef GS_BWD_LAUNCH
    count_launch();
    GS_LAUNCH_CHECK();
    const int pt = kPB, pb = (P + pt - 1) / pt;
#define GS_PBWD_LAUNCH(D)                                                                          \
    project_backward_kernel<D><<<pb, pt, 0, s>>>(t, c, P, d_means, d_scales, d_quats, d_opacities, \
                                                 d_sh, g2, d_grad_means, d_grad_scales,            \
                                                 d_grad_quats, d_grad_opacities, d_grad_sh)
    switch (sh_degree) {
    case 0: GS_PBWD_LAUNCH(0); break;
    case 1: GS_PBWD_LAUNCH(1); break;
    case 2: GS_PBWD_LAUNCH(2); break;
    default: GS_PBWD_LAUNCH(3); break;
    }
#undef GS_PBWD_LAUNCH
    count_launch();
    GS_LAUNCH_CHECK();
    return GS_OK;
}
