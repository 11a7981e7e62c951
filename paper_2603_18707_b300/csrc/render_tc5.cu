// render_tc5.cu — the quadric of every (pixel, splat) pair on the fifth-
// generation tensor cores (tcgen05, TMEM accumulators), sm_103a.
//
// The paper's Sec. 5.1 argument (a matrix engine evaluates the quadric for
// many pixels and splats at once) for a 16x16 tile:
//   Q[p][s] = sum_k Phi[p][k] W[s][k],  k < 8,
// Phi = (x^2, x y, y^2, x, y, 1, 0, 0) of the tile-centred pixel position and
// W = (A, 2B, C, -2(A dx0 + B dy0), -2(B dx0 + C dy0), Q(tile centre), 0, 0)
// of the splat (conic (A, B, C), mean offset (dx0, dy0) from the tile centre).
// Phi is exact in TF32 (quarter integers below 57); W is split into two TF32
// parts, hi + lo, so that Phi W_lo + Phi W_hi carries W's FP32 precision.
//
// One CTA per tile, 256 threads, one pixel per thread (thread t = pixel t of
// the row-major tile). Phi sits in shared memory once, as two 128-row K-major
// operands (the canonical no-swizzle layout: 8-row x 16-byte core matrices,
// 128 bytes apart along K, 256 bytes apart along M). Per batch of kT5B splats
// the threads write W_hi and W_lo in the same layout; one thread issues four
// tcgen05.mma.kind::tf32 (M = 128 pixels, N = kT5B splats, K = 8: two pixel
// halves x {lo, hi}) into a TMEM accumulator of 2 kT5B columns and commits
// them to an mbarrier. Every thread waits on it (bounded), reads its pixel's
// row with tcgen05.ld (warp w reaches TMEM lanes 32 (w mod 4) ..; half w / 4
// is the column block), and composites in FP32 with the thresholds and order
// of the FP32 path. f1 and exp are affine in Q, so their opacity-folded
// coefficients go into the weights (W' = p1 W, plus p0 on the constant
// monomial): the accumulator holds f1's alpha, or exp's exponent, directly,
// and a pixel-entry below eps costs one compare. f'2 and f3 read Q and
// evaluate their polynomial (alpha_of_q). Forward only.
#include <algorithm>

#include "blend_math.cuh"

namespace gs {
namespace {

constexpr int kT5B = 64;              // splats per batch: the MMA's N
constexpr int kT5Cols = 2 * kT5B;     // TMEM columns: one N-wide block per pixel half
constexpr int kT5Spin = 1 << 16;      // mbarrier polls before a wait gives up
// Dynamic shared memory per CTA. The operands need ~14 KB; asking for 56 KB
// keeps at most four CTAs on an SM (228 KB), so that four 128-column TMEM
// allocations always fit in the SM's 512 columns and tcgen05.alloc never waits.
constexpr int kT5Smem = 56 * 1024;
// Instruction descriptor of tcgen05.mma .kind::tf32: D FP32 (bits 4-5 = 1),
// A and B TF32 (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kT5Idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kT5B >> 3) << 17) |
                              ((128u >> 4) << 24);

__device__ uint32_t g_tc5_err; // GS_ERR_TIMEOUT when a wait gave up (read by gs_render_status_async)

struct __align__(16) T5Smem {
    uint32_t a[2][16][2][8][4];      // Phi: pixel half, 8-row group, K chunk, row, element (8 KB)
    uint32_t bhi[kT5B / 8][2][8][4]; // W_hi: 8-splat group, K chunk, row, element (2 KB)
    uint32_t blo[kT5B / 8][2][8][4]; // W_lo
    float4 coef_b[kT5B];             // per splat: v0, p0, p1, p2 (blend_math.cuh make_coef)
    float4 coef_c[kT5B];             // per splat: colour, p3
    unsigned long long mbar;         // MMA completion
    uint32_t tmem;                   // TMEM address written by tcgen05.alloc
};

__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K)
// byte offset and stride (M / N) byte offset, each >> 4; bits 46-48 = 0b001;
// base offset 0; no swizzle.
__device__ __forceinline__ unsigned long long smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)(lbo >> 4) << 16) |
           ((unsigned long long)(sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, unsigned long long adesc, unsigned long long bdesc,
                                         uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %3, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %4, p;\n\t}"
                 ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(accumulate), "r"(kT5Idesc)
                 : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Polls the mbarrier for the completion of phase `parity`, at most `limit`
// times; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int limit)
{
    for (int i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// 16 consecutive accumulator columns of this warp's 32 TMEM lanes: lane l
// receives row (lane base + l), columns c .. c + 15.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&q)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]),
                   "=r"(q[7]), "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]),
                   "=r"(q[14]), "=r"(q[15])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int KIND>
__global__ void __launch_bounds__(256, 4) // four CTAs per SM: the TMEM and shared-memory plan
render_tc5_kernel(const __grid_constant__ CamTable cams, const __grid_constant__ CfgDev cfg,
                  const __grid_constant__ RenderArgs g)
{
    // f1 and exp: the MMA yields alpha / the exponent (see the file header)
    constexpr bool AFFINE = KIND == GS_K_POLY1 || KIND == GS_K_EXP;
    extern __shared__ __align__(1024) unsigned char t5_smem[];
    T5Smem &S = *reinterpret_cast<T5Smem *>(t5_smem);
    const int gtile = blockIdx.x;
    int c = 0;
    while (c + 1 < cams.ncam && cams.cam[c + 1].tile_base <= gtile) ++c;
    const CamDev &cm = cams.cam[c];
    const int lt = gtile - cm.tile_base;
    const int tx = lt % cm.tiles_x, ty = lt / cm.tiles_x;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int lx = tid & 15, ly = tid >> 4;
    const int px = tx * 16 + lx, py = ty * 16 + ly;
    const float ox = (float)(tx * 16), oy = (float)(ty * 16);
    const float ocx = ox + 8.f, ocy = oy + 8.f; // tile centre
    const uint2 rg = g.ranges[gtile];
    // an empty or inverted range (only possible after a timed-out sort wait)
    // reads nothing: every range gs_bin_sort writes lies within its output
    const uint32_t n = rg.y > rg.x ? rg.y - rg.x : 0u;
    const float eps = cfg.eps, amax = cfg.alpha_max, tmin = cfg.t_min;

    // Phi row of this thread's pixel (row tid: half tid / 128, row tid mod 128)
    {
        const float xc = lx + 0.5f - 8.f, yc = ly + 0.5f - 8.f;
        const int h = tid >> 7, r = tid & 127;
        uint32_t *row0 = &S.a[h][r >> 3][0][r & 7][0], *row1 = &S.a[h][r >> 3][1][r & 7][0];
        *reinterpret_cast<uint4 *>(row0) = make_uint4(to_tf32(xc * xc), to_tf32(xc * yc), to_tf32(yc * yc), to_tf32(xc));
        *reinterpret_cast<uint4 *>(row1) = make_uint4(to_tf32(yc), to_tf32(1.f), 0u, 0u);
    }
    const uint32_t mbar = smem_u32(&S.mbar);
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                     "r"(kT5Cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem(); // Phi and the mbarrier, visible to the tensor core's (async) proxy
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const unsigned long long desc_a0 = smem_desc(smem_u32(&S.a[0][0][0][0][0]), 128, 256);
    const unsigned long long desc_a1 = smem_desc(smem_u32(&S.a[1][0][0][0][0]), 128, 256);
    const unsigned long long desc_hi = smem_desc(smem_u32(&S.bhi[0][0][0][0]), 128, 256);
    const unsigned long long desc_lo = smem_desc(smem_u32(&S.blo[0][0][0][0]), 128, 256);
    // this warp's TMEM lanes and column block
    const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * kT5B);

    bool active = px < cm.W && py < cm.H;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t lastc = 0, ne = n, parity = 0;
    // affine kernels: the accumulator's value that can reach eps (exp: its
    // exponent, 2^-8 below log2 eps so that ex2's rounding decides), +inf once
    // the pixel has stopped or lies off the frame
    const float thr_on = KIND == GS_K_EXP ? log2f(eps) - 1.f / 256.f : eps;
    float thr = active ? thr_on : INFINITY;
    bool failed = false;
    // the records of a batch are gathered one batch ahead (by the threads
    // that stage them), so that the loads overlap the previous batch's MMA
    // and compositing
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
    const auto gather = [&](uint32_t b) {
        if (tid < kT5B && b + tid < n) {
            uint32_t v = g.vals[rg.x + b + tid];
            if (v >= g.n_records) v = 0; // only after a timed-out sort wait
            r0 = g.rec[3 * (size_t)v + 0];
            r1 = g.rec[3 * (size_t)v + 1];
            r2 = g.rec[3 * (size_t)v + 2];
        }
    };
    gather(0);
    for (uint32_t base = 0; base < n; base += kT5B) {
        if (__syncthreads_count(active) == 0) break;
        const int cnt = (int)min((uint32_t)kT5B, n - base);
        if (tid < kT5B) {
            float w[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float4 bb = make_float4(0.f, 0.f, 0.f, 0.f), cc = bb;
            if (tid < cnt) {
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
                if (AFFINE) { // alpha (f1) or exponent (exp) = p0 + p1 Q
#pragma unroll
                    for (int kk = 0; kk < 6; ++kk) w[kk] *= k.b.z;
                    w[5] += k.b.y;
                }
            } else if (AFFINE) {
                w[5] = -1e30f; // padding: below any threshold
            }
            uint32_t hi[8], lo[8];
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                hi[kk] = to_tf32(w[kk]);
                lo[kk] = to_tf32(w[kk] - __uint_as_float(hi[kk]));
            }
            const int grp = tid >> 3, row = tid & 7;
            *reinterpret_cast<uint4 *>(&S.bhi[grp][0][row][0]) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(&S.bhi[grp][1][row][0]) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
            *reinterpret_cast<uint4 *>(&S.blo[grp][0][row][0]) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            *reinterpret_cast<uint4 *>(&S.blo[grp][1][row][0]) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
            S.coef_b[tid] = bb;
            S.coef_c[tid] = cc;
        }
        fence_async_smem();
        tc_fence_before(); // the previous batch's TMEM reads come before the next MMAs
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            mma_tf32(tmem, desc_a0, desc_lo, 0u); // small parts first
            mma_tf32(tmem, desc_a0, desc_hi, 1u);
            mma_tf32(tmem + kT5B, desc_a1, desc_lo, 0u);
            mma_tf32(tmem + kT5B, desc_a1, desc_hi, 1u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                         : "memory");
        }
        gather(base + kT5B); // the next batch's records, while the MMAs run
        const bool ok = mbar_wait(mbar, parity, kT5Spin);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        tc_fence_after();
        for (int c0 = 0; c0 < cnt; c0 += 16) {
            if (!__any_sync(0xffffffffu, active)) break; // warp-uniform: tcgen05.ld is warp-wide
            uint32_t q[16];
            tmem_ld16(taddr + (uint32_t)c0, q);
            if constexpr (AFFINE) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float x = __uint_as_float(q[j]);
                    if (!(x >= thr)) continue; // padding entries lie far below
                    const float al0 = KIND == GS_K_EXP ? ex2_approx(x) : x;
                    if (!(al0 >= eps)) continue;
                    const float4 cj = S.coef_c[c0 + j];
                    const float al = fminf(amax, al0);
                    const float Tn = fmaf(-al, T, T);
                    const uint32_t pos = base + c0 + j + 1;
                    if (Tn < tmin) {
                        active = false;
                        thr = INFINITY;
                        ne = pos;
                        continue;
                    }
                    const float wgt = al * T;
                    C0 = fmaf(cj.x, wgt, C0);
                    C1 = fmaf(cj.y, wgt, C1);
                    C2 = fmaf(cj.z, wgt, C2);
                    T = Tn;
                    lastc = pos;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (!active || c0 + j >= cnt) continue;
                    const float4 cj = S.coef_c[c0 + j];
                    const float al0 = alpha_of_q<KIND>(cfg, S.coef_b[c0 + j], cj.w, __uint_as_float(q[j]));
                    if (!(al0 >= eps)) continue;
                    const float al = fminf(amax, al0);
                    const float Tn = fmaf(-al, T, T);
                    const uint32_t pos = base + c0 + j + 1;
                    if (Tn < tmin) {
                        active = false;
                        ne = pos;
                        continue;
                    }
                    const float wgt = al * T;
                    C0 = fmaf(cj.x, wgt, C0);
                    C1 = fmaf(cj.y, wgt, C1);
                    C2 = fmaf(cj.z, wgt, C2);
                    T = Tn;
                    lastc = pos;
                }
            }
        }
    }
    if (failed) {
        if (tid == 0) atomicOr(&g_tc5_err, (uint32_t)GS_ERR_TIMEOUT);
        (void)mbar_wait(mbar, parity ^ 1u, kT5Spin); // the MMAs in flight, once more (bounded)
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kT5Cols) : "memory");
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

// One thread waits on an mbarrier that expects one arrival and gets none.
__global__ void tc5_wait_selftest_kernel(uint32_t *err, int limit)
{
    __shared__ unsigned long long mb;
    const uint32_t a = smem_u32(&mb);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    if (!mbar_wait(a, 0u, limit)) atomicOr(err, (uint32_t)GS_ERR_TIMEOUT);
}

template <int KIND>
cudaError_t launch_kind(cudaStream_t s, const CamTable &t, const CfgDev &c, const RenderArgs &g)
{
    // the shared-memory opt-in is set once per device (so that later calls,
    // e.g. under stream capture, only launch)
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError();
    if (dev >= 64 || !attr_set[dev]) {
        const cudaError_t e =
            cudaFuncSetAttribute(render_tc5_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, kT5Smem);
        if (e != cudaSuccess) return e;
        if (dev < 64) attr_set[dev] = true;
    }
    render_tc5_kernel<KIND><<<t.total_tiles, 256, kT5Smem, s>>>(t, c, g);
    return cudaPeekAtLastError();
}

} // namespace

static_assert(sizeof(T5Smem) <= kT5Smem, "tcgen05 blend: operands exceed the shared memory asked for");

cudaError_t launch_render_tc5(int kind, cudaStream_t s, const CamTable &t, const CfgDev &c, const RenderArgs &g)
{
    switch (kind) {
    case GS_K_EXP: return launch_kind<GS_K_EXP>(s, t, c, g);
    case GS_K_POLY1: return launch_kind<GS_K_POLY1>(s, t, c, g);
    case GS_K_POLY2: return launch_kind<GS_K_POLY2>(s, t, c, g);
    default: return launch_kind<GS_K_POLY3>(s, t, c, g);
    }
}

cudaError_t launch_tc5_wait_selftest(cudaStream_t s, uint32_t *err, int limit)
{
    tc5_wait_selftest_kernel<<<1, 1, 0, s>>>(err, limit);
    return cudaPeekAtLastError();
}

} // namespace gs

using namespace gs;

extern "C" gs_status gs_render_status_async(void *stream, uint32_t *dst)
{
    if (!dst) return GS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tc5_err) != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    if (cudaMemcpyAsync(dst, p, sizeof(uint32_t), cudaMemcpyDefault, s) != cudaSuccess ||
        cudaMemsetAsync(p, 0, sizeof(uint32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    return GS_OK;
}
