/*
 * gs.h — C ABI of the B300 (sm_103a) tile-based Gaussian splatting renderer
 * with the exponential kernel and the polynomial-plus-ReLU kernels of
 * "From ex(p) to poly: Gaussian Splatting with Polynomial Kernels"
 * (Mueller, Winter, Steinberger; arXiv 2603.18707).
 *
 * Pipeline (one stream, all stream-ordered):
 *   gs_preprocess       project splats into every camera, per-splat support
 *                       threshold and tile rectangle (Eq. 1, Eq. 3-6, Sec. 3.4, App. B)
 *   gs_bin_sort         depth order + tile binning: compaction, depth radix
 *                       sort, row and column splits, per-tile ranges
 *   gs_render           front-to-back alpha blending per tile (Sec. 2, Eq. 1/2/6)
 *   gs_render_backward  reverse blend + chain rule to the splat inputs (Sec. 4.3)
 * Scene preparation (once per scene, not per frame):
 *   gs_spatial_order    Z-order permutation of the splats; gs_gather_rows applies it
 *
 * Conventions shared by every entry point:
 *  - Pointers named d_* are DEVICE pointers; everything else is host memory.
 *  - The caller allocates every buffer; no entry point allocates or frees
 *    device or host memory. Workspace sizes come from the *_bytes queries.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued asynchronously; host-side arguments (cameras, config)
 *    are copied into kernel parameters before the call returns.
 *  - Errors: every call returns gs_status. Argument errors are detected on
 *    the host before anything is launched. Conditions only the device can see
 *    (overlap capacity exceeded, a bounded spin-wait that timed out) are OR-ed
 *    into an error word inside the bin/sort workspace; read it with
 *    gs_workspace_status. No entry point exits, traps or prints.
 *  - Floating point: every device computation is FP32 (FP16x2 where the config
 *    asks for it); no FP64 on the device.
 *  - Splat inputs are the activated values the paper's Sec. 2 names: means mu
 *    [P][3]; scales s [P][3] (> 0); rotation quaternions q [P][4] in
 *    (w, x, y, z) order (any non-zero norm: they are normalised internally);
 *    opacities o [P] in [0, 1]; SH coefficients [P][(d+1)^2][3], degree d <= 3.
 *    All row-major FP32.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_ABI_VERSION 1
#define GS_MAX_CAMERAS 64

typedef enum {
    GS_OK = 0,
    GS_ERR_ARG = 1,         /* invalid argument (host check, nothing launched) */
    GS_ERR_CUDA = 2,        /* a CUDA launch or copy failed */
    GS_ERR_CAPACITY = 4,    /* device: more tile overlaps than the given capacity */
    GS_ERR_TIMEOUT = 8,     /* device: a bounded spin-wait gave up */
    GS_ERR_UNSUPPORTED = 16 /* valid but not implemented for this config */
} gs_status;

/* Kernel k(x) on the quadric x = Q(v) (Sec. 3):
 *   GS_K_EXP   g(x) = exp(-x/2)                                  (Eq. 1)
 *   GS_K_POLY1 f1(x) = max(c0 + c1 x, 0)                         (Eq. 2)
 *   GS_K_POLY2 f'2(x) = c0 + c1 x + c2 x^2 if x < x0, else 0     (Eq. 6)
 *   GS_K_POLY3 f3(x) = max(c0 + c1 x + c2 x^2 + c3 x^3, 0)      (Eq. 2)
 * x0 is the first positive root of the polynomial. */
typedef enum { GS_K_EXP = 0, GS_K_POLY1 = 1, GS_K_POLY2 = 2, GS_K_POLY3 = 3 } gs_kernel_kind;

/* Support threshold (culling radius), in quadric units:
 *   GS_CULL_UNIVERSAL opacity-free: poly x0 (Eq. 5, App. B with eps = 0);
 *                     exp -2 ln(eps) (3.3 sigma, Sec. 3.1)
 *   GS_CULL_OPACITY   per splat: exp 2 ln(o'/eps) (Eq. 3); f1 (eps - o' c0)/(o' c1)
 *                     (Eq. 4); f'2/f3 first root of poly = eps/o' (App. B);
 *                     splats with o' k(0) < eps are dropped
 *   GS_CULL_LEGACY3   3 sigma (x = 9) of the original 3DGS (Sec. 2.1); not
 *                     pixel-exact for exp */
typedef enum { GS_CULL_UNIVERSAL = 0, GS_CULL_OPACITY = 1, GS_CULL_LEGACY3 = 2 } gs_cull;

/* Which tiles a splat is binned to, around its support ellipse
 * {d : d^T conic d <= x_cut}: every tile of the ellipse's exact axis-aligned
 * bounding box (AABB); of the 3DGS square around the circle of radius
 * sqrt(x_cut * lambda_max) (CIRCLE); or, per tile row, only the tiles whose
 * pixel centres the ellipse can reach (ELLIPSE: the per-tile test of
 * StopThePop that the paper's Baseline uses, Sec. 2.1, done analytically row
 * by row). All three are conservative: the image is the same. */
typedef enum { GS_RECT_AABB = 0, GS_RECT_CIRCLE = 1, GS_RECT_ELLIPSE = 2 } gs_rect_mode;

/* Pinhole camera. viewmat: world -> camera, row-major 4x4; camera looks
 * along +z with +x right and +y down. A world point p maps to
 * t = R p + T and to pixel coordinates (fx tx/tz + cx, fy ty/tz + cy);
 * pixel (i, j) has its centre at (i + 0.5, j + 0.5). Splats with
 * tz <= znear are dropped. */
typedef struct {
    float viewmat[16];
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear;
    int32_t reserved;
} gs_camera;

typedef struct {
    int32_t kind;         /* gs_kernel_kind */
    float c[4];           /* polynomial coefficients c0..c3 (unused ones 0) */
    int32_t cull;         /* gs_cull */
    float eps;            /* alpha threshold, 1/255 (Sec. 3.1) */
    float alpha_max;      /* alpha clamp, 0.99 (3DGS) */
    float t_min;          /* transmittance stop, 1e-4 (3DGS) */
    int32_t aa_normalize; /* 1: o' = o sqrt(|Sigma'| / |Sigma' + v I|) (Sec. 3.4) */
    float aa_dilation;    /* v added to the 2D covariance diagonal, 0.3 */
    int32_t tile_w;       /* tile width in pixels: 8, 16 or 32 */
    int32_t tile_h;       /* tile height in pixels: 8, 16 or 32; at most 512 pixels per
                             tile, and at most 256 threads (tile pixels / px_per_thread)
                             in the blend; the reverse pass needs tiles of <= 256 pixels */
    int32_t rect_mode;    /* gs_rect_mode */
    int32_t batch;        /* splats staged in shared memory per round: 32..256 */
    int32_t px_per_thread;/* pixels per thread in the blend: 1, 2 or 4 */
    int32_t fp16x2;       /* 1: quadric and polynomial in packed FP16x2 */
    int32_t tensor_alpha; /* quadric of every (pixel, splat) pair on the tensor cores
                             (Sec. 5.1), weights split in two TF32 parts: 1 warp-level
                             mma.sync TF32 (32 splats per batch); 2 tcgen05.mma
                             kind::tf32 into TMEM (64 splats per batch, M = 128).
                             Needs 16x16 tiles, fp16x2 = 0 and the one-CTA-per-tile
                             launch; forward only (gs_render_backward:
                             GS_ERR_UNSUPPORTED) */
    int32_t reserved[3];
} gs_config;

/* Fills a config with the defaults above for a kernel kind (plus 16x16
 * tiles, GS_RECT_AABB, batch 256, 4 pixels per thread, FP32). f1 uses the
 * paper's coefficients (Sec. 3.1, with the printed c0/c1 labels swapped:
 * c0 = 0.773, c1 = -0.773/4.386, root 4.386); f'2 and f3 use this library's
 * L1 fits by the Sec. 3.1 procedure (the paper does not print them). */
gs_status gs_config_default(int32_t kind, int32_t cull, gs_config *cfg);

/* Byte size of the per-(camera, splat) record buffer that gs_preprocess
 * writes and the later stages read, for ncam * P records. Layout, with
 * N = ncam * P and records camera-major (index c * P + i):
 *   float4 rec[N][3]   (mean.x, mean.y, o', depth), (A, B, C, x_cut),
 *                      (red, green, blue, rho) with conic (A, B, C) = (Sigma'+vI)^-1
 *                      and rho the AA factor
 *   uint16 rect[N][4]  tile x0, y0, x1, y1 (inclusive) of the support rectangle
 *   uint32 tiles[N]    number of tiles in rect; 0 = splat not drawn
 *   uint32 dkey[N]     float bits of depth
 *   rec, rect and dkey are written only for records with tiles > 0.
 * each array 256-byte aligned. */
size_t gs_splat2d_bytes(int32_t ncam, int32_t P);

/* Projection of P splats into ncam cameras (ncam <= GS_MAX_CAMERAS): EWA
 * covariance Sigma' = J W Sigma W^T J^T + v I (Eq. 1; 3DGS), the AA factor of
 * Sec. 3.4, conic, depth, SH colour (3DGS real SH + 0.5, clamped at 0),
 * support threshold x_cut (Eq. 3-5, App. B) and tile rectangle.
 * d_splat2d: gs_splat2d_bytes(ncam, P) bytes of device memory. */
gs_status gs_preprocess(void *stream, const gs_camera *cams, int32_t ncam, int32_t P,
                        const float *d_means, const float *d_scales, const float *d_quats,
                        const float *d_opacities, const float *d_sh, int32_t sh_degree,
                        const gs_config *cfg, void *d_splat2d);

/* Total tile count over all cameras; the global tile id of camera c's tile
 * (tx, ty) is base_c + ty * ceil(W_c / tile_w) + tx, cameras in order. */
int64_t gs_total_tiles(const gs_camera *cams, int32_t ncam, const gs_config *cfg);

/* Workspace bytes for gs_bin_sort with these cameras and tile shape, P
 * splats and room for `capacity` splat-tile overlaps; 0 for invalid
 * arguments (the checks of gs_bin_sort). */
size_t gs_bin_sort_workspace_bytes(const gs_camera *cams, int32_t ncam, int32_t P,
                                   const gs_config *cfg, int64_t capacity);

/* Depth-ordered tile binning of the records written by gs_preprocess.
 * Result: for global tile t, d_vals[d_ranges[2t] .. d_ranges[2t+1]) are the
 * record indices (c * P + i) of the splats whose rectangle contains t, in
 * increasing (depth, i) order — a stable sort of the 64-bit keys
 * (tile << 32 | depth bits) 3DGS uses. Implemented as a stable LSD radix sort
 * of each camera's drawn records by depth (Onesweep: one pass per 8-bit
 * digit, decoupled look-back with a bounded wait), then two stable splits of
 * the depth-sorted records: by tile row (one span per covered row) and by
 * tile column, the latter writing every record index to its final place.
 * Tiles of a camera: at most 2048 per row and per column.
 *   d_vals:      uint32 [capacity]
 *   d_ranges:    uint32 [2 * total_tiles] (start, end) per tile; (0, 0)
 *                for a tile that no record covers
 *   d_keys64:    optional uint64 [capacity] (may be NULL): the sorted keys
 *   d_count:     optional uint32 [3] (may be NULL): drawn records, overlaps
 *                stored, overlaps counted (the capacity needed)
 * Overlaps beyond `capacity` are dropped and GS_ERR_CAPACITY is raised in the
 * workspace error word (the ranges then stay inside [0, capacity)). At most
 * 2^30 - 1 records and overlaps per call. */
gs_status gs_bin_sort(void *stream, const gs_camera *cams, int32_t ncam, int32_t P,
                      const gs_config *cfg, const void *d_splat2d, int64_t capacity,
                      void *d_workspace, size_t workspace_bytes, uint32_t *d_vals,
                      uint32_t *d_ranges, uint64_t *d_keys64, uint32_t *d_count);

/* Front-to-back blending per tile (Sec. 2): for each pixel, over its tile's
 * list in order, alpha = min(alpha_max, o' k(Q)) with Q the quadric at the
 * pixel centre; entries with alpha < eps are skipped; the walk stops at the
 * first entry whose T (1 - alpha) would drop below t_min, without adding it;
 * out = sum c alpha T + T bg.
 *   d_out_rgb:   float [sum_c H_c W_c][3], cameras back to back, row-major
 *   d_final_T:   float [sum_c H_c W_c] (may be NULL)
 *   d_last:      uint32 [sum_c H_c W_c] 1 + list position of the last
 *                contributing entry, 0 if none (may be NULL; the backward
 *                pass needs it)
 *   d_n_eval:    uint32 [sum_c H_c W_c] list entries evaluated (may be NULL)
 *                With d_last and d_n_eval both NULL the blend keeps no
 *                per-pixel list positions and runs faster; the image and
 *                d_final_T are the same bit for bit.
 *   bg:          host float[3] background colour
 *   d_work:      NULL for one CTA per tile; otherwise gs_render_work_bytes()
 *                bytes of device memory (4-byte aligned) and the blend runs as
 *                one persistent launch: a grid that fills every SM once, each
 *                CTA taking the next tile of any camera from a counter in
 *                d_work (reset by the call, on the stream).
 * Pixel values do not depend on px_per_thread, batch or the launch mode; the
 * tile shape changes only FP32 rounding (the per-tile coefficients are taken
 * relative to the tile's corner). */
size_t gs_render_work_bytes(void);
gs_status gs_render(void *stream, const gs_camera *cams, int32_t ncam, int32_t P,
                    const gs_config *cfg, const void *d_splat2d, const uint32_t *d_vals,
                    const uint32_t *d_ranges, const float *bg, float *d_out_rgb,
                    float *d_final_T, uint32_t *d_last, uint32_t *d_n_eval, void *d_work);

/* Device error word of the blend: GS_ERR_TIMEOUT when a bounded wait of the
 * tcgen05 tensor-core variant (tensor_alpha = 2) gave up (its tiles are then
 * incomplete). One word per device, shared by every gs_render call of the
 * process: enqueues on `stream` a copy of it to dst (uint32, device or pinned
 * host memory) and clears it. GS_ERR_ARG for a null dst, GS_ERR_CUDA if a copy
 * cannot be enqueued. */
gs_status gs_render_status_async(void *stream, uint32_t *dst);

/* Reverse pass of gs_render and gs_preprocess for one or more cameras:
 * gradients of a loss L with respect to the splat inputs, given
 * dL/d(out_rgb). Needs the forward's d_final_T and d_last. Output gradient
 * buffers are ACCUMULATED into (the caller zeroes them): d_grad_means [P][3],
 * d_grad_scales [P][3], d_grad_quats [P][4] (for the quaternion as given,
 * before normalisation), d_grad_opacities [P], d_grad_sh [P][(d+1)^2][3].
 * d_grad2d: scratch of gs_grad2d_bytes(ncam, P) bytes (zeroed by the call).
 * Tiles of up to 512 pixels (two pixels per thread); larger tiles, and a
 * forward run with fp16x2 or tensor_alpha (whose skip / stop decisions the
 * FP32 reverse pass could not reproduce), return GS_ERR_UNSUPPORTED. */
size_t gs_grad2d_bytes(int32_t ncam, int32_t P);
gs_status gs_render_backward(void *stream, const gs_camera *cams, int32_t ncam, int32_t P,
                             const gs_config *cfg, const float *d_means,
                             const float *d_scales, const float *d_quats,
                             const float *d_opacities, const float *d_sh, int32_t sh_degree,
                             const void *d_splat2d, const uint32_t *d_vals,
                             const uint32_t *d_ranges, const float *bg,
                             const float *d_final_T, const uint32_t *d_last,
                             const float *d_grad_out, void *d_grad2d,
                             float *d_grad_means, float *d_grad_scales, float *d_grad_quats,
                             float *d_grad_opacities, float *d_grad_sh);

/* gs_bin_sort for callers that cannot allocate device memory — a plugin
 * whose host application owns all device allocations through its own pool,
 * or a real-time frame loop that may not allocate once it is running. The
 * paper has no counterpart; this is a deployment convenience of this library.
 *
 * Same arguments, results and errors as gs_bin_sort, minus the workspace: the
 * scratch is one fixed array of GS_NOALLOC_WORKSPACE_BYTES in static device
 * memory, held until the process exits. Sizes whose workspace
 * (gs_bin_sort_workspace_bytes(cams, ncam, P, cfg, capacity): about 17 bytes
 * per record plus 8 bytes per overlap of capacity) would not fit are
 * rejected with GS_ERR_ARG before anything is launched.
 *  - Set-up happens in the first call on each device: with that device
 *    current it looks up the array's device address and caches it. Under
 *    CUDA's lazy module loading (the default) that lookup is also what loads
 *    this part of the library's device code, and with it reserves the array:
 *    the first call can therefore allocate, take time, and fail with
 *    GS_ERR_CUDA if the device is out of memory. Make that first call at
 *    set-up time (a call with P = 0 is enough), before any stream capture and
 *    before the loop that must not allocate. Later calls allocate nothing.
 *  - All calls on a device share the one array; each call clears the parts
 *    that must start at zero. Calls that overlap on the GPU (other streams,
 *    or host threads without ordering between them) race: serialise them.
 *  - d_error (optional, may be NULL): uint32, device or pinned host memory;
 *    receives, stream-ordered at the end of the call, the device error word
 *    of this call (OR of GS_ERR_CAPACITY and GS_ERR_TIMEOUT, 0 if none).
 *    The word lives in the shared array, so gs_workspace_status cannot reach
 *    it: without d_error a timed-out wait goes unseen (an overflowing
 *    capacity still shows in d_count: overlaps counted > capacity). */
#define GS_NOALLOC_WORKSPACE_BYTES ((size_t)32 << 20)
gs_status gs_bin_sort_noalloc(void *stream, const gs_camera *cams, int32_t ncam, int32_t P,
                              const gs_config *cfg, const void *d_splat2d, int64_t capacity,
                              uint32_t *d_vals, uint32_t *d_ranges, uint64_t *d_keys64,
                              uint32_t *d_count, uint32_t *d_error);

/* Reads (synchronously, on `stream`) the device error word of a bin/sort
 * workspace into *code (OR of GS_ERR_CAPACITY / GS_ERR_TIMEOUT) and clears
 * it. Returns GS_ERR_CUDA if the copy fails. */
gs_status gs_workspace_status(void *stream, void *d_workspace, int32_t *code);

/* Non-blocking form of gs_workspace_status: enqueues on `stream` a copy of
 * the error word (one uint32) to dst, then clears the word. dst may be
 * device memory or pinned host memory; it holds the value once the stream
 * reaches this point (wait on an event recorded after the call). Returns
 * GS_ERR_ARG for a null pointer, GS_ERR_CUDA if a copy cannot be enqueued. */
gs_status gs_workspace_status_async(void *stream, void *d_workspace, uint32_t *dst);

/* Self-test of the bounded waits (failure detection without a fault; not
 * part of the rendering path). Runs one of the bounded waits against an
 * event that never comes: which = 0 the scalar decoupled look-back of
 * gs_bin_sort (compaction) against a predecessor partition that
 * never publishes its count; which = 1 the per-digit look-back of a radix
 * pass; which = 2 the mbarrier wait of the tcgen05 blend on a barrier that
 * no arrival completes. The wait gives up after spin_limit polls (short
 * sleeps for the look-backs) and ORs GS_ERR_TIMEOUT into the error word
 * d_scratch[0]; the launch returns and the context stays usable.
 * d_scratch: GS_SELFTEST_SCRATCH_BYTES of device memory (4-byte aligned),
 * cleared by the call. Returns GS_ERR_ARG for a null pointer, which not 0/1/2,
 * or spin_limit outside [1, 2^20]. */
#define GS_SELFTEST_SCRATCH_BYTES 4096
gs_status gs_selftest_lookback_timeout(void *stream, int32_t which, uint32_t *d_scratch, int32_t spin_limit);

/* Arithmetic peak microbenchmark (measurement helper, not part of the
 * rendering path). The blend (gs_render) is bound by the FP32 FMA pipe, or
 * by the packed FP16x2 pipe when fp16x2 is set, so its roofline denominator
 * is the rate at which this GPU retires FFMA / HFMA2 lanes. Launches `blocks`
 * CTAs of 256 threads; each thread runs 8 independent FMA chains for
 * iters x 16 rounds (FP32 FFMA if half2 == 0, packed HFMA2 if half2 == 1) and
 * writes one float to d_sink[blocks * 256] (device, caller-owned; the values
 * are meaningless). *flop (host) receives the FLOP the launch performs
 * (2 per FMA lane, 2 lanes per HFMA2); time the launch on `stream` with
 * events. Returns GS_ERR_ARG for blocks <= 0, iters <= 0, a null pointer or
 * half2 not 0/1, GS_ERR_CUDA if the launch fails. */
gs_status gs_fma_peak(void *stream, int32_t half2, int32_t blocks, int32_t iters, float *d_sink,
                      double *flop);

/* Number of kernels this library has launched in this process (all entry
 * points), for launch accounting. */
uint64_t gs_launch_count(void);

/* Human-readable name of a status bit. */
const char *gs_status_string(int32_t status);

/* Spatial order of a scene (a one-time preparation when a scene is loaded,
 * not part of a frame; the paper has no counterpart). d_perm[k] is the index
 * of the k-th splat along a Z-order (Morton) curve: each mean's coordinates
 * are scaled into 10 bits over the bounding box of the finite means and
 * interleaved (x in bit 0); equal codes keep ascending index order; a
 * non-finite coordinate counts as the box's lower end. Storing the splats in
 * this order (gs_gather_rows) lets warps of nearby splats project, cull and
 * gather records together; rendered images change only where two splats
 * share a tile at exactly equal depth (their order follows the index).
 * d_means [P][3] FP32 (device); d_perm [P] uint32 (device, written);
 * d_workspace: gs_spatial_order_workspace_bytes(P) bytes of device memory,
 * 256-byte aligned, owned by the caller (contents need no initialisation).
 * Stream-ordered. GS_ERR_ARG for P < 0, P >= 2^30 or a null / misaligned
 * pointer with P > 0; P = 0 does nothing. */
size_t gs_spatial_order_workspace_bytes(int32_t P);
gs_status gs_spatial_order(void *stream, int32_t P, const float *d_means, void *d_workspace,
                           uint32_t *d_perm);

/* Row gather for reordering a scene: dst row k = src row perm[k], for n rows
 * of row_bytes bytes each (a positive multiple of 4; src, dst 4-byte
 * aligned, not overlapping). A perm entry >= n writes a zero row.
 * Stream-ordered; GS_ERR_ARG for a bad size or pointer. */
gs_status gs_gather_rows(void *stream, int32_t n, int32_t row_bytes, const void *d_src,
                         const uint32_t *d_perm, void *d_dst);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
