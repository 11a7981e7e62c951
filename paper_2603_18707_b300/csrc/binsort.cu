// binsort.cu — depth-ordered tile binning (sm_103a).
//
// Result: per global tile, the records whose support rectangle covers it,
// in increasing (depth, record index) order. That is the order a stable sort
// of 3DGS's 64-bit keys (tile << 32 | depth bits) over records emitted in
// index order gives. It is produced here without ever materialising 64-bit
// keys:
//   1. compact   drawn records (tiles > 0) -> (depth bits, record index),
//                in index order (single-pass scan with decoupled look-back)
//   2. sort      stable LSD radix sort of those by depth: 4 Onesweep passes
//   3. emit      walk the depth-sorted records, scan their tile counts and
//                write one (tile id, record index) pair per covered tile;
//                warp-cooperative so that every store is coalesced
//   4. sort      stable LSD radix sort of the pairs by tile id:
//                ceil(bits(total tiles) / 8) Onesweep passes
//   5. ranges    first / one-past-last position of every tile id
// The depth digits are sorted once per record instead of once per overlap,
// which moves far fewer bytes than sorting the 64-bit keys directly.
//
// Onesweep (one kernel per 8-bit digit): each CTA claims the next partition
// of 4096 keys from an atomic counter, ranks its keys per digit with warp
// match/ballot, publishes per-digit counts and resolves its global offsets by
// decoupled look-back over earlier partitions, then scatters through shared
// memory so that global stores are contiguous per digit. Every spin-wait is
// bounded: on expiry it raises GS_ERR_TIMEOUT in the workspace error word and
// carries on with what it has.
#include <algorithm>
#include <utility>

#include "gs_common.cuh"

namespace gs {
namespace {

constexpr uint32_t kValMask = (1u << 30) - 1;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagIncl = 2u << 30;
constexpr int kSpinLimit = 1 << 20;

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems; // keys per partition
constexpr int kCompactItems = 8;
constexpr int kCompactTile = 256 * kCompactItems;
constexpr int kEmitItems = 8;
constexpr int kEmitTile = 256 * kEmitItems;

enum Counter {
    CTR_COMPACT = 0,
    CTR_DEPTH = 1,   // 4 passes
    CTR_EMIT = 5,
    CTR_TILE = 6,    // up to 4 passes
    CTR_COUNT = 10
};

struct WsHeader {
    uint32_t err;
    uint32_t n_vis;      // drawn records
    uint32_t n_over;     // overlaps stored (<= capacity)
    uint32_t n_over_raw; // overlaps counted
    uint32_t ctr[CTR_COUNT];
    uint32_t pad[64 - 4 - CTR_COUNT];
};

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b)
{
    uint32_t s = a + b;
    return (s > kValMask || s < a) ? kValMask : s;
}

// Decoupled look-back of a scalar scan, executed by one full warp. Publishes
// this partition's aggregate, accumulates predecessors 32 at a time until an
// inclusive prefix is found, publishes the inclusive prefix and returns the
// exclusive one (same value in every lane).
__device__ uint32_t lookback_scalar(uint32_t *state, uint32_t part, uint32_t agg, uint32_t *err)
{
    const int lane = threadIdx.x & 31;
    if (part == 0) {
        if (lane == 0) st_relaxed(&state[0], kFlagIncl | (agg & kValMask));
        return 0;
    }
    if (lane == 0) st_relaxed(&state[part], kFlagAgg | (agg & kValMask));
    uint32_t excl = 0;
    int64_t p = (int64_t)part - 1;
    int spins = 0;
    while (true) {
        const int64_t idx = p - lane;
        uint32_t s = idx >= 0 ? ld_relaxed(&state[idx]) : kFlagIncl;
        while (__any_sync(0xffffffffu, (s >> 30) == 0)) {
            if (++spins > kSpinLimit) {
                if (lane == 0) atomicOr(err, (uint32_t)GS_ERR_TIMEOUT);
                if ((s >> 30) == 0) s = kFlagIncl;
                break;
            }
            __nanosleep(64);
            if ((s >> 30) == 0) s = ld_relaxed(&state[idx]);
        }
        const uint32_t incl = __ballot_sync(0xffffffffu, (s >> 30) == 2);
        const int first = incl ? __ffs(incl) - 1 : 32;
        const uint32_t v = warp_sum(lane <= first ? (s & kValMask) : 0u);
        excl = sat_add(excl, v);
        if (first < 32) break;
        p -= 32;
    }
    if (lane == 0) st_relaxed(&state[part], kFlagIncl | sat_add(excl, agg));
    return excl;
}

// Block-wide exclusive scan of one value per thread (blockDim.x == 256).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t wex = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t t = s_warp[w];
        wex += (w < warp) ? t : 0u;
        tot += t;
    }
    total = tot;
    return wex + x - v;
}

// 1. compaction of drawn records, index order preserved.
__global__ void __launch_bounds__(256)
compact_kernel(const uint32_t *__restrict__ tiles, const uint32_t *__restrict__ dkey, uint32_t N,
               uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, WsHeader *hdr,
               uint32_t *state)
{
    __shared__ uint32_t s_part, s_excl, s_warp[8];
    if (threadIdx.x == 0) s_part = atomicAdd(&hdr->ctr[CTR_COMPACT], 1u);
    __syncthreads();
    const uint32_t part = s_part;
    const uint32_t nparts = (N + kCompactTile - 1) / kCompactTile;
    if (part >= nparts) return;
    const uint32_t base = part * kCompactTile + threadIdx.x * kCompactItems;
    uint32_t flags = 0, cnt = 0;
#pragma unroll
    for (int j = 0; j < kCompactItems; ++j) {
        const uint32_t idx = base + j;
        const bool f = idx < N && tiles[idx] > 0;
        flags |= (uint32_t)f << j;
        cnt += f;
    }
    uint32_t total;
    const uint32_t excl_t = block_excl_scan(cnt, s_warp, total);
    if (threadIdx.x < 32) {
        const uint32_t e = lookback_scalar(state, part, total, &hdr->err);
        if (threadIdx.x == 0) s_excl = e;
    }
    __syncthreads();
    uint32_t pos = s_excl + excl_t;
#pragma unroll
    for (int j = 0; j < kCompactItems; ++j) {
        if (flags >> j & 1u) {
            if (pos < N) { // always true unless a look-back wait timed out
                keys_out[pos] = dkey[base + j];
                vals_out[pos] = base + j;
            }
            ++pos;
        }
    }
    if (part == nparts - 1 && threadIdx.x == 255) hdr->n_vis = pos;
}

// Histograms of every digit position used by the passes of one sort.
__global__ void __launch_bounds__(256)
histogram_kernel(const uint32_t *__restrict__ keys, const uint32_t *n_ptr, int passes,
                 uint32_t *__restrict__ hist)
{
    __shared__ uint32_t s_h[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += 256) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const uint32_t n = *n_ptr;
    for (uint32_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
        const uint32_t v = s_h[p][threadIdx.x];
        if (v) atomicAdd(&hist[p * 256 + threadIdx.x], v);
    }
}

// One Onesweep pass over 8 bits starting at `shift`.
__global__ void __launch_bounds__(kSortThreads)
onesweep_kernel(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                const uint32_t *n_ptr, int shift, const uint32_t *__restrict__ hist,
                uint32_t *state, uint32_t *ctr, uint32_t *err)
{
    __shared__ uint32_t s_keys[kSortTile];
    __shared__ uint32_t s_vals[kSortTile];
    __shared__ uint32_t s_whist[8][256];
    __shared__ uint32_t s_bexcl[256];
    __shared__ uint32_t s_goff[256];
    __shared__ uint32_t s_warp[8];
    __shared__ uint32_t s_part;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_part = atomicAdd(ctr, 1u);
#pragma unroll
    for (int w = 0; w < 8; ++w) s_whist[w][tid] = 0;
    __syncthreads();
    const uint32_t n = *n_ptr;
    const uint32_t part = s_part;
    const uint32_t nparts = (n + kSortTile - 1) / kSortTile;
    if (part >= nparts) return;

    // warp-striped load: warp w owns keys [base + 512 w, base + 512 (w + 1))
    const uint32_t wbase = part * kSortTile + warp * (32 * kSortItems);
    uint32_t k[kSortItems], v[kSortItems], r[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t idx = wbase + j * 32 + lane;
        const bool ok = idx < n;
        k[j] = ok ? keys_in[idx] : 0xffffffffu; // invalid keys rank last (digit 255, highest index)
        v[j] = ok ? vals_in[idx] : 0u;
    }
    // rank within the warp: match lanes with equal digits
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t d = (k[j] >> shift) & 255u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader) {
            old = s_whist[warp][d];
            s_whist[warp][d] = old + __popc(peers);
        }
        old = __shfl_sync(0xffffffffu, old, leader);
        r[j] = old + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    // per digit (thread = digit): warp-exclusive offsets and block count
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t c = s_whist[w][tid];
        s_whist[w][tid] = cnt;
        cnt += c;
    }
    uint32_t tot;
    const uint32_t bex = block_excl_scan(cnt, s_warp, tot);
    s_bexcl[tid] = bex;
    // global digit offsets from the histogram (every CTA rescans 256 values)
    __syncthreads();
    uint32_t htot;
    const uint32_t hex = block_excl_scan(hist[tid], s_warp + 0, htot);
    (void)htot;
    // invalid keys exist only in the last partition, all with digit 255
    const uint32_t last_valid = n - part * kSortTile;
    const uint32_t n_invalid = last_valid < (uint32_t)kSortTile ? kSortTile - last_valid : 0u;
    const uint32_t agg = cnt - (tid == 255 ? n_invalid : 0u);
    // decoupled look-back, one digit per thread
    uint32_t *st = state + (size_t)part * 256;
    uint32_t excl = 0;
    if (part == 0) {
        st_relaxed(&st[tid], kFlagIncl | agg);
    } else {
        st_relaxed(&st[tid], kFlagAgg | agg);
        int64_t p = (int64_t)part - 1;
        int spins = 0;
        while (p >= 0) {
            const uint32_t s = ld_relaxed(&state[(size_t)p * 256 + tid]);
            const uint32_t f = s >> 30;
            if (f == 0) {
                if (++spins > kSpinLimit) {
                    atomicOr(err, (uint32_t)GS_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(32);
                continue;
            }
            excl = sat_add(excl, s & kValMask);
            if (f == 2) break;
            --p;
        }
        st_relaxed(&st[tid], kFlagIncl | sat_add(excl, agg));
    }
    s_goff[tid] = hex + excl;
    __syncthreads();
    // scatter into shared memory in digit order
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t d = (k[j] >> shift) & 255u;
        const uint32_t lp = s_bexcl[d] + s_whist[warp][d] + r[j];
        s_keys[lp] = k[j];
        s_vals[lp] = v[j];
    }
    __syncthreads();
    const uint32_t nvalid = min(last_valid, (uint32_t)kSortTile);
    for (uint32_t i = tid; i < nvalid; i += kSortThreads) {
        const uint32_t key = s_keys[i];
        const uint32_t d = (key >> shift) & 255u;
        const uint32_t o = s_goff[d] + i - s_bexcl[d];
        if (o < n) { // always true unless a look-back wait timed out
            keys_out[o] = key;
            vals_out[o] = s_vals[i];
        }
    }
}

// 3. overlap emission in depth order.
__global__ void __launch_bounds__(256)
emit_kernel(const __grid_constant__ CamTable cams, int P, uint32_t n_records,
            const uint32_t *__restrict__ sorted_vals,
            const uint32_t *__restrict__ tiles, const ushort4 *__restrict__ rects,
            uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, uint32_t capacity,
            WsHeader *hdr, uint32_t *state)
{
    __shared__ uint32_t s_part, s_excl, s_warp[8];
    if (threadIdx.x == 0) s_part = atomicAdd(&hdr->ctr[CTR_EMIT], 1u);
    __syncthreads();
    const uint32_t nv = hdr->n_vis;
    const uint32_t part = s_part;
    const uint32_t nparts = (nv + kEmitTile - 1) / kEmitTile;
    if (part >= nparts) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // warp-striped: item j of lane l is record wbase + 32 j + l (depth order)
    const uint32_t wbase = part * kEmitTile + warp * (32 * kEmitItems);
    uint32_t v[kEmitItems], cnt[kEmitItems], incl[kEmitItems], off[kEmitItems];
    ushort4 rc[kEmitItems];
    uint32_t running = 0;
#pragma unroll
    for (int j = 0; j < kEmitItems; ++j) {
        const uint32_t idx = wbase + 32 * j + lane;
        uint32_t vv = idx < nv ? sorted_vals[idx] : 0u;
        const bool valid = idx < nv && vv < n_records; // ids are < n_records unless a wait timed out
        if (!valid) vv = 0u;
        v[j] = vv;
        cnt[j] = valid ? tiles[vv] : 0u;
        rc[j] = valid ? rects[vv] : make_ushort4(0, 0, 0, 0);
        uint32_t x = cnt[j];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        incl[j] = x;
        off[j] = running;
        running += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) s_warp[warp] = running;
    __syncthreads();
    uint32_t warp_excl = 0, total = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t t = s_warp[w];
        warp_excl += (w < warp) ? t : 0u;
        total += t;
    }
    if (threadIdx.x < 32) {
        const uint32_t e = lookback_scalar(state, part, total, &hdr->err);
        if (threadIdx.x == 0) s_excl = e;
    }
    __syncthreads();
    const uint32_t part_excl = s_excl;
#pragma unroll
    for (int j = 0; j < kEmitItems; ++j) {
        const uint32_t w_incl = incl[j];
        const uint32_t w_total = __shfl_sync(0xffffffffu, w_incl, 31);
        const uint32_t out_base = part_excl + warp_excl + off[j];
        const int cam = (int)(v[j] / (uint32_t)P);
        const int tiles_x = cams.cam[cam].tiles_x;
        const uint32_t tbase = (uint32_t)cams.cam[cam].tile_base + (uint32_t)rc[j].y * tiles_x + rc[j].x;
        const uint32_t rw = (uint32_t)rc[j].z - rc[j].x + 1u;
        const uint32_t beg = w_incl - cnt[j];
        // the warp walks these overlaps 32 at a time; every lane takes part
        // in every shuffle, lanes past the end only skip the store
        for (uint32_t b = 0; b < w_total; b += 32) {
            const uint32_t p = b + lane;
            const uint32_t pq = min(p, w_total - 1u);
            int e = 0; // owner lane: number of lanes whose inclusive prefix is <= pq
#pragma unroll
            for (int sft = 16; sft > 0; sft >>= 1) {
                const uint32_t c = __shfl_sync(0xffffffffu, w_incl, e + sft - 1);
                if (c <= pq) e += sft;
            }
            const uint32_t ev = __shfl_sync(0xffffffffu, v[j], e);
            const uint32_t ebeg = __shfl_sync(0xffffffffu, beg, e);
            const uint32_t erw = __shfl_sync(0xffffffffu, rw, e);
            const uint32_t etb = __shfl_sync(0xffffffffu, tbase, e);
            const uint32_t etx = __shfl_sync(0xffffffffu, (uint32_t)tiles_x, e);
            const uint32_t l = pq - ebeg;
            const uint32_t row = l / erw, col = l - row * erw;
            const uint32_t o = out_base + p;
            if (p < w_total && o < capacity) {
                keys_out[o] = etb + row * etx + col;
                vals_out[o] = ev;
            }
        }
    }
    if (part == nparts - 1 && threadIdx.x == 0) {
        const uint32_t tot = sat_add(part_excl, total);
        hdr->n_over_raw = tot;
        hdr->n_over = min(tot, capacity);
        if (tot > capacity || tot >= kValMask) atomicOr(&hdr->err, (uint32_t)GS_ERR_CAPACITY);
    }
}

// 5. per-tile [start, end) and optional 64-bit keys.
__global__ void __launch_bounds__(256)
ranges_kernel(const uint32_t *__restrict__ tkeys, const uint32_t *__restrict__ vals,
              const uint32_t *__restrict__ dkey, const WsHeader *hdr, uint2 *__restrict__ ranges,
              unsigned long long *__restrict__ keys64, uint32_t total_tiles, uint32_t n_records)
{
    const uint32_t n = hdr->n_over;
    for (uint32_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) {
        const uint32_t t = tkeys[i];
        if (t >= total_tiles) continue; // only after a timed-out wait
        if (i == 0 || tkeys[i - 1] != t) ranges[t].x = i;
        if (i + 1 == n || tkeys[i + 1] != t) ranges[t].y = i + 1;
        if (keys64) {
            const uint32_t v = vals[i];
            keys64[i] = ((unsigned long long)t << 32) | (v < n_records ? dkey[v] : 0xffffffffu);
        }
    }
}

struct WsLayout {
    size_t hdr, hist, st_compact, st_depth, st_emit, st_tile, zero_end;
    size_t dk0, dk1, dv0, dv1, tk0, tk1, tv1, total;
    uint32_t parts_depth, parts_tile;
};

WsLayout ws_layout(int64_t N, int64_t cap)
{
    WsLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += align256(bytes); return r; };
    L.parts_depth = (uint32_t)((N + kSortTile - 1) / kSortTile);
    L.parts_tile = (uint32_t)((cap + kSortTile - 1) / kSortTile);
    L.hdr = take(sizeof(WsHeader));
    L.hist = take(sizeof(uint32_t) * 8 * 256);
    L.st_compact = take(sizeof(uint32_t) * ((N + kCompactTile - 1) / kCompactTile + 1));
    L.st_depth = take(sizeof(uint32_t) * 4 * 256 * (size_t)(L.parts_depth + 1));
    L.st_emit = take(sizeof(uint32_t) * ((N + kEmitTile - 1) / kEmitTile + 1));
    L.st_tile = take(sizeof(uint32_t) * 4 * 256 * (size_t)(L.parts_tile + 1));
    L.zero_end = o;
    L.dk0 = take(sizeof(uint32_t) * N);
    L.dk1 = take(sizeof(uint32_t) * N);
    L.dv0 = take(sizeof(uint32_t) * N);
    L.dv1 = take(sizeof(uint32_t) * N);
    L.tk0 = take(sizeof(uint32_t) * cap);
    L.tk1 = take(sizeof(uint32_t) * cap);
    L.tv1 = take(sizeof(uint32_t) * cap);
    L.total = o;
    return L;
}

int tile_bits(int64_t total_tiles)
{
    int b = 1;
    while (((int64_t)1 << b) < total_tiles) ++b;
    return b;
}

} // namespace
} // namespace gs

using namespace gs;

extern "C" size_t gs_bin_sort_workspace_bytes(int64_t n_records, int64_t capacity, int64_t total_tiles)
{
    (void)total_tiles;
    if (n_records < 0 || capacity < 0) return 0;
    return ws_layout(n_records, capacity).total;
}

extern "C" gs_status gs_bin_sort(void *stream, const gs_camera *cams, int32_t ncam, int32_t P,
                                 const gs_config *cfg, const void *d_splat2d, int64_t capacity,
                                 void *d_workspace, size_t workspace_bytes, uint32_t *d_vals,
                                 uint32_t *d_ranges, uint64_t *d_keys64, uint32_t *d_count)
{
    if (!cams || !cfg || ncam <= 0 || ncam > kMaxCams || P < 0 || capacity < 0) return GS_ERR_ARG;
    const int64_t N = (int64_t)ncam * P;
    if (N >= (int64_t)kValMask || capacity >= (int64_t)kValMask) return GS_ERR_ARG;
    if (!d_workspace || ((uintptr_t)d_workspace & 255) || !d_ranges || (capacity > 0 && !d_vals))
        return GS_ERR_ARG;
    if (N > 0 && (!d_splat2d || ((uintptr_t)d_splat2d & 255))) return GS_ERR_ARG;
    CamTable t;
    if (!build_cam_table(cams, ncam, cfg, &t)) return GS_ERR_ARG;
    const WsLayout L = ws_layout(N, capacity);
    if (workspace_bytes < L.total) return GS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(d_workspace);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws + L.hdr);
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws + L.hist);
    auto U = [&](size_t off) { return reinterpret_cast<uint32_t *>(ws + off); };

    if (cudaMemsetAsync(ws, 0, L.zero_end, s) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemsetAsync(d_ranges, 0, sizeof(uint32_t) * 2 * (size_t)t.total_tiles, s) != cudaSuccess)
        return GS_ERR_CUDA;
    if (N > 0) {
        Splat2DConst sp = splat2d_const(d_splat2d, N);
        // 1. compaction
        compact_kernel<<<(unsigned)((N + kCompactTile - 1) / kCompactTile), 256, 0, s>>>(
            sp.tiles, sp.dkey, (uint32_t)N, U(L.dk0), U(L.dv0), hdr, U(L.st_compact));
        count_launch();
        GS_LAUNCH_CHECK();
        // 2. depth sort, 4 passes ping-pong: result back in (dk0, dv0)
        const int hist_blocks = 148 * 4;
        histogram_kernel<<<hist_blocks, 256, 0, s>>>(U(L.dk0), &hdr->n_vis, 4, hist);
        count_launch();
        GS_LAUNCH_CHECK();
        uint32_t *kin = U(L.dk0), *vin = U(L.dv0), *kout = U(L.dk1), *vout = U(L.dv1);
        for (int p = 0; p < 4; ++p) {
            onesweep_kernel<<<L.parts_depth ? L.parts_depth : 1, kSortThreads, 0, s>>>(
                kin, vin, kout, vout, &hdr->n_vis, 8 * p, hist + 256 * p,
                U(L.st_depth) + (size_t)p * 256 * (L.parts_depth + 1), &hdr->ctr[CTR_DEPTH + p],
                &hdr->err);
            count_launch();
            GS_LAUNCH_CHECK();
            std::swap(kin, kout);
            std::swap(vin, vout);
        }
        if (capacity > 0) {
            // 3. emission into the buffers that make the last tile pass land in d_vals
            const int tb = tile_bits(t.total_tiles);
            const int passes = (tb + 7) / 8;
            uint32_t *ek = U(L.tk0);
            uint32_t *ev = (passes % 2 == 0) ? d_vals : U(L.tv1);
            emit_kernel<<<(unsigned)((N + kEmitTile - 1) / kEmitTile), 256, 0, s>>>(
                t, P, (uint32_t)N, vin, sp.tiles, sp.rect, ek, ev, (uint32_t)capacity, hdr, U(L.st_emit));
            count_launch();
            GS_LAUNCH_CHECK();
            // 4. tile sort
            histogram_kernel<<<hist_blocks, 256, 0, s>>>(ek, &hdr->n_over, passes, hist + 4 * 256);
            count_launch();
            GS_LAUNCH_CHECK();
            uint32_t *tki = ek, *tvi = ev, *tko = U(L.tk1), *tvo = (ev == d_vals) ? U(L.tv1) : d_vals;
            for (int p = 0; p < passes; ++p) {
                onesweep_kernel<<<L.parts_tile ? L.parts_tile : 1, kSortThreads, 0, s>>>(
                    tki, tvi, tko, tvo, &hdr->n_over, 8 * p, hist + 256 * (4 + p),
                    U(L.st_tile) + (size_t)p * 256 * (L.parts_tile + 1), &hdr->ctr[CTR_TILE + p],
                    &hdr->err);
                count_launch();
                GS_LAUNCH_CHECK();
                std::swap(tki, tko);
                std::swap(tvi, tvo);
            }
            // 5. ranges (tki / tvi hold the sorted tile keys / record ids; tvi == d_vals)
            const unsigned rblocks = (unsigned)std::min<int64_t>((capacity + 255) / 256, 148 * 16);
            ranges_kernel<<<rblocks ? rblocks : 1, 256, 0, s>>>(
                tki, tvi, sp.dkey, hdr, reinterpret_cast<uint2 *>(d_ranges),
                reinterpret_cast<unsigned long long *>(d_keys64), (uint32_t)t.total_tiles, (uint32_t)N);
            count_launch();
            GS_LAUNCH_CHECK();
        }
    }
    if (d_count) {
        if (cudaMemcpyAsync(d_count, &hdr->n_vis, 3 * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
            return GS_ERR_CUDA;
    }
    return GS_OK;
}

extern "C" gs_status gs_workspace_status(void *stream, void *d_workspace, int32_t *code)
{
    if (!d_workspace || !code) return GS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(d_workspace);
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, &hdr->err, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return GS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemsetAsync(&hdr->err, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    *code = (int32_t)v;
    return GS_OK;
}
