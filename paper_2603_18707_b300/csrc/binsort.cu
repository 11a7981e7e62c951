// binsort.cu — depth-ordered tile binning (sm_103a).
//
// Result: per global tile, the records whose support rectangle covers it,
// in increasing (depth, record index) order. That is the order a stable sort
// of 3DGS's 64-bit keys (tile << 32 | depth bits) over records emitted in
// index order gives. It is produced here without materialising keys per
// overlap and without sorting overlaps at all:
//   1. compact   drawn records (tiles > 0) -> (depth bits, record index),
//                in index order, i.e. grouped by camera (single-pass scan
//                with decoupled look-back); also the per-camera histograms
//                of the four depth digits, the per-camera start offsets, and
//                per camera a difference array of the tile rows the records
//                cover
//   2. plan      one CTA: partition tables of the record and row segments,
//                span count and first span of every tile row
//   3. sort      stable LSD radix sort by depth within each camera: 4
//                Onesweep passes of 8 bits over camera segments
//   4. rows      split the depth-sorted records of each camera by tile row:
//                one span (record, first and last tile column) per covered
//                row, stored grouped by (camera, row) in depth order
//   5. count     tile counts from the spans (per-row difference arrays)
//   6. scan      exclusive scan of the tile counts: the per-tile ranges
//   7. columns   split the spans of each row by tile column, writing every
//                record index straight to its final place in its tile's list
// Steps 4 and 7 are one "stable split" each: items (records, then spans)
// that cover a contiguous range of digits (rows, then columns) are expanded
// in item order and ranked per digit, Onesweep style: each CTA takes the
// next partition of a segment (camera, then tile row) from a counter,
// publishes its per-digit counts and resolves its offsets by decoupled
// look-back over the segment's earlier partitions. The depth digits are
// sorted once per record instead of once per overlap, and each overlap is
// written once, as its final 4-byte record index.
//
// Every spin-wait is bounded: on expiry it raises GS_ERR_TIMEOUT in the
// workspace error word and carries on with what it has; stores are checked
// against the buffers' capacities, so the results are then wrong but every
// access stays in bounds.
#include <algorithm>
#include <utility>

#include "blend_math.cuh"

namespace gs {
namespace {

constexpr uint32_t kValMask = (1u << 30) - 1;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagIncl = 2u << 30;
constexpr int kSpinLimit = 1 << 20;

// Launch-shape constants (compile-time; -D overrides for tuning builds).
#ifndef GS_SORT_ITEMS
#define GS_SORT_ITEMS 20
#endif
#ifndef GS_SORT_MIN_BLOCKS
#define GS_SORT_MIN_BLOCKS 3
#endif
#ifndef GS_LOOK_WINDOW
#define GS_LOOK_WINDOW 1
#endif
#ifndef GS_SPLIT_BLOCKS
#define GS_SPLIT_BLOCKS 3 // register budget of the split kernels: CTAs per SM it allows
#endif
#define GS_SPLIT_BOUNDS __launch_bounds__(256, GS_SPLIT_BLOCKS)
constexpr int kSortThreads = 256;
constexpr int kSortItems = GS_SORT_ITEMS;
constexpr int kSortTile = kSortThreads * kSortItems; // keys per partition
#ifndef GS_COMPACT_VEC
#define GS_COMPACT_VEC 8
#endif
constexpr int kCompactVec = GS_COMPACT_VEC;          // uint4 loads per lane
constexpr int kCompactTile = 256 * 4 * kCompactVec;  // records per partition
constexpr int kRowItems = kSortItems;                // records per thread of the row split
constexpr int kRowTile = 256 * kRowItems;            // records per row-split partition
static_assert(kRowTile == kSortTile, "the row split reuses the depth sort's partition table");
constexpr int kColItems = 20;                        // spans per thread of the column split
constexpr int kColTile = 256 * kColItems;            // spans per column-split partition
constexpr int kScanItems = 16;
constexpr int kScanTile = 256 * kScanItems;          // tiles per scan partition
constexpr int kMaxDigits = 2048;                     // tile rows / columns per camera (16384 px / 8)
constexpr int kLookWindow = GS_LOOK_WINDOW;
#ifndef GS_SPLIT_WINDOW
#define GS_SPLIT_WINDOW 1
#endif
// Look-back window of the split kernels (predecessors loaded per round): one,
// as for the depth passes, measured fastest (row split 0.589 ms at 1, 0.611
// at 4, 0.628 at 16 predecessors per round).
constexpr int kSplitWindow = GS_SPLIT_WINDOW;

enum Counter {
    CTR_COMPACT = 0,
    CTR_DEPTH = 1, // 4 passes
    CTR_ROWS = 5,
    CTR_COUNT_COLS = 6,
    CTR_SCAN = 7,
    CTR_COLS = 8,
    CTR_N = 10
};

struct WsHeader {
    uint32_t err;
    uint32_t n_vis;       // drawn records
    uint32_t n_over;      // overlaps stored (<= capacity)
    uint32_t n_over_raw;  // overlaps counted (the capacity needed)
    uint32_t n_span;      // row spans
    uint32_t n_rec_parts; // partitions of the record segments
    uint32_t n_span_parts;
    uint32_t pad0;
    unsigned long long k_total; // sum of the drawn records' tile counts
    uint32_t ctr[CTR_N];
    uint32_t pad[64 - 10 - CTR_N];
};
static_assert(sizeof(WsHeader) == 256, "header size");

// Division of n < 2^31 by a fixed d >= 1 as a multiply-high and a shift:
// with s = ceil(log2 d) and m = ceil(2^(31+s) / d) < 2^32, floor(n m / 2^(31+s))
// = floor(n / d), since the error n (m - 2^(31+s)/d) / 2^(31+s) < n / 2^(31+s)
// < 2^-s <= 1/d never carries past the next multiple of d.
struct FastDiv {
    uint32_t m;
    int sh; // s - 1, or -1 for d == 1
    static FastDiv make(uint32_t d)
    {
        FastDiv f;
        if (d <= 1) {
            f.m = 0;
            f.sh = -1;
            return f;
        }
        int s = 0;
        while ((1ull << s) < d) ++s;
        f.m = (uint32_t)(((1ull << (31 + s)) + d - 1) / d);
        f.sh = s - 1;
        return f;
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return sh < 0 ? n : __umulhi(n, m) >> sh; }
};

// Per-call geometry of the binning, a kernel parameter. Tile rows of all
// cameras are numbered back to back with one padding row after each camera
// ("padded rows"): camera c's row y is padded row gpad + y, and its padding
// row gpad + tiles_y closes its difference array.
struct BinCam {
    int tiles_x, tiles_y;
    int tile_base; // first global tile id
    int gpad;      // first padded row
    int W, H;
};
struct BinPlan {
    int ncam;
    int G; // padded rows: sum of (tiles_y + 1)
    int max_tx, max_ty;
    int tile_w, tile_h;
    uint32_t P;
    FastDiv pdiv;
    BinCam cam[kMaxCams];
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

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Lane that owns sub-item q of a warp's expansion: the number of lanes whose
// inclusive prefix of sub-item counts is <= q (binary search over the lanes).
__device__ __forceinline__ int owner_lane(uint32_t incl, uint32_t q)
{
    int e = 0;
#pragma unroll
    for (int sft = 16; sft > 0; sft >>= 1) {
        const uint32_t c = __shfl_sync(0xffffffffu, incl, e + sft - 1);
        if (c <= q) e += sft;
    }
    return e;
}

// Lanes of the warp whose BITS-bit digit equals this lane's: one ballot per
// bit (GS_SORT_BALLOT, the default) or the match instruction.
#ifndef GS_SORT_BALLOT
#define GS_SORT_BALLOT 1
#endif
template <int BITS>
__device__ __forceinline__ uint32_t warp_peers(uint32_t d)
{
#if GS_SORT_BALLOT
    uint32_t m = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t v = __ballot_sync(0xffffffffu, bit);
        m &= bit ? v : ~v;
    }
    return m;
#else
    return __match_any_sync(0xffffffffu, d);
#endif
}

#ifndef GS_SPLIT_RANK
#define GS_SPLIT_RANK 1
#endif
// Place of this lane's item among the warp's items with the same digit d
// (d < 2048), in lane order, after the warp's running count of d in wc[d];
// advances wc[d] by the group's size. Inactive lanes take no place. Peers by
// ballots over the digit bits (GS_SPLIT_RANK 1) or the match instruction (0).
__device__ __forceinline__ uint32_t split_rank(uint32_t *wc, uint32_t d, bool act, uint32_t lt)
{
    const int lane = threadIdx.x & 31;
#if GS_SPLIT_RANK
    const uint32_t peers = warp_peers<11>(d) & __ballot_sync(0xffffffffu, act);
#else
    const uint32_t peers = __match_any_sync(0xffffffffu, act ? d : 0x10000u + lane) & __ballot_sync(0xffffffffu, act);
#endif
    // every lane of a group reads the count before its first lane moves it on
    const uint32_t base = act ? wc[d] : 0u;
    __syncwarp();
    if (act && lane == __ffs(peers) - 1) wc[d] = base + __popc(peers);
    __syncwarp();
    return base + __popc(peers & lt);
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
__device__ uint32_t lookback_scalar(uint32_t *state, uint32_t part, uint32_t agg, uint32_t *err,
                                   int limit = kSpinLimit)
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
            if (++spins > limit) {
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

// Decoupled look-back of one digit (one thread per digit): sums the
// published counts of digit d in the partitions before `part` (state row
// stride R, kLookWindow per load round) until one with an inclusive prefix.
// The first partition of every segment publishes an inclusive prefix, so the
// walk never leaves the segment. A predecessor that has published nothing is
// re-read after a short sleep, at most `limit` times; then GS_ERR_TIMEOUT is
// raised and what was summed is returned.
template <int WIN = kLookWindow>
__device__ uint32_t lookback_digit(const uint32_t *state, uint32_t part, int R, int d, uint32_t *err,
                                   int limit)
{
    uint32_t excl = 0;
    int64_t p = (int64_t)part - 1;
    int spins = 0;
    bool done = false;
    while (!done && p >= 0) {
        uint32_t s[WIN];
#pragma unroll
        for (int w = 0; w < WIN; ++w)
            s[w] = (p - w >= 0) ? ld_relaxed(&state[(size_t)(p - w) * R + d]) : kFlagIncl;
        int used = 0;
        bool stall = false;
#pragma unroll
        for (int w = 0; w < WIN; ++w) {
            if (done || stall) continue;
            const uint32_t f = s[w] >> 30;
            if (f == 0) {
                stall = true;
                continue;
            }
            excl = sat_add(excl, s[w] & kValMask);
            ++used;
            if (f == 2) done = true;
        }
        p -= used;
        if (stall && !done) {
            if (++spins > limit) {
                atomicOr(err, (uint32_t)GS_ERR_TIMEOUT);
                break;
            }
            __nanosleep(32);
        }
    }
    return excl;
}

// Publishes digit d's count of partition `part` (chunk > 0: of a segment
// that began in an earlier partition) and returns the digit's exclusive
// prefix within the segment; WIN predecessors per load round.
template <int WIN>
__device__ __forceinline__ uint32_t publish_digit(uint32_t *state, uint32_t part, uint32_t chunk, int R, int d,
                                                  uint32_t agg, uint32_t *err)
{
    uint32_t *st = state + (size_t)part * R + d;
    if (chunk == 0) {
        st_relaxed(st, kFlagIncl | agg);
        return 0;
    }
    st_relaxed(st, kFlagAgg | agg);
    const uint32_t excl = lookback_digit<WIN>(state, part, R, d, err, kSpinLimit);
    st_relaxed(st, kFlagIncl | sat_add(excl, agg));
    return excl;
}

// Block-wide exclusive scan of one value per thread (WARPS warps).
template <int WARPS>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t x = warp_incl_scan(v);
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t wex = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
        const uint32_t t = s_warp[w];
        wex += (w < warp) ? t : 0u;
        tot += t;
    }
    total = tot;
    return wex + x - v;
}

// Row-difference slot of camera c, tile row y (y == tiles_y: the padding row).
__device__ __forceinline__ uint32_t *rowdiff_at(const BinPlan &bp, uint32_t *rowdiff, int c, int y)
{
    return rowdiff + bp.cam[c].gpad + y;
}

// 1. compaction of drawn records, index order preserved. Lane l of warp w
// holds records base + (kCompactTile / 8) w + 4 (32 j + l) + e, e < 4,
// j < kCompactVec (uint4 loads). Also: seg[c] = drawn records before camera
// c's first record (seg[ncam] = all drawn records); per camera the
// histograms of the four depth digits (hist[c][pass][256]) and the row
// difference array (+1 at the first covered row, -1 after the last); the
// sum of the tile counts. A partition holds records of camera c0 (its first
// record's) and usually c0 + 1, counted in shared memory; records of other
// cameras (only when P < kCompactTile) go to global memory directly.
__global__ void __launch_bounds__(256)
compact_kernel(const __grid_constant__ BinPlan bp, const uint32_t *__restrict__ tiles,
               const uint32_t *__restrict__ dkey, const ushort4 *__restrict__ rects, uint32_t N,
               uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, WsHeader *hdr,
               uint32_t *state, uint32_t *__restrict__ hist, uint32_t *__restrict__ rowdiff,
               uint32_t *__restrict__ seg)
{
    __shared__ uint32_t s_part, s_excl, s_warp[8];
    __shared__ uint32_t s_h[2][4][256];
    __shared__ uint32_t s_rd[2][kMaxDigits + 1];
    __shared__ unsigned long long s_k[8];
    if (threadIdx.x == 0) s_part = atomicAdd(&hdr->ctr[CTR_COMPACT], 1u);
    __syncthreads();
    const uint32_t part = s_part;
    const uint32_t nparts = (N + kCompactTile - 1) / kCompactTile;
    if (part >= nparts) return;
    const uint32_t c0 = bp.pdiv.div(part * kCompactTile);
    const int nrd0 = bp.cam[c0].tiles_y + 1;
    const int nrd1 = (int)c0 + 1 < bp.ncam ? bp.cam[c0 + 1].tiles_y + 1 : 0;
    for (int i = threadIdx.x; i < 2 * 4 * 256; i += 256) (&s_h[0][0][0])[i] = 0;
    for (int i = threadIdx.x; i < nrd0; i += 256) s_rd[0][i] = 0;
    for (int i = threadIdx.x; i < nrd1; i += 256) s_rd[1][i] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t wbase = part * kCompactTile + warp * (kCompactTile / 8);
    uint32_t flags[kCompactVec], incl[kCompactVec], off[kCompactVec];
    uint32_t running = 0;
    unsigned long long ksum = 0;
#pragma unroll
    for (int j = 0; j < kCompactVec; ++j) {
        const uint32_t e0 = wbase + 4 * (32 * j + lane);
        uint32_t f = 0;
        if (e0 + 3 < N) {
            const uint4 t4 = reinterpret_cast<const uint4 *>(tiles)[e0 / 4];
            f = (t4.x > 0) | (t4.y > 0) << 1 | (t4.z > 0) << 2 | (t4.w > 0) << 3;
            ksum += (unsigned long long)t4.x + t4.y + t4.z + t4.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t t = e0 + e < N ? tiles[e0 + e] : 0u;
                if (t > 0) f |= 1u << e;
                ksum += t;
            }
        }
        flags[j] = f;
        const uint32_t x = warp_incl_scan(__popc(f));
        incl[j] = x;
        off[j] = running;
        running += __shfl_sync(0xffffffffu, x, 31);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ksum += __shfl_xor_sync(0xffffffffu, ksum, o);
    if (lane == 0) {
        s_warp[warp] = running;
        s_k[warp] = ksum;
    }
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
        if (threadIdx.x == 0) {
            s_excl = e;
            unsigned long long k = 0;
            for (int w = 0; w < 8; ++w) k += s_k[w];
            if (k) atomicAdd(&hdr->k_total, k);
        }
    }
    __syncthreads();
    const uint32_t excl = s_excl;
#pragma unroll
    for (int j = 0; j < kCompactVec; ++j) {
        uint32_t pos = excl + warp_excl + off[j] + incl[j] - __popc(flags[j]);
        const uint32_t e0 = wbase + 4 * (32 * j + lane);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t i = e0 + e;
            if (i >= N) continue;
            const uint32_t c = bp.pdiv.div(i);
            if (c * bp.P == i) seg[c] = pos; // first record of camera c
            if (flags[j] >> e & 1u) {
                const uint32_t key = dkey[i];
                const ushort4 r = rects[i];
                if (pos < N) { // always true unless a look-back wait timed out
                    keys_out[pos] = key;
                    vals_out[pos] = i;
                }
                ++pos;
                const uint32_t slot = c - c0;
                if (slot < 2) {
#pragma unroll
                    for (int p = 0; p < 4; ++p) atomicAdd(&s_h[slot][p][(key >> (8 * p)) & 255u], 1u);
                    atomicAdd(&s_rd[slot][r.y], 1u);
                    atomicAdd(&s_rd[slot][r.w + 1], 0xffffffffu);
                } else {
#pragma unroll
                    for (int p = 0; p < 4; ++p) atomicAdd(&hist[(c * 4 + p) * 256 + ((key >> (8 * p)) & 255u)], 1u);
                    atomicAdd(rowdiff_at(bp, rowdiff, c, r.y), 1u);
                    atomicAdd(rowdiff_at(bp, rowdiff, c, r.w + 1), 0xffffffffu);
                }
            }
        }
    }
    if (part == nparts - 1 && threadIdx.x == 0) seg[bp.ncam] = sat_add(excl, total);
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * 4 * 256; i += 256) {
        const uint32_t slot = i >> 10;
        const uint32_t v = (&s_h[0][0][0])[i];
        if (v && c0 + slot < (uint32_t)bp.ncam) atomicAdd(&hist[(c0 + slot) * 1024 + (i & 1023)], v);
    }
    for (int i = threadIdx.x; i < nrd0; i += 256)
        if (s_rd[0][i]) atomicAdd(rowdiff_at(bp, rowdiff, c0, i), s_rd[0][i]);
    for (int i = threadIdx.x; i < nrd1; i += 256)
        if (s_rd[1][i]) atomicAdd(rowdiff_at(bp, rowdiff, c0 + 1, i), s_rd[1][i]);
}

// 2. plan (one CTA of 1024 threads): record partitions per camera (kSortTile
// records each: rec_parts[p] = (camera, chunk, first, end)); span count of every padded
// row (the inclusive prefix of the row differences: each camera's block sums
// to zero, so the prefix restarts at every camera) and its first span
// (rowbase, exclusive prefix over all rows); span partitions per row
// (kColTile spans each: span_parts[q] = (row | camera << 18, chunk, first, end)); the
// overlap totals and the capacity check.
__global__ void __launch_bounds__(1024)
plan_kernel(const __grid_constant__ BinPlan bp, WsHeader *hdr, const uint32_t *__restrict__ seg,
            uint4 *__restrict__ rec_parts, uint32_t max_rec_parts, const uint32_t *__restrict__ rowdiff,
            uint32_t *__restrict__ rowbase, uint4 *__restrict__ span_parts, uint32_t max_span_parts,
            uint32_t *__restrict__ rowq, uint32_t span_cap, uint32_t capacity, int ell)
{
    __shared__ uint32_t s_cum[kMaxCams + 1];
    __shared__ uint32_t s_warp[32];
    const int tid = threadIdx.x;
    if (tid == 0) {
        uint32_t acc = 0;
        for (int c = 0; c < bp.ncam; ++c) {
            s_cum[c] = acc;
            acc += (seg[c + 1] - seg[c] + kSortTile - 1) / kSortTile;
        }
        s_cum[bp.ncam] = acc;
        hdr->n_rec_parts = min(acc, max_rec_parts);
        hdr->n_vis = seg[bp.ncam];
    }
    __syncthreads();
    const uint32_t nrp = min(s_cum[bp.ncam], max_rec_parts);
    for (uint32_t p = tid; p < nrp; p += 1024) {
        int c = 0;
        while (c + 1 < bp.ncam && s_cum[c + 1] <= p) ++c;
        const uint32_t k = p - s_cum[c], beg = seg[c] + k * kSortTile;
        rec_parts[p] = make_uint4((uint32_t)c, k, beg, min(seg[c + 1], beg + kSortTile));
    }
    // rows: thread t owns padded rows [g0, g1)
    const int G = bp.G;
    const int per = (G + 1023) / 1024;
    const int g0 = min(G, tid * per), g1 = min(G, g0 + per);
    uint32_t dsum = 0;
    for (int g = g0; g < g1; ++g) dsum += rowdiff[g];
    uint32_t tot;
    uint32_t run = block_excl_scan<32>(dsum, s_warp, tot);
    uint32_t csum = 0;
    for (int g = g0; g < g1; ++g) {
        run += rowdiff[g];
        rowbase[g] = run; // span count of row g, for now
        csum += run;
    }
    __syncthreads();
    uint32_t R;
    uint32_t acc = block_excl_scan<32>(csum, s_warp, R);
    uint32_t nq = 0;
    for (int g = g0; g < g1; ++g) {
        const uint32_t cnt = rowbase[g];
        const uint32_t lo = min(acc, span_cap), hi = min(acc + cnt, span_cap);
        rowbase[g] = acc;
        acc += cnt;
        nq += (hi - lo + kColTile - 1) / kColTile;
    }
    if (tid == 1023) rowbase[G] = R;
    __syncthreads();
    uint32_t NQ;
    uint32_t q = block_excl_scan<32>(nq, s_warp, NQ);
    int c = 0;
    if (tid == 1023) rowq[G] = min(NQ, max_span_parts);
    for (int g = g0; g < g1; ++g) {
        while (c + 1 < bp.ncam && bp.cam[c + 1].gpad <= g) ++c;
        rowq[g] = min(q, max_span_parts);
        const uint32_t lo = min(rowbase[g], span_cap);
        const uint32_t hi = min(g + 1 == G ? R : rowbase[g + 1], span_cap);
        const uint32_t n = (hi - lo + kColTile - 1) / kColTile;
        for (uint32_t k = 0; k < n; ++k, ++q)
            if (q < max_span_parts)
                span_parts[q] = make_uint4((uint32_t)g | ((uint32_t)c << 18), k, lo + k * kColTile,
                                           min(hi, lo + (k + 1) * kColTile));
    }
    if (tid == 0) {
        hdr->n_span = R;
        hdr->n_span_parts = min(NQ, max_span_parts);
        unsigned long long raw = hdr->k_total;
        if (ell && (unsigned long long)R > raw) raw = R; // empty spans of rows the ellipse misses
        const uint32_t raw32 = raw >= kValMask ? kValMask : (uint32_t)raw;
        hdr->n_over_raw = raw32;
        hdr->n_over = min(raw32, capacity);
        if (raw > capacity || raw >= kValMask || R > span_cap) atomicOr(&hdr->err, (uint32_t)GS_ERR_CAPACITY);
    }
}

// One Onesweep pass over BITS bits starting at `shift`, over segments: the
// keys of segment c are [seg[c], seg[c+1]); partition p covers chunk k of
// segment c, keys [first, end): parts[p] = (c, k, first, end) (parts == NULL:
// one segment, chunk p). Keys
// move only within their segment. hist + c * hist_stride holds the
// segment's counts of this pass's digits. Dynamic shared memory: keys,
// values, per-warp digit counters, two per-digit tables.
template <int BITS>
constexpr size_t onesweep_smem()
{
    return sizeof(uint32_t) * (2 * kSortTile + 8 * (1 << BITS) + 2 * (1 << BITS) + 8 + 4);
}

template <int BITS>
__global__ void __launch_bounds__(kSortThreads, GS_SORT_MIN_BLOCKS) // the pass is latency-bound
onesweep_kernel(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                uint32_t *__restrict__ keys_out /* NULL: sorted keys not kept */, uint32_t *__restrict__ vals_out,
                const uint32_t *__restrict__ seg, const uint4 *__restrict__ parts, const uint32_t *nparts_ptr,
                int shift, const uint32_t *__restrict__ hist, int hist_stride, uint32_t *state, uint32_t *ctr,
                uint32_t *err)
{
    constexpr int R = 1 << BITS;
    constexpr uint32_t M = R - 1;
    constexpr int DPT = R / kSortThreads; // digits per thread (consecutive)
    extern __shared__ uint32_t smem[];
    uint32_t *s_keys = smem;
    uint32_t *s_vals = s_keys + kSortTile;
    uint32_t *s_whist = s_vals + kSortTile; // [8][R]
    uint32_t *s_bexcl = s_whist + 8 * R;
    uint32_t *s_goff = s_bexcl + R;
    uint32_t *s_warp = s_goff + R;
    uint32_t *s_part = s_warp + 8;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) *s_part = atomicAdd(ctr, 1u);
    for (int i = tid; i < 8 * R; i += kSortThreads) s_whist[i] = 0;
    __syncthreads();
    const uint32_t part = *s_part;
    const uint32_t nparts = parts ? *nparts_ptr : (seg[1] - seg[0] + kSortTile - 1) / kSortTile;
    if (part >= nparts) return;
    uint32_t c = 0, chunk = part, beg, end;
    if (parts) {
        const uint4 d = parts[part];
        c = d.x, chunk = d.y, beg = d.z, end = d.w;
    } else {
        beg = seg[0] + part * kSortTile;
        end = min(seg[1], beg + kSortTile);
    }
    const uint32_t sbeg = seg[c], send = seg[c + 1];

    // warp-striped load: warp w owns keys [beg + 32 I w, beg + 32 I (w + 1)), I = kSortItems
    const uint32_t wbase = beg + warp * (32 * kSortItems);
    uint32_t k[kSortItems], v[kSortItems], r[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t idx = wbase + j * 32 + lane;
        const bool ok = idx < end;
        k[j] = ok ? keys_in[idx] : 0xffffffffu; // invalid keys rank last (top digit, highest index)
        v[j] = ok ? vals_in[idx] : 0u;
    }
    // this thread's digits' segment counts, loaded now so that the latency
    // overlaps the ranking
    const uint32_t *hseg = hist + (size_t)c * hist_stride;
    uint32_t hv[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) hv[q] = hseg[tid * DPT + q];
    // rank within the warp: match lanes with equal digits
    const uint32_t lt = lanemask_lt();
    uint32_t *wh = s_whist + warp * R;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t d = (k[j] >> shift) & M;
        const uint32_t peers = warp_peers<BITS>(d);
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader) {
            old = wh[d];
            wh[d] = old + __popc(peers);
        }
        old = __shfl_sync(0xffffffffu, old, leader);
        r[j] = old + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    // per digit: warp-exclusive offsets and block counts
    uint32_t cnt[DPT], csum = 0, hsum = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = tid * DPT + q;
        uint32_t cc = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const uint32_t x = s_whist[w * R + d];
            s_whist[w * R + d] = cc;
            cc += x;
        }
        cnt[q] = cc;
        csum += cc;
        hsum += hv[q];
    }
    uint32_t tot;
    uint32_t bex = block_excl_scan<8>(csum, s_warp, tot);
    __syncthreads();
    uint32_t hex = sbeg + block_excl_scan<8>(hsum, s_warp, tot);
    // invalid keys exist only in a segment's last partition, all with the top digit
    const uint32_t n_here = end > beg ? end - beg : 0u;
    const uint32_t n_invalid = kSortTile - n_here;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = tid * DPT + q;
        s_bexcl[d] = bex;
        bex += cnt[q];
        const uint32_t agg = cnt[q] - (d == (int)M ? n_invalid : 0u);
        const uint32_t excl = publish_digit<kLookWindow>(state, part, chunk, R, d, agg, err);
        s_goff[d] = hex + excl;
        hex += hv[q];
    }
    __syncthreads();
    // scatter into shared memory in digit order
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t d = (k[j] >> shift) & M;
        const uint32_t lp = s_bexcl[d] + wh[d] + r[j];
        s_keys[lp] = k[j];
        s_vals[lp] = v[j];
    }
    __syncthreads();
    for (uint32_t i = tid; i < n_here; i += kSortThreads) {
        const uint32_t key = s_keys[i];
        const uint32_t d = (key >> shift) & M;
        const uint32_t o = s_goff[d] + i - s_bexcl[d];
        if (o < send) { // always true unless a look-back wait timed out
            if (keys_out) keys_out[o] = key;
            vals_out[o] = s_vals[i];
        }
    }
}

// Shared-memory words of the split kernels: per warp a counter per digit
// (D = max digits + 1 slots), plus the partition id.
inline size_t split_smem(int max_digits) { return sizeof(uint32_t) * (8 * (size_t)(max_digits + 1) + 4); }

// 4. row split. Partition p = chunk k of camera c's depth-sorted records
// (the depth sort's partition table). Warp w takes records
// [beg + 32 I w, beg + 32 I (w + 1)), I = kRowItems, and expands them in
// order into one span per covered tile row; a span's place is its row's
// first span (rowbase) + the counts of that row in the camera's earlier
// partitions (look-back) + in earlier warps of this partition + earlier in
// this warp. Span = (record index, first column | last column << 16); a row
// the ellipse misses (GS_RECT_ELLIPSE) gets an empty span (first > last).
template <bool ELL>
__global__ void __launch_bounds__(256, 2)
rows_kernel(const __grid_constant__ BinPlan bp, const uint32_t *__restrict__ seg, const uint4 *__restrict__ parts,
            const WsHeader *hdr, const uint32_t *__restrict__ ids, const ushort4 *__restrict__ rects,
            const float4 *__restrict__ rec, uint32_t N, const uint32_t *__restrict__ rowbase,
            uint2 *__restrict__ spans, uint32_t span_cap, uint32_t *state, uint32_t *ctr, uint32_t *err)
{
    extern __shared__ uint32_t smem[];
    const int D = bp.max_ty + 1;
    uint32_t *s_cnt = smem; // [8][D]
    uint32_t *s_part = smem + 8 * D;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t nparts = hdr->n_rec_parts;
    uint32_t *wc = s_cnt + warp * D;
    while (true) {
        for (int i = tid; i < 8 * D; i += 256) s_cnt[i] = 0;
        if (tid == 0) *s_part = atomicAdd(ctr, 1u);
        __syncthreads();
        const uint32_t part = *s_part;
        if (part >= nparts) break;
        const uint4 pc = parts[part];
        const int c = (int)pc.x;
        const uint32_t chunk = pc.y, beg = pc.z, end = pc.w;
        const int ty = bp.cam[c].tiles_y, tx = bp.cam[c].tiles_x;
        const uint32_t wb = beg + warp * (32 * kRowItems);
        // a drawn record's rectangle lies inside its camera's tile grid; the
        // checks only matter after a timed-out wait left stale entries
        auto usable = [&](uint32_t id, ushort4 r) {
            return id < N && r.y <= r.w && r.w < ty && r.x <= r.z && r.z < tx;
        };
        // this thread's records, all loads in flight at once: index, then
        // rectangle as first | last column and first | last row (rows
        // 0xffff | 0 marks a record to skip)
        uint32_t rid[kRowItems], rxr[kRowItems], ryr[kRowItems];
#pragma unroll
        for (int j = 0; j < kRowItems; ++j) {
            const uint32_t idx = wb + 32 * j + lane;
            rid[j] = idx < end ? ids[idx] : N;
        }
#pragma unroll
        for (int j = 0; j < kRowItems; ++j) {
            const ushort4 r = rid[j] < N ? rects[rid[j]] : make_ushort4(1, 1, 0, 0);
            const bool ok = usable(rid[j], r);
            rxr[j] = (uint32_t)r.x | ((uint32_t)r.z << 16);
            ryr[j] = ok ? ((uint32_t)r.y | ((uint32_t)r.w << 16)) : 0xffffu;
        }
        // per-warp row counts as a difference array
#pragma unroll
        for (int j = 0; j < kRowItems; ++j) {
            const uint32_t y0 = ryr[j] & 0xffffu, y1 = ryr[j] >> 16;
            if (y0 <= y1) {
                atomicAdd(&wc[y0], 1u);
                atomicAdd(&wc[y1 + 1], 0xffffffffu);
            }
        }
        __syncwarp();
        uint32_t carry = 0;
        for (int y0 = 0; y0 < ty; y0 += 32) {
            const int y = y0 + lane;
            const uint32_t x = warp_incl_scan(y < ty ? wc[y] : 0u) + carry;
            if (y < ty) wc[y] = x;
            carry = __shfl_sync(0xffffffffu, x, 31);
        }
        __syncthreads();
        const int gp = bp.cam[c].gpad;
        for (int y = tid; y < ty; y += 256) {
            uint32_t a = 0;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const uint32_t x = s_cnt[w * D + y];
                s_cnt[w * D + y] = a;
                a += x;
            }
            const uint32_t base = rowbase[gp + y] + publish_digit<kSplitWindow>(state, part, chunk, bp.max_ty, y, a, err);
#pragma unroll
            for (int w = 0; w < 8; ++w) s_cnt[w * D + y] += base;
        }
        __syncthreads();
        const int W = bp.cam[c].W, H = bp.cam[c].H;
#pragma unroll
        for (int j = 0; j < kRowItems; ++j) {
            if (wb + 32 * j >= end) break; // uniform per warp
            const uint32_t id = rid[j], xr = rxr[j], yr = ryr[j];
            const uint32_t y0 = yr & 0xffffu, y1 = yr >> 16;
            const uint32_t h = y0 <= y1 ? y1 - y0 + 1u : 0u;
            const uint32_t incl = warp_incl_scan(h);
            const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
            for (uint32_t b = 0; b < tot; b += 32) {
                const uint32_t p = b + lane;
                const uint32_t pq = min(p, tot - 1u);
                const int e = owner_lane(incl, pq);
                const uint32_t eid = __shfl_sync(0xffffffffu, id, e);
                const uint32_t exr = __shfl_sync(0xffffffffu, xr, e);
                const uint32_t eyr = __shfl_sync(0xffffffffu, yr, e);
                const uint32_t ebeg = __shfl_sync(0xffffffffu, incl - h, e);
                const bool act = p < tot;
                const uint32_t y = (eyr & 0xffffu) + (pq - ebeg);
                uint32_t span_x = exr;
                if (ELL && act) {
                    const int x0 = (int)(exr & 0xffffu), x1 = (int)(exr >> 16);
                    const bool simple = x0 == x1 || (eyr & 0xffffu) == (eyr >> 16);
                    if (!simple) {
                        const float4 g0 = rec[3 * (size_t)eid], g1 = rec[3 * (size_t)eid + 1];
                        int a0, a1;
                        span_x = row_cols(g0.x, g0.y, g1.x, g1.y, g1.z, g1.w, (int)y, bp.tile_w, bp.tile_h, W, H,
                                          x0, x1, a0, a1)
                                     ? ((uint32_t)a0 | ((uint32_t)a1 << 16))
                                     : 0xffffu;
                    }
                }
                const uint32_t pos = split_rank(wc, act ? y : 0u, act, lt);
                if (act && pos < span_cap) spans[pos] = make_uint2(eid, span_x);
            }
        }
        __syncthreads();
    }
}

// Camera c, tile row y and [beg, end) of span partition `part`.
struct SpanPart {
    int c, y;
    uint32_t chunk, beg, end;
};
__device__ __forceinline__ SpanPart span_part(const BinPlan &bp, const uint4 pc)
{
    SpanPart s;
    const int g = (int)(pc.x & 0x3ffffu);
    s.c = (int)(pc.x >> 18);
    s.y = g - bp.cam[s.c].gpad;
    s.chunk = pc.y;
    s.beg = pc.z;
    s.end = pc.w;
    return s;
}

// 5. tile counts: per span partition a difference array over the row's
// columns; either written as the partition's row of the column-count matrix
// (colmat[q][x], turned into offsets by col_offsets_kernel) or added to the
// tiles' counters.
__global__ void GS_SPLIT_BOUNDS
cols_count_kernel(const __grid_constant__ BinPlan bp, const uint4 *__restrict__ parts, const WsHeader *hdr,
                  const uint32_t *__restrict__ rowbase, const uint2 *__restrict__ spans, uint32_t span_cap,
                  uint32_t *__restrict__ tile_cnt, uint32_t *__restrict__ colmat, uint32_t *ctr)
{
    extern __shared__ uint32_t smem[];
    const int D = bp.max_tx + 1;
    uint32_t *s_d = smem;
    uint32_t *s_part = smem + 8 * D;
    const int tid = threadIdx.x;
    const uint32_t nparts = hdr->n_span_parts;
    while (true) {
        for (int i = tid; i < D; i += 256) s_d[i] = 0;
        if (tid == 0) *s_part = atomicAdd(ctr, 1u);
        __syncthreads();
        const uint32_t part = *s_part;
        if (part >= nparts) break;
        const SpanPart sp = span_part(bp, parts[part]);
        const int tx = bp.cam[sp.c].tiles_x;
        const uint32_t end = sp.y < bp.cam[sp.c].tiles_y ? sp.end : sp.beg; // the padding row has no spans
        for (uint32_t i = sp.beg + tid; i < end; i += 256) {
            const uint32_t xr = spans[i].y;
            const uint32_t x0 = xr & 0xffffu, x1 = xr >> 16;
            if (x0 <= x1 && x1 < (uint32_t)tx) {
                atomicAdd(&s_d[x0], 1u);
                atomicAdd(&s_d[x1 + 1], 0xffffffffu);
            }
        }
        __syncthreads();
        if (tid < 32) {
            uint32_t *tc = tile_cnt + bp.cam[sp.c].tile_base + (uint32_t)sp.y * tx;
            uint32_t *cm = colmat ? colmat + (size_t)part * bp.max_tx : nullptr;
            uint32_t carry = 0;
            for (int x0 = 0; x0 < tx; x0 += 32) {
                const int x = x0 + tid;
                const uint32_t v = warp_incl_scan(x < tx ? s_d[x] : 0u) + carry;
                if (cm) {
                    if (x < tx) cm[x] = v;
                } else if (x < tx && v) {
                    atomicAdd(&tc[x], v);
                }
                carry = __shfl_sync(0xffffffffu, v, 31);
            }
        }
        __syncthreads();
    }
}

// 5b. per tile (c, y, x): the exclusive prefix of colmat[q][x] over row
// (c, y)'s partitions q in order, in place, and the tile's count. One CTA per
// padded row.
__global__ void __launch_bounds__(128)
col_offsets_kernel(const __grid_constant__ BinPlan bp, const uint32_t *__restrict__ rowq,
                   uint32_t *__restrict__ colmat, uint32_t *__restrict__ tile_cnt)
{
    const int g = blockIdx.x;
    int c = 0;
    while (c + 1 < bp.ncam && bp.cam[c + 1].gpad <= g) ++c;
    const int y = g - bp.cam[c].gpad, tx = bp.cam[c].tiles_x;
    if (y >= bp.cam[c].tiles_y) return; // the padding row
    const uint32_t q0 = rowq[g], q1 = rowq[g + 1];
    uint32_t *tc = tile_cnt + bp.cam[c].tile_base + (uint32_t)y * tx;
    for (int x = threadIdx.x; x < tx; x += 128) {
        uint32_t acc = 0;
        for (uint32_t q = q0; q < q1; ++q) {
            uint32_t *m = colmat + (size_t)q * bp.max_tx + x;
            const uint32_t v = *m;
            *m = acc;
            acc += v;
        }
        tc[x] = acc;
    }
}

// 6. per-tile ranges: exclusive scan of the tile counts (single pass,
// decoupled look-back), clamped to the capacity; (0, 0) for an empty tile.
__global__ void __launch_bounds__(256)
tile_scan_kernel(const uint32_t *__restrict__ tile_cnt, uint32_t T, uint2 *__restrict__ ranges, uint32_t cap,
                 WsHeader *hdr, uint32_t *state)
{
    __shared__ uint32_t s_part, s_excl, s_warp[8];
    if (threadIdx.x == 0) s_part = atomicAdd(&hdr->ctr[CTR_SCAN], 1u);
    __syncthreads();
    const uint32_t part = s_part;
    const uint32_t t0 = part * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems], sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = t0 + i < T ? tile_cnt[t0 + i] : 0u;
        sum += v[i];
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan<8>(sum, s_warp, tot);
    if (threadIdx.x < 32) {
        const uint32_t e = lookback_scalar(state, part, tot, &hdr->err);
        if (threadIdx.x == 0) s_excl = e;
    }
    __syncthreads();
    uint32_t base = s_excl + ex;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        // an empty tile reads (0, 0), as a zero-filled table would
        if (t0 + i < T) ranges[t0 + i] = v[i] ? make_uint2(min(base, cap), min(base + v[i], cap)) : make_uint2(0u, 0u);
        base += v[i];
    }
}

// 7. column split. Partition q = chunk k of row (c, y)'s spans. Warp w
// takes spans [beg + 32 I w, beg + 32 I (w + 1)), I = kColItems, and expands
// them in order into one entry per covered column; the entry's place is its
// tile's range start + the counts of that column in the row's earlier
// partitions (look-back) + in earlier warps + earlier in this warp. Writes
// the record index there (places at or past the capacity are dropped; the
// overflow is flagged by the plan).
__global__ void __launch_bounds__(256, 2)
cols_kernel(const __grid_constant__ BinPlan bp, const uint4 *__restrict__ parts, const WsHeader *hdr,
            const uint32_t *__restrict__ rowbase, const uint2 *__restrict__ spans, uint32_t span_cap,
            const uint2 *__restrict__ ranges, uint32_t *__restrict__ vals, uint32_t cap, uint32_t *state,
            uint32_t *ctr, uint32_t *err)
{
    extern __shared__ uint32_t smem[];
    const int D = bp.max_tx + 1;
    uint32_t *s_cnt = smem; // [8][D]
    uint32_t *s_part = smem + 8 * D;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t nparts = hdr->n_span_parts;
    uint32_t *wc = s_cnt + warp * D;
    while (true) {
        for (int i = tid; i < 8 * D; i += 256) s_cnt[i] = 0;
        if (tid == 0) *s_part = atomicAdd(ctr, 1u);
        __syncthreads();
        const uint32_t part = *s_part;
        if (part >= nparts) break;
        SpanPart sp = span_part(bp, parts[part]);
        const int tx = bp.cam[sp.c].tiles_x;
        if (sp.y >= bp.cam[sp.c].tiles_y) sp.end = sp.beg; // the padding row has no spans
        const uint32_t wb = sp.beg + warp * (32 * kColItems);
        // this thread's spans, all loads in flight at once (columns 0xffff | 0
        // mark an empty span or a slot past the partition)
        uint32_t sid[kColItems], sxr[kColItems];
#pragma unroll
        for (int j = 0; j < kColItems; ++j) {
            const uint32_t idx = wb + 32 * j + lane;
            const uint2 v = idx < sp.end ? spans[idx] : make_uint2(0u, 0xffffu);
            const uint32_t x0 = v.y & 0xffffu, x1 = v.y >> 16;
            sid[j] = v.x;
            sxr[j] = (x0 <= x1 && x1 < (uint32_t)tx) ? v.y : 0xffffu;
        }
#pragma unroll
        for (int j = 0; j < kColItems; ++j) {
            const uint32_t x0 = sxr[j] & 0xffffu, x1 = sxr[j] >> 16;
            if (x0 <= x1) {
                atomicAdd(&wc[x0], 1u);
                atomicAdd(&wc[x1 + 1], 0xffffffffu);
            }
        }
        __syncwarp();
        uint32_t carry = 0;
        for (int x0 = 0; x0 < tx; x0 += 32) {
            const int x = x0 + lane;
            const uint32_t v = warp_incl_scan(x < tx ? wc[x] : 0u) + carry;
            if (x < tx) wc[x] = v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
        __syncthreads();
        const uint32_t trow = (uint32_t)bp.cam[sp.c].tile_base + (uint32_t)sp.y * tx;
        for (int x = tid; x < tx; x += 256) {
            uint32_t a = 0;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const uint32_t v = s_cnt[w * D + x];
                s_cnt[w * D + x] = a;
                a += v;
            }
            const uint32_t base = ranges[trow + x].x + publish_digit<kSplitWindow>(state, part, sp.chunk, bp.max_tx, x, a, err);
#pragma unroll
            for (int w = 0; w < 8; ++w) s_cnt[w * D + x] += base;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kColItems; ++j) {
            if (wb + 32 * j >= sp.end) break; // uniform per warp
            const uint32_t id = sid[j], x0 = sxr[j] & 0xffffu, x1 = sxr[j] >> 16;
            const uint32_t n = x0 <= x1 ? x1 - x0 + 1u : 0u;
            const uint32_t incl = warp_incl_scan(n);
            const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
            for (uint32_t b = 0; b < tot; b += 32) {
                const uint32_t p = b + lane;
                const uint32_t pq = min(p, tot - 1u);
                const int e = owner_lane(incl, pq);
                const uint32_t eid = __shfl_sync(0xffffffffu, id, e);
                const uint32_t ex0 = __shfl_sync(0xffffffffu, x0, e);
                const uint32_t ebeg = __shfl_sync(0xffffffffu, incl - n, e);
                const bool act = p < tot;
                const uint32_t x = ex0 + (pq - ebeg);
                const uint32_t pos = split_rank(wc, act ? x : 0u, act, lt);
                if (act && pos < cap) vals[pos] = eid;
            }
        }
        __syncthreads();
    }
}

// ---- split kernels with thread-private counters ---------------------------
// The same two splits for cameras of at most kThreadDigits tile rows /
// columns. Thread t of a partition owns its items [beg + I t, beg + I (t + 1)),
// I = 20, in order, and a private 16-bit counter per digit in shared memory
// (cnt[d][t]). Stable places then need no ranking inside a warp: count each
// thread's items per digit, turn the counters into the exclusive prefix over
// the threads (plus the digit's offset from the look-back), and let every
// thread write its items in order, taking and advancing its own counter.
// Counts per thread are at most I x (digits covered), prefixes at most the
// partition's items (kSortTile or kColTile records / spans): 16 bits hold both
// as long as a digit's prefix stays below 2^16, i.e. any partition here.
constexpr int kThreadDigits = 384;
constexpr int kTItems = 20;
static_assert(kTItems * 256 == kSortTile && kTItems * 256 == kColTile, "partition sizes");

inline size_t tsplit_smem(int max_digits)
{
    return sizeof(uint16_t) * 256 * (size_t)max_digits + sizeof(uint32_t) * ((size_t)max_digits + 4) + 32;
}

// cnt[d][0..256) for d < nd: exclusive prefix over the threads in place; the
// digit's total to tot[d]. Warp w takes digits w, w + 8, ..., two at a time
// (independent chains); lane l holds threads 8 l .. 8 l + 7 (one 16-byte word).
__device__ __forceinline__ uint32_t tsplit_prefix8(uint4 &q)
{
    uint32_t w[4] = {q.x, q.y, q.z, q.w}, v[8], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = w[k] & 0xffffu;
        v[2 * k + 1] = w[k] >> 16;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t x = v[k];
        v[k] = s;
        s += x;
    }
    q = make_uint4(v[0] | (v[1] << 16), v[2] | (v[3] << 16), v[4] | (v[5] << 16), v[6] | (v[7] << 16));
    return s;
}

__device__ __forceinline__ uint4 add16x2(uint4 q, uint32_t e)
{
    const uint32_t ee = e | (e << 16); // no carries: every sum stays below 2^16
    return make_uint4(q.x + ee, q.y + ee, q.z + ee, q.w + ee);
}

__device__ __forceinline__ void tsplit_scan(uint16_t *cnt, uint32_t *tot, int nd)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = warp; d < nd; d += 16) {
        const int d2 = d + 8;
        const bool two = d2 < nd;
        uint4 *r0 = reinterpret_cast<uint4 *>(cnt + (size_t)d * 256);
        uint4 *r1 = reinterpret_cast<uint4 *>(cnt + (size_t)(two ? d2 : d) * 256);
        uint4 q0 = r0[lane], q1 = two ? r1[lane] : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t s0 = tsplit_prefix8(q0), s1 = tsplit_prefix8(q1);
        const uint32_t i0 = warp_incl_scan(s0), i1 = warp_incl_scan(s1);
        r0[lane] = add16x2(q0, i0 - s0);
        if (two) r1[lane] = add16x2(q1, i1 - s1);
        if (lane == 31) {
            tot[d] = i0;
            if (two) tot[d2] = i1;
        }
    }
}

// A persistent split kernel claims a partition only when it is ready to
// process it (a partition claimed early would hold up the look-back of every
// later one); thread 0 claims it and loads its descriptor for the CTA.
struct NextPart {
    uint32_t part;
    uint4 desc;
};

template <bool ELL>
__global__ void __launch_bounds__(256, 2)
rows_t_kernel(const __grid_constant__ BinPlan bp, const uint32_t *__restrict__ seg, const uint4 *__restrict__ parts,
              const WsHeader *hdr, const uint32_t *__restrict__ ids, const ushort4 *__restrict__ rects,
              const float4 *__restrict__ rec, uint32_t N, const uint32_t *__restrict__ rowbase,
              uint2 *__restrict__ spans, uint32_t span_cap, uint32_t *state, uint32_t *ctr, uint32_t *err)
{
    extern __shared__ uint32_t smem[];
    const int ND = bp.max_ty;
    uint16_t *cnt = reinterpret_cast<uint16_t *>(smem); // [ND][256]
    uint32_t *sbase = smem + (size_t)ND * 128;           // [ND]
    NextPart *s_next = reinterpret_cast<NextPart *>(sbase + ((ND + 3) & ~3));
    const int tid = threadIdx.x;
    const uint32_t nparts = hdr->n_rec_parts;
    uint4 *z = reinterpret_cast<uint4 *>(smem);
    while (true) {
        for (int i = tid; i < ND * 32; i += 256) z[i] = make_uint4(0u, 0u, 0u, 0u);
        if (tid == 0) {
            const uint32_t p0 = atomicAdd(ctr, 1u);
            s_next->part = p0;
            s_next->desc = p0 < nparts ? parts[p0] : make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        const uint32_t part = s_next->part;
        if (part >= nparts) break;
        const uint4 pc = s_next->desc;
        const int c = (int)pc.x;
        const uint32_t chunk = pc.y, beg = pc.z, end = pc.w;
        const int ty = bp.cam[c].tiles_y, tx = bp.cam[c].tiles_x;
        const int gp = bp.cam[c].gpad;
        // this thread's digits' first spans, used after the look-back
        const uint32_t rb0 = tid < ty ? rowbase[gp + tid] : 0u;
        const uint32_t rb1 = tid + 256 < ty ? rowbase[gp + tid + 256] : 0u;
        const uint32_t t0 = beg + tid * kTItems;
        uint32_t rid[kTItems], rxr[kTItems], ryr[kTItems];
#pragma unroll
        for (int j = 0; j < kTItems; ++j) rid[j] = t0 + j < end ? ids[t0 + j] : N;
#pragma unroll
        for (int j = 0; j < kTItems; ++j) {
            const ushort4 r = rid[j] < N ? rects[rid[j]] : make_ushort4(1, 1, 0, 0);
            // a drawn record's rectangle lies inside its camera's grid; the
            // check only matters after a timed-out wait left stale entries
            const bool ok = rid[j] < N && r.y <= r.w && r.w < ty && r.x <= r.z && r.z < tx;
            rxr[j] = (uint32_t)r.x | ((uint32_t)r.z << 16);
            ryr[j] = ok ? ((uint32_t)r.y | ((uint32_t)r.w << 16)) : 0xffffu;
        }
        uint16_t *my = cnt + tid;
#pragma unroll
        for (int j = 0; j < kTItems; ++j) {
            const int y1 = (int)(ryr[j] >> 16);
            for (int y = (int)(ryr[j] & 0xffffu); y <= y1; ++y) my[y * 256] += 1;
        }
        __syncthreads();
        tsplit_scan(cnt, sbase, ty);
        __syncthreads();
        if (tid < ty)
            sbase[tid] = rb0 + publish_digit<kSplitWindow>(state, part, chunk, bp.max_ty, tid, sbase[tid], err);
        if (tid + 256 < ty)
            sbase[tid + 256] =
                rb1 + publish_digit<kSplitWindow>(state, part, chunk, bp.max_ty, tid + 256, sbase[tid + 256], err);
        __syncthreads();
        const int W = bp.cam[c].W, H = bp.cam[c].H;
#pragma unroll
        for (int j = 0; j < kTItems; ++j) {
            const int y0 = (int)(ryr[j] & 0xffffu), y1 = (int)(ryr[j] >> 16);
            const uint32_t id = rid[j];
            const int x0 = (int)(rxr[j] & 0xffffu), x1 = (int)(rxr[j] >> 16);
            float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
            const bool cut = ELL && y0 < y1 && x0 < x1; // a single row or column keeps its tiles
            if (cut) {
                g0 = rec[3 * (size_t)id];
                g1 = rec[3 * (size_t)id + 1];
            }
            for (int y = y0; y <= y1; ++y) {
                const uint32_t k = my[y * 256];
                my[y * 256] = (uint16_t)(k + 1u);
                const uint32_t pos = sbase[y] + k;
                uint32_t sx = rxr[j];
                if (cut) {
                    int a0, a1;
                    sx = row_cols(g0.x, g0.y, g1.x, g1.y, g1.z, g1.w, y, bp.tile_w, bp.tile_h, W, H, x0, x1, a0, a1)
                             ? ((uint32_t)a0 | ((uint32_t)a1 << 16))
                             : 0xffffu;
                }
                if (pos < span_cap) spans[pos] = make_uint2(id, sx);
            }
        }
        __syncthreads();
    }
}

__global__ void GS_SPLIT_BOUNDS
cols_t_kernel(const __grid_constant__ BinPlan bp, const uint4 *__restrict__ parts, const WsHeader *hdr,
              const uint32_t *__restrict__ rowbase, const uint2 *__restrict__ spans, uint32_t span_cap,
              const uint32_t *__restrict__ colmat, const uint2 *__restrict__ ranges, uint32_t *__restrict__ vals,
              uint32_t cap, uint32_t *state, uint32_t *ctr, uint32_t *err)
{
    extern __shared__ uint32_t smem[];
    const int ND = bp.max_tx;
    uint16_t *cnt = reinterpret_cast<uint16_t *>(smem); // [ND][256]
    uint32_t *sbase = smem + (size_t)ND * 128;           // [ND]
    NextPart *s_next = reinterpret_cast<NextPart *>(sbase + ((ND + 3) & ~3));
    const int tid = threadIdx.x;
    const uint32_t nparts = hdr->n_span_parts;
    uint4 *z = reinterpret_cast<uint4 *>(smem);
    while (true) {
        for (int i = tid; i < ND * 32; i += 256) z[i] = make_uint4(0u, 0u, 0u, 0u);
        if (tid == 0) {
            const uint32_t p0 = atomicAdd(ctr, 1u);
            s_next->part = p0;
            s_next->desc = p0 < nparts ? parts[p0] : make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        const uint32_t part = s_next->part;
        if (part >= nparts) break;
        SpanPart sp = span_part(bp, s_next->desc);
        const int tx = bp.cam[sp.c].tiles_x;
        if (sp.y >= bp.cam[sp.c].tiles_y) sp.end = sp.beg; // the padding row has no spans
        const uint32_t trow = (uint32_t)bp.cam[sp.c].tile_base + (uint32_t)sp.y * tx;
        // this thread's digits' first places: the tile's start, plus with the
        // column-count matrix the counts of the row's earlier partitions
        const uint32_t *cm = colmat ? colmat + (size_t)part * bp.max_tx : nullptr;
        const uint32_t tb0 = tid < tx ? ranges[trow + tid].x + (cm ? cm[tid] : 0u) : 0u;
        const uint32_t tb1 = tid + 256 < tx ? ranges[trow + tid + 256].x + (cm ? cm[tid + 256] : 0u) : 0u;
        const uint32_t t0 = sp.beg + tid * kTItems;
        uint32_t sid[kTItems], sxr[kTItems];
#pragma unroll
        for (int j = 0; j < kTItems; ++j) {
            const uint2 v = t0 + j < sp.end ? spans[t0 + j] : make_uint2(0u, 0xffffu);
            const uint32_t x0 = v.y & 0xffffu, x1 = v.y >> 16;
            sid[j] = v.x;
            sxr[j] = (x0 <= x1 && x1 < (uint32_t)tx) ? v.y : 0xffffu;
        }
        uint16_t *my = cnt + tid;
#pragma unroll
        for (int j = 0; j < kTItems; ++j) {
            const int x1 = (int)(sxr[j] >> 16);
            for (int x = (int)(sxr[j] & 0xffffu); x <= x1; ++x) my[x * 256] += 1;
        }
        __syncthreads();
        tsplit_scan(cnt, sbase, tx);
        __syncthreads();
        if (cm) {
            if (tid < tx) sbase[tid] = tb0;
            if (tid + 256 < tx) sbase[tid + 256] = tb1;
        } else {
            if (tid < tx)
                sbase[tid] = tb0 + publish_digit<kSplitWindow>(state, part, sp.chunk, bp.max_tx, tid, sbase[tid], err);
            if (tid + 256 < tx)
                sbase[tid + 256] = tb1 + publish_digit<kSplitWindow>(state, part, sp.chunk, bp.max_tx, tid + 256,
                                                                     sbase[tid + 256], err);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kTItems; ++j) {
            const int x1 = (int)(sxr[j] >> 16);
            const uint32_t id = sid[j];
            for (int x = (int)(sxr[j] & 0xffffu); x <= x1; ++x) {
                const uint32_t k = my[x * 256];
                my[x * 256] = (uint16_t)(k + 1u);
                const uint32_t pos = sbase[x] + k;
                if (pos < cap) vals[pos] = id;
            }
        }
        __syncthreads();
    }
}

// Optional 64-bit keys of the sorted lists (tile << 32 | depth bits): one
// warp per tile.
__global__ void __launch_bounds__(256)
keys64_kernel(const uint2 *__restrict__ ranges, uint32_t T, const uint32_t *__restrict__ vals,
              const uint32_t *__restrict__ dkey, uint32_t N, unsigned long long *__restrict__ keys64)
{
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t t = (blockIdx.x * 256 + threadIdx.x) >> 5; t < T; t += gridDim.x * 8) {
        const uint2 rg = ranges[t];
        for (uint32_t i = rg.x + lane; i < rg.y; i += 32) {
            const uint32_t v = vals[i];
            keys64[i] = ((unsigned long long)t << 32) | (v < N ? dkey[v] : 0xffffffffu);
        }
    }
}

struct WsLayout {
    size_t hdr, hist, rowdiff, seg, st_compact, st_depth, st_rows, st_cols, st_scan, tile_cnt, zero_end;
    size_t rowbase, rowq, rec_parts, span_parts, colmat, dk0, dk1, dv0, dv1, spans, total;
    uint32_t max_rec_parts, max_span_parts;
    size_t st_depth_stride; // uint32 entries per pass
};

WsLayout ws_layout(const BinPlan &bp, int64_t N, int64_t cap, int64_t total_tiles)
{
    WsLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += align256(bytes); return r; };
    L.max_rec_parts = (uint32_t)((N + kSortTile - 1) / kSortTile + bp.ncam);
    L.max_span_parts = (uint32_t)((cap + kColTile - 1) / kColTile + bp.G);
    L.st_depth_stride = (size_t)256 * L.max_rec_parts;
    L.hdr = take(sizeof(WsHeader));
    L.hist = take(sizeof(uint32_t) * 1024 * bp.ncam);
    L.rowdiff = take(sizeof(uint32_t) * bp.G);
    L.seg = take(sizeof(uint32_t) * (bp.ncam + 1));
    L.st_compact = take(sizeof(uint32_t) * ((N + kCompactTile - 1) / kCompactTile + 1));
    L.st_depth = take(sizeof(uint32_t) * 4 * L.st_depth_stride);
    L.st_rows = take(sizeof(uint32_t) * (size_t)bp.max_ty * L.max_rec_parts);
    L.st_cols = take(sizeof(uint32_t) * (size_t)bp.max_tx * L.max_span_parts);
    L.st_scan = take(sizeof(uint32_t) * ((total_tiles + kScanTile - 1) / kScanTile + 1));
    L.tile_cnt = take(sizeof(uint32_t) * total_tiles);
    L.zero_end = o;
    L.rowbase = take(sizeof(uint32_t) * (bp.G + 1));
    L.rowq = take(sizeof(uint32_t) * (bp.G + 1));
    L.rec_parts = take(sizeof(uint4) * L.max_rec_parts);
    L.span_parts = take(sizeof(uint4) * L.max_span_parts);
    L.colmat = take(bp.max_tx <= kThreadDigits ? sizeof(uint32_t) * (size_t)bp.max_tx * L.max_span_parts : 0);
    L.dk0 = take(sizeof(uint32_t) * N + 16);
    L.dk1 = take(sizeof(uint32_t) * N);
    L.dv0 = take(sizeof(uint32_t) * N);
    L.dv1 = take(sizeof(uint32_t) * N);
    L.spans = take(sizeof(uint2) * cap);
    L.total = o;
    return L;
}

bool make_bin_plan(const CamTable &t, const gs_config *cfg, int32_t P, BinPlan *bp)
{
    bp->ncam = t.ncam;
    bp->P = (uint32_t)std::max(P, 1);
    bp->pdiv = FastDiv::make(bp->P);
    bp->tile_w = cfg->tile_w;
    bp->tile_h = cfg->tile_h;
    int g = 0, mx = 1, my = 1;
    for (int c = 0; c < kMaxCams; ++c) {
        BinCam &b = bp->cam[c];
        if (c >= t.ncam) {
            b = BinCam{0, 0, 0, g, 0, 0};
            continue;
        }
        const CamDev &d = t.cam[c];
        if (d.tiles_x > kMaxDigits || d.tiles_y > kMaxDigits) return false;
        b = BinCam{d.tiles_x, d.tiles_y, d.tile_base, g, d.W, d.H};
        g += d.tiles_y + 1;
        mx = std::max(mx, d.tiles_x);
        my = std::max(my, d.tiles_y);
    }
    bp->G = g;
    bp->max_tx = mx;
    bp->max_ty = my;
    return true;
}

// Sets the dynamic shared-memory opt-in of a kernel once per device (so that
// later calls, e.g. under stream capture, only launch).
template <typename K>
cudaError_t smem_optin(K kernel, size_t bytes, bool *done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && dev < 64) done[dev] = true;
    return e;
}

template <int BITS>
cudaError_t launch_onesweep(unsigned grid, cudaStream_t s, const uint32_t *ki, const uint32_t *vi,
                            uint32_t *ko, uint32_t *vo, const uint32_t *seg, const uint4 *parts,
                            const uint32_t *nparts, int shift, const uint32_t *hist, int hist_stride,
                            uint32_t *state, uint32_t *ctr, uint32_t *err)
{
    const size_t sm = onesweep_smem<BITS>();
    static bool attr_set[64] = {};
    cudaError_t e = smem_optin(onesweep_kernel<BITS>, sm, attr_set);
    if (e != cudaSuccess) return e;
    onesweep_kernel<BITS><<<grid ? grid : 1, kSortThreads, sm, s>>>(ki, vi, ko, vo, seg, parts, nparts, shift,
                                                                   hist, hist_stride, state, ctr, err);
    count_launch();
    return cudaPeekAtLastError();
}

// Grid of a persistent split kernel: as many CTAs as fit on every SM at once
// (so that no partition waits for a CTA that is not resident), never more
// than partitions can exist.
template <typename K>
unsigned split_grid(K kernel, size_t smem, uint32_t max_parts)
{
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    int n = dev < 64 ? sms[dev] : 0;
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        if (dev < 64) sms[dev] = n;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem) != cudaSuccess || per_sm <= 0) {
        cudaGetLastError();
        per_sm = 1;
    }
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)n * per_sm, max_parts));
}

} // namespace
} // namespace gs

using namespace gs;

extern "C" size_t gs_bin_sort_workspace_bytes(const gs_camera *cams, int32_t ncam, int32_t P,
                                              const gs_config *cfg, int64_t capacity)
{
    if (!cams || !cfg || ncam <= 0 || ncam > kMaxCams || P < 0 || capacity < 0) return 0;
    const int64_t N = (int64_t)ncam * P;
    if (N >= (int64_t)kValMask || capacity >= (int64_t)kValMask) return 0;
    CamTable t;
    BinPlan bp;
    if (!build_cam_table(cams, ncam, cfg, &t) || !make_bin_plan(t, cfg, P, &bp)) return 0;
    return ws_layout(bp, N, capacity, t.total_tiles).total;
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
    BinPlan bp;
    if (!build_cam_table(cams, ncam, cfg, &t) || !make_bin_plan(t, cfg, P, &bp)) return GS_ERR_ARG;
    const WsLayout L = ws_layout(bp, N, capacity, t.total_tiles);
    if (workspace_bytes < L.total) return GS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(d_workspace);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws + L.hdr);
    auto U = [&](size_t off) { return reinterpret_cast<uint32_t *>(ws + off); };
    auto U2 = [&](size_t off) { return reinterpret_cast<uint2 *>(ws + off); };
    auto U4 = [&](size_t off) { return reinterpret_cast<uint4 *>(ws + off); };
    uint2 *ranges = reinterpret_cast<uint2 *>(d_ranges);
    const uint32_t T = (uint32_t)t.total_tiles;
    const uint32_t cap = (uint32_t)capacity;

    if (cudaMemsetAsync(ws, 0, L.zero_end, s) != cudaSuccess) return GS_ERR_CUDA;
    if (N == 0) {
        if (cudaMemsetAsync(d_ranges, 0, sizeof(uint2) * (size_t)T, s) != cudaSuccess) return GS_ERR_CUDA;
    } else {
        static bool optin_rows[2][64] = {}, optin_rows_t[2][64] = {}, optin_cc[64] = {}, optin_cols[64] = {},
                    optin_cols_t[64] = {};
        Splat2DConst sp = splat2d_const(d_splat2d, N);
        const bool ell = cfg->rect_mode == GS_RECT_ELLIPSE;
        // 1. compaction, per-camera histograms and row differences
        compact_kernel<<<(unsigned)((N + kCompactTile - 1) / kCompactTile), 256, 0, s>>>(
            bp, sp.tiles, sp.dkey, sp.rect, (uint32_t)N, U(L.dk0), U(L.dv0), hdr, U(L.st_compact), U(L.hist),
            U(L.rowdiff), U(L.seg));
        count_launch();
        GS_LAUNCH_CHECK();
        // 2. plan
        plan_kernel<<<1, 1024, 0, s>>>(bp, hdr, U(L.seg), U4(L.rec_parts), L.max_rec_parts, U(L.rowdiff),
                                       U(L.rowbase), U4(L.span_parts), L.max_span_parts, U(L.rowq), cap, cap,
                                       ell ? 1 : 0);
        count_launch();
        GS_LAUNCH_CHECK();
        // 3. depth sort within each camera, 4 passes ping-pong: result back in (dk0, dv0)
        uint32_t *kin = U(L.dk0), *vin = U(L.dv0), *kout = U(L.dk1), *vout = U(L.dv1);
        for (int p = 0; p < 4; ++p) {
            // the last pass writes only the record indices: the splits read
            // nothing else, and 64-bit keys are gathered by index
            if (launch_onesweep<8>(L.max_rec_parts, s, kin, vin, p == 3 ? nullptr : kout, vout, U(L.seg),
                                   U4(L.rec_parts),
                                   &hdr->n_rec_parts, 8 * p, U(L.hist) + 256 * p, 1024,
                                   U(L.st_depth) + p * L.st_depth_stride, &hdr->ctr[CTR_DEPTH + p],
                                   &hdr->err) != cudaSuccess) {
                cudaGetLastError();
                return GS_ERR_CUDA;
            }
            std::swap(kin, kout);
            std::swap(vin, vout);
        }
        if (capacity > 0) {
            uint2 *spans = U2(L.spans);
            // the dynamic shared-memory opt-ins are caps on every later launch:
            // each is set once, to the largest table any camera can need
            const size_t smw_max = split_smem(kMaxDigits), smt_max = tsplit_smem(kThreadDigits);
            const bool rows_t = bp.max_ty <= kThreadDigits, cols_t = bp.max_tx <= kThreadDigits;
            cudaError_t e = cudaSuccess;
            // 4. row split
            const size_t sm_r = rows_t ? tsplit_smem(bp.max_ty) : split_smem(bp.max_ty);
            unsigned gr = 0;
            if (rows_t && ell) {
                e = smem_optin(rows_t_kernel<true>, smt_max, optin_rows_t[1]);
                gr = split_grid(rows_t_kernel<true>, sm_r, L.max_rec_parts);
            } else if (rows_t) {
                e = smem_optin(rows_t_kernel<false>, smt_max, optin_rows_t[0]);
                gr = split_grid(rows_t_kernel<false>, sm_r, L.max_rec_parts);
            } else if (ell) {
                e = smem_optin(rows_kernel<true>, smw_max, optin_rows[1]);
                gr = split_grid(rows_kernel<true>, sm_r, L.max_rec_parts);
            } else {
                e = smem_optin(rows_kernel<false>, smw_max, optin_rows[0]);
                gr = split_grid(rows_kernel<false>, sm_r, L.max_rec_parts);
            }
            if (e != cudaSuccess) {
                cudaGetLastError();
                return GS_ERR_CUDA;
            }
#define GS_ROWS_ARGS                                                                                           \
    bp, U(L.seg), U4(L.rec_parts), hdr, vin, sp.rect, sp.rec, (uint32_t)N, U(L.rowbase), spans, cap, U(L.st_rows), \
        &hdr->ctr[CTR_ROWS], &hdr->err
            if (rows_t && ell)
                rows_t_kernel<true><<<gr, 256, sm_r, s>>>(GS_ROWS_ARGS);
            else if (rows_t)
                rows_t_kernel<false><<<gr, 256, sm_r, s>>>(GS_ROWS_ARGS);
            else if (ell)
                rows_kernel<true><<<gr, 256, sm_r, s>>>(GS_ROWS_ARGS);
            else
                rows_kernel<false><<<gr, 256, sm_r, s>>>(GS_ROWS_ARGS);
#undef GS_ROWS_ARGS
            count_launch();
            GS_LAUNCH_CHECK();
            // 5. tile counts, 6. tile ranges, 7. column split into the tiles' lists
            const bool use_colmat = cols_t; // column offsets from the count matrix, no look-back
            const size_t sm_cc = split_smem(bp.max_tx);
            const size_t sm_c = cols_t ? tsplit_smem(bp.max_tx) : sm_cc;
            if (smem_optin(cols_count_kernel, smw_max, optin_cc) != cudaSuccess ||
                (cols_t ? smem_optin(cols_t_kernel, smt_max, optin_cols_t)
                        : smem_optin(cols_kernel, smw_max, optin_cols)) != cudaSuccess) {
                cudaGetLastError();
                return GS_ERR_CUDA;
            }
            cols_count_kernel<<<split_grid(cols_count_kernel, sm_cc, L.max_span_parts), 256, sm_cc, s>>>(
                bp, U4(L.span_parts), hdr, U(L.rowbase), spans, cap, U(L.tile_cnt), use_colmat ? U(L.colmat) : nullptr,
                &hdr->ctr[CTR_COUNT_COLS]);
            count_launch();
            GS_LAUNCH_CHECK();
            if (use_colmat) {
                col_offsets_kernel<<<bp.G, 128, 0, s>>>(bp, U(L.rowq), U(L.colmat), U(L.tile_cnt));
                count_launch();
                GS_LAUNCH_CHECK();
            }
            tile_scan_kernel<<<(T + kScanTile - 1) / kScanTile, 256, 0, s>>>(U(L.tile_cnt), T, ranges, cap, hdr,
                                                                            U(L.st_scan));
            count_launch();
            GS_LAUNCH_CHECK();
            if (cols_t)
                cols_t_kernel<<<split_grid(cols_t_kernel, sm_c, L.max_span_parts), 256, sm_c, s>>>(
                    bp, U4(L.span_parts), hdr, U(L.rowbase), spans, cap, U(L.colmat), ranges, d_vals, cap,
                    U(L.st_cols), &hdr->ctr[CTR_COLS], &hdr->err);
            else
                cols_kernel<<<split_grid(cols_kernel, sm_c, L.max_span_parts), 256, sm_c, s>>>(
                    bp, U4(L.span_parts), hdr, U(L.rowbase), spans, cap, ranges, d_vals, cap, U(L.st_cols),
                    &hdr->ctr[CTR_COLS], &hdr->err);
            count_launch();
            GS_LAUNCH_CHECK();
            if (d_keys64) {
                const unsigned gk = (unsigned)std::min<int64_t>((T + 7) / 8, 148 * 16);
                keys64_kernel<<<gk ? gk : 1, 256, 0, s>>>(ranges, T, d_vals, sp.dkey, (uint32_t)N,
                                                         reinterpret_cast<unsigned long long *>(d_keys64));
                count_launch();
                GS_LAUNCH_CHECK();
            }
        } else {
            if (cudaMemsetAsync(d_ranges, 0, sizeof(uint2) * (size_t)T, s) != cudaSuccess) return GS_ERR_CUDA;
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

extern "C" gs_status gs_workspace_status_async(void *stream, void *d_workspace, uint32_t *dst)
{
    if (!d_workspace || !dst) return GS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(d_workspace);
    if (cudaMemcpyAsync(dst, &hdr->err, sizeof(uint32_t), cudaMemcpyDefault, s) != cudaSuccess)
        return GS_ERR_CUDA;
    if (cudaMemsetAsync(&hdr->err, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    return GS_OK;
}

// Self-test of the bounded waits (fault injection without a fault): the two
// look-back routines above run against a predecessor that never publishes
// (all-zero flags in d_scratch). They must give up after `limit` sleeps,
// raise GS_ERR_TIMEOUT in the error word and return, leaving the context
// usable.
namespace gs {
namespace {
__global__ void lookback_selftest_kernel(int which, uint32_t *state, uint32_t *err, int limit)
{
    if (which == 0) {
        if (threadIdx.x < 32) (void)lookback_scalar(state, 1u, 5u, err, limit);
    } else {
        (void)lookback_digit<kLookWindow>(state, 1u, 256, (int)threadIdx.x, err, limit);
    }
}
} // namespace
} // namespace gs

extern "C" gs_status gs_selftest_lookback_timeout(void *stream, int32_t which, uint32_t *d_scratch,
                                                  int32_t spin_limit)
{
    if (!d_scratch || which < 0 || which > 2 || spin_limit < 1 || spin_limit > kSpinLimit) return GS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // d_scratch: [0] error word, [64, 64 + 512) look-back flags of partitions 0 and 1
    if (cudaMemsetAsync(d_scratch, 0, GS_SELFTEST_SCRATCH_BYTES, s) != cudaSuccess) return GS_ERR_CUDA;
    if (which == 2) {
        // the tcgen05 blend's mbarrier wait (render_tc5.cu)
        if (launch_tc5_wait_selftest(s, d_scratch, spin_limit) != cudaSuccess) {
            cudaGetLastError();
            return GS_ERR_CUDA;
        }
        count_launch();
        return GS_OK;
    }
    lookback_selftest_kernel<<<1, which == 0 ? 32 : 256, 0, s>>>(which, d_scratch + 64, d_scratch, spin_limit);
    count_launch();
    if (cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

// ---- spatial order of a scene (one-time preparation) ---------------------
// Bounding box of the finite means (order-preserving integer images of the
// floats, so that atomicMin / atomicMax compare them), 30-bit Morton codes
// with the four 8-bit digit histograms, then four Onesweep passes of
// (code, index): a stable sort, ties in index order.
namespace gs {
namespace {

struct OrderWs {
    size_t hdr, box, seg, hist, st, k0, k1, v1, total;
    uint32_t parts;
    size_t st_stride;
};

OrderWs order_layout(int64_t P)
{
    OrderWs L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += align256(bytes); return r; };
    L.parts = (uint32_t)((P + kSortTile - 1) / kSortTile);
    L.st_stride = (size_t)256 * (L.parts + 1);
    L.hdr = take(sizeof(WsHeader));
    L.box = take(sizeof(uint32_t) * 6);
    L.seg = take(sizeof(uint32_t) * 2);
    L.hist = take(sizeof(uint32_t) * 4 * 256);
    L.st = take(sizeof(uint32_t) * 4 * L.st_stride);
    L.k0 = take(sizeof(uint32_t) * P + 16);
    L.k1 = take(sizeof(uint32_t) * P + 16);
    L.v1 = take(sizeof(uint32_t) * P + 16);
    L.total = o;
    return L;
}

__device__ __forceinline__ uint32_t ford(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float funord(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// box[0..2] = images of the minima (start at all ones), box[3..5] = of the
// maxima (start at zero); also writes the sorts' one segment, [0, P).
__global__ void __launch_bounds__(256) bbox_kernel(const float *__restrict__ means, int P, uint32_t *box,
                                                   uint32_t *seg)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        seg[0] = 0;
        seg[1] = (uint32_t)P;
    }
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float v = means[3 * (size_t)i + k];
            if (isfinite(v)) {
                lo[k] = fminf(lo[k], v);
                hi[k] = fmaxf(hi[k], v);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint32_t a = ford(lo[k]), b = ford(hi[k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = min(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&box[k], a);
            atomicMax(&box[3 + k], b);
        }
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t x)
{
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void __launch_bounds__(256) morton_kernel(const float *__restrict__ means, int P,
                                                     const uint32_t *box, uint32_t *__restrict__ keys,
                                                     uint32_t *__restrict__ vals, uint32_t *hist)
{
    __shared__ uint32_t s_h[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += 256) (&s_h[0][0])[i] = 0;
    __syncthreads();
    float lo[3], sc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = funord(box[k]);
        const float ext = funord(box[3 + k]) - lo[k];
        // no finite mean (ext = -inf) or a flat box: every code is 0 on that axis
        sc[k] = (ext > 0.f && isfinite(ext)) ? 1023.f / ext : 0.f;
        if (!isfinite(lo[k])) lo[k] = 0.f;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        uint32_t code = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            // fmaxf / fminf drop a NaN operand: a non-finite coordinate maps to 0 or 1023
            const float q = fminf(fmaxf((means[3 * (size_t)i + k] - lo[k]) * sc[k], 0.f), 1023.f);
            code |= spread10((uint32_t)q) << k;
        }
        keys[i] = code;
        vals[i] = (uint32_t)i;
#pragma unroll
        for (int p = 0; p < 4; ++p) atomicAdd(&s_h[p][(code >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * 256; i += 256) {
        const uint32_t v = (&s_h[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

__global__ void __launch_bounds__(256) gather_rows_kernel(int64_t total, int words,
                                                          const uint32_t *__restrict__ src,
                                                          const uint32_t *__restrict__ perm, int n,
                                                          uint32_t *__restrict__ dst)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / words, w = e - k * words;
        const uint32_t p = perm[k];
        dst[e] = p < (uint32_t)n ? src[(int64_t)p * words + w] : 0u;
    }
}

} // namespace
} // namespace gs

extern "C" size_t gs_spatial_order_workspace_bytes(int32_t P)
{
    if (P < 0 || P >= (int32_t)kValMask) return 0;
    return order_layout(P).total;
}

extern "C" gs_status gs_spatial_order(void *stream, int32_t P, const float *d_means, void *d_workspace,
                                      uint32_t *d_perm)
{
    if (P < 0 || P >= (int32_t)kValMask) return GS_ERR_ARG;
    if (P == 0) return GS_OK;
    if (!d_means || !d_workspace || !d_perm || ((uintptr_t)d_workspace & 255) || ((uintptr_t)d_means & 3) ||
        ((uintptr_t)d_perm & 3))
        return GS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const OrderWs L = order_layout(P);
    char *ws = static_cast<char *>(d_workspace);
    auto U = [&](size_t off) { return reinterpret_cast<uint32_t *>(ws + off); };
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws + L.hdr);
    // zero the header, histograms and look-back states; the box's minima start at all ones
    if (cudaMemsetAsync(ws, 0, L.k0, s) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemsetAsync(U(L.box), 0xff, sizeof(uint32_t) * 3, s) != cudaSuccess) return GS_ERR_CUDA;
    const unsigned blocks = (unsigned)std::min<int64_t>((P + 255) / 256, 148 * 8);
    bbox_kernel<<<blocks, 256, 0, s>>>(d_means, P, U(L.box), U(L.seg));
    count_launch();
    GS_LAUNCH_CHECK();
    // (code, index) into (k0, d_perm); the passes ping-pong back into them
    morton_kernel<<<blocks, 256, 0, s>>>(d_means, P, U(L.box), U(L.k0), d_perm, U(L.hist));
    count_launch();
    GS_LAUNCH_CHECK();
    uint32_t *kin = U(L.k0), *vin = d_perm, *kout = U(L.k1), *vout = U(L.v1);
    for (int p = 0; p < 4; ++p) {
        if (launch_onesweep<8>(L.parts, s, kin, vin, kout, vout, U(L.seg), nullptr, nullptr, 8 * p,
                               U(L.hist) + 256 * p, 0, U(L.st) + p * L.st_stride, &hdr->ctr[p],
                               &hdr->err) != cudaSuccess) {
            cudaGetLastError();
            return GS_ERR_CUDA;
        }
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    return GS_OK;
}

extern "C" gs_status gs_gather_rows(void *stream, int32_t n, int32_t row_bytes, const void *d_src,
                                    const uint32_t *d_perm, void *d_dst)
{
    if (n < 0 || row_bytes <= 0 || (row_bytes & 3)) return GS_ERR_ARG;
    if (n == 0) return GS_OK;
    if (!d_src || !d_perm || !d_dst || ((uintptr_t)d_src & 3) || ((uintptr_t)d_dst & 3) ||
        ((uintptr_t)d_perm & 3))
        return GS_ERR_ARG;
    const int words = row_bytes / 4;
    const int64_t total = (int64_t)n * words;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 148 * 16);
    gather_rows_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(total, words, static_cast<const uint32_t *>(d_src),
                                                           d_perm, n, static_cast<uint32_t *>(d_dst));
    count_launch();
    GS_LAUNCH_CHECK();
    return GS_OK;
}
