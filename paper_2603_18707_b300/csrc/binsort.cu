// binsort.cu — depth-ordered tile binning (sm_103a).
//
// Result: per global tile, the records whose support rectangle covers it,
// in increasing (depth, record index) order. That is the order a stable sort
// of 3DGS's 64-bit keys (tile << 32 | depth bits) over records emitted in
// index order gives. It is produced here without ever materialising 64-bit
// keys:
//   1. compact   drawn records (tiles > 0) -> (depth bits, record index),
//                in index order (single-pass scan with decoupled look-back);
//                also histograms the four depth digits
//   2. sort      stable LSD radix sort of those by depth: 4 Onesweep passes
//   3. emit      walk the depth-sorted records, scan their tile counts and
//                write one (tile id, record index) pair per covered tile;
//                warp-cooperative so that every store is coalesced; also
//                histograms the tile-id digits
//   4. sort      stable LSD radix sort of the pairs by tile id: 1 pass of 8
//                bits, 2 of 8, 2 of 9 or 3 of 8-9 bits, whatever covers the
//                tile ids
//   5. ranges    first / one-past-last position of every tile id
// The depth digits are sorted once per record instead of once per overlap,
// which moves far fewer bytes than sorting the 64-bit keys directly.
//
// Onesweep (one kernel per digit): each CTA claims the next partition of 5120
// keys from an atomic counter, ranks its keys per digit with warp
// match/ballot, publishes per-digit counts and resolves its global offsets by
// decoupled look-back over earlier partitions (kLookWindow predecessors per
// load round), then scatters through shared memory so that global stores are
// contiguous per digit. Every spin-wait is bounded: on expiry it raises
// GS_ERR_TIMEOUT in the workspace error word and carries on with what it has.
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
#ifndef GS_EMIT_MIN_BLOCKS
// 0: no register cap from the occupancy target. 8 (32 registers, some
// spills to L1) measured fastest: the emission waits on memory, and 8 CTAs
// per SM hide more of it than 4 (64 registers, no spills) or 6.
#define GS_EMIT_MIN_BLOCKS 8
#endif
#if GS_EMIT_MIN_BLOCKS
#define GS_EMIT_BOUNDS __launch_bounds__(256, GS_EMIT_MIN_BLOCKS)
#else
#define GS_EMIT_BOUNDS __launch_bounds__(256)
#endif
#ifndef GS_EMIT_RUNS
#define GS_EMIT_RUNS 1 // tile-digit histogram adds of the higher digits per run of equal digits
#endif
#ifndef GS_EMIT_ITEMS
#define GS_EMIT_ITEMS 8
#endif
constexpr int kSortThreads = 256;
constexpr int kSortItems = GS_SORT_ITEMS;
constexpr int kSortTile = kSortThreads * kSortItems; // keys per partition
#ifndef GS_COMPACT_VEC
#define GS_COMPACT_VEC 8
#endif
constexpr int kCompactVec = GS_COMPACT_VEC;          // uint4 loads per lane
constexpr int kCompactTile = 256 * 4 * kCompactVec;  // records per partition
constexpr int kEmitItems = GS_EMIT_ITEMS;
constexpr int kEmitTile = 256 * kEmitItems;          // records per partition
constexpr int kHistSlot = 512;                       // histogram entries per pass
constexpr int kLookWindow = GS_LOOK_WINDOW;

enum Counter {
    CTR_COMPACT = 0,
    CTR_DEPTH = 1, // 4 passes
    CTR_EMIT = 5,
    CTR_TILE = 6,  // up to 3 passes
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

// Digit plan of the tile-id sort.
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

struct TilePlan {
    int passes;
    int bits[3];
    int shift[3];
};

TilePlan tile_plan(int64_t total_tiles)
{
    // as few passes as 9-bit digits allow, and within them as many 8-bit
    // digits as possible (an 8-bit pass is ~25% cheaper per key); the widest
    // digit first (the look-back state is sized by it). Up to 27 bits
    // (< 2^30 tiles is checked by the caller).
    int b = 1;
    while (((int64_t)1 << b) < total_tiles) ++b;
    TilePlan p{};
    p.passes = std::max(1, (b + 8) / 9);
    const int nine = std::max(0, b - 8 * p.passes);
    int s = 0;
    for (int i = 0; i < p.passes; ++i) {
        p.bits[i] = i < nine ? 9 : 8;
        p.shift[i] = s;
        s += p.bits[i];
    }
    return p;
}

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

// Decoupled look-back of one digit of a Onesweep pass (one thread per
// digit): sums the published counts of this digit in the partitions before
// `part` (kLookWindow per load round) until one with an inclusive prefix.
// A predecessor that has published nothing is re-read after a short sleep,
// at most `limit` times; then GS_ERR_TIMEOUT is raised and what was summed
// is returned.
__device__ uint32_t lookback_digit(const uint32_t *state, uint32_t part, int R, int d, uint32_t *err,
                                   int limit)
{
    uint32_t excl = 0;
    int64_t p = (int64_t)part - 1;
    int spins = 0;
    bool done = false;
    while (!done && p >= 0) {
        uint32_t s[kLookWindow];
#pragma unroll
        for (int w = 0; w < kLookWindow; ++w)
            s[w] = (p - w >= 0) ? ld_relaxed(&state[(size_t)(p - w) * R + d]) : kFlagIncl;
        int used = 0;
        bool stall = false;
#pragma unroll
        for (int w = 0; w < kLookWindow; ++w) {
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

// Block-wide exclusive scan of one value per thread (blockDim.x == 256).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t x = warp_incl_scan(v);
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

// 1. compaction of drawn records, index order preserved, plus the histograms
// of the four depth digits. Lane l of warp w holds records
// base + (kCompactTile / 8) w + 4 (32 j + l) + e, e < 4, j < kCompactVec
// (uint4 loads).
__global__ void __launch_bounds__(256)
compact_kernel(const uint32_t *__restrict__ tiles, const uint32_t *__restrict__ dkey, uint32_t N,
               uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, WsHeader *hdr,
               uint32_t *state, uint32_t *__restrict__ hist)
{
    __shared__ uint32_t s_part, s_excl, s_warp[8];
    __shared__ uint32_t s_h[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += 256) (&s_h[0][0])[i] = 0;
    if (threadIdx.x == 0) s_part = atomicAdd(&hdr->ctr[CTR_COMPACT], 1u);
    __syncthreads();
    const uint32_t part = s_part;
    const uint32_t nparts = (N + kCompactTile - 1) / kCompactTile;
    if (part >= nparts) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t wbase = part * kCompactTile + warp * (kCompactTile / 8);
    uint32_t flags[kCompactVec], incl[kCompactVec], off[kCompactVec];
    uint32_t running = 0;
#pragma unroll
    for (int j = 0; j < kCompactVec; ++j) {
        const uint32_t e0 = wbase + 4 * (32 * j + lane);
        uint32_t f = 0;
        if (e0 + 3 < N) {
            const uint4 t4 = reinterpret_cast<const uint4 *>(tiles)[e0 / 4];
            f = (t4.x > 0) | (t4.y > 0) << 1 | (t4.z > 0) << 2 | (t4.w > 0) << 3;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (e0 + e < N && tiles[e0 + e] > 0) f |= 1u << e;
        }
        flags[j] = f;
        const uint32_t x = warp_incl_scan(__popc(f));
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
    const uint32_t excl = s_excl;
#pragma unroll
    for (int j = 0; j < kCompactVec; ++j) {
        uint32_t pos = excl + warp_excl + off[j] + incl[j] - __popc(flags[j]);
        const uint32_t e0 = wbase + 4 * (32 * j + lane);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (flags[j] >> e & 1u) {
                const uint32_t key = dkey[e0 + e];
                if (pos < N) { // always true unless a look-back wait timed out
                    keys_out[pos] = key;
                    vals_out[pos] = e0 + e;
                }
                ++pos;
#pragma unroll
                for (int p = 0; p < 4; ++p) atomicAdd(&s_h[p][(key >> (8 * p)) & 255u], 1u);
            }
        }
    }
    if (part == nparts - 1 && threadIdx.x == 0) hdr->n_vis = sat_add(excl, total);
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * 256; i += 256) {
        const uint32_t v = (&s_h[0][0])[i];
        if (v) atomicAdd(&hist[(i >> 8) * kHistSlot + (i & 255)], v);
    }
}

// One Onesweep pass over BITS bits starting at `shift`. Dynamic shared
// memory: keys, values, per-warp digit counters, two per-digit tables.
template <int BITS>
constexpr size_t onesweep_smem()
{
    return sizeof(uint32_t) * (2 * kSortTile + 8 * (1 << BITS) + 2 * (1 << BITS) + 8 + 1);
}

template <int BITS>
__global__ void __launch_bounds__(kSortThreads, GS_SORT_MIN_BLOCKS) // the pass is latency-bound
onesweep_kernel(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                const uint32_t *n_ptr, int shift, const uint32_t *__restrict__ hist,
                uint32_t *state, uint32_t *ctr, uint32_t *err)
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
    const uint32_t n = *n_ptr;
    const uint32_t part = *s_part;
    const uint32_t nparts = (n + kSortTile - 1) / kSortTile;
    if (part >= nparts) return;

    // warp-striped load: warp w owns keys [base + 32 I w, base + 32 I (w + 1)), I = kSortItems
    const uint32_t wbase = part * kSortTile + warp * (32 * kSortItems);
    uint32_t k[kSortItems], v[kSortItems], r[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t idx = wbase + j * 32 + lane;
        const bool ok = idx < n;
        k[j] = ok ? keys_in[idx] : 0xffffffffu; // invalid keys rank last (top digit, highest index)
        v[j] = ok ? vals_in[idx] : 0u;
    }
    // this thread's digits' global counts, loaded now so that the latency
    // overlaps the ranking
    uint32_t hv[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) hv[q] = hist[tid * DPT + q];
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
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const uint32_t x = s_whist[w * R + d];
            s_whist[w * R + d] = c;
            c += x;
        }
        cnt[q] = c;
        csum += c;
        hsum += hv[q];
    }
    uint32_t tot;
    uint32_t bex = block_excl_scan(csum, s_warp, tot);
    __syncthreads();
    uint32_t hex = block_excl_scan(hsum, s_warp, tot);
    // invalid keys exist only in the last partition, all with the top digit
    const uint32_t last_valid = n - part * kSortTile;
    const uint32_t n_invalid = last_valid < (uint32_t)kSortTile ? kSortTile - last_valid : 0u;
    uint32_t *st = state + (size_t)part * R;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = tid * DPT + q;
        s_bexcl[d] = bex;
        bex += cnt[q];
        const uint32_t agg = cnt[q] - (d == (int)M ? n_invalid : 0u);
        uint32_t excl = 0;
        if (part == 0) {
            st_relaxed(&st[d], kFlagIncl | agg);
        } else {
            st_relaxed(&st[d], kFlagAgg | agg);
            excl = lookback_digit(state, part, R, d, err, kSpinLimit);
            st_relaxed(&st[d], kFlagIncl | sat_add(excl, agg));
        }
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
    const uint32_t nvalid = min(last_valid, (uint32_t)kSortTile);
    for (uint32_t i = tid; i < nvalid; i += kSortThreads) {
        const uint32_t key = s_keys[i];
        const uint32_t d = (key >> shift) & M;
        const uint32_t o = s_goff[d] + i - s_bexcl[d];
        if (o < n) { // always true unless a look-back wait timed out
            keys_out[o] = key;
            vals_out[o] = s_vals[i];
        }
    }
}

// 3. overlap emission in depth order, plus the tile-digit histograms. ELL:
// only the tiles of each rectangle row that the support ellipse reaches
// (GS_RECT_ELLIPSE), else the whole rectangle.
template <bool ELL>
__global__ void GS_EMIT_BOUNDS
emit_kernel(const __grid_constant__ CamTable cams, FastDiv pdiv, uint32_t n_records,
            const uint32_t *__restrict__ sorted_vals,
            const uint32_t *__restrict__ tiles, const ushort4 *__restrict__ rects,
            const float4 *__restrict__ rec, int tile_w, int tile_h,
            uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, uint32_t capacity,
            WsHeader *hdr, uint32_t *state, TilePlan plan, uint32_t *__restrict__ hist)
{
    __shared__ uint32_t s_part, s_excl, s_warp[8];
    __shared__ uint32_t s_h[3][kHistSlot];
    __shared__ uint32_t s_tb[kMaxCams], s_tx[kMaxCams]; // per camera: first tile id, tiles per row
    for (int i = threadIdx.x; i < 3 * kHistSlot; i += 256) (&s_h[0][0])[i] = 0;
    if (threadIdx.x < cams.ncam) {
        s_tb[threadIdx.x] = (uint32_t)cams.cam[threadIdx.x].tile_base;
        s_tx[threadIdx.x] = (uint32_t)cams.cam[threadIdx.x].tiles_x;
    }
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
        rc[j] = valid ? rects[vv] : make_ushort4(0, 0, 0, 0);
        // a drawn record's rectangle holds exactly its tiles unless rows are
        // cut to the ellipse: one gather per record instead of two
        if (ELL)
            cnt[j] = valid ? tiles[vv] : 0u;
        else
            cnt[j] = valid ? ((uint32_t)rc[j].z - rc[j].x + 1u) * ((uint32_t)rc[j].w - rc[j].y + 1u) : 0u;
        const uint32_t x = warp_incl_scan(cnt[j]);
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
    if (ELL) {
        // two levels: the warp expands its records into tile rows (32 rows at
        // a time), each lane finds its row's tile columns, then the warp
        // writes those rows' tiles 32 at a time
#pragma unroll 1
        for (int j = 0; j < kEmitItems; ++j) {
            const uint32_t rows = cnt[j] ? (uint32_t)(rc[j].w - rc[j].y + 1) : 0u;
            const uint32_t r_incl = warp_incl_scan(rows);
            const uint32_t r_total = __shfl_sync(0xffffffffu, r_incl, 31);
            const uint32_t out_base = part_excl + warp_excl + off[j];
            uint32_t emitted = 0;
            for (uint32_t rb = 0; rb < r_total; rb += 32) {
                const uint32_t r = rb + lane;
                const uint32_t rq = min(r, r_total - 1u);
                int e = 0;
#pragma unroll
                for (int sft = 16; sft > 0; sft >>= 1) {
                    const uint32_t c = __shfl_sync(0xffffffffu, r_incl, e + sft - 1);
                    if (c <= rq) e += sft;
                }
                const uint32_t ev = __shfl_sync(0xffffffffu, v[j], e);
                const uint32_t rexcl = __shfl_sync(0xffffffffu, r_incl - rows, e);
                uint32_t cnt2 = 0, kb = 0;
                if (r < r_total) {
                    const float4 g0 = rec[3 * (size_t)ev], g1 = rec[3 * (size_t)ev + 1];
                    const ushort4 rr = rects[ev];
                    const CamDev &cm = cams.cam[pdiv.div(ev)];
                    const int ty = (int)rr.y + (int)(rq - rexcl);
                    int c0 = rr.x, c1 = rr.z;
                    // a single-row or single-column rectangle keeps all its tiles
                    const bool simple = rr.z == rr.x || rr.w == rr.y;
                    if (simple || row_cols(g0.x, g0.y, g1.x, g1.y, g1.z, g1.w, ty, tile_w, tile_h, cm.W,
                                           cm.H, rr.x, rr.z, c0, c1)) {
                        cnt2 = (uint32_t)(c1 - c0 + 1);
                        kb = (uint32_t)cm.tile_base + (uint32_t)ty * cm.tiles_x + (uint32_t)c0;
                    }
                }
                const uint32_t c_incl = warp_incl_scan(cnt2);
                const uint32_t seg = __shfl_sync(0xffffffffu, c_incl, 31);
                for (uint32_t b2 = 0; b2 < seg; b2 += 32) {
                    const uint32_t p = b2 + lane;
                    const uint32_t pq = min(p, seg - 1u);
                    int f = 0;
#pragma unroll
                    for (int sft = 16; sft > 0; sft >>= 1) {
                        const uint32_t c = __shfl_sync(0xffffffffu, c_incl, f + sft - 1);
                        if (c <= pq) f += sft;
                    }
                    const uint32_t fkb = __shfl_sync(0xffffffffu, kb, f);
                    const uint32_t fbeg = __shfl_sync(0xffffffffu, c_incl - cnt2, f);
                    const uint32_t fv = __shfl_sync(0xffffffffu, ev, f);
                    const uint32_t o = out_base + emitted + p;
                    if (p < seg && o < capacity) {
                        const uint32_t key = fkb + (pq - fbeg);
                        keys_out[o] = key;
                        vals_out[o] = fv;
                        for (int q = 0; q < plan.passes; ++q)
                            atomicAdd(&s_h[q][(key >> plan.shift[q]) & ((1u << plan.bits[q]) - 1u)], 1u);
                    }
                }
                emitted += seg;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < (ELL ? 0 : kEmitItems); ++j) {
        const uint32_t w_incl = incl[j];
        const uint32_t w_total = __shfl_sync(0xffffffffu, w_incl, 31);
        const uint32_t out_base = part_excl + warp_excl + off[j];
        const uint32_t cam = pdiv.div(v[j]);
        const uint32_t tiles_x = s_tx[cam];
        const uint32_t tbase = s_tb[cam] + (uint32_t)rc[j].y * tiles_x + rc[j].x;
        const uint32_t rw = (uint32_t)rc[j].z - rc[j].x + 1u;
        const float rrw = 1.f / (float)rw;
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
            const uint32_t etx = __shfl_sync(0xffffffffu, tiles_x, e);
            const float errw = __shfl_sync(0xffffffffu, rrw, e);
            const uint32_t l = pq - ebeg;
            // l / erw from the reciprocal (l < 2^22: off by at most one), corrected
            uint32_t row = (uint32_t)((float)l * errw);
            row -= (row * erw > l) ? 1u : 0u;
            row += ((row + 1u) * erw <= l) ? 1u : 0u;
            const uint32_t col = l - row * erw;
            const uint32_t o = out_base + p;
            const bool act = p < w_total && o < capacity; // a prefix of the warp's lanes
            const uint32_t key = etb + row * etx + col;
            if (act) {
                keys_out[o] = key;
                vals_out[o] = ev;
                atomicAdd(&s_h[0][(key >> plan.shift[0]) & ((1u << plan.bits[0]) - 1u)], 1u);
            }
#if GS_EMIT_RUNS
            // higher digits: consecutive lanes mostly hold consecutive tile
            // ids with one digit; one atomic per run of equal digits
            const uint32_t nact = __popc(__ballot_sync(0xffffffffu, act));
            for (int q = 1; q < plan.passes; ++q) {
                const uint32_t d = (key >> plan.shift[q]) & ((1u << plan.bits[q]) - 1u);
                const uint32_t dp = __shfl_up_sync(0xffffffffu, d, 1);
                const bool head = act && (lane == 0 || dp != d);
                const uint32_t heads = __ballot_sync(0xffffffffu, head);
                if (head) {
                    const uint32_t after = heads & (0xfffffffeu << lane);
                    const uint32_t next = after ? (uint32_t)(__ffs(after) - 1) : 32u;
                    atomicAdd(&s_h[q][d], min(next, nact) - (uint32_t)lane);
                }
            }
#else
            if (act)
                for (int q = 1; q < plan.passes; ++q)
                    atomicAdd(&s_h[q][(key >> plan.shift[q]) & ((1u << plan.bits[q]) - 1u)], 1u);
#endif
        }
    }
    if (part == nparts - 1 && threadIdx.x == 0) {
        const uint32_t tot = sat_add(part_excl, total);
        hdr->n_over_raw = tot;
        hdr->n_over = min(tot, capacity);
        if (tot > capacity || tot >= kValMask) atomicOr(&hdr->err, (uint32_t)GS_ERR_CAPACITY);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < plan.passes * kHistSlot; i += 256) {
        const uint32_t x = (&s_h[0][0])[i];
        if (x) atomicAdd(&hist[i], x);
    }
}

// 5. per-tile [start, end) and optional 64-bit keys. Each thread takes four
// consecutive sorted keys (one 16-byte load); the neighbours across thread
// boundaries come from the adjacent lanes, or from memory at warp edges.
__global__ void __launch_bounds__(256)
ranges_kernel(const uint32_t *__restrict__ tkeys, const uint32_t *__restrict__ vals,
              const uint32_t *__restrict__ dkey, const WsHeader *hdr, uint2 *__restrict__ ranges,
              unsigned long long *__restrict__ keys64, uint32_t total_tiles, uint32_t n_records)
{
    const uint32_t n = hdr->n_over;
    const uint32_t nq = (n + 3) / 4;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * 256;
    // every lane of a warp runs the same number of rounds (full-mask shuffles)
    for (uint32_t q0 = blockIdx.x * 256 + (threadIdx.x & ~31u); q0 < nq; q0 += stride) {
        const uint32_t q = q0 + lane;
        const uint32_t i0 = 4 * q;
        uint32_t k[4];
        if (i0 + 3 < n) {
            const uint4 t = *reinterpret_cast<const uint4 *>(tkeys + i0);
            k[0] = t.x, k[1] = t.y, k[2] = t.z, k[3] = t.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) k[e] = i0 + e < n ? tkeys[i0 + e] : 0xffffffffu;
        }
        uint32_t prev = __shfl_up_sync(0xffffffffu, k[3], 1);
        uint32_t next = __shfl_down_sync(0xffffffffu, k[0], 1);
        if (lane == 0) prev = (i0 > 0 && i0 - 1 < n) ? tkeys[i0 - 1] : 0xfffffffeu;
        if (lane == 31) next = i0 + 4 < n ? tkeys[i0 + 4] : 0xfffffffeu;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t i = i0 + e;
            const uint32_t t = k[e];
            if (i >= n || t >= total_tiles) continue; // t >= total_tiles only after a timed-out wait
            const uint32_t before = e == 0 ? prev : k[e - 1];
            const uint32_t after = e == 3 ? next : (i + 1 < n ? k[e + 1] : 0xfffffffeu);
            if (i == 0 || before != t) ranges[t].x = i;
            if (i + 1 == n || after != t) ranges[t].y = i + 1;
            if (keys64) {
                const uint32_t v = vals[i];
                keys64[i] = ((unsigned long long)t << 32) | (v < n_records ? dkey[v] : 0xffffffffu);
            }
        }
    }
}

struct WsLayout {
    size_t hdr, hist, st_compact, st_depth, st_emit, st_tile, zero_end;
    size_t dk0, dk1, dv0, dv1, tk0, tk1, tv1, total;
    uint32_t parts_depth, parts_tile;
    size_t st_depth_stride, st_tile_stride; // uint32 entries per pass
};

WsLayout ws_layout(int64_t N, int64_t cap, const TilePlan &plan)
{
    WsLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += align256(bytes); return r; };
    L.parts_depth = (uint32_t)((N + kSortTile - 1) / kSortTile);
    L.parts_tile = (uint32_t)((cap + kSortTile - 1) / kSortTile);
    const int rt = 1 << plan.bits[0];
    L.st_depth_stride = (size_t)256 * (L.parts_depth + 1);
    L.st_tile_stride = (size_t)rt * (L.parts_tile + 1);
    L.hdr = take(sizeof(WsHeader));
    L.hist = take(sizeof(uint32_t) * 8 * kHistSlot);
    L.st_compact = take(sizeof(uint32_t) * ((N + kCompactTile - 1) / kCompactTile + 1));
    L.st_depth = take(sizeof(uint32_t) * 4 * L.st_depth_stride);
    L.st_emit = take(sizeof(uint32_t) * ((N + kEmitTile - 1) / kEmitTile + 1));
    L.st_tile = take(sizeof(uint32_t) * plan.passes * L.st_tile_stride);
    L.zero_end = o;
    L.dk0 = take(sizeof(uint32_t) * N + 16);
    L.dk1 = take(sizeof(uint32_t) * N);
    L.dv0 = take(sizeof(uint32_t) * N);
    L.dv1 = take(sizeof(uint32_t) * N);
    L.tk0 = take(sizeof(uint32_t) * cap);
    L.tk1 = take(sizeof(uint32_t) * cap);
    L.tv1 = take(sizeof(uint32_t) * cap);
    L.total = o;
    return L;
}

template <int BITS>
cudaError_t launch_onesweep(unsigned grid, cudaStream_t s, const uint32_t *ki, const uint32_t *vi,
                            uint32_t *ko, uint32_t *vo, const uint32_t *n, int shift,
                            const uint32_t *hist, uint32_t *state, uint32_t *ctr, uint32_t *err)
{
    const size_t sm = onesweep_smem<BITS>();
    // the shared-memory opt-in is set once per device (so that later calls,
    // e.g. under stream capture, only launch)
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError();
    if (dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(onesweep_kernel<BITS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        if (dev < 64) attr_set[dev] = true;
    }
    onesweep_kernel<BITS><<<grid ? grid : 1, kSortThreads, sm, s>>>(ki, vi, ko, vo, n, shift, hist,
                                                                   state, ctr, err);
    count_launch();
    return cudaPeekAtLastError();
}

} // namespace
} // namespace gs

using namespace gs;

extern "C" size_t gs_bin_sort_workspace_bytes(int64_t n_records, int64_t capacity, int64_t total_tiles)
{
    if (n_records < 0 || capacity < 0 || total_tiles < 0) return 0;
    return ws_layout(n_records, capacity, tile_plan(total_tiles)).total;
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
    const TilePlan plan = tile_plan(t.total_tiles);
    const WsLayout L = ws_layout(N, capacity, plan);
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
        // 1. compaction + depth-digit histograms
        compact_kernel<<<(unsigned)((N + kCompactTile - 1) / kCompactTile), 256, 0, s>>>(
            sp.tiles, sp.dkey, (uint32_t)N, U(L.dk0), U(L.dv0), hdr, U(L.st_compact), hist);
        count_launch();
        GS_LAUNCH_CHECK();
        // 2. depth sort, 4 passes ping-pong: result back in (dk0, dv0)
        uint32_t *kin = U(L.dk0), *vin = U(L.dv0), *kout = U(L.dk1), *vout = U(L.dv1);
        for (int p = 0; p < 4; ++p) {
            if (launch_onesweep<8>(L.parts_depth, s, kin, vin, kout, vout, &hdr->n_vis, 8 * p,
                                   hist + kHistSlot * p, U(L.st_depth) + p * L.st_depth_stride,
                                   &hdr->ctr[CTR_DEPTH + p], &hdr->err) != cudaSuccess) {
                cudaGetLastError();
                return GS_ERR_CUDA;
            }
            std::swap(kin, kout);
            std::swap(vin, vout);
        }
        if (capacity > 0) {
            // 3. emission into the buffers that make the last tile pass land in d_vals
            uint32_t *ek = U(L.tk0);
            uint32_t *ev = (plan.passes % 2 == 0) ? d_vals : U(L.tv1);
            uint32_t *thist = hist + 4 * kHistSlot;
            const unsigned eblocks = (unsigned)((N + kEmitTile - 1) / kEmitTile);
            const FastDiv pdiv = FastDiv::make((uint32_t)std::max(P, 1));
            if (cfg->rect_mode == GS_RECT_ELLIPSE)
                emit_kernel<true><<<eblocks, 256, 0, s>>>(t, pdiv, (uint32_t)N, vin, sp.tiles, sp.rect, sp.rec,
                                                          cfg->tile_w, cfg->tile_h, ek, ev, (uint32_t)capacity,
                                                          hdr, U(L.st_emit), plan, thist);
            else
                emit_kernel<false><<<eblocks, 256, 0, s>>>(t, pdiv, (uint32_t)N, vin, sp.tiles, sp.rect, sp.rec,
                                                           cfg->tile_w, cfg->tile_h, ek, ev, (uint32_t)capacity,
                                                           hdr, U(L.st_emit), plan, thist);
            count_launch();
            GS_LAUNCH_CHECK();
            // 4. tile sort
            uint32_t *tki = ek, *tvi = ev, *tko = U(L.tk1), *tvo = (ev == d_vals) ? U(L.tv1) : d_vals;
            for (int p = 0; p < plan.passes; ++p) {
                cudaError_t e;
                if (plan.bits[p] == 9)
                    e = launch_onesweep<9>(L.parts_tile, s, tki, tvi, tko, tvo, &hdr->n_over,
                                           plan.shift[p], thist + kHistSlot * p,
                                           U(L.st_tile) + p * L.st_tile_stride,
                                           &hdr->ctr[CTR_TILE + p], &hdr->err);
                else
                    e = launch_onesweep<8>(L.parts_tile, s, tki, tvi, tko, tvo, &hdr->n_over,
                                           plan.shift[p], thist + kHistSlot * p,
                                           U(L.st_tile) + p * L.st_tile_stride,
                                           &hdr->ctr[CTR_TILE + p], &hdr->err);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    return GS_ERR_CUDA;
                }
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
        (void)lookback_digit(state, 1u, 256, (int)threadIdx.x, err, limit);
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
    size_t hdr, box, hist, st, k0, k1, v1, total;
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
    L.hist = take(sizeof(uint32_t) * 4 * kHistSlot);
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
// maxima (start at zero); also publishes the element count for the sorts.
__global__ void __launch_bounds__(256) bbox_kernel(const float *__restrict__ means, int P, uint32_t *box,
                                                   WsHeader *hdr)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) hdr->n_vis = (uint32_t)P;
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
        if (v) atomicAdd(&hist[(i >> 8) * kHistSlot + (i & 255)], v);
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
    bbox_kernel<<<blocks, 256, 0, s>>>(d_means, P, U(L.box), hdr);
    count_launch();
    GS_LAUNCH_CHECK();
    // (code, index) into (k0, d_perm); the passes ping-pong back into them
    morton_kernel<<<blocks, 256, 0, s>>>(d_means, P, U(L.box), U(L.k0), d_perm, U(L.hist));
    count_launch();
    GS_LAUNCH_CHECK();
    uint32_t *kin = U(L.k0), *vin = d_perm, *kout = U(L.k1), *vout = U(L.v1);
    for (int p = 0; p < 4; ++p) {
        if (launch_onesweep<8>(L.parts, s, kin, vin, kout, vout, &hdr->n_vis, 8 * p, U(L.hist) + kHistSlot * p,
                               U(L.st) + p * L.st_stride, &hdr->ctr[p], &hdr->err) != cudaSuccess) {
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
