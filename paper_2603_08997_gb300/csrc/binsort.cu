// gs_bin_sort: tile binning and depth order ("depth-sorted Gaussians
// overlapping a given pixel", Sec. 3).
//
// The required order is the stable sort of the 64-bit keys
// (global tile id << 32 | float32 depth bits) in emission order (Gaussian
// index ascending, tiles row-major).  It is produced in two stages that give
// the same permutation without materialising or sorting any pair key:
//   1. sort the V*N (view, Gaussian) entries by depth bits (stable, so equal
//      depths keep ascending index), then stably by view;
//   2. place every pair by a counting sort over tiles that walks the entries
//      in that order (see bin_count .. coarse_place below).
// A stable sort by tile of a depth-ordered list is ordered by
// (tile, depth, index), i.e. exactly the 64-bit key order.  Stage 2 runs in
// two levels: a chunked counting sort of the entries by 4 x 4-tile
// super-tile (coarse_place), then, per super-tile, warps selecting each
// tile's entries from the super-tile's depth-ordered list (stage 2b below).
// gs_bin_sort_coarse stops after the first level: its lists are the output.
//
// Every kernel reads the counts it needs from device memory, so the whole
// call can be captured in a CUDA graph.  The radix sort is a reduce-then-scan
// LSD sort: an upsweep histogram per block, one exclusive scan over the
// digit-major (digit, block) counts, and a downsweep that ranks each tile of
// 2048 keys with warp ballots (one per digit bit), reorders the tile by digit
// in shared memory and writes each digit's run contiguously.  Keys are
// sorted relative to the visible keys' range (key_range_kernel), so passes
// above the range's bit length are copies; for one view in the super-tile
// form they do nothing at all, the last pass that sorts bits writing the depth
// order and the entries' rectangles directly (RsFinal).
#include "common.cuh"

using namespace gsr;

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int RS_MAX_BLOCKS = 1024;  // measured best of 304, 608, 1024 at 3M keys
constexpr int SCAN_THREADS = 1024;
static_assert(RS_THREADS == RADIX, "the downsweep gives each thread one digit");

static_assert(RS_MAX_BLOCKS <= 4 * RS_THREADS, "rs_scan holds at most four counts per thread");

struct ViewTiles {
    int64_t off;  // first global tile id
    int tx, ty;   // tile grid
};

__device__ __forceinline__ ViewTiles view_tiles(const gs_camera &cam, int tile) {
    ViewTiles vt;
    vt.off = cam.tile_offset;
    vt.tx = (cam.width + tile - 1) / tile;
    vt.ty = (cam.height + tile - 1) / tile;
    return vt;
}

__device__ __forceinline__ bool view_fits(const ViewTiles &vt, int64_t tiles, int max_vt) {
    const int64_t T = (int64_t)vt.tx * vt.ty;
    return vt.tx > 0 && vt.ty > 0 && T <= max_vt && vt.off >= 0 && vt.off + T <= tiles;
}

// The last pass of the depth sort may write, instead of the next ping-pong
// buffer, the entry ids alone to a buffer of their own (vals_final) and, for a
// single view, each entry's packed rectangle beside them (dst[pos] =
// src[entry], zero when the view's tile grid does not fit the tables): the
// pass after it then has nothing to copy, and the rectangles need no gather
// of their own.
struct RsFinal {
    uint32_t *vals;     // nullptr: every pass ping-pongs
    const ushort4 *src; // optional: rectangles by entry id
    ushort4 *dst;       //           and by depth position
    const gs_camera *cam;
    int tile, max_vt;
    int64_t tiles;
};

__device__ __forceinline__ int64_t effective_count(const int64_t *d_count, int64_t cap) {
    if (!d_count) return cap;
    const int64_t c = *d_count;
    return c < 0 ? 0 : (c < cap ? c : cap);
}

__device__ __forceinline__ void block_range(int64_t count, int G, int b, int64_t &begin, int64_t &end) {
    const int64_t per = ceil_div(ceil_div(count, G), RS_TILE) * RS_TILE;
    begin = (int64_t)b * per;
    if (begin > count) begin = count;
    end = begin + per;
    if (end > count) end = count;
}

// Depth-key range.  Keys are float32 bits of positive depths, 0xffffffff for
// culled entries.  Sorting k - min over the visible keys (culled ones mapped
// to the largest value: they emit no pairs, so where they land is
// irrelevant) gives the same order of the visible entries, ties included;
// passes whose digit lies above the range's bit length are then no-ops of
// the stable sort and are replaced by a copy.  krange = {min, max} over the
// visible keys (start {0xffffffff, 0}); one pair of atomics per block.
__global__ void key_range_kernel(const uint32_t *__restrict__ keys, int64_t count, uint32_t *__restrict__ krange) {
    __shared__ uint32_t s_lo[32], s_hi[32];
    uint32_t lo = 0xffffffffu, hi = 0u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += 4 * stride) {
        uint32_t k[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) k[j] = i + j * stride < count ? keys[i + j * stride] : 0xffffffffu;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (k[j] != 0xffffffffu) {
                lo = min(lo, k[j]);
                hi = max(hi, k[j]);
            }
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nwarps = blockDim.x >> 5;
        lo = threadIdx.x < nwarps ? s_lo[threadIdx.x] : 0xffffffffu;
        hi = threadIdx.x < nwarps ? s_hi[threadIdx.x] : 0u;
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if (threadIdx.x == 0) {
            atomicMin(&krange[0], lo);
            atomicMax(&krange[1], hi);
        }
    }
}

// Bits of the range (0: at most one distinct visible key).
__device__ __forceinline__ int range_bits(const uint32_t *krange) {
    const uint32_t lo = krange[0], hi = krange[1];
    return hi > lo ? 32 - __clz(hi - lo) : 0;
}

// The range as read once per thread: keys map to k - lo, culled ones to
// hi - lo, everything to 0 when no key is visible.
struct KeyRange {
    uint32_t lo, hi;
    bool on;
    __device__ __forceinline__ KeyRange(const uint32_t *krange, bool first) {
        on = first && krange;
        lo = on ? krange[0] : 0u;
        hi = on ? krange[1] : 0u;
    }
    __device__ __forceinline__ uint32_t operator()(uint32_t k) const {
        if (!on) return k;
        if (hi < lo) return 0u;
        return k == 0xffffffffu ? hi - lo : k - lo;
    }
};

template <bool FIRST>
__global__ void __launch_bounds__(RS_THREADS) rs_upsweep(const uint32_t *__restrict__ keys, const int64_t *d_count,
                                                         int64_t cap, int shift, uint32_t mask,
                                                         uint32_t *__restrict__ counts,
                                                         const uint32_t *__restrict__ krange) {
    __shared__ uint32_t hist[RADIX];
    if (krange && shift >= range_bits(krange)) return;  // a no-op pass (copied by the downsweep)
    for (int i = threadIdx.x; i < RADIX; i += RS_THREADS) hist[i] = 0;
    __syncthreads();
    const int64_t count = effective_count(d_count, cap);
    int64_t begin, end;
    block_range(count, gridDim.x, blockIdx.x, begin, end);
    const KeyRange kr(krange, FIRST);
    for (int64_t i = begin + threadIdx.x; i < end; i += RS_THREADS) atomicAdd(&hist[(kr(keys[i]) >> shift) & mask], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) counts[(int64_t)d * gridDim.x + blockIdx.x] = hist[d];
}

// Exclusive scan across a block of SCAN_THREADS threads; returns the
// thread's exclusive prefix and writes the block total to *total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *warp_sums, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t w = lane < nw ? warp_sums[lane] : 0u;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;  // inclusive
    }
    __syncthreads();
    const uint32_t before = warp > 0 ? warp_sums[warp - 1] : 0u;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + inc - x;
}

// Digit offsets, part 1: block d scans row d of the digit-major counts
// [RADIX][G] (exclusive, in place) and writes the row total.  The downsweep
// adds each digit's base (exclusive scan of the totals) itself.
__global__ void __launch_bounds__(RS_THREADS) rs_scan(uint32_t *a, int G, uint32_t *totals, int shift,
                                                      const uint32_t *__restrict__ krange) {
    __shared__ uint32_t warp_sums[32];
    if (krange && shift >= range_bits(krange)) return;
    uint32_t *row = a + (int64_t)blockIdx.x * G;
    const int per = (G + RS_THREADS - 1) / RS_THREADS;
    const int lo = min(G, (int)threadIdx.x * per), hi = min(G, lo + per);
    uint32_t v[4] = {0u, 0u, 0u, 0u};  // per <= 4 (G <= RS_MAX_BLOCKS <= 4 * RS_THREADS)
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (lo + j < hi) { v[j] = row[lo + j]; sum += v[j]; }
    uint32_t total;
    uint32_t run = block_exclusive_scan(sum, warp_sums, &total);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (lo + j < hi) { row[lo + j] = run; run += v[j]; }
    if (threadIdx.x == 0) totals[blockIdx.x] = total;
}

template <bool FIRST>
__global__ void __launch_bounds__(RS_THREADS) rs_downsweep(const uint32_t *__restrict__ keys_in,
                                                           const uint32_t *__restrict__ vals_in,
                                                           uint32_t *__restrict__ keys_out,
                                                           uint32_t *__restrict__ vals_out, const int64_t *d_count,
                                                           int64_t cap, int shift, uint32_t mask,
                                                           const uint32_t *__restrict__ offsets,
                                                           const uint32_t *__restrict__ totals,
                                                           const uint32_t *__restrict__ krange, RsFinal fin) {
    __shared__ uint32_t s_run[RADIX];   // global start of this block's next run per digit
    __shared__ uint32_t s_tot[RADIX];   // tile count per digit
    __shared__ uint32_t s_loc[RADIX];   // tile-local start per digit
    __shared__ uint32_t s_wcnt[RS_WARPS][RADIX];
    __shared__ uint32_t s_k[RS_TILE];
    __shared__ uint32_t s_v[RS_TILE];
    __shared__ uint32_t s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const KeyRange kr(krange, FIRST);
    const int rb = krange ? range_bits(krange) : 32;
    bool last = false;  // this pass writes fin.vals (and the rectangles)
    bool rfits = false;
    if (fin.vals) {  // with krange: the passes after the last one that sorts bits are no-ops
        const int last_shift = rb > 0 ? ((rb - 1) / RADIX_BITS) * RADIX_BITS : 0;
        if (shift > last_shift) return;
        last = shift == last_shift;
        rfits = last && fin.dst && view_fits(view_tiles(*fin.cam, fin.tile), fin.tiles, fin.max_vt);
    }
    // the last pass's outputs for entry id `val` at sorted position `pos`
    auto put_last = [&](int64_t pos, uint32_t val) {
        fin.vals[pos] = val;
        if (fin.dst) fin.dst[pos] = rfits ? fin.src[val] : make_ushort4(0, 0, 0, 0);
    };
    if (krange && shift >= rb) {  // every key's digit is 0: the stable pass keeps the order
        const int64_t count = effective_count(d_count, cap);
        int64_t begin, end;
        block_range(count, gridDim.x, blockIdx.x, begin, end);
        for (int64_t i = begin + threadIdx.x; i < end; i += RS_THREADS) {
            const uint32_t val = vals_in ? vals_in[i] : (uint32_t)i;
            if (last) {
                put_last(i, val);
            } else {
                keys_out[i] = kr(keys_in[i]);
                vals_out[i] = val;
            }
        }
        return;
    }
    {
        // digit base = exclusive scan of the digit totals (thread d owns digit d)
        uint32_t all;
        const uint32_t dbase = block_exclusive_scan(totals[threadIdx.x], s_warp, &all);
        s_run[threadIdx.x] = dbase + offsets[(int64_t)threadIdx.x * gridDim.x + blockIdx.x];
    }
    const int64_t count = effective_count(d_count, cap);
    int64_t begin, end;
    block_range(count, gridDim.x, blockIdx.x, begin, end);
    for (int64_t base = begin; base < end; base += RS_TILE) {
        const int n_tile = (int)min((int64_t)RS_TILE, end - base);
        for (int i = threadIdx.x; i < RS_WARPS * RADIX; i += RS_THREADS) (&s_wcnt[0][0])[i] = 0u;
        __syncthreads();
        // rank every item among the items of its digit in this tile (stable:
        // warp-major, then round, then lane = item order)
        uint32_t k[RS_ITEMS], v[RS_ITEMS], lr[RS_ITEMS];
        int dg[RS_ITEMS];
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {  // every load of the thread first
            const int li = warp * 32 * RS_ITEMS + r * 32 + lane;
            const bool valid = li < n_tile;
            k[r] = valid ? keys_in[base + li] : 0u;
            v[r] = valid ? (vals_in ? vals_in[base + li] : (uint32_t)(base + li)) : 0u;  // no values: the index
        }
        if constexpr (FIRST) {  // into the range, after every load is in flight
#pragma unroll
            for (int r = 0; r < RS_ITEMS; ++r) k[r] = kr(k[r]);
        }
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {
            const int li = warp * 32 * RS_ITEMS + r * 32 + lane;
            const bool valid = li < n_tile;
            const int d = valid ? (int)((k[r] >> shift) & mask) : RADIX + lane;
            // lanes with the same digit: intersect one ballot per digit bit
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int bit = 0; bit < RADIX_BITS; ++bit) {
                const uint32_t bb = __ballot_sync(0xffffffffu, (d >> bit) & 1);
                peers &= ((d >> bit) & 1) ? bb : ~bb;
            }
            const uint32_t rank = __popc(peers & lt_mask);
            uint32_t basec = 0;
            if (valid) basec = s_wcnt[warp][d];
            __syncwarp();
            if (valid && rank == 0) s_wcnt[warp][d] = basec + __popc(peers);
            __syncwarp();
            lr[r] = basec + rank;
            dg[r] = d;
        }
        __syncthreads();
        // per digit: exclusive prefix across warps and the tile total
        uint32_t tot = 0;
        for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) {
                const uint32_t c = s_wcnt[w][d];
                s_wcnt[w][d] = run;
                run += c;
            }
            s_tot[d] = run;
            tot = run;
        }
        // tile-local digit starts (RS_THREADS == RADIX: thread d owns digit d)
        uint32_t all;
        const uint32_t loc = block_exclusive_scan(tot, s_warp, &all);
        s_loc[threadIdx.x] = loc;
        __syncthreads();
        // reorder the tile by digit in shared memory
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {
            if (dg[r] < RADIX) {
                const uint32_t lp = s_loc[dg[r]] + s_wcnt[warp][dg[r]] + lr[r];
                s_k[lp] = k[r];
                s_v[lp] = v[r];
            }
        }
        __syncthreads();
        // write out: consecutive items of one digit go to consecutive addresses
        for (int i = threadIdx.x; i < n_tile; i += RS_THREADS) {
            const uint32_t key = s_k[i];
            const uint32_t d = (key >> shift) & mask;
            const uint32_t pos = s_run[d] + (uint32_t)i - s_loc[d];
            if (last) {
                put_last(pos, s_v[i]);
            } else {
                keys_out[pos] = key;
                vals_out[pos] = s_v[i];
            }
        }
        __syncthreads();
        for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) s_run[d] += s_tot[d];
        __syncthreads();
    }
}

int rs_blocks(int64_t cap) {
    int64_t g = ceil_div(cap, RS_TILE);
    if (g < 1) g = 1;
    if (g > RS_MAX_BLOCKS) g = RS_MAX_BLOCKS;
    return (int)g;
}

// Stable LSD sort of (key, value) pairs on the low `bits` bits of the keys.
// Ping-pongs between (ka, va) and (kb, vb); returns 0 when the result is in
// (ka, va), 1 when it is in (kb, vb).
// If k0 is given, the first pass reads its keys from k0 (left unchanged) with
// each key's index as its value, instead of from (ka, va).
// krange (device, nullable): the depth-key range of key_range_kernel; the
// first pass then sorts keys relative to it and passes above its bit length
// copy (see key_range_kernel).
// fin.vals (with krange): the last pass that sorts bits writes the entry ids
// (and the rectangles) there and the passes after it do nothing; the return
// value is then meaningless.
int radix_sort(uint32_t *ka, uint32_t *va, uint32_t *kb, uint32_t *vb, const int64_t *d_count, int64_t cap,
               int bits, uint32_t *counts, cudaStream_t stream, const uint32_t *k0 = nullptr,
               const uint32_t *krange = nullptr, RsFinal fin = RsFinal{}) {
    const int G = rs_blocks(cap);
    int cur = 0;
    for (int shift = 0; shift < bits; shift += RADIX_BITS) {
        const int nb = bits - shift < RADIX_BITS ? bits - shift : RADIX_BITS;
        const uint32_t mask = (1u << nb) - 1u;
        const uint32_t *ki = cur ? kb : ka;
        const uint32_t *vi = cur ? vb : va;
        if (shift == 0 && k0) {
            ki = k0;
            vi = nullptr;
        }
        uint32_t *ko = cur ? ka : kb, *vo = cur ? va : vb;
        uint32_t *totals = counts + (size_t)RADIX * RS_MAX_BLOCKS;
        if (shift == 0 && krange)  // the first pass maps the keys into the range
            rs_upsweep<true><<<G, RS_THREADS, 0, stream>>>(ki, d_count, cap, shift, mask, counts, krange);
        else
            rs_upsweep<false><<<G, RS_THREADS, 0, stream>>>(ki, d_count, cap, shift, mask, counts, krange);
        rs_scan<<<RADIX, RS_THREADS, 0, stream>>>(counts, G, totals, shift, krange);
        if (shift == 0 && krange)
            rs_downsweep<true><<<G, RS_THREADS, 0, stream>>>(ki, vi, ko, vo, d_count, cap, shift, mask, counts, totals,
                                                             krange, krange ? fin : RsFinal{});
        else
            rs_downsweep<false><<<G, RS_THREADS, 0, stream>>>(ki, vi, ko, vo, d_count, cap, shift, mask, counts,
                                                              totals, krange, krange ? fin : RsFinal{});
        cur ^= 1;
    }
    return cur;
}

// depth keys: float32 bits of the depth (positive, so the bit patterns order
// like the values); culled entries sort last and emit nothing.
__global__ void depth_keys_kernel(const float *__restrict__ rec, const int32_t *__restrict__ touched, int64_t total,
                                  uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    keys[e] = touched[e] > 0 ? __float_as_uint(rec[e * kRecFloats + 9]) : 0xffffffffu;
    vals[e] = (uint32_t)e;
}

// entry -> view key, for the stable pass that groups the depth order by view
__global__ void view_keys_kernel(const uint32_t *__restrict__ order, int64_t total, int64_t n,
                                 uint32_t *__restrict__ keys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) keys[i] = (uint32_t)(order[i] / n);
}

// ----------------------------------------------------------------------------
// Stage 2: counting sort of the pairs by tile, in depth order.
//
// The depth-ordered entries of view v are cut into chunks of C entries.  For
// chunk c of view v and tile t of that view, let cnt(c, t) be the number of
// the chunk's entries whose rectangle covers t.  The pair of entry e at tile t
// then lands at
//   start(t) + sum_{c' < c} cnt(c', t) + #(earlier entries of chunk c covering t),
// with start(t) the exclusive scan of the tile totals over global tile ids.
// That is the position of the pair in the stable sort by tile of the
// depth-ordered pair list, so no pair key is ever materialised or sorted.
//   bin_rects:   the clipped rectangles in depth order (one gather, or
//                written by the depth sort's last pass);
//   bin_count:   one block per chunk: per-tile counts in shared memory, written
//                as the chunk's row of the count matrix (chunk-major per view)
//                and added into the per-group sums (BIN_GROUP chunks a group);
//   bin_groups:  per tile, exclusive scan over its groups and the tile total;
//   bin_starts:  exclusive scan of the tile totals (one block), pair count and
//                capacity check;
//   bin_offsets: per (group, tile), the count matrix becomes the chunks' first
//                slots, and group 0 writes the tile's range;
//   coarse_place: one block per chunk places the chunk's pairs (below).
// On the tile grid only the tile totals are used (bin_count, bin_groups,
// bin_starts: each tile's start and range); the placement runs on the grid of
// super-tiles (BinGeom.sup), where coarse_place writes the super-tile lists,
// and stage 2b fills the tiles (or, in the super-tile form, the compositing
// kernels filter them).
constexpr int BIN_GROUP = 16;
constexpr int COUNT_THREADS = 1024;

constexpr int SUP = kSup;         // tiles per super-tile side
constexpr int SUP_T = SUP * SUP;  // tiles per super-tile: one mask bit each

// Bits k = 4 row + column of the super-tile's tiles (its first tile at
// (x0, y0)) that the clipped tile rectangle r covers.
__device__ __forceinline__ uint32_t cover_mask(ushort4 r, int x0, int y0) {
    if (r.z == 0) return 0u;
    const int c0 = max((int)r.x - x0, 0), c1 = min((int)r.x + (int)r.z - x0, SUP);
    const int r0 = max((int)r.y - y0, 0), r1 = min((int)r.y + (int)r.w - y0, SUP);
    if (c0 >= c1 || r0 >= r1) return 0u;
    const uint32_t cols = ((1u << c1) - 1u) & ~((1u << c0) - 1u);
    uint32_t m = 0;
#pragma unroll
    for (int y = 0; y < SUP; ++y)
        if (y >= r0 && y < r1) m |= cols << (SUP * y);
    return m;
}

struct BinGeom {
    int64_t n;       // entries per view
    int64_t chunk;   // entries per chunk
    int64_t n_c;     // chunks per view
    int64_t n_g;     // groups per view
    int64_t tiles;   // total tiles over all views (of this grid)
    int tile;        // pixels per tile side
    int max_vt;      // tiles per view the shared-memory tables hold
    int sup;         // 1: the tile grid; SUP: the grid of SUP x SUP super-tiles
    const int64_t *coff;  // sup > 1: first super-tile id of each view, [n_views + 1] (device)
};

// Entries per chunk: n / `chunks` (about two chunks per SM for one view on
// the tile grid), at least 1024, in multiples of 256.
int64_t bin_chunk(int64_t n, int64_t chunks = 304) {
    int64_t c = ceil_div(n, chunks);
    c = ceil_div(c, (int64_t)256) * 256;
    return c < 1024 ? 1024 : c;
}

// The grid a BinGeom counts and places on: the view's tiles, or its
// super-tiles (SUP x SUP tiles each; the view's first super-tile id from
// g.coff).
__device__ __forceinline__ ViewTiles view_grid(const BinGeom &g, const gs_camera *cams, int64_t v) {
    ViewTiles vt = view_tiles(cams[v], g.tile);
    if (g.sup > 1) {
        vt.tx = (vt.tx + g.sup - 1) / g.sup;
        vt.ty = (vt.ty + g.sup - 1) / g.sup;
        vt.off = g.coff[v];
    }
    return vt;
}

// A clipped tile rectangle (x0, y0, width, height) in the geometry's grid.
__device__ __forceinline__ ushort4 grid_rect(const BinGeom &g, ushort4 r) {
    if (g.sup == 1 || r.z == 0) return r;
    const int x0 = r.x / g.sup, y0 = r.y / g.sup;
    const int x1 = (r.x + r.z - 1) / g.sup, y1 = (r.y + r.w - 1) / g.sup;
    return make_ushort4((unsigned short)x0, (unsigned short)y0, (unsigned short)(x1 - x0 + 1),
                        (unsigned short)(y1 - y0 + 1));
}

// The view a global id of the geometry's grid belongs to.
__device__ __forceinline__ int view_of_grid_tile(const BinGeom &g, const gs_camera *cams, int n_views, int64_t gt) {
    if (g.sup == 1) return view_of_tile(cams, n_views, gt);
    int v = 0;
    while (v + 1 < n_views && g.coff[v + 1] <= gt) ++v;
    return v;
}

// Does the view's tile table fit the shared-memory tables and the global
// tile range?  (Tile offsets that disagree with total_tiles would not.)

// Rectangle of an entry clipped to its view's tile grid, packed as
// (x0, y0, width, height) in 16 bits each; width 0 = no pair (culled/empty).
__global__ void bin_rects(const int4 *__restrict__ rect, const int32_t *__restrict__ touched,
                          const uint32_t *__restrict__ order, const gs_camera *__restrict__ cams, BinGeom g,
                          int64_t total, ushort4 *__restrict__ srect) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const uint32_t e = order[i];
    const ViewTiles vt = view_tiles(cams[i / g.n], g.tile);
    ushort4 o = make_ushort4(0, 0, 0, 0);
    if (touched[e] > 0 && view_fits(vt, g.tiles, g.max_vt)) {
        const int4 r = rect[e];
        const int x0 = max(r.x, 0), y0 = max(r.y, 0), x1 = min(r.z, vt.tx - 1), y1 = min(r.w, vt.ty - 1);
        if (x0 <= x1 && y0 <= y1)
            o = make_ushort4((unsigned short)x0, (unsigned short)y0, (unsigned short)(x1 - x0 + 1),
                             (unsigned short)(y1 - y0 + 1));
    }
    srect[i] = o;
}

// Pair counts of one chunk per tile by a 2D difference array: each entry adds
// +1 / -1 / -1 / +1 at the four corners of its rectangle on a (tx + 1) x
// (ty + 1) grid, and prefix sums along rows, then columns, give every tile the
// number of the chunk's rectangles covering it (four shared atomics per entry
// instead of one per pair, and no divergence on large rectangles).
// The same from the packed rectangles gs_project wrote (already clipped).
__global__ void bin_rects16(const ushort4 *__restrict__ rect16, const uint32_t *__restrict__ order,
                            const gs_camera *__restrict__ cams, BinGeom g, int64_t total, ushort4 *__restrict__ srect) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const ViewTiles vt = view_tiles(cams[i / g.n], g.tile);
    srect[i] = view_fits(vt, g.tiles, g.max_vt) ? rect16[order[i]] : make_ushort4(0, 0, 0, 0);
}

__global__ void __launch_bounds__(COUNT_THREADS) bin_count(const ushort4 *__restrict__ srect,
                                                           const gs_camera *__restrict__ cams, BinGeom g,
                                                           uint32_t *__restrict__ M, uint32_t *__restrict__ G1,
                                                           int32_t *dev_status) {
    extern __shared__ int s_d[];  // [(tx + 1) * (ty + 1)] <= 2 max_vt + 2
    const int64_t v = blockIdx.x / g.n_c, c = blockIdx.x % g.n_c;
    const ViewTiles vt = view_grid(g, cams, v);
    if (!view_fits(vt, g.tiles, g.max_vt)) {
        if (threadIdx.x == 0) set_status(dev_status, GS_ERR_INVALID_ARG);
        return;
    }
    const int T = vt.tx * vt.ty, W = vt.tx + 1, D = W * (vt.ty + 1);
    for (int t = threadIdx.x; t < D; t += COUNT_THREADS) s_d[t] = 0;
    __syncthreads();
    const int64_t e0 = v * g.n + c * g.chunk, e1 = v * g.n + min((c + 1) * g.chunk, g.n);
    for (int64_t i = e0 + threadIdx.x; i < e1; i += COUNT_THREADS) {
        const ushort4 r = grid_rect(g, srect[i]);
        if (r.z == 0) continue;
        const int x0 = r.x, y0 = r.y, x1 = x0 + r.z, y1 = y0 + r.w;
        atomicAdd(&s_d[y0 * W + x0], 1);
        atomicSub(&s_d[y0 * W + x1], 1);
        atomicSub(&s_d[y1 * W + x0], 1);
        atomicAdd(&s_d[y1 * W + x1], 1);
    }
    __syncthreads();
    for (int y = threadIdx.x; y < vt.ty; y += COUNT_THREADS) {  // along rows
        int run = 0;
        for (int x = 0; x < vt.tx; ++x) {
            run += s_d[y * W + x];
            s_d[y * W + x] = run;
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < vt.tx; x += COUNT_THREADS) {  // along columns
        int run = 0;
        for (int y = 0; y < vt.ty; ++y) {
            run += s_d[y * W + x];
            s_d[y * W + x] = run;
        }
    }
    __syncthreads();
    uint32_t *row = M ? M + g.n_c * vt.off + c * T : nullptr;  // no M: only the group sums are needed
    uint32_t *grp = G1 + (c / BIN_GROUP) * g.tiles + vt.off;
    for (int t = threadIdx.x; t < T; t += COUNT_THREADS) {
        const uint32_t h = (uint32_t)s_d[(t / vt.tx) * W + (t % vt.tx)];
        if (row) row[t] = h;
        if (h) atomicAdd(&grp[t], h);
    }
}

// Per global tile: exclusive scan of its group sums (in place) and its total.
__global__ void bin_groups(BinGeom g, uint32_t *__restrict__ G1, uint32_t *__restrict__ tile_total) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt >= g.tiles) return;
    uint32_t run = 0;
    for (int64_t k0 = 0; k0 < g.n_g; k0 += 16) {  // 16 independent loads in flight, then their prefix
        uint32_t x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] = k0 + j < g.n_g ? G1[(k0 + j) * g.tiles + gt] : 0u;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (k0 + j < g.n_g) G1[(k0 + j) * g.tiles + gt] = run;
            run += x[j];
        }
    }
    tile_total[gt] = run;
}

// Exclusive scan of the tile totals by one block: each thread sums a
// contiguous run of tiles, the block scans the run sums, each thread writes
// its run's starts.  Writes the pair count; over capacity (or past 32-bit
// slots) sets GS_ERR_CAPACITY and a sort count of 0, which stops the later
// stages and leaves the ranges empty.
__global__ void __launch_bounds__(SCAN_THREADS) bin_starts(BinGeom g, const uint32_t *__restrict__ tile_total,
                                                           uint32_t *__restrict__ tile_start, int64_t cap,
                                                           int64_t *dev_pair_count, int64_t *sort_count,
                                                           int32_t *dev_status) {
    __shared__ unsigned long long s[SCAN_THREADS];
    const int64_t per = ceil_div(g.tiles, (int64_t)SCAN_THREADS);
    const int64_t lo = min(g.tiles, (int64_t)threadIdx.x * per), hi = min(g.tiles, lo + per);
    unsigned long long sum = 0;
    for (int64_t t = lo; t < hi; ++t) sum += tile_total[t];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < SCAN_THREADS; off <<= 1) {
        const unsigned long long y = threadIdx.x >= off ? s[threadIdx.x - off] : 0ull;
        __syncthreads();
        s[threadIdx.x] += y;
        __syncthreads();
    }
    const unsigned long long P = s[SCAN_THREADS - 1];
    const bool ok = (int64_t)P <= cap && P < 0xffffffffull;
    unsigned long long run = s[threadIdx.x] - sum;
    if (ok) {
        for (int64_t t = lo; t < hi; ++t) {
            tile_start[t] = (uint32_t)run;
            run += tile_total[t];
        }
    }
    if (threadIdx.x == 0) {
        *dev_pair_count = (int64_t)P;
        *sort_count = ok ? (int64_t)P : 0;
        if (!ok) set_status(dev_status, GS_ERR_CAPACITY);
    }
}

// Per (group, global tile): rewrite the group's counts cnt(c, t) as the
// chunks' first slots; group 0 also writes the tile's range.  The group's
// counts are read before any is written back.
__global__ void bin_offsets(BinGeom g, const gs_camera *__restrict__ cams, int n_views,
                            const uint32_t *__restrict__ G1, const uint32_t *__restrict__ tile_start,
                            const uint32_t *__restrict__ tile_total, const int64_t *sort_count,
                            uint32_t *__restrict__ M, uint2 *__restrict__ ranges) {
    if (*sort_count == 0) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_g * g.tiles) return;
    const int64_t k = i / g.tiles, gt = i % g.tiles;
    const int v = view_of_grid_tile(g, cams, n_views, gt);
    const ViewTiles vt = view_grid(g, cams, v);
    if (!view_fits(vt, g.tiles, g.max_vt)) return;
    const int T = vt.tx * vt.ty;
    const int64_t t = gt - vt.off;
    if (t < 0 || t >= T) return;
    uint32_t run = tile_start[gt] + G1[k * g.tiles + gt];
    const int64_t c0 = k * BIN_GROUP, c1 = min(g.n_c, c0 + BIN_GROUP);
    uint32_t *col = M + g.n_c * vt.off + t;
    uint32_t x[BIN_GROUP];
#pragma unroll
    for (int j = 0; j < BIN_GROUP; ++j) x[j] = c0 + j < c1 ? col[(c0 + j) * T] : 0u;
#pragma unroll
    for (int j = 0; j < BIN_GROUP; ++j) {
        if (c0 + j < c1) col[(c0 + j) * T] = run;
        run += x[j];
    }
    if (k == 0 && ranges) {
        const uint32_t tot = tile_total[gt];
        ranges[gt] = tot ? make_uint2(tile_start[gt], tile_start[gt] + tot) : make_uint2(0u, 0u);
    }
}

// The super-tile lists, placed by warps.  One block per chunk of a view's
// depth-ordered entries (the chunks of the count matrix M, whose row for the
// chunk holds each super-tile's first slot); each of its warps takes a
// contiguous part of the chunk.  Phase 1: every warp counts its pairs per
// super-tile (shared atomics into its own row).  Phase 2: per super-tile, the
// warps' first slots follow from the chunk's first slot and the counts of
// the warps before.  Phase 3, per window of 32 entries: lane j sets bit j of
// the window's word of every super-tile of its rectangle (shared atomicOr),
// so a pair's rank among the window's pairs of its super-tile is the
// popcount of the bits below j; the window's pairs, spread evenly over the
// lanes (a warp scan of the entries' pair counts; lane l takes pairs
// p0 + l for p0 = 0, 32, ...), are written there (Gaussian index and the
// super-tile's covered-tile mask), and the pair of each word's lowest entry
// advances the warp's slot and clears the word.  Warps never wait on one
// another (only __syncwarp inside a warp); the order is the stable one the
// count matrix implies.  Shared memory: two rows of max_vt words per warp.
constexpr int CP_MAX_WARPS = 16;

// Window of 32 entries of a warp: lane j holds entry j's rectangle (in the
// super-tile grid) and the inclusive prefix of the pair counts.
struct PairWindow {
    ushort4 r;
    int incl, total;
    // pair p of the window -> its entry j and super-tile (cx, cy)
    __device__ __forceinline__ void pair(int p, int &j, int &cx, int &cy) const {
        int lo = 0;  // the first lane whose inclusive prefix exceeds p
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int probe = __shfl_sync(0xffffffffu, incl, lo + step - 1);
            if (probe <= p) lo += step;
        }
        j = lo;
        const uint32_t xy = __shfl_sync(0xffffffffu, (uint32_t)r.x | ((uint32_t)r.y << 16), j);
        const int w = __shfl_sync(0xffffffffu, (int)r.z, j);
        const int before = __shfl_sync(0xffffffffu, incl - (int)r.z * r.w, j);
        const int k = p - before;
        int dy = 0;
        if (w > 1) {  // k / w from the float reciprocal, corrected by one step (k, w < 2^16)
            dy = __float2int_rz((float)k * __frcp_rn((float)w));
            if (dy * w > k) --dy;
            else if ((dy + 1) * w <= k) ++dy;
        } else {
            dy = k;
        }
        cx = (int)(xy & 0xffffu) + (k - dy * w);
        cy = (int)(xy >> 16) + dy;
    }
};

__device__ __forceinline__ PairWindow pair_window(ushort4 r, int lane) {
    PairWindow pw;
    pw.r = r;
    int inc = (int)r.z * r.w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    pw.incl = inc;
    pw.total = __shfl_sync(0xffffffffu, inc, 31);
    return pw;
}

__global__ void __launch_bounds__(CP_MAX_WARPS * 32) coarse_place(const ushort4 *__restrict__ srect,
                                                                  const uint32_t *__restrict__ order,
                                                                  const gs_camera *__restrict__ cams, BinGeom g,
                                                                  const uint32_t *__restrict__ M,
                                                                  const int64_t *sort_count,
                                                                  uint32_t *__restrict__ gid_out,
                                                                  uint16_t *__restrict__ mask_out) {
    extern __shared__ uint32_t s_tab[];  // [warps][max_vt] counts, then slots; [warps][max_vt] window bits
    if (*sort_count == 0) return;
    const int64_t v = blockIdx.x / g.n_c, c = blockIdx.x % g.n_c;
    const ViewTiles vt = view_grid(g, cams, v);
    if (!view_fits(vt, g.tiles, g.max_vt)) return;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int T = vt.tx * vt.ty;
    uint32_t *slot = s_tab + (size_t)warp * g.max_vt;
    uint32_t *bits = s_tab + (size_t)(nw + warp) * g.max_vt;
    for (int t = threadIdx.x; t < nw * T; t += blockDim.x) {
        s_tab[(size_t)(t / T) * g.max_vt + t % T] = 0u;
        s_tab[(size_t)(nw + t / T) * g.max_vt + t % T] = 0u;
    }
    __syncthreads();
    const int64_t e0 = v * g.n + c * g.chunk, e1 = v * g.n + min((c + 1) * g.chunk, g.n);
    const int64_t per = ((e1 - e0 + nw - 1) / nw + 31) / 32 * 32;  // whole windows per warp
    const int64_t w0 = min(e1, e0 + warp * per), w1 = min(e1, w0 + per);
    // phase 1: the warp's pairs per super-tile (each lane its own entry's, row by row)
    for (int64_t base = w0; base < w1; base += 32) {
        const int64_t i = base + lane;
        const ushort4 r = i < w1 ? grid_rect(g, srect[i]) : make_ushort4(0, 0, 0, 0);
        const int area = (int)r.z * r.w;
        int t = r.y * vt.tx + r.x, x = 0;
        for (int k = 0; k < area; ++k) {
            atomicAdd(&slot[t], 1u);
            if (++x == r.z) {
                x = 0;
                t += vt.tx - (r.z - 1);
            } else {
                ++t;
            }
        }
    }
    __syncthreads();
    // phase 2: the warps' first slots per super-tile
    const uint32_t *row = M + g.n_c * vt.off + c * T;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        uint32_t run = row[t];
        for (int w = 0; w < nw; ++w) {
            uint32_t *x = s_tab + (size_t)w * g.max_vt + t;
            const uint32_t cnt = *x;
            *x = run;
            run += cnt;
        }
    }
    __syncthreads();
    // phase 3: place (the next window's entries load while this one is placed)
    ushort4 fr_next = make_ushort4(0, 0, 0, 0);
    uint32_t g_next = 0;
    if (w0 + lane < w1) {
        fr_next = srect[w0 + lane];
        g_next = (uint32_t)((int64_t)order[w0 + lane] - v * g.n);
    }
    for (int64_t base = w0; base < w1; base += 32) {
        const ushort4 fr = fr_next;  // lane j: entry j's tile rectangle and Gaussian index
        const uint32_t gi = g_next;
        const int64_t nx = base + 32 + lane;
        if (nx < w1) {
            fr_next = srect[nx];
            g_next = (uint32_t)((int64_t)order[nx] - v * g.n);
        }
        const ushort4 r = base + lane < w1 ? grid_rect(g, fr) : make_ushort4(0, 0, 0, 0);
        const int area = (int)r.z * r.w;
        const int t0 = r.y * vt.tx + r.x;
        {  // pass A: the lane's own pairs, row by row
            int t = t0, x = 0;
            for (int k = 0; k < area; ++k) {
                atomicOr(&bits[t], 1u << lane);
                if (++x == r.z) {
                    x = 0;
                    t += vt.tx - (r.z - 1);
                } else {
                    ++t;
                }
            }
        }
        __syncwarp();
        // pass B: the window's pairs spread evenly over the lanes
        const PairWindow pw = pair_window(r, lane);
        const uint32_t fxy = (uint32_t)fr.x | ((uint32_t)fr.y << 16), fwh = (uint32_t)fr.z | ((uint32_t)fr.w << 16);
        for (int p0 = 0; p0 < pw.total; p0 += 32) {
            int j = 0, cx = 0, cy = 0;
            pw.pair(p0 + lane, j, cx, cy);
            const uint32_t jxy = __shfl_sync(0xffffffffu, fxy, j);
            const uint32_t jwh = __shfl_sync(0xffffffffu, fwh, j);
            const uint32_t gj = __shfl_sync(0xffffffffu, gi, j);
            if (p0 + lane < pw.total) {
                const int t = cy * vt.tx + cx;
                const uint32_t d = slot[t] + (uint32_t)__popc(bits[t] & ((1u << j) - 1u));
                const ushort4 frj = make_ushort4((unsigned short)(jxy & 0xffffu), (unsigned short)(jxy >> 16),
                                                 (unsigned short)(jwh & 0xffffu), (unsigned short)(jwh >> 16));
                gid_out[d] = gj;
                mask_out[d] = (uint16_t)cover_mask(frj, cx * SUP, cy * SUP);
            }
        }
        __syncwarp();
        {  // pass C: the lane's own pairs again
            int t = t0, x = 0;
            for (int k = 0; k < area; ++k) {
                const uint32_t b = bits[t];
                if (b != 0u && (b & lt) == 0u) {  // the word's lowest entry (others see it or 0)
                    slot[t] += (uint32_t)__popc(b);
                    bits[t] = 0u;
                }
                if (++x == r.z) {
                    x = 0;
                    t += vt.tx - (r.z - 1);
                } else {
                    ++t;
                }
            }
        }
        __syncwarp();
    }
}

// Warps per block of coarse_place: the most (up to CP_MAX_WARPS, a power of
// two) whose tables fit 200 KB of shared memory.
int coarse_place_warps(int64_t max_vt) {
    int w = CP_MAX_WARPS;
    while (w > 1 && (size_t)2 * w * max_vt * sizeof(uint32_t) > (size_t)200 * 1024) w >>= 1;
    return w;
}

// ----------------------------------------------------------------------------
// Stage 2b: placement by super-tile.
//
// The chunked counting sort above, run on the grid of SUP x SUP super-tiles
// with entry positions as values, gives every super-tile the depth-ordered
// list of the entries whose rectangle meets it (its "coarse list").  A coarse
// list is cut into work items of WI entries, one warp each.  The warp takes
// its entries 32 at a time; each lane reads its entry's 16-bit mask of the
// super-tile's tiles it covers (written by the scatter), and one ballot per
// tile gives each covering lane its rank among the group's covering lanes: the
// tile's pairs from the item, in depth order, go to consecutive slots.  A
// count pass gives each (item, tile) its pair count, a scan per super-tile
// over its items (after the tile's start) the first slots, and the place pass
// writes.  Every pair is written once, each tile's run contiguously, and no
// warp waits on another.
constexpr int WI = 512;           // coarse-list entries per work item (one warp)
constexpr int FP_THREADS = 256;   // threads of the placement blocks (8 warps)

// coff[v]: first super-tile id of view v; coff[n_views]: the total.
__global__ void coarse_offsets(const gs_camera *__restrict__ cams, int n_views, int tile, int64_t *__restrict__ coff) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t run = 0;
    for (int v = 0; v < n_views; ++v) {
        coff[v] = run;
        const int64_t tx = (cams[v].width + tile - 1) / tile, ty = (cams[v].height + tile - 1) / tile;
        if (tx > 0 && ty > 0) run += ((tx + SUP - 1) / SUP) * ((ty + SUP - 1) / SUP);
    }
    coff[n_views] = run;
}

// Work items: seg_base[ct] = exclusive scan of ceil(ctotal[ct] / WI) over
// the super-tiles (one block), seg_base[tiles] = the item count (0 when the
// pairs exceeded the capacity).
__global__ void __launch_bounds__(SCAN_THREADS) seg_layout(int64_t tiles, const uint32_t *__restrict__ ctotal,
                                                           const int64_t *sort_count, uint32_t *__restrict__ seg_base) {
    __shared__ uint32_t s[SCAN_THREADS];
    const bool ok = *sort_count != 0;
    const int64_t per = ceil_div(tiles, (int64_t)SCAN_THREADS);
    const int64_t lo = min(tiles, (int64_t)threadIdx.x * per), hi = min(tiles, lo + per);
    uint32_t sum = 0;
    for (int64_t t = lo; t < hi; ++t) sum += ok ? (ctotal[t] + WI - 1) / WI : 0u;
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < SCAN_THREADS; off <<= 1) {
        const uint32_t y = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += y;
        __syncthreads();
    }
    uint32_t run = s[threadIdx.x] - sum;
    for (int64_t t = lo; t < hi; ++t) {
        seg_base[t] = run;
        run += ok ? (ctotal[t] + WI - 1) / WI : 0u;
    }
    if (threadIdx.x == 0) seg_base[tiles] = s[SCAN_THREADS - 1];
}

__global__ void seg_fill(int64_t tiles, const uint32_t *__restrict__ seg_base, uint32_t *__restrict__ item_ct) {
    const int64_t ct = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ct >= tiles) return;
    for (uint32_t it = seg_base[ct]; it < seg_base[ct + 1]; ++it) item_ct[it] = (uint32_t)ct;
}

// Geometry of work item `item`: its view and its entries of the super-tile's list.
struct ItemGeom {
    int v, cnt;
    uint32_t b0;
    bool fits;
};

__device__ __forceinline__ ItemGeom item_geom(uint32_t item, const BinGeom &gc, const gs_camera *cams, int n_views,
                                              const uint32_t *cstart, const uint32_t *ctotal,
                                              const uint32_t *seg_base, const uint32_t *item_ct, int64_t fine_tiles,
                                              int fine_max_vt) {
    ItemGeom ig;
    const uint32_t ct = item_ct[item];
    const uint32_t sg = item - seg_base[ct];
    ig.v = view_of_grid_tile(gc, cams, n_views, ct);
    const ViewTiles ft = view_tiles(cams[ig.v], gc.tile);
    ig.fits = view_fits(ft, fine_tiles, fine_max_vt);
    ig.b0 = cstart[ct] + sg * WI;
    ig.cnt = (int)min((uint32_t)WI, ctotal[ct] - sg * WI);
    return ig;
}

// PLACE = false: per item and tile of its super-tile, the number of the
// item's entries covering the tile (into run_of[item][k]).  PLACE = true:
// run_of[item][k] holds the tile's first slot for the item; the covering
// entries' Gaussian indices are written from there in list order.  Warps
// take items in a grid-stride loop (the item count is on the device); the
// item's records are read in order (coalesced).
template <bool PLACE>
__global__ void __launch_bounds__(FP_THREADS) fine_pass(const uint16_t *__restrict__ cmask,
                                                        const uint32_t *__restrict__ cgid,
                                                        const gs_camera *__restrict__ cams, int n_views, BinGeom gc,
                                                        const uint32_t *__restrict__ cstart,
                                                        const uint32_t *__restrict__ ctotal,
                                                        const uint32_t *__restrict__ seg_base,
                                                        const uint32_t *__restrict__ item_ct,
                                                        uint32_t *__restrict__ run_of, uint32_t *__restrict__ vals,
                                                        int64_t fine_tiles, int fine_max_vt, int64_t cap) {
    const uint32_t n_items = seg_base[gc.tiles];
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint32_t warps = gridDim.x * (FP_THREADS / 32);
    for (uint32_t item = blockIdx.x * (FP_THREADS / 32) + (threadIdx.x >> 5); item < n_items; item += warps) {
        const ItemGeom ig = item_geom(item, gc, cams, n_views, cstart, ctotal, seg_base, item_ct, fine_tiles,
                                      fine_max_vt);
        uint32_t run[SUP_T];
#pragma unroll
        for (int k = 0; k < SUP_T; ++k) run[k] = PLACE ? run_of[(size_t)item * SUP_T + k] : 0u;
        if (ig.fits) {  // else no pairs (the tile counts flagged the view)
            for (int g0 = 0; g0 < ig.cnt; g0 += 32) {
                const int j = g0 + lane;
                uint32_t m = 0, gid = 0;
                if (j < ig.cnt) {
                    m = cmask[ig.b0 + j];
                    if (PLACE) gid = cgid[ig.b0 + j];
                }
#pragma unroll
                for (int k = 0; k < SUP_T; ++k) {
                    const bool cov = (m >> k) & 1u;
                    const uint32_t b = __ballot_sync(0xffffffffu, cov);
                    if (PLACE && cov) {
                        const uint32_t d = run[k] + __popc(b & lt_mask);
                        if (d < cap) vals[d] = gid;  // always below: the tile counts bound the runs
                    }
                    run[k] += __popc(b);
                }
            }
        }
        if (!PLACE && lane < SUP_T) {
            uint32_t mine = 0;
#pragma unroll
            for (int k = 0; k < SUP_T; ++k) mine = lane == k ? run[k] : mine;
            run_of[(size_t)item * SUP_T + lane] = mine;
        }
    }
}

// One warp per super-tile: the counts of its items become first slots (per
// tile, an exclusive scan over the items after the tile's start: lanes take
// 32 items at a time, shuffle scans per tile), and its tiles' ranges are
// written.
__global__ void __launch_bounds__(256) fine_prefix(const gs_camera *__restrict__ cams, int n_views, BinGeom gc,
                                                   int64_t tiles, int fine_max_vt,
                                                   const uint32_t *__restrict__ tile_start,
                                                   const uint32_t *__restrict__ tile_total,
                                                   const uint32_t *__restrict__ seg_base, const int64_t *sort_count,
                                                   uint32_t *__restrict__ run_of, uint2 *__restrict__ ranges) {
    if (*sort_count == 0) return;
    const int64_t ct = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (ct >= gc.tiles || ct >= gc.coff[n_views]) return;  // whole warps
    const int v = view_of_grid_tile(gc, cams, n_views, ct);
    const ViewTiles ft = view_tiles(cams[v], gc.tile);
    if (!view_fits(ft, tiles, fine_max_vt)) return;
    const int ctx = (ft.tx + SUP - 1) / SUP;
    const int64_t lct = ct - gc.coff[v];
    const int x0 = (int)(lct % ctx) * SUP, y0 = (int)(lct / ctx) * SUP;
    // lane k < 16: tile k of the super-tile, its start and range
    int64_t gt = -1;
    uint32_t carry = 0;
    if (lane < SUP_T) {
        const int fx = x0 + lane % SUP, fy = y0 + lane / SUP;
        if (fx < ft.tx && fy < ft.ty) {
            gt = ft.off + (int64_t)fy * ft.tx + fx;
            carry = tile_start[gt];
            const uint32_t tot = tile_total[gt];
            ranges[gt] = tot ? make_uint2(carry, carry + tot) : make_uint2(0u, 0u);
        }
    }
    const uint32_t i0 = seg_base[ct], i1 = seg_base[ct + 1];
    for (uint32_t base = i0; base < i1; base += 32) {
        const uint32_t it = base + lane;
        const bool valid = it < i1;
        uint32_t c[SUP_T];
#pragma unroll
        for (int q = 0; q < SUP_T / 4; ++q) {
            const uint4 x = valid ? reinterpret_cast<const uint4 *>(run_of + (size_t)it * SUP_T)[q]
                                  : make_uint4(0u, 0u, 0u, 0u);
            c[4 * q] = x.x;
            c[4 * q + 1] = x.y;
            c[4 * q + 2] = x.z;
            c[4 * q + 3] = x.w;
        }
#pragma unroll
        for (int k = 0; k < SUP_T; ++k) {
            uint32_t inc = c[k];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const uint32_t start_k = __shfl_sync(0xffffffffu, carry, k);  // tile k's running slot
            const uint32_t total_k = __shfl_sync(0xffffffffu, inc, 31);
            c[k] = start_k + inc - c[k];
            if (lane == k) carry += total_k;
        }
        if (valid) {
#pragma unroll
            for (int q = 0; q < SUP_T / 4; ++q)
                reinterpret_cast<uint4 *>(run_of + (size_t)it * SUP_T)[q] =
                    make_uint4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]);
        }
    }
    (void)gt;
}

// 64-bit keys of the sorted pairs (for checking the order): one block per tile.
__global__ void keys64_kernel(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
                              const int64_t *sort_count, const gs_camera *__restrict__ cams, int n_views, int64_t n,
                              const float *__restrict__ rec, uint64_t *__restrict__ keys) {
    if (*sort_count == 0) return;
    const int64_t gt = blockIdx.x;
    const uint2 rg = ranges[gt];
    if (rg.y <= rg.x) return;
    const int v = view_of_tile(cams, n_views, gt);
    for (uint32_t i = rg.x + threadIdx.x; i < rg.y; i += blockDim.x) {
        const int64_t e = (int64_t)v * n + vals[i];
        keys[i] = ((uint64_t)gt << 32) | (uint64_t)__float_as_uint(rec[e * kRecFloats + 9]);
    }
}

int bits_for(int64_t values) {  // bits needed to represent 0 .. values-1
    int b = 0;
    while (b < 63 && ((int64_t)1 << b) < values) ++b;
    return b < 1 ? 1 : b;
}

BinGeom bin_geom(int64_t n, int64_t total_tiles, int tile, int max_vt) {
    BinGeom g;
    g.n = n;
    g.chunk = bin_chunk(n);
    g.n_c = ceil_div(n > 0 ? n : 1, g.chunk);
    g.n_g = ceil_div(g.n_c, (int64_t)BIN_GROUP);
    g.tiles = total_tiles;
    g.tile = tile;
    g.max_vt = max_vt;
    g.sup = 1;
    g.coff = nullptr;
    return g;
}

// The super-tile grid: a view of T tiles (tx * ty <= max_vt) has at most
// ceil(tx / SUP) * ceil(ty / SUP) <= (T + 3 (tx + ty) + 9) / 16 <= max_vt / 4
// + 1 super-tiles (tx + ty <= T + 1), so all views together at most
// total_tiles / 4 + n_views.  Smaller tables allow shorter chunks (about four
// per SM).
// max_super > 0: the caller's bound on one view's super-tiles (at most the
// above), which sizes the shared-memory tables of the placement.
BinGeom coarse_geom(int64_t n, int64_t total_tiles, int64_t n_views, int tile, int max_vt, const int64_t *coff,
                    int max_super = 0) {
    BinGeom g;
    g.n = n;
    g.chunk = bin_chunk(n, 608);
    g.n_c = ceil_div(n > 0 ? n : 1, g.chunk);
    g.n_g = ceil_div(g.n_c, (int64_t)BIN_GROUP);
    g.tiles = total_tiles / 4 + n_views;
    g.tile = tile;
    g.max_vt = max_vt / 4 + 1;
    if (max_super > 0 && max_super < g.max_vt) g.max_vt = max_super;
    g.sup = SUP;
    g.coff = coff;
    return g;
}

int64_t fine_items_cap(int64_t pair_capacity, int64_t coarse_tiles) {
    return ceil_div(pair_capacity, (int64_t)WI) + coarse_tiles;
}

struct BinWorkspace {
    uint32_t *dk[2], *dv[2];   // depth (then view) keys / entry ids, ping-pong, [V*N]
    uint32_t *dvf;             // super-tile form: entry ids in depth order from the last radix pass, [V*N]
    uint32_t *counts;          // [RADIX * RS_MAX_BLOCKS] + [RADIX] digit totals
    uint32_t *G1;              // [n_g * total_tiles] group sums of the tile counts
    uint32_t *tile_total;      // [total_tiles]
    uint32_t *tile_start;      // [total_tiles]
    ushort4 *srect;            // [V*N] clipped rectangles in depth order
    int64_t *sort_count;       // [1]
    // the super-tile grid (coarse)
    int64_t *coff;             // [V + 1] first super-tile of each view
    uint32_t *Mc;              // [n_c' * Tc] chunk x super-tile counts, then first slots
    uint32_t *G1c;             // [n_g' * Tc]
    uint32_t *ctotal, *cstart; // [Tc]
    uint16_t *cmask;           // [pair_capacity] covered-tile masks by super-tile, in depth order
    uint32_t *cgid;            // [pair_capacity] their Gaussian indices
    int64_t *c_count;          // [2] super-tile pair count, its sort count
    // placement work items
    uint32_t *seg_base;        // [Tc + 1]
    uint32_t *item_ct;         // [items]
    uint32_t *run_of;          // [items * SUP_T] counts, then first slots
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// coarse_only: the super-tile form (gs_bin_sort_coarse), whose lists live in
// the caller's buffers and which has no placement pass.
size_t bin_ws_layout(int64_t n, int64_t n_views, int64_t total_tiles, int64_t pair_capacity, BinWorkspace *w,
                     char *base, bool coarse_only = false) {
    const int64_t total = n * n_views;
    const BinGeom g = bin_geom(n, total_tiles, 16, 0);
    const BinGeom gc = coarse_geom(n, total_tiles, n_views, 16, 0, nullptr);
    if (coarse_only) pair_capacity = 0;
    const int64_t items = coarse_only ? 0 : fine_items_cap(pair_capacity, gc.tiles);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += align256(bytes > 0 ? bytes : 1);
        return p;
    };
    for (int i = 0; i < 2; ++i) {
        char *a = take(sizeof(uint32_t) * (size_t)(total > 0 ? total : 1));
        char *b = take(sizeof(uint32_t) * (size_t)(total > 0 ? total : 1));
        if (w) { w->dk[i] = (uint32_t *)a; w->dv[i] = (uint32_t *)b; }
    }
    char *dvf = coarse_only ? take(sizeof(uint32_t) * (size_t)(total > 0 ? total : 1)) : nullptr;
    char *counts = take(sizeof(uint32_t) * RADIX * (RS_MAX_BLOCKS + 1) + 2 * sizeof(uint32_t));
    char *G1 = take(sizeof(uint32_t) * (size_t)(g.n_g * total_tiles));
    char *tt = take(sizeof(uint32_t) * (size_t)total_tiles);
    char *ts = take(sizeof(uint32_t) * (size_t)total_tiles);
    char *sr = take(sizeof(ushort4) * (size_t)(total > 0 ? total : 1));
    char *sc = take(sizeof(int64_t));
    char *coff = take(sizeof(int64_t) * (size_t)(n_views + 1));
    char *Mc = take(sizeof(uint32_t) * (size_t)(gc.n_c * gc.tiles));
    char *G1c = take(sizeof(uint32_t) * (size_t)(gc.n_g * gc.tiles));
    char *ct = take(sizeof(uint32_t) * (size_t)gc.tiles);
    char *cs = take(sizeof(uint32_t) * (size_t)gc.tiles);
    char *cl = take(sizeof(uint16_t) * (size_t)pair_capacity);
    char *cg = take(sizeof(uint32_t) * (size_t)pair_capacity);
    char *cc = take(sizeof(int64_t) * 2);
    char *sb = take(sizeof(uint32_t) * (size_t)(gc.tiles + 1));
    char *ic = take(sizeof(uint32_t) * (size_t)items);
    char *ro = take(sizeof(uint32_t) * (size_t)items * SUP_T);
    if (w) {
        w->dvf = (uint32_t *)dvf;
        w->counts = (uint32_t *)counts;
        w->G1 = (uint32_t *)G1;
        w->tile_total = (uint32_t *)tt;
        w->tile_start = (uint32_t *)ts;
        w->srect = (ushort4 *)sr;
        w->sort_count = (int64_t *)sc;
        w->coff = (int64_t *)coff;
        w->Mc = (uint32_t *)Mc;
        w->G1c = (uint32_t *)G1c;
        w->ctotal = (uint32_t *)ct;
        w->cstart = (uint32_t *)cs;
        w->cmask = (uint16_t *)cl;
        w->cgid = (uint32_t *)cg;
        w->c_count = (int64_t *)cc;
        w->seg_base = (uint32_t *)sb;
        w->item_ct = (uint32_t *)ic;
        w->run_of = (uint32_t *)ro;
    }
    return off;
}

// The super-tile form's tile totals: TT_SPLIT blocks per super-tile count,
// per tile of it, the list entries whose mask has the tile's bit (the pairs
// the tile lists would hold), each over a contiguous part of the list read
// eight masks at a time, and add them to tile_total (zero at launch).  A view
// whose tile grid is larger than the tables hold gets GS_ERR_INVALID_ARG and
// no pairs, as on the tile grid; nothing is counted when the lists did not
// fit.  The masks are 16-byte aligned.
constexpr int TT_THREADS = 256;
constexpr int TT_SPLIT = 8;
__global__ void __launch_bounds__(TT_THREADS) coarse_tile_totals(
    const gs_camera *__restrict__ cams, int n_views, BinGeom gc, int64_t fine_tiles, int fine_max_vt,
    const uint32_t *__restrict__ cstart, const uint32_t *__restrict__ ctotal, const uint16_t *__restrict__ cmask,
    const int64_t *coarse_sort_count, uint32_t *__restrict__ tile_total, int32_t *dev_status) {
    __shared__ uint32_t s_c[TT_THREADS / 32][SUP_T];
    const int64_t ct = blockIdx.x / TT_SPLIT;
    const int part = (int)(blockIdx.x % TT_SPLIT);
    if (ct >= gc.coff[n_views]) return;  // whole block
    const int v = view_of_grid_tile(gc, cams, n_views, ct);
    const ViewTiles ft = view_tiles(cams[v], gc.tile);
    if (!view_fits(ft, fine_tiles, fine_max_vt)) {
        if (threadIdx.x == 0 && part == 0) set_status(dev_status, GS_ERR_INVALID_ARG);
        return;
    }
    if (*coarse_sort_count == 0) return;
    const uint32_t len = ctotal[ct];
    const uint32_t lo = cstart[ct] + (uint32_t)(((uint64_t)len * part) / TT_SPLIT);
    const uint32_t hi = cstart[ct] + (uint32_t)(((uint64_t)len * (part + 1)) / TT_SPLIT);
    uint32_t c[SUP_T];
#pragma unroll
    for (int k = 0; k < SUP_T; ++k) c[k] = 0;
    for (uint32_t p = (lo & ~7u) + 8u * threadIdx.x; p < hi; p += 8u * TT_THREADS) {
        uint32_t w[4];
        if (p + 8 <= hi) {
            const uint4 x = *reinterpret_cast<const uint4 *>(cmask + p);
            w[0] = x.x;
            w[1] = x.y;
            w[2] = x.z;
            w[3] = x.w;
        } else {  // the part's last vector: plain loads inside it
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t a = p + 2 * e < hi ? cmask[p + 2 * e] : 0u;
                const uint32_t b = p + 2 * e + 1 < hi ? cmask[p + 2 * e + 1] : 0u;
                w[e] = a | (b << 16);
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {  // masks before lo (the aligned head) are not this part's
            if (p + 2 * e < lo) w[e] &= 0xffff0000u;
            if (p + 2 * e + 1 < lo) w[e] &= 0x0000ffffu;
        }
        // four-bit counters: nibble n of acc[j] counts bit 4 (n % 4) + j of
        // the masks (each word holds two), at most 4 per nibble here
        uint32_t acc[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] += (w[e] >> j) & 0x11111111u;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int nb = 0; nb < 8; ++nb) c[4 * (nb % 4) + j] += (acc[j] >> (4 * nb)) & 15u;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < SUP_T; ++k) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) c[k] += __shfl_xor_sync(0xffffffffu, c[k], off);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < SUP_T; ++k) s_c[warp][k] = c[k];
    }
    __syncthreads();
    if (threadIdx.x < SUP_T) {
        const int k = threadIdx.x;
        const int ctx = (ft.tx + SUP - 1) / SUP;
        const int64_t lct = ct - gc.coff[v];
        const int x = (int)(lct % ctx) * SUP + k % SUP, y = (int)(lct / ctx) * SUP + k / SUP;
        uint32_t t = 0;
#pragma unroll
        for (int w = 0; w < TT_THREADS / 32; ++w) t += s_c[w][k];
        if (x < ft.tx && y < ft.ty && t) atomicAdd(&tile_total[ft.off + (int64_t)y * ft.tx + x], t);
    }
}

// The super-tile form's tile ranges: where each tile's pairs would lie in
// gs_bin_sort's vals (the checkpoint slots and the tile order use them).
// Written only when both the pairs and the super-tile lists fit.
__global__ void tile_ranges(int64_t tiles, const uint32_t *__restrict__ tile_start,
                            const uint32_t *__restrict__ tile_total, const int64_t *sort_count,
                            const int64_t *coarse_sort_count, uint2 *__restrict__ ranges) {
    if (*sort_count == 0 || *coarse_sort_count == 0) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tiles) return;
    const uint32_t tot = tile_total[t];
    ranges[t] = tot ? make_uint2(tile_start[t], tile_start[t] + tot) : make_uint2(0u, 0u);
}

// Tables of up to this many tiles per view fit the shared memory of the
// counting and scatter kernels (the scatter holds two 4-byte tables).
constexpr int kMaxViewTiles = 20480;

// Raise the dynamic shared-memory limit of the table kernels to the largest
// table, once per device (before any stream capture, on the first call).
gs_status bin_smem_attributes() {
    static bool done[kMaxDevices] = {};
    const int dev = cached_device_index();
    if (dev < 0) return GS_ERR_UNSUPPORTED;
    if (done[dev]) return GS_OK;
    const int bytes = (int)(sizeof(uint32_t) * kMaxViewTiles);
    GS_TRY(cudaFuncSetAttribute(bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * bytes + 8));
    // the super-tile placement: its warps' tables within 200 KB (coarse_place_warps)
    GS_TRY(cudaFuncSetAttribute(coarse_place, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(200 * 1024)));
    done[dev] = true;
    return GS_OK;
}

}  // namespace

extern "C" {

size_t gs_bin_sort_workspace_size(int64_t n, int32_t n_views, int64_t pair_capacity, int64_t total_tiles) {
    if (n < 0 || n_views <= 0 || pair_capacity < 0 || total_tiles <= 0) return 0;
    return bin_ws_layout(n, n_views, total_tiles, pair_capacity, nullptr, nullptr);
}

}  // extern "C"

namespace {

// gs_bin_sort (coarse == nullptr) and gs_bin_sort_coarse (the super-tile
// lists into the caller's buffers, without the placement of the pairs).
gs_status bin_sort_impl(const gs_projected *proj, const gs_camera *cams, int32_t n_views, int64_t n,
                        int64_t total_tiles, int32_t max_view_tiles, int32_t max_super, const gs_raster_config *cfg,
                        void *workspace,
                        size_t workspace_bytes, uint64_t *keys, uint32_t *vals, const gs_coarse_lists *coarse,
                        int64_t pair_capacity, uint32_t *ranges, int64_t *dev_pair_count, int32_t *dev_status,
                        cudaStream_t stream) {
    if (!proj || !cams || !cfg || n_views <= 0 || n < 0 || total_tiles <= 0 || !ranges || !dev_pair_count)
        return GS_ERR_INVALID_ARG;
    if (!coarse && !vals) return GS_ERR_INVALID_ARG;
    if (max_super < 0) return GS_ERR_INVALID_ARG;
    if (coarse && (!coarse->gid || !coarse->mask || !coarse->start || !coarse->count || !coarse->view_first ||
                   !coarse->total || coarse->capacity < 0 || coarse->capacity > ((int64_t)1 << 32) - 65536 ||
                   ((uintptr_t)coarse->mask & 15)))
        return GS_ERR_INVALID_ARG;
    if (cfg->tile != 8 && cfg->tile != 16 && cfg->tile != 32) return GS_ERR_INVALID_ARG;
    if (pair_capacity < 0 || pair_capacity >= ((int64_t)1 << 32) - 1) return GS_ERR_INVALID_ARG;
    if (total_tiles >= ((int64_t)1 << 31)) return GS_ERR_INVALID_ARG;
    const int64_t mvt = max_view_tiles > 0 ? max_view_tiles : total_tiles;
    if (mvt > total_tiles || mvt > kMaxViewTiles) return GS_ERR_UNSUPPORTED;
    const int64_t total = n * n_views;
    if (total >= ((int64_t)1 << 32) - 1) return GS_ERR_INVALID_ARG;
    if (total > 0 && (!proj->rec || !proj->rect || !proj->tiles_touched)) return GS_ERR_INVALID_ARG;
    const bool co = coarse != nullptr;
    if (!workspace ||
        workspace_bytes < bin_ws_layout(n, n_views, total_tiles, pair_capacity, nullptr, nullptr, co))
        return GS_ERR_WORKSPACE;
    if ((uintptr_t)workspace & 255) return GS_ERR_WORKSPACE;
    BinWorkspace w;
    bin_ws_layout(n, n_views, total_tiles, pair_capacity, &w, (char *)workspace, co);
    int64_t coarse_capacity = pair_capacity;  // at most one super-tile entry per pair
    int64_t *coarse_total = w.c_count;
    if (co) {  // the lists go to the caller's buffers
        w.cgid = coarse->gid;
        w.cmask = coarse->mask;
        w.cstart = coarse->start;
        w.ctotal = coarse->count;
        w.coff = coarse->view_first;
        coarse_capacity = coarse->capacity;
        coarse_total = coarse->total;
    }

    GS_TRY(cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)total_tiles, stream));
    if (total == 0) {
        GS_TRY(cudaMemsetAsync(dev_pair_count, 0, sizeof(int64_t), stream));
        if (co) {
            GS_TRY(cudaMemsetAsync(coarse->total, 0, sizeof(int64_t), stream));
            const BinGeom gc0 = coarse_geom(n, total_tiles, n_views, cfg->tile, (int)mvt, nullptr);
            GS_TRY(cudaMemsetAsync(coarse->count, 0, sizeof(uint32_t) * (size_t)gc0.tiles, stream));
            coarse_offsets<<<1, 32, 0, stream>>>(cams, n_views, cfg->tile, coarse->view_first);
            GS_TRY_LAUNCH();
        }
        return GS_OK;
    }
    const BinGeom g = bin_geom(n, total_tiles, cfg->tile, (int)mvt);
    // 1. depth order of all (view, Gaussian) entries, then grouped by view
    int sel;
    uint32_t *krange = w.counts + (size_t)RADIX * (RS_MAX_BLOCKS + 1);
    GS_TRY(cudaMemsetAsync(krange, 0xff, sizeof(uint32_t), stream));
    GS_TRY(cudaMemsetAsync(krange + 1, 0, sizeof(uint32_t), stream));
    const unsigned kr_blocks = (unsigned)min((int64_t)device_sm_count() * 4, ceil_div(total, (int64_t)256));
    // one view in the super-tile form: the last radix pass writes the depth
    // order to dvf with the packed rectangles beside it (no bin_rects16)
    const bool fused = co && n_views == 1 && proj->depth_key && proj->rect16 && w.dvf;
    if (proj->depth_key) {  // written by gs_project
        key_range_kernel<<<kr_blocks, 256, 0, stream>>>(proj->depth_key, total, krange);
        GS_TRY_LAUNCH();
        RsFinal fin{};
        if (fused)
            fin = RsFinal{w.dvf, reinterpret_cast<const ushort4 *>(proj->rect16), w.srect, cams, g.tile, g.max_vt,
                          g.tiles};
        sel = radix_sort(w.dk[0], w.dv[0], w.dk[1], w.dv[1], nullptr, total, 32, w.counts, stream, proj->depth_key,
                         krange, fin);
    } else {
        depth_keys_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, stream>>>(proj->rec, proj->tiles_touched, total,
                                                                             w.dk[0], w.dv[0]);
        GS_TRY_LAUNCH();
        key_range_kernel<<<kr_blocks, 256, 0, stream>>>(w.dk[0], total, krange);
        GS_TRY_LAUNCH();
        sel = radix_sort(w.dk[0], w.dv[0], w.dk[1], w.dv[1], nullptr, total, 32, w.counts, stream, nullptr, krange);
    }
    GS_TRY_LAUNCH();
    if (n_views > 1) {
        view_keys_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, stream>>>(w.dv[sel], total, n, w.dk[sel]);
        GS_TRY_LAUNCH();
        sel ^= radix_sort(w.dk[sel], w.dv[sel], w.dk[sel ^ 1], w.dv[sel ^ 1], nullptr, total, bits_for(n_views),
                          w.counts, stream);
        GS_TRY_LAUNCH();
    }
    const uint32_t *order = fused ? w.dvf : w.dv[sel];
    const int4 *rect = reinterpret_cast<const int4 *>(proj->rect);
    // 2. the pairs by tile, in depth order: tile totals and starts (chunked
    // counts on the tile grid), then the entries by super-tile (the chunked
    // counting sort on the super-tile grid), then each super-tile's tiles
    // filled from its depth-ordered entry list
    const size_t smem = sizeof(uint32_t) * (size_t)mvt;
    {
        const gs_status st = bin_smem_attributes();
        if (st != GS_OK) return st;
    }
    if (!fused) {  // (fused: the rectangles came with the depth order)
        if (proj->rect16)  // written by gs_project
            bin_rects16<<<(unsigned)ceil_div(total, 256), 256, 0, stream>>>(
                reinterpret_cast<const ushort4 *>(proj->rect16), order, cams, g, total, w.srect);
        else
            bin_rects<<<(unsigned)ceil_div(total, 256), 256, 0, stream>>>(rect, proj->tiles_touched, order, cams, g,
                                                                         total, w.srect);
        GS_TRY_LAUNCH();
    }
    if (co) {  // the tile totals come from the lists' masks, after the scatter
        GS_TRY(cudaMemsetAsync(w.tile_total, 0, sizeof(uint32_t) * (size_t)total_tiles, stream));
    } else {
        GS_TRY(cudaMemsetAsync(w.G1, 0, sizeof(uint32_t) * (size_t)(g.n_g * total_tiles), stream));
        const unsigned n_chunks = (unsigned)(g.n_c * n_views);
        bin_count<<<n_chunks, COUNT_THREADS, 2 * smem + 8, stream>>>(w.srect, cams, g, nullptr, w.G1, dev_status);
        GS_TRY_LAUNCH();
        bin_groups<<<(unsigned)ceil_div(total_tiles, (int64_t)256), 256, 0, stream>>>(g, w.G1, w.tile_total);
        GS_TRY_LAUNCH();
        bin_starts<<<1, SCAN_THREADS, 0, stream>>>(g, w.tile_total, w.tile_start, pair_capacity, dev_pair_count,
                                                   w.sort_count, dev_status);
        GS_TRY_LAUNCH();
    }
    // the super-tile grid
    coarse_offsets<<<1, 32, 0, stream>>>(cams, n_views, cfg->tile, w.coff);
    GS_TRY_LAUNCH();
    const BinGeom gc = coarse_geom(n, total_tiles, n_views, cfg->tile, (int)mvt, w.coff, max_super);
    const size_t csmem = sizeof(uint32_t) * (size_t)gc.max_vt;
    GS_TRY(cudaMemsetAsync(w.G1c, 0, sizeof(uint32_t) * (size_t)(gc.n_g * gc.tiles), stream));
    const unsigned n_cchunks = (unsigned)(gc.n_c * n_views);
    bin_count<<<n_cchunks, COUNT_THREADS, 2 * csmem + 8, stream>>>(w.srect, cams, gc, w.Mc, w.G1c, dev_status);
    GS_TRY_LAUNCH();
    bin_groups<<<(unsigned)ceil_div(gc.tiles, (int64_t)256), 256, 0, stream>>>(gc, w.G1c, w.ctotal);
    GS_TRY_LAUNCH();
    // at most as many entry x super-tile pairs as pairs: within the capacity
    // whenever the pairs are
    bin_starts<<<1, SCAN_THREADS, 0, stream>>>(gc, w.ctotal, w.cstart, coarse_capacity, coarse_total,
                                               w.c_count + 1, dev_status);
    GS_TRY_LAUNCH();
    bin_offsets<<<(unsigned)ceil_div(gc.n_g * gc.tiles, (int64_t)256), 256, 0, stream>>>(
        gc, cams, n_views, w.G1c, w.cstart, w.ctotal, w.c_count + 1, w.Mc, nullptr);
    GS_TRY_LAUNCH();
    {
        const int cw = coarse_place_warps(gc.max_vt);
        const size_t cp_smem = (size_t)2 * cw * gc.max_vt * sizeof(uint32_t);
        coarse_place<<<n_cchunks, cw * 32, cp_smem, stream>>>(w.srect, order, cams, gc, w.Mc, w.c_count + 1, w.cgid,
                                                             w.cmask);
    }
    GS_TRY_LAUNCH();
    if (co) {
        coarse_tile_totals<<<(unsigned)(gc.tiles * TT_SPLIT), TT_THREADS, 0, stream>>>(cams, n_views, gc, total_tiles, (int)mvt,
                                                                           w.cstart, w.ctotal, w.cmask,
                                                                           w.c_count + 1, w.tile_total, dev_status);
        GS_TRY_LAUNCH();
        bin_starts<<<1, SCAN_THREADS, 0, stream>>>(g, w.tile_total, w.tile_start, pair_capacity, dev_pair_count,
                                                   w.sort_count, dev_status);
        GS_TRY_LAUNCH();
        tile_ranges<<<(unsigned)ceil_div(total_tiles, (int64_t)256), 256, 0, stream>>>(
            total_tiles, w.tile_start, w.tile_total, w.sort_count, w.c_count + 1, reinterpret_cast<uint2 *>(ranges));
        GS_TRY_LAUNCH();
        return GS_OK;
    }
    // placement work items (segments of the super-tiles' lists)
    seg_layout<<<1, SCAN_THREADS, 0, stream>>>(gc.tiles, w.ctotal, w.sort_count, w.seg_base);
    GS_TRY_LAUNCH();
    seg_fill<<<(unsigned)ceil_div(gc.tiles, (int64_t)256), 256, 0, stream>>>(gc.tiles, w.seg_base, w.item_ct);
    GS_TRY_LAUNCH();
    const int64_t items_cap = fine_items_cap(pair_capacity, gc.tiles);
    const int64_t resident = (int64_t)device_sm_count() * 8;  // blocks of 8 warps
    const int64_t want = ceil_div(items_cap, (int64_t)(FP_THREADS / 32));
    const unsigned fp_blocks = (unsigned)(want < resident ? (want > 0 ? want : 1) : resident);
    fine_pass<false><<<fp_blocks, FP_THREADS, 0, stream>>>(w.cmask, w.cgid, cams, n_views, gc, w.cstart, w.ctotal,
                                                           w.seg_base, w.item_ct, w.run_of, vals, total_tiles,
                                                           (int)mvt, pair_capacity);
    GS_TRY_LAUNCH();
    fine_prefix<<<(unsigned)ceil_div(gc.tiles * 32, (int64_t)256), 256, 0, stream>>>(
        cams, n_views, gc, total_tiles, (int)mvt, w.tile_start, w.tile_total, w.seg_base, w.sort_count, w.run_of,
        reinterpret_cast<uint2 *>(ranges));
    GS_TRY_LAUNCH();
    fine_pass<true><<<fp_blocks, FP_THREADS, 0, stream>>>(w.cmask, w.cgid, cams, n_views, gc, w.cstart, w.ctotal,
                                                          w.seg_base, w.item_ct, w.run_of, vals, total_tiles,
                                                          (int)mvt, pair_capacity);
    GS_TRY_LAUNCH();
    if (keys) {
        keys64_kernel<<<(unsigned)total_tiles, 128, 0, stream>>>(reinterpret_cast<const uint2 *>(ranges), vals,
                                                                 w.sort_count, cams, n_views, n, proj->rec, keys);
        GS_TRY_LAUNCH();
    }
    return GS_OK;
}

}  // namespace

extern "C" {

gs_status gs_bin_sort(const gs_projected *proj, const gs_camera *cams, int32_t n_views, int64_t n,
                      int64_t total_tiles, int32_t max_view_tiles, const gs_raster_config *cfg, void *workspace,
                      size_t workspace_bytes, uint64_t *keys, uint32_t *vals, int64_t pair_capacity,
                      uint32_t *ranges, int64_t *dev_pair_count, int32_t *dev_status, cudaStream_t stream) {
    if (!vals) return GS_ERR_INVALID_ARG;
    return bin_sort_impl(proj, cams, n_views, n, total_tiles, max_view_tiles, 0, cfg, workspace, workspace_bytes,
                         keys, vals, nullptr, pair_capacity, ranges, dev_pair_count, dev_status, stream);
}

size_t gs_bin_sort_coarse_workspace_size(int64_t n, int32_t n_views, int64_t total_tiles) {
    if (n < 0 || n_views <= 0 || total_tiles <= 0) return 0;
    return bin_ws_layout(n, n_views, total_tiles, 0, nullptr, nullptr, true);
}

gs_status gs_bin_sort_coarse(const gs_projected *proj, const gs_camera *cams, int32_t n_views, int64_t n,
                             int64_t total_tiles, int32_t max_view_tiles, int32_t max_view_super_tiles,
                             const gs_raster_config *cfg, void *workspace, size_t workspace_bytes,
                             const gs_coarse_lists *lists, int64_t pair_capacity, uint32_t *ranges,
                             int64_t *dev_pair_count, int32_t *dev_status, cudaStream_t stream) {
    if (!lists) return GS_ERR_INVALID_ARG;
    return bin_sort_impl(proj, cams, n_views, n, total_tiles, max_view_tiles, max_view_super_tiles, cfg, workspace,
                         workspace_bytes, nullptr, nullptr, lists, pair_capacity, ranges, dev_pair_count, dev_status,
                         stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// gs_bin_sort_noalloc: gs_bin_sort with its scratch in a fixed device array.
//
// For callers that cannot allocate device memory: code that issues its work
// while a CUDA graph is being captured (cudaMalloc cannot be captured),
// plugins whose host application owns all device memory through its own
// pool, and real-time loops that must not block on the allocator.  The
// caller still owns and passes every input and output; only the scratch
// comes from here.
namespace {

constexpr int64_t kNoAllocMaxEntries = (int64_t)1 << 18;  // n * n_views
constexpr size_t kNoAllocBytes = (size_t)16 << 20;        // the whole scratch

// One copy per device that loads the library, held until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

void *g_noalloc_ptr[kMaxDevices] = {};

}  // namespace

extern "C" gs_status gs_bin_sort_noalloc(const gs_projected *proj, const gs_camera *cams, int32_t n_views, int64_t n,
                                         int64_t total_tiles, int32_t max_view_tiles, const gs_raster_config *cfg,
                                         uint64_t *keys, uint32_t *vals, int64_t pair_capacity, uint32_t *ranges,
                                         int64_t *dev_pair_count, int32_t *dev_status, cudaStream_t stream) {
    if (n < 0 || n_views <= 0 || pair_capacity < 0 || total_tiles <= 0) return GS_ERR_INVALID_ARG;
    if (n * n_views > kNoAllocMaxEntries) return GS_ERR_WORKSPACE;
    if (total_tiles >= ((int64_t)1 << 31)) return GS_ERR_INVALID_ARG;
    if (bin_ws_layout(n, n_views, total_tiles, pair_capacity, nullptr, nullptr) > kNoAllocBytes)
        return GS_ERR_WORKSPACE;
    const int dev = cached_device_index();
    if (dev < 0) return GS_ERR_UNSUPPORTED;
    // Host code cannot use the array's name as a device address: look the
    // address up with the device current.  Outside stream capture it is looked
    // up on every call (so a context torn down and recreated, e.g. after
    // cudaDeviceReset, gets the new address); during capture the address of
    // the last call outside capture on this device is used.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    GS_TRY(cudaStreamIsCapturing(stream, &cap));
    if (cap == cudaStreamCaptureStatusNone || !g_noalloc_ptr[dev]) {
        void *p = nullptr;
        GS_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    return gs_bin_sort(proj, cams, n_views, n, total_tiles, max_view_tiles, cfg, g_noalloc_ptr[dev], kNoAllocBytes,
                       keys, vals, pair_capacity, ranges, dev_pair_count, dev_status, stream);
}
