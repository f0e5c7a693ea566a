// gs_bin_sort: tile binning and depth order ("depth-sorted Gaussians
// overlapping a given pixel", Sec. 3).
//
// The required order is the stable sort of the 64-bit keys
// (global tile id << 32 | float32 depth bits) in emission order (Gaussian
// index ascending, tiles row-major).  It is produced in two stages that give
// the same permutation with far less traffic than sorting 64-bit pair keys:
//   1. sort the V*N (view, Gaussian) entries by depth bits (stable, so equal
//      depths keep ascending index);
//   2. emit each entry's pairs in that order and stably sort the pairs by
//      tile id alone (ceil(log2(tiles)) bits, 8 per pass).
// A stable sort by tile of a depth-ordered list is ordered by
// (tile, depth, index), i.e. exactly the 64-bit key order.
//
// Every kernel reads the pair count from device memory, so the whole call
// can be captured in a CUDA graph.  The radix sort is a reduce-then-scan LSD
// sort: an upsweep histogram per block, one exclusive scan over the
// digit-major (digit, block) counts, and a downsweep that ranks each tile of
// 2048 keys with warp ballots (one per digit bit), reorders the tile by digit in shared
// memory and writes each digit's run contiguously.
#include "common.cuh"

using namespace gsr;

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int RS_MAX_BLOCKS = 608;  // 4 x 152 SMs
constexpr int SCAN_THREADS = 1024;
static_assert(RS_THREADS == RADIX, "the downsweep gives each thread one digit");

static_assert(RS_MAX_BLOCKS <= 4 * RS_THREADS, "rs_scan holds at most four counts per thread");

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

__global__ void __launch_bounds__(RS_THREADS) rs_upsweep(const uint32_t *__restrict__ keys, const int64_t *d_count,
                                                         int64_t cap, int shift, uint32_t mask,
                                                         uint32_t *__restrict__ counts) {
    __shared__ uint32_t hist[RADIX];
    for (int i = threadIdx.x; i < RADIX; i += RS_THREADS) hist[i] = 0;
    __syncthreads();
    const int64_t count = effective_count(d_count, cap);
    int64_t begin, end;
    block_range(count, gridDim.x, blockIdx.x, begin, end);
    for (int64_t i = begin + threadIdx.x; i < end; i += RS_THREADS) atomicAdd(&hist[(keys[i] >> shift) & mask], 1u);
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
__global__ void __launch_bounds__(RS_THREADS) rs_scan(uint32_t *a, int G, uint32_t *totals) {
    __shared__ uint32_t warp_sums[32];
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

__global__ void __launch_bounds__(RS_THREADS) rs_downsweep(const uint32_t *__restrict__ keys_in,
                                                           const uint32_t *__restrict__ vals_in,
                                                           uint32_t *__restrict__ keys_out,
                                                           uint32_t *__restrict__ vals_out, const int64_t *d_count,
                                                           int64_t cap, int shift, uint32_t mask,
                                                           const uint32_t *__restrict__ offsets,
                                                           const uint32_t *__restrict__ totals) {
    __shared__ uint32_t s_run[RADIX];   // global start of this block's next run per digit
    __shared__ uint32_t s_tot[RADIX];   // tile count per digit
    __shared__ uint32_t s_loc[RADIX];   // tile-local start per digit
    __shared__ uint32_t s_wcnt[RS_WARPS][RADIX];
    __shared__ uint32_t s_k[RS_TILE];
    __shared__ uint32_t s_v[RS_TILE];
    __shared__ uint32_t s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
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
        for (int r = 0; r < RS_ITEMS; ++r) {
            const int li = warp * 32 * RS_ITEMS + r * 32 + lane;
            const bool valid = li < n_tile;
            k[r] = valid ? keys_in[base + li] : 0u;
            v[r] = valid ? vals_in[base + li] : 0u;
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
            keys_out[pos] = key;
            vals_out[pos] = s_v[i];
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
int radix_sort(uint32_t *ka, uint32_t *va, uint32_t *kb, uint32_t *vb, const int64_t *d_count, int64_t cap,
               int bits, uint32_t *counts, cudaStream_t stream) {
    const int G = rs_blocks(cap);
    int cur = 0;
    for (int shift = 0; shift < bits; shift += RADIX_BITS) {
        const int nb = bits - shift < RADIX_BITS ? bits - shift : RADIX_BITS;
        const uint32_t mask = (1u << nb) - 1u;
        uint32_t *ki = cur ? kb : ka, *vi = cur ? vb : va, *ko = cur ? ka : kb, *vo = cur ? va : vb;
        uint32_t *totals = counts + (size_t)RADIX * RS_MAX_BLOCKS;
        rs_upsweep<<<G, RS_THREADS, 0, stream>>>(ki, d_count, cap, shift, mask, counts);
        rs_scan<<<RADIX, RS_THREADS, 0, stream>>>(counts, G, totals);
        rs_downsweep<<<G, RS_THREADS, 0, stream>>>(ki, vi, ko, vo, d_count, cap, shift, mask, counts, totals);
        cur ^= 1;
    }
    return cur;
}

int radix_passes(int bits) { return (bits + RADIX_BITS - 1) / RADIX_BITS; }

// depth keys: float32 bits of the depth (positive, so the bit patterns order
// like the values); culled entries sort last and emit nothing.
__global__ void depth_keys_kernel(const float *__restrict__ rec, const int32_t *__restrict__ touched, int64_t total,
                                  uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    keys[e] = touched[e] > 0 ? __float_as_uint(rec[e * kRecFloats + 9]) : 0xffffffffu;
    vals[e] = (uint32_t)e;
}

// Scan of the tile counts in depth order, reduce phase: one block per chunk of
// RS_THREADS entries writes the chunk's pair count.
__global__ void __launch_bounds__(RS_THREADS) count_reduce(const int32_t *__restrict__ touched,
                                                           const uint32_t *__restrict__ order, int64_t total,
                                                           unsigned long long *__restrict__ chunk_sums) {
    const int64_t m = (int64_t)blockIdx.x * RS_THREADS + threadIdx.x;
    unsigned long long s = m < total ? (unsigned)touched[order[m]] : 0u;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __shared__ unsigned long long ws[RS_WARPS];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < RS_WARPS; ++w) t += ws[w];
        chunk_sums[blockIdx.x] = t;
    }
}

// Exclusive scan of the chunk sums by one block (SCAN_THREADS values per
// round); writes the total pair count and the count the pair sort will use
// (0 when over capacity).
__global__ void __launch_bounds__(SCAN_THREADS) count_top(unsigned long long *chunk_sums, int64_t n_chunks, int64_t cap,
                                                          int64_t *dev_pair_count, int64_t *sort_count,
                                                          int32_t *dev_status) {
    __shared__ unsigned long long s[SCAN_THREADS];
    unsigned long long carry = 0;
    for (int64_t base = 0; base < n_chunks; base += SCAN_THREADS) {
        const int64_t i = base + threadIdx.x;
        const unsigned long long x = i < n_chunks ? chunk_sums[i] : 0ull;
        s[threadIdx.x] = x;
        __syncthreads();
        for (int off = 1; off < SCAN_THREADS; off <<= 1) {
            const unsigned long long y = threadIdx.x >= off ? s[threadIdx.x - off] : 0ull;
            __syncthreads();
            s[threadIdx.x] += y;
            __syncthreads();
        }
        if (i < n_chunks) chunk_sums[i] = carry + s[threadIdx.x] - x;
        carry += s[SCAN_THREADS - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *dev_pair_count = (int64_t)carry;
        if ((int64_t)carry > cap) {
            set_status(dev_status, GS_ERR_CAPACITY);
            *sort_count = 0;
        } else {
            *sort_count = (int64_t)carry;
        }
    }
}

// Scan phase fused with pair emission.  Each block takes its range of
// entries in depth order, RS_THREADS at a time: a block scan gives every
// entry's first pair slot; each entry writes its own pairs (tiles of its
// rectangle, row-major) into a shared staging buffer, which the block then
// copies out contiguously.  A chunk with more pairs than the buffer holds
// writes straight to global memory instead.
constexpr int EMIT_STAGE = 4096;

__global__ void __launch_bounds__(RS_THREADS) emit_pairs(const int32_t *__restrict__ touched,
                                                         const int4 *__restrict__ rect,
                                                         const uint32_t *__restrict__ order, int64_t total,
                                                         int64_t n, const gs_camera *__restrict__ cams, int tile,
                                                         const unsigned long long *__restrict__ block_offsets,
                                                         const int64_t *sort_count, uint32_t *__restrict__ pkeys,
                                                         uint32_t *__restrict__ pvals) {
    if (*sort_count == 0) return;  // nothing to emit, or over capacity
    __shared__ uint32_t s_k[EMIT_STAGE];
    __shared__ uint32_t s_v[EMIT_STAGE];
    __shared__ uint32_t s_warp[32];
    const int64_t end = total;
    uint64_t run = block_offsets[blockIdx.x];
    {
        const int64_t m = (int64_t)blockIdx.x * RS_THREADS + threadIdx.x;
        uint32_t c = 0, gi = 0;
        int4 r = make_int4(0, 0, -1, -1);
        int base = 0, tx_n = 0;
        if (m < end) {
            const uint32_t e = order[m];
            c = (uint32_t)touched[e];
            if (c > 0) {
                const int64_t v = (int64_t)e / n;
                r = rect[e];
                const gs_camera &cam = cams[v];
                tx_n = (cam.width + tile - 1) / tile;
                base = cam.tile_offset;
                gi = (uint32_t)((int64_t)e - v * n);
            }
        }
        uint32_t chunk_total;
        const uint32_t excl = block_exclusive_scan(c, s_warp, &chunk_total);
        if (chunk_total <= EMIT_STAGE) {
            uint32_t o = excl;
            for (int ty = r.y; ty <= r.w; ++ty)
                for (int tx = r.x; tx <= r.z; ++tx, ++o) {
                    s_k[o] = (uint32_t)(base + ty * tx_n + tx);
                    s_v[o] = gi;
                }
            __syncthreads();
            for (uint32_t k = threadIdx.x; k < chunk_total; k += RS_THREADS) {
                pkeys[run + k] = s_k[k];
                pvals[run + k] = s_v[k];
            }
        } else {
            uint64_t o = run + excl;
            for (int ty = r.y; ty <= r.w; ++ty)
                for (int tx = r.x; tx <= r.z; ++tx, ++o) {
                    pkeys[o] = (uint32_t)(base + ty * tx_n + tx);
                    pvals[o] = gi;
                }
        }
    }
}

__global__ void ranges_kernel(const uint32_t *__restrict__ keys, const int64_t *sort_count, uint2 *__restrict__ ranges) {
    const int64_t count = *sort_count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 4 * c < count; c += stride) {
        const int64_t i0 = 4 * c;
        uint32_t k[6];
        k[0] = i0 > 0 ? keys[i0 - 1] : 0xffffffffu;
        if (i0 + 4 <= count) {
            const uint4 q = *reinterpret_cast<const uint4 *>(keys + i0);
            k[1] = q.x; k[2] = q.y; k[3] = q.z; k[4] = q.w;
        } else {
            for (int j = 0; j < 4; ++j) k[1 + j] = i0 + j < count ? keys[i0 + j] : 0xffffffffu;
        }
        k[5] = i0 + 4 < count ? keys[i0 + 4] : 0xffffffffu;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t i = i0 + j;
            if (i >= count) break;
            const uint32_t t = k[1 + j];
            if (k[j] != t || i == 0) ranges[t].x = (uint32_t)i;
            if (k[2 + j] != t || i == count - 1) ranges[t].y = (uint32_t)(i + 1);
        }
    }
}

__global__ void keys64_kernel(const uint32_t *__restrict__ tkeys, const uint32_t *__restrict__ vals,
                              const int64_t *sort_count, const gs_camera *__restrict__ cams, int n_views, int64_t n,
                              const float *__restrict__ rec, uint64_t *__restrict__ keys) {
    const int64_t count = *sort_count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = tkeys[i];
        const int v = view_of_tile(cams, n_views, t);
        const int64_t e = (int64_t)v * n + vals[i];
        keys[i] = ((uint64_t)t << 32) | (uint64_t)__float_as_uint(rec[e * kRecFloats + 9]);
    }
}

int bits_for(int64_t values) {  // bits needed to represent 0 .. values-1
    int b = 0;
    while (b < 63 && ((int64_t)1 << b) < values) ++b;
    return b < 1 ? 1 : b;
}

struct BinWorkspace {
    uint32_t *dk[2], *dv[2];        // depth keys / entry ids, ping-pong, [V*N]
    uint32_t *pk[2], *pv;           // pair tile keys ping-pong [cap], pair values scratch [cap]
    uint32_t *counts;               // [RADIX * RS_MAX_BLOCKS] + [RADIX] digit totals
    unsigned long long *block_sums; // [ceil(total / RS_THREADS) + 1] chunk pair counts, then offsets
    int64_t *sort_count;            // [1]
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t bin_ws_layout(int64_t total, int64_t cap, BinWorkspace *w, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    for (int i = 0; i < 2; ++i) {
        char *a = take(sizeof(uint32_t) * (size_t)(total > 0 ? total : 1));
        char *b = take(sizeof(uint32_t) * (size_t)(total > 0 ? total : 1));
        if (w) { w->dk[i] = (uint32_t *)a; w->dv[i] = (uint32_t *)b; }
    }
    for (int i = 0; i < 2; ++i) {
        char *a = take(sizeof(uint32_t) * (size_t)(cap > 0 ? cap : 1));
        if (w) w->pk[i] = (uint32_t *)a;
    }
    char *pv = take(sizeof(uint32_t) * (size_t)(cap > 0 ? cap : 1));
    char *counts = take(sizeof(uint32_t) * RADIX * (RS_MAX_BLOCKS + 1));
    char *bs = take(sizeof(unsigned long long) * (size_t)(ceil_div(total > 0 ? total : 1, RS_THREADS) + 1));
    char *sc = take(sizeof(int64_t));
    if (w) {
        w->pv = (uint32_t *)pv;
        w->counts = (uint32_t *)counts;
        w->block_sums = (unsigned long long *)bs;
        w->sort_count = (int64_t *)sc;
    }
    return off;
}

}  // namespace

extern "C" {

size_t gs_bin_sort_workspace_size(int64_t n, int32_t n_views, int64_t pair_capacity, int64_t total_tiles) {
    (void)total_tiles;
    if (n < 0 || n_views <= 0 || pair_capacity < 0) return 0;
    return bin_ws_layout(n * n_views, pair_capacity, nullptr, nullptr);
}

gs_status gs_bin_sort(const gs_projected *proj, const gs_camera *cams, int32_t n_views, int64_t n,
                      int64_t total_tiles, const gs_raster_config *cfg, void *workspace, size_t workspace_bytes,
                      uint64_t *keys, uint32_t *vals, int64_t pair_capacity, uint32_t *ranges,
                      int64_t *dev_pair_count, int32_t *dev_status, cudaStream_t stream) {
    if (!proj || !cams || !cfg || n_views <= 0 || n < 0 || total_tiles <= 0 || !vals || !ranges || !dev_pair_count)
        return GS_ERR_INVALID_ARG;
    if (cfg->tile != 8 && cfg->tile != 16 && cfg->tile != 32) return GS_ERR_INVALID_ARG;
    if (pair_capacity < 0 || pair_capacity >= ((int64_t)1 << 32) - 1) return GS_ERR_INVALID_ARG;
    if (total_tiles >= ((int64_t)1 << 31)) return GS_ERR_INVALID_ARG;
    const int64_t total = n * n_views;
    if (total >= ((int64_t)1 << 32) - 1) return GS_ERR_INVALID_ARG;
    if (total > 0 && (!proj->rec || !proj->rect || !proj->tiles_touched)) return GS_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < bin_ws_layout(total, pair_capacity, nullptr, nullptr)) return GS_ERR_WORKSPACE;
    if ((uintptr_t)workspace & 255) return GS_ERR_WORKSPACE;
    BinWorkspace w;
    bin_ws_layout(total, pair_capacity, &w, (char *)workspace);

    GS_TRY(cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)total_tiles, stream));
    if (total == 0) {
        GS_TRY(cudaMemsetAsync(dev_pair_count, 0, sizeof(int64_t), stream));
        return GS_OK;
    }
    // 1. depth order of all (view, Gaussian) entries
    depth_keys_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, stream>>>(proj->rec, proj->tiles_touched, total,
                                                                         w.dk[0], w.dv[0]);
    GS_TRY_LAUNCH();
    const int dsel = radix_sort(w.dk[0], w.dv[0], w.dk[1], w.dv[1], nullptr, total, 32, w.counts, stream);
    GS_TRY_LAUNCH();
    const uint32_t *order = w.dv[dsel];
    // 2. pair offsets in depth order, fused pair emission (one block per chunk)
    const int64_t n_chunks = ceil_div(total, RS_THREADS);
    count_reduce<<<(unsigned)n_chunks, RS_THREADS, 0, stream>>>(proj->tiles_touched, order, total, w.block_sums);
    count_top<<<1, SCAN_THREADS, 0, stream>>>(w.block_sums, n_chunks, pair_capacity, dev_pair_count, w.sort_count,
                                             dev_status);
    // The final pass must land in (pk[0], vals): emit into the buffer that an
    // even or odd number of passes maps there.
    const int tbits = bits_for(total_tiles);
    const int passes = radix_passes(tbits);
    uint32_t *ek = (passes & 1) ? w.pk[1] : w.pk[0];
    uint32_t *ev = (passes & 1) ? w.pv : vals;
    emit_pairs<<<(unsigned)n_chunks, RS_THREADS, 0, stream>>>(proj->tiles_touched, reinterpret_cast<const int4 *>(proj->rect), order,
                                             total, n, cams, cfg->tile, w.block_sums, w.sort_count, ek, ev);
    GS_TRY_LAUNCH();
    // 3. stable sort of the pairs by tile id
    const int psel = (passes & 1) ? radix_sort(w.pk[1], w.pv, w.pk[0], vals, w.sort_count, pair_capacity, tbits,
                                               w.counts, stream)
                                  : radix_sort(w.pk[0], vals, w.pk[1], w.pv, w.sort_count, pair_capacity, tbits,
                                               w.counts, stream);
    GS_TRY_LAUNCH();
    (void)psel;  // by construction the result is in (pk[0], vals)
    // 4. per-tile ranges and, on request, the 64-bit keys
    ranges_kernel<<<4 * 152, 256, 0, stream>>>(w.pk[0], w.sort_count, reinterpret_cast<uint2 *>(ranges));
    GS_TRY_LAUNCH();
    if (keys) {
        keys64_kernel<<<4 * 152, 256, 0, stream>>>(w.pk[0], vals, w.sort_count, cams, n_views, n, proj->rec, keys);
        GS_TRY_LAUNCH();
    }
    return GS_OK;
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
constexpr int64_t kNoAllocMaxPairs = (int64_t)1 << 20;    // pair_capacity

// Size of the gs_bin_sort workspace at the limits above (same layout as
// bin_ws_layout: each buffer rounded up to 256 bytes).
constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kNoAllocBytes = 4 * al256(4 * (size_t)kNoAllocMaxEntries) + 3 * al256(4 * (size_t)kNoAllocMaxPairs) +
                                 al256(4 * (size_t)RADIX * (RS_MAX_BLOCKS + 1)) +
                                 al256(8 * (size_t)(kNoAllocMaxEntries / RS_THREADS + 1)) + al256(8);

// One copy per device that loads the library, held until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void *g_noalloc_ptr[kMaxDevices] = {};

}  // namespace

extern "C" gs_status gs_bin_sort_noalloc(const gs_projected *proj, const gs_camera *cams, int32_t n_views, int64_t n,
                                         int64_t total_tiles, const gs_raster_config *cfg, uint64_t *keys,
                                         uint32_t *vals, int64_t pair_capacity, uint32_t *ranges,
                                         int64_t *dev_pair_count, int32_t *dev_status, cudaStream_t stream) {
    if (n < 0 || n_views <= 0 || pair_capacity < 0) return GS_ERR_INVALID_ARG;
    if (n * n_views > kNoAllocMaxEntries || pair_capacity > kNoAllocMaxPairs) return GS_ERR_WORKSPACE;
    int dev = 0;
    GS_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return GS_ERR_UNSUPPORTED;
    if (!g_noalloc_ptr[dev]) {
        // Host code cannot use the array's name as a device address: look the
        // address up once per device, with that device current.
        void *p = nullptr;
        GS_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    return gs_bin_sort(proj, cams, n_views, n, total_tiles, cfg, g_noalloc_ptr[dev], kNoAllocBytes, keys, vals,
                       pair_capacity, ranges, dev_pair_count, dev_status, stream);
}
