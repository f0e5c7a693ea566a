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
// 2048 keys with warp match/ballot and scatters them stably.
#include "common.cuh"

using namespace gsr;

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int RS_MAX_BLOCKS = 1024;
constexpr int SCAN_THREADS = 1024;

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

// In-place exclusive scan of n uint32 values by one block.
__global__ void __launch_bounds__(SCAN_THREADS) rs_scan(uint32_t *a, int n) {
    __shared__ uint32_t s[SCAN_THREADS];
    const int per = (n + SCAN_THREADS - 1) / SCAN_THREADS;
    const int lo = threadIdx.x * per;
    const int hi = min(n, lo + per);
    uint32_t sum = 0;
    for (int i = lo; i < hi; ++i) sum += a[i];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < SCAN_THREADS; off <<= 1) {
        const uint32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    uint32_t run = s[threadIdx.x] - sum;
    for (int i = lo; i < hi; ++i) {
        const uint32_t t = a[i];
        a[i] = run;
        run += t;
    }
}

__global__ void __launch_bounds__(RS_THREADS) rs_downsweep(const uint32_t *__restrict__ keys_in,
                                                           const uint32_t *__restrict__ vals_in,
                                                           uint32_t *__restrict__ keys_out,
                                                           uint32_t *__restrict__ vals_out, const int64_t *d_count,
                                                           int64_t cap, int shift, uint32_t mask,
                                                           const uint32_t *__restrict__ offsets) {
    __shared__ uint32_t s_run[RADIX];
    __shared__ uint32_t s_tot[RADIX];
    __shared__ uint32_t s_wcnt[RS_WARPS][RADIX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) s_run[d] = offsets[(int64_t)d * gridDim.x + blockIdx.x];
    const int64_t count = effective_count(d_count, cap);
    int64_t begin, end;
    block_range(count, gridDim.x, blockIdx.x, begin, end);
    for (int64_t base = begin; base < end; base += RS_TILE) {
        for (int i = threadIdx.x; i < RS_WARPS * RADIX; i += RS_THREADS) (&s_wcnt[0][0])[i] = 0u;
        __syncthreads();
        uint32_t k[RS_ITEMS], v[RS_ITEMS], lr[RS_ITEMS];
        int dg[RS_ITEMS];
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {
            const int64_t idx = base + (int64_t)warp * 32 * RS_ITEMS + r * 32 + lane;
            const bool valid = idx < end;
            k[r] = valid ? keys_in[idx] : 0u;
            v[r] = valid ? vals_in[idx] : 0u;
            const int d = valid ? (int)((k[r] >> shift) & mask) : RADIX + lane;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
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
        for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) {
                const uint32_t c = s_wcnt[w][d];
                s_wcnt[w][d] = run;
                run += c;
            }
            s_tot[d] = run;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {
            if (dg[r] < RADIX) {
                const uint32_t pos = s_run[dg[r]] + s_wcnt[warp][dg[r]] + lr[r];
                keys_out[pos] = k[r];
                vals_out[pos] = v[r];
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
int radix_sort(uint32_t *ka, uint32_t *va, uint32_t *kb, uint32_t *vb, const int64_t *d_count, int64_t cap,
               int bits, uint32_t *counts, cudaStream_t stream) {
    const int G = rs_blocks(cap);
    int cur = 0;
    for (int shift = 0; shift < bits; shift += RADIX_BITS) {
        const int nb = bits - shift < RADIX_BITS ? bits - shift : RADIX_BITS;
        const uint32_t mask = (1u << nb) - 1u;
        uint32_t *ki = cur ? kb : ka, *vi = cur ? vb : va, *ko = cur ? ka : kb, *vo = cur ? va : vb;
        rs_upsweep<<<G, RS_THREADS, 0, stream>>>(ki, d_count, cap, shift, mask, counts);
        rs_scan<<<1, SCAN_THREADS, 0, stream>>>(counts, RADIX * G);
        rs_downsweep<<<G, RS_THREADS, 0, stream>>>(ki, vi, ko, vo, d_count, cap, shift, mask, counts);
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

// Scan of the tile counts in depth order, reduce phase: per-block sums.
__global__ void __launch_bounds__(RS_THREADS) count_reduce(const int32_t *__restrict__ touched,
                                                           const uint32_t *__restrict__ order, int64_t total,
                                                           unsigned long long *__restrict__ block_sums) {
    int64_t begin, end;
    block_range(total, gridDim.x, blockIdx.x, begin, end);
    unsigned long long s = 0;
    for (int64_t m = begin + threadIdx.x; m < end; m += RS_THREADS) s += (unsigned)touched[order[m]];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __shared__ unsigned long long ws[RS_WARPS];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < RS_WARPS; ++w) t += ws[w];
        block_sums[blockIdx.x] = t;
    }
}

// Exclusive scan of the block sums (one block); writes the total pair count
// and the count the pair sort will use (0 when over capacity).
__global__ void count_top(unsigned long long *block_sums, int G, int64_t cap, int64_t *dev_pair_count,
                          int64_t *sort_count, int32_t *dev_status) {
    if (threadIdx.x != 0) return;
    unsigned long long run = 0;
    for (int b = 0; b < G; ++b) {
        const unsigned long long t = block_sums[b];
        block_sums[b] = run;
        run += t;
    }
    *dev_pair_count = (int64_t)run;
    if ((int64_t)run > cap) {
        set_status(dev_status, GS_ERR_CAPACITY);
        *sort_count = 0;
    } else {
        *sort_count = (int64_t)run;
    }
}

// Scan phase fused with pair emission: every entry, in depth order, writes
// one (tile id, Gaussian index) pair per tile of its rectangle, row-major.
__global__ void __launch_bounds__(RS_THREADS) emit_pairs(const int32_t *__restrict__ touched,
                                                         const int4 *__restrict__ rect,
                                                         const uint32_t *__restrict__ order, int64_t total,
                                                         int64_t n, const gs_camera *__restrict__ cams, int tile,
                                                         const unsigned long long *__restrict__ block_offsets,
                                                         const int64_t *sort_count, uint32_t *__restrict__ pkeys,
                                                         uint32_t *__restrict__ pvals) {
    if (*sort_count == 0) return;  // nothing to emit, or over capacity
    __shared__ unsigned long long s_scan[RS_THREADS];
    int64_t begin, end;
    block_range(total, gridDim.x, blockIdx.x, begin, end);
    unsigned long long run = block_offsets[blockIdx.x];
    for (int64_t base = begin; base < end; base += RS_THREADS) {
        const int64_t m = base + threadIdx.x;
        uint32_t e = 0;
        unsigned long long c = 0;
        if (m < end) {
            e = order[m];
            c = (unsigned)touched[e];
        }
        s_scan[threadIdx.x] = c;
        __syncthreads();
        for (int off = 1; off < RS_THREADS; off <<= 1) {
            const unsigned long long t = threadIdx.x >= off ? s_scan[threadIdx.x - off] : 0ull;
            __syncthreads();
            s_scan[threadIdx.x] += t;
            __syncthreads();
        }
        const unsigned long long incl = s_scan[threadIdx.x];
        const unsigned long long tile_total = s_scan[RS_THREADS - 1];
        if (c > 0) {
            uint64_t off = run + incl - c;
            const int64_t v = (int64_t)e / n;
            const uint32_t gi = (uint32_t)((int64_t)e - v * n);
            const gs_camera &cam = cams[v];
            const int tiles_x = (cam.width + tile - 1) / tile;
            const int4 r = rect[e];
            for (int ty = r.y; ty <= r.w; ++ty)
                for (int tx = r.x; tx <= r.z; ++tx) {
                    pkeys[off] = (uint32_t)(cam.tile_offset + ty * tiles_x + tx);
                    pvals[off] = gi;
                    ++off;
                }
        }
        run += tile_total;
        __syncthreads();
    }
}

__global__ void ranges_kernel(const uint32_t *__restrict__ keys, const int64_t *sort_count, uint2 *__restrict__ ranges) {
    const int64_t count = *sort_count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = keys[i];
        if (i == 0 || keys[i - 1] != t) ranges[t].x = (uint32_t)i;
        if (i == count - 1 || keys[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
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
    uint32_t *counts;               // [RADIX * RS_MAX_BLOCKS]
    unsigned long long *block_sums; // [RS_MAX_BLOCKS]
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
    char *counts = take(sizeof(uint32_t) * RADIX * RS_MAX_BLOCKS);
    char *bs = take(sizeof(unsigned long long) * RS_MAX_BLOCKS);
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
    // 2. pair offsets in depth order, fused pair emission
    const int G = rs_blocks(total);
    count_reduce<<<G, RS_THREADS, 0, stream>>>(proj->tiles_touched, order, total, w.block_sums);
    count_top<<<1, 32, 0, stream>>>(w.block_sums, G, pair_capacity, dev_pair_count, w.sort_count, dev_status);
    // The final pass must land in (pk[0], vals): emit into the buffer that an
    // even or odd number of passes maps there.
    const int tbits = bits_for(total_tiles);
    const int passes = radix_passes(tbits);
    uint32_t *ek = (passes & 1) ? w.pk[1] : w.pk[0];
    uint32_t *ev = (passes & 1) ? w.pv : vals;
    emit_pairs<<<G, RS_THREADS, 0, stream>>>(proj->tiles_touched, reinterpret_cast<const int4 *>(proj->rect), order,
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
