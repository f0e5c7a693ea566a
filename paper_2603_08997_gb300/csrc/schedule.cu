// gs_tile_order: the order in which the compositing kernels visit tiles.
//
// One CTA composites one tile, and the hardware hands out CTAs in launch
// order, so launching the tiles with the longest lists first (longest
// processing time first) keeps a long tile from starting last and running
// alone at the end of the grid.  The work of a tile is its list length; tiles
// are grouped by that length on a logarithmic scale (eight buckets per
// doubling) and the buckets are visited longest first.  The order inside a
// bucket is not specified: compositing results do not depend on the order.
#include "common.cuh"

using namespace gsr;

namespace {

constexpr int ORDER_THREADS = 1024;
constexpr int ORDER_BUCKETS = 256;

// 8 log2(len + 1) rounded down: the bit length and the next three bits.
__device__ __forceinline__ int work_bucket(uint32_t len) {
    const uint32_t x = len + 1u;  // >= 1 (len < 2^32 - 1)
    const int lz = __clz(x);
    const int e = 31 - lz;
    const uint32_t frac = e >= 3 ? (x >> (e - 3)) & 7u : (x << (3 - e)) & 7u;
    return 8 * e + (int)frac;
}

__global__ void __launch_bounds__(ORDER_THREADS) tile_order_kernel(const uint2 *__restrict__ ranges, int64_t tiles,
                                                                   uint32_t *__restrict__ order) {
    __shared__ uint32_t s_cnt[ORDER_BUCKETS];
    for (int b = threadIdx.x; b < ORDER_BUCKETS; b += ORDER_THREADS) s_cnt[b] = 0u;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < tiles; t += ORDER_THREADS) {
        const uint2 r = ranges[t];
        atomicAdd(&s_cnt[work_bucket(r.y > r.x ? r.y - r.x : 0u)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // first slot of each bucket, longest bucket first
        uint32_t run = 0;
        for (int b = ORDER_BUCKETS - 1; b >= 0; --b) {
            const uint32_t c = s_cnt[b];
            s_cnt[b] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < tiles; t += ORDER_THREADS) {
        const uint2 r = ranges[t];
        order[atomicAdd(&s_cnt[work_bucket(r.y > r.x ? r.y - r.x : 0u)], 1u)] = (uint32_t)t;
    }
}

}  // namespace

extern "C" gs_status gs_tile_order(const uint32_t *ranges, int64_t total_tiles, uint32_t *tile_order,
                                   cudaStream_t stream) {
    if (!ranges || !tile_order || total_tiles <= 0 || total_tiles >= ((int64_t)1 << 31)) return GS_ERR_INVALID_ARG;
    tile_order_kernel<<<1, ORDER_THREADS, 0, stream>>>(reinterpret_cast<const uint2 *>(ranges), total_tiles,
                                                       tile_order);
    GS_TRY_LAUNCH();
    return GS_OK;
}
