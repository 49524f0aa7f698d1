// Device-wide exclusive prefix sum (see scan.cuh).
#include "scan.cuh"

namespace gipc {
namespace {

// Block-wide exclusive scan of per-thread values; returns the block total to all threads.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t& total) {
    __shared__ int64_t warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int64_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;
    }
    __syncthreads();
    total = warp_tot[(blockDim.x >> 5) - 1];
    const int64_t before = wid > 0 ? warp_tot[wid - 1] : 0;
    __syncthreads();
    return before + x - v;
}

template <typename TIn>
__global__ void __launch_bounds__(kScanThreads)
tile_scan_kernel(const TIn* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                 int64_t* __restrict__ tile_tot) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems], sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = (base + j < n) ? (int64_t)in[base + j] : 0;
        sum += v[j];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(sum, total);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == 0 && tile_tot) tile_tot[blockIdx.x] = total;
    if (!tile_tot && threadIdx.x == blockDim.x - 1) out[n] = run;  // single tile: write total
}

__global__ void add_tile_offsets_kernel(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += off[i / kScanTile];
    if (i == 0) out[n] = off[(n + kScanTile - 1) / kScanTile];
}

}  // namespace

template <typename TIn>
cudaError_t exclusive_scan(const TIn* in, int64_t* out, int64_t n, int64_t* scratch, cudaStream_t s) {
    if (n <= kScanTile) {
        tile_scan_kernel<TIn><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        return cudaGetLastError();
    }
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    int64_t* tot = scratch;               // [tiles + 1]
    tile_scan_kernel<TIn><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, tot);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan<int64_t>(tot, tot, tiles, scratch + tiles + 1, s);  // in place is safe per tile
    if (e != cudaSuccess) return e;
    add_tile_offsets_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, tot);
    return cudaGetLastError();
}

template cudaError_t exclusive_scan<int32_t>(const int32_t*, int64_t*, int64_t, int64_t*, cudaStream_t);
template cudaError_t exclusive_scan<int64_t>(const int64_t*, int64_t*, int64_t, int64_t*, cudaStream_t);

}  // namespace gipc
