// mpm_sort.cuh -- stable re-ordering of particles by key (Sec. 3 step xii).
//
// The paper re-orders particles so that those in the first cell come first,
// then those of the second cell, and so on, keeping their current order
// inside a cell (a stable counting sort over the per-cell particle lists).
// Here: an LSD radix sort of (key, index) pairs with per-block stable ranks,
// followed by one gather of the particle state and the cell-start table.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mpm {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;                       // per thread
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide inclusive scan of one value per thread (warp shuffles + smem).
__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t v, uint32_t* warp_sums)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_sums[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < nw ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    if (warp > 0) v += warp_sums[warp - 1];
    __syncthreads();
    return v;
}

// Phase 1: per-tile sums (block blk of the scan).
__device__ __forceinline__ void scan_reduce_block(const uint32_t* in, int64_t n, uint32_t* partial, int64_t blk)
{
    __shared__ uint32_t ws[32];
    const int64_t base = blk * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    s = block_inclusive_scan(s, ws);
    if (threadIdx.x == blockDim.x - 1) partial[blk] = s;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* in, int64_t n, uint32_t* partial)
{
    scan_reduce_block(in, n, partial, blockIdx.x);
}

// Phase 2: exclusive scan of the per-tile sums by one block.
__device__ __forceinline__ void scan_partials_block(uint32_t* partial, int64_t m)
{
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < m; b += blockDim.x) {
        int64_t i = b + threadIdx.x;
        uint32_t v = i < m ? partial[i] : 0u;
        uint32_t inc = block_inclusive_scan(v, ws);
        uint32_t c = carry;
        if (i < m) partial[i] = c + inc - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + inc;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partials(uint32_t* partial, int64_t m)
{
    scan_partials_block(partial, m);
}

// Phase 3: exclusive scan inside each tile plus its offset; out[n] = total
// when write_total is set (out must then hold n + 1 values).
__device__ __forceinline__ void scan_down_block(const uint32_t* in, int64_t n, const uint32_t* partial, uint32_t* out,
                                                int write_total, int64_t blk)
{
    __shared__ uint32_t ws[32];
    const int64_t base = blk * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems], s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        s += v[i];
    }
    uint32_t inc = block_inclusive_scan(s, ws);
    uint32_t run = partial[blk] + inc - s;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
        if (write_total && base + i == n - 1) out[n] = run;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* in, int64_t n, const uint32_t* partial,
                                                           uint32_t* out, int write_total)
{
    scan_down_block(in, n, partial, out, write_total, blockIdx.x);
}

__host__ __device__ inline int64_t scan_blocks(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// Exclusive scan of n u32 values; partial needs scan_blocks(n) entries.
inline void scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* partial, int write_total,
                           cudaStream_t st, int64_t* launches)
{
    const int64_t nb = scan_blocks(n);
    if (n <= 0) return;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, partial);
    k_scan_partials<<<1, kScanThreads, 0, st>>>(partial, nb);
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, partial, out, write_total);
    if (launches) *launches += 3;
}

// ------------------------------------------------------------- radix sort

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;                      // per thread
constexpr int kSortTile = kSortThreads * kSortItems; // elements per block
constexpr int kWarpSpan = kSortTile / kSortWarps;   // contiguous elements per warp
constexpr int kRadixBitsMax = 9;                    // digits of up to 9 bits
constexpr int kRadixMax = 1 << kRadixBitsMax;

// Digit histogram of each block, stored digit-major: hist[d * nblocks + b].
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* keys, int64_t n, int shift, int bits,
                                                             uint32_t* hist, const int* active)
{
    if (active && !*active) return;
    __shared__ uint32_t h[kRadixMax];
    const int radix = 1 << bits;
    for (int i = threadIdx.x; i < radix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) {
        int64_t j = base + i;
        if (j < n) atomicAdd(&h[(keys[j] >> shift) & (radix - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < radix; d += blockDim.x) hist[(int64_t)d * gridDim.x + blockIdx.x] = h[d];
}

// Stable scatter: each warp owns a contiguous run of kWarpSpan elements and
// places them in order, 32 at a time, using __match_any_sync to rank equal
// digits inside the warp; warps are ordered by a per-digit prefix over warps.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t* keys_in, const uint32_t* idx_in,
                                                                uint32_t* keys_out, uint32_t* idx_out, int64_t n,
                                                                int shift, int bits, const uint32_t* offsets,
                                                                const int* active, int first_pass)
{
    if (active && !*active) return;
    __shared__ uint32_t cnt[kSortWarps][kRadixMax];
    const int radix = 1 << bits;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kRadixMax; i += blockDim.x) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * kWarpSpan;
    constexpr int R = kWarpSpan / 32;
    // the warp's keys and indices stay in registers between counting and placing
    uint32_t kr[R], ir[R];
#pragma unroll
    for (int c = 0; c < R; ++c) {
        const int64_t j = wbase + c * 32 + lane;
        const bool valid = j < n;
        kr[c] = valid ? keys_in[j] : 0u;
        ir[c] = valid ? (first_pass ? (uint32_t)j : idx_in[j]) : 0u;
    }
#pragma unroll
    for (int c = 0; c < R; ++c) {
        const bool valid = wbase + c * 32 + lane < n;
        const uint32_t d = valid ? ((kr[c] >> shift) & (radix - 1)) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&cnt[warp][d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    // exclusive prefix over warps, plus the global offset of (digit, block)
    for (int d = threadIdx.x; d < radix; d += blockDim.x) {
        uint32_t run = offsets[(int64_t)d * gridDim.x + blockIdx.x];
        for (int w = 0; w < kSortWarps; ++w) {
            uint32_t t = cnt[w][d];
            cnt[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < R; ++c) {
        const bool valid = wbase + c * 32 + lane < n;
        const uint32_t d = valid ? ((kr[c] >> shift) & (radix - 1)) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        const int leader = __ffs(peers) - 1;
        uint32_t basev = 0;
        if (valid && lane == leader) basev = cnt[warp][d];
        basev = __shfl_sync(0xffffffffu, basev, leader);
        if (valid) {
            const uint32_t pos = basev + rank;
            keys_out[pos] = kr[c];
            idx_out[pos] = ir[c];
        }
        __syncwarp();
        if (valid && lane == leader) cnt[warp][d] = basev + __popc(peers);
        __syncwarp();
    }
}

// Cell-start table from sorted keys: start[k] = first position with key >= k.
__global__ void k_cell_start(const uint32_t* keys, int64_t n, int64_t nkey, uint32_t* start, const int* active)
{
    if (active && !*active) return;
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j > n) return;
    int64_t lo = (j == 0) ? 0 : (int64_t)keys[j - 1] + 1;
    int64_t hi = (j == n) ? nkey : (int64_t)keys[j];
    if (j == 0) lo = 0;
    for (int64_t k = lo; k <= hi && k <= nkey; ++k) start[k] = (uint32_t)j;
}

}  // namespace mpm
