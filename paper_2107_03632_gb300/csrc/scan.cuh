// Device-wide exclusive prefix sum (three passes: tile scan, scan of tile
// totals, add-back).  Deterministic; no atomics.
#pragma once

#include "common.cuh"

namespace rbffd {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048 elements per block

// Exclusive block scan of one value per thread; returns the block total.
template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* sh, T& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) RB_AT(sh, wid, kScanThreads / 32) = x;
    __syncthreads();
    if (wid == 0) {
        T w = (lane < kScanThreads / 32) ? sh[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) sh[lane] = w;
    }
    __syncthreads();
    T warp_prefix = (wid > 0) ? RB_AT(sh, wid - 1, kScanThreads / 32) : T(0);
    total = sh[kScanThreads / 32 - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

// out[i] = sum of load(j) for tile-local j < i; tile totals to sums.
// `in` is read through `load(i)` so callers can scan derived values.
template <class T, class Load>
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(Load load, int64_t n, T* out, T* sums) {
    __shared__ T sh[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        v[k] = (i < n) ? load(i) : T(0);
        local += v[k];
    }
    T total;
    T run = block_exclusive_scan<T>(local, sh, total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Exclusive scan of the tile totals in place (one block, chunks of
// kScanTile with a running carry, so any number of tiles); writes the grand
// total to *grand.
template <class T>
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(T* sums, int ntiles, T* grand) {
    __shared__ T sh[kScanThreads / 32];
    T carry = 0;
    for (int chunk = 0; chunk < ntiles; chunk += kScanTile) {
        const int base = chunk + threadIdx.x * kScanItems;
        T v[kScanItems];
        T local = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            v[k] = (base + k < ntiles) ? sums[base + k] : T(0);
            local += v[k];
        }
        T total;
        T run = carry + block_exclusive_scan<T>(local, sh, total);
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (base + k < ntiles) sums[base + k] = run;
            run += v[k];
        }
        carry += total;
    }
    if (threadIdx.x == 0) *grand = carry;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) scan_add_kernel(T* out, int64_t n, const T* sums) {
    const T add = sums[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
        const int64_t i = base + k;
        if (i < n) out[i] += add;
    }
}

inline int scan_tiles(int64_t n) { return (int)((n + kScanTile - 1) / kScanTile); }

// Exclusive scan of load(0..n-1) into out[0..n-1], grand total into *grand
// (device).  `sums` needs scan_tiles(n) elements.
template <class T, class Load>
inline cudaError_t exclusive_scan(Load load, int64_t n, T* out, T* sums, T* grand, cudaStream_t st) {
    const int tiles = scan_tiles(n);
    if (tiles == 0) {
        return cudaMemsetAsync(grand, 0, sizeof(T), st);
    }
    scan_tiles_kernel<T, Load><<<tiles, kScanThreads, 0, st>>>(load, n, out, sums);
    scan_sums_kernel<T><<<1, kScanThreads, 0, st>>>(sums, tiles, grand);
    scan_add_kernel<T><<<tiles, kScanThreads, 0, st>>>(out, n, sums);
    note_launches(3);
    return cudaGetLastError();
}

}  // namespace rbffd
