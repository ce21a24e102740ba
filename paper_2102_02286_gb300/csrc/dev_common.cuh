// Device helpers shared by the index build and the search kernels:
// CUDA error plumbing and a multi-block exclusive scan.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "hicops_internal.h"

#define HC_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            hicops::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? HICOPS_ENOMEM : HICOPS_ECUDA;         \
        }                                                                                  \
    } while (0)

namespace hicops {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide inclusive scan of one value per thread (256 threads).
__device__ __forceinline__ uint64_t block_inclusive_scan(uint64_t v, uint64_t* warp_tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    if (lane == 31) warp_tot[w] = v;
    __syncthreads();
    if (w == 0) {
        uint64_t t = lane < (kScanThreads / 32) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t n = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += n;
        }
        if (lane < (kScanThreads / 32)) warp_tot[lane] = t;
    }
    __syncthreads();
    if (w > 0) v += warp_tot[w - 1];
    __syncthreads();
    return v;
}

template <class T>
__global__ void scan_reduce_kernel(const T* __restrict__ in, uint64_t n, uint64_t* __restrict__ block_sums) {
    __shared__ uint64_t wt[kScanThreads / 32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint64_t s = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        uint64_t g = base + i;
        if (g < n) s += (uint64_t)in[g];
    }
    s = block_inclusive_scan(s, wt);
    if (threadIdx.x == kScanThreads - 1) block_sums[blockIdx.x] = s;
}

// exclusive scan of one tile with a carried-in block offset
template <class T>
__global__ void scan_tile_kernel(const T* __restrict__ in, uint64_t n, const uint64_t* __restrict__ block_off,
                                 uint64_t* __restrict__ out, uint64_t* __restrict__ total) {
    __shared__ uint64_t wt[kScanThreads / 32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint64_t v[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        uint64_t g = base + i;
        v[i] = g < n ? (uint64_t)in[g] : 0;
        s += v[i];
    }
    uint64_t incl = block_inclusive_scan(s, wt);
    uint64_t run = incl - s + (block_off ? block_off[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        uint64_t g = base + i;
        if (g < n) out[g] = run;
        run += v[i];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) *total = run;
}

// Exclusive scan in[0..n) -> out[0..n), total -> *total (device pointers).
// tmp must hold scan_tmp_words(n) uint64 words.
inline uint64_t scan_tmp_words(uint64_t n) {
    uint64_t words = 0;
    while (n > (uint64_t)kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        words += 2 * n;
    }
    return words + 1;
}

template <class T>
cudaError_t exclusive_scan(const T* in, uint64_t n, uint64_t* out, uint64_t* total, uint64_t* tmp,
                           cudaStream_t s) {
    if (n == 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint64_t), s);
        return cudaSuccess;
    }
    const uint64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        scan_tile_kernel<T><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out, total);
        count_launches(1);
        return cudaGetLastError();
    }
    uint64_t* sums = tmp;
    uint64_t* sums_scanned = tmp + nb;
    scan_reduce_kernel<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
    count_launches(1);
    cudaError_t e = exclusive_scan<uint64_t>(sums, nb, sums_scanned, nullptr, tmp + 2 * nb, s);
    if (e != cudaSuccess) return e;
    scan_tile_kernel<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums_scanned, out, total);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace hicops
