// Device exclusive prefix sums (three launches: tile sums, a single-block scan of the
// tile sums, tile-local scans).  Shared by the CSR assembly and the preconditioner.
#pragma once

#include <algorithm>

#include "ms_internal.cuh"

namespace {

constexpr int kScanBS = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBS * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T* total, T* sh) {
    // inclusive warp scan
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        T t = lane < kScanBS / 32 ? sh[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanBS / 32) sh[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    const T before = (w > 0 ? sh[w - 1] : T(0)) + x - v;
    *total = sh[kScanBS / 32 - 1];
    __syncthreads();
    return before;
}

template <typename Tin, typename Tout>
__global__ void k_scan_tiles(const Tin* in, int64_t n, Tout* tile_sums) {
    const int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
    Tout s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += (Tout)in[base + k];
    __shared__ Tout sh[kScanBS / 32];
    Tout total;
    block_exclusive_scan<Tout>(s, &total, sh);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Exclusive scan of a[0..n) in place by one block; a[n] receives the total.
template <typename T>
__global__ void k_scan_single(T* a, int64_t n) {
    __shared__ T sh[kScanBS / 32];
    T carry = 0;
    for (int64_t s = 0; s < n; s += kScanBS) {
        const int64_t i = s + threadIdx.x;
        T v = i < n ? a[i] : T(0);
        T total;
        T ex = block_exclusive_scan<T>(v, &total, sh);
        if (i < n) a[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) a[n] = carry;
}

template <typename Tin, typename Tout>
__global__ void k_scan_apply(const Tin* in, int64_t n, const Tout* tile_off, int64_t ntiles, Tout* out) {
    const int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
    Tout loc[kScanItems];
    Tout s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = (base + k < n) ? (Tout)in[base + k] : Tout(0);
        s += loc[k];
    }
    __shared__ Tout sh[kScanBS / 32];
    Tout total;
    Tout ex = block_exclusive_scan<Tout>(s, &total, sh) + tile_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += loc[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tile_off[ntiles];
}

// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.  tmp holds ntiles+1 Tout.
template <typename Tin, typename Tout>
void exclusive_scan(const Tin* in, int64_t n, Tout* out, Tout* tmp, cudaStream_t s) {
    const int64_t ntiles = std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile);
    k_scan_tiles<Tin, Tout><<<(unsigned)ntiles, kScanBS, 0, s>>>(in, n, tmp); ms_count_launch();
    k_scan_single<Tout><<<1, kScanBS, 0, s>>>(tmp, ntiles); ms_count_launch();
    k_scan_apply<Tin, Tout><<<(unsigned)ntiles, kScanBS, 0, s>>>(in, n, tmp, ntiles, out); ms_count_launch();
}

}  // namespace
