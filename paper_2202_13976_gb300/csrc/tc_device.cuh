// Device helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tcg {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(FULL, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Inclusive warp scan.
template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T w = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += w;
    }
    return v;
}

// Appends `want` (per lane) to a global list with one atomic per warp; returns the
// lane's slot (valid only where want is true).  All 32 lanes must call it.
__device__ __forceinline__ unsigned warp_append(bool want, unsigned* counter) {
    unsigned mask = __ballot_sync(FULL, want);
    unsigned base = 0;
    int leader = __ffs(mask) - 1;
    if (mask && lane_id() == leader) base = atomicAdd(counter, (unsigned)__popc(mask));
    base = __shfl_sync(FULL, base, leader < 0 ? 0 : leader);
    return base + __popc(mask & lanemask_lt());
}

// First index in [lo, hi) of sorted a[] whose value is >= x.
template <typename P>
__device__ __forceinline__ int lower_bound(P a, int lo, int hi, int x) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__host__ __device__ __forceinline__ int next_pow2_int(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace tcg
