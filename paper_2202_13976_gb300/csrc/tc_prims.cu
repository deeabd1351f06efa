// Device-wide primitives: exclusive scan and a stable LSD radix sort.
#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-wide exclusive scan of one value per thread; returns the exclusive prefix
// and writes the block total to *total.
template <typename T>
__device__ T block_exclusive_scan(T v, T* total) {
    __shared__ T warp_tot[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_inclusive_scan(v);
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < SCAN_THREADS / 32 ? warp_tot[lane] : T(0);
        T wi = warp_inclusive_scan(w);
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - w;
        if (lane == SCAN_THREADS / 32 - 1) *total = wi;
    }
    __syncthreads();
    T out = warp_tot[warp] + inc - v;
    __syncthreads();
    return out;
}

template <typename In, typename Acc>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_reduce(const In* __restrict__ in, int64_t count,
                                                              Acc* __restrict__ partials) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    Acc s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < count) s += (Acc)in[i];
    }
    s = warp_sum(s);
    __shared__ Acc ws[SCAN_THREADS / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        Acc t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += ws[w];
        partials[blockIdx.x] = t;
    }
}

// One block: exclusive scan of partials[0..num) in place; partials[num] = total.
template <typename Acc>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_partials(Acc* partials, int64_t num) {
    __shared__ Acc carry_sh;
    Acc carry = 0;
    for (int64_t base = 0; base < num; base += SCAN_TILE) {
        Acc v[SCAN_ITEMS];
        Acc s = 0;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
            v[k] = i < num ? partials[i] : Acc(0);
            s += v[k];
        }
        Acc tot;
        Acc ex = block_exclusive_scan(s, &carry_sh);
        tot = carry_sh;
        Acc run = carry + ex;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
            if (i < num) partials[i] = run;
            run += v[k];
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[num] = carry;
}

template <typename In, typename Out, typename Acc>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const In* in, Out* out, int64_t count,
                                                            const Acc* __restrict__ partials,
                                                            int64_t num_tiles) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    Acc v[SCAN_ITEMS];
    Acc s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        v[k] = i < count ? (Acc)in[i] : Acc(0);
        s += v[k];
    }
    __shared__ Acc tot;
    Acc run = partials[blockIdx.x] + block_exclusive_scan(s, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        if (i < count) out[i] = (Out)run;
        run += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[count] = (Out)partials[num_tiles];
}

template <typename In, typename Out, typename Acc>
void scan_impl(const In* in, Out* out, int64_t count, void* tmp, const Launch& L) {
    int64_t tiles = (count + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles < 1) tiles = 1;
    Acc* partials = static_cast<Acc*>(tmp);
    k_tile_reduce<In, Acc><<<(unsigned)tiles, SCAN_THREADS, 0, L.stream>>>(in, count, partials); count_launch();
    k_scan_partials<Acc><<<1, SCAN_THREADS, 0, L.stream>>>(partials, tiles); count_launch();
    k_tile_scan<In, Out, Acc><<<(unsigned)tiles, SCAN_THREADS, 0, L.stream>>>(in, out, count, partials, tiles); count_launch();
}

// ---- radix sort --------------------------------------------------------------

constexpr int RADIX_THREADS = 256;
constexpr int RADIX_WARPS = RADIX_THREADS / 32;
constexpr int RADIX_ITEMS = 8;
constexpr int RADIX_TILE = RADIX_THREADS * RADIX_ITEMS;  // 2048 keys
constexpr int RADIX_BINS = 256;

// Key index of item k of this thread: warp w owns 256 consecutive keys; item k of
// lane l is key w*256 + k*32 + l.  Loads are coalesced and, within a warp, the
// (item, lane) order is the input order.
__device__ __forceinline__ int64_t radix_index(int64_t tile_base, int k) {
    return tile_base + (threadIdx.x >> 5) * (32 * RADIX_ITEMS) + k * 32 + (threadIdx.x & 31);
}

__global__ void __launch_bounds__(RADIX_THREADS) k_radix_hist(const uint64_t* __restrict__ keys,
                                                              int64_t count, int shift, int bits,
                                                              uint32_t* __restrict__ hist,
                                                              int64_t tiles) {
    __shared__ uint32_t h[RADIX_BINS];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RADIX_TILE;
    const uint64_t mask = (1ull << bits) - 1;
#pragma unroll
    for (int k = 0; k < RADIX_ITEMS; ++k) {
        int64_t i = radix_index(base, k);
        if (i < count) atomicAdd(&h[(keys[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RADIX_THREADS) k_radix_scatter(const uint64_t* __restrict__ in,
                                                                 uint64_t* __restrict__ out,
                                                                 int64_t count, int shift, int bits,
                                                                 const uint32_t* __restrict__ offs,
                                                                 int64_t tiles) {
    __shared__ uint32_t wcnt[RADIX_WARPS][RADIX_BINS];
    for (int i = threadIdx.x; i < RADIX_WARPS * RADIX_BINS; i += RADIX_THREADS)
        (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * RADIX_TILE;
    const uint64_t mask = (1ull << bits) - 1;
    uint64_t key[RADIX_ITEMS];
    int dig[RADIX_ITEMS];
    uint32_t pos[RADIX_ITEMS];
#pragma unroll
    for (int k = 0; k < RADIX_ITEMS; ++k) {
        int64_t i = radix_index(base, k);
        bool valid = i < count;
        key[k] = valid ? in[i] : 0;
        // invalid lanes get a private value so they never join a digit group
        int d = valid ? (int)((key[k] >> shift) & mask) : RADIX_BINS + lane;
        dig[k] = d;
        unsigned peers = __match_any_sync(FULL, d);
        uint32_t before = valid ? wcnt[warp][d] : 0;
        pos[k] = before + __popc(peers & lanemask_lt());
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // exclusive prefix over warps, one digit per thread
        uint32_t run = 0;
        for (int w = 0; w < RADIX_WARPS; ++w) {
            uint32_t c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RADIX_ITEMS; ++k) {
        int64_t i = radix_index(base, k);
        if (i < count) {
            int d = dig[k];
            uint32_t p = offs[(int64_t)d * tiles + blockIdx.x] + wcnt[warp][d] + pos[k];
            out[p] = key[k];
        }
    }
}

}  // namespace

size_t scan_tmp_bytes(int64_t count) {
    int64_t tiles = (count + SCAN_TILE - 1) / SCAN_TILE + 2;
    return (size_t)tiles * 8 + 256;
}

void scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t count, void* tmp, const Launch& L) {
    scan_impl<uint32_t, int64_t, long long>(in, out, count, tmp, L);
}

void scan_u32_to_u32(const uint32_t* in, uint32_t* out, int64_t count, void* tmp, const Launch& L) {
    scan_impl<uint32_t, uint32_t, unsigned long long>(in, out, count, tmp, L);
}

size_t radix_tmp_bytes(int64_t count) {
    int64_t tiles = (count + RADIX_TILE - 1) / RADIX_TILE;
    if (tiles < 1) tiles = 1;
    size_t hist = (size_t)(RADIX_BINS * tiles + 1) * 4;
    hist = (hist + 255) & ~(size_t)255;
    return hist + scan_tmp_bytes(RADIX_BINS * tiles);
}

uint64_t* radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t count, int lo, int hi, void* tmp,
                         const Launch& L) {
    if (count <= 1 || hi <= lo) return keys;
    int64_t tiles = (count + RADIX_TILE - 1) / RADIX_TILE;
    uint32_t* hist = static_cast<uint32_t*>(tmp);
    size_t hist_bytes = ((size_t)(RADIX_BINS * tiles + 1) * 4 + 255) & ~(size_t)255;
    void* scan_tmp = static_cast<char*>(tmp) + hist_bytes;
    uint64_t* a = keys;
    uint64_t* b = alt;
    for (int shift = lo; shift < hi; shift += 8) {
        int bits = hi - shift < 8 ? hi - shift : 8;
        k_radix_hist<<<(unsigned)tiles, RADIX_THREADS, 0, L.stream>>>(a, count, shift, bits, hist, tiles); count_launch();
        scan_u32_to_u32(hist, hist, RADIX_BINS * tiles, scan_tmp, L);
        k_radix_scatter<<<(unsigned)tiles, RADIX_THREADS, 0, L.stream>>>(a, b, count, shift, bits, hist, tiles); count_launch();
        uint64_t* t = a;
        a = b;
        b = t;
    }
    return a;
}

}  // namespace tcg
