// tc_count_noalloc: the whole count for a small graph in one kernel launch, with
// every intermediate array in a fixed device array of this file, so that the call
// allocates no memory at all.
//
// Who needs it: code that must not allocate device memory while it runs, for
// example a caller that has handed all free HBM to its own caching allocator, or
// real-time code that forbids allocation after start-up.  The call reads its status
// words back to the host and synchronises the caller's stream before it returns.
//
// The scratch array below is reserved on every GPU that loads the library for as
// long as the process lives (TC_NOALLOC_SCRATCH_BYTES); with lazy module loading the
// runtime places it during the first call on each device, so that call belongs at
// start-up, before the free memory is handed to another allocator.  All calls share it and it
// keeps the previous call's contents; the kernel clears what it needs before use.
// Calls whose work overlaps on the GPU (two streams, or two host threads) race on
// it and give wrong results: the caller must order them.
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <mutex>

#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {
namespace {

constexpr int NA_THREADS = 1024;
constexpr int NA_WARPS = NA_THREADS / 32;
constexpr int64_t NA_MAX_N = TC_NOALLOC_MAX_N;
constexpr int64_t NA_MAX_M = TC_NOALLOC_MAX_M;

// Layout of the scratch array, in 8-byte words.
constexpr int64_t W_CTL = 0;                        // [0] error flags, [1] pairs, [2] distinct edges, [3] sum t
constexpr int64_t W_KEYS = 16;                      // NA_MAX_M pair keys
constexpr int64_t W_VKEYS = W_KEYS + NA_MAX_M;      // NA_MAX_N vertex keys
constexpr int64_t W_T = W_VKEYS + NA_MAX_N;         // NA_MAX_N per-rank counts
constexpr int64_t W_I32 = W_T + NA_MAX_N;           // 32-bit arrays from here
constexpr int64_t I_COL = 0;                        // NA_MAX_M
constexpr int64_t I_ROWSTART = I_COL + NA_MAX_M;    // NA_MAX_N + 1
constexpr int64_t I_ROWLEN = I_ROWSTART + NA_MAX_N + 2;
constexpr int64_t I_DMULTI = I_ROWLEN + NA_MAX_N;
constexpr int64_t I_RANK = I_DMULTI + NA_MAX_N;
constexpr int64_t I_DEG = I_RANK + NA_MAX_N;
constexpr int64_t I_END = I_DEG + NA_MAX_N;
constexpr int64_t NA_WORDS = W_I32 + (I_END + 1) / 2;
static_assert(NA_WORDS * 8 == TC_NOALLOC_SCRATCH_BYTES, "scratch size stated in include/tc.h");

static __device__ __align__(256) unsigned long long g_noalloc_scratch[NA_WORDS];

// Exclusive scan of one value per thread across the block; *total receives the sum.
__device__ int block_scan_excl(int x, int* warp_tot, int* total) {
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int inc = warp_inclusive_scan(x);
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int v = warp_tot[lane];
        const int vi = warp_inclusive_scan(v);
        warp_tot[lane] = vi - v;
        if (lane == 31) *total = vi;
    }
    __syncthreads();
    const int out = warp_tot[w] + inc - x;
    __syncthreads();
    return out;
}

// Ascending bitonic network over a[0, len) with virtual +inf padding to a power of
// two: every comparator sends the minimum to the lower index, so padded slots are
// never touched.
__device__ void block_sort_u64(unsigned long long* a, int len) {
    const int P = next_pow2_int(len > 1 ? len : 1);
    for (int k = 2; k <= P; k <<= 1) {
        const int half = k >> 1;
        for (int i = threadIdx.x; i < (P >> 1); i += NA_THREADS) {
            const int blk = i / half, off = i - blk * half;
            const int lo = blk * k + off, hi = blk * k + k - 1 - off;
            if (hi < len) {
                const unsigned long long x = a[lo], y = a[hi];
                if (x > y) {
                    a[lo] = y;
                    a[hi] = x;
                }
            }
        }
        __syncthreads();
        for (int j = half >> 1; j >= 1; j >>= 1) {
            for (int i = threadIdx.x; i < (P >> 1); i += NA_THREADS) {
                const int blk = i / j, off = i - blk * j;
                const int lo = blk * 2 * j + off, hi = lo + j;
                if (hi < len) {
                    const unsigned long long x = a[lo], y = a[hi];
                    if (x > y) {
                        a[lo] = y;
                        a[hi] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// One block.  Same definitions as the multi-kernel path: self-loops and repeated
// pairs dropped, (degree, id) ranks, oriented rows sorted, t[u] += c, t[v] += c and
// t[w] += 1 for every common neighbour w of the suffix of N+(u) after v and N+(v),
// LCC by Eq. 2 with the simple degree.
__global__ void __launch_bounds__(NA_THREADS) k_tc_noalloc(int32_t n, int32_t m, const int32_t* __restrict__ src,
                                                           const int32_t* __restrict__ dst,
                                                           unsigned long long* __restrict__ S,
                                                           unsigned long long* __restrict__ t_out,
                                                           double* __restrict__ lcc_out) {
    __shared__ int warp_tot[NA_WARPS];
    __shared__ int total;
    __shared__ unsigned long long boundary;
    unsigned long long* ctl = S + W_CTL;
    unsigned long long* keys = S + W_KEYS;
    unsigned long long* vkeys = S + W_VKEYS;
    unsigned long long* t = S + W_T;
    int32_t* I = reinterpret_cast<int32_t*>(S + W_I32);
    int32_t* col = I + I_COL;
    int32_t* rowstart = I + I_ROWSTART;
    int32_t* rowlen = I + I_ROWLEN;
    uint32_t* dmulti = reinterpret_cast<uint32_t*>(I + I_DMULTI);
    int32_t* rank = I + I_RANK;
    int32_t* deg = I + I_DEG;
    const int tid = threadIdx.x;

    // clear what the previous call left behind
    if (tid < 16) ctl[tid] = 0;
    for (int v = tid; v < n; v += NA_THREADS) {
        t[v] = 0;
        dmulti[v] = 0;
        rowlen[v] = 0;
        deg[v] = 0;
    }
    __syncthreads();
    // degrees of the multigraph (non-loop pairs), id check
    for (int i = tid; i < m; i += NA_THREADS) {
        const int32_t u = src[i], v = dst[i];
        if ((uint32_t)u >= (uint32_t)n || (uint32_t)v >= (uint32_t)n) {
            atomicOr(&ctl[0], (unsigned long long)ERR_BAD_ID);
        } else if (u != v) {
            atomicAdd(&dmulti[u], 1u);
            atomicAdd(&dmulti[v], 1u);
        }
    }
    __syncthreads();
    if (ctl[0] != 0) return;
    // ranks in (degree, id) order
    for (int v = tid; v < n; v += NA_THREADS) vkeys[v] = ((unsigned long long)dmulti[v] << 32) | (uint32_t)v;
    __syncthreads();
    block_sort_u64(vkeys, n);
    for (int r = tid; r < n; r += NA_THREADS) rank[(uint32_t)vkeys[r]] = r;
    __syncthreads();
    // oriented pair keys (lower rank << 32 | higher rank), sorted
    for (int i = tid; i < m; i += NA_THREADS) {
        const int32_t u = src[i], v = dst[i];
        if (u != v) {
            const unsigned long long a = (unsigned long long)rank[u], b = (unsigned long long)rank[v];
            const unsigned long long p = atomicAdd(&ctl[1], 1ull);
            keys[p] = a < b ? (a << 32) | b : (b << 32) | a;
        }
    }
    __syncthreads();
    const int mp = (int)ctl[1];
    block_sort_u64(keys, mp);
    // distinct keys, compacted in place, in order; rows are contiguous and sorted
    if (tid == 0) boundary = ~0ull;
    __syncthreads();
    int kept = 0;
    for (int c = 0; c < mp; c += NA_THREADS) {
        const int i = c + tid;
        const unsigned long long x = i < mp ? keys[i] : 0ull;
        const unsigned long long prev = (i > 0 && tid > 0 && i < mp) ? keys[i - 1] : boundary;
        const bool keep = i < mp && (i == 0 || x != prev);
        const unsigned long long last = keys[min(c + NA_THREADS, mp) - 1];
        const int pos = block_scan_excl(keep ? 1 : 0, warp_tot, &total);
        const int tot = total;
        if (keep) {
            const int32_t s = (int32_t)(x >> 32), d = (int32_t)(x & 0xffffffffu);
            keys[kept + pos] = x;
            col[kept + pos] = d;
            atomicAdd(&rowlen[s], 1);
            atomicAdd(&deg[s], 1);
            atomicAdd(&deg[d], 1);
        }
        kept += tot;
        if (tid == 0) boundary = last;
        __syncthreads();
    }
    const int mu = kept;
    // row starts: exclusive scan of rowlen
    int carry = 0;
    for (int c = 0; c < n; c += NA_THREADS) {
        const int v = c + tid;
        const int len = v < n ? rowlen[v] : 0;
        const int pos = block_scan_excl(len, warp_tot, &total);
        if (v < n) rowstart[v] = carry + pos;
        carry += total;
    }
    if (tid == 0) {
        rowstart[n] = carry;
        ctl[2] = (unsigned long long)mu;
    }
    __syncthreads();
    // one thread per oriented edge (u, v): Alg. 2 over the suffix of N+(u) after v and N+(v)
    for (int k = tid; k < mu; k += NA_THREADS) {
        const int32_t u = (int32_t)(keys[k] >> 32), v = col[k];
        int i = k + 1;
        const int iend = rowstart[u] + rowlen[u];
        int j = rowstart[v];
        const int jend = j + rowlen[v];
        unsigned long long c = 0;
        while (i < iend && j < jend) {
            const int32_t a = col[i], b = col[j];
            if (a == b) {
                atomicAdd(&t[a], 1ull);
                ++c;
                ++i;
                ++j;
            } else if (a < b) {
                ++i;
            } else {
                ++j;
            }
        }
        if (c) {
            atomicAdd(&t[u], c);
            atomicAdd(&t[v], c);
        }
    }
    __syncthreads();
    // outputs in the caller's ids; sum of t for T
    unsigned long long s = 0;
    for (int v = tid; v < n; v += NA_THREADS) {
        const int32_t r = rank[v];
        const unsigned long long tv = t[r];
        s += tv;
        if (t_out) t_out[v] = tv;
        if (lcc_out) {
            const long long d = deg[r];
            lcc_out[v] = d < 2 ? 0.0 : __ddiv_rn((double)(2ull * tv), (double)(d * (d - 1)));
        }
    }
    s = warp_sum(s);
    if (lane_id() == 0 && s) atomicAdd(&ctl[3], s);
}

std::mutex g_na_mutex;
unsigned long long* g_na_ptr[64] = {};

}  // namespace
}  // namespace tcg

using namespace tcg;

extern "C" tc_status tc_count_noalloc(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                      uint64_t* T_out, uint64_t* t_out, double* lcc_out, void* cuda_stream) {
    if (!T_out || n < 0 || m < 0 || (m > 0 && (!src || !dst))) return TC_EINVAL;
    if (n > NA_MAX_N || m > NA_MAX_M) return TC_EINVAL;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return TC_ECUDA;
    unsigned long long* S = nullptr;
    {
        // Once per device, with that device current: the device address of the
        // scratch array (its name in host code is not a device address).
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return TC_ECUDA;
            g_na_ptr[dev] = static_cast<unsigned long long*>(p);
        }
        S = g_na_ptr[dev];
    }
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    k_tc_noalloc<<<1, NA_THREADS, 0, stream>>>(n, (int32_t)m, src, dst, S, reinterpret_cast<unsigned long long*>(t_out),
                                               lcc_out);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return TC_ECUDA;
    unsigned long long ctl[4] = {0, 0, 0, 0};
    e = cudaMemcpyAsync(ctl, S + W_CTL, sizeof(ctl), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return TC_ECUDA;
    if (ctl[0] & ERR_BAD_ID) return TC_EINVAL;
    if (ctl[3] % 3 != 0) return TC_EINTERNAL;
    *T_out = ctl[3] / 3;
    return TC_OK;
}
