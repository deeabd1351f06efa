// Graph build on the device: simple-graph normalisation (Sec. II-A), CSR
// (Sec. II-B) and the degree orientation that replaces the id-order upper
// triangle of Sec. II-C.
//
// Pipeline (all in device memory, ids are int32):
//  1. canon_degree  drop self-loops, count every non-loop pair at both ends
//                   (multigraph degree), flag ids outside [0, n)
//  2. rank          sort vertices by (degree, id): rank[v] = position
//  3. orient        every non-loop pair {u, v} becomes the oriented entry
//                   min(rank u, rank v) -> max(rank u, rank v); rows are filled by a
//                   counting sort on the source rank
//  4. segsort       each row is sorted (bitonic networks in a thread's or a warp's
//                   registers, in a block's shared memory or, for very long rows, in
//                   global memory) and repeated entries are removed;
//                   the simple-graph degree of every vertex is its distinct
//                   out-entries plus its in-entries before deduplication minus the
//                   repeats dropped at it
// Any strict total order finds each triangle once; the (degree, id) order keeps
// every oriented row short (d+(u) <= sqrt(2m)).  The degree used for the order is
// the count of non-loop input pairs at a vertex, which equals the simple degree
// unless the input repeats pairs; LCC always uses the simple degree.
#include <climits>

#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {

namespace {

constexpr int THREADS = 256;
constexpr int WARP_SORT_MAX = 1024;   // rows up to this length: one warp, registers
constexpr int CTA_SORT_MAX = 16384;   // rows up to this length: one block, shared memory
constexpr int SEG_WARPS = 8;          // warps per block in the warp sorter

// CSR offsets check: offsets[0] == 0, non-decreasing, offsets[n] <= limit.
__global__ void k_check_offsets(const int64_t* __restrict__ offsets, int32_t n, int64_t limit, DevStats* stats) {
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        if (offsets[i + 1] < offsets[i]) bad = 1;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (offsets[0] != 0 || offsets[n] > limit || offsets[n] < 0)) bad = 1;
    bad = __reduce_or_sync(FULL, bad);
    if (lane_id() == 0 && bad) atomicOr(&stats->err, ERR_BAD_OFFSETS);
}

// Row expansion of a CSR input: rows[k] = i for offsets[i] <= k < offsets[i+1].
// One warp per row.  Offsets must start at 0 and not decrease.
__global__ void k_expand_csr(const int64_t* __restrict__ offsets, int32_t n, int32_t* __restrict__ rows,
                             DevStats* stats) {
    const int lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        int64_t a = offsets[i], b = offsets[i + 1];
        if (b < a || a < 0) {
            if (lane == 0) atomicOr(&stats->err, ERR_BAD_OFFSETS);
            continue;
        }
        for (int64_t k = a + lane; k < b; k += 32) rows[k] = (int32_t)i;
    }
}

// Multigraph degree counts.  Each block keeps the counts of the vertices it meets
// first in a shared-memory hash table (open addressing, at most DEG_PROBES slots
// looked at); hub vertices occur often enough to take a slot early, so their many
// increments stay in shared memory and reach dmulti with one atomic per block.
// Vertices that find no slot add to dmulti directly.
constexpr int PAIR_UNROLL = 8;  // pairs per thread and round in the pair passes
constexpr int DEG_SLOTS = 4096;
constexpr int DEG_PROBES = 4;

__device__ __forceinline__ void deg_add(int32_t x, int32_t* hk, uint32_t* hc, uint32_t* __restrict__ dmulti) {
    unsigned h = ((unsigned)x * 0x9e3779b1u) >> (32 - 12);
#pragma unroll
    for (int k = 0; k < DEG_PROBES; ++k) {
        int32_t cur = hk[h];
        if (cur == -1) cur = atomicCAS(&hk[h], -1, x);
        if (cur == -1 || cur == x) {
            atomicAdd(&hc[h], 1u);
            return;
        }
        h = (h + 1) & (DEG_SLOTS - 1);
    }
    atomicAdd(&dmulti[x], 1u);
}

__global__ void __launch_bounds__(THREADS) k_canon_degree(const int32_t* __restrict__ src,
                                                          const int32_t* __restrict__ dst, int64_t m, int32_t n,
                                                          uint32_t* __restrict__ dmulti, DevStats* stats) {
    static_assert(DEG_SLOTS == 1 << 12, "hash width");
    __shared__ int32_t hk[DEG_SLOTS];
    __shared__ uint32_t hc[DEG_SLOTS];
    for (int i = threadIdx.x; i < DEG_SLOTS; i += blockDim.x) {
        hk[i] = -1;
        hc[i] = 0;
    }
    __syncthreads();
    unsigned long long loops = 0;
    int err = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < m; i0 += PAIR_UNROLL * stride) {
        int32_t a[PAIR_UNROLL], c[PAIR_UNROLL];
#pragma unroll
        for (int k = 0; k < PAIR_UNROLL; ++k) {
            const int64_t i = i0 + k * stride;
            a[k] = i < m ? src[i] : 0;
            c[k] = i < m ? dst[i] : 0;
        }
#pragma unroll
        for (int k = 0; k < PAIR_UNROLL; ++k) {
            if (i0 + k * stride >= m) break;
            if ((uint32_t)a[k] >= (uint32_t)n || (uint32_t)c[k] >= (uint32_t)n) {
                err = ERR_BAD_ID;
            } else if (a[k] == c[k]) {
                ++loops;
            } else {
                deg_add(a[k], hk, hc, dmulti);
                deg_add(c[k], hk, hc, dmulti);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < DEG_SLOTS; i += blockDim.x)
        if (hc[i]) atomicAdd(&dmulti[hk[i]], hc[i]);
    loops = warp_sum(loops);
    err = __reduce_or_sync(FULL, err);
    if (lane_id() == 0) {
        if (loops) atomicAdd(&stats->loops, loops);
        if (err) atomicOr(&stats->err, err);
    }
}

__global__ void k_max_deg(const uint32_t* __restrict__ dmulti, int32_t n, DevStats* stats) {
    uint32_t mx = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        mx = max(mx, dmulti[i]);
    mx = __reduce_max_sync(FULL, mx);
    if (lane_id() == 0 && mx) atomicMax(&stats->max_deg, mx);
}

__global__ void k_rank_keys(const uint32_t* __restrict__ dmulti, int32_t n, uint64_t* __restrict__ keys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        keys[i] = ((uint64_t)dmulti[i] << 32) | (uint32_t)i;
}

// rank[id] = position in (degree, id) order; dmulti is rewritten in rank space
// (dmulti_rank[r] = degree of the vertex of rank r, the high word of its key).
__global__ void k_rank_invert(const uint64_t* __restrict__ sorted, int32_t n, int32_t* __restrict__ rank,
                              uint32_t* __restrict__ dmulti) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const uint64_t key = sorted[r];
        rank[(uint32_t)key] = (int32_t)r;
        dmulti[r] = (uint32_t)(key >> 32);
    }
}

// Both passes take PAIR_UNROLL pairs per thread and round (pair i0 + k * stride), so
// that the loads, the rank gathers and the atomics of the pairs are in flight
// together instead of one dependent chain per pair.  The count pass keeps every
// pair's oriented form (source rank, target rank) in input order ((-1, -1): a loop
// or a bad id), so the scatter pass reads it back in order instead of gathering the
// two ranks again; the scatter's cursors start at the rows' first slots, so one
// atomic gives the slot.
__global__ void k_orient_count(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                               int32_t n, const int32_t* __restrict__ rank, uint32_t* __restrict__ rowcnt,
                               int2* __restrict__ oriented, bool dir_bits) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < m; i0 += PAIR_UNROLL * stride) {
        int32_t u[PAIR_UNROLL], v[PAIR_UNROLL];
#pragma unroll
        for (int k = 0; k < PAIR_UNROLL; ++k) {
            const int64_t i = i0 + k * stride;
            u[k] = i < m ? src[i] : 0;
            v[k] = i < m ? dst[i] : 0;
        }
        // every pair's two rank gathers first, so that they are in flight together
        int32_t a[PAIR_UNROLL], b[PAIR_UNROLL];
#pragma unroll
        for (int k = 0; k < PAIR_UNROLL; ++k) {
            const bool ok = i0 + k * stride < m && u[k] != v[k] && (uint32_t)u[k] < (uint32_t)n &&
                            (uint32_t)v[k] < (uint32_t)n;
            a[k] = ok ? rank[u[k]] : -1;
            b[k] = ok ? rank[v[k]] : -1;
        }
#pragma unroll
        for (int k = 0; k < PAIR_UNROLL; ++k) {
            const int64_t i = i0 + k * stride;
            if (i >= m) break;
            int2 o = make_int2(-1, -1);
            if (a[k] >= 0) {
                o = make_int2(min(a[k], b[k]), max(a[k], b[k]));
                if (dir_bits) o.y = (o.y << 2) | (a[k] < b[k] ? 1 : 2);
                atomicAdd(&rowcnt[o.x], 1u);
            }
            oriented[i] = o;
        }
    }
}

__global__ void k_orient_scatter(const int2* __restrict__ oriented, int64_t m,
                                 uint32_t* __restrict__ cursor, int32_t* __restrict__ col,
                                 DevStats* stats) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int err = 0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < m; i0 += PAIR_UNROLL * stride) {
        int2 o[PAIR_UNROLL];
#pragma unroll
        for (int k = 0; k < PAIR_UNROLL; ++k) {
            const int64_t i = i0 + k * stride;
            o[k] = i < m ? oriented[i] : make_int2(-1, -1);
        }
        uint32_t p[PAIR_UNROLL];
#pragma unroll
        for (int k = 0; k < PAIR_UNROLL; ++k) p[k] = o[k].x >= 0 ? atomicAdd(&cursor[o[k].x], 1u) : 0u;
#pragma unroll
        for (int k = 0; k < PAIR_UNROLL; ++k) {
            if (o[k].x < 0) continue;
            if ((int64_t)p[k] < m)  // always true unless the passes disagree
                col[p[k]] = o[k].y;
            else
                err = ERR_OVERFLOW;
        }
    }
    err = __reduce_or_sync(FULL, err);
    if (err && lane_id() == 0) atomicOr(&stats->err, err);
}

// Row counts and row fill by buckets of consecutive source ranks (2^shift rows each,
// nb buckets), with no per-pair global atomic:
//  k_bucket_count  counts the pairs of each bucket (shared-memory histogram, one
//                  global atomic per bucket and block) and keeps every pair's
//                  (source rank, target rank), read back in input order;
//  k_orient_part   takes PART_TILE pairs per block, groups them by bucket in shared
//                  memory, reserves each bucket's run with one atomic and writes
//                  (source, target) into the bucket's segment of `pairs`;
//  k_bucket_fill   takes one bucket per block: counts its rows in shared memory,
//                  scans them into rowstart and rowcnt, and moves every pair into its
//                  row through shared-memory cursors.
// Used for flat degree distributions when a bucket's rows fit in shared memory
// (BUCKET_ROWS_MAX) and nb is at most BUCKET_MAX.  Skewed graphs take the direct
// count and scatter above: their heavy rows would pile onto a few buckets and onto
// single shared-memory counters, while in the direct scatter they stay in cache.
constexpr int PART_ITEMS = 16;
constexpr int PART_THREADS = 1024;  // large tiles: one reservation per bucket and 16384 pairs
constexpr int PART_TILE = PART_THREADS * PART_ITEMS;
constexpr int FILL_THREADS = 1024;

__global__ void __launch_bounds__(THREADS) k_bucket_count(const int32_t* __restrict__ src,
                                                          const int32_t* __restrict__ dst, int64_t m, int32_t n,
                                                          const int32_t* __restrict__ rank, int shift, int nb,
                                                          uint32_t* __restrict__ bcount, int2* __restrict__ oriented,
                                                          bool dir_bits) {
    extern __shared__ uint32_t hist[];  // nb
    for (int b = threadIdx.x; b < nb; b += THREADS) hist[b] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < m; i0 += PAIR_UNROLL * stride) {
        int32_t u[PAIR_UNROLL], v[PAIR_UNROLL];
#pragma unroll
        for (int k = 0; k < PAIR_UNROLL; ++k) {
            const int64_t i = i0 + k * stride;
            u[k] = i < m ? src[i] : 0;
            v[k] = i < m ? dst[i] : 0;
        }
#pragma unroll
        for (int k = 0; k < PAIR_UNROLL; ++k) {
            const int64_t i = i0 + k * stride;
            if (i >= m) break;
            int2 o = make_int2(-1, -1);  // loop or invalid id: no entry
            if (u[k] != v[k] && (uint32_t)u[k] < (uint32_t)n && (uint32_t)v[k] < (uint32_t)n) {
                const int32_t a = rank[u[k]], b = rank[v[k]];
                o = make_int2(min(a, b), max(a, b));
                if (dir_bits) o.y = (o.y << 2) | (a < b ? 1 : 2);
                atomicAdd(&hist[o.x >> shift], 1u);
            }
            oriented[i] = o;  // the partition pass reads these instead of gathering ranks again
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += THREADS)
        if (hist[b]) atomicAdd(&bcount[b], hist[b]);
}

__global__ void __launch_bounds__(PART_THREADS) k_orient_part(const int2* __restrict__ oriented, int64_t m,
                                                         int shift, int nb, const int64_t* __restrict__ bstart,
                                                         uint32_t* __restrict__ bcur, int2* __restrict__ pairs,
                                                         DevStats* stats) {
    extern __shared__ __align__(8) unsigned char part_sh[];
    int64_t* base = reinterpret_cast<int64_t*>(part_sh);  // nb
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + nb);  // nb
    for (int64_t t0 = (int64_t)blockIdx.x * PART_TILE; t0 < m; t0 += (int64_t)gridDim.x * PART_TILE) {
        for (int b = threadIdx.x; b < nb; b += PART_THREADS) hist[b] = 0;
        __syncthreads();
        int32_t sv[PART_ITEMS], tv[PART_ITEMS];
        uint32_t loc[PART_ITEMS];
#pragma unroll
        for (int k = 0; k < PART_ITEMS; ++k) {
            const int64_t i = t0 + (int64_t)k * PART_THREADS + threadIdx.x;
            sv[k] = -1;
            if (i < m) {
                const int2 o = oriented[i];
                sv[k] = o.x;
                tv[k] = o.y;
                if (o.x >= 0) loc[k] = atomicAdd(&hist[o.x >> shift], 1u);
            }
        }
        __syncthreads();
        for (int b = threadIdx.x; b < nb; b += PART_THREADS) {
            const uint32_t c = hist[b];
            if (c) base[b] = bstart[b] + atomicAdd(&bcur[b], c);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PART_ITEMS; ++k)
            if (sv[k] >= 0) {
                const int b = sv[k] >> shift;
                const int64_t pos = base[b] + loc[k];
                if (pos < bstart[b + 1])  // always true unless the two passes disagree
                    pairs[pos] = make_int2(sv[k], tv[k]);
                else
                    atomicOr(&stats->err, ERR_OVERFLOW);
            }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(FILL_THREADS) k_bucket_fill(int32_t n, int shift, int nb,
                                                              const int64_t* __restrict__ bstart,
                                                              const int2* __restrict__ pairs,
                                                              int64_t* __restrict__ rowstart,
                                                              uint32_t* __restrict__ rowcnt, int32_t* __restrict__ col,
                                                              DevStats* stats) {
    extern __shared__ uint32_t rc[];  // 2^shift row counters, then row cursors
    __shared__ uint32_t part[FILL_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int32_t r0 = b << shift;
        const int nr = (int)min((int64_t)1 << shift, (int64_t)n - r0);
        const int64_t e0 = bstart[b], e1 = bstart[b + 1];
        for (int i = threadIdx.x; i < nr; i += FILL_THREADS) rc[i] = 0;
        __syncthreads();
        for (int64_t e = e0 + threadIdx.x; e < e1; e += FILL_THREADS) {
            const int r = pairs[e].x - r0;
            if ((unsigned)r < (unsigned)nr)
                atomicAdd(&rc[r], 1u);
            else
                atomicOr(&stats->err, ERR_OVERFLOW);
        }
        __syncthreads();
        // exclusive scan of rc[0, nr): thread k sums rows [k*per, (k+1)*per)
        const int per = (nr + FILL_THREADS - 1) / FILL_THREADS;
        const int i0 = min(threadIdx.x * per, nr), i1 = min(i0 + per, nr);
        uint32_t sum = 0;
        for (int i = i0; i < i1; ++i) sum += rc[i];
        const uint32_t inc = warp_inclusive_scan(sum);
        if (lane == 31) part[w] = inc;
        __syncthreads();
        if (w == 0) {
            const uint32_t pv = lane < FILL_THREADS / 32 ? part[lane] : 0u;
            const uint32_t pi = warp_inclusive_scan(pv);
            if (lane < FILL_THREADS / 32) part[lane] = pi - pv;
        }
        __syncthreads();
        uint32_t run = part[w] + inc - sum;
        for (int i = i0; i < i1; ++i) {
            const uint32_t c = rc[i];
            rowstart[r0 + i] = e0 + run;
            rowcnt[r0 + i] = c;
            rc[i] = run;
            run += c;
        }
        __syncthreads();
        for (int64_t e = e0 + threadIdx.x; e < e1; e += FILL_THREADS) {
            const int2 st = pairs[e];
            const int r = st.x - r0;
            if ((unsigned)r < (unsigned)nr) col[e0 + atomicAdd(&rc[r], 1u)] = st.y;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rowstart[n] = bstart[nb];
}

// Simple degree in rank space: distinct out-entries + in-entries before
// deduplication (non-loop pairs at v minus those where v is the source) - repeats
// dropped at v.  dmulti, rowcnt, rowlen and dupin are all indexed by rank here.
__global__ void k_degree(int32_t n, const int32_t* __restrict__ rowlen, const uint32_t* __restrict__ dmulti,
                         const uint32_t* __restrict__ rowcnt, const uint32_t* __restrict__ dupin,
                         int32_t* __restrict__ deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        deg[v] = rowlen[v] + (int32_t)(dmulti[v] - rowcnt[v]) - (int32_t)dupin[v];
}

struct WarpSync {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Bitonic sorting network over P (power of two) elements of `s`, ascending, in the
// form where every comparator sends the minimum to the lower index: the first
// comparator layer of each merge compares mirrored positions, the later layers are
// half-cleaners.  Padding with INT_MAX at the end is therefore inert.  `lanes`
// workers with ids `me` share the work; `sync` orders the layers.
template <typename Sync>
__device__ __forceinline__ void bitonic_sort(int32_t* s, int P, int me, int lanes, Sync sync) {
    for (int k = 2; k <= P; k <<= 1) {
        const int half = k >> 1;
        for (int i = me; i < (P >> 1); i += lanes) {
            int blk = i / half, off = i - blk * half;
            int lo = blk * k + off, hi = blk * k + k - 1 - off;
            int32_t x = s[lo], y = s[hi];
            if (x > y) {
                s[lo] = y;
                s[hi] = x;
            }
        }
        sync();
        for (int j = half >> 1; j >= 1; j >>= 1) {
            for (int i = me; i < (P >> 1); i += lanes) {
                int blk = i / j, off = i - blk * j;
                int lo = blk * 2 * j + off, hi = lo + j;
                int32_t x = s[lo], y = s[hi];
                if (x > y) {
                    s[lo] = y;
                    s[hi] = x;
                }
            }
            sync();
        }
    }
}

// Same network on a global-memory row of arbitrary length len (virtual +inf
// padding up to the next power of two): comparators touching a padded slot are
// skipped.
__device__ void bitonic_sort_global(int32_t* s, int len, int me, int lanes) {
    const int P = next_pow2_int(len);
    for (int k = 2; k <= P; k <<= 1) {
        const int half = k >> 1;
        for (int i = me; i < (P >> 1); i += lanes) {
            int blk = i / half, off = i - blk * half;
            int lo = blk * k + off, hi = blk * k + k - 1 - off;
            if (hi < len) {
                int32_t x = s[lo], y = s[hi];
                if (x > y) {
                    s[lo] = y;
                    s[hi] = x;
                }
            }
        }
        __syncthreads();
        for (int j = half >> 1; j >= 1; j >>= 1) {
            for (int i = me; i < (P >> 1); i += lanes) {
                int blk = i / j, off = i - blk * j;
                int lo = blk * 2 * j + off, hi = lo + j;
                if (hi < len) {
                    int32_t x = s[lo], y = s[hi];
                    if (x > y) {
                        s[lo] = y;
                        s[hi] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Sorting network on N registers (bitonic, all indices known at compile time).
template <int N>
__device__ __forceinline__ void reg_bitonic(int32_t (&v)[N]) {
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const int32_t a = v[i], b = v[l];
                    if ((i & k) == 0) {
                        v[i] = min(a, b);
                        v[l] = max(a, b);
                    } else {
                        v[i] = max(a, b);
                        v[l] = min(a, b);
                    }
                }
            }
        }
    }
}

// Sorts a row of len <= N entries in registers, writes the distinct entries back
// to its start and counts each dropped repeat at its target; returns how many were kept.
template <int N>
__device__ __forceinline__ int sort_row_regs(int32_t* __restrict__ row, int len, uint32_t* __restrict__ dupin) {
    int32_t v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = i < len ? row[i] : INT_MAX;
    reg_bitonic<N>(v);
    int kept = 0;
    int32_t prev = INT_MIN;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i < len) {
            if (v[i] != prev)
                row[kept++] = v[i];
            else if (dupin)
                atomicAdd(&dupin[v[i]], 1u);
        }
        prev = v[i];
    }
    return kept;
}

// One thread per row for rows of at most 16 entries; longer rows are listed for the
// warp sorter (<= WARP_SORT_MAX) or the block sorter.
__global__ void __launch_bounds__(256) k_segsort_thread(int32_t n, const int64_t* __restrict__ rowstart,
                                                        const uint32_t* __restrict__ rowcnt, int32_t* __restrict__ col,
                                                        int32_t* __restrict__ rowlen, int2* __restrict__ rowinfo,
                                                        uint32_t* __restrict__ dupin, int32_t* __restrict__ midlist,
                                                        int32_t* __restrict__ midlist2, int32_t* __restrict__ longlist,
                                                        DevStats* stats) {
    unsigned long long kept_total = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // the loop bound is uniform across a warp, as warp_append needs all 32 lanes
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < n; b += stride) {
        const int64_t r = b + lane_id();
        const int len = r < n ? (int)rowcnt[r] : 0;
        const bool mid = len > 16 && len <= 256, mid2 = len > 256 && len <= WARP_SORT_MAX, lng = len > WARP_SORT_MAX;
        const unsigned pm = warp_append(mid, &stats->mid_count);
        const unsigned pm2 = warp_append(mid2, &stats->mid2_count);
        const unsigned pl = warp_append(lng, &stats->long_count);
        if (mid) midlist[pm] = (int32_t)r;
        if (mid2) midlist2[pm2] = (int32_t)r;
        if (lng) longlist[pl] = (int32_t)r;
        if (r < n && len <= 16) {
            const int64_t base = rowstart[r];
            const int kept = len <= 8 ? sort_row_regs<8>(col + base, len, dupin) : sort_row_regs<16>(col + base, len, dupin);
            rowlen[r] = kept;
            rowinfo[r] = make_int2((int)base, kept);
            kept_total += (unsigned long long)kept;
        }
    }
    kept_total = warp_sum(kept_total);
    if (lane_id() == 0 && kept_total) atomicAdd(&stats->m_simple, kept_total);
}

// Bitonic network over the 32*K entries a warp holds in registers, lane L holding
// entries L*K .. L*K + K - 1 (ascending overall when done).  Comparator partners
// closer than K sit in the same lane; farther partners are exchanged with shfl_xor.
template <int K>
__device__ __forceinline__ void warp_reg_sort(int32_t (&v)[K], int lane) {
    constexpr int N = 32 * K;
#pragma unroll
    for (int s = 2; s <= N; s <<= 1) {
#pragma unroll
        for (int j = s >> 1; j > 0; j >>= 1) {
            if (j < K) {
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    if ((r & j) == 0) {
                        const int e = lane * K + r;
                        const bool asc = (e & s) == 0;
                        const int32_t a = v[r], b = v[r | j];
                        v[r] = asc ? min(a, b) : max(a, b);
                        v[r | j] = asc ? max(a, b) : min(a, b);
                    }
                }
            } else {
                const int lm = j / K;
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    const int e = lane * K + r;
                    const int32_t w = __shfl_xor_sync(FULL, v[r], lm);
                    const bool asc = (e & s) == 0;
                    const bool lower = (e & j) == 0;
                    v[r] = (asc == lower) ? min(v[r], w) : max(v[r], w);
                }
            }
        }
    }
}

// Sorts one row of len <= 32 K entries with a warp, writes the distinct entries
// back to the row's start, counts dropped repeats at their targets; returns the
// number kept (all lanes).
template <int K>
__device__ __forceinline__ int warp_sort_row(int32_t* __restrict__ row, int len, uint32_t* __restrict__ dupin,
                                             int lane) {
    int32_t v[K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const int e = lane * K + r;
        v[r] = e < len ? row[e] : INT_MAX;
    }
    warp_reg_sort<K>(v, lane);
    int32_t prev = __shfl_up_sync(FULL, v[K - 1], 1);
    if (lane == 0) prev = INT_MIN;
    unsigned keepmask = 0;
    int nk = 0;
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const int e = lane * K + r;
        if (e < len) {
            if (v[r] != prev) {
                keepmask |= 1u << r;
                ++nk;
            } else if (dupin) {
                atomicAdd(&dupin[v[r]], 1u);
            }
        }
        prev = v[r];
    }
    const int incl = warp_inclusive_scan(nk);
    const int total = __shfl_sync(FULL, incl, 31);
    __syncwarp();  // every lane has read its entries before any is overwritten
    int pos = incl - nk;
#pragma unroll
    for (int r = 0; r < K; ++r)
        if (keepmask & (1u << r)) row[pos++] = v[r];
    return total;
}

// One warp per listed row, sorted in registers: MAXK = 8 takes the rows of 17..256
// entries, MAXK = 32 those of 257..1024 (separate kernels keep the register budget
// of the short classes small).
template <int MAXK>
__global__ void __launch_bounds__(SEG_WARPS * 32) k_segsort_warp(const int64_t* __restrict__ rowstart,
                                                                 const uint32_t* __restrict__ rowcnt,
                                                                 int32_t* __restrict__ col, int32_t* __restrict__ rowlen,
                                                                 int2* __restrict__ rowinfo, uint32_t* __restrict__ dupin,
                                                                 const int32_t* __restrict__ list,
                                                                 const unsigned* __restrict__ count, DevStats* stats) {
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const unsigned nrows = *count;
    const unsigned warps = gridDim.x * SEG_WARPS;
    unsigned long long kept_total = 0;
    for (unsigned q = blockIdx.x * SEG_WARPS + w; q < nrows; q += warps) {
        const int32_t r = list[q];
        const int len = (int)rowcnt[r];
        const int64_t base = rowstart[r];
        int32_t* row = col + base;
        int kept;
        if (MAXK <= 8) {
            if (len <= 32)
                kept = warp_sort_row<1>(row, len, dupin, lane);
            else if (len <= 64)
                kept = warp_sort_row<2>(row, len, dupin, lane);
            else if (len <= 128)
                kept = warp_sort_row<4>(row, len, dupin, lane);
            else
                kept = warp_sort_row<8>(row, len, dupin, lane);
        } else if (MAXK <= 16) {
            kept = warp_sort_row<16>(row, len, dupin, lane);
        } else {
            if (len <= 512)
                kept = warp_sort_row<16>(row, len, dupin, lane);
            else
                kept = warp_sort_row<32>(row, len, dupin, lane);
        }
        if (lane == 0) {
            rowlen[r] = kept;
            rowinfo[r] = make_int2((int)base, kept);
            kept_total += (unsigned long long)kept;
        }
        __syncwarp();
    }
    if (lane == 0 && kept_total) atomicAdd(&stats->m_simple, kept_total);
}

// One block per long row: shared-memory network up to CTA_SORT_MAX, global-memory
// network beyond; then in-place compaction of repeated entries.
__global__ void __launch_bounds__(1024) k_segsort_block(const int64_t* __restrict__ rowstart,
                                                        const uint32_t* __restrict__ rowcnt,
                                                        int32_t* __restrict__ col, int32_t* __restrict__ rowlen,
                                                        int2* __restrict__ rowinfo, uint32_t* __restrict__ dupin,
                                                        const int32_t* __restrict__ longlist,
                                                        DevStats* stats) {
    extern __shared__ int32_t sh[];  // CTA_SORT_MAX entries
    __shared__ int wk[32];
    __shared__ int32_t boundary;
    const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned nlong = stats->long_count;
    for (unsigned q = blockIdx.x; q < nlong; q += gridDim.x) {
        const int32_t r = longlist[q];
        const int len = (int)rowcnt[r];
        const int64_t base = rowstart[r];
        int32_t* s;
        if (len <= CTA_SORT_MAX) {
            const int P = next_pow2_int(len);
            for (int i = threadIdx.x; i < P; i += blockDim.x) sh[i] = i < len ? col[base + i] : INT_MAX;
            __syncthreads();
            bitonic_sort(sh, P, threadIdx.x, blockDim.x, BlockSync());
            s = sh;
        } else {
            bitonic_sort_global(col + base, len, threadIdx.x, blockDim.x);
            s = col + base;
        }
        // compaction in chunks of blockDim; the last element of the previous chunk
        // is kept in `boundary` because in-place writes may overwrite it.
        int kept = 0;
        if (threadIdx.x == 0) boundary = 0;
        __syncthreads();
        for (int c = 0; c < len; c += blockDim.x) {
            int i = c + threadIdx.x;
            int32_t x = i < len ? s[i] : 0;
            int32_t prev = (i > 0 && threadIdx.x > 0 && i < len) ? s[i - 1] : boundary;
            bool keep = i < len && (i == 0 || x != prev);
            unsigned mk = __ballot_sync(FULL, keep);
            if (lane == 0) wk[w] = __popc(mk);
            __syncthreads();
            int before = 0, tot = 0;
            for (int k = 0; k < nw; ++k) {
                before += k < w ? wk[k] : 0;
                tot += wk[k];
            }
            int32_t last = s[min(c + (int)blockDim.x, len) - 1];
            __syncthreads();
            if (keep)
                col[base + kept + before + __popc(mk & lanemask_lt())] = x;
            else if (i < len && dupin)
                atomicAdd(&dupin[x], 1u);
            kept += tot;
            if (threadIdx.x == 0) boundary = last;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            rowlen[r] = kept;
            rowinfo[r] = make_int2((int)base, kept);
            atomicAdd(&stats->m_simple, (unsigned long long)kept);
        }
        __syncthreads();
    }
}

}  // namespace

void launch_check_offsets(const int64_t* offsets, int32_t n, int64_t limit, DevStats* stats, const Launch& L) {
    k_check_offsets<<<grid_for(n + 1, THREADS, L.sms), THREADS, 0, L.stream>>>(offsets, n, limit, stats); count_launch();
}

void launch_expand_csr(const int64_t* offsets, int32_t n, int32_t* rows, DevStats* stats, const Launch& L) {
    if (n <= 0) return;
    k_expand_csr<<<grid_for((int64_t)n * 32, THREADS, L.sms), THREADS, 0, L.stream>>>(offsets, n, rows, stats); count_launch();
}

void launch_canon_degree_part(const BuildBuffers& B, int64_t first, int64_t count, const Launch& L) {
    if (count <= 0) return;
    // 32 KB of shared memory per block: four blocks per SM stay resident
    k_canon_degree<<<grid_for(count, THREADS, L.sms, 4), THREADS, 0, L.stream>>>(B.src + first, B.dst + first, count,
                                                                               B.n, B.dmulti, B.stats);
    count_launch();
}

void launch_max_deg(const BuildBuffers& B, const Launch& L) {
    if (B.n > 0) { k_max_deg<<<grid_for(B.n, THREADS, L.sms), THREADS, 0, L.stream>>>(B.dmulti, B.n, B.stats); count_launch(); }
}

void launch_canon_degree(const BuildBuffers& B, const Launch& L) {
    launch_canon_degree_part(B, 0, B.m, L);
    launch_max_deg(B, L);
}

// Batches: the graph of every vertex (one warp per graph), then keys
// (graph, degree, local id) whose stable sort on the graph and degree fields ranks the
// vertices graph by graph.
__global__ void k_seg_of(const int32_t* __restrict__ vbase, int32_t G, uint32_t* __restrict__ seg) {
    const int lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += warps)
        for (int64_t v = vbase[g] + lane; v < vbase[g + 1]; v += 32) seg[v] = (uint32_t)g;
}

__global__ void k_rank_keys_seg(const uint32_t* __restrict__ dmulti, const uint32_t* __restrict__ seg,
                                const int32_t* __restrict__ vbase, int32_t n, int deg_bits, int local_bits,
                                uint64_t* __restrict__ keys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t g = seg[i];
        keys[i] = ((uint64_t)g << (deg_bits + local_bits)) | ((uint64_t)dmulti[i] << local_bits) |
                  (uint64_t)(i - vbase[g]);
    }
}

__global__ void k_rank_invert_seg(const uint64_t* __restrict__ sorted, const int32_t* __restrict__ vbase, int32_t n,
                                  int deg_bits, int local_bits, int32_t* __restrict__ rank,
                                  uint32_t* __restrict__ dmulti) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t lmask = (1ull << local_bits) - 1, dmask = (1ull << deg_bits) - 1;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const uint64_t key = sorted[r];
        const int64_t g = (int64_t)(key >> (deg_bits + local_bits));
        rank[vbase[g] + (int64_t)(key & lmask)] = (int32_t)r;
        dmulti[r] = (uint32_t)((key >> local_bits) & dmask);
    }
}

void launch_rank(const BuildBuffers& B, int deg_bits, const Launch& L) {
    if (B.n <= 0) return;
    if (B.seg_vbase && B.seg_count > 0 && B.seg_bits + B.seg_deg_bits + B.local_bits <= 64) {
        uint32_t* seg = B.cursor;  // free until the row fill
        k_seg_of<<<grid_for((int64_t)B.seg_count * 32, THREADS, L.sms), THREADS, 0, L.stream>>>(B.seg_vbase,
                                                                                               B.seg_count, seg);
        count_launch();
        k_rank_keys_seg<<<grid_for(B.n, THREADS, L.sms), THREADS, 0, L.stream>>>(B.dmulti, seg, B.seg_vbase, B.n,
                                                                               B.seg_deg_bits, B.local_bits, B.keys);
        count_launch();
        uint64_t* sorted = radix_sort_u64(B.keys, B.keys_alt, B.n, B.local_bits,
                                          B.local_bits + B.seg_deg_bits + B.seg_bits, B.tmp, L);
        k_rank_invert_seg<<<grid_for(B.n, THREADS, L.sms), THREADS, 0, L.stream>>>(
            sorted, B.seg_vbase, B.n, B.seg_deg_bits, B.local_bits, B.rank, B.dmulti);
        count_launch();
        return;
    }
    k_rank_keys<<<grid_for(B.n, THREADS, L.sms), THREADS, 0, L.stream>>>(B.dmulti, B.n, B.keys); count_launch();
    // the keys start in id order, so a stable sort on the degree bits yields (degree, id)
    uint64_t* sorted = radix_sort_u64(B.keys, B.keys_alt, B.n, 32, 32 + deg_bits, B.tmp, L);
    k_rank_invert<<<grid_for(B.n, THREADS, L.sms), THREADS, 0, L.stream>>>(sorted, B.n, B.rank, B.dmulti); count_launch();
}

void bucket_shape(int32_t n, int* shift, int* nb) {
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < (int64_t)n) ++bits;
    int sh = bits - BUCKET_BITS;
    if (sh < 0) sh = 0;
    if (((int64_t)1 << sh) > BUCKET_ROWS_MAX) sh = 0;
    while (((int64_t)1 << sh) < BUCKET_ROWS_MAX && (((int64_t)n + ((int64_t)1 << sh) - 1) >> sh) > BUCKET_MAX) ++sh;
    const int64_t b = ((int64_t)n + ((int64_t)1 << sh) - 1) >> sh;
    *shift = sh;
    *nb = b <= BUCKET_MAX ? (int)b : 0;  // 0: too many rows for the bucket path
}

void launch_orient(const BuildBuffers& B, const Launch& L, cudaEvent_t* ev, const PlanStreams* ps) {
    if (B.n <= 0) return;
    cudaMemsetAsync(B.cursor, 0, sizeof(uint32_t) * (size_t)B.n, L.stream);
    cudaMemsetAsync(B.dupin, 0, sizeof(uint32_t) * (size_t)B.n, L.stream);
    int shift = 0, nb = 0;
    bucket_shape(B.n, &shift, &nb);
    if (B.bucket_fill && nb > 0) {
        cudaMemsetAsync(B.bcount, 0, sizeof(uint32_t) * (size_t)nb, L.stream);
        cudaMemsetAsync(B.bcur, 0, sizeof(uint32_t) * (size_t)nb, L.stream);
        if (B.m > 0) {
            k_bucket_count<<<grid_for(B.m, THREADS * PAIR_UNROLL, L.sms, 8), THREADS, sizeof(uint32_t) * nb, L.stream>>>(
                B.src, B.dst, B.m, B.n, B.rank, shift, nb, B.bcount, B.oriented, B.dir_bits);
            count_launch();
        }
        scan_u32_to_i64(B.bcount, B.bstart, nb, B.tmp, L);
        if (ev) cudaEventRecord(ev[BP_COUNT], L.stream);
        if (B.m > 0) {
            k_orient_part<<<grid_for(B.m, PART_TILE, L.sms, 1), PART_THREADS, (sizeof(int64_t) + sizeof(uint32_t)) * nb,
                            L.stream>>>(B.oriented, B.m, shift, nb, B.bstart, B.bcur, B.pairs, B.stats);
            count_launch();
        }
        const int fill_blocks = nb < 4 * L.sms ? nb : 4 * L.sms;
        k_bucket_fill<<<fill_blocks, FILL_THREADS, sizeof(uint32_t) << shift, L.stream>>>(
            B.n, shift, nb, B.bstart, B.pairs, B.rowstart, B.rowcnt, B.col, B.stats);
        count_launch();
    } else {
        cudaMemsetAsync(B.rowcnt, 0, sizeof(uint32_t) * (size_t)B.n, L.stream);
        if (B.m > 0) {
            k_orient_count<<<grid_for(B.m, THREADS, L.sms), THREADS, 0, L.stream>>>(B.src, B.dst, B.m, B.n, B.rank,
                                                                                  B.rowcnt, B.oriented, B.dir_bits);
            count_launch();
        }
        scan_u32_to_i64(B.rowcnt, B.rowstart, B.n, B.tmp, L);
        if (ev) cudaEventRecord(ev[BP_COUNT], L.stream);
        if (B.m > 0) {
            // 32-bit cursors in the rank keys' buffer (free once the ranks are known),
            // starting at every row's first slot (slots stay below m <= 2^31 - 1)
            scan_u32_to_u32(B.rowcnt, reinterpret_cast<uint32_t*>(B.keys), B.n, B.tmp, L);
            k_orient_scatter<<<grid_for(B.m, THREADS, L.sms), THREADS, 0, L.stream>>>(
                B.oriented, B.m, reinterpret_cast<uint32_t*>(B.keys), B.col, B.stats);
            count_launch();
        }
    }
    if (ev) cudaEventRecord(ev[BP_FILL], L.stream);
    // with direction bits the entries are not ranks: repeats are not counted at targets
    uint32_t* const dupin = B.dir_bits ? nullptr : B.dupin;
    k_segsort_thread<<<grid_for(B.n, THREADS, L.sms), THREADS, 0, L.stream>>>(
        B.n, B.rowstart, B.rowcnt, B.col, B.rowlen, B.rowinfo, dupin, B.midlist, B.midlist2, B.longlist, B.stats);
    count_launch();
    // the three sorters take disjoint rows: with a second stream the long rows are
    // sorted there while the main stream sorts the rows of 17..256
    Launch S = L;
    if (ps) {
        cudaEventRecord(ps->fork, L.stream);
        cudaStreamWaitEvent(ps->side, ps->fork, 0);
        S.stream = ps->side;
    }
    k_segsort_warp<WARP_SORT_MAX / 32><<<S.sms * 2, SEG_WARPS * 32, 0, S.stream>>>(B.rowstart, B.rowcnt, B.col,
                                                                                  B.rowlen, B.rowinfo, dupin,
                                                                                  B.midlist2, &B.stats->mid2_count,
                                                                                  B.stats);
    count_launch();
    k_segsort_block<<<S.sms * 2, 1024, CTA_SORT_MAX * sizeof(int32_t), S.stream>>>(
        B.rowstart, B.rowcnt, B.col, B.rowlen, B.rowinfo, dupin, B.longlist, B.stats);
    count_launch();
    if (ps) cudaEventRecord(ps->join, S.stream);
    k_segsort_warp<8><<<L.sms * 4, SEG_WARPS * 32, 0, L.stream>>>(B.rowstart, B.rowcnt, B.col, B.rowlen, B.rowinfo,
                                                                 dupin, B.midlist, &B.stats->mid_count, B.stats);
    count_launch();
    if (ps) cudaStreamWaitEvent(L.stream, ps->join, 0);
    if (ev) cudaEventRecord(ev[BP_SORT], L.stream);
    k_degree<<<grid_for(B.n, THREADS, L.sms), THREADS, 0, L.stream>>>(B.n, B.rowlen, B.dmulti, B.rowcnt, B.dupin,
                                                                     B.deg);
    count_launch();
}

// Dynamic shared memory: 64 KB for the block sorter, up to BUCKET_ROWS_MAX row
// counters for the bucket fill and BUCKET_MAX buckets for the partition pass.
cudaError_t build_init_attributes() {
    cudaError_t e = cudaFuncSetAttribute(k_segsort_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         CTA_SORT_MAX * (int)sizeof(int32_t));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_bucket_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             BUCKET_ROWS_MAX * (int)sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_orient_part, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             BUCKET_MAX * (int)(sizeof(int64_t) + sizeof(uint32_t)));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_bucket_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                BUCKET_MAX * (int)sizeof(uint32_t));
}

}  // namespace tcg
