// Per-edge set intersection over the degree-oriented CSR (Sec. II-C, Sec. IV-C),
// the planner that splits the edges into buckets, and the final reduction to T
// (Sec. II-C) and LCC (Eq. 2).
//
// Counting rule.  Vertices are ranked by (degree, id) and every oriented row N+(u)
// is sorted and holds only ranks above u.  For the oriented edge (u, v) with
// v = N+(u)[j], the common neighbours are W = N+(u)[j+1 ..] ∩ N+(v): every element
// of N+(v) exceeds v, so only the suffix of N+(u) after v can match.  With c = |W|,
// a triangle {u, v, w} (u < v < w in rank order) is met exactly once, and t[u] += c,
// t[v] += c, t[w] += 1 for every w in W.
//
// Buckets (each oriented edge belongs to exactly one):
//  hub    edges into the highest-ranked vertices ("hubs").  One thread block per hub
//         v stages N+(v) once in shared memory (a bitmap over its rank window with
//         per-word prefix counts, or the sorted list), then streams the suffix
//         N+(u)[j+1 ..] of every in-edge (u, v) against it.  This is the on-chip
//         analogue of the paper's caching of remote adjacency lists ranked by degree
//         (Sec. IV-B, Observations 1 and 2): the list that most edges need is read
//         from memory once and reused by all of them.  t[w] increments are summed
//         per position of N+(v) in shared memory and flushed once per hub.
//  small  other edges whose source has 2 <= |N+(u)| <= 32: a group of 8, 16 or 32
//         lanes stages N+(u); lane j intersects edge j sequentially, by SSI (Alg. 2)
//         or binary search (Alg. 1), chosen per edge by Eq. 3.
//  block  other edges whose source has |N+(u)| > 32: one thread block stages N+(u),
//         one warp per edge, methods:
//           MERGE   merge path: the merge of A (suffix) and B = N+(v) is cut into 32
//                   equal diagonal ranges, one per lane, each running Alg. 2
//           SEARCH  every key of A is looked up in B by binary search (Alg. 1)
//           PROBE   every element of B is looked up in A (shared memory) by binary
//                   search; the scan of B stops above max N+(u)
//           BITMAP  like PROBE against a bitmap of N+(u) over its rank window
//           AUTO    Eq. 3 per edge: merge if |B|/|A| <= f (log2|B| - 1) (|A| <= |B|),
//                   else the keys of the shorter list are searched in the longer
#include <climits>

#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {

namespace {

constexpr int THREADS = 256;
constexpr int SMALL_WARPS = 8;         // warps per block in the small-bucket kernel
constexpr int SMALL_BLOCKS = 8;        // its resident blocks per SM (the grid is one wave of them)
constexpr int SMALL_WIDE_MAX = 256;    // longest N+(u) the warp-per-source kernel stages
constexpr int HASH_CUT = 64;           // rows longer than this are cut at max N+(u) by the hash kernel
constexpr int CTA_THREADS = 256;       // block push kernel
constexpr int CTA_WARPS = CTA_THREADS / 32;
constexpr int CTA_LIST_MAX = 2048;     // staged list capacity of the block push kernel
constexpr int BITMAP_WORDS = 4096;     // its bitmap window: 131072 ranks
constexpr int HUB_THREADS = 256;
constexpr int HUB_WARPS = HUB_THREADS / 32;
constexpr int HUB_BM_WORDS = HUB_BM_BITS / 32;
constexpr int HUB_CNT_MAX = 1024;      // hub lists longer than this count matches globally
constexpr int HUB_BLOCKS = 6;          // resident blocks of the hub kernel per SM (registers and shared memory)
constexpr int HUB_WARP_MAX = 256;      // longest N+(v) a single warp stages
constexpr int HUB_HASH_LOAD = 2;       // its hash table has at least this many slots per key
constexpr int HUB_HASH_MAX = HUB_HASH_LOAD * HUB_WARP_MAX;
constexpr int SCAT_STEPS = 4;          // lockstep steps of the row-walk scatter in flight together
constexpr int HUB_BATCH = 32;          // in-edges per batch of a big hub
constexpr int HUB_LONG = 16;           // suffixes at least this long are read by lane groups
constexpr int HUB_GROUPS = 4;          // long suffixes one warp reads at a time
constexpr int HUB_GLANES = 32 / HUB_GROUPS;
constexpr int HUB_UNROLL = 8;          // entries a lane reads per round of a long suffix

struct Sink {
    uint32_t* cnt;               // per-position counters (shared), or null
    unsigned long long* t;       // global counts, used when cnt is null
    const int32_t* Lu;           // N+(u) (shared or global)
    uint32_t* supA;              // per-edge support of the entries of N+(u) when cnt is null, or null
    uint32_t* supB;              // per-edge support of the entries of N+(v), or null
    __device__ __forceinline__ void hit(int p) const {
        if (cnt) {
            atomicAdd(&cnt[p], 1u);
        } else {
            atomicAdd(&t[Lu[p]], 1ull);
            if (supA) atomicAdd(&supA[p], 1u);
        }
    }
    __device__ __forceinline__ void hitB(int k) const {
        if (supB) atomicAdd(&supB[k], 1u);
    }
};

// Number of elements of sorted B[0, b) that are <= x.
__device__ __forceinline__ int count_le(const int32_t* __restrict__ B, int b, int32_t x) {
    int lo = 0, hi = b;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (B[mid] <= x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool eq3_prefers_merge(int a, int b, float factor) {
    int s = min(a, b), l = max(a, b);
    return (float)l <= factor * (log2f((float)l) - 1.0f) * (float)s;
}

// Lane-per-edge choice between the batched merge and binary search: Eq. 3, except
// that an N+(v) of at most 16 entries (two 8-entry loads of the merge) is always
// merged, since one merge round costs less than the dependent loads of a search.
__device__ __forceinline__ int small_auto(int a, int dv, float factor) {
    return dv <= 16 || eq3_prefers_merge(a, dv, factor) || dv < a ? TC_STRAT_MERGE : TC_STRAT_SEARCH;
}

// ---- warp-cooperative methods (block push kernel) -----------------------------

__device__ uint32_t edge_merge(const Sink& S, int a0, int du, const int32_t* __restrict__ B, int b) {
    const int lane = lane_id();
    const int32_t* A = S.Lu + a0;
    const int a = du - a0;
    b = count_le(B, b, A[a - 1]);  // elements of B above max(A) cannot match
    const int64_t total = (int64_t)a + b;
    const int d0 = (int)((total * lane) >> 5);
    const int d1 = (int)((total * (lane + 1)) >> 5);
    int lo = max(0, d0 - b), hi = min(d0, a);
    while (lo < hi) {  // A elements among the first d0 merged items (ties: A first)
        int mid = (lo + hi) >> 1;
        if (A[mid] <= B[d0 - mid - 1])
            lo = mid + 1;
        else
            hi = mid;
    }
    int i = lo, j = d0 - lo;
    int32_t bj = j < b ? B[j] : INT_MAX;
    uint32_t c = 0;
    for (int step = d0; step < d1; ++step) {
        if (i < a && A[i] <= bj) {
            if (A[i] == bj) {
                S.hit(a0 + i);
                S.hitB(j);
                ++c;
            }
            ++i;
        } else {
            ++j;
            bj = j < b ? B[j] : INT_MAX;
        }
    }
    return warp_sum(c);
}

__device__ uint32_t edge_search(const Sink& S, int a0, int du, const int32_t* __restrict__ B, int b) {
    const int lane = lane_id();
    uint32_t c = 0;
    int lo = 0;
    for (int k = a0 + lane; k < du; k += 32) {
        int32_t y = S.Lu[k];
        int p = lower_bound(B, lo, b, y);
        lo = p;  // keys of this lane increase
        if (p < b && B[p] == y) {
            S.hit(k);
            S.hitB(p);
            ++c;
        }
    }
    return warp_sum(c);
}

__device__ uint32_t edge_probe(const Sink& S, int a0, int du, const int32_t* __restrict__ B, int b) {
    const int lane = lane_id();
    const int32_t maxu = S.Lu[du - 1];
    uint32_t c = 0;
    for (int k0 = 0; k0 < b; k0 += 32) {
        int k = k0 + lane;
        int32_t x = k < b ? B[k] : INT_MAX;
        if (x <= maxu) {
            int p = lower_bound(S.Lu, a0, du, x);
            if (S.Lu[p] == x) {  // p < du because x <= max
                S.hit(p);
                S.hitB(k);
                ++c;
            }
        }
        if (__any_sync(FULL, x > maxu)) break;  // B is sorted: later chunks exceed too
    }
    return warp_sum(c);
}

// Bitmap over ranks (u, maxu]: bit (x - u - 1) set iff x in N+(u); pre[w] = number of
// set bits in the words before w, i.e. the position in N+(u) of the word's first member.
__device__ uint32_t edge_bitmap(const uint32_t* bm, const uint16_t* pre, int32_t u, int32_t maxu,
                                uint32_t* cnt, const int32_t* __restrict__ B, int b, uint32_t* __restrict__ supB) {
    const int lane = lane_id();
    uint32_t c = 0;
    for (int k0 = 0; k0 < b; k0 += 32) {
        int k = k0 + lane;
        int32_t x = k < b ? B[k] : INT_MAX;
        if (x <= maxu) {
            int off = x - u - 1;
            uint32_t w = bm[off >> 5], bit = 1u << (off & 31);
            if (w & bit) {
                atomicAdd(&cnt[pre[off >> 5] + __popc(w & (bit - 1))], 1u);
                if (supB) atomicAdd(&supB[k], 1u);
                ++c;
            }
        }
        if (__any_sync(FULL, x > maxu)) break;
    }
    return warp_sum(c);
}

__device__ __forceinline__ uint32_t edge_dispatch(int method, const Sink& S, int a0, int du,
                                                  const int32_t* __restrict__ B, int b) {
    switch (method) {
        case TC_STRAT_MERGE: return edge_merge(S, a0, du, B, b);
        case TC_STRAT_SEARCH: return edge_search(S, a0, du, B, b);
        default: return edge_probe(S, a0, du, B, b);
    }
}

// Builds the bitmap of the staged list L[0, d) over ranks (base, base + 32 W] and its
// per-word prefix counts; a whole block calls it.
template <int THREADS_>
__device__ void build_bitmap(uint32_t* bm, uint16_t* pre, uint32_t* slice, const int32_t* __restrict__ L, int d,
                             int32_t base, int W) {
    const int lane = lane_id(), w = threadIdx.x >> 5;
    constexpr int WARPS = THREADS_ / 32;
    for (int i = threadIdx.x; i < W; i += THREADS_) bm[i] = 0;
    __syncthreads();
    for (int p = threadIdx.x; p < d; p += THREADS_) {
        int off = L[p] - base - 1;
        atomicOr(&bm[off >> 5], 1u << (off & 31));
    }
    __syncthreads();
    // exclusive prefix of per-word popcounts: within 32-word slices (one warp each),
    // then over slice totals (warp 0), then the slice offsets are added
    const int slices = (W + 31) >> 5;
    for (int s = w; s < slices; s += WARPS) {
        const int i = s * 32 + lane;
        const int pc = i < W ? __popc(bm[i]) : 0;
        const int inc = warp_inclusive_scan(pc);
        if (i < W) pre[i] = (uint16_t)(inc - pc);
        if (lane == 31) slice[s] = (uint32_t)inc;
    }
    __syncthreads();
    if (w == 0) {
        uint32_t carry = 0;
        for (int c0 = 0; c0 < slices; c0 += 32) {
            const int i = c0 + lane;
            const uint32_t v = i < slices ? slice[i] : 0u;
            const uint32_t inc = warp_inclusive_scan(v);
            if (i < slices) slice[i] = carry + inc - v;
            carry += __shfl_sync(FULL, inc, 31);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += THREADS_) pre[i] = (uint16_t)(pre[i] + slice[i >> 5]);
    __syncthreads();
}

// ---- lane-sequential methods (small bucket) -----------------------------------
// A = Lu[a0, du) (shared, sorted), B = N+(v) (global, sorted).  A match at position
// p of Lu adds one to cnt[p].

__device__ uint32_t lane_merge(const int32_t* Lu, int a0, int du, const int32_t* __restrict__ B, int b,
                               uint32_t* cnt) {
    if (a0 >= du || b == 0) return 0;
    uint32_t c = 0;
    int i = a0, k = 0;
    int32_t x = Lu[i], y = B[0];
    for (;;) {
        if (x == y) {
            atomicAdd(&cnt[i], 1u);
            ++c;
            if (++i >= du || ++k >= b) break;
            x = Lu[i];
            y = B[k];
        } else if (x < y) {
            if (++i >= du) break;
            x = Lu[i];
        } else {
            if (++k >= b) break;
            y = B[k];
        }
    }
    return c;
}

// Merge with B read eight entries at a time (independent loads), A in shared memory.
__device__ uint32_t lane_merge_batched(const int32_t* Lu, int a0, int du, const int32_t* __restrict__ B, int b,
                                       uint32_t* cnt, uint32_t* __restrict__ supB) {
    uint32_t c = 0;
    int i = a0;
    const int32_t mx = Lu[du - 1];
    for (int k0 = 0; k0 < b && i < du; k0 += 8) {
        int32_t y[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) y[q] = k0 + q < b ? B[k0 + q] : INT_MAX;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            while (i < du && Lu[i] < y[q]) ++i;
            if (i < du && Lu[i] == y[q]) {
                atomicAdd(&cnt[i], 1u);
                if (supB) atomicAdd(&supB[k0 + q], 1u);
                ++c;
                ++i;
            }
        }
        if (y[7] >= mx) break;
    }
    return c;
}

// keys of A looked up in B
__device__ uint32_t lane_search(const int32_t* Lu, int a0, int du, const int32_t* __restrict__ B, int b,
                                uint32_t* cnt, uint32_t* __restrict__ supB) {
    uint32_t c = 0;
    int lo = 0;
    for (int i = a0; i < du && lo < b; ++i) {
        const int32_t x = Lu[i];
        const int p = lower_bound(B, lo, b, x);
        lo = p;
        if (p < b && B[p] == x) {
            atomicAdd(&cnt[i], 1u);
            if (supB) atomicAdd(&supB[p], 1u);
            ++c;
        }
    }
    return c;
}

// keys of B looked up in A
__device__ uint32_t lane_search_rev(const int32_t* Lu, int a0, int du, const int32_t* __restrict__ B, int b,
                                    uint32_t* cnt, uint32_t* __restrict__ supB) {
    uint32_t c = 0;
    int lo = a0;
    const int32_t mx = Lu[du - 1];
    for (int k = 0; k < b && lo < du; ++k) {
        const int32_t y = B[k];
        if (y > mx) break;
        const int p = lower_bound(Lu, lo, du, y);
        lo = p;
        if (p < du && Lu[p] == y) {
            atomicAdd(&cnt[p], 1u);
            if (supB) atomicAdd(&supB[k], 1u);
            ++c;
        }
    }
    return c;
}

// ---- planner -----------------------------------------------------------------

__global__ void k_hub_candidates(int32_t n, const int32_t* __restrict__ deg, int min_degree, DevStats* stats) {
    unsigned c = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride)
        c += deg[r] >= min_degree ? 1u : 0u;
    c = warp_sum(c);
    if (lane_id() == 0 && c) atomicAdd(&stats->hub_candidates, c);
}

__global__ void k_hub_count(int32_t hub_cap, int hub_max, int core_max, DevStats* stats) {
    unsigned k = stats->hub_candidates;
    k = min(k, (unsigned)hub_max);
    k = min(k, (unsigned)hub_cap);
    stats->hub_count = k;
    stats->core_n = min(k, (unsigned)core_max);
}

// In-degree d-(v) = deg(v) - d+(v) of every hub slot (0 for slots below the hubs),
// less the in-edges from the dense core, which the core count covers.
__global__ void k_hub_indeg(int32_t n, int32_t hub_cap, const int32_t* __restrict__ deg,
                            const int32_t* __restrict__ rowlen, const uint32_t* __restrict__ core_cnt,
                            uint32_t* __restrict__ cnt, DevStats* stats) {
    const int32_t R = n - (int32_t)stats->hub_count;
    const int32_t c0 = n - (int32_t)stats->core_n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hub_cap; i += stride) {
        const int32_t r = n - hub_cap + (int32_t)i;
        uint32_t d = r >= R ? (uint32_t)(deg[r] - rowlen[r]) : 0u;
        if (r >= c0) d -= core_cnt[r - c0];
        cnt[i] = d;
    }
}

// The hub in-edge records are written by tiles of entries (k_row_of, k_hub_scatter)
// when the hub in-edges are at least a quarter of the entries of the non-core rows,
// else by a walk over the rows' hub tails (k_hub_scatter_rows).  All three kernels
// are launched and read the choice from the planned counts.
__device__ __forceinline__ bool scatter_by_tiles(const int64_t* __restrict__ hub_start, int32_t hub_cap,
                                                 const int64_t* __restrict__ rowstart, int32_t c0) {
    return 4 * hub_start[hub_cap] >= rowstart[c0];
}

// Source row of every entry of the non-core rows (whole row capacity, so that the
// slots left free by deduplication also name a valid row).  A lane writes its own
// row when it holds at most 32 entries; longer rows are written by the whole warp.
__global__ void k_row_of(int32_t n, int32_t hub_cap, const int64_t* __restrict__ rowstart,
                         const int64_t* __restrict__ hub_start, int32_t* __restrict__ rowof, const DevStats* stats) {
    const int32_t c0 = n - (int32_t)stats->core_n;
    if (!scatter_by_tiles(hub_start, hub_cap, rowstart, c0)) return;
    const int lane = lane_id();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // the loop bound is uniform across a warp, as the ballot needs all 32 lanes
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < c0; b += stride) {
        const int64_t u = b + lane;
        const int64_t a0 = u < c0 ? rowstart[u] : 0, a1 = u < c0 ? rowstart[u + 1] : 0;
        const bool longrow = a1 - a0 > 32;
        if (!longrow)
            for (int64_t p = a0; p < a1; ++p) rowof[p] = (int32_t)u;
        unsigned lm = __ballot_sync(FULL, longrow);
        while (lm) {
            const int r = __ffs(lm) - 1;
            lm &= lm - 1;
            const int64_t ar = __shfl_sync(FULL, a0, r), br = __shfl_sync(FULL, a1, r);
            for (int64_t p = ar + lane; p < br; p += 32) rowof[p] = (int32_t)(b + r);
        }
    }
}

// Every oriented entry (u -> v) of a row outside the dense core with v a hub becomes
// an in-edge record of v: {u, index after v in N+(u), end of N+(u), 0}, one 16-byte
// store into v's segment.  Blocks take tiles of SCAT_TILE consecutive entries (16
// bytes per thread and load), so the work is spread evenly whatever the row lengths;
// entries in the slots deduplication left free are skipped.  The SCAT_TOP highest
// hubs, whose cursors every tile would contend for, are served per tile: shared-
// memory counters give each entry its offset, then one global atomic per hub and
// tile reserves the tile's run; the other hubs take their slot from a global
// cursor per entry.  Records of one tile stay together, nearly in source order.
constexpr int SCAT_THREADS = 256;
constexpr int SCAT_ITEMS = 8;  // entries per thread and tile (two 16-byte loads)
constexpr int SCAT_TILE = SCAT_THREADS * SCAT_ITEMS;
constexpr int SCAT_TOP = 2048;

__global__ void __launch_bounds__(SCAT_THREADS) k_hub_scatter(int32_t n, int32_t hub_cap,
                                                              const int64_t* __restrict__ rowstart,
                                                              const int2* __restrict__ rowinfo,
                                                              const int32_t* __restrict__ col,
                                                              const int32_t* __restrict__ rowof,
                                                              const int64_t* __restrict__ hub_start,
                                                              unsigned long long* __restrict__ cur,
                                                              int4* __restrict__ in_rec, int32_t src_lo,
                                                              int32_t src_hi, DevStats* stats) {
    __shared__ uint32_t lcnt[SCAT_TOP];
    __shared__ int64_t gbase[SCAT_TOP];
    const int32_t R = n - (int32_t)stats->hub_count;
    const int32_t c0 = n - (int32_t)stats->core_n;  // rows of the dense core are counted there
    const int top = min((int)stats->hub_count, SCAT_TOP);
    const int32_t T0 = n - top;  // top hubs: ranks T0 .. n-1 (all hubs)
    const int32_t H0 = n - hub_cap;  // rank of hub slot 0
    if (!scatter_by_tiles(hub_start, hub_cap, rowstart, c0)) return;
    const int64_t mend = rowstart[c0];
    const int64_t total = hub_start[hub_cap];
    for (int64_t t0 = (int64_t)blockIdx.x * SCAT_TILE; t0 < mend; t0 += (int64_t)gridDim.x * SCAT_TILE) {
        for (int h = threadIdx.x; h < top; h += SCAT_THREADS) lcnt[h] = 0;
        __syncthreads();
        int32_t x[SCAT_ITEMS], u[SCAT_ITEMS], end[SCAT_ITEMS];
        uint32_t loc[SCAT_ITEMS];
#pragma unroll
        for (int k = 0; k < SCAT_ITEMS / 4; ++k) {
            const int64_t e0 = t0 + ((int64_t)k * SCAT_THREADS + threadIdx.x) * 4;
            if (e0 + 3 < mend) {
                const int4 q = *reinterpret_cast<const int4*>(col + e0);
                x[4 * k] = q.x, x[4 * k + 1] = q.y, x[4 * k + 2] = q.z, x[4 * k + 3] = q.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) x[4 * k + j] = e0 + j < mend ? col[e0 + j] : -1;
            }
        }
#pragma unroll
        for (int e = 0; e < SCAT_ITEMS; ++e) {
            const int64_t p = t0 + ((int64_t)(e >> 2) * SCAT_THREADS + threadIdx.x) * 4 + (e & 3);
            if (x[e] >= R) {
                u[e] = rowof[p];
                const int2 ri = rowinfo[u[e]];
                end[e] = ri.x + ri.y;
                if (p >= end[e]) x[e] = -1;  // a slot freed by deduplication
                // a source outside the counted shard keeps its slot with an empty suffix
                if (u[e] < src_lo || u[e] >= src_hi) end[e] = (int32_t)(p + 1);
            }
        }
        // the slot reservations of all items first, so that their round trips overlap,
        // then the records of the hubs below the top ones
        unsigned long long gslot[SCAT_ITEMS];
#pragma unroll
        for (int e = 0; e < SCAT_ITEMS; ++e) {
            gslot[e] = 0;
            if (x[e] >= T0)
                loc[e] = atomicAdd(&lcnt[x[e] - T0], 1u);
            else if (x[e] >= R)
                gslot[e] = atomicAdd(&cur[x[e] - H0], 1ull);
        }
#pragma unroll
        for (int e = 0; e < SCAT_ITEMS; ++e) {
            if (x[e] < R || x[e] >= T0) continue;
            const int64_t p = t0 + ((int64_t)(e >> 2) * SCAT_THREADS + threadIdx.x) * 4 + (e & 3);
            if ((int64_t)gslot[e] < total)  // counts and entries disagree only on a bug: never write outside
                in_rec[gslot[e]] = make_int4(u[e], (int32_t)(p + 1), end[e], 0);
            else
                atomicOr(&stats->err, ERR_OVERFLOW);
        }
        __syncthreads();
        for (int h = threadIdx.x; h < top; h += SCAT_THREADS) {
            const uint32_t c = lcnt[h];
            if (c) gbase[h] = (int64_t)atomicAdd(&cur[T0 + h - H0], (unsigned long long)c);
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < SCAT_ITEMS; ++e) {
            if (x[e] < T0) continue;
            const int64_t p = t0 + ((int64_t)(e >> 2) * SCAT_THREADS + threadIdx.x) * 4 + (e & 3);
            const int64_t slot = gbase[x[e] - T0] + loc[e];
            if (slot < total)
                in_rec[slot] = make_int4(u[e], (int32_t)(p + 1), end[e], 0);
            else
                atomicOr(&stats->err, ERR_OVERFLOW);
        }
        __syncthreads();  // lcnt and gbase are reused by the next tile
    }
}

// After the scatter every hub's cursor must stand at the start of the next segment:
// a count and a scatter that disagree are reported instead of trusted.
__global__ void k_hub_cur_check(int32_t hub_cap, const int64_t* __restrict__ hub_start,
                                const unsigned long long* __restrict__ cur, DevStats* stats) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hub_cap; i += stride)
        if (cur[i] != (unsigned long long)hub_start[i + 1]) atomicOr(&stats->err, ERR_OVERFLOW);
}

// The same records when hub entries are a small share of the entries (flat degree
// distributions): a warp takes 32 consecutive rows (one per lane) and walks their
// hub tails from the end backwards in lockstep, so rows without a hub cost one
// load; the highest-ranked hubs end almost every row, so lanes that name the same
// hub in a step reserve their slots with one atomic.
__global__ void k_hub_scatter_rows(int32_t n, int32_t hub_cap, const int64_t* __restrict__ rowstart,
                                   const int32_t* __restrict__ rowlen, const int32_t* __restrict__ col,
                                   const int64_t* __restrict__ hub_start, unsigned long long* __restrict__ cur,
                                   int4* __restrict__ in_rec, int32_t src_lo, int32_t src_hi,
                                   DevStats* stats) {
    const int32_t R = n - (int32_t)stats->hub_count;
    const int32_t c0 = n - (int32_t)stats->core_n;  // rows of the dense core are counted there
    if (scatter_by_tiles(hub_start, hub_cap, rowstart, c0)) return;
    const int64_t total = hub_start[hub_cap];
    const int lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; w0 < c0; w0 += warps * 32) {
        const int64_t u = w0 + lane;
        const int du = u < c0 ? rowlen[u] : 0;
        const int64_t base = u < n ? rowstart[u] : 0;
        const bool inshard = u >= src_lo && u < src_hi;  // else its records get empty suffixes
        int p = du - 1;
        // SCAT_STEPS steps at a time: their loads, then their slot reservations, are
        // independent and in flight together.  Walking backwards, the hub entries of a
        // row come first, so a lane's active steps are a prefix.
        for (int step = 0;; step += SCAT_STEPS) {
            int32_t x[SCAT_STEPS];
#pragma unroll
            for (int j = 0; j < SCAT_STEPS; ++j) x[j] = p - j >= 0 ? col[base + p - j] : -1;
            if (!__any_sync(FULL, x[0] >= R)) break;
            unsigned peers[SCAT_STEPS];
            int64_t slot0[SCAT_STEPS];
#pragma unroll
            for (int j = 0; j < SCAT_STEPS; ++j) {
                const bool active = x[j] >= R;
                // the first steps meet the most contended (highest) hubs: aggregate them;
                // afterwards every lane reserves its own slot
                peers[j] = __match_any_sync(FULL, active && step + j < 16 ? x[j] : -1 - lane);
                slot0[j] = 0;
                if (active && lane == __ffs(peers[j]) - 1)
                    slot0[j] = (int64_t)atomicAdd(&cur[x[j] - (n - hub_cap)], (unsigned long long)__popc(peers[j]));
            }
#pragma unroll
            for (int j = 0; j < SCAT_STEPS; ++j) {
                slot0[j] = __shfl_sync(FULL, slot0[j], __ffs(peers[j]) - 1);
                if (x[j] >= R) {
                    const int64_t slot = slot0[j] + __popc(peers[j] & lanemask_lt());
                    if (slot < total)  // counts and entries disagree only on a bug: never write outside
                        in_rec[slot] = make_int4((int32_t)u, (int32_t)(base + p - j + 1),
                                                 inshard ? (int32_t)(base + du) : (int32_t)(base + p - j + 1), 0);
                    else
                        atomicOr(&stats->err, ERR_OVERFLOW);
                }
            }
            p = x[SCAT_STEPS - 1] >= R ? p - SCAT_STEPS : -1;
        }
    }
}

// Hub slot i (0 = highest rank) is big when its in-degree reaches big_in or its list
// is too long for one warp.
__global__ void k_hub_flags(int32_t n, const int32_t* __restrict__ rowlen, const uint32_t* __restrict__ indeg,
                            int32_t hub_cap, int big_in, uint32_t* __restrict__ big, DevStats* stats) {
    const int64_t K = stats->hub_count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += stride) {
        const int32_t v = n - 1 - (int32_t)i;
        const uint32_t din = indeg[v - (n - hub_cap)];
        big[i] = (din >= (uint32_t)big_in || rowlen[v] > HUB_WARP_MAX) && rowlen[v] > 0 && din > 0 ? 1u : 0u;
    }
}

// Ordered split of the hubs (highest rank first) into the big and medium lists.
__global__ void k_hub_lists(int32_t n, const uint32_t* __restrict__ big, const uint32_t* __restrict__ pos,
                            int32_t* __restrict__ big_list, int32_t* __restrict__ med_list, DevStats* stats) {
    const int64_t K = stats->hub_count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += stride) {
        const int32_t v = n - 1 - (int32_t)i;
        if (big[i])
            big_list[pos[i]] = v;
        else
            med_list[i - pos[i]] = v;
        if (i == K - 1) stats->hub_big = pos[i] + big[i];
    }
}

// Push lists: sources with at least one non-hub target and a non-empty suffix.  A
// block classifies PLAN_ITEMS vertices per thread and appends them with one global
// atomic per list and block (warp ballots, then shared-memory offsets), since one
// atomic per warp and list serialises on the four list counters.
constexpr int PLAN_ITEMS = 4;
constexpr int PLAN_LISTS = 5;  // d+ classes <= 8, <= 16, <= 32, <= SMALL_WIDE_MAX, larger

__global__ void __launch_bounds__(THREADS) k_plan(int32_t n, const int64_t* __restrict__ rowstart,
                                                  const int32_t* __restrict__ rowlen, const int32_t* __restrict__ col,
                                                  int32_t* __restrict__ l8, int32_t* __restrict__ l16,
                                                  int32_t* __restrict__ l32, int32_t* __restrict__ l256,
                                                  int32_t* __restrict__ lcta, int32_t src_lo, int32_t src_hi,
                                                  DevStats* stats) {
    __shared__ unsigned bcount[PLAN_LISTS];
    __shared__ unsigned bbase[PLAN_LISTS];
    const int32_t R = n - (int32_t)stats->hub_count;
    const int lane = lane_id();
    unsigned* counters[PLAN_LISTS] = {&stats->small_count[0], &stats->small_count[1], &stats->small_count[2],
                                      &stats->small_count[3], &stats->cta_count};
    int32_t* lists[PLAN_LISTS] = {l8, l16, l32, l256, lcta};
    const int64_t tile = (int64_t)THREADS * PLAN_ITEMS;
    for (int64_t t0 = (int64_t)blockIdx.x * tile; t0 < n; t0 += (int64_t)gridDim.x * tile) {
        if (threadIdx.x < PLAN_LISTS) bcount[threadIdx.x] = 0;
        __syncthreads();
        int cls[PLAN_ITEMS];
        unsigned off[PLAN_ITEMS];
#pragma unroll
        for (int k = 0; k < PLAN_ITEMS; ++k) {
            const int64_t u = t0 + (int64_t)k * THREADS + threadIdx.x;
            int d = u < n && u >= src_lo && u < src_hi ? rowlen[u] : 0;  // sources outside the shard: none
            if (d >= 2 && col[rowstart[u]] >= R) d = 0;  // every target is a hub
            cls[k] = d < 2 ? -1 : d <= 8 ? 0 : d <= 16 ? 1 : d <= 32 ? 2 : d <= SMALL_WIDE_MAX ? 3 : 4;
#pragma unroll
            for (int c = 0; c < PLAN_LISTS; ++c) {
                const unsigned mk = __ballot_sync(FULL, cls[k] == c);
                unsigned wb = 0;
                if (mk && lane == 0) wb = atomicAdd(&bcount[c], (unsigned)__popc(mk));
                wb = __shfl_sync(FULL, wb, 0);
                if (cls[k] == c) off[k] = wb + __popc(mk & lanemask_lt());
            }
        }
        __syncthreads();
        if (threadIdx.x < PLAN_LISTS)
            bbase[threadIdx.x] = bcount[threadIdx.x] ? atomicAdd(counters[threadIdx.x], bcount[threadIdx.x]) : 0u;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PLAN_ITEMS; ++k)
            if (cls[k] >= 0) lists[cls[k]][bbase[cls[k]] + off[k]] = (int32_t)(t0 + (int64_t)k * THREADS + threadIdx.x);
        __syncthreads();
    }
}

// ---- small bucket: groups of G lanes, one lane per edge -----------------------

template <int G, bool SUP>
__global__ void __launch_bounds__(SMALL_WARPS * 32, SMALL_BLOCKS) k_tc_small(int32_t n, const int64_t* __restrict__ rowstart,
                                                               const int32_t* __restrict__ rowlen,
                                                               const int2* __restrict__ rowinfo,
                                                               const int32_t* __restrict__ col,
                                                               const int32_t* __restrict__ list, int cls,
                                                               unsigned long long* __restrict__ t, DevStats* stats,
                                                               int strategy, float factor,
                                                               uint32_t* __restrict__ sup_arg) {
    uint32_t* const sup = SUP ? sup_arg : nullptr;  // per-edge support (tc_edge_support) or none
    constexpr int GPW = 32 / G;
    __shared__ int32_t sLu[SMALL_WARPS * 32];
    __shared__ uint32_t sCnt[SMALL_WARPS * 32];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int grp = lane / G, g = lane % G;
    const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1u) << (grp * G));
    int32_t* Lu = sLu + w * 32 + grp * G;
    uint32_t* cnt = sCnt + w * 32 + grp * G;
    const unsigned count = stats->small_count[cls];
    const int32_t R = n - (int32_t)stats->hub_count;
    const unsigned groups = gridDim.x * SMALL_WARPS * GPW;
    // the next source and its row are fetched while the current one is counted
    unsigned q = (blockIdx.x * SMALL_WARPS + w) * GPW + grp;
    int32_t u = q < count ? list[q] : 0;
    int2 ru = q < count ? rowinfo[u] : make_int2(0, 0);
    for (; q < count; q += groups) {
        const unsigned qn = q + groups;
        const int32_t un = qn < count ? list[qn] : 0;
        const int du = ru.y;
        const int64_t base = ru.x;
        Lu[g] = g < du ? col[base + g] : INT_MAX;
        cnt[g] = 0;
        const int2 run = qn < count ? rowinfo[un] : make_int2(0, 0);
        __syncwarp(gmask);
        uint32_t c = 0;
        if (g < du - 1) {
            const int32_t v = Lu[g];
            const int2 ri = v < R ? rowinfo[v] : make_int2(0, 0);
            const int dv = ri.y;
            if (dv > 0) {
                const int32_t* B = col + ri.x;
                uint32_t* supB = sup ? sup + ri.x : nullptr;
                const int a = du - g - 1;
                int method = strategy;
                if (method == TC_STRAT_AUTO) method = small_auto(a, dv, factor);
                if (method == TC_STRAT_MERGE)
                    c = lane_merge_batched(Lu, g + 1, du, B, dv, cnt, supB);
                else
                    c = a <= dv ? lane_search(Lu, g + 1, du, B, dv, cnt, supB)
                                : lane_search_rev(Lu, g + 1, du, B, dv, cnt, supB);
                if (c) atomicAdd(&cnt[g], c);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) c += __shfl_down_sync(gmask, c, o, G);
        __syncwarp(gmask);
        const uint32_t cv = cnt[g];
        if (g < du && cv) {
            atomicAdd(&t[Lu[g]], (unsigned long long)cv);
            if (sup) atomicAdd(&sup[base + g], cv);  // edge (u, Lu[g]): as v of its edge and as w of others
        }
        if (g == 0 && c) atomicAdd(&t[u], (unsigned long long)c);
        __syncwarp(gmask);
        u = un;
        ru = run;
    }
}

// Sources with 32 < |N+(u)| <= SMALL_WIDE_MAX: a group of SMALL_WIDE_G lanes per
// source stages N+(u) in shared memory and its lanes take the edges (u, v) with v a
// non-hub (the first jh entries), one at a time, with the same per-edge choice
// (Eq. 3) between the batched merge and binary search as the small kernel.  Such
// sources mostly point to hubs and have few non-hub edges, so a block (or a whole
// warp) per source would idle.
constexpr int SMALL_WIDE_G = 16;
constexpr int SMALL_WIDE_BLOCKS = 6;  // blocks per SM
constexpr int SMALL_WIDE_GROUPS = SMALL_WARPS * 32 / SMALL_WIDE_G;  // per block

template <bool SUP>
__global__ void __launch_bounds__(SMALL_WARPS * 32) k_tc_small_wide(int32_t n, const int2* __restrict__ rowinfo,
                                                                   const int32_t* __restrict__ col,
                                                                   const int32_t* __restrict__ list,
                                                                   unsigned long long* __restrict__ t,
                                                                   DevStats* stats, int strategy, float factor,
                                                                   uint32_t* __restrict__ sup_arg) {
    uint32_t* const sup = SUP ? sup_arg : nullptr;
    extern __shared__ __align__(16) unsigned char wide_sh[];
    constexpr int G = SMALL_WIDE_G;
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int grp = lane / G, g = lane % G;
    const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1u) << (grp * G));
    const int gi = w * (32 / G) + grp;  // group index in the block
    int32_t* Lu = reinterpret_cast<int32_t*>(wide_sh) + gi * SMALL_WIDE_MAX;
    uint32_t* cnt = reinterpret_cast<uint32_t*>(wide_sh) + (SMALL_WIDE_GROUPS + gi) * SMALL_WIDE_MAX;
    const unsigned count = stats->small_count[3];
    const int32_t R = n - (int32_t)stats->hub_count;
    const unsigned groups = gridDim.x * SMALL_WIDE_GROUPS;
    for (unsigned q = blockIdx.x * SMALL_WIDE_GROUPS + gi; q < count; q += groups) {
        const int32_t u = list[q];
        const int2 ru = rowinfo[u];
        const int du = ru.y;  // 33 .. SMALL_WIDE_MAX
        for (int p = g; p < du; p += G) {
            Lu[p] = col[ru.x + p];
            cnt[p] = 0;
        }
        __syncwarp(gmask);
        const int jh = min(du - 1, lower_bound(Lu, 0, du, R));  // edges into non-hubs
        uint32_t c = 0;
        for (int j = g; j < jh; j += G) {
            const int32_t v = Lu[j];
            const int2 ri = rowinfo[v];
            const int dv = ri.y;
            if (dv == 0) continue;
            const int32_t* B = col + ri.x;
            uint32_t* supB = sup ? sup + ri.x : nullptr;
            const int a = du - j - 1;
            int method = strategy;
            if (method == TC_STRAT_AUTO) method = small_auto(a, dv, factor);
            const uint32_t cj = method == TC_STRAT_MERGE
                                    ? lane_merge_batched(Lu, j + 1, du, B, dv, cnt, supB)
                                    : (a <= dv ? lane_search(Lu, j + 1, du, B, dv, cnt, supB)
                                               : lane_search_rev(Lu, j + 1, du, B, dv, cnt, supB));
            if (cj) atomicAdd(&cnt[j], cj);
            c += cj;
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) c += __shfl_down_sync(gmask, c, o, G);
        __syncwarp(gmask);
        for (int p = g; p < du; p += G) {
            const uint32_t cv = cnt[p];
            if (cv) {
                atomicAdd(&t[Lu[p]], (unsigned long long)cv);
                if (sup) atomicAdd(&sup[ru.x + p], cv);
            }
        }
        if (g == 0 && c) atomicAdd(&t[u], (unsigned long long)c);
        __syncwarp(gmask);
    }
}

// ---- block bucket: |N+(u)| > 32, non-hub targets ------------------------------

// Open-addressing hash set of a staged list in shared memory (Fibonacci hashing, linear
// probing, empty slots hold -1).  The table has at least twice as many slots as
// keys, so a probe meets an empty slot after about two steps at most on average.
struct HashProbe {
    const int32_t* keys;
    unsigned shift, mask;
    __device__ __forceinline__ int operator()(int32_t x) const {
        unsigned h = ((unsigned)x * 0x9e3779b1u) >> shift;
        for (;;) {
            const int32_t k = keys[h];
            if (k == x) return (int)h;
            if (k < 0) return -1;
            h = (h + 1) & mask;
        }
    }
};

// ---- small bucket, hash strategy: N+(u) as a hash set, target rows end to end ----
//
// A group of G lanes takes one source u at a time.  N+(u) (at most AMAX entries) goes
// into an open-addressing hash set of SL >= 2 AMAX slots in shared memory.  Its edges
// (u, v) into non-hubs are taken G at a time; their rows N+(v) are laid end to end and
// the group reads G entries per round, one per lane, each entry probed once in the
// set (entries above max N+(u) are skipped).  A hit at x in N+(v) is a triangle: x is
// above v, so it lies in the suffix of N+(u) after v, which is W for the edge (u, v).
// Hits add to the slot's counter (t[x], flushed once per source) and to the edge's
// counter (t[v]); their sum goes to t[u].  Every lane reads at every round, so the
// lanes stay busy whatever the lengths of the rows.
template <int G, int SL, bool SUP>
__global__ void __launch_bounds__(SMALL_WARPS * 32) k_tc_small_hash(int32_t n, const int2* __restrict__ rowinfo,
                                                                   const int32_t* __restrict__ col,
                                                                   const int32_t* __restrict__ list, int cls,
                                                                   unsigned long long* __restrict__ t,
                                                                   DevStats* stats, uint32_t* __restrict__ sup_arg) {
    uint32_t* const sup = SUP ? sup_arg : nullptr;
    static_assert(G == 8 || G == 16 || G == 32, "lane groups within a warp");
    static_assert((SL & (SL - 1)) == 0 && SL >= 2 * G, "power-of-two table");
    constexpr int GROUPS = SMALL_WARPS * 32 / G;
    constexpr int LG = SL == 16 ? 4 : SL == 32 ? 5 : SL == 64 ? 6 : SL == 128 ? 7 : SL == 256 ? 8 : 9;
    static_assert((1 << LG) == SL, "table size");
    __shared__ int32_t skeys[GROUPS][SL];
    __shared__ uint32_t shcnt[GROUPS][SL];
    __shared__ uint32_t secnt[GROUPS][G];
    __shared__ uint16_t shpos[GROUPS][SL];  // position in N+(u) of each key (support only)
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int grp = lane / G, g = lane % G;
    const int gi = w * (32 / G) + grp;
    const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1u) << (grp * G));
    const unsigned below = (1u << g) - 1u;  // group lanes under this one (group-relative bits)
    int32_t* keys = skeys[gi];
    uint32_t* hcnt = shcnt[gi];
    uint32_t* ecnt = secnt[gi];
    uint16_t* hpos = shpos[gi];
    for (int i = g; i < SL; i += G) {
        keys[i] = -1;
        hcnt[i] = 0;
    }
    ecnt[g] = 0;
    __syncwarp(gmask);
    const unsigned count = stats->small_count[cls];
    const int32_t R = n - (int32_t)stats->hub_count;
    const unsigned groups = gridDim.x * GROUPS;
    const HashProbe P{keys, 32u - LG, SL - 1u};
    auto gballot = [&](bool p) { return (__ballot_sync(gmask, p) >> (grp * G)) & (G == 32 ? FULL : ((1u << G) - 1u)); };
    for (unsigned q = blockIdx.x * GROUPS + gi; q < count; q += groups) {
        const int32_t u = list[q];
        const int2 ru = rowinfo[u];
        const int du = ru.y;
        const int64_t base = ru.x;
        int jh = 0;  // entries below the hubs: the rows are sorted, so they come first
        for (int i0 = 0; i0 < du; i0 += G) {  // every lane of the group takes every round
            const bool valid = i0 + g < du;
            const int32_t x = valid ? col[base + i0 + g] : INT_MAX;
            if (valid) {
                unsigned h = ((unsigned)x * 0x9e3779b1u) >> (32 - LG);
                while (atomicCAS(&keys[h], -1, x) != -1) h = (h + 1) & (SL - 1);  // keys are distinct
                if (sup) hpos[h] = (uint16_t)(i0 + g);
            }
            jh += __popc(gballot(x < R));
        }
        const int32_t maxu = col[base + du - 1];
        const int ne = min(jh, du - 1);  // the last entry has an empty suffix
        __syncwarp(gmask);
        uint32_t cu = 0;
        for (int e0 = 0; e0 < ne; e0 += G) {
            const bool has = e0 + g < ne;
            const int32_t v0 = has ? col[base + e0 + g] : 0;
            const int2 r0 = has ? rowinfo[v0] : make_int2(0, 0);
            // only entries up to max N+(u) can match: long rows are cut there; an edge
            // whose cut row is longer than the suffix a of N+(u) after v by more than
            // Eq. 3 allows (factor 8: one lane's dependent search steps cost more than the
            // group's parallel probes) is left to its own lane, which searches the a keys
            // in the row (a log b instead of b probes)
            int b0 = r0.y;
            if (b0 > HASH_CUT) b0 = lower_bound(col + r0.x, 0, b0, maxu + 1);
            const int a0 = du - (e0 + g) - 1;
            const bool live = has && b0 > 0;
            const bool srch0 = live && a0 > 0 && b0 > a0 && !eq3_prefers_merge(a0, b0, 8.0f);
            // lanes reordered: the streamed edges first (ce of them), then the searching
            // ones (cq), then nothing
            const unsigned sm = gballot(live && !srch0);
            const unsigned qm = gballot(srch0);
            const int ce_n = __popc(sm), cq = __popc(qm);
            if (ce_n + cq == 0) continue;
            const int src = g < ce_n ? (int)__fns(sm, 0, g + 1) : (g < ce_n + cq ? (int)__fns(qm, 0, g - ce_n + 1) : g);
            const int32_t v = __shfl_sync(gmask, v0, src, G);
            const int jv = e0 + src;  // position of v in N+(u)
            const int rs = __shfl_sync(gmask, r0.x, src, G);
            int b = __shfl_sync(gmask, b0, src, G);
            if (g >= ce_n + cq) b = 0;
            const bool search = g >= ce_n && g < ce_n + cq;
            const int streamed = g < ce_n ? b : 0;
            int incl = streamed;
#pragma unroll
            for (int o = 1; o < G; o <<= 1) {
                const int y = __shfl_up_sync(gmask, incl, o, G);
                if (g >= o) incl += y;
            }
            const int total = __shfl_sync(gmask, incl, G - 1, G);
            const int excl = incl - streamed;
            for (int r = 0; r < total; r += G) {
                // the edge of entry r + g: i0 holds entry r, and every later streamed
                // edge that starts inside the round marks its first entry in mk
                const int i0 = __popc(gballot(g < ce_n && incl <= r));
                const unsigned mk = __reduce_or_sync(gmask, (g > i0 && g < ce_n && excl - r < G) ? (1u << (excl - r)) : 0u);
                const int idx = min(i0 + __popc(mk & (below | (1u << g))), G - 1);
                const int bs = __shfl_sync(gmask, rs, idx, G);
                const int bx = __shfl_sync(gmask, excl, idx, G);
                const int k = r + g;
                if (k < total) {
                    const int64_t px = (int64_t)bs + (k - bx);
                    const int32_t x = col[px];
                    if (x <= maxu) {
                        const int h = P(x);
                        if (h >= 0) {
                            atomicAdd(&hcnt[h], 1u);
                            atomicAdd(&ecnt[idx], 1u);
                            if (sup) atomicAdd(&sup[px], 1u);  // edge (v, x)
                        }
                    }
                }
            }
            uint32_t cs = 0;  // a searching lane: the suffix keys after v looked up in N+(v)
            if (search) {
                const int32_t* B = col + rs;
                int lo = 0;
                for (int i = jv + 1; i < du && lo < b; ++i) {
                    const int32_t y = col[base + i];
                    const int p = lower_bound(B, lo, b, y);
                    lo = p;
                    if (p < b && B[p] == y) {
                        atomicAdd(&hcnt[P(y)], 1u);
                        if (sup) atomicAdd(&sup[rs + p], 1u);  // edge (v, y)
                        ++cs;
                    }
                }
            }
            __syncwarp(gmask);
            const uint32_t ce = ecnt[g] + cs;
            ecnt[g] = 0;
            if (ce) {
                atomicAdd(&t[v], (unsigned long long)ce);
                if (sup) atomicAdd(&sup[base + jv], ce);  // edge (u, v)
                cu += ce;
            }
            __syncwarp(gmask);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) cu += __shfl_down_sync(gmask, cu, o, G);
        if (g == 0 && cu) atomicAdd(&t[u], (unsigned long long)cu);
        for (int i = g; i < SL; i += G) {  // flush the per-entry counts, empty the set
            const int32_t x = keys[i];
            if (x >= 0) {
                const uint32_t c = hcnt[i];
                if (c) {
                    atomicAdd(&t[x], (unsigned long long)c);
                    if (sup) atomicAdd(&sup[base + hpos[i]], c);  // edge (u, x)
                }
                keys[i] = -1;
                hcnt[i] = 0;
            }
        }
        __syncwarp(gmask);
    }
}


// Warp per edge: the entries of B = N+(v) (sorted) are probed in a set of the
// staged N+(u), two per lane per round, stopping above max N+(u); hits add to the
// set's per-slot counter.  Returns the edge's count (all lanes).
template <class Probe>
__device__ uint32_t edge_probe_set(const Probe& P, int32_t maxu, uint32_t* hcnt, const int32_t* __restrict__ B, int b,
                               uint32_t* __restrict__ supB) {
    const int lane = lane_id();
    uint32_t c = 0;
    for (int k0 = 0; k0 < b; k0 += 64) {
        const int k1 = k0 + lane, k2 = k1 + 32;
        const int32_t x1 = k1 < b ? B[k1] : INT_MAX;
        const int32_t x2 = k2 < b ? B[k2] : INT_MAX;
        if (x1 <= maxu) {
            const int p = P(x1);
            if (p >= 0) {
                atomicAdd(&hcnt[p], 1u);
                if (supB) atomicAdd(&supB[k1], 1u);
                ++c;
            }
        }
        if (x2 <= maxu) {
            const int p = P(x2);
            if (p >= 0) {
                atomicAdd(&hcnt[p], 1u);
                if (supB) atomicAdd(&supB[k2], 1u);
                ++c;
            }
        }
        if (__any_sync(FULL, x2 > maxu)) break;  // B is sorted
    }
    return warp_sum(c);
}

struct CtaShared {
    int32_t Lu[CTA_LIST_MAX];
    uint32_t cnt[CTA_LIST_MAX];
    union {
        struct {  // bitmap of N+(u) over its rank window
            uint32_t bm[BITMAP_WORDS];
            uint16_t pre[BITMAP_WORDS];
            uint32_t slice[BITMAP_WORDS / 32];
        } b;
        struct {  // hash set of N+(u) when the window is wider than the bitmap
            int32_t keys[2 * CTA_LIST_MAX];
            uint32_t hcnt[2 * CTA_LIST_MAX];
        } h;
    } s;
    unsigned long long utot[CTA_WARPS];
    int q;
};

template <bool SUP>
__global__ void __launch_bounds__(CTA_THREADS) k_tc_cta(int32_t n, const int64_t* __restrict__ rowstart,
                                                        const int32_t* __restrict__ rowlen,
                                                        const int2* __restrict__ rowinfo,
                                                        const int32_t* __restrict__ col,
                                                        const int32_t* __restrict__ list,
                                                        unsigned long long* __restrict__ t,
                                                        DevStats* stats, int strategy, float factor,
                                                        uint32_t* __restrict__ sup_arg) {
    uint32_t* const sup = SUP ? sup_arg : nullptr;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaShared& sh = *reinterpret_cast<CtaShared*>(smem_raw);
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const unsigned count = stats->cta_count;
    const int32_t R = n - (int32_t)stats->hub_count;
    for (;;) {
        if (threadIdx.x == 0) sh.q = (int)atomicAdd(&stats->cta_next, 1u);
        __syncthreads();
        const int q = sh.q;
        if ((unsigned)q >= count) break;
        const int32_t u = list[q];
        const int du = rowlen[u];
        const int64_t base = rowstart[u];
        const bool staged = du <= CTA_LIST_MAX;
        if (staged) {
            for (int p = threadIdx.x; p < du; p += CTA_THREADS) {
                sh.Lu[p] = col[base + p];
                sh.cnt[p] = 0;
            }
        }
        __syncthreads();
        const int32_t* Lu = staged ? sh.Lu : col + base;
        const int32_t maxu = Lu[du - 1];
        const int jh = min(du - 1, lower_bound(Lu, 0, du, R));  // edges into non-hubs
        const int span = maxu - u;  // ranks u+1 .. maxu
        const bool bitmap = staged && strategy == TC_STRAT_BITMAP && span <= BITMAP_WORDS * 32;
        const bool hashed = staged && strategy == TC_STRAT_BITMAP && !bitmap;
        if (bitmap) build_bitmap<CTA_THREADS>(sh.s.b.bm, sh.s.b.pre, sh.s.b.slice, sh.Lu, du, u, (span + 31) >> 5);
        unsigned hshift = 0, hmask = 0;
        if (hashed) {  // uniform across the block
            int lg = 6;
            while ((1 << lg) < 2 * du) ++lg;  // du <= CTA_LIST_MAX: at most 2 * CTA_LIST_MAX slots
            hmask = (1u << lg) - 1u;
            hshift = 32u - (unsigned)lg;
            for (int p = threadIdx.x; p <= (int)hmask; p += CTA_THREADS) {
                sh.s.h.keys[p] = -1;
                sh.s.h.hcnt[p] = 0;
            }
            __syncthreads();
            for (int p = threadIdx.x; p < du; p += CTA_THREADS) {
                const int32_t x = sh.Lu[p];
                unsigned h = ((unsigned)x * 0x9e3779b1u) >> hshift;
                while (atomicCAS(&sh.s.h.keys[h], -1, x) != -1) h = (h + 1) & hmask;  // keys are distinct
            }
            __syncthreads();
        }
        uint32_t* supA = sup ? sup + base : nullptr;
        Sink S{staged ? sh.cnt : nullptr, t, Lu, staged ? nullptr : supA, nullptr};
        unsigned long long utot = 0;
        for (int j = w; j < jh; j += CTA_WARPS) {
            const int32_t v = Lu[j];
            const int2 ri = rowinfo[v];
            const int dv = ri.y;
            if (dv == 0) continue;
            const int32_t* B = col + ri.x;
            uint32_t* supB = sup ? sup + ri.x : nullptr;
            S.supB = supB;
            uint32_t c;
            if (bitmap) {
                c = edge_bitmap(sh.s.b.bm, sh.s.b.pre, u, maxu, sh.cnt, B, dv, supB);
            } else if (hashed) {
                c = edge_probe_set(HashProbe{sh.s.h.keys, hshift, hmask}, maxu, sh.s.h.hcnt, B, dv, supB);
            } else {
                int method = strategy;
                if (method == TC_STRAT_AUTO) {
                    const int a = du - j - 1;
                    method = eq3_prefers_merge(a, dv, factor) ? TC_STRAT_MERGE
                                                              : (a <= dv ? TC_STRAT_SEARCH : TC_STRAT_PROBE);
                } else if (method == TC_STRAT_BITMAP) {
                    method = TC_STRAT_PROBE;
                }
                c = edge_dispatch(method, S, j + 1, du, B, dv);
            }
            if (lane == 0 && c) {
                if (staged) {
                    atomicAdd(&sh.cnt[j], c);
                } else {
                    atomicAdd(&t[v], (unsigned long long)c);
                    if (supA) atomicAdd(&supA[j], c);  // edge (u, v)
                }
            }
            utot += c;
        }
        if (lane == 0) sh.utot[w] = utot;
        __syncthreads();
        if (staged) {
            for (int p = threadIdx.x; p < du; p += CTA_THREADS) {
                const uint32_t cv = sh.cnt[p];
                if (cv) {
                    atomicAdd(&t[sh.Lu[p]], (unsigned long long)cv);
                    if (supA) atomicAdd(&supA[p], cv);
                }
            }
        }
        if (hashed) {
            for (int p = threadIdx.x; p <= (int)hmask; p += CTA_THREADS) {
                const int32_t x = sh.s.h.keys[p];
                const uint32_t cv = sh.s.h.hcnt[p];
                if (x >= 0 && cv) {
                    atomicAdd(&t[x], (unsigned long long)cv);
                    if (supA) atomicAdd(&supA[lower_bound(sh.Lu, 0, du, x)], cv);
                }
            }
        }
        if (threadIdx.x == 0) {
            unsigned long long s = 0;
            for (int k = 0; k < CTA_WARPS; ++k) s += sh.utot[k];
            if (s) atomicAdd(&t[u], s);
        }
        __syncthreads();
    }
}

// ---- hub bucket ----------------------------------------------------------------
// Big hubs (in-degree >= the planner's threshold, or lists too long for one warp) are processed
// by a whole block over a bitmap of N+(v); the remaining hubs by one warp each over
// a hash set of N+(v) in shared memory.  One persistent kernel drains the big-hub
// queue first, then every warp takes medium hubs independently.


struct BitmapProbe {
    const uint32_t* bm;
    const uint16_t* pre;
    int32_t v;
    __device__ __forceinline__ int operator()(int32_t x) const {
        const int off = x - v - 1;
        const uint32_t word = bm[off >> 5], bit = 1u << (off & 31);
        return (word & bit) ? (int)pre[off >> 5] + __popc(word & (bit - 1)) : -1;
    }
};

struct ListProbe {
    const int32_t* L;
    int d;
    __device__ __forceinline__ int operator()(int32_t x) const {
        const int p = lower_bound(L, 0, d, x);  // x <= max(L), so p < d
        return L[p] == x ? p : -1;
    }
};

// One batch of up to 32 in-edges [k0, min(k0 + 32, e1)) of hub v, processed by one
// warp.  Suffixes of 32 or more entries are read one in-edge at a time by all lanes
// (the read stops above max N+(v)); shorter ones are laid end to end and read 32
// entries at a time.  Matches add to cnt[p] (or t[x] when cnt is null) and to the
// per-in-edge total, which goes to t[u].  Returns the batch total (all lanes).
template <bool SUP, class Probe>
__device__ uint32_t hub_batch(int64_t k0, int64_t e1, const int4* __restrict__ in_rec,
                              const int32_t* __restrict__ col, int32_t maxv, const Probe& probe, uint32_t* cnt,
                              unsigned long long* __restrict__ t, uint32_t* cw, uint32_t* __restrict__ sup_arg,
                              int64_t vbase) {
    uint32_t* const sup = SUP ? sup_arg : nullptr;
    const int lane = lane_id();
    const int64_t k = k0 + lane;
    const int4 rec = k < e1 ? in_rec[k] : make_int4(0, 0, 0, 0);
    int32_t uu = rec.x;
    int32_t b0 = rec.y;
    int a = rec.z - rec.y;
    uint32_t total_c = 0;
    const bool islong = a >= HUB_LONG;
    const int nlong = __popc(__ballot_sync(FULL, islong));
    // the long suffixes by decreasing length (bitonic sort of (length, lane) keys across
    // the warp), so that the groups that run their rounds together take suffixes of
    // similar length and wait less for each other
    uint32_t key = islong ? ((uint32_t)min(a, (1 << 26) - 1) << 5) | (uint32_t)lane : 0u;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const uint32_t other = __shfl_xor_sync(FULL, key, j);
            const bool keep_max = ((lane & j) == 0) == ((lane & k) == 0);
            key = keep_max ? max(key, other) : min(key, other);
        }
    }
    // HUB_GROUPS long suffixes at a time, one per group of HUB_GLANES lanes, each lane
    // reading HUB_UNROLL entries per round with all loads in flight before any is used
    const int g = lane / HUB_GLANES, gl = lane % HUB_GLANES;
    const unsigned gmask = (HUB_GLANES == 32 ? FULL : ((1u << HUB_GLANES) - 1u)) << (g * HUB_GLANES);
    for (int k0 = 0; k0 < nlong; k0 += HUB_GROUPS) {
        const int pos = k0 + g;
        const uint32_t kp = __shfl_sync(FULL, key, min(pos, 31));
        const int my = pos < nlong ? (int)(kp & 31u) : -1;  // batch lane holding this group's in-edge
        const int src = my < 0 ? 0 : my;
        const int32_t bL = __shfl_sync(FULL, b0, src);
        int aL = __shfl_sync(FULL, a, src);
        const int32_t uL = __shfl_sync(FULL, uu, src);
        if (my < 0) aL = 0;
        uint32_t c = 0;
        for (int o0 = 0;; o0 += HUB_GLANES * HUB_UNROLL) {
            int32_t x[HUB_UNROLL];
#pragma unroll
            for (int j = 0; j < HUB_UNROLL; ++j) {
                const int o = o0 + j * HUB_GLANES + gl;
                x[j] = o < aL ? col[bL + o] : INT_MAX;
            }
#pragma unroll
            for (int j = 0; j < HUB_UNROLL; ++j) {
                if (x[j] <= maxv) {
                    const int p = probe(x[j]);
                    if (p >= 0) {
                        if (cnt) {
                            atomicAdd(&cnt[p], 1u);
                        } else {
                            atomicAdd(&t[x[j]], 1ull);
                            if (sup) atomicAdd(&sup[vbase + p], 1u);  // edge (v, x)
                        }
                        if (sup) atomicAdd(&sup[bL + o0 + j * HUB_GLANES + gl], 1u);  // edge (u, x)
                        ++c;
                    }
                }
            }
            // the suffix is sorted: a group is done once one of its lanes read past maxv
            // (or past the end of the suffix)
            if (__ballot_sync(FULL, x[HUB_UNROLL - 1] > maxv) & gmask) aL = 0;
            if (__all_sync(FULL, aL == 0)) break;
        }
#pragma unroll
        for (int off = HUB_GLANES / 2; off > 0; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
        if (gl == 0 && my >= 0 && c) {
            atomicAdd(&t[uL], (unsigned long long)c);
            if (sup) atomicAdd(&sup[bL - 1], c);  // edge (u, v): bL is the entry after v
        }
        total_c += __reduce_add_sync(FULL, gl == 0 ? c : 0u);
    }
    if (a >= HUB_LONG) a = 0;  // done above
    const unsigned nz = __ballot_sync(FULL, a > 0);
    const int cz = __popc(nz);
    if (cz == 0) return total_c;
    // lane i takes the i-th short in-edge
    const int src = lane < cz ? (int)__fns(nz, 0, lane + 1) : lane;
    uu = __shfl_sync(FULL, uu, src);
    b0 = __shfl_sync(FULL, b0, src);
    a = __shfl_sync(FULL, a, src);
    if (lane >= cz) a = 0;
    int incl = warp_inclusive_scan(a);
    const int total = __shfl_sync(FULL, incl, 31);
    const int excl = incl - a;
    if (lane >= cz) incl = INT_MAX;
    cw[lane] = 0;
    __syncwarp();
    for (int r = 0; r < total; r += 32) {
        const int i0 = __popc(__ballot_sync(FULL, incl <= r));
        unsigned mk = (lane > i0 && lane < cz && excl - r < 32) ? (1u << (excl - r)) : 0u;
        mk = __reduce_or_sync(FULL, mk);
        const int idx = min(i0 + __popc(mk & (lane == 31 ? FULL : ((2u << lane) - 1u))), 31);
        const int bi = __shfl_sync(FULL, b0, idx);
        const int xi = __shfl_sync(FULL, excl, idx);
        const int item = r + lane;
        if (item < total) {
            const int32_t x = col[bi + (item - xi)];
            if (x <= maxv) {
                const int p = probe(x);
                if (p >= 0) {
                    if (cnt) {
                        atomicAdd(&cnt[p], 1u);
                    } else {
                        atomicAdd(&t[x], 1ull);
                        if (sup) atomicAdd(&sup[vbase + p], 1u);  // edge (v, x)
                    }
                    if (sup) atomicAdd(&sup[bi + (item - xi)], 1u);  // edge (u, x)
                    atomicAdd(&cw[idx], 1u);
                }
            }
        }
    }
    __syncwarp();
    const uint32_t cu = cw[lane];
    if (lane < cz && cu) {
        atomicAdd(&t[uu], (unsigned long long)cu);
        if (sup) atomicAdd(&sup[b0 - 1], cu);  // edge (u, v)
    }
    __syncwarp();
    return total_c + __reduce_add_sync(FULL, lane < cz ? cu : 0u);
}

struct HubShared {
    union {
        struct {  // big hub, one block
            union {
                struct {
                    uint32_t bm[HUB_BM_WORDS];
                    uint16_t pre[HUB_BM_WORDS];
                } b;
                int32_t list[HUB_CNT_MAX];
            } s;
            uint32_t cnt[HUB_CNT_MAX];
            uint32_t slice[HUB_BM_WORDS / 32];
        } big;
        struct {  // medium hubs, one per warp
            int32_t keys[HUB_WARPS][HUB_HASH_MAX];
            uint32_t cnt[HUB_WARPS][HUB_HASH_MAX];
        } med;
    } u;
    uint32_t cw[HUB_WARPS][32];
    unsigned long long vt[HUB_WARPS];
    int q;
    unsigned bq;  // next batch of the current big hub
};

template <bool SUP>
__global__ void __launch_bounds__(HUB_THREADS) k_tc_hub(int32_t n, int32_t hub_cap, const int64_t* __restrict__ rowstart,
                                                        const int32_t* __restrict__ rowlen,
                                                        const int32_t* __restrict__ col,
                                                        const int64_t* __restrict__ hub_start,
                                                        const int32_t* __restrict__ big_list,
                                                        const int32_t* __restrict__ med_list,
                                                        const int4* __restrict__ in_rec,
                                                        unsigned long long* __restrict__ t, DevStats* stats,
                                                        int probe_mode, uint32_t* __restrict__ sup_arg) {
    uint32_t* const sup = SUP ? sup_arg : nullptr;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    HubShared& sh = *reinterpret_cast<HubShared*>(smem_raw);
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const unsigned nbig = stats->hub_big, nmed = stats->hub_count - stats->hub_big;
    // phase 1: big hubs, one block each
    for (;;) {
        if (threadIdx.x == 0) {
            sh.q = (int)atomicAdd(&stats->hub_next, 1u);
            sh.bq = 0;
        }
        __syncthreads();
        const int q = sh.q;
        if ((unsigned)q >= nbig) break;
        const int32_t v = big_list[q];
        const int hi = v - (n - hub_cap);
        const int64_t e0 = hub_start[hi], e1 = hub_start[hi + 1];
        const int dv = rowlen[v];
        const int64_t base = rowstart[v];
        const int32_t maxv = col[base + dv - 1];  // big hubs have dv >= 1
        const bool staged = dv <= HUB_CNT_MAX;
        const int W = (maxv - v + 31) >> 5;  // maxv - v < hub_cap <= HUB_BM_BITS
        if (staged)
            for (int p = threadIdx.x; p < dv; p += HUB_THREADS) sh.u.big.cnt[p] = 0;
        if (!probe_mode) {
            build_bitmap<HUB_THREADS>(sh.u.big.s.b.bm, sh.u.big.s.b.pre, sh.u.big.slice, col + base, dv, v, W);
        } else {
            if (staged)
                for (int p = threadIdx.x; p < dv; p += HUB_THREADS) sh.u.big.s.list[p] = col[base + p];
            __syncthreads();
        }
        uint32_t* cnt = staged ? sh.u.big.cnt : nullptr;
        unsigned long long vtot = 0;
        // batches of bs in-edges, claimed by the warps from a shared counter (the block
        // waits for its slowest warp); small hubs use smaller batches so that every
        // warp gets some
        const int64_t din = e1 - e0;
        const int bs = din >= 2 * HUB_WARPS * HUB_BATCH ? HUB_BATCH
                                                        : max(8, (int)((din + 2 * HUB_WARPS - 1) / (2 * HUB_WARPS)));
        if (!probe_mode) {
            const BitmapProbe P{sh.u.big.s.b.bm, sh.u.big.s.b.pre, v};
            for (;;) {
                unsigned k = 0;
                if (lane == 0) k = atomicAdd(&sh.bq, 1u);
                const int64_t bb = e0 + (int64_t)__shfl_sync(FULL, k, 0) * bs;
                if (bb >= e1) break;
                vtot += hub_batch<SUP>(bb, min(bb + bs, e1), in_rec, col, maxv, P, cnt, t, sh.cw[w], sup, base);
            }
        } else {
            const ListProbe P{staged ? sh.u.big.s.list : col + base, dv};
            for (;;) {
                unsigned k = 0;
                if (lane == 0) k = atomicAdd(&sh.bq, 1u);
                const int64_t bb = e0 + (int64_t)__shfl_sync(FULL, k, 0) * bs;
                if (bb >= e1) break;
                vtot += hub_batch<SUP>(bb, min(bb + bs, e1), in_rec, col, maxv, P, cnt, t, sh.cw[w], sup, base);
            }
        }
        if (lane == 0) sh.vt[w] = vtot;
        __syncthreads();
        if (staged) {
            if (!probe_mode) {
                for (int i = threadIdx.x; i < W; i += HUB_THREADS) {
                    const uint32_t word = sh.u.big.s.b.bm[i];
                    uint32_t rest = word;
                    while (rest) {
                        const int bpos = __ffs(rest) - 1;
                        rest &= rest - 1;
                        const int p = sh.u.big.s.b.pre[i] + __popc(word & ((1u << bpos) - 1u));
                        const uint32_t c = sh.u.big.cnt[p];
                        if (c) {
                            atomicAdd(&t[v + 1 + i * 32 + bpos], (unsigned long long)c);
                            if (sup) atomicAdd(&sup[base + p], c);  // edge (v, x)
                        }
                    }
                }
            } else {
                for (int p = threadIdx.x; p < dv; p += HUB_THREADS) {
                    const uint32_t c = sh.u.big.cnt[p];
                    if (c) {
                        atomicAdd(&t[sh.u.big.s.list[p]], (unsigned long long)c);
                        if (sup) atomicAdd(&sup[base + p], c);  // edge (v, x)
                    }
                }
            }
        }
        if (threadIdx.x == 0) {
            unsigned long long s = 0;
            for (int k = 0; k < HUB_WARPS; ++k) s += sh.vt[k];
            if (s) atomicAdd(&t[v], s);
        }
        __syncthreads();
    }
    // phase 2: medium hubs, one warp each (no block barriers from here on), probed
    // through a hash set of N+(v); every slot is empty again after each hub
    int32_t* K = sh.u.med.keys[w];
    uint32_t* cnt = sh.u.med.cnt[w];
    for (int p = lane; p < HUB_HASH_MAX; p += 32) {
        K[p] = -1;
        cnt[p] = 0;
    }
    __syncwarp();
    for (;;) {
        unsigned q = 0;
        if (lane == 0) q = atomicAdd(&stats->hub_next2, 1u);
        q = __shfl_sync(FULL, q, 0);
        if (q >= nmed) break;
        const int32_t v = med_list[q];
        const int hi = v - (n - hub_cap);
        const int64_t e0 = hub_start[hi], e1 = hub_start[hi + 1];
        const int dv = rowlen[v];
        if (dv == 0 || e1 == e0) continue;
        if (dv > HUB_WARP_MAX) {  // the flags never make such a hub medium: do not overrun the table
            if (lane == 0) atomicOr(&stats->err, ERR_OVERFLOW);
            continue;
        }
        const int64_t base = rowstart[v];
        int lg = 5;
        while ((1 << lg) < HUB_HASH_LOAD * dv) ++lg;
        const unsigned shift = 32u - (unsigned)lg, mask = (1u << lg) - 1u;
        for (int p = lane; p < dv; p += 32) {
            const int32_t x = col[base + p];
            unsigned h = ((unsigned)x * 0x9e3779b1u) >> shift;
            while (atomicCAS(&K[h], -1, x) != -1) h = (h + 1) & mask;  // keys are distinct
        }
        const int32_t maxv = col[base + dv - 1];
        __syncwarp();
        const HashProbe P{K, shift, mask};
        unsigned long long vtot = 0;
        for (int64_t bb = e0; bb < e1; bb += 32)
            vtot += hub_batch<SUP>(bb, e1, in_rec, col, maxv, P, cnt, t, sh.cw[w], sup, base);
        __syncwarp();
        for (int p = lane; p <= (int)mask; p += 32) {
            const int32_t x = K[p];
            if (x >= 0) {
                const uint32_t c = cnt[p];
                if (c) {
                    atomicAdd(&t[x], (unsigned long long)c);
                    if (sup) atomicAdd(&sup[base + lower_bound(col + base, 0, dv, x)], c);  // edge (v, x)
                }
                K[p] = -1;
                cnt[p] = 0;
            }
        }
        if (lane == 0 && vtot) atomicAdd(&t[v], vtot);
        __syncwarp();
    }
}

// ---- reductions ---------------------------------------------------------------

__global__ void k_sum_t(int32_t n, const unsigned long long* __restrict__ t, DevStats* stats) {
    unsigned long long s = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) s += t[i];
    s = warp_sum(s);
    if (lane_id() == 0 && s) atomicAdd(&stats->sum_t, s);
}

// Eq. 2 with the simple degree; both operands are exact integers below 2^53, so
// the IEEE round-to-nearest division gives the correctly rounded quotient.
__global__ void k_finalize(int32_t n, const int32_t* __restrict__ rank, const unsigned long long* __restrict__ t_rank,
                           const int32_t* __restrict__ deg, unsigned long long* __restrict__ t_out,
                           double* __restrict__ lcc_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t r = rank[v];
        const unsigned long long tv = t_rank[r];
        if (t_out) t_out[v] = tv;
        if (lcc_out) {
            const long long d = deg[r];
            // t = 0 gives +0.0 without a double division (FP64 runs at a small fraction of FP32)
            lcc_out[v] = d < 2 || tv == 0 ? 0.0 : __ddiv_rn((double)(2ull * tv), (double)(d * (d - 1)));
        }
    }
}

// Per-bucket work: edges and sum of d+(u) + d+(v) over them (one thread per u).
__global__ void k_plan_stats(int32_t n, const int64_t* __restrict__ rowstart, const int32_t* __restrict__ rowlen,
                             const int32_t* __restrict__ col, const DevStats* stats,
                             unsigned long long* __restrict__ out) {
    const int32_t R = n - (int32_t)stats->hub_count;
    unsigned long long e[TC_NUM_BUCKETS + 1] = {}, ids[TC_NUM_BUCKETS + 1] = {};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const int d = rowlen[u];
        for (int k = 0; k < d; ++k) {
            const int32_t v = col[rowstart[u] + k];
            const int b = v >= R ? TC_BUCKET_HUB
                                 : (d < 2 ? TC_NUM_BUCKETS : (d <= SMALL_WIDE_MAX ? TC_BUCKET_SMALL : TC_BUCKET_CTA));
            e[b] += 1;
            ids[b] += (unsigned long long)(d + rowlen[v]);
        }
    }
#pragma unroll
    for (int b = 0; b <= TC_NUM_BUCKETS; ++b) {
        const unsigned long long x = warp_sum(e[b]), y = warp_sum(ids[b]);
        if (lane_id() == 0) {
            if (x) atomicAdd(&out[b], x);
            if (y) atomicAdd(&out[TC_NUM_BUCKETS + 1 + b], y);
        }
    }
}

}  // namespace

void launch_plan_stats(const CountBuffers& C, unsigned long long* out, const Launch& L) {
    if (C.n <= 0) return;
    k_plan_stats<<<grid_for(C.n, THREADS, L.sms), THREADS, 0, L.stream>>>(C.n, C.rowstart, C.rowlen, C.col,
                                                                         C.stats, out);
    count_launch();
}

bool launch_plan(const CountBuffers& C, const Strategy& S, const Launch& L, const PlanStreams* ps) {
    if (C.n <= 0) return false;
    const int hub_max = S.hub_max < 0 ? 0 : S.hub_max;
    const bool hubs = C.hub_cap > 0 && hub_max > 0;
    if (hubs) {
        k_hub_candidates<<<grid_for(C.n, THREADS, L.sms), THREADS, 0, L.stream>>>(C.n, C.deg, S.hub_min_degree,
                                                                                 C.stats);
        count_launch();
    }
    const int core_max = hubs && C.core_cap > 0 && S.hub_core > 0 ? (S.hub_core < C.core_cap ? S.hub_core : C.core_cap) : 0;
    k_hub_count<<<1, 1, 0, L.stream>>>(C.hub_cap, hub_max, core_max, C.stats);
    count_launch();
    // the hub lists and the dense core need only the hub count: with a second stream
    // they are built while the main stream lists and counts the push buckets
    const bool forked = hubs && ps != nullptr;
    Launch H = L;
    if (forked) {
        cudaEventRecord(ps->fork, L.stream);
        cudaStreamWaitEvent(ps->side, ps->fork, 0);
        H.stream = ps->side;
    }
    if (hubs) {
        if (core_max > 0) launch_core_plan(C, H);
        k_hub_indeg<<<grid_for(C.hub_cap, THREADS, H.sms), THREADS, 0, H.stream>>>(C.n, C.hub_cap, C.deg, C.rowlen,
                                                                                  C.core_cnt, C.hub_cnt, C.stats);
        count_launch();
        scan_u32_to_i64(C.hub_cnt, C.hub_start, C.hub_cap, C.tmp, H);
        // 64-bit cursors starting at every hub's first slot
        cudaMemcpyAsync(C.hub_cur64, C.hub_start, sizeof(int64_t) * (size_t)C.hub_cap, cudaMemcpyDeviceToDevice,
                        H.stream);
        k_row_of<<<grid_for((int64_t)C.n, THREADS, H.sms), THREADS, 0, H.stream>>>(C.n, C.hub_cap, C.rowstart,
                                                                                  C.hub_start, C.rowof, C.stats);
        count_launch();
        k_hub_scatter_rows<<<grid_for(C.n, THREADS, H.sms), THREADS, 0, H.stream>>>(
            C.n, C.hub_cap, C.rowstart, C.rowlen, C.col, C.hub_start, C.hub_cur64, C.in_rec, C.src_lo, C.src_hi,
            C.stats);
        count_launch();
        k_hub_scatter<<<grid_for((int64_t)C.m_cap / SCAT_ITEMS + 1, SCAT_THREADS, H.sms), SCAT_THREADS, 0, H.stream>>>(
            C.n, C.hub_cap, C.rowstart, C.rowinfo, C.col, C.rowof, C.hub_start, C.hub_cur64, C.in_rec, C.src_lo,
            C.src_hi, C.stats);
        count_launch();
        k_hub_cur_check<<<grid_for(C.hub_cap, THREADS, H.sms), THREADS, 0, H.stream>>>(C.hub_cap, C.hub_start,
                                                                                      C.hub_cur64, C.stats);
        count_launch();
        // hub_cur is free again: it holds the big flags, hub_cnt (still the in-degrees
        // until here) is overwritten by their exclusive scan
        k_hub_flags<<<grid_for(C.hub_cap, THREADS, H.sms), THREADS, 0, H.stream>>>(
            C.n, C.rowlen, C.hub_cnt, C.hub_cap, S.hub_big_in > 0 ? S.hub_big_in : 1, C.hub_cur, C.stats);
        count_launch();
        scan_u32_to_u32(C.hub_cur, C.hub_cnt, C.hub_cap, C.tmp, H);
        k_hub_lists<<<grid_for(C.hub_cap, THREADS, H.sms), THREADS, 0, H.stream>>>(C.n, C.hub_cur, C.hub_cnt,
                                                                                  C.big_list, C.med_list, C.stats);
        count_launch();
    }
    if (forked) cudaEventRecord(ps->join, H.stream);
    k_plan<<<grid_for(C.n, THREADS * PLAN_ITEMS, L.sms), THREADS, 0, L.stream>>>(C.n, C.rowstart, C.rowlen, C.col,
                                                                   C.small_list[0], C.small_list[1],
                                                                   C.small_list[2], C.small_list[3], C.cta_list,
                                                                   C.src_lo, C.src_hi, C.stats);
    count_launch();
    return forked;
}

cudaError_t intersect_init_attributes() {
    const int wide = 2 * SMALL_WIDE_GROUPS * SMALL_WIDE_MAX * (int)sizeof(int32_t);
    cudaError_t e = cudaSuccess;
    if ((e = cudaFuncSetAttribute(k_tc_cta<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CtaShared))) ||
        (e = cudaFuncSetAttribute(k_tc_cta<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CtaShared))) ||
        (e = cudaFuncSetAttribute(k_tc_small_wide<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, wide)) ||
        (e = cudaFuncSetAttribute(k_tc_small_wide<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, wide)) ||
        (e = cudaFuncSetAttribute(k_tc_hub<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(HubShared))))
        return e;
    return cudaFuncSetAttribute(k_tc_hub<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(HubShared));
}

template <bool SUP>
void intersect_impl(const CountBuffers& C, const Strategy& S, cudaEvent_t* ev, const Launch& L) {
    if (C.n <= 0) return;
    if (ev) cudaEventRecord(ev[PH_SMALL], L.stream);
    const int ss = S.strat[TC_BUCKET_SMALL];
    const float sf = S.factor[TC_BUCKET_SMALL];
    if (ss == TC_STRAT_HASH) {
        // sources of at most 16 entries: one edge per lane (Eq. 3 per edge), whose
        // short merges cost less than building and flushing a set per source
        k_tc_small<8, SUP><<<L.sms * SMALL_BLOCKS, SMALL_WARPS * 32, 0, L.stream>>>(
            C.n, C.rowstart, C.rowlen, C.rowinfo, C.col, C.small_list[0], 0, C.t_rank, C.stats, TC_STRAT_AUTO, sf, C.sup);
        count_launch();
        k_tc_small<16, SUP><<<L.sms * SMALL_BLOCKS, SMALL_WARPS * 32, 0, L.stream>>>(
            C.n, C.rowstart, C.rowlen, C.rowinfo, C.col, C.small_list[1], 1, C.t_rank, C.stats, TC_STRAT_AUTO, sf, C.sup);
        count_launch();
        k_tc_small_hash<32, 64, SUP><<<L.sms * SMALL_BLOCKS, SMALL_WARPS * 32, 0, L.stream>>>(
            C.n, C.rowinfo, C.col, C.small_list[2], 2, C.t_rank, C.stats, C.sup);
        count_launch();
        k_tc_small_hash<32, 2 * SMALL_WIDE_MAX, SUP><<<L.sms * SMALL_WIDE_BLOCKS, SMALL_WARPS * 32, 0, L.stream>>>(
            C.n, C.rowinfo, C.col, C.small_list[3], 3, C.t_rank, C.stats, C.sup);
        count_launch();
    } else {
        k_tc_small<8, SUP><<<L.sms * SMALL_BLOCKS, SMALL_WARPS * 32, 0, L.stream>>>(
            C.n, C.rowstart, C.rowlen, C.rowinfo, C.col, C.small_list[0], 0, C.t_rank, C.stats, ss, sf, C.sup);
        count_launch();
        k_tc_small<16, SUP><<<L.sms * SMALL_BLOCKS, SMALL_WARPS * 32, 0, L.stream>>>(
            C.n, C.rowstart, C.rowlen, C.rowinfo, C.col, C.small_list[1], 1, C.t_rank, C.stats, ss, sf, C.sup);
        count_launch();
        k_tc_small<32, SUP><<<L.sms * SMALL_BLOCKS, SMALL_WARPS * 32, 0, L.stream>>>(
            C.n, C.rowstart, C.rowlen, C.rowinfo, C.col, C.small_list[2], 2, C.t_rank, C.stats, ss, sf, C.sup);
        count_launch();
        k_tc_small_wide<SUP><<<L.sms * SMALL_WIDE_BLOCKS, SMALL_WARPS * 32,
                          2 * SMALL_WIDE_GROUPS * SMALL_WIDE_MAX * sizeof(int32_t), L.stream>>>(
            C.n, C.rowinfo, C.col, C.small_list[3], C.t_rank, C.stats, ss, sf, C.sup);
        count_launch();
    }
    if (ev) cudaEventRecord(ev[PH_CTA], L.stream);
    cudaMemsetAsync(&C.stats->cta_next, 0, sizeof(unsigned), L.stream);
    k_tc_cta<SUP><<<L.sms * 4, CTA_THREADS, sizeof(CtaShared), L.stream>>>(C.n, C.rowstart, C.rowlen, C.rowinfo, C.col,
                                                                     C.cta_list,
                                                                     C.t_rank, C.stats, S.strat[TC_BUCKET_CTA],
                                                                     S.factor[TC_BUCKET_CTA], C.sup);
    count_launch();
    // the hub lists and the dense core come from the planner's second stream
    if (C.hub_ready) cudaStreamWaitEvent(L.stream, C.hub_ready, 0);
    if (ev) cudaEventRecord(ev[PH_HUB], L.stream);
    if (C.hub_cap > 0) {
        if (S.hub_core > 0) launch_core_count(C, L);
        cudaMemsetAsync(&C.stats->hub_next, 0, 2 * sizeof(unsigned), L.stream);
        k_tc_hub<SUP><<<L.sms * HUB_BLOCKS, HUB_THREADS, sizeof(HubShared), L.stream>>>(
            C.n, C.hub_cap, C.rowstart, C.rowlen, C.col, C.hub_start, C.big_list, C.med_list, C.in_rec, C.t_rank,
            C.stats, S.strat[TC_BUCKET_HUB] == TC_STRAT_PROBE ? 1 : 0, C.sup);
        count_launch();
    }
    if (ev) cudaEventRecord(ev[PH_END], L.stream);
}

// The plain count, or the count that also records every triangle's three edges in
// C.sup (tc_edge_support), from the same kernels compiled twice.
void launch_intersect(const CountBuffers& C, const Strategy& S, cudaEvent_t* ev, const Launch& L) {
    if (C.sup)
        intersect_impl<true>(C, S, ev, L);
    else
        intersect_impl<false>(C, S, ev, L);
}

void launch_sum_t(const CountBuffers& C, const Launch& L) {
    if (C.n <= 0) return;
    k_sum_t<<<grid_for(C.n, THREADS, L.sms), THREADS, 0, L.stream>>>(C.n, C.t_rank, C.stats);
    count_launch();
}

void launch_finalize(int32_t n, const int32_t* rank, const unsigned long long* t_rank, const int32_t* deg,
                     unsigned long long* t_out, double* lcc_out, const Launch& L) {
    if (n <= 0) return;
    k_finalize<<<grid_for(n, THREADS, L.sms), THREADS, 0, L.stream>>>(n, rank, t_rank, deg, t_out, lcc_out);
    count_launch();
}

}  // namespace tcg
