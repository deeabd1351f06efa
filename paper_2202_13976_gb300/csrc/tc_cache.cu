// Remote adjacency reads of the distributed algorithm (Sec. IV-A, Alg. 4) and the
// caches of Sec. IV-B, evaluated for many cache sizes at once.
//
// 1D partition: process k owns the ids [floor(k n / p), floor((k+1) n / p)).  Process k
// walks its vertices v_i in id order and every v_j of the sorted list adj(v_i); when
// v_j belongs to another process it reads adj(v_j) remotely (4 deg(v_j) bytes) after
// reading the offsets of v_j (one 16-byte entry).  Two caches sit in front of the two
// remote windows (adjacency lists, offsets), each under two policies:
//  - LRU: a miss inserts the entry as the most recent and evicts the least recent
//    until the entries fit.  Whatever the size, the cache holds the longest run of
//    most recently read entries that fits, so the read at time t of x hits a cache of
//    K bytes iff x was read before (at p = prev(t)) and
//      D(t) = size(x) + sum of the sizes of the distinct entries read in (p, t) <= K.
//    The distinct entries of (p, t) are the reads t' in (p, t) with prev(t') < p, so
//      D(t) = size(x) + F(t, p) - S(p),  F(t, p) = sum over t' < t with prev(t') < p,
//    S(p) = sum over t' <= p (every such t' has prev(t') < p).  F is a sum over points
//    (t', prev(t') + 1) dominated by the query (t, p + 1): answered for all reads
//    together by a merge-sort tree over time, level by level (level l holds the keys
//    sorted within aligned blocks of 2^l reads, with prefix sums of the weights);
//    [0, t) splits into one block per set bit of t, the blocks of the five lowest bits
//    read directly.  All levels are kept (12 bytes per read and level), so a query
//    walks them in one thread with its sums in registers.
//  - degree score (Sec. IV-B2): whenever an entry must be evicted, the victim is the
//    cached entry of the lowest (degree, id); a miss is stored after evicting the
//    lowest entries until it fits, unless it is larger than the whole cache (then it
//    is not stored and nothing is evicted).  This policy has no inclusion property
//    across sizes (a small entry admitted into the free room of a small cache can be
//    missing from a larger one), so every (cache, process, capacity) is simulated
//    directly: one warp per simulation walks the process's reads in time order, the
//    cache a two-level bitmap over the process's distinct entries ranked by score
//    (bit r of level 1 set iff the entry of rank r is cached; a bit of level 2 per
//    non-zero word of level 1), with the 32 lowest cached entries and their sizes in
//    a sorted buffer across the warp's registers, so that an eviction is a shuffle
//    and the sizes of evicted entries are loaded 32 at a time.  32 reads are tested
//    at once; each miss is applied (evictions, then the insertion) and the reads after
//    it are tested again.
#include <cuda_runtime.h>

#include <climits>
#include <cstring>
#include <vector>

#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {
namespace {

constexpr int RC_THREADS = 256;
constexpr uint32_t RC_NEVER = 0xffffffffu;  // a key no threshold counts
constexpr int RC_LOW = 5;                   // tree levels below this are read directly

__host__ __device__ __forceinline__ int32_t owner_of(int64_t i, int64_t n, int64_t parts) {
    return (int32_t)(((i + 1) * parts - 1) / n);
}

__global__ void k_rc_id_of(int32_t n, const int32_t* __restrict__ rank, int32_t* __restrict__ id_of) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) id_of[rank[v]] = (int32_t)v;
}

// Simple degree per id, and score keys (degree << b) | id: a stable sort of the degree
// field orders the ids by (degree, id); prank[id] = position.
__global__ void k_rc_score_keys(int32_t n, const int32_t* __restrict__ rank, const int32_t* __restrict__ deg_rank,
                                int b, uint32_t* __restrict__ sdeg, uint64_t* __restrict__ vkeys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t d = (uint32_t)deg_rank[rank[v]];
        sdeg[v] = d;
        vkeys[v] = ((uint64_t)d << b) | (uint64_t)v;
    }
}

__global__ void k_rc_prank(int32_t n, const uint64_t* __restrict__ vsorted, int b, int32_t* __restrict__ prank) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t mask = (1ull << b) - 1;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
        prank[vsorted[p] & mask] = (int32_t)p;
}

// Both directions of every oriented entry as id keys (i << b) | j, at 2 (estart[r] + p).
__global__ void k_rc_sym_keys(int32_t n, const int64_t* __restrict__ rowstart, const int32_t* __restrict__ rowlen,
                              const int32_t* __restrict__ col, const int64_t* __restrict__ estart,
                              const int32_t* __restrict__ id_of, int b, uint64_t* __restrict__ keys) {
    const int lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        const int d = rowlen[r];
        const int64_t a0 = rowstart[r], e0 = estart[r];
        const uint64_t iu = (uint32_t)id_of[r];
        for (int p = lane; p < d; p += 32) {
            const uint64_t iv = (uint32_t)id_of[col[a0 + p]];
            keys[2 * (e0 + p)] = (iu << b) | iv;
            keys[2 * (e0 + p) + 1] = (iv << b) | iu;
        }
    }
}

// flag[s] = 1 for a symmetric entry (i, j) whose ends lie in different processes.
__global__ void k_rc_remote_flags(int64_t ms2, const uint64_t* __restrict__ sym, int b, int32_t n, int32_t parts,
                                  uint32_t* __restrict__ flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t mask = (1ull << b) - 1;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ms2; s += stride) {
        const uint64_t key = sym[s];
        flag[s] = owner_of((int64_t)(key >> b), n, parts) != owner_of((int64_t)(key & mask), n, parts) ? 1u : 0u;
    }
}

// Adds v to field[k] once per group of lanes that share k (k < 0: nothing); every lane
// of the warp calls it.
__device__ __forceinline__ void part_add3(int32_t k, unsigned long long v0, unsigned long long v1,
                                          unsigned long long v2, unsigned long long* f0, unsigned long long* f1,
                                          unsigned long long* f2) {
    unsigned pending = __ballot_sync(FULL, k >= 0);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int32_t kl = __shfl_sync(FULL, k, leader);
        const bool mine = k == kl;
        const unsigned long long s0 = warp_sum(mine ? v0 : 0ull);
        const unsigned long long s1 = warp_sum(mine ? v1 : 0ull);
        const unsigned long long s2 = warp_sum(mine ? v2 : 0ull);
        if (lane_id() == leader) {
            if (s0 && f0) atomicAdd(f0 + 4 * kl, s0);
            if (s1 && f1) atomicAdd(f1 + 4 * kl, s1);
            if (s2 && f2) atomicAdd(f2 + 4 * kl, s2);
        }
        pending &= ~__ballot_sync(FULL, mine);
    }
}

// The read stream: item[t] = v_j, part[t] = process of v_i, in (i, j) order; per-process
// reads, reads of the top decile (score rank >= n - ceil(n / 10)) and bytes.
__global__ void k_rc_stream(int64_t ms2, const uint64_t* __restrict__ sym, int b, int32_t n, int32_t parts,
                            const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                            const int32_t* __restrict__ prank, const uint32_t* __restrict__ sdeg,
                            int32_t* __restrict__ item, int32_t* __restrict__ part, PartCounters* __restrict__ pc) {
    const int lane = lane_id();
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t mask = (1ull << b) - 1;
    const int32_t top_rank = n - (int32_t)(((int64_t)n + 9) / 10);  // ranks >= this: the top decile
    for (int64_t base = warp0 * 32; base < ms2; base += wstride * 32) {  // uniform per warp
        const int64_t s = base + lane;
        int32_t k = -1;
        unsigned long long top = 0, bytes = 0;
        if (s < ms2 && flag[s]) {
            const uint64_t key = sym[s];
            const int32_t i = (int32_t)(key >> b), j = (int32_t)(key & mask);
            const int64_t t = pos[s];
            k = owner_of(i, n, parts);
            item[t] = j;
            part[t] = k;
            top = prank[j] >= top_rank ? 1 : 0;
            bytes = 4ull * (unsigned long long)sdeg[j];
        }
        part_add3(k, 1ull, top, bytes, &pc->reads, &pc->top_reads, &pc->read_bytes);
    }
}

// Reuse keys (item << 32) | t: a stable sort of the item field lists every item's
// reads in time order.
__global__ void k_rc_item_keys(int64_t N, const int32_t* __restrict__ item, uint64_t* __restrict__ keys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += stride)
        keys[t] = ((uint64_t)(uint32_t)item[t] << 32) | (uint64_t)t;
}

// prev[t] = the previous read of the same item by the same process (-1: first read).
// The processes' reads are contiguous in time, so it is the item's previous read when
// that read belongs to the same process.
__global__ void k_rc_prev(int64_t N, const uint64_t* __restrict__ sorted, const int32_t* __restrict__ part,
                          int64_t* __restrict__ prev) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += stride) {
        const uint64_t key = sorted[s];
        const int64_t t = (int64_t)(key & 0xffffffffull);
        int64_t p = -1;
        if (s > 0) {
            const uint64_t q = sorted[s - 1];
            const int64_t tq = (int64_t)(q & 0xffffffffull);
            if ((q >> 32) == (key >> 32) && part[tq] == part[t]) p = tq;
        }
        prev[t] = p;
    }
}

// Inputs of the LRU dominance sum and its queries: key = prev + 1, weight deg; query
// (t, prev(t) + 1) for every read.  Also counts every process's first reads.
__global__ void k_rc_inputs(int64_t N, const int32_t* __restrict__ item, const int32_t* __restrict__ part,
                            const int64_t* __restrict__ prev, const uint32_t* __restrict__ sdeg,
                            uint32_t* __restrict__ key_lru, uint32_t* __restrict__ wdeg,
                            int64_t* __restrict__ q_lru, uint32_t* __restrict__ th_lru,
                            PartCounters* __restrict__ pc) {
    const int lane = lane_id();
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp0 * 32; base < N; base += wstride * 32) {  // uniform per warp
        const int64_t t = base + lane;
        int32_t first_k = -1;
        if (t < N) {
            const int32_t x = item[t];
            const int64_t p = prev[t];
            key_lru[t] = (uint32_t)(p + 1);
            wdeg[t] = sdeg[x];
            q_lru[t] = t;
            th_lru[t] = (uint32_t)(p + 1);
            if (p < 0) first_k = part[t];
        }
        part_add3(first_k, 1ull, 0ull, 0ull, &pc->distinct, nullptr, nullptr);
    }
}

// pstart[k] = first read of process k (k = 0 .. parts).
__global__ void k_rc_pstart(int64_t N, int32_t parts, const int32_t* __restrict__ part, int64_t* __restrict__ pstart) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= parts; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = N;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (part[mid] < k)
                lo = mid + 1;
            else
                hi = mid;
        }
        pstart[k] = lo;
    }
}

// Level l -> l + 1 of the merge-sort tree: the two sorted halves of each block of
// 2^(l+1) reads are merged (stable: the left half first among equal keys).
__global__ void k_rc_merge(int64_t N, int l, const uint32_t* __restrict__ key, const uint32_t* __restrict__ wa,
                           uint32_t* __restrict__ key2, uint32_t* __restrict__ wa2) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t B = (int64_t)1 << l;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const int64_t base = (i >> (l + 1)) << (l + 1);
        const bool left = i - base < B;
        const uint32_t x = key[i];
        int64_t lo, hi;
        if (left) {  // count the right half's keys < x
            lo = base + B;
            hi = min(base + 2 * B, N);
            const int64_t r0 = lo;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (key[mid] < x)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            const int64_t out = base + (i - base) + (lo - r0);
            key2[out] = x;
            wa2[out] = wa[i];
        } else {  // count the left half's keys <= x
            lo = base;
            hi = base + B;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (key[mid] <= x)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            const int64_t out = base + (i - base - B) + (lo - base);
            key2[out] = x;
            wa2[out] = wa[i];
        }
    }
}

// Level RC_LOW of the tree: each aligned block of 32 reads sorted by key, one warp per
// block (the order among equal keys does not matter to the sums).
__global__ void k_rc_sort32(int64_t N, const uint32_t* __restrict__ key0, const uint32_t* __restrict__ w0,
                            uint32_t* __restrict__ key, uint32_t* __restrict__ wa) {
    static_assert(RC_LOW == 5, "one warp per block of 2^RC_LOW reads");
    const int lane = lane_id();
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp0 * 32; base < N; base += wstride * 32) {  // uniform per warp
        const int64_t t = base + lane;
        const uint32_t x = t < N ? key0[t] : 0xffffffffu;
        int r = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const uint32_t y = __shfl_sync(FULL, x, j);
            r += (y < x) || (y == x && j < lane);
        }
        if (t < N) {
            key[base + r] = x;
            wa[base + r] = w0[t];
        }
    }
}

// Every query in one thread: the reads [q & ~31, q) directly in time order, then for
// every level l >= RC_LOW with bit l of q set, the block [(q >> (l+1)) << (l+1), + 2^l)
// of level l adds the entry sizes of its keys < th (sa) and their number (sb).
__global__ void k_rc_query(int64_t M, const int64_t* __restrict__ q, const uint32_t* __restrict__ th,
                           const uint32_t* __restrict__ key0, const uint32_t* __restrict__ w0, int64_t N, int nlev,
                           const uint32_t* __restrict__ lk, const int64_t* __restrict__ le,
                           int64_t* __restrict__ sa, int64_t* __restrict__ sb) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        const int64_t qi = q[i];
        const uint32_t x = th[i];
        int64_t a = 0, c = 0;
        for (int64_t t = qi & ~(int64_t)((1 << RC_LOW) - 1); t < qi; ++t)
            if (key0[t] < x) {
                a += w0[t];
                ++c;
            }
        for (int j = 0; j < nlev; ++j) {
            const int l = RC_LOW + j;
            if (!((qi >> l) & 1)) continue;
            const int64_t start = (qi >> (l + 1)) << (l + 1);
            const uint32_t* K = lk + (int64_t)j * N;
            int64_t lo = start, hi = start + ((int64_t)1 << l);
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (K[mid] < x)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            const int64_t* E = le + (int64_t)j * (N + 1);
            a += E[lo] - E[start];
            c += lo - start;
        }
        sa[i] = a;
        sb[i] = c;
    }
}

// LRU hits per (cache, process, first capacity that holds the read); cache 0 holds
// adjacency lists, cache 1 offsets.
__global__ void k_rc_hist(int64_t N, int32_t parts, int ncap, const uint64_t* __restrict__ caps,
                          const int32_t* __restrict__ part, const int64_t* __restrict__ prev,
                          const uint32_t* __restrict__ wdeg, const int64_t* __restrict__ e0deg,
                          const int64_t* __restrict__ f_lru_deg, const int64_t* __restrict__ f_lru_one,
                          unsigned long long* __restrict__ cnt, unsigned long long* __restrict__ byt) {
    extern __shared__ unsigned long long sh[];
    const int cells = 2 * parts * ncap;
    const bool local = cells <= RC_HIST_SHARED;
    unsigned long long* scnt = sh;
    unsigned long long* sbyt = sh + (local ? cells : 0);
    if (local)
        for (int i = threadIdx.x; i < 2 * cells; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += stride) {
        const int64_t p = prev[t];
        if (p < 0) continue;  // a first read misses every cache
        const int k = part[t];
        const uint64_t d = wdeg[t];  // deg(v_j)
        uint64_t need[2], size[2];
        need[0] = 4 * (d + (uint64_t)(f_lru_deg[t] - e0deg[p + 1]));  // adjacency
        need[1] = 16 * (1 + (uint64_t)(f_lru_one[t] - (p + 1)));       // offsets
        size[0] = 4 * d;
        size[1] = 16;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            int lo = 0, hi = ncap;  // first capacity >= need
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (caps[mid] < need[c])
                    lo = mid + 1;
                else
                    hi = mid;
            }
            if (lo == ncap) continue;
            const int cell = (c * parts + k) * ncap + lo;
            if (local) {
                atomicAdd(&scnt[cell], 1ull);
                atomicAdd(&sbyt[cell], (unsigned long long)size[c]);
            } else {
                atomicAdd(&cnt[cell], 1ull);
                atomicAdd(&byt[cell], (unsigned long long)size[c]);
            }
        }
    }
    if (local) {
        __syncthreads();
        for (int i = threadIdx.x; i < cells; i += blockDim.x) {
            if (scnt[i]) atomicAdd(&cnt[i], scnt[i]);
            if (sbyt[i]) atomicAdd(&byt[i], sbyt[i]);
        }
    }
}

// ---- degree-score caches: direct simulation ---------------------------------------

// Score keys of the reads: (process << b) | score position of the entry read.
__global__ void k_rc_ukeys(int64_t N, const int32_t* __restrict__ item, const int32_t* __restrict__ part,
                           const int32_t* __restrict__ prank, int b, uint64_t* __restrict__ ukeys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += stride)
        ukeys[t] = ((uint64_t)(uint32_t)part[t] << b) | (uint64_t)(uint32_t)prank[item[t]];
}

__global__ void k_rc_uflags(int64_t N, const uint64_t* __restrict__ sorted, uint32_t* __restrict__ flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        flag[i] = (i == 0 || sorted[i] != sorted[i - 1]) ? 1u : 0u;
}

// The distinct (process, entry) keys in order, with the degree of each entry (the
// degree field of its (degree << b) | id score key).
__global__ void k_rc_ucompact(int64_t N, const uint64_t* __restrict__ sorted, const uint32_t* __restrict__ flag,
                              const uint32_t* __restrict__ pos, const uint64_t* __restrict__ vsorted, int b,
                              uint64_t* __restrict__ ukeys, uint32_t* __restrict__ udeg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t mask = (1ull << b) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        if (flag[i]) {
            const uint32_t u = pos[i];
            ukeys[u] = sorted[i];
            udeg[u] = (uint32_t)(vsorted[sorted[i] & mask] >> b);
        }
}

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* __restrict__ a, int64_t count, uint64_t x) {
    int64_t lo = 0, hi = count;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// ubase[k] = index of process k's first distinct key (k = 0 .. parts).
__global__ void k_rc_ubase(int32_t parts, const uint64_t* __restrict__ ukeys, const uint32_t* __restrict__ U, int b,
                           int64_t* __restrict__ ubase) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= parts; k += (int64_t)gridDim.x * blockDim.x)
        ubase[k] = lower_bound_u64(ukeys, (int64_t)*U, (uint64_t)k << b);
}

// lr[t] = score rank of the entry read at t among its process's distinct entries
// (0 = lowest (degree, id)).
__global__ void k_rc_local_rank(int64_t N, const int32_t* __restrict__ item, const int32_t* __restrict__ part,
                                const int32_t* __restrict__ prank, int b, const uint64_t* __restrict__ ukeys,
                                const uint32_t* __restrict__ U, const int64_t* __restrict__ ubase,
                                int32_t* __restrict__ lr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t u = (int64_t)*U;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += stride) {
        const int32_t k = part[t];
        const uint64_t key = ((uint64_t)(uint32_t)k << b) | (uint64_t)(uint32_t)prank[item[t]];
        lr[t] = (int32_t)(lower_bound_u64(ukeys, u, key) - ubase[k]);
    }
}

constexpr uint32_t RC_EMPTY = 0xffffffffu;

// Refill of a simulation's buffer: the up to 32 lowest cached ranks >= F, found in the
// level-1 bitmap 32 words at a time, empty stretches skipped through level 2.  Lane l
// receives the l-th of them (RC_EMPTY beyond the count); *F_out = one past the 32nd
// (RC_EMPTY when fewer than 32 remain, i.e. every cached rank is now in the buffer).
__device__ int rc_refill(const uint32_t* L1, const uint32_t* L2, uint32_t W1, uint32_t W2, uint32_t F,
                         uint32_t* sbuf, uint32_t* rank_out, uint32_t* F_out) {
    const int lane = lane_id();
    int found = 0;
    uint32_t w0 = F >> 5;
    bool first = true;
    while (found < 32 && w0 < W1) {
        const uint32_t w = w0 + lane;
        uint32_t word = w < W1 ? L1[w] : 0u;
        if (first && lane == 0) word &= 0xffffffffu << (F & 31);
        first = false;
        const int c = __popc(word);
        const int incl = warp_inclusive_scan(c);
        const int tot = __shfl_sync(FULL, incl, 31);
        if (tot == 0) {  // next non-zero level-1 word at or after w0 + 32, from level 2
            uint32_t q = w0 + 32, nxt = RC_EMPTY;
            while (q < W1) {
                const uint32_t w2 = (q >> 5) + lane;
                uint32_t x = w2 < W2 ? L2[w2] : 0u;
                if (lane == 0) x &= 0xffffffffu << (q & 31);
                const unsigned nz = __ballot_sync(FULL, x != 0u);
                if (nz) {
                    const int l = __ffs(nz) - 1;
                    const uint32_t xl = __shfl_sync(FULL, x, l);
                    nxt = (((q >> 5) + (uint32_t)l) << 5) + (uint32_t)(__ffs(xl) - 1);
                    break;
                }
                q = ((q >> 5) + 32) << 5;
            }
            if (nxt == RC_EMPTY) break;
            w0 = nxt;
            continue;
        }
        int slot = found + incl - c;
        uint32_t x = word;
        while (x && slot < 32) {
            const int bit = __ffs(x) - 1;
            x &= x - 1;
            sbuf[slot++] = (w << 5) + (uint32_t)bit;
        }
        found = min(32, found + tot);
        w0 += 32;
    }
    __syncwarp();
    *rank_out = lane < found ? sbuf[lane] : RC_EMPTY;
    *F_out = found == 32 ? sbuf[31] + 1 : RC_EMPTY;
    __syncwarp();
    return found;
}

// One warp per simulation job = (cache, process, capacity); cache 0 holds adjacency
// lists (4 deg bytes per entry), cache 1 offsets (16 bytes).  The cache is a bitmap
// over the process's score ranks (L1: a bit per rank; L2: a bit per non-zero L1 word),
// in shared memory (SHARED) or at gstate + job * (W1 + W2).  The lowest cached ranks
// and their sizes sit in a buffer in registers, sorted across the lanes: lane l holds
// the l-th lowest of the nb buffered entries, and every cached rank below F is in the
// buffer.  An eviction takes lane 0's entry; an insertion below F goes into the
// buffer (pushing its highest entry out, which lowers F, when it is full); an empty
// buffer is refilled from the bitmap.
template <bool SHARED>
__global__ void __launch_bounds__(32) k_rc_score_sim(int32_t parts, int ncap, const uint64_t* __restrict__ caps,
                                                     const int64_t* __restrict__ pstart,
                                                     const int32_t* __restrict__ lr,
                                                     const uint32_t* __restrict__ wdeg,
                                                     const int64_t* __restrict__ ubase,
                                                     const uint32_t* __restrict__ udeg, uint32_t W1, uint32_t W2,
                                                     uint32_t* __restrict__ gstate,
                                                     unsigned long long* __restrict__ out_cnt,
                                                     unsigned long long* __restrict__ out_byt) {
    extern __shared__ uint32_t rc_sim_sh[];
    __shared__ uint32_t sbuf[32];
    const int lane = threadIdx.x;
    const int64_t per_kind = (int64_t)parts * ncap;
    const int64_t jobs = 2 * per_kind;
    const uint32_t words = W1 + W2;
    for (int64_t job = blockIdx.x; job < jobs; job += gridDim.x) {
        const int kind = (int)(job / per_kind);
        const int64_t rem = job - kind * per_kind;
        const int32_t k = (int32_t)(rem / ncap);
        const int c = (int)(rem - (int64_t)k * ncap);
        uint32_t* L1 = SHARED ? rc_sim_sh : gstate + job * (int64_t)words;
        uint32_t* L2 = L1 + W1;
        for (uint32_t i = lane; i < words; i += 32) L1[i] = 0;
        __syncwarp();
        const uint64_t K = caps[c];
        const int64_t t0 = pstart[k], t1 = pstart[k + 1];
        const uint32_t* ud = udeg + ubase[k];
        unsigned long long h = 0, hb = 0;
        uint64_t used = 0;  // bytes held (the same in every lane)
        uint32_t brank = RC_EMPTY, F = RC_EMPTY;
        uint64_t bsize = 0;
        int nb = 0;
        bool broken = false;  // the buffer found no entry to evict (cannot happen while used > 0)
        for (int64_t base = t0; base < t1 && !broken; base += 32) {
            const int64_t t = base + lane;
            const bool valid = t < t1;
            const uint32_t r = valid ? (uint32_t)lr[t] : 0u;
            const uint64_t sz = valid ? (kind == 0 ? 4ull * wdeg[t] : 16ull) : 0ull;
            unsigned pending = __ballot_sync(FULL, valid);
            while (pending) {
                const bool in = ((pending >> lane) & 1u) && ((L1[r >> 5] >> (r & 31)) & 1u);
                const unsigned inm = __ballot_sync(FULL, in);
                const unsigned missm = pending & ~inm;
                const int i = missm ? __ffs(missm) - 1 : 32;
                const unsigned before = i == 32 ? 0xffffffffu : ((1u << i) - 1u);
                if (in && ((before >> lane) & 1u)) {
                    ++h;
                    hb += sz;
                }
                if (i == 32) break;
                pending &= i == 31 ? 0u : (0xffffffffu << (i + 1));
                const uint32_t ri = __shfl_sync(FULL, r, i);
                const uint64_t si = __shfl_sync(FULL, sz, i);
                if (si > K) continue;  // larger than the cache: not stored, nothing evicted
                while (used + si > K) {  // used > 0: the cache holds an entry
                    if (nb == 0) {
                        nb = rc_refill(L1, L2, W1, W2, F, sbuf, &brank, &F);
                        bsize = lane < nb ? (kind == 0 ? 4ull * ud[brank] : 16ull) : 0ull;
                        if (nb == 0) {
                            broken = true;
                            break;
                        }
                    }
                    const uint32_t v = __shfl_sync(FULL, brank, 0);
                    used -= __shfl_sync(FULL, bsize, 0);
                    if (lane == 0) {  // clear bit v
                        const uint32_t w = v >> 5, nw = L1[w] & ~(1u << (v & 31));
                        L1[w] = nw;
                        if (!nw) L2[w >> 5] &= ~(1u << (w & 31));
                    }
                    __syncwarp();
                    brank = __shfl_down_sync(FULL, brank, 1);
                    bsize = __shfl_down_sync(FULL, bsize, 1);
                    --nb;
                    if (lane >= nb) brank = RC_EMPTY;
                }
                if (broken) break;
                if (lane == 0) {  // set bit ri
                    const uint32_t w = ri >> 5, o = L1[w];
                    L1[w] = o | (1u << (ri & 31));
                    if (!o) L2[w >> 5] |= 1u << (w & 31);
                }
                __syncwarp();
                used += si;
                if (ri < F) {
                    const uint32_t top = __shfl_sync(FULL, brank, 31);
                    if (nb == 32 && ri > top) {
                        F = ri;
                    } else {
                        const int pos = __popc(__ballot_sync(FULL, brank < ri));
                        const uint32_t up_r = __shfl_up_sync(FULL, brank, 1);
                        const uint64_t up_s = __shfl_up_sync(FULL, bsize, 1);
                        if (lane > pos) {
                            brank = up_r;
                            bsize = up_s;
                        } else if (lane == pos) {
                            brank = ri;
                            bsize = si;
                        }
                        if (nb == 32)
                            F = top;  // the highest entry left the buffer
                        else
                            ++nb;
                    }
                }
            }
        }
        h = warp_sum(h);
        hb = warp_sum(hb);
        if (lane == 0) {
            out_cnt[job] = broken ? RC_SIM_BROKEN : h;
            out_byt[job] = hb;
        }
        __syncwarp();
    }
}

}  // namespace

int rc_levels(int64_t N) {
    int k = 0;
    while (((int64_t)1 << (RC_LOW + k)) <= N) ++k;
    return k;
}

int rc_key_bits(int32_t n) {
    int b = 1;
    while (b < 31 && ((int64_t)1 << b) < (int64_t)n) ++b;
    return b;
}

void launch_rc_stream(RemoteCacheBuffers& R, const Launch& L) {
    const int sms = L.sms;
    const int b = rc_key_bits(R.n);
    k_rc_id_of<<<grid_for(R.n, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(R.n, R.rank, R.id_of);
    count_launch();
    k_rc_score_keys<<<grid_for(R.n, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(R.n, R.rank, R.deg, b, R.sdeg,
                                                                                 R.vkeys);
    count_launch();
    uint64_t* vs = radix_sort_u64(R.vkeys, R.vkeys_alt, R.n, b, 2 * b, R.radix_tmp, L);
    R.vsorted = vs;
    k_rc_prank<<<grid_for(R.n, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(R.n, vs, b, R.prank);
    count_launch();
    scan_u32_to_i64(reinterpret_cast<const uint32_t*>(R.rowlen), R.estart, R.n, R.scan_tmp, L);
    k_rc_sym_keys<<<grid_for((int64_t)R.n * 32, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(
        R.n, R.rowstart, R.rowlen, R.col, R.estart, R.id_of, b, R.keys);
    count_launch();
    uint64_t* sym = radix_sort_u64(R.keys, R.keys_alt, R.ms2, 0, 2 * b, R.radix_tmp, L);
    k_rc_remote_flags<<<grid_for(R.ms2, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(R.ms2, sym, b, R.n, R.parts,
                                                                                     R.flag);
    count_launch();
    scan_u32_to_u32(R.flag, R.pos, R.ms2, R.scan_tmp, L);
    k_rc_stream<<<grid_for(R.ms2, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(
        R.ms2, sym, b, R.n, R.parts, R.flag, R.pos, R.prank, R.sdeg, R.item, R.part, R.pc);
    count_launch();
}

void launch_rc_caches(const RemoteCacheBuffers& R, int64_t N, const Launch& L) {
    const int sms = L.sms;
    const int b = rc_key_bits(R.n);
    // previous reads
    k_rc_item_keys<<<grid_for(N, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(N, R.item, R.keys);
    count_launch();
    uint64_t* byitem = radix_sort_u64(R.keys, R.keys_alt, N, 32, 32 + b, R.radix_tmp, L);
    k_rc_prev<<<grid_for(N, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(N, byitem, R.part, R.prev);
    count_launch();
    k_rc_pstart<<<1, RC_THREADS, 0, L.stream>>>(N, R.parts, R.part, R.pstart);
    count_launch();
    k_rc_inputs<<<grid_for(N, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(
        N, R.item, R.part, R.prev, R.sdeg, R.key_lru, R.wdeg, R.q_lru, R.th_lru, R.pc);
    count_launch();
    // S(p): prefix sums of the weights in time order (level 0)
    scan_u32_to_i64(R.wdeg, R.e0deg, N, R.scan_tmp, L);
    // the LRU merge-sort tree: every level is built and kept, then each query walks
    // them all in one thread
    const int nlev = rc_levels(N);
    if (nlev > 0) {
        k_rc_sort32<<<grid_for(N, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(N, R.key_lru, R.wdeg, R.lk, R.la[0]);
        count_launch();
    }
    for (int j = 0; j < nlev; ++j) {
        uint32_t* wa = R.la[j & 1];
        scan_u32_to_i64(wa, R.le + (int64_t)j * (N + 1), N, R.scan_tmp, L);
        if (j + 1 < nlev) {
            k_rc_merge<<<grid_for(N, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(
                N, RC_LOW + j, R.lk + (int64_t)j * N, wa, R.lk + (int64_t)(j + 1) * N, R.la[(j + 1) & 1]);
            count_launch();
        }
    }
    k_rc_query<<<grid_for(N, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(N, R.q_lru, R.th_lru, R.key_lru, R.wdeg, N,
                                                                          nlev, R.lk, R.le, R.f_lru_deg, R.f_lru_one);
    count_launch();
    const int cells = 2 * R.parts * R.ncap;
    const size_t shmem = cells <= RC_HIST_SHARED ? 2 * sizeof(unsigned long long) * (size_t)cells : 0;
    k_rc_hist<<<grid_for(N, RC_THREADS, sms, 4), RC_THREADS, shmem, L.stream>>>(
        N, R.parts, R.ncap, R.caps, R.part, R.prev, R.wdeg, R.e0deg, R.f_lru_deg, R.f_lru_one, R.cnt, R.byt);
    count_launch();
    // score ranks of the reads within their processes, for the score simulations
    k_rc_ukeys<<<grid_for(N, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(N, R.item, R.part, R.prank, b, R.keys);
    count_launch();
    const uint64_t* sorted = radix_sort_u64(R.keys, R.keys_alt, N, 0, 2 * b, R.radix_tmp, L);
    k_rc_uflags<<<grid_for(N, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(N, sorted, R.flag);
    count_launch();
    scan_u32_to_u32(R.flag, R.pos, N, R.scan_tmp, L);
    k_rc_ucompact<<<grid_for(N, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(N, sorted, R.flag, R.pos, R.vsorted, b,
                                                                             R.ukeys, R.udeg);
    count_launch();
    k_rc_ubase<<<1, RC_THREADS, 0, L.stream>>>(R.parts, R.ukeys, R.pos + N, b, R.ubase);
    count_launch();
    k_rc_local_rank<<<grid_for(N, RC_THREADS, sms), RC_THREADS, 0, L.stream>>>(N, R.item, R.part, R.prank, b, R.ukeys,
                                                                               R.pos + N, R.ubase, R.lr);
    count_launch();
}

RcSimShape rc_sim_shape(int64_t max_distinct) {
    RcSimShape S;
    S.W1 = (uint32_t)((max_distinct + 31) / 32);
    if (S.W1 == 0) S.W1 = 1;
    S.W2 = (S.W1 + 31) / 32;
    S.bytes = 4 * (size_t)(S.W1 + S.W2);
    S.shared = S.bytes <= RC_SIM_SHARED_MAX;
    return S;
}

void launch_rc_score(const RemoteCacheBuffers& R, const RcSimShape& S, const Launch& L) {
    const int64_t jobs = 2 * (int64_t)R.parts * R.ncap;
    if (jobs == 0) return;
    const unsigned grid = (unsigned)(jobs < (int64_t)INT_MAX ? jobs : (int64_t)INT_MAX);
    if (S.shared) {
        if (S.bytes > 40 * 1024)
            cudaFuncSetAttribute(k_rc_score_sim<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.bytes);
        k_rc_score_sim<true><<<grid, 32, S.bytes, L.stream>>>(R.parts, R.ncap, R.caps, R.pstart, R.lr, R.wdeg,
                                                               R.ubase, R.udeg, S.W1, S.W2, nullptr, R.sc_cnt,
                                                               R.sc_byt);
    } else {
        k_rc_score_sim<false><<<grid, 32, 0, L.stream>>>(R.parts, R.ncap, R.caps, R.pstart, R.lr, R.wdeg, R.ubase,
                                                          R.udeg, S.W1, S.W2, R.sim_state, R.sc_cnt, R.sc_byt);
    }
    count_launch();
}

}  // namespace tcg
