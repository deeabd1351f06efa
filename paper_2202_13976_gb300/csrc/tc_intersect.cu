// Per-edge set intersection over the degree-oriented CSR (Sec. II-C, Sec. IV-C),
// the planner that groups source vertices into degree buckets, and the final
// reduction to T (Sec. II-C) and LCC (Eq. 2).
//
// Counting rule.  In rank space every oriented row N+(u) is sorted and holds only
// ranks above u.  For the oriented edge (u, v) with v = N+(u)[j], the common
// neighbours are W = N+(u)[j+1 ..] ∩ N+(v): an element of N+(v) exceeds v, so only
// the suffix of N+(u) after v can match.  With c = |W|, a triangle {u, v, w}
// (u < v < w in rank order) is met exactly once, and t[u] += c, t[v] += c,
// t[w] += 1 for every w in W.
//
// Source-vertex staging.  One warp (d+(u) <= 32) or one thread block (d+(u) > 32)
// owns u: N+(u) is copied into shared memory once and reused by all d+(u) edges of
// u, and every increment aimed at an entry of N+(u) (t[v] += c and t[w] += 1) is
// first added to a shared-memory counter for that position.  One global atomic per
// non-zero counter and one for t[u] flush them.  This is the on-chip analogue of the
// paper's reuse of adjacency lists (Sec. IV-B): the staged list plays the role of a
// cached entry, kept for as long as its owner is processed.
//
// Methods for one edge (a warp; A = suffix of N+(u), B = N+(v)):
//  MERGE   merge path: the merge of A and B is cut into 32 equal diagonal ranges,
//          one per lane; each lane runs Alg. 2 over its range (Sec. II-C, SSI)
//  SEARCH  every key of A is looked up in B by binary search (Alg. 1)
//  PROBE   every element of B is looked up in A (staged, shared memory) by binary
//          search; the scan of B stops at the first element above max(N+(u))
//  BITMAP  like PROBE, but N+(u) is a bitmap over the rank window (u, max N+(u)]
//          with per-word prefix counts, so a probe is one shared-memory load
//  AUTO    Eq. 3 per edge: if |B|/|A| <= f (log2|B| - 1) with |A| <= |B| the
//          lists are merged (MERGE), otherwise the keys of the shorter list are
//          searched in the longer (SEARCH when A is shorter, PROBE when B is)
#include <climits>

#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {

namespace {

constexpr int THREADS = 256;
constexpr int WK_WARPS = 8;            // warps per block in the warp-bucket kernel
constexpr int CTA_THREADS = 256;       // block-bucket kernel
constexpr int CTA_WARPS = CTA_THREADS / 32;
constexpr int CTA_LIST_MAX = 2048;     // staged list capacity of one block
constexpr int BITMAP_WORDS = 4096;     // bitmap window of one block: 131072 ranks

struct Sink {
    uint32_t* cnt;               // per-position counters (shared), or null
    unsigned long long* t;       // global counts, used when cnt is null
    const int32_t* Lu;           // N+(u) (shared or global)
    __device__ __forceinline__ void hit(int p) const {
        if (cnt)
            atomicAdd(&cnt[p], 1u);
        else
            atomicAdd(&t[Lu[p]], 1ull);
    }
};

// Number of elements of sorted B[0, b) that are <= x (warp-uniform inputs).
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
                ++c;
            }
        }
        if (__any_sync(FULL, x > maxu)) break;  // B is sorted: later chunks exceed too
    }
    return warp_sum(c);
}

// Bitmap over ranks (u, maxu]: bit (x - u - 1) set iff x in N+(u); pre[w] = number of
// set bits in words before w, i.e. the position in N+(u) of the word's first member.
__device__ uint32_t edge_bitmap(const uint32_t* bm, const uint16_t* pre, int32_t u, int32_t maxu,
                                uint32_t* cnt, const int32_t* __restrict__ B, int b) {
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
                ++c;
            }
        }
        if (__any_sync(FULL, x > maxu)) break;
    }
    return warp_sum(c);
}

__device__ __forceinline__ int auto_method(int a, int b, float factor) {
    int s = min(a, b), l = max(a, b);
    bool ssi = (float)l <= factor * (log2f((float)l) - 1.0f) * (float)s;
    if (ssi) return TC_STRAT_MERGE;
    return a <= b ? TC_STRAT_SEARCH : TC_STRAT_PROBE;
}

__device__ __forceinline__ uint32_t edge_dispatch(int method, const Sink& S, int a0, int du,
                                                  const int32_t* __restrict__ B, int b) {
    switch (method) {
        case TC_STRAT_MERGE: return edge_merge(S, a0, du, B, b);
        case TC_STRAT_SEARCH: return edge_search(S, a0, du, B, b);
        default: return edge_probe(S, a0, du, B, b);
    }
}

// ---- planner -----------------------------------------------------------------

__global__ void k_plan(int32_t n, const int32_t* __restrict__ rowlen, int32_t* __restrict__ warp_list,
                       int32_t* __restrict__ cta_list, DevStats* stats) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // the loop bound is uniform across a warp, as warp_append needs all 32 lanes
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < n; b += stride) {
        const int64_t u = b + lane_id();
        const int d = u < n ? rowlen[u] : 0;
        const bool w = d >= 2 && d <= 32, c = d > 32;
        const unsigned pw = warp_append(w, &stats->warp_count);
        const unsigned pc = warp_append(c, &stats->cta_count);
        if (w) warp_list[pw] = (int32_t)u;
        if (c) cta_list[pc] = (int32_t)u;
    }
}

// ---- warp bucket: 2 <= d+(u) <= 32 ------------------------------------------------

__global__ void __launch_bounds__(WK_WARPS * 32) k_tc_warp(const int64_t* __restrict__ rowstart,
                                                           const int32_t* __restrict__ rowlen,
                                                           const int32_t* __restrict__ col,
                                                           const int32_t* __restrict__ list,
                                                           unsigned long long* __restrict__ t,
                                                           DevStats* stats, int strategy, float factor) {
    __shared__ int32_t sLu[WK_WARPS][32];
    __shared__ uint32_t sCnt[WK_WARPS][32];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const unsigned count = stats->warp_count;
    const unsigned warps = gridDim.x * WK_WARPS;
    for (unsigned q = blockIdx.x * WK_WARPS + w; q < count; q += warps) {
        const int32_t u = list[q];
        const int du = rowlen[u];
        const int64_t base = rowstart[u];
        sLu[w][lane] = lane < du ? col[base + lane] : INT_MAX;
        sCnt[w][lane] = 0;
        __syncwarp();
        Sink S{sCnt[w], t, sLu[w]};
        unsigned long long utot = 0;
        for (int j = 0; j < du - 1; ++j) {
            const int32_t v = sLu[w][j];
            const int dv = rowlen[v];
            if (dv == 0) continue;
            const int32_t* B = col + rowstart[v];
            const int a = du - j - 1;
            int method = strategy == TC_STRAT_AUTO ? auto_method(a, dv, factor) : strategy;
            uint32_t c = edge_dispatch(method, S, j + 1, du, B, dv);
            if (lane == 0 && c) atomicAdd(&sCnt[w][j], c);
            utot += c;
        }
        __syncwarp();
        uint32_t cv = sCnt[w][lane];
        if (lane < du && cv) atomicAdd(&t[sLu[w][lane]], (unsigned long long)cv);
        if (lane == 0 && utot) atomicAdd(&t[u], utot);
        __syncwarp();
    }
}

// ---- block bucket: d+(u) > 32 ----------------------------------------------------

struct CtaShared {
    int32_t Lu[CTA_LIST_MAX];
    uint32_t cnt[CTA_LIST_MAX];
    uint32_t bm[BITMAP_WORDS];
    uint16_t pre[BITMAP_WORDS];
    uint32_t slice[BITMAP_WORDS / 32];
    unsigned long long utot[CTA_WARPS];
    int q;
};

__global__ void __launch_bounds__(CTA_THREADS) k_tc_cta(const int64_t* __restrict__ rowstart,
                                                        const int32_t* __restrict__ rowlen,
                                                        const int32_t* __restrict__ col,
                                                        const int32_t* __restrict__ list,
                                                        unsigned long long* __restrict__ t,
                                                        DevStats* stats, int strategy, float factor) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaShared& sh = *reinterpret_cast<CtaShared*>(smem_raw);
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const unsigned count = stats->cta_count;
    for (;;) {
        if (threadIdx.x == 0) sh.q = (int)atomicAdd(&stats->work_next, 1u);
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
        const int32_t* Lu = staged ? sh.Lu : col + base;
        const int32_t maxu = col[base + du - 1];
        const int span = maxu - u;  // ranks u+1 .. maxu
        const bool bitmap = staged && strategy == TC_STRAT_BITMAP && span <= BITMAP_WORDS * 32;
        const int W = (span + 31) >> 5;
        if (bitmap) {
            for (int i = threadIdx.x; i < W; i += CTA_THREADS) sh.bm[i] = 0;
        }
        __syncthreads();
        if (bitmap) {
            for (int p = threadIdx.x; p < du; p += CTA_THREADS) {
                int off = sh.Lu[p] - u - 1;
                atomicOr(&sh.bm[off >> 5], 1u << (off & 31));
            }
            __syncthreads();
            // exclusive prefix of per-word popcounts: within 32-word slices (one warp
            // each), then over slice totals (warp 0), then the slice offsets are added
            const int slices = (W + 31) >> 5;
            for (int s = w; s < slices; s += CTA_WARPS) {
                const int i = s * 32 + lane;
                const int pc = i < W ? __popc(sh.bm[i]) : 0;
                const int inc = warp_inclusive_scan(pc);
                if (i < W) sh.pre[i] = (uint16_t)(inc - pc);
                if (lane == 31) sh.slice[s] = (uint32_t)inc;
            }
            __syncthreads();
            if (w == 0) {
                uint32_t carry = 0;
                for (int c0 = 0; c0 < slices; c0 += 32) {
                    const int i = c0 + lane;
                    const uint32_t v = i < slices ? sh.slice[i] : 0u;
                    const uint32_t inc = warp_inclusive_scan(v);
                    if (i < slices) sh.slice[i] = carry + inc - v;
                    carry += __shfl_sync(FULL, inc, 31);
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < W; i += CTA_THREADS) sh.pre[i] = (uint16_t)(sh.pre[i] + sh.slice[i >> 5]);
            __syncthreads();
        }
        Sink S{staged ? sh.cnt : nullptr, t, Lu};
        unsigned long long utot = 0;
        for (int j = w; j < du - 1; j += CTA_WARPS) {
            const int32_t v = Lu[j];
            const int dv = rowlen[v];
            if (dv == 0) continue;
            const int32_t* B = col + rowstart[v];
            uint32_t c;
            if (bitmap) {
                c = edge_bitmap(sh.bm, sh.pre, u, maxu, sh.cnt, B, dv);
            } else {
                int method = strategy == TC_STRAT_AUTO ? auto_method(du - j - 1, dv, factor)
                                                       : (strategy == TC_STRAT_BITMAP ? TC_STRAT_PROBE : strategy);
                c = edge_dispatch(method, S, j + 1, du, B, dv);
            }
            if (lane == 0 && c) {
                if (staged)
                    atomicAdd(&sh.cnt[j], c);
                else
                    atomicAdd(&t[v], (unsigned long long)c);
            }
            utot += c;
        }
        if (lane == 0) sh.utot[w] = utot;
        __syncthreads();
        if (staged) {
            for (int p = threadIdx.x; p < du; p += CTA_THREADS) {
                uint32_t cv = sh.cnt[p];
                if (cv) atomicAdd(&t[sh.Lu[p]], (unsigned long long)cv);
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
            lcc_out[v] = d < 2 ? 0.0 : __ddiv_rn((double)(2ull * tv), (double)(d * (d - 1)));
        }
    }
}

}  // namespace

void launch_plan(const CountBuffers& C, const Launch& L) {
    if (C.n <= 0) return;
    k_plan<<<grid_for(C.n, THREADS, L.sms), THREADS, 0, L.stream>>>(C.n, C.rowlen, C.warp_list, C.cta_list,
                                                                   C.stats);
}

size_t cta_smem_bytes() { return sizeof(CtaShared); }

cudaError_t intersect_init_attributes() {
    return cudaFuncSetAttribute(k_tc_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CtaShared));
}

void launch_intersect(const CountBuffers& C, const Strategy& S, cudaEvent_t ev[3], const Launch& L) {
    if (C.n <= 0) return;
    if (ev) cudaEventRecord(ev[0], L.stream);
    k_tc_warp<<<L.sms * 8, WK_WARPS * 32, 0, L.stream>>>(C.rowstart, C.rowlen, C.col, C.warp_list, C.t_rank,
                                                        C.stats, S.strat[TC_BUCKET_WARP],
                                                        S.factor[TC_BUCKET_WARP]);
    if (ev) cudaEventRecord(ev[1], L.stream);
    cudaMemsetAsync(&C.stats->work_next, 0, sizeof(unsigned), L.stream);
    k_tc_cta<<<L.sms * 4, CTA_THREADS, sizeof(CtaShared), L.stream>>>(C.rowstart, C.rowlen, C.col, C.cta_list,
                                                                     C.t_rank, C.stats, S.strat[TC_BUCKET_CTA],
                                                                     S.factor[TC_BUCKET_CTA]);
    if (ev) cudaEventRecord(ev[2], L.stream);
}

void launch_sum_t(const CountBuffers& C, const Launch& L) {
    if (C.n <= 0) return;
    k_sum_t<<<grid_for(C.n, THREADS, L.sms), THREADS, 0, L.stream>>>(C.n, C.t_rank, C.stats);
}

void launch_finalize(int32_t n, const int32_t* rank, const unsigned long long* t_rank, const int32_t* deg,
                     unsigned long long* t_out, double* lcc_out, const Launch& L) {
    if (n <= 0) return;
    k_finalize<<<grid_for(n, THREADS, L.sms), THREADS, 0, L.stream>>>(n, rank, t_rank, deg, t_out, lcc_out);
}

}  // namespace tcg
