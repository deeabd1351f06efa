// Shards of the count for several GPUs, and the LCC from summed counts.
//
// Every triangle is counted once, from its lowest-ranked vertex u: the oriented
// edges (u, v) and the suffixes of N+(u) after them (Alg. 2 on the degree-oriented
// graph, Sec. III).  So the triangles split into disjoint shards by ranges of u, and
// the per-vertex counts of the shards sum to t(v).  A shard's range is cut where the
// prefix of a per-source cost crosses an equal share of the total; the cost of u is
// d+(u) (d+(u) + 1) / 2 + 1, the suffix entries its edges read plus one, which
// balances the work rather than the number of edges (the paper's 1D partition splits
// vertices evenly and reports the imbalance this causes, Sec. V).  The graph is
// read-only and replicated; one sum of t[] over the shards is the only exchange, and
// Eq. 2 then gives the LCC from the summed t[] and the degrees.
#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {
namespace {

constexpr int SH_THREADS = 256;

__global__ void k_shard_cost(int32_t n, const int32_t* __restrict__ rowlen, uint32_t* __restrict__ cost) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const uint64_t d = (uint64_t)rowlen[u];
        const uint64_t c = d * (d + 1) / 2 + 1;
        cost[u] = c > 0xffffffffull ? 0xffffffffu : (uint32_t)c;
    }
}

// First index i in [0, n] with prefix[i] >= target (prefix is strictly increasing
// over [0, n), every cost being at least 1; prefix[n] is the total).
__device__ int32_t first_at_least(const int64_t* __restrict__ prefix, int32_t n, int64_t target) {
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        const int32_t mid = lo + (hi - lo) / 2;
        if (prefix[mid] >= target)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// floor(total * s / N) without overflow: total = q N + r, so the product is
// q s N + r s with r s < N^2 <= 2^62.
__device__ int64_t share_of(int64_t total, int32_t s, int32_t N) {
    const int64_t q = total / N, r = total % N;
    return q * s + (r * s) / N;
}

// Shard s takes the sources u with share_of(total, s) <= prefix[u] < share_of(total, s + 1).
__global__ void k_shard_cut(int32_t n, const int64_t* __restrict__ prefix, int32_t shard, int32_t nshards,
                            int32_t* __restrict__ bounds) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int64_t total = prefix[n];
    bounds[0] = shard == 0 ? 0 : first_at_least(prefix, n, share_of(total, shard, nshards));
    bounds[1] = shard + 1 == nshards ? n : first_at_least(prefix, n, share_of(total, shard + 1, nshards));
}

// Eq. 2 per vertex id from summed counts: the same arithmetic as the count's own
// finalisation (one correctly rounded double division of exact integers).
__global__ void k_lcc_counts(int32_t n, const int32_t* __restrict__ rank, const int32_t* __restrict__ deg,
                             const unsigned long long* __restrict__ t, double* __restrict__ lcc_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const unsigned long long tv = t[v];
        const long long d = deg[rank[v]];
        lcc_out[v] = d < 2 || tv == 0 ? 0.0 : __ddiv_rn((double)(2ull * tv), (double)(d * (d - 1)));
    }
}

}  // namespace

void launch_shard_bounds(int32_t n, const int32_t* rowlen, uint32_t* cost, int64_t* prefix, void* tmp, int32_t shard,
                         int32_t nshards, int32_t* bounds, const Launch& L) {
    if (n > 0) {
        k_shard_cost<<<grid_for(n, SH_THREADS, L.sms), SH_THREADS, 0, L.stream>>>(n, rowlen, cost);
        count_launch();
    }
    scan_u32_to_i64(cost, prefix, n, tmp, L);
    k_shard_cut<<<1, 32, 0, L.stream>>>(n, prefix, shard, nshards, bounds);
    count_launch();
}

void launch_lcc_from_counts(int32_t n, const int32_t* rank, const int32_t* deg, const unsigned long long* t,
                            double* lcc_out, const Launch& L) {
    if (n <= 0) return;
    k_lcc_counts<<<grid_for(n, SH_THREADS, L.sms), SH_THREADS, 0, L.stream>>>(n, rank, deg, t, lcc_out);
    count_launch();
}

}  // namespace tcg
