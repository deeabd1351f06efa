// Batched counting: G independent graphs are counted as one disjoint union.
//
// Graph g's pairs use local ids in [0, n_g); in the union they become
// vbase[g] + id, with vbase the exclusive prefix sum of the n_g.  A disjoint union
// has no triangle across graphs, so the union's t(v) and LCC(v) are exactly the
// per-graph values and T_g is the sum of t over graph g's vertex range divided by 3.
// Counting the union with the single-graph kernels keeps every multiprocessor
// busy even when most graphs are tiny (the planner's persistent, dynamically
// scheduled bucket kernels take vertices of all graphs from one queue), instead of
// one short launch sequence per graph.
#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {

namespace {

// One block per graph (grid-stride): union ids; a pair with a local id outside
// [0, n_g) becomes a self-loop at vbase[g] (dropped later) and raises ERR_BAD_ID.
__global__ void k_batch_relabel(int32_t G, const int64_t* __restrict__ edge_off, const int32_t* __restrict__ vbase,
                                const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                int32_t* __restrict__ usrc, int32_t* __restrict__ udst, int* __restrict__ err) {
    for (int g = blockIdx.x; g < G; g += gridDim.x) {
        const int64_t e0 = edge_off[g], e1 = edge_off[g + 1];
        const int32_t b = vbase[g], ng = vbase[g + 1] - b;
        int bad = 0;
        for (int64_t k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
            int32_t u = src[k], v = dst[k];
            if ((uint32_t)u >= (uint32_t)ng || (uint32_t)v >= (uint32_t)ng) {
                bad = 1;
                u = 0;
                v = 0;
            }
            usrc[k] = b + u;
            udst[k] = b + v;
        }
        bad = __syncthreads_or(bad);
        if (threadIdx.x == 0 && bad) atomicOr(err, ERR_BAD_ID);
    }
}

// One block per graph (grid-stride): T_g = (sum of t over the graph's vertices) / 3.
__global__ void k_batch_T(int32_t G, const int32_t* __restrict__ vbase, const int32_t* __restrict__ rank,
                          const unsigned long long* __restrict__ t_rank, unsigned long long* __restrict__ T_out,
                          int* __restrict__ err) {
    __shared__ unsigned long long ws[32];
    for (int g = blockIdx.x; g < G; g += gridDim.x) {
        unsigned long long s = 0;
        for (int32_t v = vbase[g] + threadIdx.x; v < vbase[g + 1]; v += blockDim.x) s += t_rank[rank[v]];
        s = warp_sum(s);
        if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += ws[w];
            if (tot % 3 != 0) atomicOr(err, ERR_OVERFLOW);
            T_out[g] = tot / 3;
        }
        __syncthreads();
    }
}

// Status word of a whole batch call: id errors, failed per-graph sums, sum of t not
// a multiple of 3.
__global__ void k_run_status(const DevStats* stats, const int* batch_err, int* status) {
    int s = stats->err | *batch_err;
    if (stats->sum_t % 3 != 0) s |= ERR_OVERFLOW;
    *status = s;
}

}  // namespace

void launch_run_status(const DevStats* stats, const int* batch_err, int* status, const Launch& L) {
    k_run_status<<<1, 1, 0, L.stream>>>(stats, batch_err, status);
    count_launch();
}

void launch_batch_relabel(int32_t G, const int64_t* edge_off, const int32_t* vbase, const int32_t* src,
                          const int32_t* dst, int32_t* usrc, int32_t* udst, int* err, const Launch& L) {
    if (G <= 0) return;
    k_batch_relabel<<<grid_for((int64_t)G * 256, 256, L.sms, 16), 256, 0, L.stream>>>(G, edge_off, vbase, src, dst,
                                                                                     usrc, udst, err);
    count_launch();
}

void launch_batch_T(int32_t G, const int32_t* vbase, const int32_t* rank, const unsigned long long* t_rank,
                    unsigned long long* T_out, int* err, const Launch& L) {
    if (G <= 0) return;
    k_batch_T<<<grid_for((int64_t)G * 256, 256, L.sms, 16), 256, 0, L.stream>>>(G, vbase, rank, t_rank, T_out, err);
    count_launch();
}

}  // namespace tcg
