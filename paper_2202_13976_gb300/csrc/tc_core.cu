// Dense core of the hub bucket: the core_n highest ranks (c0 = n - core_n .. n-1).
//
// Every out-neighbour of a core vertex has a higher rank, so it lies in the core too:
// a triangle whose lowest vertex is in the core lies wholly in the core.  On
// scale-free graphs the top ranks are densely linked, and their triangles make up a
// large part of the wedges the hub kernel would probe one by one (each in-edge
// (u -> v) reads the suffix of N+(u) after v, Sec. III / Eq. 1).  In the core the
// same counts come from bit-parallel intersections with the rows of one symmetric
// bit matrix over core indices i = rank - c0:
//   Z[i] : bit j set iff i and j are adjacent
// For a core edge (x -> y), x < y, let S(x, y) = |{w > x : x -> w, w adjacent to y}|,
// the popcount of (Z[x] above bit x) AND Z[y].  A triangle a < b < c of the core
// is seen in S(a, b) (w = c) and in S(a, c) (w = b) and in no other S, so
//   t[y] += S(x, y) for every core edge, and t[x] += (sum over y of S(x, y)) / 2
// gives every core triangle once at each of its vertices (b and c through their own
// edge from a, a through the two).  The hub in-edge lists then leave out the
// in-edges whose source lies in the core.
#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {
namespace {

constexpr int CORE_THREADS = 256;
constexpr int CORE_WARPS = CORE_THREADS / 32;
constexpr int CORE_LANE_WORDS = 8;  // bitmap words each lane holds: 32 * 8 * 32 bits = CORE_MAX
static_assert(32 * CORE_LANE_WORDS * 32 == CORE_MAX, "lane words cover the core");

// One warp per core vertex x: its row sets the bits of both ends in Z; lo and hi
// collect the lowest and highest neighbour of every core vertex, hiout[i] is the
// highest out-neighbour of i (-1 for an empty row), cnt[j] the core in-degree of j.
__global__ void __launch_bounds__(CORE_THREADS) k_core_build(int32_t n, const int64_t* __restrict__ rowstart,
                                                             const int32_t* __restrict__ rowlen,
                                                             const int32_t* __restrict__ col, int words,
                                                             uint32_t* __restrict__ z, int32_t* __restrict__ lo,
                                                             int32_t* __restrict__ hi, int32_t* __restrict__ hiout,
                                                             uint32_t* __restrict__ cnt, const DevStats* stats) {
    const int core_n = (int)stats->core_n;
    const int32_t c0 = n - core_n;
    const int lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * CORE_WARPS;
    for (int64_t i = (int64_t)blockIdx.x * CORE_WARPS + (threadIdx.x >> 5); i < core_n; i += warps) {
        const int32_t x = c0 + (int32_t)i;
        const int d = rowlen[x];
        const int64_t base = rowstart[x];
        for (int p = lane; p < d; p += 32) {
            const int j = col[base + p] - c0;  // > i: the row lies above x
            atomicOr(&z[i * words + (j >> 5)], 1u << (j & 31));
            atomicOr(&z[(int64_t)j * words + (i >> 5)], 1u << (i & 31));
            atomicMin(&lo[j], (int32_t)i);
            atomicMax(&hi[j], (int32_t)i);
            atomicAdd(&cnt[j], 1u);
        }
        if (d > 0 && lane == 0) {  // the row is sorted: its ends bound i's out-neighbours
            atomicMin(&lo[i], col[base] - c0);
            atomicMax(&hi[i], col[base + d - 1] - c0);
        }
        if (lane == 0) hiout[i] = d > 0 ? col[base + d - 1] - c0 : -1;
    }
}

// Sum of popc(a & b) over the lane's words that fall in [w0, w1] (word indices).
__device__ __forceinline__ uint32_t and_popc(const uint32_t* __restrict__ row, const uint32_t (&mine)[CORE_LANE_WORDS],
                                             int first, int w0, int w1) {
    uint32_t c = 0;
    if (w0 > w1) return 0;  // empty range
#pragma unroll
    for (int h = 0; h < CORE_LANE_WORDS / 4; ++h) {
        const int q = first + 4 * h;  // word index of this uint4
        if (q + 3 >= w0 && q <= w1) {
            const uint4 v = *reinterpret_cast<const uint4*>(row + q);
            c += __popc(v.x & mine[4 * h]) + __popc(v.y & mine[4 * h + 1]) + __popc(v.z & mine[4 * h + 2]) +
                 __popc(v.w & mine[4 * h + 3]);
        }
    }
    return c;
}

// One block per core vertex x; its warps take the entries y of N+(x) in turn.  Lane
// l holds words [8l, 8l + 8) of Z[x] with the bits at or below x cleared (that is,
// N+(x)) in registers and reads the same words of Z[y] where the bit ranges can
// overlap: (x, hiout[x]] against [lo[y], hi[y]].  Words outside that range are zero in
// one operand, so skipping them changes no count.
__global__ void __launch_bounds__(CORE_THREADS) k_core_count(int32_t n, const int64_t* __restrict__ rowstart,
                                                             const int32_t* __restrict__ rowlen,
                                                             const int32_t* __restrict__ col, int words,
                                                             const uint32_t* __restrict__ z,
                                                             const int32_t* __restrict__ lo,
                                                             const int32_t* __restrict__ hi,
                                                             const int32_t* __restrict__ hiout,
                                                             unsigned long long* __restrict__ t, int32_t src_lo,
                                                             int32_t src_hi, const DevStats* stats) {
    __shared__ unsigned long long tx_w[CORE_WARPS];
    const int core_n = (int)stats->core_n;
    const int32_t c0 = n - core_n;
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int first = lane * CORE_LANE_WORDS;
    for (int64_t i = blockIdx.x; i < core_n; i += gridDim.x) {
        const int32_t x = c0 + (int32_t)i;
        const int d = x >= src_lo && x < src_hi ? rowlen[x] : 0;  // sources outside the counted shard: none
        if (d < 2) continue;  // no triangle has x lowest; uniform across the block
        const int64_t base = rowstart[x];
        uint32_t ox[CORE_LANE_WORDS];
#pragma unroll
        for (int h = 0; h < CORE_LANE_WORDS; h += 4) {
            uint4 a = make_uint4(0, 0, 0, 0);
            if (first + h < words) a = *reinterpret_cast<const uint4*>(z + i * words + first + h);
            ox[h] = a.x, ox[h + 1] = a.y, ox[h + 2] = a.z, ox[h + 3] = a.w;
        }
#pragma unroll
        for (int h = 0; h < CORE_LANE_WORDS; ++h) {  // keep the bits above x
            const int b0 = (first + h) * 32;
            if (b0 + 31 <= (int)i)
                ox[h] = 0;
            else if (b0 <= (int)i)
                ox[h] &= (~0u << ((int)i - b0)) << 1;
        }
        const int xlo = (int)i + 1, xhi = hiout[i];
        unsigned long long tx = 0;
        for (int p = w; p < d; p += CORE_WARPS) {
            const int j = col[base + p] - c0;
            const int b0 = max(xlo, lo[j]), b1 = min(xhi, hi[j]);
            uint32_t s = 0;
            if (b0 <= b1 && first < words) s = and_popc(z + (int64_t)j * words, ox, first, b0 >> 5, b1 >> 5);
            tx += s;
            s = __reduce_add_sync(FULL, s);
            if (lane == 0 && s) atomicAdd(&t[c0 + j], (unsigned long long)s);
        }
        tx = warp_sum(tx);
        if (lane == 0) tx_w[w] = tx;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long s = 0;
            for (int k = 0; k < CORE_WARPS; ++k) s += tx_w[k];
            if (s) atomicAdd(&t[x], s / 2);  // every triangle with x lowest was seen twice
        }
        __syncthreads();
    }
}

}  // namespace

int core_words_for(int32_t core_cap) {
    int w = (core_cap + 31) / 32;
    return (w + 7) & ~7;  // rows start on 32-byte boundaries; lanes read uint4
}

void launch_core_plan(const CountBuffers& C, const Launch& L) {
    if (C.core_cap <= 0) return;
    const size_t rows = (size_t)C.core_cap * (size_t)C.core_words;
    // z and cnt are one zeroed block; lo starts above and hi below every core index
    cudaMemsetAsync(C.core_z, 0, sizeof(uint32_t) * (rows + (size_t)C.core_cap), L.stream);
    cudaMemsetAsync(C.core_lo, 0x7f, sizeof(int32_t) * (size_t)C.core_cap, L.stream);
    cudaMemsetAsync(C.core_hi, 0xff, sizeof(int32_t) * (size_t)C.core_cap, L.stream);
    k_core_build<<<grid_for((int64_t)C.core_cap * 32, CORE_THREADS, L.sms), CORE_THREADS, 0, L.stream>>>(
        C.n, C.rowstart, C.rowlen, C.col, C.core_words, C.core_z, C.core_lo, C.core_hi, C.core_hiout, C.core_cnt,
        C.stats);
    count_launch();
}

void launch_core_count(const CountBuffers& C, const Launch& L) {
    if (C.core_cap <= 0) return;
    k_core_count<<<C.core_cap, CORE_THREADS, 0, L.stream>>>(C.n, C.rowstart, C.rowlen, C.col, C.core_words, C.core_z,
                                                           C.core_lo, C.core_hi, C.core_hiout, C.t_rank, C.src_lo,
                                                           C.src_hi, C.stats);
    count_launch();
}

}  // namespace tcg
