// Dense core of the hub bucket: the core_n highest ranks (c0 = n - core_n .. n-1).
//
// Every out-neighbour of a core vertex has a higher rank, so it lies in the core too:
// a triangle whose lowest vertex is in the core lies wholly in the core.  On
// scale-free graphs the top ranks are densely linked, and their triangles make up a
// large part of the wedges the hub kernel would probe one by one (each in-edge
// (u -> v) reads the suffix of N+(u) after v, Sec. III / Eq. 1).  In the core the
// same counts come from bit-parallel intersections of rows of two bit matrices over
// core indices i = rank - c0:
//   Out[i] : bit j set iff j is in N+(i)   (bits above i only)
//   In[j]  : bit i set iff j is in N+(i)   (bits below j only)
// For a core edge (x -> y), x < y:
//   c1 = |Out[x] & Out[y]| = triangles x < y < w (x lowest, y middle),
//   c2 = |In[x] & In[y]|   = triangles u < x < y (y highest).
// A triangle a < b < c of the core is seen as c1 of edge (a, b) and as c2 of edge
// (b, c) and nowhere else, so t[x] += c1 and t[y] += c1 + c2 over all core edges
// gives every core triangle once at each of its vertices.  The hub in-edge lists then
// leave out the in-edges whose source lies in the core.
#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {
namespace {

constexpr int CORE_THREADS = 256;
constexpr int CORE_WARPS = CORE_THREADS / 32;
constexpr int CORE_LANE_WORDS = 8;  // bitmap words each lane holds: 32 * 8 * 32 bits = CORE_MAX
static_assert(32 * CORE_LANE_WORDS * 32 == CORE_MAX, "lane words cover the core");

// One warp per core vertex x: its row sets the bits of Out[x] and of the In rows of
// its targets; lo[j] = lowest core in-neighbour of j, hi[i] = highest out-neighbour
// of i (-1 for an empty row), cnt[j] = core in-degree of j.
__global__ void __launch_bounds__(CORE_THREADS) k_core_build(int32_t n, const int64_t* __restrict__ rowstart,
                                                             const int32_t* __restrict__ rowlen,
                                                             const int32_t* __restrict__ col, int words,
                                                             uint32_t* __restrict__ out, uint32_t* __restrict__ in,
                                                             int32_t* __restrict__ lo, int32_t* __restrict__ hi,
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
            atomicOr(&out[i * words + (j >> 5)], 1u << (j & 31));
            atomicOr(&in[(int64_t)j * words + (i >> 5)], 1u << (i & 31));
            atomicMin(&lo[j], (int32_t)i);
            atomicAdd(&cnt[j], 1u);
        }
        if (lane == 0) hi[i] = d > 0 ? col[base + d - 1] - c0 : -1;
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
// l holds words [8l, 8l + 8) of Out[x] and In[x] in registers and reads the same
// words of Out[y] and In[y], only where the bit ranges can overlap: Out bits lie in
// (y, min(hi[x], hi[y])], In bits in [max(lo[x], lo[y]), x).  Words outside those
// ranges are zero in one operand, so skipping them changes no count.
__global__ void __launch_bounds__(CORE_THREADS) k_core_count(int32_t n, const int64_t* __restrict__ rowstart,
                                                             const int32_t* __restrict__ rowlen,
                                                             const int32_t* __restrict__ col, int words,
                                                             const uint32_t* __restrict__ out,
                                                             const uint32_t* __restrict__ in,
                                                             const int32_t* __restrict__ lo,
                                                             const int32_t* __restrict__ hi,
                                                             unsigned long long* __restrict__ t, const DevStats* stats) {
    __shared__ unsigned long long tx_w[CORE_WARPS];
    const int core_n = (int)stats->core_n;
    const int32_t c0 = n - core_n;
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int first = lane * CORE_LANE_WORDS;
    for (int64_t i = blockIdx.x; i < core_n; i += gridDim.x) {
        const int32_t x = c0 + (int32_t)i;
        const int d = rowlen[x];
        if (d == 0) continue;  // uniform across the block
        const int64_t base = rowstart[x];
        uint32_t ox[CORE_LANE_WORDS], ix[CORE_LANE_WORDS];
#pragma unroll
        for (int h = 0; h < CORE_LANE_WORDS; h += 4) {
            uint4 a = make_uint4(0, 0, 0, 0), b = make_uint4(0, 0, 0, 0);
            if (first + h < words) {
                a = *reinterpret_cast<const uint4*>(out + i * words + first + h);
                b = *reinterpret_cast<const uint4*>(in + i * words + first + h);
            }
            ox[h] = a.x, ox[h + 1] = a.y, ox[h + 2] = a.z, ox[h + 3] = a.w;
            ix[h] = b.x, ix[h + 1] = b.y, ix[h + 2] = b.z, ix[h + 3] = b.w;
        }
        const int hix = hi[i], lox = lo[i];
        unsigned long long tx = 0;
        for (int p = w; p < d; p += CORE_WARPS) {
            const int j = col[base + p] - c0;
            const int ohi = min(hix, hi[j]);
            const int ilo = max(lox, lo[j]);
            uint32_t c1 = 0, c2 = 0;
            if (ohi > j && first < words) c1 = and_popc(out + (int64_t)j * words, ox, first, (j + 1) >> 5, ohi >> 5);
            if (ilo < (int)i && first < words) c2 = and_popc(in + (int64_t)j * words, ix, first, ilo >> 5, ((int)i - 1) >> 5);
            const uint32_t c12 = __reduce_add_sync(FULL, c1 + c2);
            tx += c1;
            if (lane == 0 && c12) atomicAdd(&t[x + (j - (int)i)], (unsigned long long)c12);  // t[y], y = c0 + j
        }
        tx = warp_sum(tx);
        if (lane == 0) tx_w[w] = tx;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long s = 0;
            for (int k = 0; k < CORE_WARPS; ++k) s += tx_w[k];
            if (s) atomicAdd(&t[x], s);
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
    // out, in and cnt are one zeroed block; lo starts above every core index
    cudaMemsetAsync(C.core_out, 0, sizeof(uint32_t) * (2 * rows + (size_t)C.core_cap), L.stream);
    cudaMemsetAsync(C.core_lo, 0x7f, sizeof(int32_t) * (size_t)C.core_cap, L.stream);
    k_core_build<<<grid_for((int64_t)C.core_cap * 32, CORE_THREADS, L.sms), CORE_THREADS, 0, L.stream>>>(
        C.n, C.rowstart, C.rowlen, C.col, C.core_words, C.core_out, C.core_in, C.core_lo, C.core_hi, C.core_cnt,
        C.stats);
    count_launch();
}

void launch_core_count(const CountBuffers& C, const Launch& L) {
    if (C.core_cap <= 0) return;
    k_core_count<<<C.core_cap, CORE_THREADS, 0, L.stream>>>(C.n, C.rowstart, C.rowlen, C.col, C.core_words,
                                                           C.core_out, C.core_in, C.core_lo, C.core_hi, C.t_rank,
                                                           C.stats);
    count_launch();
}

}  // namespace tcg
