// Directed local clustering coefficient (Eq. 1, Sec. II-C).
//
// For a directed simple graph (e_ij from v_i to v_j, Sec. II-A) with adj(v_i) the
// out-neighbours of v_i, Eq. 1 counts
//   c(i) = |{e_jk in E : v_j, v_k in adj(v_i)}|,   C(i) = c(i) / (deg+(i) (deg+(i) - 1)).
// Every pair counted in c(i) closes a triangle {i, j, k} of the undirected graph U
// that underlies G, so the count runs on U with the undirected path's orientation
// (every triangle met once, at the edge joining its two lowest ranks, Sec. II-C's
// offset).  Each edge of U carries two direction bits relative to rank order:
// bit 0 = lower -> higher exists in G, bit 1 = higher -> lower.  A triangle
// u < v < w (ranks) found at the oriented edge (u, v) adds to each corner x, with y
// and z the other two corners, the number of its ordered pairs:
//   [x -> y] [x -> z] ([y -> z] + [z -> y]).
//
// Phases (all on the device):
//  1. U itself by the undirected build (ids checked, loops and repeats dropped,
//     vertices ranked by (degree, id), oriented rows sorted; one synchronisation
//     reads its size); its rows are laid out without gaps as keys
//     (lower rank, higher rank, bits) and as col;
//  2. every input pair finds its oriented entry by binary search in its lower end's
//     row and sets the bit of its direction; the bits give dirf, the distinct
//     directed edges and the out-degrees;
//  3. in-edge lists of the hubs: a stable sort of the entries by target;
//  4. count, pull: vertices with many in-edges (hubs) stage N+(v) as a 2-bit map of
//     direction bits in shared memory, and every in-edge (u -> v) streams N+(u) after v
//     against it;
//     count, push: a thread per other oriented entry (u, v), highest ranks first: N+(u)
//     after v against N+(v), by a merge (Alg. 2) or a binary search of the shorter
//     list (Alg. 1), as Eq. 3 decides, the direction bits read at the matched positions;
//  5. c and C per input id, and the sum of c.
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <cstring>
#include <vector>

#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {
namespace {

constexpr int DG_THREADS = 256;
constexpr int DGH_WINDOW = 131072;   // ranks above a hub covered by its 2-bit map (32 KB)
constexpr int DGH_MIN_IN = 32;       // in-edges that make a vertex a hub
constexpr int DGH_BLOCKS = 5;        // resident hub blocks per SM (40.1 KB shared memory each)
constexpr int DGH_UNROLL = 8;        // suffix loads in flight per lane of the hub kernel
constexpr int DGH_TOP = 1024;        // highest ranks whose c the hub kernel sums in shared memory

struct DgStats {
    unsigned long long loops;       // self-loops dropped
    unsigned long long m_directed;  // distinct directed edges
    unsigned long long sum_c;       // sum over i of c(i)
    unsigned long long entries;     // list entries read by the count (timed calls)
    int err;                        // an id outside [0, n)
    int pad;
};

int key_bits(int32_t n) {
    int b = 1;
    while (b < 31 && ((int64_t)1 << b) < (int64_t)n) ++b;
    return b;
}

// Phase 1: the rows of U without gaps: col[k] and okeys[k] = (u << (b + 2)) |
// (v << 2) for the k-th entry, rowstart the exclusive scan of the row lengths.  One
// warp per row.
__global__ void k_dg_compact(int32_t n, const int2* __restrict__ rowinfo, const int32_t* __restrict__ ucol,
                             const int64_t* __restrict__ rowstart, int b, int32_t* __restrict__ col,
                             uint64_t* __restrict__ okeys) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int2 ri = rowinfo[u];
        const int64_t d0 = rowstart[u];
        const uint64_t hi = (uint64_t)u << (b + 2);
        for (int i = lane; i < ri.y; i += 32) {
            const int32_t x = ucol[(int64_t)ri.x + i];
            col[d0 + i] = x;
            okeys[d0 + i] = hi | ((uint64_t)(uint32_t)x << 2);
        }
    }
}

// Phase 2a: every non-loop pair a -> c sets its direction bit at the entry of
// {a, c}: bit 0 when a has the lower rank, bit 1 otherwise.  The ids were checked by
// the build; the entry exists because the build kept one entry per distinct pair.
__global__ void k_dg_bits(int64_t m, const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                          const int32_t* __restrict__ rank, const int64_t* __restrict__ rowstart,
                          const int32_t* __restrict__ col, unsigned long long* __restrict__ okeys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += stride) {
        const int32_t a = src[k], c = dst[k];
        if (a == c) continue;
        const int32_t ra = rank[a], rc = rank[c];
        const int32_t lo = min(ra, rc), hi = max(ra, rc);
        const int64_t s0 = rowstart[lo];
        const int len = (int)(rowstart[lo + 1] - s0);
        const int p = lower_bound(col + s0, 0, len, hi);
        if (p < len && col[s0 + p] == hi) atomicOr(&okeys[s0 + p], ra < rc ? 1ull : 2ull);
    }
}

// Phase 1-2 with carried bits: the entries of a row are (rank << 2) | bit, sorted,
// exact repeats dropped, so a pair read in both directions left (v, 1) and (v, 2)
// next to each other.  A row keeps one entry per v, whose bits are the OR of the two.
// One warp per row; merge_count gives the merged lengths, merge_write the rows
// without gaps (col, dirf and the keys (u << (b + 2)) | (v << 2) | bits), the
// distinct directed edges and the out-degrees by id.
__global__ void k_dg_merge_count(int32_t n, const int2* __restrict__ rowinfo, const int32_t* __restrict__ ucol,
                                 uint32_t* __restrict__ merged) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int2 ri = rowinfo[u];
        uint32_t kept = 0;
        for (int i0 = 0; i0 < ri.y; i0 += 32) {  // ri.y is the same in every lane
            const int i = i0 + lane;
            bool keep = false;
            if (i < ri.y) {
                const int64_t p = (int64_t)ri.x + i;
                keep = i == 0 || (ucol[p - 1] >> 2) != (ucol[p] >> 2);
            }
            kept += __popc(__ballot_sync(FULL, keep));
        }
        if (lane == 0) merged[u] = kept;
    }
}

__global__ void k_dg_merge_write(int32_t n, const int2* __restrict__ rowinfo, const int32_t* __restrict__ ucol,
                                 const int64_t* __restrict__ rowstart, int b, const int32_t* __restrict__ idof,
                                 int32_t* __restrict__ col, uint8_t* __restrict__ dirf, uint64_t* __restrict__ okeys,
                                 uint32_t* __restrict__ dout, DgStats* st) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long distinct = 0;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int2 ri = rowinfo[u];
        int64_t d = rowstart[u];
        const uint64_t hi = (uint64_t)u << (b + 2);
        uint32_t out_u = 0;  // entries with bit 0: u -> v, tail u
        for (int i0 = 0; i0 < ri.y; i0 += 32) {
            const int i = i0 + lane;
            bool keep = false;
            int32_t v = 0;
            uint32_t f = 0;
            if (i < ri.y) {
                const int64_t p = (int64_t)ri.x + i;
                const int32_t x = ucol[p];
                v = x >> 2;
                keep = i == 0 || (ucol[p - 1] >> 2) != v;
                if (keep) {
                    f = (uint32_t)(x & 3);
                    if (i + 1 < ri.y) {
                        const int32_t y = ucol[p + 1];
                        if ((y >> 2) == v) f |= (uint32_t)(y & 3);
                    }
                }
            }
            const unsigned km = __ballot_sync(FULL, keep);
            if (keep) {
                const int64_t q = d + __popc(km & lanemask_lt());
                col[q] = v;
                dirf[q] = (uint8_t)f;
                okeys[q] = hi | ((uint64_t)(uint32_t)v << 2) | f;
                distinct += __popc(f);
                if (f & 1u) ++out_u;
                if (f & 2u) atomicAdd(&dout[idof[v]], 1u);  // v -> u, tail v
            }
            d += __popc(km);
        }
        out_u = __reduce_add_sync(FULL, out_u);
        if (lane == 0 && out_u) atomicAdd(&dout[idof[u]], out_u);
    }
    distinct = warp_sum(distinct);
    if (lane == 0 && distinct) atomicAdd(&st->m_directed, distinct);
}

// idof[rank[v]] = v.
__global__ void k_dg_idof(int32_t n, const int32_t* __restrict__ rank, int32_t* __restrict__ idof) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) idof[rank[v]] = (int32_t)v;
}

// Phase 2b: dirf[k] = the bits of entry k; each bit is one distinct directed edge,
// counted with its tail's out-degree (by id; the lower ends aggregated per warp: the
// entries are sorted by their lower end).
__global__ void k_dg_flags(int64_t mu, const uint64_t* __restrict__ okeys, int b, const int32_t* __restrict__ idof,
                           uint8_t* __restrict__ dirf, uint32_t* __restrict__ dout, DgStats* st) {
    const int lane = lane_id();
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t mask = (1ull << b) - 1;
    unsigned long long distinct = 0;
    for (int64_t base = warp0 * 32; base < mu; base += wstride * 32) {  // uniform per warp
        const int64_t e = base + lane;
        int32_t lo_tail = -1;
        if (e < mu) {
            const uint64_t key = okeys[e];
            const uint32_t f = (uint32_t)(key & 3);
            dirf[e] = (uint8_t)f;
            distinct += __popc(f);
            if (f & 1u) lo_tail = idof[key >> (b + 2)];
            if (f & 2u) atomicAdd(&dout[idof[(key >> 2) & mask]], 1u);
        }
        const unsigned same = __match_any_sync(FULL, lo_tail);
        if (lo_tail >= 0 && lane == __ffs(same) - 1) atomicAdd(&dout[lo_tail], (unsigned)__popc(same));
    }
    distinct = warp_sum(distinct);
    if (lane == 0 && distinct) atomicAdd(&st->m_directed, distinct);
}

// One matched corner w of the triangle (u, v, w): fa = bits of (u, w), fb = bits of
// (v, w), fuv = bits of (u, v), all in rank order (u < v < w).
struct DgAcc {
    uint32_t uv, vu, pop_uv;
    unsigned long long cu, cv;
    __device__ __forceinline__ void match(uint32_t fa, uint32_t fb, int32_t w, unsigned long long* __restrict__ c) {
        if (uv & fa & 1u) cu += __popc(fb);                   // [u->v][u->w]([v->w] + [w->v])
        if (vu & fb & 1u) cv += __popc(fa);                   // [v->u][v->w]([u->w] + [w->u])
        if ((fa >> 1) & (fb >> 1)) atomicAdd(&c[w], (unsigned long long)pop_uv);  // [w->u][w->v]([u->v] + [v->u])
    }
};

// Phase 4, pull: the in-edges (u -> v) of a vertex v, in rank order; ikey = (v << 31) | k
// for the entry k of (u, v) in col, so that a stable sort of the v field lists every
// vertex's in-edges together, in entry order.
__global__ void k_dg_in_keys(int64_t mu, const int32_t* __restrict__ col, uint64_t* __restrict__ ikeys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < mu; k += stride)
        ikeys[k] = ((uint64_t)(uint32_t)col[k] << 31) | (uint64_t)k;
}

// instart[a] = first sorted in-key whose target is >= a (a = 0 .. n).
__global__ void k_dg_instart(int32_t n, int64_t mu, const uint64_t* __restrict__ ikeys,
                             int64_t* __restrict__ instart) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a <= n; a += stride) {
        int64_t lo = 0, hi = mu;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)(ikeys[mid] >> 31) < a)
                lo = mid + 1;
            else
                hi = mid;
        }
        instart[a] = lo;
    }
}

// Hubs: at least DGH_MIN_IN in-edges, a non-empty N+(v) and a rank window
// (v, max N+(v)] that the shared 2-bit map covers.  hubflag is indexed by q = n-1-v so
// that the scanned list runs from the highest rank down.
__global__ void k_dg_hub_flags(int32_t n, const int64_t* __restrict__ rowstart, const int32_t* __restrict__ col,
                               const int64_t* __restrict__ instart, uint32_t* __restrict__ hubflag,
                               uint8_t* __restrict__ ishub) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t r0 = rowstart[v], r1 = rowstart[v + 1];
        const bool hub = instart[v + 1] - instart[v] >= DGH_MIN_IN && r1 > r0 && col[r1 - 1] - v <= DGH_WINDOW;
        ishub[v] = hub ? 1 : 0;
        hubflag[n - 1 - v] = hub ? 1u : 0u;
    }
}

__global__ void k_dg_hub_list(int32_t n, const uint32_t* __restrict__ hubflag, const uint32_t* __restrict__ hubpos,
                              int32_t* __restrict__ hubs) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride)
        if (hubflag[q]) hubs[hubpos[q]] = n - 1 - (int32_t)q;
}

// In-edge records of the hubs: rec[i] = {u, first entry after v in N+(u), end of
// N+(u), bits of (u, v)} for the sorted in-key i of (u -> v).
__global__ void k_dg_in_rec(int64_t mu, const uint64_t* __restrict__ ikeys, const uint64_t* __restrict__ okeys, int b,
                            const int64_t* __restrict__ rowstart, const uint8_t* __restrict__ ishub,
                            int4* __restrict__ rec) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t kmask = (1ull << 31) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < mu; i += stride) {
        const uint64_t ik = ikeys[i];
        if (!ishub[ik >> 31]) continue;
        const int64_t k = (int64_t)(ik & kmask);
        const uint64_t key = okeys[k];
        const int32_t u = (int32_t)(key >> (b + 2));
        rec[i] = make_int4(u, (int)(k + 1), (int)rowstart[u + 1], (int)(key & 3));
    }
}

// One block per hub v (claimed from the list, highest rank first).  N+(v) is staged as
// a 2-bit map over the window (v, max N+(v)]: position w - v - 1 holds the direction
// bits of (v, w), 0 when w is not an out-neighbour.  Groups of 8 lanes take the
// in-edges (u -> v); each streams N+(u) after v (stopping above max N+(v)) and probes
// the map: a non-zero code fb is a triangle u < v < w with fa = bits of (u, w) read
// beside w, fuv = bits of (u, v).  The map is cleared once per block; each hub resets
// only the words its own entries set, so a hub costs O(|N+(v)|) on top of its in-edges'
// suffixes, not O(window).  Matches that add to one of the DGH_TOP highest ranks (the
// vertices most in-edges lead to) are summed in shared memory and flushed once per
// block; the others add to c[] directly.
__global__ void __launch_bounds__(DG_THREADS, DGH_BLOCKS) k_dg_hub(int32_t n, const uint32_t* __restrict__ nh_ptr,
                                                       const int32_t* __restrict__ hubs,
                                                       const int64_t* __restrict__ rowstart,
                                                       const int32_t* __restrict__ col,
                                                       const uint8_t* __restrict__ dirf,
                                                       const int4* __restrict__ rec,
                                                       const int64_t* __restrict__ instart,
                                                       unsigned long long* __restrict__ c,
                                                       unsigned* __restrict__ counter) {
    __shared__ uint32_t map[DGH_WINDOW / 16];
    __shared__ unsigned long long top[DGH_TOP];  // c of ranks n - DGH_TOP .. n - 1, this block's share
    __shared__ unsigned long long cv_w[DG_THREADS / 32];
    __shared__ unsigned next;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const int grp = lane >> 3, gl = lane & 7;
    const unsigned nh = *nh_ptr;
    const int32_t top0 = n - DGH_TOP;
    for (int i = threadIdx.x; i < DGH_WINDOW / 16; i += DG_THREADS) map[i] = 0;  // once; each hub clears its own
    for (int i = threadIdx.x; i < DGH_TOP; i += DG_THREADS) top[i] = 0;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1u);
        __syncthreads();  // the previous hub is finished and cleared by every thread
        const unsigned q = next;
        if (q >= nh) break;
        const int32_t v = hubs[q];
        const int64_t s0 = rowstart[v];
        const int dv = (int)(rowstart[v + 1] - s0);
        const int32_t hi = col[s0 + dv - 1];  // dv > 0 for every hub
        for (int j = threadIdx.x; j < dv; j += DG_THREADS) {
            const int off = col[s0 + j] - v - 1;
            atomicOr(&map[off >> 4], (uint32_t)dirf[s0 + j] << (2 * (off & 15)));
        }
        __syncthreads();
        unsigned long long cv = 0;
        const int64_t i0 = instart[v], i1 = instart[v + 1];
        for (int64_t base = i0 + (int64_t)warp * 4; base < i1; base += DG_THREADS / 8) {  // uniform per warp
            const int64_t i = base + grp;
            unsigned long long cu = 0;
            int4 r = make_int4(-1, 0, 0, 0);
            if (i < i1) r = rec[i];
            const uint32_t fuv = (uint32_t)r.w;
            // the group's lanes take positions sb + gl + 8 j, DGH_UNROLL loads in flight
            for (int p0 = r.y + gl; p0 < r.z; p0 += 8 * DGH_UNROLL) {
                int32_t w[DGH_UNROLL];
                uint32_t fa[DGH_UNROLL];
#pragma unroll
                for (int j = 0; j < DGH_UNROLL; ++j) {
                    const int p = p0 + 8 * j;
                    w[j] = p < r.z ? col[p] : INT_MAX;
                    fa[j] = p < r.z ? dirf[p] : 0u;
                }
#pragma unroll
                for (int j = 0; j < DGH_UNROLL; ++j) {
                    if (w[j] > hi) break;  // the row is sorted: nothing further lies in the window
                    const int off = w[j] - v - 1;
                    const uint32_t fb = (map[off >> 4] >> (2 * (off & 15))) & 3u;
                    if (fb) {
                        if (fuv & fa[j] & 1u) cu += __popc(fb);         // [u->v][u->w]([v->w] + [w->v])
                        if ((fuv >> 1) & fb & 1u) cv += __popc(fa[j]);  // [v->u][v->w]([u->w] + [w->u])
                        if ((fa[j] >> 1) & (fb >> 1)) {                 // [w->u][w->v]([u->v] + [v->u])
                            const unsigned long long x = (unsigned long long)__popc(fuv);
                            if (w[j] >= top0)
                                atomicAdd(&top[w[j] - top0], x);
                            else
                                atomicAdd(&c[w[j]], x);
                        }
                    }
                }
                if (w[DGH_UNROLL - 1] > hi) break;
            }
            cu += __shfl_xor_sync(FULL, cu, 1);
            cu += __shfl_xor_sync(FULL, cu, 2);
            cu += __shfl_xor_sync(FULL, cu, 4);
            if (gl == 0 && cu) atomicAdd(&c[r.x], cu);
        }
        cv = warp_sum(cv);
        if (lane == 0) cv_w[warp] = cv;
        __syncthreads();  // every probe of this hub is done
        if (threadIdx.x == 0) {
            unsigned long long sv = 0;
            for (int k = 0; k < DG_THREADS / 32; ++k) sv += cv_w[k];
            if (sv) atomicAdd(&c[v], sv);
        }
        for (int j = threadIdx.x; j < dv; j += DG_THREADS) map[(col[s0 + j] - v - 1) >> 4] = 0;
    }
    for (int i = threadIdx.x; i < DGH_TOP; i += DG_THREADS)  // after the final barrier of the loop
        if (top0 + i >= 0 && top[i]) atomicAdd(&c[top0 + i], top[i]);
}

// Phase 4, push: a thread per oriented entry whose target is not a hub, from the last
// (highest ranks) down.
__global__ void __launch_bounds__(DG_THREADS) k_dg_count(int64_t mu, const uint64_t* __restrict__ okeys, int b,
                                                         const int64_t* __restrict__ rowstart,
                                                         const int32_t* __restrict__ col,
                                                         const uint8_t* __restrict__ dirf,
                                                         const uint8_t* __restrict__ ishub,
                                                         unsigned long long* __restrict__ c) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t mask = (1ull << b) - 1;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < mu; q += stride) {
        const int64_t k = mu - 1 - q;
        const uint64_t key = okeys[k];
        const int32_t u = (int32_t)(key >> (b + 2)), v = (int32_t)((key >> 2) & mask);
        if (ishub[v]) continue;  // pulled by k_dg_hub
        DgAcc acc;
        const uint32_t fuv = (uint32_t)(key & 3);
        acc.uv = fuv & 1u;
        acc.vu = fuv >> 1;
        acc.pop_uv = __popc(fuv);
        acc.cu = 0;
        acc.cv = 0;
        const int64_t r1 = rowstart[u + 1];
        const int32_t* A = col + k + 1;
        const uint8_t* FA = dirf + k + 1;
        const int a = (int)(r1 - k - 1);
        const int64_t s0 = rowstart[v];
        const int32_t* B = col + s0;
        const uint8_t* FB = dirf + s0;
        const int bl = (int)(rowstart[v + 1] - s0);
        if (a > 0 && bl > 0) {
            const int s = min(a, bl), l = max(a, bl);
            if (l <= 16 || (float)l <= (log2f((float)l) - 1.0f) * (float)s) {  // Eq. 3: merge
                int i = 0, j = 0;
                while (i < a && j < bl) {
                    const int32_t x = A[i], y = B[j];
                    if (x == y) acc.match(FA[i], FB[j], x, c);
                    i += x <= y;
                    j += y <= x;
                }
            } else if (a <= bl) {  // keys from the suffix of N+(u), looked up in N+(v)
                int lo = 0;
                for (int i = 0; i < a && lo < bl; ++i) {
                    const int32_t x = A[i];
                    lo = lower_bound(B, lo, bl, x);
                    if (lo < bl && B[lo] == x) acc.match(FA[i], FB[lo], x, c);
                }
            } else {  // keys from N+(v), looked up in the suffix of N+(u)
                int lo = 0;
                for (int j = 0; j < bl && lo < a; ++j) {
                    const int32_t y = B[j];
                    lo = lower_bound(A, lo, a, y);
                    if (lo < a && A[lo] == y) acc.match(FA[lo], FB[j], y, c);
                }
            }
        }
        if (acc.cu) atomicAdd(&c[u], acc.cu);
        if (acc.cv) atomicAdd(&c[v], acc.cv);
    }
}

// Sum over oriented entries (u, v) of d+(u) + d+(v): the list entries the count reads.
__global__ void k_dg_list_entries(int64_t mu, const uint64_t* __restrict__ okeys, int b,
                                  const int64_t* __restrict__ rowstart, DgStats* st) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t mask = (1ull << b) - 1;
    unsigned long long s = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < mu; k += stride) {
        const uint64_t key = okeys[k];
        const int64_t u = (int64_t)(key >> (b + 2)), v = (int64_t)((key >> 2) & mask);
        s += (unsigned long long)(rowstart[u + 1] - rowstart[u] + rowstart[v + 1] - rowstart[v]);
    }
    s = warp_sum(s);
    if (lane_id() == 0 && s) atomicAdd(&st->entries, s);
}

// Phase 5: outputs in input ids and the sum of c.
__global__ void k_dg_finalize(int32_t n, const int32_t* __restrict__ rank, const unsigned long long* __restrict__ c_rank,
                              const uint32_t* __restrict__ dout, unsigned long long* __restrict__ c_out,
                              double* __restrict__ lcc_out, DgStats* st) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long sum = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const unsigned long long cv = c_rank[rank[v]];
        sum += cv;
        if (c_out) c_out[v] = cv;
        if (lcc_out) {
            const long long d = dout[v];
            lcc_out[v] = d < 2 || cv == 0 ? 0.0 : __ddiv_rn((double)cv, (double)(d * (d - 1)));
        }
    }
    sum = warp_sum(sum);
    if (lane_id() == 0 && sum) atomicAdd(&st->sum_c, sum);
}

// Pool allocations of one call, released (stream-ordered) when it ends.
struct Arena {
    cudaMemPool_t pool;
    cudaStream_t stream;
    std::vector<void*> list;
    bool failed = false;
    template <typename T>
    T* get(size_t count) {
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        bytes = (bytes + 255) & ~(size_t)255;
        void* p = nullptr;
        if (failed) return nullptr;
        if (cudaMallocFromPoolAsync(&p, bytes, pool, stream) != cudaSuccess) {
            cudaGetLastError();
            failed = true;
            return nullptr;
        }
        list.push_back(p);
        return static_cast<T*>(p);
    }
    ~Arena() {
        for (void* p : list) cudaFreeAsync(p, stream);
    }
};

// CUDA events around the phases of a timed call (none otherwise).
struct Events {
    cudaEvent_t e[4] = {};
    bool on = false, ok = true;
    explicit Events(bool timed) : on(timed) {
        for (int k = 0; on && k < 4; ++k)
            if (cudaEventCreate(&e[k]) != cudaSuccess) {
                cudaGetLastError();
                ok = false;
                on = false;
            }
    }
    void record(int k, cudaStream_t s) {
        if (on) cudaEventRecord(e[k], s);
    }
    float ms(int a, int b) const {
        float t = 0.0f;
        if (on && cudaEventElapsedTime(&t, e[a], e[b]) != cudaSuccess) {
            cudaGetLastError();
            t = 0.0f;
        }
        return t;
    }
    ~Events() {
        for (int k = 0; k < 4; ++k)
            if (e[k]) cudaEventDestroy(e[k]);
    }
};

tc_status fail(const char* where, cudaError_t e) {
    set_last_error(where, e);
    return TC_ECUDA;
}

}  // namespace
}  // namespace tcg

using namespace tcg;

extern "C" tc_status tc_directed_lcc(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, int mem_kind,
                                     void* cuda_stream, uint64_t* c_out, double* lcc_out, tc_directed_stats* stats,
                                     int flags) {
    if (n < 0 || m < 0 || m > INT32_MAX || (m > 0 && (!src || !dst)) ||
        (mem_kind != TC_MEM_HOST && mem_kind != TC_MEM_DEVICE) || (flags & ~TC_DIRECTED_TIMED))
        return TC_EINVAL;
    const bool timed = (flags & TC_DIRECTED_TIMED) != 0;
    const bool host = mem_kind == TC_MEM_HOST;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail("tc_directed_lcc: device", e);
    cudaMemPool_t pool = device_pool(dev);
    if (!pool) return TC_ECUDA;
    const Launch L{stream, sms};
    const size_t nn = (size_t)n, mm = (size_t)m;
    Arena A{pool, stream};

    if (m == 0) {  // no edge: every count and coefficient is zero
        if (host) {
            if (c_out) memset(c_out, 0, sizeof(uint64_t) * nn);
            if (lcc_out) memset(lcc_out, 0, sizeof(double) * nn);
        } else {
            if (c_out && nn) e = cudaMemsetAsync(c_out, 0, sizeof(uint64_t) * nn, stream);
            if (e == cudaSuccess && lcc_out && nn) e = cudaMemsetAsync(lcc_out, 0, sizeof(double) * nn, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) return fail("tc_directed_lcc", e);
        }
        if (stats) *stats = tc_directed_stats{};
        return TC_OK;
    }

    const int b = key_bits(n);
    const int32_t* dsrc = src;
    const int32_t* ddst = dst;
    if (host) {
        int32_t* s = A.get<int32_t>(mm);
        int32_t* d = A.get<int32_t>(mm);
        if (A.failed) return TC_ENOMEM;
        e = cudaMemcpyAsync(s, src, sizeof(int32_t) * mm, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d, dst, sizeof(int32_t) * mm, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return fail("tc_directed_lcc: copy in", e);
        dsrc = s;
        ddst = d;
    }
    Events ev(timed);
    if (!ev.ok) return fail("tc_directed_lcc: events", cudaErrorMemoryAllocation);
    ev.record(0, stream);
    // phase 1: U by the undirected build (its graph object is released with the call);
    // up to 2^29 vertices its entries carry the direction bits of their pairs
    const bool carried = n <= (1 << 29);
    tc_graph* ug = nullptr;
    UndirectedRows U{};
    tc_status ust = build_undirected_rows(n, m, dsrc, ddst, stream, carried, &ug, &U);
    struct GraphHold {
        tc_graph* g;
        ~GraphHold() {
            if (g) tc_graph_destroy(g);
        }
    } hold{ug};
    if (ust != TC_OK) return ust;
    const unsigned long long loops = (unsigned long long)U.loops;
    const int32_t* rank = U.rank;
    void* scan_tmp = A.get<char>(scan_tmp_bytes((int64_t)nn + 1));
    uint32_t* dout = A.get<uint32_t>(nn);
    int32_t* idof = A.get<int32_t>(nn);
    DgStats* st = A.get<DgStats>(1);
    int64_t* rowstart = A.get<int64_t>(nn + 1);
    uint32_t* merged = carried ? A.get<uint32_t>(nn) : nullptr;
    if (A.failed) return TC_ENOMEM;
    int64_t mu = U.m_simple;
    if (carried) {
        // a pair read in both directions left two neighbouring entries: rows merged
        k_dg_merge_count<<<grid_for((int64_t)n * 32, DG_THREADS, sms), DG_THREADS, 0, stream>>>(n, U.rowinfo, U.col,
                                                                                              merged);
        count_launch();
        scan_u32_to_i64(merged, rowstart, n, scan_tmp, L);
        e = cudaMemcpyAsync(&mu, rowstart + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return fail("tc_directed_lcc: merged rows", e);
    } else {
        scan_u32_to_i64(reinterpret_cast<const uint32_t*>(U.rowlen), rowstart, n, scan_tmp, L);
    }
    const int64_t big = mu > (int64_t)n + 1 ? mu : (int64_t)n + 1;
    void* radix_tmp = A.get<char>(radix_tmp_bytes(big));
    uint64_t* keys = A.get<uint64_t>((size_t)mu);
    uint64_t* alt = A.get<uint64_t>((size_t)mu);
    int32_t* col = A.get<int32_t>((size_t)mu);
    uint8_t* dirf = A.get<uint8_t>((size_t)mu);
    unsigned long long* c_rank = A.get<unsigned long long>(nn);
    unsigned long long* dc = nullptr;
    double* dl = nullptr;
    if (host && c_out) dc = A.get<unsigned long long>(nn);
    if (host && lcc_out) dl = A.get<double>(nn);
    if (A.failed) return TC_ENOMEM;
    DgStats hst_v{};
    DgStats* hst = &hst_v;  // the host copy is read only after the stream is synchronised
    cudaMemsetAsync(st, 0, sizeof(DgStats), stream);
    cudaMemsetAsync(dout, 0, sizeof(uint32_t) * nn, stream);
    k_dg_idof<<<grid_for(n, DG_THREADS, sms), DG_THREADS, 0, stream>>>(n, rank, idof);
    count_launch();
    if (carried) {
        // phase 2 from the carried bits: merged rows, keys, dirf, out-degrees
        k_dg_merge_write<<<grid_for((int64_t)n * 32, DG_THREADS, sms), DG_THREADS, 0, stream>>>(
            n, U.rowinfo, U.col, rowstart, b, idof, col, dirf, keys, dout, st);
        count_launch();
    } else {
        k_dg_compact<<<grid_for((int64_t)n * 32, DG_THREADS, sms), DG_THREADS, 0, stream>>>(n, U.rowinfo, U.col,
                                                                                          rowstart, b, col, keys);
        count_launch();
        // phase 2: direction bits by a binary search per pair
        k_dg_bits<<<grid_for(m, DG_THREADS, sms), DG_THREADS, 0, stream>>>(m, dsrc, ddst, rank, rowstart, col,
                                                                            reinterpret_cast<unsigned long long*>(keys));
        count_launch();
        k_dg_flags<<<grid_for(mu, DG_THREADS, sms), DG_THREADS, 0, stream>>>(mu, keys, b, idof, dirf, dout, st);
        count_launch();
    }
    uint64_t* osorted = keys;  // the rows are laid out in (lower, higher) order already
    // in-edge lists and hubs (the phase-1 buffer that does not hold osorted is free)
    uint64_t* ikeys = osorted == keys ? alt : keys;
    uint64_t* ialt = A.get<uint64_t>((size_t)mu);
    int64_t* instart = A.get<int64_t>(nn + 1);
    uint32_t* hubflag = A.get<uint32_t>(nn + 1);
    uint32_t* hubpos = A.get<uint32_t>(nn + 1);
    int32_t* hubs = A.get<int32_t>(nn);
    uint8_t* ishub = A.get<uint8_t>(nn);
    unsigned* counter = A.get<unsigned>(1);
    int4* rec = A.get<int4>((size_t)mu);
    if (A.failed) return TC_ENOMEM;
    k_dg_in_keys<<<grid_for(mu, DG_THREADS, sms), DG_THREADS, 0, stream>>>(mu, col, ikeys);
    count_launch();
    uint64_t* isorted = radix_sort_u64(ikeys, ialt, mu, 31, 31 + b, radix_tmp, L);
    k_dg_instart<<<grid_for((int64_t)n + 1, DG_THREADS, sms), DG_THREADS, 0, stream>>>(n, mu, isorted, instart);
    count_launch();
    k_dg_hub_flags<<<grid_for(n, DG_THREADS, sms), DG_THREADS, 0, stream>>>(n, rowstart, col, instart, hubflag,
                                                                             ishub);
    count_launch();
    scan_u32_to_u32(hubflag, hubpos, n, scan_tmp, L);
    k_dg_hub_list<<<grid_for(n, DG_THREADS, sms), DG_THREADS, 0, stream>>>(n, hubflag, hubpos, hubs);
    count_launch();
    k_dg_in_rec<<<grid_for(mu, DG_THREADS, sms), DG_THREADS, 0, stream>>>(mu, isorted, osorted, b, rowstart, ishub,
                                                                           rec);
    count_launch();
    // phase 4: count
    cudaMemsetAsync(c_rank, 0, sizeof(unsigned long long) * nn, stream);
    cudaMemsetAsync(counter, 0, sizeof(unsigned), stream);
    if (timed) {
        k_dg_list_entries<<<grid_for(mu, DG_THREADS, sms), DG_THREADS, 0, stream>>>(mu, osorted, b, rowstart, st);
        count_launch();
    }
    ev.record(1, stream);
    k_dg_hub<<<sms * DGH_BLOCKS, DG_THREADS, 0, stream>>>(n, hubpos + n, hubs, rowstart, col, dirf, rec, instart,
                                                          c_rank, counter);
    count_launch();
    k_dg_count<<<grid_for(mu, DG_THREADS, sms), DG_THREADS, 0, stream>>>(mu, osorted, b, rowstart, col, dirf, ishub,
                                                                          c_rank);
    count_launch();
    ev.record(2, stream);
    // phase 5
    k_dg_finalize<<<grid_for(n, DG_THREADS, sms), DG_THREADS, 0, stream>>>(
        n, rank, c_rank, dout, host ? dc : reinterpret_cast<unsigned long long*>(c_out), host ? dl : lcc_out, st);
    count_launch();
    ev.record(3, stream);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hst, st, sizeof(DgStats), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess && host && c_out && nn)
        e = cudaMemcpyAsync(c_out, dc, sizeof(uint64_t) * nn, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess && host && lcc_out && nn)
        e = cudaMemcpyAsync(lcc_out, dl, sizeof(double) * nn, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail("tc_directed_lcc", e);
    if (stats) {
        *stats = tc_directed_stats{};
        stats->m_directed = (int64_t)hst->m_directed;
        stats->m_undirected = mu;
        stats->loops_dropped = (int64_t)loops;
        stats->total = hst->sum_c;
        stats->list_entries = hst->entries;
        if (timed) {
            stats->build_ms = ev.ms(0, 1);
            stats->count_ms = ev.ms(1, 2);
            stats->finalize_ms = ev.ms(2, 3);
        }
    }
    return TC_OK;
}
