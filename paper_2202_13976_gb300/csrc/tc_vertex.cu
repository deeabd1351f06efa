// The paper's unoriented per-vertex formula on the GPU (Alg. 3 with the Sec. II-C
// offset), as an alternative to the oriented count for comparison and ablation:
//   t(v_i) = sum over v_j in adj(v_i) of |adj(v_i) ∩ {v_k in adj(v_j) : k > j}|.
// Vertices carry their ranks as labels, so {v_k in adj(v_j) : k > j} is N+(j), the
// oriented row the build already holds, and only the symmetric rows adj(i) are
// built here: the oriented entries u -> v are turned into keys (v, u), radix sorted,
// and written as the lower part of each row (in-neighbours, ascending), the oriented
// row N+(i) copied after them.  In adj(i) = [lower part, N+(i)] the entries after
// j = adj(i)[k] are exactly those above j, and only they can lie in N+(j), so a lane
// intersects adj(i)[k+1..] with N+(j), by a merge (Alg. 2) or by binary
// search of the shorter list in the longer (Alg. 1) as Eq. 3 decides.  One warp forms
// each vertex's sum and writes it once; vertices are taken from the highest rank
// (largest degree) down through a counter.
#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {
namespace {

constexpr int VF_THREADS = 256;

// Keys of the oriented entries: key = (v << b) | u for u -> v; the slots that
// deduplication left free get the all-ones key, which sorts after every entry.
__global__ void k_vf_keys(int32_t n, const int64_t* __restrict__ rowstart, const int32_t* __restrict__ rowlen,
                          const int32_t* __restrict__ col, int b, uint64_t* __restrict__ keys) {
    const int lane = lane_id();
    const uint64_t none = (b >= 32 ? ~0ull : ((1ull << (2 * b)) - 1));
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int64_t a0 = rowstart[u], a1 = rowstart[u + 1];
        const int d = rowlen[u];
        for (int64_t p = a0 + lane; p < a1; p += 32)
            keys[p] = p - a0 < d ? ((uint64_t)(uint32_t)col[p] << b) | (uint64_t)u : none;
    }
}

// Lower parts: sorted key k = (v, u) goes to adj(v) at position k - instart[v].
__global__ void k_vf_lower(int64_t m, const uint64_t* __restrict__ keys, int b, const int64_t* __restrict__ sym_start,
                           const int64_t* __restrict__ instart, int32_t* __restrict__ sym) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t umask = (1ull << b) - 1;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += stride) {
        const uint64_t key = keys[k];
        const int64_t v = (int64_t)(key >> b), u = (int64_t)(key & umask);
        sym[sym_start[v] + (k - instart[v])] = (int32_t)u;
    }
}

// Upper parts: N+(u) copied after the lower part of adj(u).
__global__ void k_vf_upper(int32_t n, const int64_t* __restrict__ rowstart, const int32_t* __restrict__ rowlen,
                           const int32_t* __restrict__ deg, const int64_t* __restrict__ sym_start,
                           const int32_t* __restrict__ col, int32_t* __restrict__ sym) {
    const int lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int d = rowlen[u];
        const int64_t dst = sym_start[u] + (deg[u] - d), src = rowstart[u];
        for (int p = lane; p < d; p += 32) sym[dst + p] = col[src + p];
    }
}

__global__ void k_vf_indeg(int32_t n, const int32_t* __restrict__ deg, const int32_t* __restrict__ rowlen,
                           uint32_t* __restrict__ indeg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        indeg[v] = (uint32_t)(deg[v] - rowlen[v]);
}

// |A ∩ B| for sorted A[0, a) and B[0, b): Eq. 3 between the merge and a binary search
// of each key of the shorter list in the longer one (lower end carried over).
__device__ uint32_t lane_count_hybrid(const int32_t* __restrict__ A, int a, const int32_t* __restrict__ B, int b) {
    if (a == 0 || b == 0) return 0;
    const int s = min(a, b), l = max(a, b);
    uint32_t c = 0;
    if ((float)l <= (log2f((float)l) - 1.0f) * (float)s) {
        int i = 0, j = 0;
        while (i < a && j < b) {
            const int32_t x = A[i], y = B[j];
            c += x == y;
            i += x <= y;
            j += y <= x;
        }
        return c;
    }
    const int32_t* S = a <= b ? A : B;
    const int32_t* L = a <= b ? B : A;
    int lo = 0;
    for (int k = 0; k < s && lo < l; ++k) {
        const int32_t x = S[k];
        lo = lower_bound(L, lo, l, x);
        if (lo < l && L[lo] == x) ++c;
    }
    return c;
}

__global__ void __launch_bounds__(VF_THREADS) k_vf_count(int32_t n, const int64_t* __restrict__ sym_start,
                                                         const int32_t* __restrict__ sym,
                                                         const int2* __restrict__ rowinfo,
                                                         const int32_t* __restrict__ col,
                                                         unsigned long long* __restrict__ t,
                                                         unsigned* __restrict__ counter) {
    const int lane = lane_id();
    for (;;) {
        unsigned q = 0;
        if (lane == 0) q = atomicAdd(counter, 1u);
        q = __shfl_sync(FULL, q, 0);
        if (q >= (unsigned)n) break;
        const int32_t i = n - 1 - (int32_t)q;
        const int64_t a0 = sym_start[i];
        const int da = (int)(sym_start[i + 1] - a0);
        const int32_t* A = sym + a0;
        unsigned long long c = 0;
        for (int k = lane; k < da; k += 32) {
            const int2 rj = rowinfo[A[k]];  // N+(j), j = A[k]
            c += lane_count_hybrid(A + k + 1, da - k - 1, col + rj.x, rj.y);
        }
        c = warp_sum(c);
        if (lane == 0) t[i] = c;
    }
}

__global__ void k_vf_id_of(int32_t n, const int32_t* __restrict__ rank, int32_t* __restrict__ id_of) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) id_of[rank[v]] = (int32_t)v;
}

// Per-edge supports out of the count: the oriented entry x -> y at col index e is the
// undirected edge {x, y}; it goes to estart[x] + position in x's row, in the caller's
// ids, smaller first, with the support the count recorded at e.
__global__ void k_support_out(int32_t n, const int2* __restrict__ rowinfo,
                              const int32_t* __restrict__ col, const uint32_t* __restrict__ sup,
                              const int32_t* __restrict__ id_of, const int64_t* __restrict__ estart,
                              int32_t* __restrict__ eu, int32_t* __restrict__ ev, uint32_t* __restrict__ support) {
    const int lane = lane_id();
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
        const int2 rx = rowinfo[x];
        const int32_t idx = id_of[x];
        const int64_t e0 = estart[x];
        for (int p = lane; p < rx.y; p += 32) {
            const int32_t idy = id_of[col[rx.x + p]];
            eu[e0 + p] = min(idx, idy);
            ev[e0 + p] = max(idx, idy);
            support[e0 + p] = sup[rx.x + p];
        }
    }
}

__global__ void k_vf_sum(int32_t n, const unsigned long long* __restrict__ t, unsigned long long* __restrict__ out) {
    unsigned long long s = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) s += t[v];
    s = warp_sum(s);
    if (lane_id() == 0 && s) atomicAdd(out, s);
}

}  // namespace

int vf_key_bits(int32_t n) {
    int b = 1;
    while (b < 31 && ((int64_t)1 << b) < (int64_t)n) ++b;
    return b;
}

void launch_symmetric_rows(const VertexFormulaBuffers& V, const Launch& L) {
    if (V.n <= 0) return;
    const int b = vf_key_bits(V.n);
    k_vf_indeg<<<grid_for(V.n, VF_THREADS, L.sms), VF_THREADS, 0, L.stream>>>(V.n, V.deg, V.rowlen, V.indeg);
    count_launch();
    scan_u32_to_i64(reinterpret_cast<const uint32_t*>(V.deg), V.sym_start, V.n, V.tmp, L);
    scan_u32_to_i64(V.indeg, V.instart, V.n, V.tmp, L);
    if (V.m_cap > 0) {
        cudaMemsetAsync(V.keys, 0xff, sizeof(uint64_t) * (size_t)V.m_cap, L.stream);  // slots past the rows
        k_vf_keys<<<grid_for((int64_t)V.n * 32, VF_THREADS, L.sms), VF_THREADS, 0, L.stream>>>(
            V.n, V.rowstart, V.rowlen, V.col, b, V.keys);
        count_launch();
        uint64_t* sorted = radix_sort_u64(V.keys, V.keys_alt, V.m_cap, 0, 2 * b, V.radix_tmp, L);
        k_vf_lower<<<grid_for(V.m, VF_THREADS, L.sms), VF_THREADS, 0, L.stream>>>(V.m, sorted, b, V.sym_start,
                                                                                V.instart, V.sym);
        count_launch();
    }
    k_vf_upper<<<grid_for((int64_t)V.n * 32, VF_THREADS, L.sms), VF_THREADS, 0, L.stream>>>(
        V.n, V.rowstart, V.rowlen, V.deg, V.sym_start, V.col, V.sym);
    count_launch();
}

void launch_vertex_formula(const VertexFormulaBuffers& V, const Launch& L) {
    if (V.n <= 0) return;
    launch_symmetric_rows(V, L);
    cudaMemsetAsync(V.counter, 0, sizeof(unsigned), L.stream);
    cudaMemsetAsync(V.sum, 0, sizeof(unsigned long long), L.stream);
    k_vf_count<<<L.sms * 8, VF_THREADS, 0, L.stream>>>(V.n, V.sym_start, V.sym, V.rowinfo, V.col, V.t,
                                                      V.counter);
    count_launch();
    k_vf_sum<<<grid_for(V.n, VF_THREADS, L.sms), VF_THREADS, 0, L.stream>>>(V.n, V.t, V.sum);
    count_launch();
}

void launch_support_out(int32_t n, const int32_t* rank, const int32_t* rowlen, const int2* rowinfo, const int32_t* col,
                        const uint32_t* sup, int32_t* id_of, int64_t* estart, void* scan_tmp, int32_t* eu, int32_t* ev,
                        uint32_t* support, const Launch& L) {
    if (n <= 0) return;
    k_vf_id_of<<<grid_for(n, VF_THREADS, L.sms), VF_THREADS, 0, L.stream>>>(n, rank, id_of);
    count_launch();
    scan_u32_to_i64(reinterpret_cast<const uint32_t*>(rowlen), estart, n, scan_tmp, L);
    k_support_out<<<grid_for((int64_t)n * 32, VF_THREADS, L.sms), VF_THREADS, 0, L.stream>>>(
        n, rowinfo, col, sup, id_of, estart, eu, ev, support);
    count_launch();
}

}  // namespace tcg
