// CPU oracle for triangle counting (TC) and the local clustering coefficient (LCC).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
// statement of what the GPU path computes.  Only the test suite, the smoke check
// and the CPU-baseline leg of the benchmark may load it; the product path never
// does.  It shares no code, header or table with the CUDA library.
//
// What it computes (arxiv 2202.13976):
//  - Sec. II-A: the input is read as a simple undirected graph G = (V, E):
//    self-loops are dropped and {u, v} / {v, u} / repeated pairs are one edge.
//  - Sec. II-B: the graph is held in CSR form (offsets, adjacencies), every
//    adjacency list sorted ascending.
//  - Sec. II-C: edge-centric counting, |adj(v_i) ∩ adj(v_j)| per edge, with the
//    double count removed by restricting the neighbour's list to an upper triangle.
//    Here the upper triangle is taken in the (degree, id) order instead of the id
//    order j < k; any strict total order finds every triangle exactly once.
//  - Alg. 2 (SSI) is the intersection used for the oriented count; Alg. 1 (binary
//    search, read as the textbook lower-bound search) and the Eq. 3 rule that picks
//    between them are used by the paper's per-vertex formula (Alg. 3).
//  - Eq. 2: LCC(i) = 2 t(i) / (deg(i) (deg(i) - 1)), with deg the undirected degree.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <list>
#include <set>
#include <unordered_map>
#include <utility>
#include <vector>

extern "C" {

// Sec. II-A/B: simple undirected graph -> sorted symmetric CSR.
// Inputs: n vertices, m pairs (src[k], dst[k]).  Outputs: offsets[n+1] and
// adj[offsets[n]] (caller provides room for 2m entries).  stats[0..2] receive the
// number of distinct undirected edges, dropped self-loops and dropped repeats.
// Returns 0, or -1 if an id lies outside [0, n).
int or_build_csr(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int64_t* offsets,
                 int32_t* adj, int64_t* stats) {
    std::vector<uint64_t> keys;
    keys.reserve((size_t)m);
    int64_t loops = 0;
    for (int64_t k = 0; k < m; ++k) {
        int64_t u = src[k], v = dst[k];
        if (u < 0 || u >= n || v < 0 || v >= n) return -1;
        if (u == v) {
            ++loops;
            continue;
        }
        uint64_t a = (uint64_t)std::min(u, v), b = (uint64_t)std::max(u, v);
        keys.push_back((a << 32) | b);
    }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    int64_t ms = (int64_t)keys.size();
    stats[0] = ms;
    stats[1] = loops;
    stats[2] = m - loops - ms;

    std::vector<int64_t> deg((size_t)n, 0);
    for (uint64_t key : keys) {
        deg[key >> 32] += 1;
        deg[key & 0xffffffffu] += 1;
    }
    offsets[0] = 0;
    for (int64_t i = 0; i < n; ++i) offsets[i + 1] = offsets[i] + deg[i];
    std::vector<int64_t> pos(offsets, offsets + n);
    for (uint64_t key : keys) {
        int64_t a = (int64_t)(key >> 32), b = (int64_t)(key & 0xffffffffu);
        adj[pos[a]++] = (int32_t)b;
        adj[pos[b]++] = (int32_t)a;
    }
    for (int64_t i = 0; i < n; ++i) std::sort(adj + offsets[i], adj + offsets[i + 1]);
    return 0;
}

// Orientation: keep u -> v iff (deg(u), u) < (deg(v), v).  Every row of the
// oriented CSR is a subsequence of a sorted row, so it stays sorted by id.
void or_orient(int64_t n, const int64_t* offsets, const int32_t* adj, int64_t* off_plus,
               int32_t* adj_plus) {
    off_plus[0] = 0;
    int64_t w = 0;
    for (int64_t u = 0; u < n; ++u) {
        int64_t du = offsets[u + 1] - offsets[u];
        for (int64_t k = offsets[u]; k < offsets[u + 1]; ++k) {
            int64_t v = adj[k];
            int64_t dv = offsets[v + 1] - offsets[v];
            if (du < dv || (du == dv && u < v)) adj_plus[w++] = (int32_t)v;
        }
        off_plus[u + 1] = w;
    }
}

// Alg. 2: sorted set intersection (two pointers) of sorted lists A and B.
int64_t or_ssi(const int32_t* A, int64_t na, const int32_t* B, int64_t nb) {
    int64_t counter = 0, i = 0, j = 0;
    while (i < na && j < nb) {
        if (A[i] == B[j]) {
            ++counter;
            ++i;
            ++j;
        } else if (A[i] < B[j]) {
            ++i;
        } else {
            ++j;
        }
    }
    return counter;
}

// Alg. 1, read as the textbook search: every key x of A is looked up in the
// sorted list B by a lower-bound binary search over [bottom, |B|).  Because A is
// sorted, the lower end carries over from one key to the next; the upper end
// starts at |B| for every key.  (The printed listing omits "bottom +" from the
// midpoint and never resets the upper end; the textbook reading is used.)
int64_t or_binary_search(const int32_t* A, int64_t na, const int32_t* B, int64_t nb) {
    int64_t counter = 0, bottom = 0;
    for (int64_t k = 0; k < na; ++k) {
        int32_t x = A[k];
        int64_t lo = bottom, hi = nb;  // first index in [lo, hi) with B[idx] >= x
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (B[mid] < x)
                lo = mid + 1;
            else
                hi = mid;
        }
        bottom = lo;
        if (lo < nb && B[lo] == x) ++counter;
    }
    return counter;
}

// Eq. 3: with |A| <= |B|, SSI is preferred iff |B| / |A| <= log2(|B|) - 1
// (a tie chooses SSI).  Returns 1 for SSI, 0 for binary search.
int or_prefer_ssi(int64_t a, int64_t b) {
    if (a > b) std::swap(a, b);
    if (a == 0) return 1;  // empty intersection; either method returns 0 at once
    return (double)b / (double)a <= std::log2((double)b) - 1.0 ? 1 : 0;
}

// Hybrid intersection count of two sorted lists (Sec. IV-C): the shorter list is
// the keys, the method is chosen by Eq. 3.
static int64_t hybrid(const int32_t* A, int64_t na, const int32_t* B, int64_t nb) {
    if (na > nb) {
        std::swap(A, B);
        std::swap(na, nb);
    }
    return or_prefer_ssi(na, nb) ? or_ssi(A, na, B, nb) : or_binary_search(A, na, B, nb);
}

// Oriented edge-centric count over the oriented CSR, for source vertices
// u in [u0, u1): for every oriented edge (u, v), W = N+(u) ∩ N+(v) (Alg. 2); then
// t[u] += |W|, t[v] += |W| and t[w] += 1 for every w in W.  Each triangle is met
// once, at the edge joining its two lowest vertices in the orientation order.
// Accumulates into t (length n).
void or_tc_oriented(int64_t n, const int64_t* off_plus, const int32_t* adj_plus, uint64_t* t,
                    int64_t u0, int64_t u1) {
    (void)n;
    for (int64_t u = u0; u < u1; ++u) {
        const int32_t* Nu = adj_plus + off_plus[u];
        int64_t du = off_plus[u + 1] - off_plus[u];
        for (int64_t k = 0; k < du; ++k) {
            int64_t v = Nu[k];
            const int32_t* Nv = adj_plus + off_plus[v];
            int64_t dv = off_plus[v + 1] - off_plus[v];
            // Alg. 2 with the matches recorded.
            int64_t i = 0, j = 0, c = 0;
            while (i < du && j < dv) {
                if (Nu[i] == Nv[j]) {
                    t[Nu[i]] += 1;
                    ++c;
                    ++i;
                    ++j;
                } else if (Nu[i] < Nv[j]) {
                    ++i;
                } else {
                    ++j;
                }
            }
            t[u] += (uint64_t)c;
            t[v] += (uint64_t)c;
        }
    }
}

// The paper's per-vertex formula (Alg. 3 with the Sec. II-C offset), on the
// symmetric CSR: t(v_i) = sum over v_j in adj(v_i) of |adj(v_i) ∩ {v_k in adj(v_j) : j < k}|,
// each intersection by the Eq. 3 hybrid.  Needs no orientation and no shared
// accumulation.  Writes t_out[q] = t(vertices[q]).
void or_tc_vertex(int64_t n, const int64_t* offsets, const int32_t* adj, const int32_t* vertices,
                  int64_t nv, uint64_t* t_out) {
    (void)n;
    for (int64_t q = 0; q < nv; ++q) {
        int64_t i = vertices[q];
        const int32_t* Ai = adj + offsets[i];
        int64_t di = offsets[i + 1] - offsets[i];
        uint64_t t = 0;
        for (int64_t k = 0; k < di; ++k) {
            int64_t j = Ai[k];
            const int32_t* Aj = adj + offsets[j];
            int64_t dj = offsets[j + 1] - offsets[j];
            // {v_k in adj(v_j) : k > j}: the suffix after the last entry <= j.
            const int32_t* up = std::upper_bound(Aj, Aj + dj, (int32_t)j);
            t += (uint64_t)hybrid(Ai, di, up, (Aj + dj) - up);
        }
        t_out[q] = t;
    }
}

// Per-edge support: for every undirected edge {u, v} (listed once, u < v, in CSR
// order) the number of triangles that contain it, |adj(u) ∩ adj(v)| (Alg. 2) -- the
// entries C(u, v) of the algebraic form C = A·A ∘ A of Sec. VI-B.  Writes eu, ev and
// support (room for offsets[n] / 2 entries); returns the number of edges written.
int64_t or_edge_support(int64_t n, const int64_t* offsets, const int32_t* adj, int32_t* eu, int32_t* ev,
                        uint32_t* support) {
    int64_t e = 0;
    for (int64_t u = 0; u < n; ++u) {
        const int32_t* Au = adj + offsets[u];
        const int64_t du = offsets[u + 1] - offsets[u];
        for (int64_t k = 0; k < du; ++k) {
            const int64_t v = Au[k];
            if (v <= u) continue;
            eu[e] = (int32_t)u;
            ev[e] = (int32_t)v;
            support[e] = (uint32_t)or_ssi(Au, du, adj + offsets[v], offsets[v + 1] - offsets[v]);
            ++e;
        }
    }
    return e;
}

// Directed graphs (Sec. II-A, II-C): e_ij is the edge from v_i to v_j and adj(v_i) the
// out-neighbours {v_j : e_ij in E}.  Self-loops are dropped and a repeated (src, dst)
// pair is one edge; (u, v) and (v, u) are two different edges.  Outputs offsets[n+1]
// and adj[offsets[n]] (room for m entries), every out-list sorted ascending.  stats[0..2]
// receive the distinct directed edges, dropped self-loops and dropped repeats.
// Returns 0, or -1 if an id lies outside [0, n).
int or_build_digraph(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int64_t* offsets,
                     int32_t* adj, int64_t* stats) {
    std::vector<uint64_t> keys;
    keys.reserve((size_t)m);
    int64_t loops = 0;
    for (int64_t k = 0; k < m; ++k) {
        int64_t u = src[k], v = dst[k];
        if (u < 0 || u >= n || v < 0 || v >= n) return -1;
        if (u == v) {
            ++loops;
            continue;
        }
        keys.push_back(((uint64_t)u << 32) | (uint64_t)v);
    }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    const int64_t md = (int64_t)keys.size();
    stats[0] = md;
    stats[1] = loops;
    stats[2] = m - loops - md;
    std::fill(offsets, offsets + n + 1, (int64_t)0);
    for (uint64_t key : keys) offsets[(key >> 32) + 1] += 1;
    for (int64_t i = 0; i < n; ++i) offsets[i + 1] += offsets[i];
    for (int64_t k = 0; k < md; ++k) adj[k] = (int32_t)(keys[(size_t)k] & 0xffffffffu);  // sorted by (src, dst)
    return 0;
}

// Eq. 1 (directed LCC) for the listed vertices of a directed CSR:
//   c(i) = |{e_jk in E : v_j, v_k in adj(v_i)}|, counted as the sum over v_j in adj(v_i)
//          of |adj(v_i) ∩ adj(v_j)| (Alg. 2), every edge e_jk met once at its tail v_j;
//   C(i) = c(i) / (deg+(i) (deg+(i) - 1)), 0.0 when deg+(i) < 2.
// Writes c_out[q] and lcc_out[q] for vertex vertices[q].
void or_directed_lcc(int64_t n, const int64_t* offsets, const int32_t* adj, const int32_t* vertices, int64_t nv,
                     uint64_t* c_out, double* lcc_out) {
    (void)n;
    for (int64_t q = 0; q < nv; ++q) {
        const int64_t i = vertices[q];
        const int32_t* Ai = adj + offsets[i];
        const int64_t d = offsets[i + 1] - offsets[i];
        uint64_t c = 0;
        for (int64_t k = 0; k < d; ++k) {
            const int64_t j = Ai[k];
            c += (uint64_t)or_ssi(Ai, d, adj + offsets[j], offsets[j + 1] - offsets[j]);
        }
        c_out[q] = c;
        lcc_out[q] = d < 2 ? 0.0 : (double)c / (double)(d * (d - 1));
    }
}

// ---------------------------------------------------------------------------
// Remote reads of the distributed algorithm (Sec. IV-A, Alg. 4) and their caches
// (Sec. IV-B).  1D partition: process k owns the ids [floor(k n / p), floor((k+1) n / p)).
// Process k walks its vertices v_i in id order and, for every v_j in adj(v_i) (sorted,
// Sec. II-B), reads adj(v_j) remotely when v_j belongs to another process.

// The read stream over a sorted symmetric CSR: item_out[t] = v_j and part_out[t] = k
// for every remote read, processes in order; returns the number of reads.
int64_t or_remote_reads(int64_t n, const int64_t* offsets, const int32_t* adj, int64_t parts, int32_t* item_out,
                        int32_t* part_out) {
    int64_t t = 0;
    for (int64_t k = 0; k < parts; ++k) {
        const int64_t lo = k * n / parts, hi = (k + 1) * n / parts;
        for (int64_t i = lo; i < hi; ++i)
            for (int64_t e = offsets[i]; e < offsets[i + 1]; ++e) {
                const int64_t j = adj[e];
                if (j < lo || j >= hi) {
                    item_out[t] = (int32_t)j;
                    part_out[t] = (int32_t)k;
                    ++t;
                }
            }
    }
    return t;
}

// LRU cache of `capacity` bytes over one process's reads (items[0..count), entry
// sizes size_of[item] bytes): a hit moves the entry to the front; a miss inserts it at
// the front and evicts from the back until the entries fit (an entry larger than the
// cache evicts everything, itself included).  Returns the hits; *hit_bytes gets their
// bytes.
uint64_t or_cache_lru(int64_t count, const int32_t* items, const uint64_t* size_of, uint64_t capacity,
                      uint64_t* hit_bytes) {
    std::list<int32_t> order;  // front = most recent
    std::unordered_map<int32_t, std::list<int32_t>::iterator> where;
    uint64_t used = 0, hits = 0, hb = 0;
    for (int64_t t = 0; t < count; ++t) {
        const int32_t x = items[t];
        auto it = where.find(x);
        if (it != where.end()) {
            ++hits;
            hb += size_of[x];
            order.splice(order.begin(), order, it->second);
            continue;
        }
        order.push_front(x);
        where[x] = order.begin();
        used += size_of[x];
        while (used > capacity) {
            const int32_t z = order.back();
            order.pop_back();
            where.erase(z);
            used -= size_of[z];
        }
    }
    *hit_bytes = hb;
    return hits;
}

// Cache with application-defined scores (Sec. IV-B2): every cached entry carries a
// score, and whenever an entry must be evicted the victim is the cached entry of the
// lowest score.  A miss of x is stored if it can be: an entry larger than the whole
// cache cannot, and evicts nothing; otherwise the lowest-scored cached entries are
// evicted, one at a time, until x fits, and x is stored (the incoming entry is never
// its own victim).  The score of a cached entry is the one given with its latest read,
// score_at[t] for the read at time t (a hit refreshes it); equal scores evict the
// smaller item first.  Returns the hits; *hit_bytes gets their bytes.
uint64_t or_cache_priority(int64_t count, const int32_t* items, const uint64_t* size_of, const int64_t* score_at,
                           uint64_t capacity, uint64_t* hit_bytes) {
    typedef std::pair<int64_t, int32_t> Entry;  // (score, item), lowest first
    std::set<Entry> cache;
    std::unordered_map<int32_t, int64_t> score_of;  // the cached entries and their scores
    uint64_t used = 0, hits = 0, hb = 0;
    for (int64_t t = 0; t < count; ++t) {
        const int32_t x = items[t];
        auto it = score_of.find(x);
        if (it != score_of.end()) {
            ++hits;
            hb += size_of[x];
            cache.erase(Entry(it->second, x));
            it->second = score_at[t];
            cache.insert(Entry(score_at[t], x));
            continue;
        }
        if (size_of[x] > capacity) continue;  // cannot be stored
        while (used + size_of[x] > capacity) {
            const Entry z = *cache.begin();
            cache.erase(cache.begin());
            score_of.erase(z.second);
            used -= size_of[z.second];
        }
        cache.insert(Entry(score_at[t], x));
        score_of[x] = score_at[t];
        used += size_of[x];
    }
    *hit_bytes = hb;
    return hits;
}

// The degree score of the TC application (Sec. IV-B2): the score of the entry of v_j is
// its degree, ties between equal degrees going to the larger id, i.e. the victim is the
// cached entry of the lowest (degree, id).  Returns the hits; *hit_bytes their bytes.
uint64_t or_cache_score(int64_t count, const int32_t* items, const uint64_t* size_of, const int64_t* degree,
                        uint64_t capacity, uint64_t* hit_bytes) {
    std::vector<int64_t> score((size_t)count);
    for (int64_t t = 0; t < count; ++t) score[(size_t)t] = (degree[items[t]] << 32) | (int64_t)items[t];
    return or_cache_priority(count, items, size_of, score.data(), capacity, hit_bytes);
}

// Eq. 2: LCC(i) = 2 t(i) / (deg(i) (deg(i) - 1)); 0.0 when deg(i) < 2.  Both the
// numerator and the denominator are exact integers below 2^53, so the single fp64
// division is correctly rounded.
void or_lcc(int64_t n, const int64_t* offsets, const uint64_t* t, double* lcc) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t d = offsets[i + 1] - offsets[i];
        lcc[i] = d < 2 ? 0.0 : (double)(2 * t[i]) / (double)(d * (d - 1));
    }
}

}  // extern "C"
