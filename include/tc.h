/*
 * tc.h -- triangle counting (TC) and local clustering coefficient (LCC) on one
 * GB300 GPU (sm_103a).  C ABI: plain pointers and sizes, no C++ or framework types.
 *
 * Problem statement (arxiv 2202.13976): the input is read as a simple, unweighted,
 * undirected graph G = (V, E), |V| = n (Sec. II-A), given as an edge list or in
 * CSR form (Sec. II-B).  The library computes
 *   t(v)   = number of triangles that contain v            (Sec. I, Sec. II-D)
 *   T      = (1/3) * sum_v t(v)                             (Sec. II-C)
 *   LCC(v) = 2 t(v) / (deg(v) (deg(v) - 1)), 0 if deg(v) < 2 (Eq. 2)
 * exactly: counts are unsigned 64-bit integers and LCC is one correctly rounded
 * IEEE fp64 division of two exact integers.
 *
 * Conventions shared by every call:
 *  - Vertex ids are int32 in [0, n); n <= 2^31 - 1.  Edge counts are int64 and at
 *    most 2^31 - 1 pairs are accepted.
 *  - Input semantics: (u, v) and (v, u) are the same edge; self-loops and repeated
 *    pairs are dropped and counted (tc_graph_info).  An id outside [0, n) makes the
 *    call fail with TC_EINVAL.
 *  - mem_kind says where a caller pointer lives: TC_MEM_HOST (pageable or pinned
 *    host memory) or TC_MEM_DEVICE (device memory of the current CUDA device).
 *  - Ownership: the library copies what it needs from the inputs before the call
 *    returns; the caller keeps ownership of every buffer it passes.  Outputs are
 *    caller-allocated.
 *  - Streams: a graph is bound to the CUDA stream given at creation (NULL = the
 *    legacy default stream); all device work of that graph is ordered on it.  Calls
 *    that return host data synchronise that stream before returning.
 *  - Errors never abort the process: every failure is a tc_status.  Device-side
 *    checks raise a flag that the host turns into a status.
 *  - Thread safety: distinct graphs may be used from distinct host threads; one
 *    graph must not be used from two threads at once.
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tc_status {
    TC_OK = 0,
    TC_EINVAL = 1,   /* bad argument: id outside [0, n), size out of range, NULL */
    TC_ENOMEM = 2,   /* device or host allocation failed */
    TC_ECUDA = 3,    /* a CUDA runtime call failed (no device, launch failure, ...) */
    TC_ETIMEOUT = 4, /* a bounded device-side wait gave up */
    TC_EBUSY = 5,    /* the object is in use (server admission full) */
    TC_EINTERNAL = 6 /* an internal consistency check failed (sum t != 0 mod 3, ...) */
} tc_status;

enum { TC_MEM_HOST = 0, TC_MEM_DEVICE = 1 };

typedef struct tc_graph tc_graph;

/*
 * Build a graph from an undirected edge list (Sec. II-A/B, Alg. 3 "build CSR").
 *   n            number of vertices (>= 0)
 *   m            number of pairs (0 <= m <= 2^31 - 1)
 *   src, dst     m int32 ids each; may be NULL when m == 0
 *   mem_kind     where src/dst live
 *   cuda_stream  a cudaStream_t (as void*), or NULL
 *   out          receives the new graph; *out is NULL on failure
 * The device copy holds the simple graph's degree-oriented CSR; the triangle count
 * itself runs at the first tc_count / lcc_compute.
 * Errors: TC_EINVAL (n < 0, m out of range, NULL pointers, id outside [0, n)),
 *         TC_ENOMEM, TC_ECUDA.
 */
tc_status tc_graph_create_from_edges(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                     int mem_kind, void* cuda_stream, tc_graph** out);

/*
 * Build a graph from CSR arrays (Sec. II-B, Fig. 2): row i lists
 * adj[offsets[i] .. offsets[i+1]).  Every entry (i, adj[k]) is read as the
 * undirected pair {i, adj[k]}, so rows need not be sorted, symmetric or free of
 * repeats; the library re-normalises.
 *   offsets  n + 1 int64 values, offsets[0] == 0, non-decreasing,
 *            offsets[n] <= 2^31 - 1
 *   adj      offsets[n] int32 ids
 * Errors: as tc_graph_create_from_edges, plus TC_EINVAL for bad offsets.
 */
tc_status tc_graph_create_from_csr(int32_t n, const int64_t* offsets, const int32_t* adj,
                                   int mem_kind, void* cuda_stream, tc_graph** out);

/*
 * Global triangle count T = (1/3) sum_v t(v) (Sec. II-C), written to the host
 * scalar *T_out.  Runs the intersection if it has not run yet; synchronises the
 * graph's stream.  Errors: TC_EINVAL (NULL), TC_ECUDA, TC_EINTERNAL (sum t is not
 * a multiple of 3).
 */
tc_status tc_count(tc_graph* g, uint64_t* T_out);

/*
 * Per-vertex triangle counts t[n] (uint64) and LCC[n] (fp64, Eq. 2), in the
 * caller's vertex ids.  Either output may be NULL to skip it.  mem_kind says where
 * the outputs live; with TC_MEM_DEVICE the results are written by kernels on the
 * graph's stream, with TC_MEM_HOST they are copied back and the stream is
 * synchronised.  Degree-0/1 vertices report t = 0 and LCC = +0.0.
 */
tc_status lcc_compute(tc_graph* g, uint64_t* t_out, double* lcc_out, int mem_kind);

/*
 * One shard of the count, for a graph replicated on several GPUs (one process per
 * GPU).
 * The shards partition the triangles. Each triangle is counted once, from its
 * lowest-ranked vertex u, the source of the oriented edges (Alg. 2 on the
 * degree-oriented graph, Sec. III).
 * Shard `shard` of `nshards` counts the triangles whose u lies in one range of
 * ranks. The ranges are cut where the prefix of the per-source cost
 * d+(u) (d+(u) + 1) / 2 + 1 crosses equal shares of the total. This balances work
 * rather than vertices, unlike the paper's 1D partition, whose imbalance Sec. V
 * reports.
 *   shard, nshards  0 <= shard < nshards; nshards = 1 counts the whole graph
 *   t_out           NULL, or n uint64: this shard's share of t(v) in the caller's
 *                   vertex ids. Summed over all shards it equals t(v).
 *   mem_kind        where t_out lives (as lcc_compute)
 *   T_out           NULL, or the host scalar that receives this shard's triangles.
 *                   Summed over all shards it equals T.
 * The graph is not changed: a later tc_count or lcc_compute counts the whole graph
 * again. Synchronises the graph's stream to read the shard's bounds.
 * Errors: TC_EINVAL (NULL graph, shard out of range, bad mem_kind), TC_ENOMEM,
 * TC_ECUDA, TC_EINTERNAL.
 */
tc_status tc_count_shard(tc_graph* g, int32_t shard, int32_t nshards, uint64_t* t_out, int mem_kind,
                         uint64_t* T_out);

/*
 * LCC[n] (fp64, Eq. 2) in the caller's vertex ids, from per-vertex counts t[n]
 * (uint64, caller's ids). t is typically the sum of the shards' t_out of
 * tc_count_shard.
 * The arithmetic is the same as lcc_compute's: LCC(v) = 2 t(v) / (d(v) (d(v) - 1)),
 * one correctly rounded division, and +0.0 for d(v) < 2 or t(v) = 0.
 * t and lcc_out both live where mem_kind says.
 * Errors: TC_EINVAL (NULL, bad mem_kind), TC_ENOMEM, TC_ECUDA.
 */
tc_status tc_lcc_from_counts(tc_graph* g, const uint64_t* t, double* lcc_out, int mem_kind);

/*
 * Per-vertex triangle counts by the paper's unoriented per-vertex formula (Alg. 3
 * with the Sec. II-C offset): t(v_i) = sum over v_j in adj(v_i) of
 * |adj(v_i) ∩ {v_k in adj(v_j) : k > j}|, each intersection chosen per pair by Eq. 3
 * (merge, Alg. 2, or binary search of the shorter list, Alg. 1), every vertex's sum
 * formed by one warp and written once (no shared accumulation).  The graph's
 * vertices are relabelled by rank, so "k > j" compares ranks; the symmetric CSR it
 * needs is built for the call (a radix sort of the transposed oriented entries) and
 * released after it.  An alternative to tc_count / lcc_compute for comparison and
 * ablation: same results, far more work on skewed graphs.  t_out[n] (uint64) in the
 * caller's ids, in mem_kind memory; the stream is synchronised.  *T_out (may be
 * NULL) receives sum t / 3.  Errors: TC_EINVAL (NULL t_out, bad mem_kind), TC_ENOMEM,
 * TC_ECUDA, TC_EINTERNAL (sum t is not a multiple of 3).
 */
tc_status tc_count_vertex_formula(tc_graph* g, uint64_t* t_out, int mem_kind, uint64_t* T_out);

/*
 * Per-edge support (an extension toward k-truss; Sec. VI-B's C = A·A ∘ A read edge
 * by edge): for every distinct undirected edge {u, v} the number of triangles that
 * contain it, |adj(u) ∩ adj(v)|.  Writes m_simple entries (tc_graph_info): u_out[k] <
 * v_out[k] in the caller's ids, support_out[k] (uint32), each edge once, in an order
 * of the library's choosing (row by row in its internal rank order); all three
 * arrays in mem_kind memory.  Runs the oriented count once more with every triangle
 * also added to its three edges (the dense core off, since it counts words of bits
 * without naming triangles); the graph's tuning is restored afterwards.
 * Synchronises the stream.  Errors: TC_EINVAL (NULL output, bad mem_kind),
 * TC_ENOMEM, TC_ECUDA, TC_EINTERNAL.
 */
tc_status tc_edge_support(tc_graph* g, int32_t* u_out, int32_t* v_out, uint32_t* support_out, int mem_kind);

/*
 * Remote adjacency reads of the distributed algorithm (Sec. IV-A, Alg. 4) and the
 * caches of Sec. IV-B, for every cache size in one call.  The graph's ids are split
 * into `parts` processes (1D partition: process k owns [floor(k n / parts),
 * floor((k+1) n / parts))); process k walks its vertices v_i in id order and every v_j
 * of the sorted list adj(v_i), and reads adj(v_j) remotely (after its offsets) when
 * v_j belongs to another process.  Four caches are evaluated per process, each at
 * every capacity (bytes) of capacity_bytes[0..ncap), which must be non-decreasing:
 *   TC_CACHE_ADJ_LRU, TC_CACHE_ADJ_SCORE   adjacency lists, an entry of 4 deg(v_j) bytes
 *   TC_CACHE_OFF_LRU, TC_CACHE_OFF_SCORE   offsets, an entry of 16 bytes
 * LRU: a miss inserts the entry as the most recent and evicts the least recent until
 * the entries fit (an entry larger than the cache is never held).  SCORE
 * (application-defined scores, Sec. IV-B2): whenever an entry must be evicted the
 * victim is the cached entry of the lowest (degree, id); a miss is stored after
 * evicting the lowest entries until it fits, unless it is larger than the whole
 * cache (then it is not stored and nothing is evicted).
 *   hits, hit_bytes   host uint64[TC_CACHE_KINDS][parts][ncap] or NULL: the reads that
 *                     hit (and their bytes) per cache, process and capacity
 *   part_stats        host tc_remote_part[parts] or NULL
 * The graph's stream is synchronised.  Errors: TC_EINVAL (NULL graph, parts < 1 or >
 * n, ncap < 0, NULL or decreasing capacities, a graph built from bad ids), TC_ENOMEM,
 * TC_ECUDA.
 */
enum { TC_CACHE_ADJ_LRU = 0, TC_CACHE_ADJ_SCORE = 1, TC_CACHE_OFF_LRU = 2, TC_CACHE_OFF_SCORE = 3,
       TC_CACHE_KINDS = 4 };

typedef struct tc_remote_part {
    int64_t reads;       /* remote reads of adjacency lists */
    int64_t top_reads;   /* of them, reads of the ceil(n / 10) vertices of highest (degree, id) */
    int64_t distinct;    /* distinct remote vertices read: the first-read misses of every cache */
    int64_t read_bytes;  /* bytes of the adjacency lists read, 4 deg(v_j) each */
} tc_remote_part;

tc_status tc_remote_cache(tc_graph* g, int32_t parts, int32_t ncap, const uint64_t* capacity_bytes, uint64_t* hits,
                          uint64_t* hit_bytes, tc_remote_part* part_stats);

/*
 * Directed local clustering coefficient, Eq. 1 (Sec. II-C), from a directed edge list.
 * Pair k is the edge e_ij from i = src[k] to j = dst[k] (Sec. II-A); self-loops are
 * dropped and a repeated (src, dst) pair is one edge, while (u, v) and (v, u) are two
 * different edges.  With adj(v_i) the out-neighbours of v_i and deg+(i) = |adj(v_i)|:
 *   c(i) = |{e_jk in E : v_j, v_k in adj(v_i)}|        (ordered pairs j != k)
 *   C(i) = c(i) / (deg+(i) (deg+(i) - 1)), +0.0 when deg+(i) < 2 or c(i) = 0,
 * one IEEE fp64 division of the two integers (the correctly rounded ratio while
 * deg+(i) < 2^26).  On a symmetric input (both directions of every edge) c = 2t and
 * C is Eq. 2's LCC.
 *   n, m          vertices (>= 0) and pairs (0 <= m <= 2^31 - 1)
 *   src, dst      int32[m] in mem_kind memory, read only (the caller keeps them)
 *   cuda_stream   stream the work is ordered on (NULL: the legacy default stream);
 *                 the call synchronises it before returning
 *   c_out         uint64[n] or NULL, in mem_kind memory, caller's ids
 *   lcc_out       double[n] or NULL, in mem_kind memory, caller's ids
 *   stats         host struct or NULL, filled on success
 *   flags         TC_DIRECTED_TIMED: time the phases with CUDA events on the stream
 *                 and count the list entries the intersections read (stats fields)
 * Works on the undirected graph underlying the input, oriented by (degree, id) as
 * tc_count is, with two direction bits per edge; scratch comes from the library's
 * device pool and is released before the call returns.  Errors: TC_EINVAL (an id
 * outside [0, n), n < 0, m out of range, NULL src/dst with m > 0, bad mem_kind or
 * flags; the outputs are then left untouched), TC_ENOMEM, TC_ECUDA.
 */
enum { TC_DIRECTED_TIMED = 1 };

typedef struct tc_directed_stats {
    int64_t m_directed;      /* distinct directed edges after dropping loops and repeats */
    int64_t m_undirected;    /* edges of the underlying undirected graph */
    int64_t loops_dropped;   /* self-loops in the input */
    uint64_t total;          /* sum over i of c(i) */
    uint64_t list_entries;   /* TC_DIRECTED_TIMED: sum over oriented edges (u, v) of d+(u) + d+(v) */
    float build_ms;          /* TC_DIRECTED_TIMED: undirected build, direction bits, in-edge lists (input copy excluded) */
    float count_ms;          /* TC_DIRECTED_TIMED: the intersection kernel */
    float finalize_ms;       /* TC_DIRECTED_TIMED: c and C in the caller's ids */
    float pad;
} tc_directed_stats;

tc_status tc_directed_lcc(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, int mem_kind,
                          void* cuda_stream, uint64_t* c_out, double* lcc_out, tc_directed_stats* stats,
                          int flags);

/*
 * Input accounting (Sec. II-A: the input is read as a simple graph, so self-loops
 * and repeated pairs leave it): number of distinct undirected edges |E|, self-loops
 * dropped and repeated pairs dropped.  Any pointer may be NULL.  Synchronises the
 * stream.  Errors: TC_EINVAL for a NULL graph; TC_ECUDA.
 */
tc_status tc_graph_info(const tc_graph* g, int64_t* m_simple, int64_t* loops_dropped,
                        int64_t* dups_dropped);

/* Number of vertices |V| and of oriented edges (Sec. II-C orients every edge of E
 * once, so this is |E|).  Errors: TC_EINVAL for a NULL graph; TC_ECUDA. */
tc_status tc_graph_size(const tc_graph* g, int32_t* n, int64_t* m_oriented);

/* Release the graph's device memory (back to the library's device pool).  NULL is
 * a no-op.  The paper defines no such call: it is this library's ownership rule
 * (the graph object owns the device CSR of Sec. II-B that tc_graph_create_* built). */
void tc_graph_destroy(tc_graph* g);

/* Static, NUL-terminated description of a status code (no counterpart in the
 * paper: the status codes are this library's error reporting).  Unknown codes give
 * "unknown tc_status". */
const char* tc_status_str(tc_status s);

/* Detail of the last failure on the calling host thread (CUDA error text or the
   failed check), NUL-terminated; empty if none.  Valid until the next call. */
const char* tc_last_error_detail(void);

/*
 * Intersection strategies (Sec. II-C, Sec. IV-C).  The result never depends on the
 * strategy, only the speed.
 *   TC_STRAT_AUTO      per-edge choice by the hybrid rule of Eq. 3 (with the
 *                      tunable factor below); bitmap staging in the hub bucket
 *   TC_STRAT_MERGE     merge of the two sorted lists (Alg. 2, SSI); in the block
 *                      bucket split across a warp along merge-path diagonals
 *   TC_STRAT_SEARCH    binary search of every key of one list in the other (Alg. 1)
 *   TC_STRAT_PROBE     the staged list (shared memory, sorted) is probed by binary
 *                      search with every element of the streamed list
 *   TC_STRAT_BITMAP    the staged list is a bitmap over its rank window, probed
 *                      with one shared-memory load per streamed element
 *   TC_STRAT_HASH      (small bucket) for sources with more than 16 entries, N+(u)
 *                      is a hash set in shared memory and the rows N+(v) of all of
 *                      u's edges are read end to end, one element per lane, each
 *                      probed once in the set; shorter sources as AUTO
 */
enum {
    TC_STRAT_AUTO = 0,
    TC_STRAT_MERGE = 1,
    TC_STRAT_SEARCH = 2,
    TC_STRAT_PROBE = 3,
    TC_STRAT_BITMAP = 4,
    TC_STRAT_HASH = 5
};

/*
 * Buckets of the planner.  Vertices are ranked by (degree, id); every edge is
 * oriented from the lower to the higher rank, and N+(u) is the oriented row of u.
 *   TC_BUCKET_SMALL  edges (u, v), v not a hub, 2 <= |N+(u)| <= 256: groups of 8, 16
 *                    or 32 lanes per source vertex; HASH (the default) reads the
 *                    rows of all of u's edges end to end across the lanes (sources
 *                    of more than 16 entries), AUTO, MERGE and SEARCH take one edge
 *                    per lane
 *   TC_BUCKET_CTA    edges (u, v), v not a hub, |N+(u)| > 32: one thread block per
 *                    source vertex, N+(u) staged in shared memory, one warp per
 *                    edge (AUTO, MERGE, SEARCH, PROBE, BITMAP)
 *   TC_BUCKET_HUB    edges (u, v) into a hub v: one thread block per hub, N+(v)
 *                    staged in shared memory once, then every edge that hits v
 *                    streams its suffix of N+(u) against it (AUTO = BITMAP, PROBE)
 * Hubs are the highest-ranked vertices whose degree reaches a threshold
 * (tc_graph_set_hubs).
 */
enum { TC_BUCKET_SMALL = 0, TC_BUCKET_CTA = 1, TC_BUCKET_HUB = 2, TC_NUM_BUCKETS = 3 };

/*
 * Per-graph tuning, applied at the next intersection (set before tc_count).
 *   strategy  one of TC_STRAT_* for the bucket
 *   factor    Eq. 3 is applied as  |B| / |A| <= factor * (log2|B| - 1)  when the
 *             strategy is TC_STRAT_AUTO; factor = 1 is the paper's rule.
 * Errors: TC_EINVAL for an unknown bucket or strategy, a strategy the bucket
 * cannot run (see the bucket list), or factor <= 0.
 */
tc_status tc_graph_set_strategy(tc_graph* g, int bucket, int strategy, double factor);

/*
 * Hub selection: vertices with degree >= min_degree are candidates, and at most
 * max_hubs of the highest-ranked candidates are staged (max_hubs is capped at
 * 131072, the bitmap window of one thread block).  max_hubs = 0 disables the hub
 * bucket.  Defaults: min_degree 32, max_hubs 131072.  Errors: TC_EINVAL for
 * negative values.
 */
tc_status tc_graph_set_hubs(tc_graph* g, int32_t min_degree, int32_t max_hubs);

/*
 * Timing of the last intersection in milliseconds (CUDA events on the graph's
 * stream): ms[0] planning (bucket lists and hub in-edge lists), ms[1] small
 * bucket, ms[2] block bucket, ms[3] hub bucket, ms[4] total.  count is the length
 * of ms (up to 5).  Synchronises the stream.  Errors: TC_EINVAL before the first
 * count.
 */
tc_status tc_graph_last_timing(const tc_graph* g, float* ms, int count);

/*
 * Timing of the graph's build in milliseconds (CUDA events): ms[0] ingest and
 * checks, ms[1] (degree, id) ranks, ms[2] row counts, ms[3] row fill, ms[4] row
 * sort and deduplication, ms[5] degrees, ms[6] total.  count up to 7.  Errors:
 * TC_EINVAL when the build was not timed (a batch recorded into a CUDA graph).
 */
tc_status tc_graph_build_timing(const tc_graph* g, float* ms, int count);

/*
 * Work accounting of the planned intersection, per bucket (b = TC_BUCKET_*):
 *   edges[b]  oriented edges handled by bucket b
 *   ids[b]    sum over those edges (u, v) of |N+(u)| + |N+(v)|: the adjacency
 *             entries that a merge of the two full lists reads (4 bytes each)
 * Edges whose source has |N+(u)| < 2 and whose target is not a hub have an empty
 * intersection and are reported in edges[TC_NUM_BUCKETS] (arrays hold
 * TC_NUM_BUCKETS + 1 entries).  Runs the planner if needed; synchronises the
 * stream; not meant for timed regions.
 */
tc_status tc_graph_plan_stats(tc_graph* g, int64_t* edges, int64_t* ids);

/*
 * Batches: G independent graphs in one object (an addition of this library; the
 * paper has no counterpart).  Graph g has n[g] vertices with local ids
 * [0, n[g]) and the pairs src/dst[edge_off[g] .. edge_off[g+1]).  The batch is
 * counted as one disjoint union: vertex (g, i) becomes union id vbase[g] + i with
 * vbase[g] = n[0] + ... + n[g-1].  t[] and LCC[] from lcc_compute on a batch are
 * indexed by union id (graph after graph); T per graph comes from tc_batch_count.
 *   G           number of graphs (>= 0)
 *   n, edge_off HOST arrays of G and G + 1 entries; edge_off[0] == 0, non-decreasing;
 *               sum of n and edge_off[G] at most 2^31 - 1
 *   src, dst    edge_off[G] int32 local ids each, in mem_kind memory
 * Ids outside [0, n[g]) are reported by tc_batch_count (TC_EINVAL); creation
 * itself does not wait for the device after copying the host arrays.
 */
tc_status tc_batch_create(int32_t G, const int32_t* n, const int64_t* edge_off, const int32_t* src,
                          const int32_t* dst, int mem_kind, void* cuda_stream, tc_graph** out);

/* T of every graph of a batch: T_out[G] (uint64) in mem_kind memory.  Runs the
   count if needed; synchronises the stream.  Errors: TC_EINVAL (not a batch, NULL,
   an id outside its graph), TC_ECUDA, TC_EINTERNAL. */
tc_status tc_batch_count(tc_graph* g, uint64_t* T_out, int mem_kind);

/* Number of graphs of a batch (TC_EINVAL for a single graph). */
tc_status tc_batch_size(const tc_graph* g, int32_t* G);

/*
 * Tuning of the intersection: strategy and Eq. 3 factor per bucket, and the hub
 * selection (min_degree, max hubs) and block-versus-warp split of hubs (hubs with
 * in-degree >= hub_big_in get a whole thread block, the others one warp).
 * hub_core: the highest min(hub_core, hubs, 8192) ranks form a dense core whose
 * triangles are counted by bit-parallel row intersections (every out-neighbour of a
 * core vertex lies in the core); 0 turns the core off.  Default 8192.
 */
typedef struct tc_tuning {
    int32_t strategy[TC_NUM_BUCKETS];
    double factor[TC_NUM_BUCKETS];
    int32_t hub_min_degree;
    int32_t hub_max;
    int32_t hub_big_in;
    int32_t hub_core;
} tc_tuning;

tc_status tc_graph_get_tuning(const tc_graph* g, tc_tuning* out);
/* Errors: TC_EINVAL for values the buckets cannot run (as tc_graph_set_strategy). */
tc_status tc_graph_set_tuning(tc_graph* g, const tc_tuning* t);

/*
 * Autotuner: times the bucket kernels of g under candidate settings (hub threshold
 * and block/warp split first, then each bucket's strategy, chosen per bucket from
 * its own kernel time), applies the fastest and writes it to *out (may be NULL).
 * Results are cached in the process by a signature of the planned work (edges and
 * list lengths per bucket, rounded to powers of two); a graph with a cached
 * signature gets the cached setting without trials unless force != 0.  Runs the
 * count several times; synchronises the stream.
 */
tc_status tc_graph_autotune(tc_graph* g, int32_t force, tc_tuning* out);

/*
 * One call for a whole batch with device buffers: create, count, per-graph T,
 * t[] and LCC[] (union ids), release.  src, dst, T_out (uint64[G]), t_out
 * (uint64[sum n], may be NULL) and lcc_out (fp64[sum n], may be NULL) are DEVICE
 * pointers; n and edge_off are host arrays as in tc_batch_create.  tuning may be
 * NULL (defaults).  With flags & TC_RUN_GRAPH the device work is recorded once
 * into a CUDA graph (cuda_stream must then not be NULL) and replayed by later calls
 * with the same sizes, buffers and tuning; the library keeps the recorded graph and
 * two small arrays per distinct call until tc_release_cached_graphs.  Synchronises
 * the stream (to report errors).  Errors: as tc_batch_create / tc_batch_count.
 */
enum { TC_RUN_GRAPH = 1 };
tc_status tc_batch_run(int32_t G, const int32_t* n, const int64_t* edge_off, const int32_t* src,
                       const int32_t* dst, uint64_t* T_out, uint64_t* t_out, double* lcc_out,
                       const tc_tuning* tuning, void* cuda_stream, int flags);

/* Frees the CUDA graphs and arrays kept by tc_batch_run. */
void tc_release_cached_graphs(void);

/*
 * Device-side generation of the synthetic inputs of the serving stream (an
 * addition of this library; the paper's graphs come from files).  Writes m pairs
 * (device memory) of an R-MAT graph (a, b, c) = (0.57, 0.19, 0.19) over n vertices
 * (scale ceil(log2 n), endpoints >= n redrawn) or m uniform pairs with
 * replacement, from the counter-based SplitMix64 stream (seed, stream_id); the
 * host generator of the test suite produces the same pairs.  Stream-ordered.
 */
enum { TC_GEN_RMAT = 0, TC_GEN_ER_REPLACE = 1 };
tc_status tc_generate_edges(int kind, int32_t n, int64_t m, uint64_t seed, uint64_t stream_id, int32_t* src,
                            int32_t* dst, void* cuda_stream);

/*
 * Serving (an addition of this library; the paper has no counterpart): a request
 * loop that accepts TC/LCC jobs on graphs of different sizes as they arrive.
 * `slots` worker threads, each with its own CUDA stream on the device current at
 * start, take the oldest waiting request as soon as they are free and the device
 * memory budget admits it (estimate 48 m + 160 n bytes + 16 MiB per request), so
 * requests arriving while others run are admitted as slots and memory free up and
 * their work overlaps on the device.  A request larger than the whole budget runs
 * alone.  Each request's graph is generated on the device (tc_generate_edges),
 * counted through this ABI and released; the result carries T, the number of
 * distinct edges, order-independent checksums of t[] and LCC[] (sum over v of
 * SplitMix64-mix(v * 0x9e3779b97f4a7c15 ^ x_v), x_v = t[v] or the bits of LCC[v]),
 * and timestamps in seconds on the server's steady clock.
 */
typedef struct tc_server tc_server;
typedef struct tc_request {
    int64_t id;          /* caller's id, returned with the result */
    int32_t kind;        /* TC_GEN_RMAT or TC_GEN_ER_REPLACE */
    int32_t n;           /* vertices */
    int64_t m;           /* generated pairs */
    uint64_t seed;
    uint64_t stream_id;
} tc_request;
typedef struct tc_result {
    int64_t id;
    int32_t status;      /* tc_status of the request */
    int32_t slot;        /* worker that ran it */
    uint64_t T;
    int64_t m_simple;
    uint64_t t_hash;
    uint64_t lcc_hash;
    double submit_s, start_s, end_s;
    uint64_t bytes;      /* admission estimate */
} tc_result;
typedef struct tc_server_stats {
    int32_t slots;
    uint64_t budget_bytes;
    uint64_t submitted, completed, running, queued, max_queue;
    uint64_t peak_bytes, in_flight_bytes;  /* admitted estimates */
    double clock_s;
} tc_server_stats;

tc_status tc_server_start(uint64_t hbm_budget_bytes, int32_t slots, tc_server** out);
/* Queues a request (non-blocking).  TC_EBUSY after tc_server_stop began. */
tc_status tc_server_submit(tc_server* s, const tc_request* r);
/* Moves up to max finished results into out (non-blocking); *count receives how many. */
tc_status tc_server_poll(tc_server* s, tc_result* out, int32_t max, int32_t* count);
/* Waits until at least `completed` requests have finished (TC_ETIMEOUT after timeout_s). */
tc_status tc_server_wait(tc_server* s, int64_t completed, double timeout_s);
tc_status tc_server_get_stats(tc_server* s, tc_server_stats* out);
/* Stops accepting, finishes every queued request, joins the workers, frees s. */
tc_status tc_server_stop(tc_server* s);
/*
 * One request alone on the caller's stream: the plain per-graph path that the serving
 * loop is measured against.  Generates the request's graph on the device, builds it,
 * counts T, t[] and LCC[] (tc_graph_create_from_edges, tc_count, lcc_compute) and
 * releases it; *out gets the fields a served request's result has (T, m_simple and
 * the checksums of t[] and LCC[]; status in out->status; end_s = seconds the call
 * took, submit_s = start_s = 0).  Synchronises the stream.  Errors: TC_EINVAL for a
 * NULL pointer or a bad request, TC_ECUDA.
 */
tc_status tc_request_run(const tc_request* r, void* cuda_stream, tc_result* out);

/*
 * Count without allocating (an addition of this library; the paper has no
 * counterpart).  For callers that cannot allocate device memory while they run: a
 * program that has handed all free HBM to its own caching allocator, or real-time
 * code that forbids allocation after start-up.
 *
 * Computes the same T, t[] and LCC[] as tc_graph_create_from_edges + tc_count +
 * lcc_compute for a small graph, in one kernel launch whose intermediate arrays
 * live in a fixed device array of TC_NOALLOC_SCRATCH_BYTES bytes inside the
 * library.  Every GPU that loads the library holds that array until the process
 * exits.  The call itself allocates nothing and calls no allocating routine.
 *   n, m        0 <= n <= TC_NOALLOC_MAX_N, 0 <= m <= TC_NOALLOC_MAX_M
 *   src, dst    m int32 ids each, DEVICE memory (may be NULL when m == 0)
 *   T_out       host scalar, receives T
 *   t_out       n uint64 in device memory, or NULL
 *   lcc_out     n fp64 in device memory, or NULL
 *   cuda_stream a cudaStream_t (as void*), or NULL; the call copies its status words
 *               to the host and synchronises this stream before it returns
 * The first call on a device looks up the device address of the array (once per
 * device, with that device current); make that first call before any stream
 * capture begins.  With lazy module loading (the CUDA default) that first call is
 * also when the runtime loads this library's device code and places the array on
 * the device, so make it at start-up, before the free memory is handed to another
 * allocator.  All calls share the array and it keeps the previous call's contents
 * (the kernel clears what it needs): calls whose work overlaps on the GPU (other
 * streams or host threads) race on it and must be ordered by the caller.
 * Errors: TC_EINVAL for sizes beyond the limits, NULL pointers or an id outside
 * [0, n); TC_ECUDA; TC_EINTERNAL.
 */
#define TC_NOALLOC_MAX_N 16384
#define TC_NOALLOC_MAX_M 262144
#define TC_NOALLOC_SCRATCH_BYTES 3735688
tc_status tc_count_noalloc(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, uint64_t* T_out,
                           uint64_t* t_out, double* lcc_out, void* cuda_stream);

/* Number of kernels this library has launched in the process so far (all devices). */
uint64_t tc_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
