// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tc.h"

namespace tcg {

// Device-side error flags (bit set by kernels, read by the host).
enum : int {
    ERR_BAD_ID = 1,        // a vertex id outside [0, n)
    ERR_BAD_OFFSETS = 2,   // CSR offsets decreasing or out of range
    ERR_OVERFLOW = 4,      // a count exceeded its storage
};

// Small device-resident record of one build / count (one allocation).
struct DevStats {
    unsigned long long loops;      // self-loops dropped
    unsigned long long m_simple;   // distinct undirected edges
    unsigned long long sum_t;      // sum over v of t(v)
    unsigned int max_deg;          // largest multigraph degree
    int err;                       // ERR_* flags
    unsigned int long_count;       // build: rows sorted by whole blocks
    unsigned int small_count[4];   // planner: vertices per small-list class (d+ <= 8, 16, 32, 256)
    unsigned int cta_count;        // planner: vertices with d+ > 32
    unsigned int cta_next;         // dynamic work counter of the block push kernel
    unsigned int hub_count;        // vertices staged as hubs (ranks n - hub_count .. n-1)
    unsigned int hub_next;         // dynamic work counter of the hub kernel (big hubs)
    unsigned int hub_next2;        // dynamic work counter of the hub kernel (medium hubs)
    unsigned int hub_candidates;   // vertices whose degree reaches the hub threshold
    unsigned int hub_big;          // hubs processed by whole blocks
    unsigned int mid_count;        // build: rows of 17..256 entries sorted by one warp
    unsigned int mid2_count;       // build: rows of 257..1024 entries sorted by one warp
    unsigned int core_n;           // planner: dense core size (ranks n - core_n .. n-1)
    unsigned int pad[1];
};
static_assert(sizeof(DevStats) == 96, "DevStats layout");

struct Launch {
    cudaStream_t stream;
    int sms;  // multiprocessors of the device
};

// The simple undirected graph of a pair list, built by the same path as
// tc_graph_create_from_edges (used by the directed count, whose triangles are those
// of this graph): vertices ranked by (degree, id), oriented rows N+(u) in rank space.
struct UndirectedRows {
    int64_t m_simple, loops;
    const int32_t* rank;    // n: the rank of each vertex id
    const int2* rowinfo;    // n, by rank: {first entry of the row in col, entries}
    const int32_t* rowlen;  // n, by rank: entries of the row
    const int32_t* col;     // the rows' entries (ranks), ascending within each row
};
// Builds it on `stream` from device pairs; *g receives the graph object that holds
// the rows (the caller destroys it).  Synchronises the stream to read the sizes.
// With dir_bits (n <= 2^29) every entry is (rank << 2) | direction bit of its pair
// (BuildBuffers::dir_bits): a pair read in both directions leaves two neighbouring
// entries, and m_simple counts entries, not edges.
tc_status build_undirected_rows(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, cudaStream_t stream,
                                bool dir_bits, tc_graph** g, UndirectedRows* out);

// A second stream for work that does not depend on what the main stream does next:
// it starts after `fork` is recorded on the main stream and records `join` when its
// part is done, which the main stream waits for before it uses the results.  The
// planner builds the hub in-edge lists and the dense core there while the main
// stream lists and counts the push buckets; the build sorts the rows of 257 entries
// or more there while the main stream sorts the rows of 17..256.
struct PlanStreams {
    cudaStream_t side;
    cudaEvent_t fork, join;
};

// ---- primitives (tc_prims.cu) ------------------------------------------------
// Exclusive scan of `count` uint32 values into int64 (out has count + 1 entries;
// out[count] = total).  `tmp` needs scan_tmp_bytes(count) bytes.
size_t scan_tmp_bytes(int64_t count);
void scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t count, void* tmp, const Launch& L);
// Exclusive scan of uint32 in place-capable (out may equal in); out[count] = total.
void scan_u32_to_u32(const uint32_t* in, uint32_t* out, int64_t count, void* tmp, const Launch& L);

// Stable LSD radix sort of uint64 keys on bits [lo, hi).  keys and alt are two
// buffers of `count`; returns the buffer holding the result.  `tmp` needs
// radix_tmp_bytes(count) bytes.
size_t radix_tmp_bytes(int64_t count);
uint64_t* radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t count, int lo, int hi, void* tmp,
                         const Launch& L);

// ---- build (tc_build.cu) -----------------------------------------------------
struct BuildBuffers {
    // inputs
    const int32_t* src;
    const int32_t* dst;
    int64_t m;
    int32_t n;
    // scratch
    uint32_t* dmulti;     // n
    uint64_t* keys;       // n
    uint64_t* keys_alt;   // n
    uint32_t* rowcnt;     // n + 1
    uint32_t* cursor;     // n
    int32_t* longlist;    // n
    int32_t* midlist;     // n: rows of 17..256 entries
    int32_t* midlist2;    // n: rows of 257..1024 entries
    uint32_t* dupin;      // n: repeated entries dropped at each target
    uint32_t* bcount;     // BUCKET_MAX + 1: pairs per source bucket
    uint32_t* bcur;       // BUCKET_MAX: bucket cursors of the partition pass
    int64_t* bstart;      // BUCKET_MAX + 1: first pair of each bucket
    int2* pairs;          // m: (source rank, target rank) grouped by bucket
    int2* oriented;       // m: (source rank, target rank) in input order ((-1, -1): no entry)
    bool bucket_fill;     // rows counted and filled by source buckets (flat degree distributions)
    // directed input (tc_directed_lcc): every entry is (target rank << 2) | direction
    // bit of its pair (1: source rank below target rank, 2: above), so a pair read in
    // both directions leaves two entries; repeats are dropped as usual, but not
    // counted into the degrees (they are not used then).  Needs n <= 2^29.
    bool dir_bits;
    // batches: vertices are ranked within their own graph (graph, degree, id), so each
    // graph keeps a contiguous block of ranks and rows; seg_vbase null for one graph
    const int32_t* seg_vbase;  // G + 1: first union id of every graph
    int32_t seg_count;         // G
    int seg_bits, seg_deg_bits, local_bits;  // key fields: graph, degree within a graph, local id
    void* tmp;            // max(scan_tmp_bytes(n + 1), radix_tmp_bytes(n))
    // outputs (kept by the graph)
    int32_t* rank;        // n: rank of each input id in (degree, id) order
    int64_t* rowstart;    // n + 1 (rank space)
    int32_t* rowlen;      // n: oriented out-degree after deduplication
    int2* rowinfo;        // n: {first index in col, rowlen} (rank space)
    int32_t* col;         // m: oriented adjacency (rank space), rows sorted
    int32_t* deg;         // n: simple-graph degree (rank space)
    DevStats* stats;
};

// Build phases timed by events (tc_graph_build_timing): ingest, rank, row counts,
// row fill, row sort + dedup, degrees.
enum { BP_START = 0, BP_INGEST, BP_RANK, BP_COUNT, BP_FILL, BP_SORT, BP_END, BP_EVENTS };

void launch_check_offsets(const int64_t* offsets, int32_t n, int64_t limit, DevStats* stats,
                          const Launch& L);
void launch_expand_csr(const int64_t* offsets, int32_t n, int32_t* rows, DevStats* stats,
                       const Launch& L);
void launch_canon_degree(const BuildBuffers& B, const Launch& L);
// The same in pieces: the degree counts of pairs [first, first + count), then the
// maximum degree once all pieces are in.
void launch_canon_degree_part(const BuildBuffers& B, int64_t first, int64_t count, const Launch& L);
void launch_max_deg(const BuildBuffers& B, const Launch& L);
void launch_rank(const BuildBuffers& B, int deg_bits, const Launch& L);
void launch_orient(const BuildBuffers& B, const Launch& L, cudaEvent_t* ev = nullptr, const PlanStreams* ps = nullptr);
// Row fill by source buckets: at most BUCKET_MAX buckets of at most BUCKET_ROWS_MAX
// rows (2^BUCKET_BITS buckets when that fits); nb = 0 selects the direct fill.
constexpr int BUCKET_BITS = 11;
constexpr int BUCKET_MAX = 8192;
constexpr int BUCKET_ROWS_MAX = 32768;
void bucket_shape(int32_t n, int* shift, int* nb);
cudaError_t build_init_attributes();

// ---- plan + intersect + finalize (tc_intersect.cu) ---------------------------
// Buckets (include/tc.h): small lists (push, lane per edge), large lists (push,
// block per source vertex), hubs (pull, block per staged hub list).
struct Strategy {
    int strat[TC_NUM_BUCKETS];
    float factor[TC_NUM_BUCKETS];
    int hub_min_degree;   // vertices of degree >= this are hub candidates (<= 0: no hubs)
    int hub_max;          // at most this many hubs (the highest ranks)
    int hub_big_in;       // hubs with at least this in-degree get a whole block (else one warp)
    int hub_core;         // the highest min(hub_core, hubs, CORE_MAX) ranks form the dense core (0: none)
};

// Capacity of the hub kernel's shared-memory bitmap (ranks above the hub).
constexpr int HUB_BM_BITS = 131072;
// Largest dense core (tc_core.cu): one core_n x core_n bit matrix.
constexpr int CORE_MAX = 8192;

struct CountBuffers {
    int32_t n;
    const int64_t* rowstart;
    const int32_t* rowlen;
    const int2* rowinfo;     // {first index in col, length} per row
    const int32_t* col;
    const int32_t* deg;
    int32_t* small_list[4];  // n each: d+ <= 8, 16, 32, 256
    int32_t* cta_list;       // n
    // hub in-edges (transpose of the oriented edges that point into the hub ranks)
    int32_t hub_cap;         // min(n, HUB_BM_BITS): slots for ranks n - hub_cap .. n-1
    uint32_t* hub_cnt;       // hub_cap + 1
    int64_t* hub_start;      // hub_cap + 1
    uint32_t* hub_cur;       // hub_cap + 1
    unsigned long long* hub_cur64;  // hub_cap + 1: next free slot of every hub's segment (planner)
    int32_t* big_list;       // hub_cap: big hubs, highest rank first
    int32_t* med_list;       // hub_cap: the other hubs, highest rank first
    int4* in_rec;            // m: in-edge {u, first suffix entry, end of N+(u), 0} (indices into col)
    int32_t* rowof;          // m: source row of each entry of the non-core rows
    int64_t m_cap;           // entries of col (and of in_rec, rowof)
    void* tmp;               // scan scratch, scan_tmp_bytes(hub_cap + 1)
    // dense core (tc_core.cu): bit rows of core_words words for core indices 0 .. core_cap-1
    int32_t core_cap;        // min(hub_cap, CORE_MAX)
    int32_t core_words;      // core_words_for(core_cap)
    uint32_t* core_z;        // core_cap * core_words: symmetric adjacency rows; followed by core_cnt
    uint32_t* core_cnt;      // core_cap: in-degree from the core
    int32_t* core_lo;        // core_cap: lowest core neighbour
    int32_t* core_hi;        // core_cap: highest core neighbour (-1: none)
    int32_t* core_hiout;     // core_cap: highest core out-neighbour (-1: none)
    unsigned long long* t_rank;  // n
    DevStats* stats;
    uint32_t* sup;           // null, or m_cap per-edge supports indexed like col (tc_edge_support)
    int32_t src_lo, src_hi;  // only triangles whose lowest vertex has a rank in [src_lo, src_hi) are counted
    cudaEvent_t hub_ready;   // null, or recorded once the hub lists and the dense core are built (PlanStreams)
};


enum { PH_PLAN = 0, PH_SMALL, PH_CTA, PH_HUB, PH_END, PH_EVENTS };

// Builds the bucket lists and the hub in-edge lists; with ps, the hub part runs on
// ps->side.  Returns whether it did (the count must then wait for ps->join).
bool launch_plan(const CountBuffers& C, const Strategy& S, const Launch& L, const PlanStreams* ps = nullptr);
// Shards of the sources (tc_vertex.cu): cost[u] = d+(u) (d+(u) + 1) / 2 + 1 (saturated),
// then the rank range [bounds[0], bounds[1]) of shard `shard` of `nshards`, cut where
// the prefix of the cost crosses shard / nshards of the total.  cost needs n entries,
// prefix n + 1, tmp scan_tmp_bytes(n).
void launch_shard_bounds(int32_t n, const int32_t* rowlen, uint32_t* cost, int64_t* prefix, void* tmp, int32_t shard,
                         int32_t nshards, int32_t* bounds, const Launch& L);
// LCC (Eq. 2) of every vertex id from per-id triangle counts t (the sum of the shards').
void launch_lcc_from_counts(int32_t n, const int32_t* rank, const int32_t* deg, const unsigned long long* t,
                            double* lcc_out, const Launch& L);
// Dense core (tc_core.cu): bit matrices after the hub count is known, and the count.
int core_words_for(int32_t core_cap);
void launch_core_plan(const CountBuffers& C, const Launch& L);
void launch_core_count(const CountBuffers& C, const Launch& L);
cudaError_t intersect_init_attributes();
// Runs the three bucket kernels; ev (may be null) holds PH_EVENTS events.
void launch_intersect(const CountBuffers& C, const Strategy& S, cudaEvent_t* ev, const Launch& L);
void launch_sum_t(const CountBuffers& C, const Launch& L);
void launch_finalize(int32_t n, const int32_t* rank, const unsigned long long* t_rank,
                     const int32_t* deg, unsigned long long* t_out, double* lcc_out,
                     const Launch& L);

// ---- per-vertex formula (tc_vertex.cu) -------------------------------------------
struct VertexFormulaBuffers {
    int32_t n;
    int64_t m;               // oriented entries (distinct edges)
    int64_t m_cap;           // entries of col, including slots freed by deduplication
    const int64_t* rowstart;
    const int32_t* rowlen;
    const int2* rowinfo;
    const int32_t* col;
    const int32_t* deg;      // simple degree (rank space)
    uint32_t* indeg;         // n
    int64_t* sym_start;      // n + 1
    int64_t* instart;        // n + 1
    int32_t* sym;            // 2 m: symmetric rows, ascending
    uint64_t* keys;          // m_cap
    uint64_t* keys_alt;      // m_cap
    void* radix_tmp;         // radix_tmp_bytes(m_cap)
    void* tmp;               // scan_tmp_bytes(n + 1)
    unsigned long long* t;   // n (rank space)
    unsigned* counter;
    unsigned long long* sum;
};
int vf_key_bits(int32_t n);
void launch_symmetric_rows(const VertexFormulaBuffers& V, const Launch& L);
void launch_vertex_formula(const VertexFormulaBuffers& V, const Launch& L);
// Per-edge supports recorded by the count (sup, indexed like col) written out as the
// edge list {u, v, support} in the caller's ids, row by row in rank order; id_of (n),
// estart (n + 1) and scan_tmp (scan_tmp_bytes(n + 1)) are scratch.
void launch_support_out(int32_t n, const int32_t* rank, const int32_t* rowlen, const int2* rowinfo, const int32_t* col,
                        const uint32_t* sup, int32_t* id_of, int64_t* estart, void* scan_tmp, int32_t* eu, int32_t* ev,
                        uint32_t* support, const Launch& L);

// ---- remote reads and caches of the 1D partition (tc_cache.cu) -------------------
struct PartCounters {  // per process; four 64-bit fields, nothing else (indexed as such)
    unsigned long long reads, top_reads, distinct, read_bytes;
};
static_assert(sizeof(PartCounters) == 32, "PartCounters layout");

// Cells of the shared-memory hit histogram (2 LRU caches x processes x capacities).
constexpr int RC_HIST_SHARED = 3072;
// Hit count a score simulation reports when its state broke an invariant.
constexpr unsigned long long RC_SIM_BROKEN = ~0ull;
// Largest bitmap set of one score simulation kept in shared memory.
constexpr size_t RC_SIM_SHARED_MAX = 200 * 1024;

struct RemoteCacheBuffers {
    int32_t n, parts, ncap;
    int64_t ms2;                 // symmetric entries (2 m)
    const int32_t* rank;         // graph: id -> rank
    const int64_t* rowstart;     // graph: oriented rows (rank space)
    const int32_t* rowlen;
    const int32_t* col;
    const int32_t* deg;          // graph: simple degree (rank space)
    const uint64_t* caps;        // ncap capacities in bytes, ascending (device)
    // stream phase
    int32_t* id_of;              // n
    uint32_t* sdeg;              // n: simple degree per id
    int32_t* prank;              // n: position in (degree, id) order
    uint64_t* vkeys;             // n
    uint64_t* vkeys_alt;         // n
    const uint64_t* vsorted;     // set by launch_rc_stream: (degree << b) | id in score order
    int64_t* estart;             // n + 1
    uint64_t* keys;              // ms2 (later: N item keys, then N score keys)
    uint64_t* keys_alt;          // ms2
    uint32_t* flag;              // ms2
    uint32_t* pos;               // ms2 + 1
    int32_t* item;               // ms2 (N used)
    int32_t* part;               // ms2 (N used)
    PartCounters* pc;            // parts
    void* radix_tmp;             // radix_tmp_bytes(max(ms2, n))
    void* scan_tmp;              // scan_tmp_bytes(max(ms2, n) + 1)
    // LRU caches (N reads)
    int64_t* prev;               // N
    int64_t* pstart;             // parts + 1
    uint32_t *key_lru, *wdeg;    // N each
    int64_t* q_lru;              // N
    uint32_t* th_lru;            // N
    int64_t* e0deg;              // N + 1
    uint32_t* lk;                // rc_levels(N) * N: the tree's keys, level RC_LOW + j at j * N
    int64_t* le;                 // rc_levels(N) * (N + 1): prefix sums of each level's entry sizes
    uint32_t* la[2];             // N each: entry sizes of the current and the next level
    int64_t *f_lru_deg, *f_lru_one;  // N each
    unsigned long long *cnt, *byt;   // 2 * parts * ncap each (adjacency, offsets)
    // score caches (N reads)
    uint64_t* ukeys;             // N: distinct (process << b | score position) keys, sorted
    uint32_t* udeg;              // N: degree of the entry of each distinct key
    int64_t* ubase;              // parts + 1: first distinct key of each process
    int32_t* lr;                 // N: score rank of each read's entry within its process
    uint32_t* sim_state;         // bitmaps of every simulation when they exceed shared memory
    unsigned long long *sc_cnt, *sc_byt;  // 2 * parts * ncap each (adjacency, offsets)
};
int rc_key_bits(int32_t n);
// Levels of the merge-sort tree kept for N reads (levels 5 .. floor(log2 N)).
int rc_levels(int64_t N);
// The read stream (N = pos[ms2] reads), then, once N is known, the LRU caches and the
// score ranks; then, once the largest count of distinct entries of a process is known,
// the score simulations.
void launch_rc_stream(RemoteCacheBuffers& R, const Launch& L);
void launch_rc_caches(const RemoteCacheBuffers& R, int64_t N, const Launch& L);
struct RcSimShape {
    uint32_t W1, W2;      // words of the two bitmap levels
    size_t bytes;         // per simulation
    bool shared;          // bitmaps in shared memory (else sim_state, bytes per job)
};
RcSimShape rc_sim_shape(int64_t max_distinct);
void launch_rc_score(const RemoteCacheBuffers& R, const RcSimShape& S, const Launch& L);

// ---- batch (tc_batch.cu) -------------------------------------------------------
void launch_batch_relabel(int32_t G, const int64_t* edge_off, const int32_t* vbase, const int32_t* src,
                          const int32_t* dst, int32_t* usrc, int32_t* udst, int* err, const Launch& L);
void launch_run_status(const DevStats* stats, const int* batch_err, int* status, const Launch& L);
void launch_batch_T(int32_t G, const int32_t* vbase, const int32_t* rank, const unsigned long long* t_rank,
                    unsigned long long* T_out, int* err, const Launch& L);

// ---- device generators (tc_gen.cu) and serving (tc_serve.cu, tc_api.cu) ---------
cudaError_t launch_generate(int kind, int32_t n, int64_t m, unsigned long long seed, unsigned long long stream_id,
                            int32_t* src, int32_t* dst, const Launch& L);
// The library's stream-ordered pool of a device (initialising the device state).
cudaMemPool_t device_pool(int dev);
// Device memory a serving request is admitted with.
uint64_t serve_estimate_bytes(int32_t n, int64_t m);

// Records "where: CUDA error text" for tc_last_error_detail on this thread.
void set_last_error(const char* where, cudaError_t e);

// Kernel launch accounting (tc_launch_count).
void count_launch(int k = 1);
uint64_t launch_total();

void launch_plan_stats(const CountBuffers& C, unsigned long long* out /* 2*TC_NUM_BUCKETS+1 */,
                       const Launch& L);

inline int grid_for(int64_t work, int threads, int sms, int per_sm = 8) {
    int64_t g = (work + threads - 1) / threads;
    int64_t cap = (int64_t)sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace tcg
