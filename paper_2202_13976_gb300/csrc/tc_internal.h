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
    unsigned int warp_count;       // planner: vertices in the warp bucket
    unsigned int cta_count;        // planner: vertices in the block bucket
    unsigned int long_count;       // build: rows sorted by whole blocks
    unsigned int work_next;        // dynamic work counter of the block bucket
    unsigned int pad[6];
};

struct Launch {
    cudaStream_t stream;
    int sms;  // multiprocessors of the device
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
    void* tmp;            // max(scan_tmp_bytes(n + 1), radix_tmp_bytes(n))
    // outputs (kept by the graph)
    int32_t* rank;        // n: rank of each input id in (degree, id) order
    int64_t* rowstart;    // n + 1 (rank space)
    int32_t* rowlen;      // n: oriented out-degree after deduplication
    int32_t* col;         // m: oriented adjacency (rank space), rows sorted
    int32_t* deg;         // n: simple-graph degree (rank space)
    DevStats* stats;
};

void launch_check_offsets(const int64_t* offsets, int32_t n, int64_t limit, DevStats* stats,
                          const Launch& L);
void launch_expand_csr(const int64_t* offsets, int32_t n, int32_t* rows, DevStats* stats,
                       const Launch& L);
void launch_canon_degree(const BuildBuffers& B, const Launch& L);
void launch_rank(const BuildBuffers& B, int deg_bits, const Launch& L);
void launch_orient(const BuildBuffers& B, const Launch& L);
cudaError_t build_init_attributes();

// ---- plan + intersect + finalize (tc_intersect.cu) ---------------------------
struct Strategy {
    int strat[TC_NUM_BUCKETS];
    float factor[TC_NUM_BUCKETS];
};

struct CountBuffers {
    int32_t n;
    const int64_t* rowstart;
    const int32_t* rowlen;
    const int32_t* col;
    int32_t* warp_list;   // n
    int32_t* cta_list;    // n
    unsigned long long* t_rank;  // n
    DevStats* stats;
};

void launch_plan(const CountBuffers& C, const Launch& L);
cudaError_t intersect_init_attributes();
// Runs both bucket kernels; events (may be null) bracket each for timing.
void launch_intersect(const CountBuffers& C, const Strategy& S, cudaEvent_t ev[3], const Launch& L);
void launch_sum_t(const CountBuffers& C, const Launch& L);
void launch_finalize(int32_t n, const int32_t* rank, const unsigned long long* t_rank,
                     const int32_t* deg, unsigned long long* t_out, double* lcc_out,
                     const Launch& L);

inline int grid_for(int64_t work, int threads, int sms, int per_sm = 8) {
    int64_t g = (work + threads - 1) / threads;
    int64_t cap = (int64_t)sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace tcg
