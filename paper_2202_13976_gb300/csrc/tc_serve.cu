// Serving loop: requests for T / t[] / LCC on graphs of different sizes arrive over
// time; each is generated on the device, counted through the C ABI and released.
//
// Continuous batching on streams: `slots` worker threads, each with its own CUDA
// stream, take the oldest waiting request as soon as they are free and the HBM
// budget has room for it (admission by an estimate of the request's device
// memory), so requests that arrive while others run are admitted as slots and
// memory free up and their kernels overlap on the device.  A request larger than
// the whole budget runs only when nothing else is in flight.  Latency is measured
// from submission to the moment the result is on the host.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {
namespace {

__device__ __forceinline__ unsigned long long h_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Order-independent checksums of the outputs: sum over v of mix(v * gamma ^ x_v).
__global__ void k_checksum(int32_t n, const unsigned long long* __restrict__ t, const double* __restrict__ lcc,
                           unsigned long long* __restrict__ out) {
    unsigned long long a = 0, b = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const unsigned long long key = (unsigned long long)v * 0x9e3779b97f4a7c15ull;
        a += h_mix(key ^ t[v]);
        b += h_mix(key ^ (unsigned long long)__double_as_longlong(lcc[v]));
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane_id() == 0) {
        atomicAdd(&out[0], a);
        atomicAdd(&out[1], b);
    }
}

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

uint64_t serve_estimate_bytes(int32_t n, int64_t m) {
    // peak of one request: its pairs and outputs, the graph (CSR, hub in-edges and
    // source rows 24 m, per-vertex arrays), the build scratch (pairs 16 m) and the core
    return (uint64_t)(48 * m + 160 * (int64_t)n) + (16ull << 20);
}

}  // namespace tcg

using namespace tcg;

struct tc_server {
    int device = 0;
    int sms = 0;
    cudaMemPool_t pool = nullptr;
    uint64_t budget = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::pair<tc_request, double>> queue;  // request, submit time
    std::vector<tc_result> done;                      // finished, not yet polled
    std::vector<std::thread> workers;
    bool stopping = false;
    uint64_t in_flight = 0;
    tc_server_stats stats{};
};

namespace {

void run_one(cudaMemPool_t pool, int sms, cudaStream_t stream, const tc_request& r, tc_result* out) {
    out->status = TC_OK;
    const size_t n = (size_t)r.n;
    Launch L{stream, sms};
    int32_t *src = nullptr, *dst = nullptr;
    unsigned long long* t = nullptr;
    double* lcc = nullptr;
    unsigned long long* sums = nullptr;
    tc_graph* g = nullptr;
    cudaError_t e = cudaSuccess;
    unsigned long long h[2] = {0, 0};
    int64_t m_simple = 0;
    auto fail = [&](tc_status st) { out->status = st; };
    do {
        const size_t me = r.m > 0 ? (size_t)r.m : 1;
        if ((e = cudaMallocFromPoolAsync((void**)&src, 4 * me, pool, stream)) != cudaSuccess ||
            (e = cudaMallocFromPoolAsync((void**)&dst, 4 * me, pool, stream)) != cudaSuccess ||
            (e = cudaMallocFromPoolAsync((void**)&t, 8 * (n ? n : 1), pool, stream)) != cudaSuccess ||
            (e = cudaMallocFromPoolAsync((void**)&lcc, 8 * (n ? n : 1), pool, stream)) != cudaSuccess ||
            (e = cudaMallocFromPoolAsync((void**)&sums, 16, pool, stream)) != cudaSuccess) {
            cudaGetLastError();
            fail(TC_ENOMEM);
            break;
        }
        if ((e = launch_generate(r.kind, r.n, r.m, r.seed, r.stream_id, src, dst, L)) != cudaSuccess) {
            fail(TC_ECUDA);
            break;
        }
        tc_status st = tc_graph_create_from_edges(r.n, r.m, src, dst, TC_MEM_DEVICE, stream, &g);
        if (st != TC_OK) {
            fail(st);
            break;
        }
        if ((st = tc_count(g, &out->T)) != TC_OK || (st = lcc_compute(g, reinterpret_cast<uint64_t*>(t), lcc, TC_MEM_DEVICE)) != TC_OK ||
            (st = tc_graph_info(g, &m_simple, nullptr, nullptr)) != TC_OK) {
            fail(st);
            break;
        }
        cudaMemsetAsync(sums, 0, 16, stream);
        k_checksum<<<grid_for(r.n, 256, sms), 256, 0, stream>>>(r.n, t, lcc, sums);
        count_launch();
        if ((e = cudaMemcpyAsync(h, sums, 16, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(stream)) != cudaSuccess) {
            fail(TC_ECUDA);
            break;
        }
    } while (false);
    if (g) tc_graph_destroy(g);
    if (src) cudaFreeAsync(src, stream);
    if (dst) cudaFreeAsync(dst, stream);
    if (t) cudaFreeAsync(t, stream);
    if (lcc) cudaFreeAsync(lcc, stream);
    if (sums) cudaFreeAsync(sums, stream);
    cudaStreamSynchronize(stream);
    out->m_simple = m_simple;
    out->t_hash = h[0];
    out->lcc_hash = h[1];
}

void worker_main(tc_server* s, int slot) {
    cudaSetDevice(s->device);
    cudaStream_t stream = nullptr;
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    for (;;) {
        tc_request r;
        double submit = 0;
        uint64_t bytes = 0;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            for (;;) {
                if (!s->queue.empty()) {
                    bytes = serve_estimate_bytes(s->queue.front().first.n, s->queue.front().first.m);
                    if (s->in_flight == 0 || s->in_flight + bytes <= s->budget) break;
                } else if (s->stopping) {
                    break;
                }
                s->cv_work.wait(lock);
            }
            if (s->queue.empty()) break;  // stopping and drained
            r = s->queue.front().first;
            submit = s->queue.front().second;
            s->queue.pop_front();
            s->in_flight += bytes;
            if (s->in_flight > s->stats.peak_bytes) s->stats.peak_bytes = s->in_flight;
            s->stats.running += 1;
        }
        s->cv_work.notify_all();  // the next request may fit as well
        tc_result res{};
        res.id = r.id;
        res.slot = slot;
        res.bytes = bytes;
        res.submit_s = submit;
        res.start_s = now_s(s->t0);
        run_one(s->pool, s->sms, stream, r, &res);
        res.end_s = now_s(s->t0);
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->in_flight -= bytes;
            s->stats.running -= 1;
            s->stats.completed += 1;
            s->done.push_back(res);
        }
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
    cudaStreamDestroy(stream);
}

}  // namespace

extern "C" tc_status tc_server_start(uint64_t hbm_budget_bytes, int32_t slots, tc_server** out) {
    if (!out || slots < 1 || slots > 64 || hbm_budget_bytes == 0) return TC_EINVAL;
    *out = nullptr;
    tc_server* s = new (std::nothrow) tc_server();
    if (!s) return TC_ENOMEM;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return TC_ECUDA;
    }
    s->pool = device_pool(s->device);  // also prepares the device for the library's kernels
    if (!s->pool) {
        delete s;
        return TC_ECUDA;
    }
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    s->budget = hbm_budget_bytes;
    s->t0 = std::chrono::steady_clock::now();
    s->stats.slots = slots;
    s->stats.budget_bytes = hbm_budget_bytes;
    for (int i = 0; i < slots; ++i) s->workers.emplace_back(worker_main, s, i);
    *out = s;
    return TC_OK;
}

extern "C" tc_status tc_server_submit(tc_server* s, const tc_request* r) {
    if (!s || !r || r->n < 0 || r->m < 0 || r->m > INT32_MAX || (r->kind != TC_GEN_RMAT && r->kind != TC_GEN_ER_REPLACE) ||
        (r->m > 0 && r->n == 0))
        return TC_EINVAL;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stopping) return TC_EBUSY;
        s->queue.emplace_back(*r, now_s(s->t0));
        s->stats.submitted += 1;
        if ((uint64_t)s->queue.size() > s->stats.max_queue) s->stats.max_queue = s->queue.size();
    }
    s->cv_work.notify_one();
    return TC_OK;
}

extern "C" tc_status tc_server_poll(tc_server* s, tc_result* out, int32_t max, int32_t* count) {
    if (!s || !count || max < 0 || (max > 0 && !out)) return TC_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    int32_t k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.back();
        s->done.pop_back();
    }
    *count = k;
    return TC_OK;
}

extern "C" tc_status tc_server_wait(tc_server* s, int64_t completed, double timeout_s) {
    if (!s) return TC_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    const bool ok = s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s),
                                        [&] { return (int64_t)s->stats.completed >= completed; });
    return ok ? TC_OK : TC_ETIMEOUT;
}

extern "C" tc_status tc_server_get_stats(tc_server* s, tc_server_stats* out) {
    if (!s || !out) return TC_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->stats;
    out->queued = s->queue.size();
    out->in_flight_bytes = s->in_flight;
    out->clock_s = now_s(s->t0);
    return TC_OK;
}

extern "C" tc_status tc_server_stop(tc_server* s) {
    if (!s) return TC_EINVAL;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& w : s->workers) w.join();
    delete s;
    return TC_OK;
}

extern "C" tc_status tc_request_run(const tc_request* r, void* cuda_stream, tc_result* out) {
    if (!r || !out || r->n < 0 || r->m < 0 || r->m > INT32_MAX || (r->kind != TC_GEN_RMAT && r->kind != TC_GEN_ER_REPLACE) ||
        (r->m > 0 && r->n == 0))
        return TC_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return TC_ECUDA;
    cudaMemPool_t pool = device_pool(dev);
    if (!pool) return TC_ECUDA;
    *out = tc_result{};
    out->id = r->id;
    out->bytes = serve_estimate_bytes(r->n, r->m);
    const auto t0 = std::chrono::steady_clock::now();
    run_one(pool, sms, static_cast<cudaStream_t>(cuda_stream), *r, out);
    out->end_s = now_s(t0);
    return TC_OK;
}

extern "C" tc_status tc_generate_edges(int kind, int32_t n, int64_t m, uint64_t seed, uint64_t stream_id, int32_t* src,
                                       int32_t* dst, void* cuda_stream) {
    if (n < 0 || m < 0 || m > INT32_MAX || (m > 0 && (!src || !dst || n == 0)) ||
        (kind != TC_GEN_RMAT && kind != TC_GEN_ER_REPLACE))
        return TC_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return TC_ECUDA;
    Launch L{static_cast<cudaStream_t>(cuda_stream), sms};
    return launch_generate(kind, n, m, seed, stream_id, src, dst, L) == cudaSuccess ? TC_OK : TC_ECUDA;
}
