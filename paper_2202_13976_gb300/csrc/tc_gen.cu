// Device-side generation of the seeded synthetic inputs used by the serving loop,
// whose request graphs are too many to stage from the host.  This file produces
// inputs only and holds none of the counting arithmetic.
//
// The definitions are the published ones the host generator also implements:
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) in counter form, draw i of stream
// (seed, s) = mix(key + (i + 1) * gamma) with key = mix(mix(seed + gamma) ^ ((s + 1) * gamma));
// R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with (a, b, c) = (0.57, 0.19, 0.19),
// one 32-bit uniform per level (high half of the draw for even levels, low half for
// odd), draw index ((e * 64 + r) * 16) + level / 2 for pair e and redraw attempt r,
// pairs with an endpoint >= n redrawn, after 64 attempts reduced modulo n; uniform
// pairs with replacement: u = (hi32 * n) >> 32, v = (lo32 * n) >> 32 of draw i.
#include <cmath>

#include "tc_device.cuh"
#include "tc_internal.h"

namespace tcg {
namespace {

constexpr unsigned long long GAMMA = 0x9e3779b97f4a7c15ull;

__host__ __device__ __forceinline__ unsigned long long sm_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long sm_draw(unsigned long long key, unsigned long long i) {
    return sm_mix(key + (i + 1) * GAMMA);
}

__global__ void k_gen_rmat(unsigned long long key, int scale, int32_t n, int64_t m, uint32_t ta, uint32_t tab,
                           uint32_t tabc, int32_t* __restrict__ src, int32_t* __restrict__ dst) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        for (unsigned long long r = 0; r < 64; ++r) {
            const unsigned long long base = (((unsigned long long)e * 64 + r) * 16);
            unsigned long long row = 0, col = 0, x = 0;
            for (int l = 0; l < scale; ++l) {
                if ((l & 1) == 0) x = sm_draw(key, base + (unsigned long long)(l >> 1));
                const uint32_t u = (l & 1) ? (uint32_t)(x & 0xffffffffu) : (uint32_t)(x >> 32);
                const unsigned long long bit = 1ull << (scale - 1 - l);
                if (u < ta) {
                } else if (u < tab) {
                    col |= bit;
                } else if (u < tabc) {
                    row |= bit;
                } else {
                    row |= bit;
                    col |= bit;
                }
            }
            if (row < (unsigned long long)n && col < (unsigned long long)n) {
                src[e] = (int32_t)row;
                dst[e] = (int32_t)col;
                break;
            }
            if (r == 63) {
                src[e] = (int32_t)(row % (unsigned long long)n);
                dst[e] = (int32_t)(col % (unsigned long long)n);
            }
        }
    }
}

__global__ void k_gen_er_replace(unsigned long long key, int32_t n, int64_t m, int32_t* __restrict__ src,
                                 int32_t* __restrict__ dst) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const unsigned long long x = sm_draw(key, (unsigned long long)i);
        src[i] = (int32_t)(((x >> 32) * (unsigned long long)n) >> 32);
        dst[i] = (int32_t)(((x & 0xffffffffu) * (unsigned long long)n) >> 32);
    }
}

}  // namespace

unsigned long long gen_stream_key(unsigned long long seed, unsigned long long stream) {
    return sm_mix(sm_mix(seed + GAMMA) ^ ((stream + 1) * GAMMA));
}

cudaError_t launch_generate(int kind, int32_t n, int64_t m, unsigned long long seed, unsigned long long stream_id,
                            int32_t* src, int32_t* dst, const Launch& L) {
    if (m <= 0) return cudaSuccess;
    const unsigned long long key = gen_stream_key(seed, stream_id);
    if (kind == TC_GEN_RMAT) {
        int scale = 1;
        while ((1ll << scale) < (long long)n) ++scale;
        const uint32_t ta = (uint32_t)std::floor(0.57 * 4294967296.0);
        const uint32_t tab = (uint32_t)std::floor((0.57 + 0.19) * 4294967296.0);
        const uint32_t tabc = (uint32_t)std::floor((0.57 + 0.19 + 0.19) * 4294967296.0);
        k_gen_rmat<<<grid_for(m, 256, L.sms), 256, 0, L.stream>>>(key, scale, n, m, ta, tab, tabc, src, dst);
    } else {
        k_gen_er_replace<<<grid_for(m, 256, L.sms), 256, 0, L.stream>>>(key, n, m, src, dst);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace tcg
