/*
 * Seeded synthetic graph generators: R-MAT and Erdos-Renyi G(n, m).
 *
 * This file produces INPUTS only.  It holds none of the triangle-counting
 * arithmetic; both the CPU oracle and the CUDA path consume its edge lists.
 *
 * Random numbers come from a counter-based form of SplitMix64 (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): draw i
 * of a stream is the SplitMix64 output function applied to key + (i + 1) * gamma,
 * gamma = 0x9e3779b97f4a7c15.  Every draw is therefore addressable by its index,
 * so generation is deterministic for any thread count, on x86 and Arm alike.
 *
 * R-MAT (Chakrabarti, Zhan, Faloutsos 2004), with the parameters the paper uses
 * for its synthetic graphs (a, b, c, d) = (0.57, 0.19, 0.19, 0.05) (Sec. V-A):
 * each generated pair descends `scale` levels of the recursive 2x2 partition of
 * the adjacency matrix.  Level l (l = 0 is the most significant bit) reads one
 * 32-bit uniform u: u < ta picks quadrant a (no bit set), u < tab picks b (column
 * bit), u < tabc picks c (row bit), otherwise d (both bits).  Thresholds are
 * floor(cumulative probability * 2^32), passed in by the caller.  No noise and no
 * vertex permutation are applied.  Two levels share one 64-bit draw (high half for
 * even l, low half for odd l); draw index = ((e * 64 + r) * 16) + l / 2, where r is
 * the redraw attempt.  A pair with an endpoint >= n (n not a power of two) is
 * redrawn with r + 1; after 64 attempts the endpoints are reduced modulo n.
 *
 * ER with replacement (the serving stream): pair i is draw i split into
 * u = (hi32 * n) >> 32 and v = (lo32 * n) >> 32; loops and repeats are kept in the
 * list (the counting library drops them).
 *
 * ER G(n, m): m distinct unordered pairs {u != v}, uniform without replacement.
 *  - when 4m >= C(n,2) (dense) every pair index p in [0, C(n,2)) (row-major over
 *    u < v) gets the key draw(p); the m pairs with the smallest (key, p) are
 *    emitted in that order;
 *  - otherwise draws i = 0, 1, ... give candidates u = (hi32 * n) >> 32,
 *    v = (lo32 * n) >> 32; loops are skipped and the first m distinct unordered
 *    pairs in draw order are emitted.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GG_GAMMA 0x9e3779b97f4a7c15ULL

static inline uint64_t gg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t gg_stream_key(uint64_t seed, uint64_t stream) {
    return gg_mix(gg_mix(seed + GG_GAMMA) ^ ((stream + 1) * GG_GAMMA));
}

uint64_t gg_draw(uint64_t key, uint64_t i) { return gg_mix(key + (i + 1) * GG_GAMMA); }

void gg_draw_many(uint64_t key, uint64_t i0, int64_t count, uint64_t* out) {
    for (int64_t k = 0; k < count; ++k) out[k] = gg_draw(key, i0 + (uint64_t)k);
}

static inline void rmat_pair(uint64_t key, int64_t e, int scale, int64_t n, uint32_t ta,
                             uint32_t tab, uint32_t tabc, int32_t* su, int32_t* sv) {
    for (uint64_t r = 0; r < 64; ++r) {
        uint64_t base = (((uint64_t)e * 64 + r) * 16);
        uint64_t row = 0, col = 0, x = 0;
        for (int l = 0; l < scale; ++l) {
            if ((l & 1) == 0) x = gg_draw(key, base + (uint64_t)(l >> 1));
            uint32_t u = (l & 1) ? (uint32_t)(x & 0xffffffffu) : (uint32_t)(x >> 32);
            uint64_t bit = 1ULL << (scale - 1 - l);
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
        if ((int64_t)row < n && (int64_t)col < n) {
            *su = (int32_t)row;
            *sv = (int32_t)col;
            return;
        }
        if (r == 63) {
            *su = (int32_t)(row % (uint64_t)n);
            *sv = (int32_t)(col % (uint64_t)n);
            return;
        }
    }
}

/* R-MAT pairs e in [e0, e0 + count); writes src[e - e0], dst[e - e0]. */
void gg_rmat(uint64_t seed, uint64_t stream, int scale, int64_t n, int64_t e0, int64_t count,
             uint32_t ta, uint32_t tab, uint32_t tabc, int32_t* src, int32_t* dst) {
    uint64_t key = gg_stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k)
        rmat_pair(key, e0 + k, scale, n, ta, tab, tabc, &src[k], &dst[k]);
}

/* ER with replacement: pairs i in [i0, i0 + count). */
void gg_er_replace(uint64_t seed, uint64_t stream, int64_t n, int64_t i0, int64_t count, int32_t* src, int32_t* dst) {
    uint64_t key = gg_stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k) {
        uint64_t x = gg_draw(key, (uint64_t)(i0 + k));
        src[k] = (int32_t)(((x >> 32) * (uint64_t)n) >> 32);
        dst[k] = (int32_t)(((x & 0xffffffffu) * (uint64_t)n) >> 32);
    }
}

typedef struct {
    uint64_t key;
    int64_t idx;
} gg_kv;

static int gg_kv_cmp(const void* a, const void* b) {
    const gg_kv* x = (const gg_kv*)a;
    const gg_kv* y = (const gg_kv*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

/* Pair index p (row-major over u < v) -> (u, v); row u starts at u(2n-u-1)/2. */
static void pair_of_index(int64_t n, int64_t p, int32_t* u, int32_t* v) {
    int64_t lo = 0, hi = n - 2; /* largest row whose start is <= p */
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (mid * (2 * n - mid - 1) / 2 <= p)
            lo = mid;
        else
            hi = mid - 1;
    }
    int64_t start = lo * (2 * n - lo - 1) / 2;
    *u = (int32_t)lo;
    *v = (int32_t)(lo + 1 + (p - start));
}

static uint64_t next_pow2(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

/* Returns the number of pairs written (m, capped at C(n,2)); -1 on allocation failure. */
int64_t gg_er(uint64_t seed, uint64_t stream, int64_t n, int64_t m, int32_t* src, int32_t* dst) {
    uint64_t key = gg_stream_key(seed, stream);
    int64_t total = n < 2 ? 0 : n * (n - 1) / 2;
    if (m > total) m = total;
    if (m <= 0) return 0;
    if (4 * m >= total) {
        /* The m smallest (key, p) are found by filtering on a key threshold that is
           raised until at least m pairs pass; the selection does not depend on it. */
        gg_kv* kv = (gg_kv*)malloc(sizeof(gg_kv) * (size_t)total);
        if (!kv) return -1;
        double frac = 2.0 * (double)m / (double)total + 1e-3;
        for (;;) {
            uint64_t thr = frac >= 1.0 ? ~0ULL : (uint64_t)(frac * 18446744073709551615.0);
            int64_t cnt = 0;
            for (int64_t p = 0; p < total; ++p) {
                uint64_t k = gg_draw(key, (uint64_t)p);
                if (k <= thr) {
                    kv[cnt].key = k;
                    kv[cnt].idx = p;
                    ++cnt;
                }
            }
            if (cnt >= m || frac >= 1.0) {
                qsort(kv, (size_t)cnt, sizeof(gg_kv), gg_kv_cmp);
                break;
            }
            frac *= 2.0;
        }
        for (int64_t k = 0; k < m; ++k) pair_of_index(n, kv[k].idx, &src[k], &dst[k]);
        free(kv);
        return m;
    }
    uint64_t cap = next_pow2((uint64_t)m * 2 + 16);
    uint64_t* table = (uint64_t*)malloc(sizeof(uint64_t) * cap);
    if (!table) return -1;
    memset(table, 0xff, sizeof(uint64_t) * cap); /* empty slot = all ones */
    int64_t got = 0;
    uint64_t i = 0;
    const int64_t chunk = 1 << 20;
    uint64_t* buf = (uint64_t*)malloc(sizeof(uint64_t) * chunk);
    if (!buf) {
        free(table);
        return -1;
    }
    while (got < m) {
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < chunk; ++k) buf[k] = gg_draw(key, i + (uint64_t)k);
        for (int64_t k = 0; k < chunk && got < m; ++k) {
            uint64_t x = buf[k];
            uint64_t u = ((x >> 32) * (uint64_t)n) >> 32;
            uint64_t v = ((x & 0xffffffffu) * (uint64_t)n) >> 32;
            if (u == v) continue;
            uint64_t a = u < v ? u : v, b = u < v ? v : u;
            uint64_t kk = (a << 32) | b;
            uint64_t h = gg_mix(kk) & (cap - 1);
            int fresh = 1;
            while (table[h] != ~0ULL) {
                if (table[h] == kk) {
                    fresh = 0;
                    break;
                }
                h = (h + 1) & (cap - 1);
            }
            if (!fresh) continue;
            table[h] = kk;
            src[got] = (int32_t)u;
            dst[got] = (int32_t)v;
            ++got;
        }
        i += (uint64_t)chunk;
    }
    free(buf);
    free(table);
    return m;
}
