/*
 * Seeded synthetic graph generators: Erdos-Renyi G(n, m), R-MAT (with optional
 * planted cliques) and a degree-ascending relabel.  Every generator returns an
 * undirected simple graph stored as a strictly upper-triangular CSR
 * (row_ptr int32[n+1], col int32[m], columns strictly increasing in a row,
 * col > row), which is the input format of Eager K-truss (Sec. II-B, Sec. III-D
 * of Blanco, Low, Kim, HPEC 2019).
 *
 * This file holds graph construction only.  It contains no triangle, support
 * or pruning arithmetic, and both the K-truss oracle and the CUDA library take
 * their inputs from it.
 *
 * Random numbers come from a counter-based generator: value i of stream `key`
 * is SplitMix64's output function applied to key + (i + 1) * 0x9E3779B97F4A7C15
 * (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014; constants as published by S. Vigna).  Every draw is
 * a pure function of (key, i), so the output is independent of thread count,
 * and no floating point touches the sampled values, so x86_64 and aarch64
 * produce the same graphs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t n;
    int64_t m;
    int32_t *row_ptr;
    int32_t *col;
} gg_csr;

#define GG_OK 0
#define GG_EINVAL -1
#define GG_ENOMEM -2

static const uint64_t GOLDEN = 0x9E3779B97F4A7C15ULL;

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Value i of the counter-based stream `key`. */
uint64_t gg_rand(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GOLDEN); }

/* Derives a stream key from (tag, seed, stream) so that generators and their
 * sub-steps never share draws. */
uint64_t gg_key(uint64_t tag, uint64_t seed, uint64_t stream) {
    return mix64(mix64(tag * GOLDEN + 0x1234567ULL) ^ (seed * 0xD1B54A32D192ED03ULL)) ^
           mix64(stream + 0x5851F42D4C957F2DULL);
}

/* Unbiased integer in [0, bound) by rejection on the top bits (bound >= 1). */
static uint64_t bounded(uint64_t key, uint64_t *ctr, uint64_t bound) {
    uint64_t lim = UINT64_MAX - (UINT64_MAX % bound);
    for (;;) {
        uint64_t r = gg_rand(key, (*ctr)++);
        if (r < lim) return r % bound;
    }
}

/* ---------------------------------------------------------------- sorting */

/* LSD radix sort of 64-bit keys on the low `bits` bits; tmp has n slots. */
static void radix_sort_u64(uint64_t *a, uint64_t *tmp, int64_t n, int bits) {
    uint64_t *src = a, *dst = tmp;
    for (int shift = 0; shift < bits; shift += 11) {
        int64_t cnt[2048];
        memset(cnt, 0, sizeof(cnt));
        for (int64_t i = 0; i < n; ++i) cnt[(src[i] >> shift) & 2047]++;
        int64_t s = 0;
        for (int d = 0; d < 2048; ++d) { int64_t c = cnt[d]; cnt[d] = s; s += c; }
        for (int64_t i = 0; i < n; ++i) dst[cnt[(src[i] >> shift) & 2047]++] = src[i];
        uint64_t *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, (size_t)n * sizeof(uint64_t));
}

/* Turns a list of packed pairs (u << 32 | v), u < v, into a sorted,
 * de-duplicated upper-triangular CSR.  Consumes `pairs`. */
static int pairs_to_csr(gg_csr *out, int32_t n, uint64_t *pairs, int64_t cnt) {
    uint64_t *tmp = (uint64_t *)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(uint64_t));
    if (!tmp) return GG_ENOMEM;
    int bits = 0;
    while (bits < 64 && (((uint64_t)1 << bits) <= (uint64_t)n)) bits++;
    radix_sort_u64(pairs, tmp, cnt, 32 + bits);
    free(tmp);
    int64_t m = 0;
    for (int64_t i = 0; i < cnt; ++i)
        if (m == 0 || pairs[i] != pairs[m - 1]) pairs[m++] = pairs[i];
    out->n = n;
    out->m = m;
    out->row_ptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    out->col = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!out->row_ptr || !out->col) return GG_ENOMEM;
    for (int64_t i = 0; i < m; ++i) {
        out->row_ptr[(pairs[i] >> 32) + 1]++;
        out->col[i] = (int32_t)(pairs[i] & 0xFFFFFFFFULL);
    }
    for (int32_t i = 0; i < n; ++i) out->row_ptr[i + 1] += out->row_ptr[i];
    return GG_OK;
}

static inline uint64_t pack(uint32_t u, uint32_t v) {
    return u < v ? ((uint64_t)u << 32) | v : ((uint64_t)v << 32) | u;
}

/* ------------------------------------------------------- relabel by degree */

/* New label of v = rank of v when vertices are sorted by (degree, old id). */
static int relabel_degree_ascending(gg_csr *g) {
    int32_t n = g->n;
    int64_t m = g->m;
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    uint64_t *keys = (uint64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint64_t));
    uint64_t *tmp = (uint64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint64_t));
    int32_t *newid = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    uint64_t *pairs = (uint64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
    if (!deg || !keys || !tmp || !newid || !pairs) return GG_ENOMEM;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t p = g->row_ptr[i]; p < g->row_ptr[i + 1]; ++p) {
            deg[i]++;
            deg[g->col[p]]++;
        }
    for (int32_t v = 0; v < n; ++v) keys[v] = ((uint64_t)deg[v] << 32) | (uint32_t)v;
    radix_sort_u64(keys, tmp, n, 64);
    for (int32_t r = 0; r < n; ++r) newid[keys[r] & 0xFFFFFFFFULL] = r;
    int64_t c = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t p = g->row_ptr[i]; p < g->row_ptr[i + 1]; ++p)
            pairs[c++] = pack((uint32_t)newid[i], (uint32_t)newid[g->col[p]]);
    free(g->row_ptr);
    free(g->col);
    int rc = pairs_to_csr(g, n, pairs, c);
    free(pairs); free(deg); free(keys); free(tmp); free(newid);
    return rc;
}

void gg_free(gg_csr *g) {
    if (!g) return;
    free(g->row_ptr);
    free(g->col);
    g->row_ptr = NULL;
    g->col = NULL;
}

/* ------------------------------------------------------------------- G(n,m) */

/* Erdos-Renyi G(n, m): unordered pairs u != v drawn uniformly, duplicates
 * rejected, until exactly m distinct edges exist (requires m <= n(n-1)/2). */
int gg_er(gg_csr *out, int32_t n, int64_t m, uint64_t seed, int relabel) {
    memset(out, 0, sizeof(*out));
    if (n < 0 || m < 0 || (n < 2 && m > 0) || m > (int64_t)n * (n - 1) / 2) return GG_EINVAL;
    uint64_t key = gg_key(1, seed, 0);
    /* open-addressing set of packed pairs, load factor <= 1/2 */
    uint64_t cap = 16;
    while (cap < (uint64_t)(2 * m + 2)) cap <<= 1;
    uint64_t *set = (uint64_t *)malloc(cap * sizeof(uint64_t));
    uint64_t *pairs = (uint64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
    if (!set || !pairs) { free(set); free(pairs); return GG_ENOMEM; }
    memset(set, 0xFF, cap * sizeof(uint64_t));
    uint64_t ctr = 0;
    int64_t have = 0;
    while (have < m) {
        uint32_t u = (uint32_t)bounded(key, &ctr, (uint64_t)n);
        uint32_t v = (uint32_t)bounded(key, &ctr, (uint64_t)n);
        if (u == v) continue;
        uint64_t k = pack(u, v);
        uint64_t h = mix64(k) & (cap - 1);
        int dup = 0;
        while (set[h] != UINT64_MAX) {
            if (set[h] == k) { dup = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (dup) continue;
        set[h] = k;
        pairs[have++] = k;
    }
    free(set);
    int rc = pairs_to_csr(out, n, pairs, m);
    free(pairs);
    if (rc == GG_OK && relabel) rc = relabel_degree_ascending(out);
    return rc;
}

/* -------------------------------------------------------------------- R-MAT */

/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004): edge_factor * 2^scale samples;
 * each picks, for every bit from the most significant down, the quadrant
 * (0,0), (0,1), (1,0), (1,1) with probabilities a, b, c, 1-a-b-c, using the
 * thresholds t1 <= t2 <= t3 given as 64-bit fixed point (probability * 2^64).
 * No noise, no vertex permutation.  Then n_cliques cliques are planted with
 * sizes clique_lo + round((clique_hi - clique_lo) * c / (n_cliques - 1)),
 * c = 0 .. n_cliques-1, each on distinct vertices drawn uniformly from
 * [0, 2^scale) (cliques may overlap one another).  The union is symmetrised,
 * self-loops dropped, de-duplicated and stored upper-triangular. */
int gg_rmat(gg_csr *out, int scale, int edge_factor, uint64_t t1, uint64_t t2, uint64_t t3,
            uint64_t seed, int n_cliques, int clique_lo, int clique_hi, int relabel) {
    memset(out, 0, sizeof(*out));
    if (scale < 1 || scale > 30 || edge_factor < 0 || n_cliques < 0 || t1 > t2 || t2 > t3)
        return GG_EINVAL;
    int32_t n = (int32_t)1 << scale;
    int64_t samples = (int64_t)edge_factor << scale;
    int64_t clique_pairs = 0;
    for (int c = 0; c < n_cliques; ++c) {
        int64_t s = n_cliques == 1 ? clique_lo
                                   : clique_lo + ((int64_t)2 * (clique_hi - clique_lo) * c + (n_cliques - 1)) /
                                                     (2 * (n_cliques - 1));
        if (s > n) return GG_EINVAL;
        clique_pairs += s * (s - 1) / 2;
    }
    uint64_t *pairs = (uint64_t *)malloc((size_t)(samples + clique_pairs + 1) * sizeof(uint64_t));
    if (!pairs) return GG_ENOMEM;
    uint64_t key = gg_key(2, seed, 0);
    int64_t kept = 0;
    /* sample in parallel into a flag-marked array, then compact serially */
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < samples; ++s) {
        uint32_t u = 0, v = 0;
        uint64_t base = (uint64_t)s * (uint64_t)scale;
        for (int l = 0; l < scale; ++l) {
            uint64_t r = gg_rand(key, base + (uint64_t)l);
            uint32_t bu = r >= t2;                 /* rows 1: quadrants c, d */
            uint32_t bv = (r >= t1 && r < t2) || r >= t3; /* cols 1: quadrants b, d */
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        pairs[s] = (u == v) ? UINT64_MAX : pack(u, v);
    }
    for (int64_t s = 0; s < samples; ++s)
        if (pairs[s] != UINT64_MAX) pairs[kept++] = pairs[s];
    /* planted cliques */
    uint64_t ckey = gg_key(3, seed, 0);
    uint64_t ctr = 0;
    int32_t *verts = (int32_t *)malloc((size_t)(clique_hi > clique_lo ? clique_hi : clique_lo) * sizeof(int32_t) + 4);
    if (!verts) { free(pairs); return GG_ENOMEM; }
    for (int c = 0; c < n_cliques; ++c) {
        int64_t s = n_cliques == 1 ? clique_lo
                                   : clique_lo + ((int64_t)2 * (clique_hi - clique_lo) * c + (n_cliques - 1)) /
                                                     (2 * (n_cliques - 1));
        int64_t got = 0;
        while (got < s) {
            int32_t v = (int32_t)bounded(ckey, &ctr, (uint64_t)n);
            int dup = 0;
            for (int64_t j = 0; j < got; ++j)
                if (verts[j] == v) { dup = 1; break; }
            if (!dup) verts[got++] = v;
        }
        for (int64_t x = 0; x < s; ++x)
            for (int64_t y = x + 1; y < s; ++y) pairs[kept++] = pack((uint32_t)verts[x], (uint32_t)verts[y]);
    }
    free(verts);
    int rc = pairs_to_csr(out, n, pairs, kept);
    free(pairs);
    if (rc == GG_OK && relabel) rc = relabel_degree_ascending(out);
    return rc;
}

/* Builds an upper-triangular CSR from an arbitrary undirected edge list
 * (u[i], v[i]); self-loops are dropped and duplicates merged. */
int gg_from_edges(gg_csr *out, int32_t n, int64_t cnt, const int32_t *u, const int32_t *v, int relabel) {
    memset(out, 0, sizeof(*out));
    if (n < 0 || cnt < 0) return GG_EINVAL;
    uint64_t *pairs = (uint64_t *)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(uint64_t));
    if (!pairs) return GG_ENOMEM;
    int64_t k = 0;
    for (int64_t i = 0; i < cnt; ++i) {
        if (u[i] < 0 || v[i] < 0 || u[i] >= n || v[i] >= n) { free(pairs); return GG_EINVAL; }
        if (u[i] != v[i]) pairs[k++] = pack((uint32_t)u[i], (uint32_t)v[i]);
    }
    int rc = pairs_to_csr(out, n, pairs, k);
    free(pairs);
    if (rc == GG_OK && relabel) rc = relabel_degree_ascending(out);
    return rc;
}
