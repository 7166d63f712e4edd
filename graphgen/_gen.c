/*
 * Seeded synthetic graph generators (input side only).
 *
 * These routines draw random graphs and turn edge lists into canonical symmetric
 * CSR (int64 row pointers, int32 sorted neighbour lists, no self-loops, no
 * duplicates). They contain none of the nucleus-decomposition arithmetic: both the
 * CPU oracle and the GPU library consume their output, and neither side shares any
 * other code.
 *
 * Random numbers: xoshiro256** (Blackman and Vigna), state seeded from a 64-bit
 * seed through SplitMix64, as both authors recommend.
 *
 * Plain C11, no intrinsics, no platform-specific assembly: it builds and gives the
 * same output on x86_64 and aarch64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t s[4];
} gg_rng;

static uint64_t gg_splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static void gg_seed(gg_rng *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = gg_splitmix64(&x);
}

static inline uint64_t gg_rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t gg_next(gg_rng *r) {
    uint64_t *s = r->s;
    const uint64_t result = gg_rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = gg_rotl(s[3], 45);
    return result;
}

/* uniform double in [0, 1) with 53 random bits */
static inline double gg_unif(gg_rng *r) { return (double)(gg_next(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, bound) (bound > 0), Lemire-style rejection-free multiply-shift
 * with a rejection step to remove bias */
static inline uint64_t gg_below(gg_rng *r, uint64_t bound) {
    uint64_t threshold = (0 - bound) % bound;
    for (;;) {
        uint64_t x = gg_next(r);
        if (x >= threshold) return x % bound;
    }
}

/* ------------------------------------------------------------------------- */
/* Edge-list growth helper                                                   */

typedef struct {
    int32_t *u, *v;
    int64_t m, cap;
} gg_edges;

static int gg_push(gg_edges *e, int32_t a, int32_t b) {
    if (e->m == e->cap) {
        int64_t nc = e->cap ? e->cap * 2 : 1024;
        int32_t *nu = (int32_t *)realloc(e->u, (size_t)nc * sizeof(int32_t));
        if (!nu) return -1;
        e->u = nu;
        int32_t *nv = (int32_t *)realloc(e->v, (size_t)nc * sizeof(int32_t));
        if (!nv) return -1;
        e->v = nv;
        e->cap = nc;
    }
    e->u[e->m] = a;
    e->v[e->m] = b;
    e->m++;
    return 0;
}

void gg_free(void *p) { free(p); }

/* ------------------------------------------------------------------------- */
/* Chung-Lu, exact O(n^2): every pair i<j is an edge with probability
 * min(1, w_i w_j / S), S = sum of weights. */
int64_t gg_chung_lu_exact(int32_t n, const double *w, uint64_t seed, int32_t **out_u, int32_t **out_v) {
    gg_rng r;
    gg_seed(&r, seed);
    double S = 0.0;
    for (int32_t i = 0; i < n; ++i) S += w[i];
    gg_edges e = {0};
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t j = i + 1; j < n; ++j) {
            double p = w[i] * w[j] / S;
            if (p > 1.0) p = 1.0;
            if (gg_unif(&r) < p) {
                if (gg_push(&e, i, j)) return -1;
            }
        }
    }
    *out_u = e.u;
    *out_v = e.v;
    return e.m;
}

/* Chung-Lu, O(n + m) skip sampling (Miller and Hagberg, 2011). Weights must be sorted
 * in non-increasing order; the pair (i,j) is an edge with probability
 * min(1, w_i w_j / S), exactly as in the O(n^2) routine. */
int64_t gg_chung_lu_fast(int32_t n, const double *w, uint64_t seed, int32_t **out_u, int32_t **out_v) {
    gg_rng r;
    gg_seed(&r, seed);
    double S = 0.0;
    for (int32_t i = 0; i < n; ++i) S += w[i];
    gg_edges e = {0};
    for (int32_t u = 0; u + 1 < n; ++u) {
        int64_t v = u + 1;
        double p = w[u] * w[v] / S;
        if (p > 1.0) p = 1.0;
        while (v < n && p > 0.0) {
            if (p < 1.0) {
                double x = gg_unif(&r);
                /* geometric skip: number of failures before the next success */
                double skip = floor(log1p(-x) / log1p(-p));
                if (skip > (double)n) skip = (double)n;
                v += (int64_t)skip;
            }
            if (v < n) {
                double q = w[u] * w[v] / S;
                if (q > 1.0) q = 1.0;
                if (gg_unif(&r) < q / p) {
                    if (gg_push(&e, u, (int32_t)v)) return -1;
                }
                p = q;
                v += 1;
            }
        }
    }
    *out_u = e.u;
    *out_v = e.v;
    return e.m;
}

/* R-MAT: `samples` directed edge samples on 2^scale vertices, quadrant
 * probabilities a, b, c, d = 1-a-b-c at every level, no noise, no permutation.
 * Self-loops and duplicates are kept here; the CSR builder drops them. */
int64_t gg_rmat(int32_t scale, int64_t samples, double a, double b, double c, uint64_t seed, int32_t *out_u,
                int32_t *out_v) {
    gg_rng r;
    gg_seed(&r, seed);
    const double ab = a + b, abc = a + b + c;
    for (int64_t k = 0; k < samples; ++k) {
        uint32_t u = 0, v = 0;
        for (int32_t l = 0; l < scale; ++l) {
            double x = gg_unif(&r);
            uint32_t bu, bv;
            if (x < a) {
                bu = 0;
                bv = 0;
            } else if (x < ab) {
                bu = 0;
                bv = 1;
            } else if (x < abc) {
                bu = 1;
                bv = 0;
            } else {
                bu = 1;
                bv = 1;
            }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        out_u[k] = (int32_t)u;
        out_v[k] = (int32_t)v;
    }
    return samples;
}

/* Planted communities: `k` disjoint groups with sizes uniform in [smin, smax], whose
 * members are the first vertices of a seeded Fisher-Yates shuffle of 0..n-1; every
 * internal pair is an edge with probability p. Returns the number of edges. */
int64_t gg_planted(int32_t n, int32_t k, int32_t smin, int32_t smax, double p, uint64_t seed, int32_t **out_u,
                   int32_t **out_v) {
    gg_rng r;
    gg_seed(&r, seed);
    int32_t *perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!perm) return -1;
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {
        int32_t j = (int32_t)gg_below(&r, (uint64_t)i + 1);
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
    gg_edges e = {0};
    int64_t at = 0;
    for (int32_t g = 0; g < k; ++g) {
        int32_t sz = smin + (int32_t)gg_below(&r, (uint64_t)(smax - smin + 1));
        if (at + sz > n) break;
        for (int32_t i = 0; i < sz; ++i)
            for (int32_t j = i + 1; j < sz; ++j)
                if (gg_unif(&r) < p) {
                    if (gg_push(&e, perm[at + i], perm[at + j])) {
                        free(perm);
                        return -1;
                    }
                }
        at += sz;
    }
    free(perm);
    *out_u = e.u;
    *out_v = e.v;
    return e.m;
}

/* G(n,p) for tiny test graphs. */
int64_t gg_gnp(int32_t n, double p, uint64_t seed, int32_t **out_u, int32_t **out_v) {
    gg_rng r;
    gg_seed(&r, seed);
    gg_edges e = {0};
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = i + 1; j < n; ++j)
            if (gg_unif(&r) < p) {
                if (gg_push(&e, i, j)) return -1;
            }
    *out_u = e.u;
    *out_v = e.v;
    return e.m;
}

/* Uniform doubles for seeded parameter draws on the Python side. */
void gg_uniform(uint64_t seed, int64_t count, double *out) {
    gg_rng r;
    gg_seed(&r, seed);
    for (int64_t i = 0; i < count; ++i) out[i] = gg_unif(&r);
}

/* ------------------------------------------------------------------------- */
/* Canonical symmetric CSR from an undirected edge list: drops self-loops, stores
 * both directions, sorts every row ascending and removes duplicates.
 * rowptr has n+1 entries; col is allocated here (free with gg_free). Returns the
 * number of stored (directed) entries, i.e. 2m, or -1 on bad input / no memory. */

static void gg_sort_i32(int32_t *a, int64_t len, int32_t *tmp) {
    /* LSD radix sort on the 32-bit pattern with the sign bit flipped (ids are >= 0) */
    int32_t *src = a, *dst = tmp;
    for (int pass = 0; pass < 4; ++pass) {
        int64_t cnt[257];
        memset(cnt, 0, sizeof(cnt));
        int sh = pass * 8;
        for (int64_t i = 0; i < len; ++i) cnt[(((uint32_t)src[i] ^ 0x80000000u) >> sh & 0xff) + 1]++;
        for (int b = 0; b < 256; ++b) cnt[b + 1] += cnt[b];
        for (int64_t i = 0; i < len; ++i) dst[cnt[((uint32_t)src[i] ^ 0x80000000u) >> sh & 0xff]++] = src[i];
        int32_t *t = src;
        src = dst;
        dst = t;
    }
    /* four passes: result is back in `a` */
}

static void gg_insertion_sort(int32_t *a, int64_t len) {
    for (int64_t i = 1; i < len; ++i) {
        int32_t x = a[i];
        int64_t j = i - 1;
        while (j >= 0 && a[j] > x) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = x;
    }
}

int64_t gg_csr_from_edges(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, int64_t *rowptr,
                          int32_t **out_col) {
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) return -1;
    for (int64_t k = 0; k < m; ++k) {
        int32_t a = eu[k], b = ev[k];
        if (a < 0 || b < 0 || a >= n || b >= n) {
            free(deg);
            return -1;
        }
        if (a == b) continue;
        deg[a]++;
        deg[b]++;
    }
    int64_t total = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t d = deg[v];
        deg[v] = total;
        total += d;
    }
    deg[n] = total;
    int32_t *col = (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    int64_t *fill = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!col || !fill) {
        free(deg);
        free(col);
        free(fill);
        return -1;
    }
    memcpy(fill, deg, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t k = 0; k < m; ++k) {
        int32_t a = eu[k], b = ev[k];
        if (a == b) continue;
        col[fill[a]++] = b;
        col[fill[b]++] = a;
    }
    free(fill);
    /* sort and dedupe each row, compacting in place */
    int64_t maxd = 0;
    for (int32_t v = 0; v < n; ++v)
        if (deg[v + 1] - deg[v] > maxd) maxd = deg[v + 1] - deg[v];
    int32_t *tmp = (int32_t *)malloc((size_t)(maxd > 0 ? maxd : 1) * sizeof(int32_t));
    if (!tmp) {
        free(deg);
        free(col);
        return -1;
    }
    int64_t w = 0;
    rowptr[0] = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t b = deg[v], e = deg[v + 1], len = e - b;
        int32_t *row = col + b;
        if (len <= 32)
            gg_insertion_sort(row, len);
        else
            gg_sort_i32(row, len, tmp);
        int64_t start = w;
        for (int64_t i = 0; i < len; ++i) {
            if (w > start && col[w - 1] == row[i]) continue;
            col[w++] = row[i];
        }
        rowptr[v + 1] = w;
    }
    free(tmp);
    free(deg);
    *out_col = col;
    return w;
}
