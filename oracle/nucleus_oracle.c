/*
 * CPU ORACLE for the (r,s) nucleus decomposition -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load this
 * library. The product (the CUDA library) never calls it and shares no code with it.
 *
 * Everything here is plain, sequential and slow on purpose, so that a reader can
 * check it against the paper by eye. All arithmetic is exact integer arithmetic.
 *
 * What the paper fixes, and where:
 *   - Definition (Section 2, "Preliminaries"): a c-(r,s) nucleus is a maximal union of
 *     s-cliques in which every r-clique lies in at least c of the s-cliques whose
 *     r-subsets are all present; the (r,s)-clique core number of an r-clique R is the
 *     largest c for which R lies in a c-(r,s) nucleus. The footnote's connectivity
 *     requirement is not part of the problem the paper solves, and not part of ours.
 *   - Algorithm 1 (rec-list-cliques, Section 4.1): grow cliques one vertex at a time,
 *     keeping the candidate set I of vertices adjacent to everything chosen so far.
 *   - Algorithm 2 (Section 4.2): Count-Func adds 1 to the count of every r-subset of
 *     every s-clique; the peeling loop repeatedly extracts the r-cliques of the lowest
 *     bucket (set A), and Update re-lists, for each R in A, the s-cliques containing R
 *     from I = intersection of the undirected neighbourhoods of R's vertices; for each
 *     such S, Update-Func returns at once if an r-subset of S outside A was peeled in
 *     an earlier round, and otherwise subtracts 1/a from every r-subset of S outside A,
 *     where a is the number of r-subsets of S inside A.
 *
 * Readings (where the paper leaves a choice):
 *   - The fraction 1/a is kept exact by storing every count multiplied by
 *     L = lcm(1, ..., C(s,r)) in a 128-bit integer; a <= C(s,r), so L/a is an integer.
 *   - "Next bucket" (Algorithm 2): the bucket structure keeps r-cliques whose count drops
 *     below the current level k in bucket k (the core number never decreases), so each
 *     round peels every unpeeled r-clique with count <= k after setting
 *     k = max(k, minimum unpeeled count). Rounds are counted under this rule.
 *   - r-cliques are identified by their rank in the lexicographic order of their sorted
 *     vertex tuples (original vertex ids). For r = 1 this is the vertex id; for r = 2 it
 *     is the order of edges (u < v) in CSR order.
 *   - Listing order: no orientation is used; cliques are grown in ascending vertex id,
 *     which is itself an acyclic orientation (Algorithm 2 lets the caller choose it).
 *
 * Graph input: symmetric CSR, rowptr int64[n+1], col int32[rowptr[n]], every row sorted
 * ascending, no self-loops, no duplicates (the caller guarantees this).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

typedef struct {
    int32_t n;
    const int64_t *rp;
    const int32_t *col;
} og;

static inline int64_t deg(const og *g, int32_t v) { return g->rp[v + 1] - g->rp[v]; }

/* Is x in the sorted list a[0..len)? Plain binary search. */
static int in_sorted(const int32_t *a, int64_t len, int32_t x) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo < len && a[lo] == x;
}

static int adjacent(const og *g, int32_t u, int32_t v) {
    /* search in the shorter of the two neighbour lists */
    if (deg(g, u) > deg(g, v)) {
        int32_t t = u;
        u = v;
        v = t;
    }
    return in_sorted(g->col + g->rp[u], deg(g, u), v);
}

/* I' = the members of I[i+1..nI) adjacent to v, ascending (I is sorted ascending).
 * Walks whichever of I[i+1..nI) and N(v) is shorter; both give the same set. */
static int64_t intersect_after(const og *g, const int32_t *I, int64_t i, int64_t nI, int32_t v, int32_t *out) {
    int64_t nn = 0, rest = nI - (i + 1);
    if (deg(g, v) < rest) {
        const int32_t *nb = g->col + g->rp[v];
        for (int64_t j = 0; j < deg(g, v); ++j)
            if (nb[j] > v && in_sorted(I + i + 1, rest, nb[j])) out[nn++] = nb[j];
    } else {
        for (int64_t j = i + 1; j < nI; ++j)
            if (adjacent(g, v, I[j])) out[nn++] = I[j];
    }
    return nn;
}

static int64_t binom(int a, int b) {
    if (b < 0 || b > a) return 0;
    int64_t r = 1;
    for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
    return r;
}

static int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

/* ------------------------------------------------------------------------- */
/* Clique listing (Algorithm 1, with ascending-id growth).                    */

typedef struct {
    const og *g;
    int c;                /* clique size to list */
    int32_t prefix[8];    /* vertices chosen so far, ascending */
    int32_t **cand;       /* candidate buffers per depth */
    void (*f)(void *ctx, const int32_t *clique);
    void *ctx;
} lister;

/* I holds the vertices (ascending) adjacent to every vertex of prefix[0..depth) and larger
 * than the last of them. */
static void grow(lister *L, int depth, const int32_t *I, int64_t nI) {
    if (depth == L->c) {
        L->f(L->ctx, L->prefix);
        return;
    }
    if (depth + 1 == L->c) {
        for (int64_t i = 0; i < nI; ++i) {
            L->prefix[depth] = I[i];
            L->f(L->ctx, L->prefix);
        }
        return;
    }
    for (int64_t i = 0; i < nI; ++i) {
        int32_t v = I[i];
        /* I' = I (after v) intersected with N(v) */
        int32_t *next = L->cand[depth + 1];
        int64_t nn = intersect_after(L->g, I, i, nI, v, next);
        L->prefix[depth] = v;
        grow(L, depth + 1, next, nn);
    }
}

/* List every c-clique (1 <= c <= 8) once, as an ascending tuple, in lexicographic order. */
static int list_all(const og *g, int c, void (*f)(void *, const int32_t *), void *ctx) {
    if (c < 1 || c > 8) return -1;
    int64_t maxd = 0;
    for (int32_t v = 0; v < g->n; ++v)
        if (deg(g, v) > maxd) maxd = deg(g, v);
    lister L;
    memset(&L, 0, sizeof(L));
    L.g = g;
    L.c = c;
    L.f = f;
    L.ctx = ctx;
    int32_t *bufs[9];
    for (int d = 0; d <= 8; ++d) {
        bufs[d] = (int32_t *)malloc((size_t)(maxd + 1) * sizeof(int32_t));
        if (!bufs[d]) {
            for (int e = 0; e < d; ++e) free(bufs[e]);
            return -2;
        }
    }
    L.cand = bufs;
    for (int32_t v = 0; v < g->n; ++v) {
        L.prefix[0] = v;
        if (c == 1) {
            f(ctx, L.prefix);
            continue;
        }
        const int32_t *nb = g->col + g->rp[v];
        int64_t nI = 0;
        for (int64_t j = 0; j < deg(g, v); ++j)
            if (nb[j] > v) bufs[1][nI++] = nb[j];
        grow(&L, 1, bufs[1], nI);
    }
    for (int d = 0; d <= 8; ++d) free(bufs[d]);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The r-clique table: all r-cliques as sorted tuples in lexicographic order; the
 * index of a tuple in this table is the r-clique's id.                        */

typedef struct {
    int r;
    int64_t count, cap;
    int32_t *t; /* t[id * r + j] */
} rtable;

static void rtable_add(void *ctx, const int32_t *c) {
    rtable *T = (rtable *)ctx;
    if (T->count == T->cap) {
        int64_t nc = T->cap ? 2 * T->cap : 1024;
        int32_t *nt = (int32_t *)realloc(T->t, (size_t)nc * T->r * sizeof(int32_t));
        if (!nt) {
            T->cap = -1;
            return;
        }
        T->t = nt;
        T->cap = nc;
    }
    if (T->cap < 0) return;
    memcpy(T->t + T->count * T->r, c, (size_t)T->r * sizeof(int32_t));
    T->count++;
}

static int rtable_build(const og *g, int r, rtable *T) {
    memset(T, 0, sizeof(*T));
    T->r = r;
    if (list_all(g, r, rtable_add, T)) return -2;
    if (T->cap < 0) return -2;
    return 0;
}

static int tuple_cmp(const int32_t *a, const int32_t *b, int r) {
    for (int j = 0; j < r; ++j) {
        if (a[j] < b[j]) return -1;
        if (a[j] > b[j]) return 1;
    }
    return 0;
}

/* id of the ascending tuple x, or -1 if x is not an r-clique */
static int64_t rtable_find(const rtable *T, const int32_t *x) {
    int64_t lo = 0, hi = T->count;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (tuple_cmp(T->t + mid * T->r, x, T->r) < 0)
            lo = mid + 1;
        else
            hi = mid;
    }
    if (lo < T->count && tuple_cmp(T->t + lo * T->r, x, T->r) == 0) return lo;
    return -1;
}

/* The ids of the C(s,r) r-subsets of the ascending s-tuple S, in a fixed order. */
static int subsets_of(const rtable *T, int s, const int32_t *S, int64_t *ids) {
    int r = T->r, k = 0;
    int32_t sub[8];
    for (unsigned mask = 0; mask < (1u << s); ++mask) {
        if (__builtin_popcount(mask) != r) continue;
        int j = 0;
        for (int i = 0; i < s; ++i)
            if (mask >> i & 1u) sub[j++] = S[i];
        ids[k++] = rtable_find(T, sub);
    }
    return k;
}

/* ------------------------------------------------------------------------- */
/* Count-Func (Algorithm 2): count[R] = number of s-cliques containing R.     */

typedef struct {
    const rtable *T;
    int s;
    int64_t *counts;
    int64_t n_s;
    int bad;
} count_ctx;

static void count_func(void *vctx, const int32_t *S) {
    count_ctx *C = (count_ctx *)vctx;
    int64_t ids[128];
    int k = subsets_of(C->T, C->s, S, ids);
    for (int i = 0; i < k; ++i) {
        if (ids[i] < 0) {
            C->bad = 1;
            continue;
        }
        C->counts[ids[i]] += 1;
    }
    C->n_s++;
}

static int check_rs(int r, int s) { return (r >= 1 && s > r && s <= 7) ? 0 : -1; }

/* Number of c-cliques; writes them (ascending tuples, lexicographic order) to out when
 * out is not NULL and cap (in tuples) is large enough. Returns -1 on bad c. */
typedef struct {
    int c;
    int32_t *out;
    int64_t cap, count;
} collect_ctx;

static void collect_func(void *vctx, const int32_t *x) {
    collect_ctx *C = (collect_ctx *)vctx;
    if (C->out && C->count < C->cap) memcpy(C->out + C->count * C->c, x, (size_t)C->c * sizeof(int32_t));
    C->count++;
}

int64_t orc_list_cliques(int32_t n, const int64_t *rp, const int32_t *col, int c, int32_t *out, int64_t cap) {
    og g = {n, rp, col};
    collect_ctx C = {c, out, cap, 0};
    if (c < 1 || c > 8) return -1;
    if (list_all(&g, c, collect_func, &C)) return -2;
    return C.count;
}

/* counts: int64[n_r] (n_r = number of r-cliques, canonical order). Returns 0, -1 on bad
 * (r,s), -2 on allocation failure. */
int orc_count(int32_t n, const int64_t *rp, const int32_t *col, int r, int s, int64_t *counts, int64_t *n_r_out,
              int64_t *n_s_out) {
    if (check_rs(r, s)) return -1;
    og g = {n, rp, col};
    rtable T;
    if (rtable_build(&g, r, &T)) return -2;
    if (counts) memset(counts, 0, (size_t)T.count * sizeof(int64_t));
    int64_t *tmp = counts;
    if (!tmp) tmp = (int64_t *)calloc((size_t)(T.count > 0 ? T.count : 1), sizeof(int64_t));
    count_ctx C = {&T, s, tmp, 0, 0};
    int rc = list_all(&g, s, count_func, &C);
    if (n_r_out) *n_r_out = T.count;
    if (n_s_out) *n_s_out = C.n_s;
    if (!counts) free(tmp);
    free(T.t);
    if (rc) return -2;
    return C.bad ? -3 : 0;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2, peeling loop with Update / Update-Func.                        */

typedef struct {
    const og *g;
    const rtable *T;
    int r, s;
    i128 *cnt;        /* count * L */
    const int32_t *round; /* -1 = not peeled; t = in A this round; < t earlier */
    int32_t t;
    int64_t L;
    int32_t R[8];
    int64_t cur;      /* id of R */
    int bad;
    int64_t listed;   /* s-cliques re-listed by Update */
    int64_t live;     /* of those, the ones with no r-subset peeled in an earlier round */
    int64_t decs;     /* r-subsets outside A whose count a live S lowers (once per S and member) */
} update_ctx;

/* Update-Func on the s-clique S = R u C (C is an (s-r)-clique in I). */
static void update_func(update_ctx *U, const int32_t *Cset) {
    int32_t S[8];
    /* merge R and C into one ascending tuple */
    int i = 0, j = 0, k = 0, r = U->r, c = U->s - U->r;
    while (i < r || j < c) {
        if (j >= c || (i < r && U->R[i] < Cset[j]))
            S[k++] = U->R[i++];
        else
            S[k++] = Cset[j++];
    }
    U->listed++;
    int64_t ids[128];
    int nsub = subsets_of(U->T, U->s, S, ids);
    int a = 0;
    for (int q = 0; q < nsub; ++q) {
        if (ids[q] < 0) {
            U->bad = 1;
            return;
        }
        if (U->round[ids[q]] == U->t) a++;
    }
    /* U' = r-subsets not in A; return if any of them was peeled in an earlier round */
    for (int q = 0; q < nsub; ++q) {
        int32_t rq = U->round[ids[q]];
        if (rq != U->t && rq >= 0) return;
    }
    U->live++;
    /* the a members of A each list S; count S's surviving members once */
    {
        int64_t first = -1;
        for (int q = 0; q < nsub; ++q)
            if (U->round[ids[q]] == U->t && (first < 0 || ids[q] < first)) first = ids[q];
        if (first == U->cur) U->decs += nsub - a;
    }
    /* subtract 1/a from every r-subset outside A (exactly: L/a on the scaled count) */
    for (int q = 0; q < nsub; ++q)
        if (U->round[ids[q]] != U->t) U->cnt[ids[q]] -= (i128)(U->L / a);
}

/* rec-list-cliques over I for the remaining s-r vertices, ascending ids */
static void update_grow(update_ctx *U, int32_t *Cset, int depth, const int32_t *I, int64_t nI, int32_t **bufs) {
    int need = U->s - U->r;
    if (depth == need) {
        update_func(U, Cset);
        return;
    }
    for (int64_t i = 0; i < nI; ++i) {
        int32_t v = I[i];
        Cset[depth] = v;
        if (depth + 1 == need) {
            update_func(U, Cset);
            continue;
        }
        int32_t *next = bufs[depth + 1];
        int64_t nn = intersect_after(U->g, I, i, nI, v, next);
        update_grow(U, Cset, depth + 1, next, nn, bufs);
    }
}

/* core: int32[n_r]; round: int32[n_r] or NULL (round in which each r-clique is peeled);
 * sizes/levels: int64[cap] or NULL (|A| and k of each round). rho_out: number of rounds.
 * Returns 0, -1 (bad r,s), -2 (no memory), -3 (internal inconsistency). */
int orc_decompose(int32_t n, const int64_t *rp, const int32_t *col, int r, int s, int32_t *core, int32_t *round_out,
                  int64_t *rho_out, int64_t *sizes, int64_t *levels, int64_t cap, int64_t *n_s_out,
                  int64_t *listed_out, int64_t *live_out, int64_t *decs_out) {
    if (check_rs(r, s)) return -1;
    og g = {n, rp, col};
    rtable T;
    if (rtable_build(&g, r, &T)) return -2;
    int64_t nr = T.count;
    int64_t *c0 = (int64_t *)calloc((size_t)(nr > 0 ? nr : 1), sizeof(int64_t));
    i128 *cnt = (i128 *)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(i128));
    int32_t *round = (int32_t *)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int32_t));
    int64_t *A = (int64_t *)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
    int64_t maxd = 0;
    for (int32_t v = 0; v < n; ++v)
        if (deg(&g, v) > maxd) maxd = deg(&g, v);
    int32_t *bufs[9];
    int okb = 1;
    for (int d = 0; d <= 8; ++d) {
        bufs[d] = (int32_t *)malloc((size_t)(maxd + 1) * sizeof(int32_t));
        if (!bufs[d]) okb = 0;
    }
    int rc = 0;
    if (!c0 || !cnt || !round || !A || !okb) {
        rc = -2;
        goto done;
    }
    /* Count-Func over all s-cliques */
    count_ctx C = {&T, s, c0, 0, 0};
    if (list_all(&g, s, count_func, &C)) {
        rc = -2;
        goto done;
    }
    if (C.bad) {
        rc = -3;
        goto done;
    }
    if (n_s_out) *n_s_out = C.n_s;
    /* L = lcm(1..C(s,r)) */
    int64_t L = 1, csr = binom(s, r);
    for (int64_t q = 2; q <= csr; ++q) L = L / gcd64(L, q) * q;
    for (int64_t i = 0; i < nr; ++i) {
        cnt[i] = (i128)c0[i] * L;
        round[i] = -1;
    }
    update_ctx U;
    memset(&U, 0, sizeof(U));
    U.g = &g;
    U.T = &T;
    U.r = r;
    U.s = s;
    U.cnt = cnt;
    U.round = round;
    U.L = L;
    int64_t finished = 0, k = 0;
    int32_t t = 0;
    while (finished < nr) {
        /* the next bucket: k = max(k, min count over unpeeled); A = unpeeled with count <= k */
        i128 mn = -1;
        for (int64_t i = 0; i < nr; ++i)
            if (round[i] < 0 && (mn < 0 || cnt[i] < mn)) mn = cnt[i];
        if (mn % L != 0) {
            rc = -3;
            goto done;
        }
        if ((int64_t)(mn / L) > k) k = (int64_t)(mn / L);
        int64_t na = 0;
        for (int64_t i = 0; i < nr; ++i)
            if (round[i] < 0 && cnt[i] <= (i128)k * L) {
                A[na++] = i;
                round[i] = t;
            }
        finished += na;
        if (sizes && t < cap) sizes[t] = na;
        if (levels && t < cap) levels[t] = k;
        /* Update(G, DG, A, T) */
        U.t = t;
        for (int64_t q = 0; q < na; ++q) {
            const int32_t *Rt = T.t + A[q] * r;
            memcpy(U.R, Rt, (size_t)r * sizeof(int32_t));
            U.cur = A[q];
            /* I = intersection of the undirected neighbourhoods of R's vertices */
            int32_t v0 = Rt[0];
            for (int j = 1; j < r; ++j)
                if (deg(&g, Rt[j]) < deg(&g, v0)) v0 = Rt[j];
            int64_t nI = 0;
            const int32_t *nb = g.col + g.rp[v0];
            for (int64_t j = 0; j < deg(&g, v0); ++j) {
                int32_t w = nb[j], all = 1;
                for (int x = 0; x < r && all; ++x)
                    if (Rt[x] == w || !adjacent(&g, Rt[x], w)) all = 0;
                if (all) bufs[0][nI++] = w;
            }
            int32_t Cset[8];
            update_grow(&U, Cset, 0, bufs[0], nI, bufs);
            if (U.bad) {
                rc = -3;
                goto done;
            }
        }
        for (int64_t q = 0; q < na; ++q) core[A[q]] = (int32_t)k;
        if (k > INT32_MAX) {
            rc = -3;
            goto done;
        }
        t++;
    }
    if (round_out) memcpy(round_out, round, (size_t)nr * sizeof(int32_t));
    if (rho_out) *rho_out = t;
    if (listed_out) *listed_out = U.listed;
    if (live_out) *live_out = U.live;
    if (decs_out) *decs_out = U.decs;
done:
    free(c0);
    free(cnt);
    free(round);
    free(A);
    for (int d = 0; d <= 8; ++d) free(bufs[d]);
    free(T.t);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* The definition, written out: for c = 1, 2, ..., X_c is the largest set of r-cliques
 * in which every member lies in at least c s-cliques whose r-subsets are all in X_c.
 * It is the greatest fixpoint of "remove every member with support < c", started from
 * X_{c-1} (the nuclei are nested). core(R) = the largest c with R in X_c (0 if none).
 * Holds all s-cliques in memory: for small graphs only. */

typedef struct {
    const rtable *T;
    int s, nsub;
    int64_t *subs;
    int64_t n_s, cap;
    int bad;
} slist_ctx;

static void slist_add(void *vctx, const int32_t *S) {
    slist_ctx *C = (slist_ctx *)vctx;
    if (C->cap < 0) return;
    if (C->n_s == C->cap) {
        int64_t nc = C->cap ? 2 * C->cap : 1024;
        int64_t *ns = (int64_t *)realloc(C->subs, (size_t)nc * C->nsub * sizeof(int64_t));
        if (!ns) {
            C->cap = -1;
            return;
        }
        C->subs = ns;
        C->cap = nc;
    }
    int k = subsets_of(C->T, C->s, S, C->subs + C->n_s * C->nsub);
    for (int i = 0; i < k; ++i)
        if (C->subs[C->n_s * C->nsub + i] < 0) C->bad = 1;
    C->n_s++;
}

int orc_decompose_fixpoint(int32_t n, const int64_t *rp, const int32_t *col, int r, int s, int32_t *core) {
    if (check_rs(r, s)) return -1;
    og g = {n, rp, col};
    rtable T;
    if (rtable_build(&g, r, &T)) return -2;
    int64_t nr = T.count;
    slist_ctx C = {&T, s, (int)binom(s, r), NULL, 0, 0, 0};
    int rc = 0;
    unsigned char *inX = (unsigned char *)malloc((size_t)(nr > 0 ? nr : 1));
    int64_t *sup = (int64_t *)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
    if (!inX || !sup || list_all(&g, s, slist_add, &C) || C.cap < 0) {
        rc = -2;
        goto done;
    }
    if (C.bad) {
        rc = -3;
        goto done;
    }
    for (int64_t i = 0; i < nr; ++i) {
        inX[i] = 1;
        core[i] = 0;
    }
    int64_t alive = nr;
    for (int64_t c = 1; alive > 0; ++c) {
        int changed = 1;
        while (changed) {
            changed = 0;
            memset(sup, 0, (size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
            for (int64_t q = 0; q < C.n_s; ++q) {
                const int64_t *ids = C.subs + q * C.nsub;
                int all = 1;
                for (int i = 0; i < C.nsub; ++i)
                    if (!inX[ids[i]]) all = 0;
                if (all)
                    for (int i = 0; i < C.nsub; ++i) sup[ids[i]]++;
            }
            for (int64_t i = 0; i < nr; ++i)
                if (inX[i] && sup[i] < c) {
                    inX[i] = 0;
                    alive--;
                    changed = 1;
                }
        }
        for (int64_t i = 0; i < nr; ++i)
            if (inX[i]) core[i] = (int32_t)c;
    }
done:
    free(inX);
    free(sup);
    free(C.subs);
    free(T.t);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Certificate of a claimed decomposition (core, peel round per r-clique), checked on the
 * r-cliques listed in ids[0..nids):
 *   validity:  #{S containing R : every r-subset R' of S has core[R'] >= core[R]} >= core[R]
 *   order:     #{S containing R : every r-subset R' of S has round[R'] >= round[R]} <= core[R]
 * plus: core is non-decreasing in round (checked by the caller over all ids). If both hold
 * for every r-clique, the claimed core numbers are the exact ones: validity makes each
 * {R : core[R] >= c} a feasible set for c, so core is a lower bound, and the order
 * condition rules out any r-clique whose true core number exceeds its claim.
 * tuples: int32[nids * r], the ascending vertex tuple of each checked r-clique (the caller
 * decodes ids); id lookups of the other r-subsets go through lookup (canonical ids).
 * Writes per checked r-clique: sup_valid[i], sup_order[i]. */
typedef int64_t (*orc_lookup_fn)(const int32_t *tuple, void *user);

typedef struct {
    const og *g;
    int r, s;
    const int32_t *core, *round;
    int32_t R[8];
    int32_t cR, tR;
    int64_t valid, order;
    orc_lookup_fn lookup;
    void *user;
    int bad;
} cert_ctx;

static void cert_func(cert_ctx *K, const int32_t *Cset) {
    int32_t S[8], sub[8];
    int i = 0, j = 0, k = 0, r = K->r, c = K->s - K->r;
    while (i < r || j < c) {
        if (j >= c || (i < r && K->R[i] < Cset[j]))
            S[k++] = K->R[i++];
        else
            S[k++] = Cset[j++];
    }
    int okv = 1, oko = 1;
    for (unsigned mask = 0; mask < (1u << K->s); ++mask) {
        if (__builtin_popcount(mask) != r) continue;
        int q = 0;
        for (int b = 0; b < K->s; ++b)
            if (mask >> b & 1u) sub[q++] = S[b];
        int64_t id = K->lookup(sub, K->user);
        if (id < 0) {
            K->bad = 1;
            return;
        }
        if (K->core[id] < K->cR) okv = 0;
        if (K->round[id] < K->tR) oko = 0;
    }
    K->valid += okv;
    K->order += oko;
}

static void cert_grow(cert_ctx *K, int32_t *Cset, int depth, const int32_t *I, int64_t nI, int32_t **bufs) {
    int need = K->s - K->r;
    if (depth == need) {
        cert_func(K, Cset);
        return;
    }
    for (int64_t i = 0; i < nI; ++i) {
        int32_t v = I[i];
        Cset[depth] = v;
        if (depth + 1 == need) {
            cert_func(K, Cset);
            continue;
        }
        int32_t *next = bufs[depth + 1];
        int64_t nn = intersect_after(K->g, I, i, nI, v, next);
        cert_grow(K, Cset, depth + 1, next, nn, bufs);
    }
}

int orc_certify(int32_t n, const int64_t *rp, const int32_t *col, int r, int s, const int32_t *core,
                const int32_t *round, const int64_t *ids, const int32_t *tuples, int64_t nids, orc_lookup_fn lookup,
                void *user, int64_t *sup_valid, int64_t *sup_order) {
    if (check_rs(r, s)) return -1;
    og g = {n, rp, col};
    int64_t maxd = 0;
    for (int32_t v = 0; v < n; ++v)
        if (deg(&g, v) > maxd) maxd = deg(&g, v);
    int32_t *bufs[9];
    int rc = 0;
    for (int d = 0; d <= 8; ++d) bufs[d] = (int32_t *)malloc((size_t)(maxd + 1) * sizeof(int32_t));
    for (int d = 0; d <= 8; ++d)
        if (!bufs[d]) rc = -2;
    cert_ctx K;
    memset(&K, 0, sizeof(K));
    K.g = &g;
    K.r = r;
    K.s = s;
    K.core = core;
    K.round = round;
    K.lookup = lookup;
    K.user = user;
    for (int64_t q = 0; q < nids && rc == 0; ++q) {
        memcpy(K.R, tuples + q * r, (size_t)r * sizeof(int32_t));
        K.cR = core[ids[q]];
        K.tR = round[ids[q]];
        K.valid = 0;
        K.order = 0;
        int32_t v0 = K.R[0];
        for (int j = 1; j < r; ++j)
            if (deg(&g, K.R[j]) < deg(&g, v0)) v0 = K.R[j];
        int64_t nI = 0;
        const int32_t *nb = g.col + g.rp[v0];
        for (int64_t j = 0; j < deg(&g, v0); ++j) {
            int32_t w = nb[j], all = 1;
            for (int x = 0; x < r && all; ++x)
                if (K.R[x] == w || !adjacent(&g, K.R[x], w)) all = 0;
            if (all) bufs[0][nI++] = w;
        }
        int32_t Cset[8];
        cert_grow(&K, Cset, 0, bufs[0], nI, bufs);
        if (K.bad) rc = -3;
        sup_valid[q] = K.valid;
        sup_order[q] = K.order;
    }
    for (int d = 0; d <= 8; ++d) free(bufs[d]);
    return rc;
}

/* Number of s-cliques containing each of the given r-cliques (tuples int32[nids*r]),
 * computed one by one from the definition: I = common neighbourhood of R, then the
 * (s-r)-cliques inside I. Used for sampled checks on graphs too large for orc_count. */
typedef struct {
    const og *g;
    int need;
    int64_t found;
} local_ctx;

static void local_grow(local_ctx *K, int depth, const int32_t *I, int64_t nI, int32_t **bufs) {
    if (depth == K->need) {
        K->found++;
        return;
    }
    if (depth + 1 == K->need) {
        K->found += nI;
        return;
    }
    for (int64_t i = 0; i < nI; ++i) {
        int32_t v = I[i];
        int32_t *next = bufs[depth + 1];
        int64_t nn = intersect_after(K->g, I, i, nI, v, next);
        local_grow(K, depth + 1, next, nn, bufs);
    }
}

int orc_local_counts(int32_t n, const int64_t *rp, const int32_t *col, int r, int s, const int32_t *tuples,
                     int64_t nids, int64_t *out) {
    if (check_rs(r, s)) return -1;
    og g = {n, rp, col};
    int64_t maxd = 0;
    for (int32_t v = 0; v < n; ++v)
        if (deg(&g, v) > maxd) maxd = deg(&g, v);
    int32_t *bufs[9];
    int rc = 0;
    for (int d = 0; d <= 8; ++d) bufs[d] = (int32_t *)malloc((size_t)(maxd + 1) * sizeof(int32_t));
    for (int d = 0; d <= 8; ++d)
        if (!bufs[d]) rc = -2;
    local_ctx K = {&g, s - r, 0};
    for (int64_t q = 0; q < nids && rc == 0; ++q) {
        const int32_t *R = tuples + q * r;
        int32_t v0 = R[0];
        for (int j = 1; j < r; ++j)
            if (deg(&g, R[j]) < deg(&g, v0)) v0 = R[j];
        int64_t nI = 0;
        const int32_t *nb = g.col + g.rp[v0];
        for (int64_t j = 0; j < deg(&g, v0); ++j) {
            int32_t w = nb[j], all = 1;
            for (int x = 0; x < r && all; ++x)
                if (R[x] == w || !adjacent(&g, R[x], w)) all = 0;
            if (all) bufs[0][nI++] = w;
        }
        K.found = 0;
        local_grow(&K, 0, bufs[0], nI, bufs);
        out[q] = K.found;
    }
    for (int d = 0; d <= 8; ++d) free(bufs[d]);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Certificate over every r-clique (or a sample), parallel, for graphs where  */
/* the peeling loop above is far too slow.                                    */
/*
 * What it checks is the same pair of conditions as orc_certify above, which together prove
 * a claimed (core, round) exact without running Algorithm 2 (Section 2 definition):
 *   validity:  #{S containing R : every r-subset R' of S has core[R'] >= core[R]} >= core[R];
 *   order:     #{S containing R : every r-subset R' of S has round[R'] >= round[R]} <= core[R];
 *   level:     core[R] == levels[round[R]], and levels[] is non-decreasing.
 * Validity makes {R : core[R] >= c} a set in which every member has support >= c, so the true
 * core number is at least the claim. For the converse take the true c-nucleus X of any R*;
 * its first member R0 to be peeled (round t0) still has all of X in rounds >= t0, so the order
 * count of R0 is at least c, hence levels[t0] = core[R0] >= c, and every member of X (R*
 * included) is peeled at a level >= levels[t0] >= c.
 *
 * Ids are looked up in a trie of ascending tuples built here (level 1: vertices; level j+1:
 * for each j-clique K with largest vertex x, the vertices w > x adjacent to all of K, in
 * ascending order). The position of an r-tuple in level r is its rank in the lexicographic
 * order of all r-cliques, i.e. the canonical id. The s-cliques are listed once each along a
 * (degree, id) order of the vertices (Section 3, orientation) and sorted before the lookups.
 * The loops over listing roots and over sampled r-cliques are split across threads (OpenMP
 * when compiled with it); the arithmetic is the same either way.
 */
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int r;              /* levels 1..r */
    int64_t cnt[9];     /* entries per level */
    int64_t *off[9];    /* off[j][i] .. off[j][i+1]: children (level j+1) of entry i of level j */
    int32_t *val[9];    /* val[j][i]: the last vertex of entry i of level j */
} trie;

static void trie_free(trie *T) {
    for (int j = 0; j <= 8; ++j) {
        free(T->off[j]);
        free(T->val[j]);
    }
}

/* vertices of entry i of level j (ascending), found by walking up with binary searches */
static void trie_tuple(const trie *T, int j, int64_t i, int32_t *out) {
    for (int lv = j; lv >= 1; --lv) {
        out[lv - 1] = T->val[lv][i];
        if (lv == 1) break;
        /* parent = largest p with off[lv-1][p] <= i */
        int64_t lo = 0, hi = T->cnt[lv - 1];
        while (hi - lo > 1) {
            int64_t mid = lo + (hi - lo) / 2;
            if (T->off[lv - 1][mid] <= i)
                lo = mid;
            else
                hi = mid;
        }
        i = lo;
    }
}

static int64_t trie_children(const og *g, const int32_t *K, int j, int32_t *out) {
    /* vertices w > K[j-1] adjacent to all of K[0..j): walk the neighbours above K[j-1] of the
     * member with the fewest neighbours and test adjacency to the others */
    int32_t x = K[j - 1], y0 = K[0];
    for (int y = 1; y < j; ++y)
        if (deg(g, K[y]) < deg(g, y0)) y0 = K[y];
    const int32_t *nb = g->col + g->rp[y0];
    int64_t d = deg(g, y0), c = 0;
    int64_t lo = 0, hi = d; /* first neighbour of y0 above x */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (nb[mid] <= x)
            lo = mid + 1;
        else
            hi = mid;
    }
    for (int64_t q = lo; q < d; ++q) {
        int32_t w = nb[q];
        int all = 1;
        for (int y = 0; y < j && all; ++y)
            if (K[y] != y0) all = adjacent(g, K[y], w);
        if (all) {
            if (out) out[c] = w;
            c++;
        }
    }
    return c;
}

static int trie_build(const og *g, int r, trie *T) {
    memset(T, 0, sizeof(*T));
    T->r = r;
    T->cnt[1] = g->n;
    T->val[1] = (int32_t *)malloc((size_t)(g->n > 0 ? g->n : 1) * sizeof(int32_t));
    if (!T->val[1]) return -2;
    for (int32_t v = 0; v < g->n; ++v) T->val[1][v] = v;
    for (int j = 1; j < r; ++j) {
        int64_t nj = T->cnt[j];
        int64_t *off = (int64_t *)malloc((size_t)(nj + 1) * sizeof(int64_t));
        if (!off) return -2;
        T->off[j] = off;
        int bad = 0;
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < nj; ++i) {
            int32_t K[8];
            trie_tuple(T, j, i, K);
            off[i + 1] = trie_children(g, K, j, NULL);
        }
        off[0] = 0;
        for (int64_t i = 0; i < nj; ++i) off[i + 1] += off[i];
        T->cnt[j + 1] = off[nj];
        T->val[j + 1] = (int32_t *)malloc((size_t)(off[nj] > 0 ? off[nj] : 1) * sizeof(int32_t));
        if (!T->val[j + 1]) return -2;
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < nj; ++i) {
            int32_t K[8];
            trie_tuple(T, j, i, K);
            int64_t c = trie_children(g, K, j, T->val[j + 1] + off[i]);
            if (c != off[i + 1] - off[i]) bad = 1;
        }
        if (bad) return -3;
    }
    return 0;
}

/* canonical id of the ascending r-tuple x, or -1 if x is not an r-clique */
static int64_t trie_find(const trie *T, const int32_t *x) {
    if (x[0] < 0 || x[0] >= T->cnt[1]) return -1;
    int64_t i = x[0];
    for (int j = 1; j < T->r; ++j) {
        int64_t lo = T->off[j][i], hi = T->off[j][i + 1];
        const int32_t *a = T->val[j + 1];
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (a[mid] < x[j])
                lo = mid + 1;
            else
                hi = mid;
        }
        if (lo >= T->off[j][i + 1] || a[lo] != x[j]) return -1;
        i = lo;
    }
    return i;
}

typedef struct {
    const og *g;
    const trie *T;
    int r, s;
    const int32_t *core, *round;
    int32_t *valid, *order; /* full mode: per r-clique tallies (atomic adds) */
    int32_t R[8];           /* sample mode: the r-clique being checked */
    int32_t cR, tR;
    int64_t v_one, o_one;   /* sample mode tallies */
    int sample;
    int bad;
} fcert;

static void isort(int32_t *a, int n) {
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && a[j - 1] > a[j]; --j) {
            int32_t t = a[j];
            a[j] = a[j - 1];
            a[j - 1] = t;
        }
}

/* one s-clique S (ascending): look up its r-subsets, then tally */
static void fcert_s(fcert *K, const int32_t *S) {
    int64_t ids[128];
    int32_t sub[8];
    int k = 0, s = K->s, r = K->r;
    int32_t mc = INT32_MAX, mr = INT32_MAX;
    for (unsigned mask = 0; mask < (1u << s); ++mask) {
        if (__builtin_popcount(mask) != r) continue;
        int q = 0;
        for (int b = 0; b < s; ++b)
            if (mask >> b & 1u) sub[q++] = S[b];
        int64_t id = trie_find(K->T, sub);
        if (id < 0) {
            K->bad = 1;
            return;
        }
        ids[k++] = id;
        if (K->core[id] < mc) mc = K->core[id];
        if (K->round[id] < mr) mr = K->round[id];
    }
    if (K->sample) {
        K->v_one += mc >= K->cR;
        K->o_one += mr >= K->tR;
        return;
    }
    for (int q = 0; q < k; ++q) {
        if (mc >= K->core[ids[q]]) __atomic_fetch_add(&K->valid[ids[q]], 1, __ATOMIC_RELAXED);
        if (mr >= K->round[ids[q]]) __atomic_fetch_add(&K->order[ids[q]], 1, __ATOMIC_RELAXED);
    }
}

/* full mode: every s-clique once, grown along the (degree, id) order; out-lists dg[] */
typedef struct {
    const int64_t *orp;
    const int32_t *ocol; /* out-neighbours (higher in the order), ascending ids */
} ograph;

static int64_t sorted_intersect(const int32_t *a, int64_t na, const int32_t *b, int64_t nb, int32_t *out) {
    int64_t i = 0, j = 0, c = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j])
            ++i;
        else if (a[i] > b[j])
            ++j;
        else {
            out[c++] = a[i];
            ++i;
            ++j;
        }
    }
    return c;
}

static void fcert_grow(fcert *K, const ograph *D, int32_t *S, int depth, const int32_t *I, int64_t nI,
                       int32_t **bufs) {
    if (depth == K->s) {
        int32_t t[8];
        memcpy(t, S, (size_t)K->s * sizeof(int32_t));
        isort(t, K->s);
        fcert_s(K, t);
        return;
    }
    for (int64_t i = 0; i < nI; ++i) {
        int32_t v = I[i];
        S[depth] = v;
        if (depth + 1 == K->s) {
            fcert_grow(K, D, S, depth + 1, NULL, 0, bufs);
            continue;
        }
        int64_t nn = sorted_intersect(I, nI, D->ocol + D->orp[v], D->orp[v + 1] - D->orp[v], bufs[depth + 1]);
        fcert_grow(K, D, S, depth + 1, bufs[depth + 1], nn, bufs);
    }
}

/* sample mode: the (s-r)-cliques in I = common neighbourhood of R, ascending growth */
static void fcert_grow_r(fcert *K, int32_t *Cset, int depth, const int32_t *I, int64_t nI, int32_t **bufs) {
    int need = K->s - K->r;
    if (depth == need) {
        int32_t S[8];
        int i = 0, j = 0, k = 0, r = K->r;
        while (i < r || j < need) {
            if (j >= need || (i < r && K->R[i] < Cset[j]))
                S[k++] = K->R[i++];
            else
                S[k++] = Cset[j++];
        }
        fcert_s(K, S);
        return;
    }
    for (int64_t i = 0; i < nI; ++i) {
        int32_t v = I[i];
        Cset[depth] = v;
        if (depth + 1 == need) {
            fcert_grow_r(K, Cset, depth + 1, NULL, 0, bufs);
            continue;
        }
        int64_t nn = intersect_after(K->g, I, i, nI, v, bufs[depth + 1]);
        fcert_grow_r(K, Cset, depth + 1, bufs[depth + 1], nn, bufs);
    }
}

static int deg_order_less(const og *g, int32_t a, int32_t b) {
    return deg(g, a) < deg(g, b) || (deg(g, a) == deg(g, b) && a < b);
}

/* Certificate of a claimed (core, round, levels) over every r-clique (ids == NULL) or over the
 * r-cliques ids[0..nids). n_r: number of r-cliques the claim covers (checked against the trie).
 * Outputs (each nullable): bad[0] validity failures, bad[1] order failures, bad[2] level
 * failures (core != levels[round], round outside [0, rho), or levels decreasing), bad[3] the
 * first failing id (-1 if none); sample mode also writes sup_valid[q], sup_order[q].
 * nthreads <= 0 uses the default. Returns 0, -1 (bad r,s), -2 (memory), -3 (a subset of an
 * s-clique is missing from the trie, or n_r does not match), -4 (r > 6). */
int orc_certify_all(int32_t n, const int64_t *rp, const int32_t *col, int r, int s, int64_t n_r, const int32_t *core,
                    const int32_t *round, const int64_t *levels, int64_t rho, const int64_t *ids, int64_t nids,
                    int nthreads, int64_t *bad, int64_t *sup_valid, int64_t *sup_order) {
    if (check_rs(r, s)) return -1;
    if (r > 6) return -4;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    og g = {n, rp, col};
    trie T;
    int rc = trie_build(&g, r, &T);
    if (rc) {
        trie_free(&T);
        return rc;
    }
    if (T.cnt[r] != n_r) {
        trie_free(&T);
        return -3;
    }
    int64_t nb[4] = {0, 0, 0, -1};
    for (int64_t t = 1; t < rho; ++t)
        if (levels[t] < levels[t - 1]) nb[2]++;
    int64_t maxd = 0;
    for (int32_t v = 0; v < n; ++v)
        if (deg(&g, v) > maxd) maxd = deg(&g, v);
    int err = 0;
    if (!ids) {
        int32_t *valid = (int32_t *)calloc((size_t)(n_r > 0 ? n_r : 1), sizeof(int32_t));
        int32_t *order = (int32_t *)calloc((size_t)(n_r > 0 ? n_r : 1), sizeof(int32_t));
        int64_t *orp = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
        int32_t *ocol = (int32_t *)malloc((size_t)(rp[n] / 2 > 0 ? rp[n] / 2 : 1) * sizeof(int32_t));
        if (!valid || !order || !orp || !ocol) err = -2;
        if (!err) {
            orp[0] = 0;
            for (int32_t v = 0; v < n; ++v) {
                int64_t c = 0;
                for (int64_t q = rp[v]; q < rp[v + 1]; ++q) c += deg_order_less(&g, v, col[q]);
                orp[v + 1] = orp[v] + c;
            }
            for (int32_t v = 0; v < n; ++v) {
                int64_t at = orp[v];
                for (int64_t q = rp[v]; q < rp[v + 1]; ++q)
                    if (deg_order_less(&g, v, col[q])) ocol[at++] = col[q];
            }
            ograph D = {orp, ocol};
#pragma omp parallel
            {
                fcert K;
                memset(&K, 0, sizeof(K));
                K.g = &g;
                K.T = &T;
                K.r = r;
                K.s = s;
                K.core = core;
                K.round = round;
                K.valid = valid;
                K.order = order;
                int32_t *bufs[9];
                int ok = 1;
                for (int d = 0; d <= 8; ++d) {
                    bufs[d] = (int32_t *)malloc((size_t)(maxd + 1) * sizeof(int32_t));
                    if (!bufs[d]) ok = 0;
                }
                if (!ok) {
#pragma omp atomic write
                    err = -2;
                }
#pragma omp for schedule(dynamic, 64)
                for (int32_t v = 0; v < n; ++v) {
                    if (!ok) continue;
                    int32_t S[8];
                    S[0] = v;
                    if (s == 1) continue;
                    fcert_grow(&K, &D, S, 1, ocol + orp[v], orp[v + 1] - orp[v], bufs);
                }
                if (K.bad) {
#pragma omp atomic write
                    err = -3;
                }
                for (int d = 0; d <= 8; ++d) free(bufs[d]);
            }
            for (int64_t R = 0; R < n_r && !err; ++R) {
                int f = 0;
                if (valid[R] < core[R]) {
                    nb[0]++;
                    f = 1;
                }
                if ((int64_t)order[R] > (int64_t)core[R]) {
                    nb[1]++;
                    f = 1;
                }
                if (round[R] < 0 || round[R] >= rho || levels[round[R]] != core[R]) {
                    nb[2]++;
                    f = 1;
                }
                if (f && nb[3] < 0) nb[3] = R;
            }
        }
        free(valid);
        free(order);
        free(orp);
        free(ocol);
    } else {
        int64_t first = INT64_MAX;
        int64_t b0 = 0, b1 = 0, b2 = 0;
#pragma omp parallel reduction(+ : b0, b1, b2) reduction(min : first)
        {
            fcert K;
            memset(&K, 0, sizeof(K));
            K.g = &g;
            K.T = &T;
            K.r = r;
            K.s = s;
            K.core = core;
            K.round = round;
            K.sample = 1;
            int32_t *bufs[9];
            int ok = 1;
            for (int d = 0; d <= 8; ++d) {
                bufs[d] = (int32_t *)malloc((size_t)(maxd + 1) * sizeof(int32_t));
                if (!bufs[d]) ok = 0;
            }
            if (!ok) {
#pragma omp atomic write
                err = -2;
            }
#pragma omp for schedule(dynamic, 16)
            for (int64_t q = 0; q < nids; ++q) {
                if (!ok) continue;
                int64_t id = ids[q];
                if (id < 0 || id >= n_r) {
                    K.bad = 1;
                    continue;
                }
                trie_tuple(&T, r, id, K.R);
                K.cR = core[id];
                K.tR = round[id];
                K.v_one = K.o_one = 0;
                int32_t v0 = K.R[0];
                for (int j = 1; j < r; ++j)
                    if (deg(&g, K.R[j]) < deg(&g, v0)) v0 = K.R[j];
                int64_t nI = 0;
                const int32_t *nbv = g.col + g.rp[v0];
                for (int64_t j = 0; j < deg(&g, v0); ++j) {
                    int32_t w = nbv[j], all = 1;
                    for (int x = 0; x < r && all; ++x)
                        if (K.R[x] == w || !adjacent(&g, K.R[x], w)) all = 0;
                    if (all) bufs[0][nI++] = w;
                }
                int32_t Cset[8];
                fcert_grow_r(&K, Cset, 0, bufs[0], nI, bufs);
                if (sup_valid) sup_valid[q] = K.v_one;
                if (sup_order) sup_order[q] = K.o_one;
                int f = 0;
                if (K.v_one < K.cR) {
                    b0++;
                    f = 1;
                }
                if (K.o_one > K.cR) {
                    b1++;
                    f = 1;
                }
                if (K.tR < 0 || K.tR >= rho || levels[K.tR] != K.cR) {
                    b2++;
                    f = 1;
                }
                if (f && id < first) first = id;
            }
            if (K.bad) {
#pragma omp atomic write
                err = -3;
            }
            for (int d = 0; d <= 8; ++d) free(bufs[d]);
        }
        nb[0] += b0;
        nb[1] += b1;
        nb[2] += b2;
        nb[3] = first == INT64_MAX ? -1 : first;
    }
    trie_free(&T);
    if (bad)
        for (int i = 0; i < 4; ++i) bad[i] = nb[i];
    return err;
}

/* ------------------------------------------------------------------------- */
/* Connectivity of a nucleus (Section 2, footnote: the original definition also requires the     */
/* r-cliques of a nucleus to be connected through s-cliques).                                    */
/*
 * For a level c, the r-cliques with core >= c form the c-(r,s) nucleus set X_c. Two of them are
 * joined when some s-clique contains both and all of that s-clique's r-subsets lie in X_c; the
 * connected nuclei at level c are the connected components of this relation. comp[R] receives the
 * smallest r-clique id of R's component (or -1 when core[R] < c); *n_comp the number of components.
 * Plain sequential union-find over every s-clique, listed once (Algorithm 1 growth).
 */
typedef struct {
    const rtable *T;
    int s;
    const int32_t *core;
    int32_t level;
    int64_t *parent;
    int bad;
} nuc_ctx;

static int64_t uf_root(int64_t *parent, int64_t x) {
    while (parent[x] != x) x = parent[x];
    return x;
}

static void nuc_func(void *vctx, const int32_t *S) {
    nuc_ctx *K = (nuc_ctx *)vctx;
    int64_t ids[128];
    int k = subsets_of(K->T, K->s, S, ids);
    for (int i = 0; i < k; ++i) {
        if (ids[i] < 0) {
            K->bad = 1;
            return;
        }
        if (K->core[ids[i]] < K->level) return; /* S is not inside X_c */
    }
    for (int i = 1; i < k; ++i) {
        int64_t a = uf_root(K->parent, ids[0]), b = uf_root(K->parent, ids[i]);
        if (a == b) continue;
        if (a < b)
            K->parent[b] = a;
        else
            K->parent[a] = b;
    }
}

int orc_nuclei(int32_t n, const int64_t *rp, const int32_t *col, int r, int s, const int32_t *core, int32_t level,
               int32_t *comp, int64_t *n_comp) {
    if (check_rs(r, s)) return -1;
    og g = {n, rp, col};
    rtable T;
    if (rtable_build(&g, r, &T)) return -2;
    int64_t nr = T.count;
    int64_t *parent = (int64_t *)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
    if (!parent) {
        free(T.t);
        return -2;
    }
    for (int64_t i = 0; i < nr; ++i) parent[i] = i;
    nuc_ctx K = {&T, s, core, level, parent, 0};
    int rc = list_all(&g, s, nuc_func, &K);
    int64_t nc = 0;
    for (int64_t i = 0; i < nr; ++i) {
        if (core[i] < level) {
            comp[i] = -1;
            continue;
        }
        int64_t root = uf_root(parent, i); /* the smallest id: unions always hang the larger root */
        comp[i] = (int32_t)root;
        if (root == i) nc++;
    }
    if (n_comp) *n_comp = nc;
    free(parent);
    free(T.t);
    if (rc) return -2;
    return K.bad ? -3 : 0;
}
