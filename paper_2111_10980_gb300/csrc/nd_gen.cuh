// Generic (r,s) listing for the counting and Update kernels of (r,s) without a dedicated kernel:
// r <= 4 and s - r <= 3 ((1,4), (2,5), (3,5), (3,6), (4,5), (4,6)). Algorithm 1 restricted to one r-clique R:
// the candidates are the entries w of R's driving list (r = 1: N(v); r = 2: the shorter of N(u),
// N(v); r = 3: the shortest of the triangle's three common-neighbour lists L(e)); w belongs to
// I = the common neighbourhood of R when it is adjacent to every vertex of R. The (s-r)-cliques C
// of I are listed once each along DG (w -> x -> y, every edge of C oriented forward), and every
// s-clique S = R + C is handed to a visitor. The ids of S's r-subsets come from the r-clique
// index: an edge (a < b) is the canonical id stored at b's position in N(a); a triangle
// (a < b < c) is the triangle id stored at c's entry in L(a,b).
#pragma once

#include "nd_common.cuh"

// the triangle whose children in the 4-clique index hold position q (largest t with qbase[t] <= q)
__device__ __forceinline__ int64_t gen_quad_parent(const GraphView& g, int64_t q) {
    int64_t lo = 0, hi = g.n3;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (g.qbase[mid] <= q)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// vertices of r-clique `id`, ascending
template <int R>
__device__ __forceinline__ void gen_verts(const GraphView& g, int64_t id, int32_t* v) {
    if (R == 1) {
        v[0] = (int32_t)id;
    } else if (R == 2) {
        v[0] = g.eu[id];
        v[1] = g.ev[id];
    } else {
        int64_t t = R == 4 ? gen_quad_parent(g, id) : id;
        int32_t e = g.tri_e[3 * t], e1 = g.tri_e[3 * t + 1];
        v[0] = g.eu[e];
        v[1] = g.ev[e];
        v[2] = g.ev[e1];
        if (R == 4) v[3] = g.qval[id];
    }
}

// position of b in N(a), or -1
__device__ __forceinline__ int64_t gen_pos(const GraphView& g, int32_t a, int32_t b) {
    int64_t lo = g.rp[a];
    int64_t i = nd_find(g.col + lo, g.rp[a + 1] - lo, b);
    return i < 0 ? -1 : lo + i;
}

__device__ __forceinline__ bool gen_adj(const GraphView& g, int32_t a, int32_t b) {
    if (g.rp[a + 1] - g.rp[a] > g.rp[b + 1] - g.rp[b]) {
        int32_t t = a;
        a = b;
        b = t;
    }
    return gen_pos(g, a, b) >= 0;
}

// canonical id of the ascending r-tuple t, or -1 if it is not an r-clique
template <int R>
__device__ __forceinline__ int64_t gen_id(const GraphView& g, const int32_t* t) {
    if (R == 1) return t[0];
    int64_t p = gen_pos(g, t[0], t[1]);
    if (p < 0) return -1;
    int64_t e = g.pos2e[p];
    if (R == 2) return e;
    int64_t lo = g.et_rp[e];
    int64_t i = nd_find(g.et_w + lo, g.et_rp[e + 1] - lo, t[2]);
    if (i < 0) return -1;
    int64_t tri = g.et_t[lo + i];
    if (R == 3) return tri;
    int64_t qb = g.qbase[tri];
    int64_t j = nd_find(g.qval + qb, g.qbase[tri + 1] - qb, t[3]);
    return j < 0 ? -1 : qb + j;
}

// the driving list of r-clique v (its candidates w)
template <int R>
__device__ __forceinline__ void gen_drive(const GraphView& g, int64_t id, const int32_t* v, const int32_t*& list,
                                          int64_t& len) {
    if (R == 1) {
        list = g.col + g.rp[v[0]];
        len = g.rp[v[0] + 1] - g.rp[v[0]];
    } else if (R == 2) {
        int64_t du = g.rp[v[0] + 1] - g.rp[v[0]], dv = g.rp[v[1] + 1] - g.rp[v[1]];
        int32_t x = du <= dv ? v[0] : v[1];
        list = g.col + g.rp[x];
        len = du <= dv ? du : dv;
    } else {
        // r = 3: the triangle's own lists; r = 4: the lists of its first three vertices' triangle
        int64_t t = R == 4 ? gen_quad_parent(g, id) : id;
        len = -1;
        for (int k = 0; k < 3; ++k) {
            int32_t e = g.tri_e[3 * t + k];
            int64_t n = g.et_rp[e + 1] - g.et_rp[e];
            if (len < 0 || n < len) {
                len = n;
                list = g.et_w + g.et_rp[e];
            }
        }
    }
}

// w is in the common neighbourhood of v (adjacent to all of v, and not one of them)
template <int R>
__device__ __forceinline__ bool gen_in(const GraphView& g, const int32_t* v, int32_t w) {
#pragma unroll
    for (int k = 0; k < R; ++k)
        if (v[k] == w || !gen_adj(g, v[k], w)) return false;
    return true;
}

// Every (S-R)-clique C of the common neighbourhood of v whose first vertex (in DG order) is the
// candidate w: visit(C, |C|) once per C (vertices in DG order, not sorted).
template <int R, int S, typename Visit>
__device__ __forceinline__ void gen_cand(const GraphView& g, const int32_t* v, int32_t w, Visit&& visit) {
    constexpr int K = S - R;
    if (!gen_in<R>(g, v, w)) return;
    int32_t C[3] = {w, 0, 0};
    if (K == 1) {
        visit(C);
        return;
    }
    for (int64_t jx = g.dg_rp[w]; jx < g.dg_rp[w + 1]; ++jx) {
        int32_t x = g.dg_col[jx];
        if (!gen_in<R>(g, v, x)) continue;
        C[1] = x;
        if (K == 2) {
            visit(C);
            continue;
        }
        for (int64_t jy = g.dg_rp[x]; jy < g.dg_rp[x + 1]; ++jy) {
            int32_t y = g.dg_col[jy];
            if (!gen_adj(g, w, y) || !gen_in<R>(g, v, y)) continue;
            C[2] = y;
            visit(C);
        }
    }
}

// S = v + C as an ascending tuple (|S| = S_ <= 6)
template <int R, int S>
__device__ __forceinline__ void gen_merge(const int32_t* v, const int32_t* C, int32_t* out) {
    constexpr int K = S - R;
    int32_t c[3] = {C[0], K > 1 ? C[1] : 0, K > 2 ? C[2] : 0};
    // sort C (at most 3 entries)
    if (K > 1 && c[1] < c[0]) { int32_t t = c[0]; c[0] = c[1]; c[1] = t; }
    if (K > 2 && c[2] < c[1]) { int32_t t = c[1]; c[1] = c[2]; c[2] = t; }
    if (K > 1 && c[1] < c[0]) { int32_t t = c[0]; c[0] = c[1]; c[1] = t; }
    int i = 0, j = 0;
#pragma unroll
    for (int k = 0; k < S; ++k) {
        bool take_v = j >= K || (i < R && v[i] < c[j]);
        out[k] = take_v ? v[i] : c[j];
        i += take_v;
        j += !take_v;
    }
}

constexpr int gen_binom(int n, int k) { return k < 0 || k > n ? 0 : (k == 0 || k == n ? 1 : gen_binom(n - 1, k - 1) + gen_binom(n - 1, k)); }

// ids of the r-subsets of the ascending s-tuple Sv other than v itself (C(s,r) - 1 of them);
// false if a lookup fails (inconsistent index)
template <int R, int S>
__device__ __forceinline__ bool gen_others(const GraphView& g, const int32_t* v, const int32_t* Sv, int32_t* o) {
    int n = 0;
    for (unsigned mask = 0; mask < (1u << S); ++mask) {
        if (__popc(mask) != R) continue;
        int32_t t[4];
        int q = 0;
        bool same = true;
#pragma unroll
        for (int b = 0; b < S; ++b)
            if (mask >> b & 1u) t[q++] = Sv[b];
#pragma unroll
        for (int k = 0; k < R; ++k) same = same && t[k] == v[k];
        if (same) continue;
        int64_t id = gen_id<R>(g, t);
        if (id < 0) return false;
        o[n++] = (int32_t)id;
    }
    return true;
}
