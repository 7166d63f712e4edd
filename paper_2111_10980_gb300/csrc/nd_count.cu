// s-clique counts per r-clique: Algorithm 2's Count-Func over every s-clique listed once by
// Algorithm 1 (rec-list-cliques) on the oriented graph DG.
//
// Two kernel shapes, one per kind of (r,s):
//   * s = r + 1  ((1,2), (2,3), (3,4)): the s-cliques containing R are R plus one vertex of
//     I(R) = ∩_{v in R} N(v), so count[R] = |I(R)|. One warp per r-clique intersects the two
//     shortest lists by merge path (or probes / bisects the longer one when it is much longer);
//     the result is written once, with no atomics.
//     For r = 3 the lists are the per-edge common-neighbour tables L(e) of the triangle index
//     (|L(e)| is the edge's triangle support, far shorter than the vertex degrees).
//   * s = r + 2  ((1,3), (2,4)): the s-cliques are listed once each over DG (Algorithm 1:
//     I' = I ∩ N_DG(v) at each level) and add 1 to each of their C(s,r) r-subsets (Count-Func),
//     with one aggregated atomic for an r-subset shared by a whole level: (1,3) one warp per
//     lowest vertex; (2,4) one warp per lowest DG edge, the pairs of its last level spread over the
//     lanes.
#include "nd_common.cuh"
#include "nd_gen.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;

int blocks_for_warps(int64_t items) {
    int64_t want = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    int64_t cap = (int64_t)nd_sm_count() * 16;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

__device__ __forceinline__ int64_t gwarp() { return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int64_t nwarps() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }

__device__ __forceinline__ int warp_sum(int v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <typename CT>
__global__ void k_count12(GraphView g, CT* __restrict__ cnt) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x)
        cnt[v] = (CT)(g.rp[v + 1] - g.rp[v]);
}

// count[e] = |N(a) ∩ N(b)|
template <typename CT>
__global__ void k_count23(GraphView g, CT* __restrict__ cnt) {
    int lane = threadIdx.x & 31;
    for (int64_t e = gwarp(); e < g.m; e += nwarps()) {
        int32_t a = g.eu[e], b = g.ev[e];
        int64_t ab = g.rp[a], ae = g.rp[a + 1], bb = g.rp[b], be = g.rp[b + 1];
        const int32_t *xs = g.col + ab, *ys = g.col + bb;
        int64_t nx = ae - ab, ny = be - bb;
        if (nx > ny) {
            const int32_t* t = xs;
            xs = ys;
            ys = t;
            int64_t tn = nx;
            nx = ny;
            ny = tn;
        }
        int c = 0;
        if (nd_prefer_merge(nx, ny))
            c = nd_merge_count(xs, (int)nx, ys, (int)ny);
        else
            for (int64_t i = lane; i < nx; i += 32) c += nd_find(ys, ny, xs[i]) >= 0 ? 1 : 0;
        c = warp_sum(c);
        if (lane == 0) cnt[e] = (CT)c;
    }
}

// count[t] = |L(ab) ∩ L(ac) ∩ L(bc)|. Any two of the lists already intersect to the common
// neighbourhood of the triangle (L(ab) ∩ L(ac) = N(a) ∩ N(b) ∩ N(c)), so the two shortest suffice.
template <typename CT>
__global__ void k_count34(GraphView g, CT* __restrict__ cnt) {
    int lane = threadIdx.x & 31;
    for (int64_t t = gwarp(); t < g.n3; t += nwarps()) {
        int32_t e0 = g.tri_e[3 * t], e1 = g.tri_e[3 * t + 1], e2 = g.tri_e[3 * t + 2];
        int64_t b0 = g.et_rp[e0], n0 = g.et_rp[e0 + 1] - b0;
        int64_t b1 = g.et_rp[e1], n1 = g.et_rp[e1 + 1] - b1;
        int64_t b2 = g.et_rp[e2], n2 = g.et_rp[e2 + 1] - b2;
        // the two shortest lists: (b0, n0) drives, (b1, n1) is searched
        if (n1 < n0) {
            int64_t tb = b0, tn = n0;
            int32_t te = e0;
            b0 = b1, n0 = n1, e0 = e1, b1 = tb, n1 = tn, e1 = te;
        }
        if (n2 < n0) {
            int64_t tb = b0, tn = n0;
            int32_t te = e0;
            b0 = b2, n0 = n2, e0 = e2, b2 = tb, n2 = tn, e2 = te;
        }
        if (n2 < n1) b1 = b2, n1 = n2, e1 = e2;
        // the longer list is probed in the hash directory once it is more than about twice the
        // shorter (measured on R-MAT scale 20: the merge pays only below that; 1x, 4x and never
        // measured slower); without a table, the merge up to 8x and bisection beyond
        int c = 0;
        const bool probe = g.htab && nd_hashed(n1) && n1 > 2 * n0 + 64;
        if (!probe && nd_prefer_merge(n0, n1)) {
            c = nd_merge_count(g.et_w + b0, (int)n0, g.et_w + b1, (int)n1);
        } else if (probe) {
            // the long list has a hash directory: one probe instead of a bisection
            const NdHashSlot* tab = g.htab + g.hoff[e1];
            int k = nd_hash_bits(n1);
            int32_t id, rnd;
            for (int64_t i = lane; i < n0; i += 32) c += nd_hash_find(tab, k, g.et_w[b0 + i], id, rnd) ? 1 : 0;
        } else {
            for (int64_t i = lane; i < n0; i += 32) c += nd_find(g.et_w + b1, n1, g.et_w[b0 + i]) >= 0 ? 1 : 0;
        }
        c = warp_sum(c);
        if (lane == 0) cnt[t] = (CT)c;
    }
}

// (1,3): every triangle (u, v, w) of DG (u -> v, u -> w, v -> w) adds 1 to u, v and w.
template <typename CT>
__global__ void k_count13(GraphView g, CT* __restrict__ cnt) {
    int lane = threadIdx.x & 31;
    for (int64_t u = gwarp(); u < g.n; u += nwarps()) {
        int64_t ub = g.dg_rp[u], ue = g.dg_rp[u + 1];
        int cu = 0;
        for (int64_t jv = ub; jv < ue; ++jv) {
            int32_t v = g.dg_col[jv];
            int64_t vb = g.dg_rp[v], vn = g.dg_rp[v + 1] - vb;
            int cv = 0;
            for (int64_t i = ub + lane; i < ue; i += 32) {
                int32_t w = g.dg_col[i];
                if (nd_find(g.dg_col + vb, vn, w) >= 0) {
                    nd_atomic_add(&cnt[w], 1);
                    cv++;
                }
            }
            cv = warp_sum(cv);
            if (lane == 0 && cv) nd_atomic_add(&cnt[v], cv);
            cu += cv;
        }
        if (lane == 0 && cu) nd_atomic_add(&cnt[u], cu);
    }
}

// (2,4), one warp per DG edge u -> v: the 4-cliques whose two lowest vertices (in the orientation)
// are u and v are u, v plus a DG edge w -> x inside I = N_DG(u) ∩ N_DG(v). The warp stages I in
// shared memory (ascending ids, with the edge ids u-w and v-w and the out-list bounds of each w),
// numbers the candidate pairs (w, k-th out-neighbour of w) through a prefix sum of the out-degrees
// and spreads them evenly over its lanes; a lane finds x in the staged I by bisection and adds 1 to
// the 4-clique's edges w-x, u-x, v-x, u-w, v-w; u-v gets the warp's total once. An edge whose I does
// not fit the stage (more than kC24 vertices) is listed by the lanes walking out-lists instead.
constexpr int kC24 = 128;

__device__ __forceinline__ int stage_find24(const int32_t* a, int n, int32_t x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < n && a[lo] == x) ? lo : -1;
}

template <typename CT>
__global__ void __launch_bounds__(kThreads) k_count24_flat(GraphView g, CT* __restrict__ cnt) {
    __shared__ int32_t s_w[kWarpsPerBlock][kC24], s_eu[kWarpsPerBlock][kC24], s_ev[kWarpsPerBlock][kC24],
        s_b[kWarpsPerBlock][kC24], s_p[kWarpsPerBlock][kC24 + 1];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *sw = s_w[wid], *seu = s_eu[wid], *sev = s_ev[wid], *sb = s_b[wid], *sp = s_p[wid];
    for (int64_t j = gwarp(); j < g.m; j += nwarps()) {
        // u: the vertex whose out-list holds DG position j
        int64_t lo = 0, hi = g.n;
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (g.dg_rp[mid] <= j)
                lo = mid;
            else
                hi = mid;
        }
        const int32_t u = (int32_t)lo, v = g.dg_col[j], e_uv = g.dg_eid[j];
        const int64_t ub = g.dg_rp[u], ue = g.dg_rp[u + 1], vb = g.dg_rp[v], vn = g.dg_rp[v + 1] - vb;
        // stage I = N_DG(u) ∩ N_DG(v) in order
        int c = 0;
        for (int64_t p0 = ub; p0 < ue; p0 += 32) {
            int64_t p = p0 + lane;
            int64_t q = p < ue ? nd_find(g.dg_col + vb, vn, g.dg_col[p]) : -1;
            unsigned mk = __ballot_sync(full, q >= 0);
            if (q >= 0) {
                int at = c + __popc(mk & nd_lanemask_lt());
                if (at < kC24) {
                    int32_t w = g.dg_col[p];
                    sw[at] = w;
                    seu[at] = g.dg_eid[p];
                    sev[at] = g.dg_eid[vb + q];
                    sb[at] = (int32_t)g.dg_rp[w];
                    sp[at] = (int32_t)(g.dg_rp[w + 1] - g.dg_rp[w]);
                }
            }
            c += __popc(mk);
        }
        __syncwarp();
        unsigned long long c_uv = 0;
        if (c <= kC24) {
            // exclusive prefix of the out-degrees (c <= kC24: at most four 32-wide chunks)
            int32_t carry = 0;
            for (int c0 = 0; c0 < c; c0 += 32) {
                int i = c0 + lane;
                int32_t d = i < c ? sp[i] : 0, inc = d;
                for (int o = 1; o < 32; o <<= 1) {
                    int32_t y = __shfl_up_sync(full, inc, o);
                    if (lane >= o) inc += y;
                }
                if (i < c) sp[i] = carry + inc - d;
                carry += __shfl_sync(full, inc, 31);
            }
            if (lane == 0) sp[c] = carry;
            __syncwarp();
            for (int32_t p = lane; p < carry; p += 32) {
                int a = 0, b = c;  // owner: the last i with sp[i] <= p
                while (b - a > 1) {
                    int mid = (a + b) >> 1;
                    if (sp[mid] <= p)
                        a = mid;
                    else
                        b = mid;
                }
                int64_t jx = (int64_t)sb[a] + (p - sp[a]);
                int k = stage_find24(sw, c, g.dg_col[jx]);
                if (k < 0) continue;
                ++c_uv;
                nd_atomic_add(&cnt[g.dg_eid[jx]], 1);
                nd_atomic_add(&cnt[seu[k]], 1);
                nd_atomic_add(&cnt[sev[k]], 1);
                nd_atomic_add(&cnt[seu[a]], 1);
                nd_atomic_add(&cnt[sev[a]], 1);
            }
        } else {
            // I does not fit the stage: the lanes take the w of N_DG(u) ∩ N_DG(v) and walk their
            // out-lists, searching x in both lists
            for (int64_t p = ub + lane; p < ue; p += 32) {
                int32_t w = g.dg_col[p];
                int64_t q = nd_find(g.dg_col + vb, vn, w);
                if (q < 0) continue;
                int32_t e_uw = g.dg_eid[p], e_vw = g.dg_eid[vb + q];
                for (int64_t jx = g.dg_rp[w]; jx < g.dg_rp[w + 1]; ++jx) {
                    int32_t x = g.dg_col[jx];
                    int64_t pux = nd_find(g.dg_col + ub, ue - ub, x);
                    if (pux < 0) continue;
                    int64_t pvx = nd_find(g.dg_col + vb, vn, x);
                    if (pvx < 0) continue;
                    ++c_uv;
                    nd_atomic_add(&cnt[g.dg_eid[jx]], 1);
                    nd_atomic_add(&cnt[g.dg_eid[ub + pux]], 1);
                    nd_atomic_add(&cnt[g.dg_eid[vb + pvx]], 1);
                    nd_atomic_add(&cnt[e_uw], 1);
                    nd_atomic_add(&cnt[e_vw], 1);
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) c_uv += __shfl_down_sync(full, c_uv, o);
        if (lane == 0 && c_uv) nd_atomic_add(&cnt[e_uv], (int64_t)c_uv);
        __syncwarp();
    }
}

// Any other supported (r,s) ((1,4), (2,5), (3,5), (3,6), (4,5), (4,6)): one warp per r-clique R counts the
// s-cliques containing it, listing the (s-r)-cliques of R's common neighbourhood from the entries
// of its driving list (nd_gen.cuh); written once, no atomics.
template <typename CT, int R_, int S_>
__global__ void k_count_gen(GraphView g, CT* __restrict__ cnt, int64_t n_r) {
    int lane = threadIdx.x & 31;
    for (int64_t id = gwarp(); id < n_r; id += nwarps()) {
        int32_t v[4];
        gen_verts<R_>(g, id, v);
        const int32_t* list = nullptr;
        int64_t len = 0;
        gen_drive<R_>(g, id, v, list, len);
        unsigned long long c = 0;
        for (int64_t j = lane; j < len; j += 32) gen_cand<R_, S_>(g, v, list[j], [&](const int32_t*) { ++c; });
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (lane == 0) cnt[id] = (CT)c;
    }
}

template <typename CT>
__global__ void k_zero(CT* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0;
}

}  // namespace

template <typename CT>
void nd_count_launch(const GraphView& g, int r, int s, CT* cnt, int64_t n_r, cudaStream_t st) {
    if (n_r <= 0) return;
    int blk = blocks_for_warps(n_r);
    if (r == 1 && s == 2) {
        ND_K(k_count12<CT><<<blk, kThreads, 0, st>>>(g, cnt));
    } else if (r == 2 && s == 3) {
        ND_K(k_count23<CT><<<blk, kThreads, 0, st>>>(g, cnt));
    } else if (r == 3 && s == 4) {
        ND_K(k_count34<CT><<<blk, kThreads, 0, st>>>(g, cnt));
    } else if (r == 1 && s == 3) {
        ND_K(k_zero<CT><<<blk, kThreads, 0, st>>>(cnt, n_r));
        ND_K(k_count13<CT><<<blocks_for_warps(g.n), kThreads, 0, st>>>(g, cnt));
    } else if (r == 2 && s == 4) {
        ND_K(k_zero<CT><<<blk, kThreads, 0, st>>>(cnt, n_r));
        ND_K(k_count24_flat<CT><<<blocks_for_warps(g.m), kThreads, 0, st>>>(g, cnt));
    } else if (r == 1 && s == 4) {
        ND_K(k_count_gen<CT, 1, 4><<<blk, kThreads, 0, st>>>(g, cnt, n_r));
    } else if (r == 2 && s == 5) {
        ND_K(k_count_gen<CT, 2, 5><<<blk, kThreads, 0, st>>>(g, cnt, n_r));
    } else if (r == 3 && s == 5) {
        ND_K(k_count_gen<CT, 3, 5><<<blk, kThreads, 0, st>>>(g, cnt, n_r));
    } else if (r == 3 && s == 6) {
        ND_K(k_count_gen<CT, 3, 6><<<blk, kThreads, 0, st>>>(g, cnt, n_r));
    } else if (r == 4 && s == 5) {
        ND_K(k_count_gen<CT, 4, 5><<<blk, kThreads, 0, st>>>(g, cnt, n_r));
    } else if (r == 4 && s == 6) {
        ND_K(k_count_gen<CT, 4, 6><<<blk, kThreads, 0, st>>>(g, cnt, n_r));
    }
}

template void nd_count_launch<int32_t>(const GraphView&, int, int, int32_t*, int64_t, cudaStream_t);
template void nd_count_launch<int64_t>(const GraphView&, int, int, int64_t*, int64_t, cudaStream_t);
