// Graph structure kernels: CSR validation, the canonical edge index (r = 2), the oriented
// graph DG (Section 3, O(alpha)-orientation; Algorithm 2, line "Orient") and the triangle
// index (r = 3; Sections 5.1-5.3: the per-edge last-level tables of the two-level T laid out
// contiguously with a prefix sum, and the inverse map from a triangle id to its edges).
//
// Layout choices for the GPU:
//   * vertex ids are never relabelled; DG's out-lists are order-preserving filters of the
//     sorted CSR rows, so every list stays sorted by vertex id and intersections of undirected
//     and oriented lists need no re-sort (the paper's relabelling, Section 5.4, is replaced by
//     this);
//   * the canonical edge id of (a<b) is its rank in CSR order, so per-edge outputs need no
//     permutation;
//   * L(a,b) stores every common neighbour w of a and b (all three edges of a triangle list
//     it), together with the triangle's canonical id; a triangle (a<b<c) gets id
//     tbase[e(a,b)] + rank of c among the entries of L(a,b) greater than b.
#include "nd_common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;

int blocks_for_warps(int64_t items) {
    int64_t want = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    int64_t cap = (int64_t)nd_sm_count() * 16;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

int blocks_for_threads(int64_t items) {
    int64_t want = (items + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)nd_sm_count() * 16;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

__device__ __forceinline__ int64_t gwarp() { return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int64_t nwarps() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }

// err bits: 1 row pointers not monotone, 2 id out of range, 4 row not strictly ascending,
// 8 self-loop, 16 missing reverse entry
__global__ void k_validate(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t n, int64_t nnz,
                           int* err) {
    int lane = threadIdx.x & 31;
    for (int64_t u = gwarp(); u < n; u += nwarps()) {
        int64_t b = rp[u], e = rp[u + 1];
        if (e < b || b < 0 || e > nnz) {
            if (lane == 0) atomicOr(err, 1);
            continue;
        }
        for (int64_t p = b + lane; p < e; p += 32) {
            int32_t v = col[p];
            if (v < 0 || v >= n) {
                atomicOr(err, 2);
                continue;
            }
            if (p > b && col[p - 1] >= v) atomicOr(err, 4);
            if (v == u) atomicOr(err, 8);
            int64_t vb = rp[v], ve = rp[v + 1];
            if (ve < vb || vb < 0 || ve > nnz || nd_find(col + vb, ve - vb, (int32_t)u) < 0) atomicOr(err, 16);
        }
    }
}

__global__ void k_split(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t n,
                        int64_t* __restrict__ split, int64_t* __restrict__ updeg) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = rp[u], e = rp[u + 1];
        int64_t s = b + nd_lower_bound(col + b, e - b, (int32_t)u + 1);
        split[u] = s;
        updeg[u] = e - s;
    }
}

// A CSR entry whose reverse entry is missing (or a self-loop) sets *err and gets edge id 0, so
// that no later kernel indexes outside the edge arrays.
__global__ void k_pos2e(GraphView g, int32_t* __restrict__ pos2e, int32_t* __restrict__ eu,
                        int32_t* __restrict__ ev, int* err) {
    int lane = threadIdx.x & 31;
    for (int64_t u = gwarp(); u < g.n; u += nwarps()) {
        int64_t b = g.rp[u], e = g.rp[u + 1];
        for (int64_t p = b + lane; p < e; p += 32) {
            int32_t v = g.col[p];
            int64_t id;
            if (v > u) {
                id = g.ebase[u] + (p - g.split[u]);
                eu[id] = (int32_t)u;
                ev[id] = v;
            } else {
                int64_t vb = g.rp[v], ve = g.rp[v + 1];
                int64_t q = vb + nd_lower_bound(g.col + vb, ve - vb, (int32_t)u);
                if (v == u || q >= ve || g.col[q] != (int32_t)u || q < g.split[v]) {
                    atomicOr(err, 1);
                    id = 0;
                } else {
                    id = g.ebase[v] + (q - g.split[v]);
                }
            }
            pos2e[p] = (int32_t)id;
        }
    }
}

__device__ __forceinline__ bool key_less(const int64_t* rp, const int32_t* key_hi, int32_t a, int32_t b) {
    int64_t ka = key_hi ? (int64_t)key_hi[a] : rp[a + 1] - rp[a];
    int64_t kb = key_hi ? (int64_t)key_hi[b] : rp[b + 1] - rp[b];
    return ka < kb || (ka == kb && a < b);
}

__global__ void k_dg_count(GraphView g, const int32_t* __restrict__ key_hi, int64_t* __restrict__ outdeg) {
    int lane = threadIdx.x & 31;
    for (int64_t u = gwarp(); u < g.n; u += nwarps()) {
        int64_t b = g.rp[u], e = g.rp[u + 1];
        int c = 0;
        for (int64_t p = b + lane; p < e; p += 32) c += key_less(g.rp, key_hi, (int32_t)u, g.col[p]) ? 1 : 0;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (lane == 0) outdeg[u] = c;
    }
}

__global__ void k_dg_fill(GraphView g, const int32_t* __restrict__ key_hi, const int64_t* __restrict__ dg_rp,
                          int32_t* __restrict__ dg_col, int32_t* __restrict__ dg_eid) {
    int lane = threadIdx.x & 31;
    for (int64_t u = gwarp(); u < g.n; u += nwarps()) {
        int64_t b = g.rp[u], e = g.rp[u + 1];
        int64_t out = dg_rp[u];
        for (int64_t p0 = b; p0 < e; p0 += 32) {
            int64_t p = p0 + lane;
            bool take = false;
            int32_t v = 0;
            if (p < e) {
                v = g.col[p];
                take = key_less(g.rp, key_hi, (int32_t)u, v);
            }
            unsigned m = __ballot_sync(0xffffffffu, take);
            if (take) {
                int64_t at = out + __popc(m & nd_lanemask_lt());
                dg_col[at] = v;
                dg_eid[at] = g.pos2e[p];
            }
            out += __popc(m);
        }
    }
}

// sigma[e] = |N(a) ∩ N(b)|, up[e] = |{w in N(a) ∩ N(b) : w > b}| for canonical edge e = (a,b)
__global__ void k_edge_support(GraphView g, int64_t* __restrict__ sigma, int64_t* __restrict__ up) {
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
        int c = 0, cu = 0;
        if (nd_prefer_merge(nx, ny)) {
            const int ix = (int)nx, iy = (int)ny;
            nd_merge_walk(xs, ix, ys, iy, nd_merge_run(xs, ix, ys, iy), [&](int, int, int32_t w) {
                c++;
                cu += w > b ? 1 : 0;
            });
        } else {
            for (int64_t i = lane; i < nx; i += 32) {
                int32_t w = xs[i];
                if (nd_find(ys, ny, w) >= 0) {
                    c++;
                    cu += (w > b) ? 1 : 0;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_down_sync(0xffffffffu, c, o);
            cu += __shfl_down_sync(0xffffffffu, cu, o);
        }
        if (lane == 0) {
            sigma[e] = c;
            up[e] = cu;
        }
    }
}

// Writes L(a,b) in ascending w with, per entry: the canonical triangle id when w > b, else
// (temporarily) the id of edge (a,w); and the edges of every triangle whose lowest edge is e.
__global__ void k_edge_fill(GraphView g, const int64_t* __restrict__ et_rp, const int64_t* __restrict__ tbase,
                            int32_t* __restrict__ et_w, int32_t* __restrict__ et_t, int32_t* __restrict__ tri_e,
                            int32_t* __restrict__ tri_pos) {
    int lane = threadIdx.x & 31;
    for (int64_t e = gwarp(); e < g.m; e += nwarps()) {
        int32_t a = g.eu[e], b = g.ev[e];
        int64_t ab = g.rp[a], ae = g.rp[a + 1], bb = g.rp[b], be = g.rp[b + 1];
        bool a_drives = (ae - ab) <= (be - bb);
        int64_t xb = a_drives ? ab : bb, xe = a_drives ? ae : be;
        int64_t yb = a_drives ? bb : ab, ye = a_drives ? be : ae;
        int64_t out = et_rp[e];
        int64_t sig = et_rp[e + 1] - out;
        int64_t split_e = sig - (tbase[e + 1] - tbase[e]);
        // writes common element w, found at driver position p and other-list position q, as entry
        // `local` of L(a,b)
        auto put = [&](int64_t local, int64_t p, int64_t q, int32_t w) {
            int64_t pa = a_drives ? p : q;  // position of w in N(a)
            int64_t pb = a_drives ? q : p;  // position of w in N(b)
            int32_t e_aw = g.pos2e[pa], e_bw = g.pos2e[pb];
            et_w[out + local] = w;
            if (w > b) {
                int64_t tid = tbase[e] + (local - split_e);
                et_t[out + local] = (int32_t)tid;
                tri_e[3 * tid + 0] = (int32_t)e;
                tri_e[3 * tid + 1] = e_aw;
                tri_e[3 * tid + 2] = e_bw;
                tri_pos[3 * tid + 0] = (int32_t)local;
            } else {
                et_t[out + local] = e_aw;
            }
        };
        if (nd_prefer_merge(xe - xb, ye - yb)) {
            // merge path: count this lane's matches, place them after the lower lanes' (exclusive
            // scan), then walk the run again and write them
            const int32_t *X = g.col + xb, *Y = g.col + yb;
            const int nx = (int)(xe - xb), ny = (int)(ye - yb);
            const NdMergeRun run = nd_merge_run(X, nx, Y, ny);
            int cnt = 0;
            nd_merge_walk(X, nx, Y, ny, run, [&](int, int, int32_t) { ++cnt; });
            int inc = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            int64_t local = inc - cnt;
            nd_merge_walk(X, nx, Y, ny, run, [&](int i, int j, int32_t w) { put(local++, xb + i, yb + j, w); });
        } else {
            int64_t pos = 0;
            for (int64_t p0 = xb; p0 < xe; p0 += 32) {
                int64_t p = p0 + lane;
                int64_t q = -1;
                if (p < xe) q = nd_find(g.col + yb, ye - yb, g.col[p]);
                unsigned m = __ballot_sync(0xffffffffu, q >= 0);
                if (q >= 0) put(pos + __popc(m & nd_lanemask_lt()), p, yb + q, g.col[p]);
                pos += __popc(m);
            }
        }
    }
}

// For entries of L(a,b) with w < b, the triangle {a,w,b} has b as its largest vertex, so its
// lowest edge is (a,w) (or (w,a)); its id is tbase[e'] + rank of b among the upper entries of L(e').
// The entry is the triangle's (a,c) entry when a < w, its (b,c) entry when w < a (slots 1, 2).
__global__ void k_edge_fill_tid(GraphView g, int32_t* __restrict__ et_t, int32_t* __restrict__ tri_pos) {
    int lane = threadIdx.x & 31;
    for (int64_t e = gwarp(); e < g.m; e += nwarps()) {
        int32_t a = g.eu[e], b = g.ev[e];
        int64_t lo = g.et_rp[e], hi = g.et_rp[e + 1];
        int64_t split_e = (hi - lo) - (g.tbase[e + 1] - g.tbase[e]);
        for (int64_t j = lo + lane; j < lo + split_e; j += 32) {
            int32_t e2 = et_t[j];
            int64_t l2 = g.et_rp[e2], h2 = g.et_rp[e2 + 1];
            int64_t s2 = (h2 - l2) - (g.tbase[e2 + 1] - g.tbase[e2]);
            int64_t at = nd_lower_bound(g.et_w + l2, h2 - l2, b);
            int64_t tid = g.tbase[e2] + (at - s2);
            et_t[j] = (int32_t)tid;
            tri_pos[3 * tid + (g.et_w[j] > a ? 1 : 2)] = (int32_t)(j - lo);
        }
    }
}

__global__ void k_tri_tuples(GraphView g, int32_t* __restrict__ out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < g.n3; t += (int64_t)gridDim.x * blockDim.x) {
        int32_t e = g.tri_e[3 * t], e1 = g.tri_e[3 * t + 1];
        out[3 * t] = g.eu[e];
        out[3 * t + 1] = g.ev[e];
        out[3 * t + 2] = g.ev[e1];
    }
}

// 4-clique index (the paper's T one level deeper, Section 5.1): the children of triangle
// t = (a<b<c) are the vertices d > c adjacent to a, b and c, ascending. Any two of the triangle's
// edge lists intersect to its common neighbourhood (L(ab) ∩ L(bc) = N(a) ∩ N(b) ∩ N(c)), so a
// warp walks the part above c of the shortest list and searches the second shortest; matches are
// compacted in order with a ballot (count pass, then fill pass at qbase[t]).
template <bool kFill>
__device__ __forceinline__ int64_t quad_children(const GraphView& g, int64_t t, int32_t* out) {
    int lane = threadIdx.x & 31;
    int32_t e[3] = {g.tri_e[3 * t], g.tri_e[3 * t + 1], g.tri_e[3 * t + 2]};
    int32_t c = g.ev[e[1]];  // edges (ab, ac, bc): the largest vertex is ac's upper end
    int64_t b[3], n[3];
    for (int k = 0; k < 3; ++k) {
        b[k] = g.et_rp[e[k]];
        n[k] = g.et_rp[e[k] + 1] - b[k];
    }
    int i0 = 0, i1 = 1;
    if (n[1] < n[0]) i0 = 1, i1 = 0;
    if (n[2] < n[i0]) i1 = i0, i0 = 2;
    else if (n[2] < n[i1]) i1 = 2;
    const int32_t* xs = g.et_w + b[i0];
    const int32_t* ys = g.et_w + b[i1];
    int64_t xlo = nd_lower_bound(xs, n[i0], c + 1), ylo = nd_lower_bound(ys, n[i1], c + 1);
    int64_t pos = 0;
    for (int64_t p0 = xlo; p0 < n[i0]; p0 += 32) {
        int64_t p = p0 + lane;
        bool hit = p < n[i0] && nd_find(ys + ylo, n[i1] - ylo, xs[p]) >= 0;
        unsigned m = __ballot_sync(0xffffffffu, hit);
        if (kFill && hit) out[pos + __popc(m & nd_lanemask_lt())] = xs[p];
        pos += __popc(m);
    }
    return pos;
}

__global__ void k_quad_count(GraphView g, int64_t* __restrict__ qcnt) {
    for (int64_t t = gwarp(); t < g.n3; t += nwarps()) {
        int64_t k = quad_children<false>(g, t, nullptr);
        if ((threadIdx.x & 31) == 0) qcnt[t] = k;
    }
}

__global__ void k_quad_fill(GraphView g, const int64_t* __restrict__ qbase, int32_t* __restrict__ qval) {
    for (int64_t t = gwarp(); t < g.n3; t += nwarps()) quad_children<true>(g, t, qval + qbase[t]);
}

// the inverse map of the 4-clique index: 4-clique q -> (a, b, c, d), one warp per triangle
__global__ void k_quad_tuples(GraphView g, int32_t* __restrict__ out) {
    int lane = threadIdx.x & 31;
    for (int64_t t = gwarp(); t < g.n3; t += nwarps()) {
        int32_t e = g.tri_e[3 * t], e1 = g.tri_e[3 * t + 1];
        int32_t a = g.eu[e], b = g.ev[e], c = g.ev[e1];
        for (int64_t q = g.qbase[t] + lane; q < g.qbase[t + 1]; q += 32) {
            out[4 * q] = a;
            out[4 * q + 1] = b;
            out[4 * q + 2] = c;
            out[4 * q + 3] = g.qval[q];
        }
    }
}

__global__ void k_edge_tuples(GraphView g, int32_t* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < g.m; e += (int64_t)gridDim.x * blockDim.x) {
        out[2 * e] = g.eu[e];
        out[2 * e + 1] = g.ev[e];
    }
}

// max over edges (u,v) of min(deg u, deg v): a bound on |N(u) ∩ N(v)| for every edge
__global__ void k_max_edge_mindeg(GraphView g, unsigned long long* __restrict__ out) {
    unsigned long long best = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < g.m; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = g.eu[e], v = g.ev[e];
        int64_t du = g.rp[u + 1] - g.rp[u], dv = g.rp[v + 1] - g.rp[v];
        unsigned long long d = (unsigned long long)(du < dv ? du : dv);
        best = d > best ? d : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
        best = y > best ? y : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(out, best);
}

__global__ void k_tri_hash_sizes(GraphView g, int64_t* __restrict__ slots) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < g.m; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t n = g.et_rp[e + 1] - g.et_rp[e];
        slots[e] = nd_hashed(n) ? ((int64_t)1 << nd_hash_bits(n)) : 0;
    }
}

// Filling one list's table: each entry claims a free slot by compare-and-swap on its (w, id) pair,
// its round is set to unpeeled and the slot is recorded for its triangle (hpos). A free slot is
// all ones. The triangle's edges are (xy, xz, yz) for x < y < z: e = (a, c) is xy when w > c, xz
// when a < w < c, yz when w < a.
__device__ __forceinline__ int hash_which(int32_t w, int32_t a, int32_t c) { return w > c ? 0 : (w > a ? 1 : 2); }

// Tables of at most 2^kHashSmemBits slots are built in shared memory, (w, id) pairs only, by one
// block per list, and written out whole and coalesced (free slots included), so the directory
// needs no clearing and the compare-and-swaps stay on chip. Each block collects the lists of
// 256 consecutive edges that qualify and then fills them one after another.
constexpr int kHashSmemBits = 13;  // 8,192 slots: 64 KiB of (w, id) pairs
constexpr int kHashBlock = 256;

__global__ void __launch_bounds__(kHashBlock) k_tri_hash_fill_smem(GraphView g, const int64_t* __restrict__ hoff,
                                                                    NdHashSlot* __restrict__ tab,
                                                                    int32_t* __restrict__ hpos) {
    extern __shared__ unsigned long long s_tab[];
    __shared__ int64_t s_list[kHashBlock];
    __shared__ int s_cnt;
    for (int64_t base = (int64_t)blockIdx.x * kHashBlock; base < g.m; base += (int64_t)gridDim.x * kHashBlock) {
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        const int64_t e0 = base + threadIdx.x;
        if (e0 < g.m) {
            int64_t n = g.et_rp[e0 + 1] - g.et_rp[e0];
            if (nd_hashed(n) && nd_hash_bits(n) <= kHashSmemBits) s_list[atomicAdd(&s_cnt, 1)] = e0;
        }
        __syncthreads();
        const int cnt = s_cnt;
        for (int q = 0; q < cnt; ++q) {
            const int64_t e = s_list[q];
            const int64_t b = g.et_rp[e], n = g.et_rp[e + 1] - b;
            const int k = nd_hash_bits(n);
            const uint32_t S = 1u << k, mask = S - 1u;
            for (uint32_t i = threadIdx.x; i < S; i += kHashBlock) s_tab[i] = ~0ull;
            __syncthreads();
            const int32_t a = g.eu[e], c = g.ev[e];
            for (int64_t p = threadIdx.x; p < n; p += kHashBlock) {
                const int32_t w = g.et_w[b + p], id = g.et_t[b + p];
                const unsigned long long key = ((unsigned long long)(uint32_t)id << 32) | (uint32_t)w;
                uint32_t sl = nd_hash_slot(w, k);
                for (uint32_t probes = 0; probes <= mask; ++probes) {
                    if (atomicCAS(&s_tab[sl], ~0ull, key) == ~0ull) {
                        hpos[3 * (int64_t)id + hash_which(w, a, c)] = (int32_t)sl;
                        break;
                    }
                    sl = (sl + 1) & mask;
                }
            }
            __syncthreads();
            int4* out = reinterpret_cast<int4*>(tab + hoff[e]);
            for (uint32_t i = threadIdx.x; i < S; i += kHashBlock) {
                const unsigned long long v = s_tab[i];
                out[i] = v == ~0ull ? make_int4(-1, -1, -1, -1)
                                    : make_int4((int32_t)(uint32_t)v, (int32_t)(v >> 32), ND_UNPEELED, -1);
            }
            __syncthreads();
        }
    }
}

// Larger tables: one warp per list clears its table, then claims slots in global memory.
__global__ void k_tri_hash_fill(GraphView g, const int64_t* __restrict__ hoff, NdHashSlot* __restrict__ tab,
                                int32_t* __restrict__ hpos) {
    int lane = threadIdx.x & 31;
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < g.m;
         e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int64_t b = g.et_rp[e], n = g.et_rp[e + 1] - b;
        if (!nd_hashed(n)) continue;
        int k = nd_hash_bits(n);
        if (k <= kHashSmemBits) continue;
        uint32_t mask = (1u << k) - 1u;
        NdHashSlot* t = tab + hoff[e];
        int4* t4 = reinterpret_cast<int4*>(t);
        for (uint32_t i = lane; i <= mask; i += 32) t4[i] = make_int4(-1, -1, -1, -1);
        __syncwarp();
        const int32_t a = g.eu[e], c = g.ev[e];  // e = (a, c), a < c
        for (int64_t p = lane; p < n; p += 32) {
            int32_t w = g.et_w[b + p], id = g.et_t[b + p];
            unsigned long long key = ((unsigned long long)(uint32_t)id << 32) | (uint32_t)w;  // little endian: w first
            uint32_t s = nd_hash_slot(w, k);
            for (uint32_t probes = 0; probes <= mask; ++probes) {
                unsigned long long* half = reinterpret_cast<unsigned long long*>(t + s);
                if (atomicCAS(half, 0xffffffffffffffffull, key) == 0xffffffffffffffffull) {
                    t[s].rnd = ND_UNPEELED;
                    hpos[3 * (int64_t)id + hash_which(w, a, c)] = (int32_t)s;
                    break;
                }
                s = (s + 1) & mask;
            }
        }
    }
}

}  // namespace

void nd_tri_hash_sizes(const GraphView& g, int64_t* slots, cudaStream_t st) {
    if (g.m <= 0) return;
    ND_K(k_tri_hash_sizes<<<blocks_for_threads(g.m), kThreads, 0, st>>>(g, slots));
}

void nd_tri_hash_fill(const GraphView& g, const int64_t* hoff, NdHashSlot* tab, int32_t* hpos, cudaStream_t st) {
    if (g.m <= 0) return;
    const int smem = (int)sizeof(unsigned long long) << kHashSmemBits;
    cudaFuncSetAttribute(k_tri_hash_fill_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int64_t want = (g.m + kHashBlock - 1) / kHashBlock, cap = (int64_t)nd_sm_count() * 3;
    int blocks = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    ND_K(k_tri_hash_fill_smem<<<blocks, kHashBlock, smem, st>>>(g, hoff, tab, hpos));
    ND_K(k_tri_hash_fill<<<blocks_for_warps(g.m), kThreads, 0, st>>>(g, hoff, tab, hpos));
}

void nd_max_edge_mindeg(const GraphView& g, unsigned long long* out, cudaStream_t st) {
    if (g.m <= 0) return;
    ND_K(k_max_edge_mindeg<<<blocks_for_threads(g.m), kThreads, 0, st>>>(g, out));
}

void nd_validate_csr(const int64_t* rp, const int32_t* col, int32_t n, int64_t nnz, int* err, cudaStream_t st) {
    if (n <= 0) return;
    ND_K(k_validate<<<blocks_for_warps(n), kThreads, 0, st>>>(rp, col, n, nnz, err));
}

void nd_build_split(const int64_t* rp, const int32_t* col, int32_t n, int64_t* split, int64_t* updeg,
                    cudaStream_t st) {
    if (n <= 0) return;
    ND_K(k_split<<<blocks_for_threads(n), kThreads, 0, st>>>(rp, col, n, split, updeg));
}

void nd_build_pos2e(const GraphView& g, int32_t* pos2e, int32_t* eu, int32_t* ev, int* err, cudaStream_t st) {
    if (g.n <= 0) return;
    ND_K(k_pos2e<<<blocks_for_warps(g.n), kThreads, 0, st>>>(g, pos2e, eu, ev, err));
}

void nd_dg_count(const GraphView& g, const int32_t* key_hi, int64_t* outdeg, cudaStream_t st) {
    if (g.n <= 0) return;
    ND_K(k_dg_count<<<blocks_for_warps(g.n), kThreads, 0, st>>>(g, key_hi, outdeg));
}

void nd_dg_fill(const GraphView& g, const int32_t* key_hi, int64_t* dg_rp, int32_t* dg_col, int32_t* dg_eid,
                cudaStream_t st) {
    if (g.n <= 0) return;
    ND_K(k_dg_fill<<<blocks_for_warps(g.n), kThreads, 0, st>>>(g, key_hi, dg_rp, dg_col, dg_eid));
}

void nd_edge_support(const GraphView& g, int64_t* sigma, int64_t* up, cudaStream_t st) {
    if (g.m <= 0) return;
    ND_K(k_edge_support<<<blocks_for_warps(g.m), kThreads, 0, st>>>(g, sigma, up));
}

void nd_edge_fill(const GraphView& g, int64_t* et_rp, int64_t* tbase, int32_t* et_w, int32_t* et_t, int32_t* tri_e,
                  int32_t* tri_pos, cudaStream_t st) {
    if (g.m <= 0) return;
    ND_K(k_edge_fill<<<blocks_for_warps(g.m), kThreads, 0, st>>>(g, et_rp, tbase, et_w, et_t, tri_e, tri_pos));
}

void nd_edge_fill_tid(const GraphView& g, int32_t* et_t, int32_t* tri_pos, cudaStream_t st) {
    if (g.m <= 0) return;
    ND_K(k_edge_fill_tid<<<blocks_for_warps(g.m), kThreads, 0, st>>>(g, et_t, tri_pos));
}


void nd_tri_tuples(const GraphView& g, int32_t* out, cudaStream_t st) {
    if (g.n3 <= 0) return;
    ND_K(k_tri_tuples<<<blocks_for_threads(g.n3), kThreads, 0, st>>>(g, out));
}

void nd_edge_tuples(const GraphView& g, int32_t* out, cudaStream_t st) {
    if (g.m <= 0) return;
    ND_K(k_edge_tuples<<<blocks_for_threads(g.m), kThreads, 0, st>>>(g, out));
}

void nd_quad_count(const GraphView& g, int64_t* qcnt, cudaStream_t st) {
    if (g.n3 <= 0) return;
    ND_K(k_quad_count<<<blocks_for_warps(g.n3), kThreads, 0, st>>>(g, qcnt));
}

void nd_quad_fill(const GraphView& g, const int64_t* qbase, int32_t* qval, cudaStream_t st) {
    if (g.n3 <= 0) return;
    ND_K(k_quad_fill<<<blocks_for_warps(g.n3), kThreads, 0, st>>>(g, qbase, qval));
}

void nd_quad_tuples(const GraphView& g, int32_t* out, cudaStream_t st) {
    if (g.n3 <= 0) return;
    ND_K(k_quad_tuples<<<blocks_for_warps(g.n3), kThreads, 0, st>>>(g, out));
}
