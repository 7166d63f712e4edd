// Connectivity of nuclei (Section 2, footnote): the original definition of a c-(r,s) nucleus also
// requires its r-cliques to be connected through s-cliques. For a level c, the r-cliques with core
// >= c form X_c; two of them are joined when an s-clique contains both and all of its r-subsets lie
// in X_c; the connected nuclei at level c are the components of that relation. Components at a
// higher level nest inside those of a lower one, so the levels together form the nucleus hierarchy.
//
// One warp per r-clique R of X_c lists the s-cliques containing R (the generic listing of
// nd_gen.cuh); an s-clique whose r-subsets all lie in X_c is handled by its owner, the smallest id
// among them, which unites the others with itself in a union-find over r-clique ids. Unions hook
// the larger root under the smaller with a compare-and-swap, so every link points to a smaller id,
// roots end as the smallest id of their component, and finds halve paths without conflicting with
// the hooks (only roots are hooked, only non-roots are shortened). Every retry loop is bounded; a
// bound that runs out sets an error bit instead of spinning.
#include "nd.h"
#include "nd_common.cuh"
#include "nd_gen.cuh"
#include "nd_host.h"

#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int64_t gwarp() { return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int64_t nwarps() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }

int blocks_for_warps(int64_t items) {
    int64_t want = (items + 7) / 8, cap = (int64_t)nd_sm_count() * 16;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

__device__ __forceinline__ int32_t uf_find(int32_t* parent, int32_t x) {
    volatile int32_t* p = parent;
    for (int it = 0; it < (1 << 26); ++it) {
        int32_t px = p[x];
        if (px == x) return x;
        int32_t gp = p[px];
        if (gp != px) p[x] = gp;  // path halving: the link moves to a smaller id
        x = px;
    }
    return x;
}

__device__ __forceinline__ void uf_union(int32_t* parent, int32_t a, int32_t b, int* err) {
    for (int it = 0; it < (1 << 20); ++it) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return;
        if (a > b) {
            int32_t t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(&parent[b], b, a) == b) return;  // hook the larger root under the smaller
    }
    atomicOr(err, 1);
}

// the number of r-subsets of an s-clique other than a given one
template <int R_, int S_>
struct Others {
    static constexpr int M = gen_binom(S_, R_) - 1;
};

// One warp per r-clique R lists the s-cliques containing R and unites the members of those inside
// X_level. Connectivity (kBucket false): every R of X_level, owner = the smallest member. Hierarchy
// (kBucket true): the R of the bucket `ids`, all of core exactly `level`, taking the s-cliques whose
// smallest member core is `level` (the ones that enter X_level at this level), owner = the smallest
// member of core exactly `level`.
template <int R_, int S_, bool kBucket>
__global__ void k_nuclei_union(GraphView g, const int32_t* __restrict__ core, int32_t level,
                               const int32_t* __restrict__ ids, int64_t count, int32_t* parent, int* err) {
    constexpr int M = Others<R_, S_>::M;
    const int lane = threadIdx.x & 31;
    for (int64_t k = gwarp(); k < count; k += nwarps()) {
        const int64_t id = kBucket ? ids[k] : k;
        if (!kBucket && core[id] < level) continue;
        int32_t v[4];
        gen_verts<R_>(g, id, v);
        const int32_t* list = nullptr;
        int64_t len = 0;
        gen_drive<R_>(g, id, v, list, len);
        for (int64_t j = lane; j < len; j += 32)
            gen_cand<R_, S_>(g, v, list[j], [&](const int32_t* C) {
                int32_t Sv[S_], o[M];
                gen_merge<R_, S_>(v, C, Sv);
                if (!gen_others<R_, S_>(g, v, Sv, o)) {
                    atomicOr(err, 2);
                    return;
                }
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    const int32_t co = core[o[i]];
                    if (co < level) return;                                  // not inside X_level
                    if (o[i] < id && (!kBucket || co == level)) return;      // not the owner
                }
#pragma unroll
                for (int i = 0; i < M; ++i) uf_union(parent, (int32_t)id, o[i], err);
            });
    }
}

__global__ void k_nuclei_label(const int32_t* __restrict__ core, int32_t level, int64_t n_r, int32_t* parent,
                               int32_t* __restrict__ comp, unsigned long long* n_comp) {
    unsigned long long roots = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
        if (core[i] < level) {
            comp[i] = -1;
            continue;
        }
        int32_t rt = uf_find(parent, (int32_t)i);
        comp[i] = rt;
        roots += rt == i;
    }
    for (int o = 16; o > 0; o >>= 1) roots += __shfl_down_sync(0xffffffffu, roots, o);
    if ((threadIdx.x & 31) == 0 && roots) atomicAdd(n_comp, roots);
}

template <int R_, int S_, bool kBucket>
void launch_union(const GraphView& g, const int32_t* core, int32_t level, const int32_t* ids, int64_t count,
                  int32_t* parent, int* err, cudaStream_t st) {
    ND_K(k_nuclei_union<R_, S_, kBucket><<<blocks_for_warps(count), kThreads, 0, st>>>(g, core, level, ids, count,
                                                                                       parent, err));
}

bool dispatch_union(int r, int s, bool bucket, const GraphView& g, const int32_t* core, int32_t level,
                    const int32_t* ids, int64_t count, int32_t* parent, int* err, cudaStream_t st) {
#define ND_NUC(R, S)                                                                      \
    if (r == R && s == S) {                                                               \
        if (bucket)                                                                       \
            launch_union<R, S, true>(g, core, level, ids, count, parent, err, st);        \
        else                                                                              \
            launch_union<R, S, false>(g, core, level, ids, count, parent, err, st);       \
        return true;                                                                      \
    }
    ND_NUC(1, 2) ND_NUC(1, 3) ND_NUC(1, 4) ND_NUC(2, 3) ND_NUC(2, 4) ND_NUC(2, 5) ND_NUC(3, 4) ND_NUC(3, 5)
    ND_NUC(3, 6) ND_NUC(4, 5) ND_NUC(4, 6)
#undef ND_NUC
    return false;
}

// ---- the hierarchy ------------------------------------------------------------------------
// Levels are taken in decreasing order with one union-find over all r-clique ids. At level c the
// bucket of r-cliques of core exactly c unites the s-cliques that enter X_c (smallest member core
// c); every s-clique is therefore listed once over all levels, and after level c the sets are the
// components of X_c (roots are smallest ids). A node is a component of X_c holding an r-clique of
// core exactly c; it is represented by the smallest such r-clique (rep). Nodes wait in a pending
// list until the first lower level at which their component's root is a node: that node is their
// parent.

__global__ void k_core_range(const int32_t* __restrict__ core, int64_t n_r, int* lo_hi) {
    int lo = INT_MAX, hi = INT_MIN;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
        lo = min(lo, core[i]);
        hi = max(hi, core[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(lo_hi, lo);
        atomicMax(lo_hi + 1, hi);
    }
}

__global__ void k_core_hist(const int32_t* __restrict__ core, int64_t n_r, unsigned* __restrict__ hist) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[core[i]], 1u);
}

// ids bucketed by core: cursor[c] starts at the bucket's offset
__global__ void k_core_scatter(const int32_t* __restrict__ core, int64_t n_r, unsigned* __restrict__ cursor,
                               int32_t* __restrict__ order) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x)
        order[atomicAdd(&cursor[core[i]], 1u)] = (int32_t)i;
}

// comp of the bucket's r-cliques (their roots after this level's unions) and the smallest of them
// per root
__global__ void k_hier_rep(const int32_t* __restrict__ ids, int64_t count, int32_t* parent, int32_t* __restrict__ comp,
                           int32_t* __restrict__ rep_tmp) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t R = ids[k], rt = uf_find(parent, R);
        comp[R] = rt;
        atomicMin(&rep_tmp[rt], R);
    }
}

// each bucket r-clique learns its node's rep; each rep opens its node (pending, for a parent below)
__global__ void k_hier_node(const int32_t* __restrict__ ids, int64_t count, int32_t level,
                            const int32_t* __restrict__ comp, const int32_t* __restrict__ rep_tmp,
                            int32_t* __restrict__ node_rep, int32_t* __restrict__ node_at,
                            int32_t* __restrict__ node_rep_at, int32_t* __restrict__ pend_root,
                            int32_t* __restrict__ pend_rep, unsigned* __restrict__ pend_n,
                            unsigned long long* __restrict__ n_nodes) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t R = ids[k], rt = comp[R], rep = rep_tmp[rt];
        node_rep[R] = rep;
        if (rep == R) {
            node_at[rt] = level;
            node_rep_at[rt] = R;
            const unsigned at = atomicAdd(pend_n, 1u);
            pend_root[at] = rt;
            pend_rep[at] = R;
            atomicAdd(n_nodes, 1ull);
        }
    }
}

__global__ void k_hier_reset(const int32_t* __restrict__ ids, int64_t count, const int32_t* __restrict__ comp,
                             int32_t* __restrict__ rep_tmp) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
        rep_tmp[comp[ids[k]]] = INT_MAX;
}

// nodes of higher levels still without a parent: the node of their component at this level, if
// there is one, is their parent; the others move on to the next list with their current root
__global__ void k_hier_resolve(const int32_t* __restrict__ in_root, const int32_t* __restrict__ in_rep,
                               const unsigned* __restrict__ in_n, int32_t level, int32_t* parent,
                               const int32_t* __restrict__ node_at, const int32_t* __restrict__ node_rep_at,
                               int32_t* __restrict__ parent_rep, int32_t* __restrict__ out_root,
                               int32_t* __restrict__ out_rep, unsigned* __restrict__ out_n) {
    const unsigned n = *in_n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rt = uf_find(parent, in_root[k]), rep = in_rep[k];
        if (node_at[rt] == level) {
            parent_rep[rep] = node_rep_at[rt];
        } else {
            const unsigned at = atomicAdd(out_n, 1u);
            out_root[at] = rt;
            out_rep[at] = rep;
        }
    }
}

__global__ void k_hier_out(const int32_t* __restrict__ core, int64_t n_r, const int32_t* __restrict__ comp,
                           const int32_t* __restrict__ node_rep, const int32_t* __restrict__ parent_rep,
                           int32_t* __restrict__ comp_out, int32_t* __restrict__ plev_out,
                           int32_t* __restrict__ pcomp_out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t pr = parent_rep[node_rep[i]];
        comp_out[i] = comp[i];
        plev_out[i] = pr >= 0 ? core[pr] : -1;
        pcomp_out[i] = pr >= 0 ? comp[pr] : -1;
    }
}

int thread_blocks(int64_t items) {
    int64_t want = (items + 255) / 256, cap = (int64_t)nd_sm_count() * 8;
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

}  // namespace

extern "C" int nd_nuclei(nd_graph* g, int r, int s, const int32_t* core, int32_t level, int32_t* comp_out, int flags,
                         int64_t* n_comp_out) {
    if (!g || !core) return nd_set_error(ND_EINVAL, "nd_nuclei: NULL graph or core");
    int64_t n_r = 0;
    int rc = nd_prepare(g, r, s, &n_r, nullptr, nullptr);
    if (rc) return rc;
    if (n_r > INT32_MAX) return nd_set_error(ND_EOVERFLOW, "nd_nuclei: %lld r-cliques exceed int32 ids", (long long)n_r);
    nd_ctx* c = g->ctx;
    cudaStream_t st = c->stream;
    const bool dev = flags & ND_PTR_DEVICE;
    DBuf dcore, parent, comp, scal;
    if ((rc = nd_alloc(c, parent, 4 * std::max<int64_t>(n_r, 1))) || (rc = nd_alloc(c, comp, 4 * std::max<int64_t>(n_r, 1))) ||
        (rc = nd_alloc(c, scal, 64)) || (!dev && (rc = nd_alloc(c, dcore, 4 * std::max<int64_t>(n_r, 1))))) {
        for (DBuf* b : {&dcore, &parent, &comp, &scal}) nd_free(c, *b);
        return rc;
    }
    const int32_t* cd = core;
    if (!dev) {
        if (n_r) cudaMemcpyAsync(dcore.p, core, 4 * n_r, cudaMemcpyHostToDevice, st);
        cd = (const int32_t*)dcore.p;
    }
    cudaMemsetAsync(scal.p, 0, 64, st);
    nd_iota_i32((int32_t*)parent.p, n_r, st);
    GraphView v = nd_view(g);
    if (n_r && !dispatch_union(r, s, false, v, cd, level, nullptr, n_r, (int32_t*)parent.p, (int*)scal.p, st))
        rc = nd_set_error(ND_EINVAL, "nd_nuclei: (r,s) = (%d,%d) is not supported", r, s);
    if (!rc && n_r) {
        int64_t want = (n_r + 255) / 256, cap = (int64_t)nd_sm_count() * 8;
        ND_K(k_nuclei_label<<<(int)std::max<int64_t>(1, std::min(want, cap)), 256, 0, st>>>(
            cd, level, n_r, (int32_t*)parent.p, (int32_t*)comp.p, (unsigned long long*)((char*)scal.p + 8)));
    }
    if (!rc) rc = nd_check_launch("nd_nuclei");
    struct {
        int err, pad;
        unsigned long long n;
    } h = {0, 0, 0};
    if (!rc) {
        cudaMemcpyAsync(c->pinned, scal.p, sizeof(h), cudaMemcpyDeviceToHost, st);
        rc = nd_sync(c, "nd_nuclei");
        if (!rc) memcpy(&h, c->pinned, sizeof(h));
    }
    if (!rc && h.err) rc = nd_set_error(ND_EINTERNAL, "nd_nuclei: union-find retries ran out or an r-subset is not in the index (%d)", h.err);
    if (!rc && comp_out && n_r) {
        cudaError_t e = cudaMemcpyAsync(comp_out, comp.p, 4 * n_r, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = nd_set_error(ND_ECUDA, "nd_nuclei: copy out: %s", cudaGetErrorString(e));
        }
        if (!rc) rc = nd_sync(c, "nd_nuclei");
    }
    if (!rc && n_comp_out) *n_comp_out = (int64_t)h.n;
    for (DBuf* b : {&dcore, &parent, &comp, &scal}) nd_free(c, *b);
    return rc;
}

// The nucleus hierarchy (Section 2, footnote). See the comment above the hierarchy kernels.
extern "C" int nd_hierarchy(nd_graph* g, int r, int s, const int32_t* core, int32_t* comp_out,
                            int32_t* parent_level_out, int32_t* parent_comp_out, int flags, int64_t* n_nodes_out) {
    if (!g || !core) return nd_set_error(ND_EINVAL, "nd_hierarchy: NULL graph or core");
    int64_t n_r = 0;
    int rc = nd_prepare(g, r, s, &n_r, nullptr, nullptr);
    if (rc) return rc;
    if (n_r > INT32_MAX) return nd_set_error(ND_EOVERFLOW, "nd_hierarchy: %lld r-cliques exceed int32 ids", (long long)n_r);
    if (n_r == 0) {
        if (n_nodes_out) *n_nodes_out = 0;
        return ND_OK;
    }
    nd_ctx* c = g->ctx;
    cudaStream_t st = c->stream;
    const bool dev = flags & ND_PTR_DEVICE;
    const size_t B = 4 * (size_t)n_r;
    enum { kCore, kParent, kComp, kRepTmp, kNodeRep, kNodeAt, kNodeRepAt, kParentRep, kOrder, kPR0, kPP0, kPR1, kPP1,
           kOutC, kOutL, kOutP, kScal, kHist, kN };
    DBuf b[kN];
    auto release = [&]() {
        for (DBuf& x : b) nd_free(c, x);
    };
    for (int i = 0; i < kScal && !rc; ++i) {
        if ((i == kCore || i >= kOutC) && dev) continue;  // caller's device arrays are used directly
        rc = nd_alloc(c, b[i], B);
    }
    if (!rc) rc = nd_alloc(c, b[kScal], 64);
    if (rc) {
        release();
        return rc;
    }
    auto I32 = [&](int i) { return (int32_t*)b[i].p; };
    const int32_t* cd = dev ? core : I32(kCore);
    int32_t* oc = dev ? comp_out : I32(kOutC);
    int32_t* ol = dev ? parent_level_out : I32(kOutL);
    int32_t* op = dev ? parent_comp_out : I32(kOutP);
    if (dev && (!comp_out || !parent_level_out || !parent_comp_out)) {
        release();
        return nd_set_error(ND_EINVAL, "nd_hierarchy: with ND_PTR_DEVICE all three outputs are required");
    }
    if (!dev) cudaMemcpyAsync(I32(kCore), core, B, cudaMemcpyHostToDevice, st);
    // scal: [0] union-find error bits, [1..2] core range, [4..5] pending counters, [8] node count
    int* sc = (int*)b[kScal].p;
    const int init[4] = {0, INT_MAX, INT_MIN, 0};
    cudaMemcpyAsync(sc, init, sizeof(init), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(sc + 4, 0, 64 - 16, st);
    ND_K(k_core_range<<<thread_blocks(n_r), 256, 0, st>>>(cd, n_r, sc + 1));
    int lo_hi[2] = {0, 0};
    cudaMemcpyAsync(c->pinned, sc + 1, sizeof(lo_hi), cudaMemcpyDeviceToHost, st);
    if ((rc = nd_check_launch("nd_hierarchy")) || (rc = nd_sync(c, "nd_hierarchy"))) {
        release();
        return rc;
    }
    memcpy(lo_hi, c->pinned, sizeof(lo_hi));
    if (lo_hi[0] < 0 || lo_hi[1] >= (1 << 26)) {
        release();
        return nd_set_error(ND_EINVAL, "nd_hierarchy: core numbers must lie in [0, 2^26) (got %d .. %d)", lo_hi[0], lo_hi[1]);
    }
    const int64_t nb = (int64_t)lo_hi[1] + 1;
    if ((rc = nd_alloc(c, b[kHist], 4 * nb))) {
        release();
        return rc;
    }
    unsigned* hist = (unsigned*)b[kHist].p;
    cudaMemsetAsync(hist, 0, 4 * nb, st);
    ND_K(k_core_hist<<<thread_blocks(n_r), 256, 0, st>>>(cd, n_r, hist));
    std::vector<unsigned> h(nb);
    cudaMemcpyAsync(h.data(), hist, 4 * nb, cudaMemcpyDeviceToHost, st);
    if ((rc = nd_check_launch("nd_hierarchy")) || (rc = nd_sync(c, "nd_hierarchy"))) {
        release();
        return rc;
    }
    std::vector<unsigned> off(nb);
    unsigned run = 0;
    for (int64_t v = 0; v < nb; ++v) {
        off[v] = run;
        run += h[v];
    }
    cudaMemcpyAsync(hist, off.data(), 4 * nb, cudaMemcpyHostToDevice, st);
    ND_K(k_core_scatter<<<thread_blocks(n_r), 256, 0, st>>>(cd, n_r, hist, I32(kOrder)));
    nd_iota_i32(I32(kParent), n_r, st);
    nd_fill_i32(I32(kRepTmp), INT_MAX, n_r, st);
    nd_fill_i32(I32(kNodeAt), -1, n_r, st);
    nd_fill_i32(I32(kParentRep), -1, n_r, st);
    GraphView v = nd_view(g);
    unsigned* pend_n = (unsigned*)(sc + 4);  // [0], [1]: counters of the two pending lists
    unsigned long long* n_nodes = (unsigned long long*)(sc + 8);
    int cur = 0;  // the list holding nodes that wait for a parent
    for (int64_t lv = nb - 1; lv >= 0 && !rc; --lv) {
        if (!h[lv]) continue;
        const int32_t* ids = I32(kOrder) + off[lv];
        const int64_t cnt = h[lv];
        const int nxt = cur ^ 1;
        int32_t* nroot = I32(nxt ? kPR1 : kPR0);
        int32_t* nrep = I32(nxt ? kPP1 : kPP0);
        if (!dispatch_union(r, s, true, v, cd, (int32_t)lv, ids, cnt, I32(kParent), sc, st)) {
            rc = nd_set_error(ND_EINVAL, "nd_hierarchy: (r,s) = (%d,%d) is not supported", r, s);
            break;
        }
        ND_K(k_hier_rep<<<thread_blocks(cnt), 256, 0, st>>>(ids, cnt, I32(kParent), I32(kComp), I32(kRepTmp)));
        // this level's nodes first (node_at marks them), then the older nodes look for them
        cudaMemsetAsync(pend_n + nxt, 0, 4, st);
        ND_K(k_hier_node<<<thread_blocks(cnt), 256, 0, st>>>(ids, cnt, (int32_t)lv, I32(kComp), I32(kRepTmp),
                                                             I32(kNodeRep), I32(kNodeAt), I32(kNodeRepAt), nroot,
                                                             nrep, pend_n + nxt, n_nodes));
        ND_K(k_hier_resolve<<<(int)nd_sm_count() * 4, 256, 0, st>>>(
            I32(cur ? kPR1 : kPR0), I32(cur ? kPP1 : kPP0), pend_n + cur, (int32_t)lv, I32(kParent), I32(kNodeAt),
            I32(kNodeRepAt), I32(kParentRep), nroot, nrep, pend_n + nxt));
        ND_K(k_hier_reset<<<thread_blocks(cnt), 256, 0, st>>>(ids, cnt, I32(kComp), I32(kRepTmp)));
        rc = nd_check_launch("nd_hierarchy");
        cur = nxt;
    }
    if (!rc) {
        ND_K(k_hier_out<<<thread_blocks(n_r), 256, 0, st>>>(cd, n_r, I32(kComp), I32(kNodeRep), I32(kParentRep), oc,
                                                            ol, op));
        rc = nd_check_launch("nd_hierarchy");
    }
    struct {
        int err;
        int pad[7];
        unsigned long long nodes;
    } hs = {0, {0}, 0};
    if (!rc) {
        cudaMemcpyAsync(c->pinned, sc, sizeof(hs), cudaMemcpyDeviceToHost, st);
        rc = nd_sync(c, "nd_hierarchy");
        if (!rc) memcpy(&hs, c->pinned, sizeof(hs));
    }
    if (!rc && hs.err)
        rc = nd_set_error(ND_EINTERNAL, "nd_hierarchy: union-find retries ran out or an r-subset is not in the index (%d)", hs.err);
    if (!rc && !dev) {
        int32_t* outs[3] = {comp_out, parent_level_out, parent_comp_out};
        const int32_t* srcs[3] = {oc, ol, op};
        for (int i = 0; i < 3 && !rc; ++i)
            if (outs[i] && cudaMemcpyAsync(outs[i], srcs[i], B, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
                cudaGetLastError();
                rc = nd_set_error(ND_ECUDA, "nd_hierarchy: copy out failed");
            }
        if (!rc) rc = nd_sync(c, "nd_hierarchy");
    }
    if (!rc && n_nodes_out) *n_nodes_out = (int64_t)hs.nodes;
    release();
    return rc;
}
