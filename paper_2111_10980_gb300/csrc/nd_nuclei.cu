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
#include <cstring>

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

template <int R_, int S_>
__global__ void k_nuclei_union(GraphView g, const int32_t* __restrict__ core, int32_t level, int64_t n_r,
                               int32_t* parent, int* err) {
    constexpr int M = Others<R_, S_>::M;
    const int lane = threadIdx.x & 31;
    for (int64_t id = gwarp(); id < n_r; id += nwarps()) {
        if (core[id] < level) continue;
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
                for (int i = 0; i < M; ++i)
                    if (core[o[i]] < level || o[i] < id) return;  // not inside X_c, or not the owner
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

template <int R_, int S_>
void launch_union(const GraphView& g, const int32_t* core, int32_t level, int64_t n_r, int32_t* parent, int* err,
                  cudaStream_t st) {
    ND_K(k_nuclei_union<R_, S_><<<blocks_for_warps(n_r), kThreads, 0, st>>>(g, core, level, n_r, parent, err));
}

bool dispatch_union(int r, int s, const GraphView& g, const int32_t* core, int32_t level, int64_t n_r, int32_t* parent,
                    int* err, cudaStream_t st) {
#define ND_NUC(R, S) \
    if (r == R && s == S) return launch_union<R, S>(g, core, level, n_r, parent, err, st), true;
    ND_NUC(1, 2) ND_NUC(1, 3) ND_NUC(1, 4) ND_NUC(2, 3) ND_NUC(2, 4) ND_NUC(2, 5) ND_NUC(3, 4) ND_NUC(3, 5)
    ND_NUC(3, 6) ND_NUC(4, 5) ND_NUC(4, 6)
#undef ND_NUC
    return false;
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
    if (n_r && !dispatch_union(r, s, v, cd, level, n_r, (int32_t*)parent.p, (int*)scal.p, st))
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
