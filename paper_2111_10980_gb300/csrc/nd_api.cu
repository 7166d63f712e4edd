// C ABI of libnd.so (declared in include/nd.h): contexts, device memory, graph lifecycle and
// the host-side sequencing of Algorithm 2 (orient, index, count, peel). Every arithmetic step
// runs in the kernels of nd_graph.cu, nd_count.cu and nd_peel.cu; this file only allocates,
// launches and copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "nd.h"
#include "nd_common.cuh"
#include "nd_host.h"

// ------------------------------------------------------------------------------------
// errors

static thread_local std::string g_last_error;

int nd_set_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

extern "C" const char* nd_last_error(void) { return g_last_error.c_str(); }

// ------------------------------------------------------------------------------------
// memory

int nd_alloc(nd_ctx* ctx, DBuf& b, size_t bytes) {
    nd_free(ctx, b);
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (ctx->budget && ctx->in_use.load() + bytes > ctx->budget)
        return nd_set_error(ND_ENOMEM, "memory budget exceeded: %zu + %zu > %zu bytes", ctx->in_use.load(), bytes,
                            ctx->budget);
    void* p = nullptr;
    if (ctx->af) {
        p = ctx->af(bytes, (void*)ctx->stream, ctx->user);
        if (!p) return nd_set_error(ND_ENOMEM, "allocator hook failed for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, ctx->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return nd_set_error(ND_ENOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
        }
    }
    b.p = p;
    b.bytes = bytes;
    ctx->in_use += bytes;
    return ND_OK;
}

void nd_free(nd_ctx* ctx, DBuf& b) {
    if (!b.p) return;
    if (ctx->ff)
        ctx->ff(b.p, b.bytes, (void*)ctx->stream, ctx->user);
    else
        cudaFreeAsync(b.p, ctx->stream);
    ctx->in_use -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
}

#define ND_TRY(x)                       \
    do {                                \
        int _rc = (x);                  \
        if (_rc != ND_OK) return _rc;   \
    } while (0)

#define ND_CUDA(x)                                                                          \
    do {                                                                                    \
        cudaError_t _e = (x);                                                               \
        if (_e != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            return nd_set_error(ND_ECUDA, "%s failed: %s", #x, cudaGetErrorString(_e));     \
        }                                                                                   \
    } while (0)

int nd_check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return nd_set_error(ND_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return ND_OK;
}

int nd_sync(nd_ctx* ctx, const char* what) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nd_set_error(ND_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    }
    return ND_OK;
}

// device scalar helpers: a small per-graph scratch holds flags and reduction results
static int scalar_zero(nd_graph* g) {
    ND_CUDA(cudaMemsetAsync(g->scal.p, 0, g->scal.bytes, g->ctx->stream));
    return ND_OK;
}

template <typename T>
static int read_back(nd_graph* g, const void* dptr, T* out, const char* what) {
    ND_CUDA(cudaMemcpyAsync(g->ctx->pinned, dptr, sizeof(T), cudaMemcpyDeviceToHost, g->ctx->stream));
    ND_TRY(nd_sync(g->ctx, what));
    memcpy(out, g->ctx->pinned, sizeof(T));
    return ND_OK;
}

static bool rs_supported(int r, int s);

// ------------------------------------------------------------------------------------
// context

extern "C" int nd_ctx_create(int device, void* stream, size_t mem_budget, nd_ctx** out) {
    if (!out) return nd_set_error(ND_EINVAL, "nd_ctx_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    ND_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return nd_set_error(ND_EINVAL, "nd_ctx_create: no CUDA device %d", device);
    ND_CUDA(cudaSetDevice(device));
    nd_ctx* c = new nd_ctx();
    c->device = device;
    c->budget = mem_budget;
    if (stream) {
        c->stream = (cudaStream_t)stream;
        c->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            cudaGetLastError();
            return nd_set_error(ND_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    // keep freed blocks in the device's default pool instead of returning them to the driver
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    if (cudaMallocHost(&c->pinned, 4096) != cudaSuccess) {
        cudaGetLastError();
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return nd_set_error(ND_ECUDA, "cudaMallocHost failed");
    }
    *out = c;
    return ND_OK;
}

extern "C" int nd_ctx_set_allocator(nd_ctx* ctx, nd_alloc_fn alloc, nd_free_fn free_fn, void* user) {
    if (!ctx) return nd_set_error(ND_EINVAL, "nd_ctx_set_allocator: NULL context");
    if ((alloc == nullptr) != (free_fn == nullptr))
        return nd_set_error(ND_EINVAL, "nd_ctx_set_allocator: give both hooks or neither");
    if (ctx->ngraphs.load() > 0) return nd_set_error(ND_EBUSY, "nd_ctx_set_allocator: graphs are still loaded");
    ctx->af = alloc;
    ctx->ff = free_fn;
    ctx->user = user;
    return ND_OK;
}

extern "C" int nd_ctx_set_limits(nd_ctx* ctx, int64_t max_rounds, int64_t barrier_timeout_ns, int64_t count_limit,
                                 int32_t flags) {
    if (!ctx) return nd_set_error(ND_EINVAL, "nd_ctx_set_limits: NULL context");
    if (max_rounds < 0 || barrier_timeout_ns < 0 || count_limit < 0 || (flags & ~ND_LIMIT_DROP_BLOCK))
        return nd_set_error(ND_EINVAL, "nd_ctx_set_limits: negative limit or unknown flag");
    ctx->max_rounds = max_rounds;
    ctx->barrier_ns = barrier_timeout_ns;
    ctx->count_limit = count_limit;
    ctx->limit_flags = flags;
    return ND_OK;
}

extern "C" int nd_ctx_set_tuning(nd_ctx* ctx, int r, int s, int64_t heavy_work, int32_t flags) {
    if (!ctx) return nd_set_error(ND_EINVAL, "nd_ctx_set_tuning: NULL context");
    if (!rs_supported(r, s)) return nd_set_error(ND_EINVAL, "nd_ctx_set_tuning: (r,s) = (%d,%d) is not supported", r, s);
    if (heavy_work < 0 || (flags & ~(ND_DENSE_BUCKETS | ND_CONTRACT_OFF)))
        return nd_set_error(ND_EINVAL, "nd_ctx_set_tuning: negative threshold or unknown flag");
    ctx->tune_heavy[r * 8 + s] = heavy_work;
    ctx->tune_flags[r * 8 + s] = flags;
    return ND_OK;
}

extern "C" int nd_ctx_destroy(nd_ctx* ctx) {
    if (!ctx) return ND_OK;
    if (ctx->ngraphs.load() > 0) return nd_set_error(ND_EBUSY, "nd_ctx_destroy: graphs are still loaded");
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->stage) cudaFreeHost(ctx->stage);
    for (cudaStream_t x : ctx->cap_st)
        if (x) cudaStreamDestroy(x);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    cudaGetLastError();
    delete ctx;
    return ND_OK;
}

extern "C" size_t nd_ctx_bytes_in_use(const nd_ctx* ctx) { return ctx ? ctx->in_use.load() : 0; }

extern "C" int64_t nd_kernel_launches(void) { return nd_total_launches(); }

// ------------------------------------------------------------------------------------
// graphs

static void free_derived(nd_graph* g) {
    nd_ctx* c = g->ctx;
    for (DBuf* b : {&g->split, &g->ebase, &g->pos2e, &g->eu, &g->ev, &g->dg_rp, &g->dg_col, &g->dg_eid, &g->et_rp,
                    &g->et_w, &g->et_t, &g->tbase, &g->tri_e, &g->tri_pos, &g->qbase, &g->qval})
        nd_free(c, *b);
    g->have_quad = false;
    g->n4 = 0;
    g->have_base = false;
    g->edge_mindeg = -1;
    g->orient = -1;
    g->have_tri = false;
    g->n3 = 0;
}

extern "C" int nd_load_csr(nd_ctx* ctx, int32_t n, const int64_t* rowptr, const int32_t* col, int flags,
                           nd_graph** out) {
    if (!ctx || !out) return nd_set_error(ND_EINVAL, "nd_load_csr: NULL context or out");
    *out = nullptr;
    if (n < 0) return nd_set_error(ND_EINVAL, "nd_load_csr: n < 0");
    if (!rowptr) return nd_set_error(ND_EINVAL, "nd_load_csr: rowptr is NULL");
    ND_CUDA(cudaSetDevice(ctx->device));
    bool dev = flags & ND_PTR_DEVICE;
    int64_t ends[2] = {0, 0};
    if (dev) {
        ND_CUDA(cudaMemcpyAsync(ctx->pinned, rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
        ND_CUDA(cudaMemcpyAsync((char*)ctx->pinned + 8, rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                ctx->stream));
        ND_TRY(nd_sync(ctx, "nd_load_csr"));
        memcpy(ends, ctx->pinned, 16);
    } else {
        ends[0] = rowptr[0];
        ends[1] = rowptr[n];
    }
    int64_t nnz = ends[1];
    if (ends[0] != 0 || nnz < 0) return nd_set_error(ND_EINVAL, "nd_load_csr: rowptr[0] must be 0 and rowptr[n] >= 0");
    if (nnz % 2) return nd_set_error(ND_EINVAL, "nd_load_csr: odd number of entries; the CSR is not symmetric");
    if (nnz / 2 > INT32_MAX) return nd_set_error(ND_EOVERFLOW, "nd_load_csr: more than 2^31-1 edges");
    if (nnz > 0 && !col) return nd_set_error(ND_EINVAL, "nd_load_csr: col is NULL");
    nd_graph* g = new nd_graph();
    g->ctx = ctx;
    g->n = n;
    g->nnz = nnz;
    g->m = nnz / 2;
    ctx->ngraphs++;
    int rc = ND_OK;
    cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if ((rc = nd_alloc(ctx, g->rp, sizeof(int64_t) * (n + 1))) || (rc = nd_alloc(ctx, g->col, sizeof(int32_t) * nnz)) ||
        (rc = nd_alloc(ctx, g->scal, 4096))) {
        nd_graph_free(g);
        return rc;
    }
    if (cudaMemcpyAsync(g->rp.p, rowptr, sizeof(int64_t) * (n + 1), kind, ctx->stream) != cudaSuccess ||
        (nnz && cudaMemcpyAsync(g->col.p, col, sizeof(int32_t) * nnz, kind, ctx->stream) != cudaSuccess)) {
        cudaGetLastError();
        nd_graph_free(g);
        return nd_set_error(ND_ECUDA, "nd_load_csr: copy failed");
    }
    if (flags & ND_VALIDATE) {
        scalar_zero(g);
        nd_validate_csr((const int64_t*)g->rp.p, (const int32_t*)g->col.p, n, nnz, (int*)g->scal.p, ctx->stream);
        int err = 0;
        if ((rc = nd_check_launch("validate")) || (rc = read_back(g, g->scal.p, &err, "validate"))) {
            nd_graph_free(g);
            return rc;
        }
        if (err) {
            nd_graph_free(g);
            return nd_set_error(ND_EINVAL,
                                "nd_load_csr: malformed CSR (flags 0x%x: 1 rowptr decreasing, 2 id out of range, "
                                "4 row not strictly ascending, 8 self-loop, 16 missing reverse entry)",
                                err);
        }
    } else {
        if ((rc = nd_sync(ctx, "nd_load_csr"))) {
            nd_graph_free(g);
            return rc;
        }
    }
    *out = g;
    return ND_OK;
}

extern "C" int nd_graph_free(nd_graph* g) {
    if (!g) return ND_OK;
    nd_ctx* c = g->ctx;
    cudaSetDevice(c->device);
    free_derived(g);
    for (DBuf* b : {&g->rp, &g->col, &g->scal}) nd_free(c, *b);
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    c->ngraphs--;
    delete g;
    return ND_OK;
}

extern "C" int nd_graph_size(const nd_graph* g, int32_t* n, int64_t* m) {
    if (!g) return nd_set_error(ND_EINVAL, "nd_graph_size: NULL graph");
    if (n) *n = g->n;
    if (m) *m = g->m;
    return ND_OK;
}

extern "C" int nd_graph_reset(nd_graph* g) {
    if (!g) return nd_set_error(ND_EINVAL, "nd_graph_reset: NULL graph");
    cudaSetDevice(g->ctx->device);
    free_derived(g);
    return ND_OK;
}

GraphView nd_view(const nd_graph* g) {
    GraphView v;
    memset(&v, 0, sizeof(v));
    v.n = g->n;
    v.m = g->m;
    v.rp = (const int64_t*)g->rp.p;
    v.col = (const int32_t*)g->col.p;
    v.split = (const int64_t*)g->split.p;
    v.ebase = (const int64_t*)g->ebase.p;
    v.pos2e = (const int32_t*)g->pos2e.p;
    v.eu = (const int32_t*)g->eu.p;
    v.ev = (const int32_t*)g->ev.p;
    v.dg_rp = (const int64_t*)g->dg_rp.p;
    v.dg_col = (const int32_t*)g->dg_col.p;
    v.dg_eid = (const int32_t*)g->dg_eid.p;
    v.et_rp = (const int64_t*)g->et_rp.p;
    v.et_w = (const int32_t*)g->et_w.p;
    v.et_t = (const int32_t*)g->et_t.p;
    v.tbase = (const int64_t*)g->tbase.p;
    v.tri_e = (const int32_t*)g->tri_e.p;
    v.tri_pos = (const int32_t*)g->tri_pos.p;
    v.n3 = g->n3;
    v.hoff = (const int64_t*)g->hoff.p;
    v.htab = (const NdHashSlot*)g->htab.p;
    v.qbase = (const int64_t*)g->qbase.p;
    v.qval = (const int32_t*)g->qval.p;
    v.n4 = g->n4;
    return v;
}

// canonical edge index (r = 2) and the degree bound
static int ensure_base(nd_graph* g) {
    if (g->have_base) return ND_OK;
    nd_ctx* c = g->ctx;
    cudaStream_t st = c->stream;
    DBuf updeg, tmp;
    int rc = ND_OK;
    if ((rc = nd_alloc(c, g->split, sizeof(int64_t) * std::max<int64_t>(g->n, 1))) ||
        (rc = nd_alloc(c, g->ebase, sizeof(int64_t) * (g->n + 1))) ||
        (rc = nd_alloc(c, updeg, sizeof(int64_t) * std::max<int64_t>(g->n, 1))) ||
        (rc = nd_alloc(c, tmp, nd_scan_tmp_bytes(g->n))) ||
        (rc = nd_alloc(c, g->pos2e, sizeof(int32_t) * std::max<int64_t>(g->nnz, 1))) ||
        (rc = nd_alloc(c, g->eu, sizeof(int32_t) * std::max<int64_t>(g->m, 1))) ||
        (rc = nd_alloc(c, g->ev, sizeof(int32_t) * std::max<int64_t>(g->m, 1)))) {
        nd_free(c, updeg);
        nd_free(c, tmp);
        return rc;
    }
    nd_build_split((const int64_t*)g->rp.p, (const int32_t*)g->col.p, g->n, (int64_t*)g->split.p,
                   (int64_t*)updeg.p, st);
    nd_scan_i64((const int64_t*)updeg.p, (int64_t*)g->ebase.p, g->n, tmp.p, st);
    int64_t m_up = 0;
    rc = nd_check_launch("edge index");
    if (!rc) rc = read_back(g, (int64_t*)g->ebase.p + g->n, &m_up, "edge index");
    nd_free(c, updeg);
    nd_free(c, tmp);
    if (rc) return rc;
    if (m_up != g->m)
        return nd_set_error(ND_EINVAL, "the CSR is not symmetric (%lld upper entries for %lld edges); load it with "
                                       "ND_VALIDATE for details",
                            (long long)m_up, (long long)g->m);
    GraphView v = nd_view(g);
    ND_TRY(scalar_zero(g));
    nd_build_pos2e(v, (int32_t*)g->pos2e.p, (int32_t*)g->eu.p, (int32_t*)g->ev.p, (int*)g->scal.p, st);
    nd_max_deg((const int64_t*)g->rp.p, g->n, (unsigned long long*)g->scal.p + 1, st);
    unsigned long long sc[2] = {0, 0};
    ND_TRY(nd_check_launch("edge index"));
    ND_TRY(read_back(g, g->scal.p, &sc, "edge index"));
    if (sc[0] & 1)
        return nd_set_error(ND_EINVAL, "the CSR is not symmetric or has a self-loop; load it with ND_VALIDATE "
                                       "for details");
    unsigned long long md = sc[1];
    g->maxdeg = (int64_t)md;
    g->have_base = true;
    return ND_OK;
}

int nd_kcore_rounds(nd_graph* g, DBuf& rnd_out);  // degeneracy ranking (below)

static int build_dg(nd_graph* g, int mode) {
    nd_ctx* c = g->ctx;
    cudaStream_t st = c->stream;
    DBuf key, outdeg, tmp;
    int rc = ND_OK;
    const int32_t* key_hi = nullptr;
    if (mode == ND_ORIENT_DEGENERACY) {
        ND_TRY(nd_kcore_rounds(g, key));
        key_hi = (const int32_t*)key.p;
    }
    for (DBuf* b : {&g->dg_rp, &g->dg_col, &g->dg_eid}) nd_free(c, *b);
    if ((rc = nd_alloc(c, outdeg, sizeof(int64_t) * std::max<int64_t>(g->n, 1))) ||
        (rc = nd_alloc(c, tmp, nd_scan_tmp_bytes(g->n))) ||
        (rc = nd_alloc(c, g->dg_rp, sizeof(int64_t) * (g->n + 1))) ||
        (rc = nd_alloc(c, g->dg_col, sizeof(int32_t) * std::max<int64_t>(g->m, 1))) ||
        (rc = nd_alloc(c, g->dg_eid, sizeof(int32_t) * std::max<int64_t>(g->m, 1)))) {
        nd_free(c, key);
        nd_free(c, outdeg);
        nd_free(c, tmp);
        return rc;
    }
    GraphView v = nd_view(g);
    nd_dg_count(v, key_hi, (int64_t*)outdeg.p, st);
    nd_scan_i64((const int64_t*)outdeg.p, (int64_t*)g->dg_rp.p, g->n, tmp.p, st);
    v = nd_view(g);
    nd_dg_fill(v, key_hi, (int64_t*)g->dg_rp.p, (int32_t*)g->dg_col.p, (int32_t*)g->dg_eid.p, st);
    scalar_zero(g);
    nd_max_deg((const int64_t*)g->dg_rp.p, g->n, (unsigned long long*)g->scal.p, st);
    unsigned long long mo = 0;
    rc = nd_check_launch("orientation");
    if (!rc) rc = read_back(g, g->scal.p, &mo, "orientation");
    nd_free(c, key);
    nd_free(c, outdeg);
    nd_free(c, tmp);
    if (rc) return rc;
    g->maxout = (int64_t)mo;
    g->orient = mode;
    return ND_OK;
}

extern "C" int nd_orient(nd_graph* g, int mode) {
    if (!g) return nd_set_error(ND_EINVAL, "nd_orient: NULL graph");
    if (mode != ND_ORIENT_DEGREE && mode != ND_ORIENT_DEGENERACY)
        return nd_set_error(ND_EINVAL, "nd_orient: unknown mode %d", mode);
    ND_CUDA(cudaSetDevice(g->ctx->device));
    ND_TRY(ensure_base(g));
    if (g->orient == mode) return ND_OK;
    ND_TRY(build_dg(g, mode));
    return nd_sync(g->ctx, "nd_orient");
}

// triangle index (r = 3)
static int ensure_tri(nd_graph* g) {
    if (g->have_tri) return ND_OK;
    nd_ctx* c = g->ctx;
    cudaStream_t st = c->stream;
    DBuf sigma, up, tmp;
    int rc = ND_OK;
    int64_t m = g->m;
    if ((rc = nd_alloc(c, sigma, sizeof(int64_t) * std::max<int64_t>(m, 1))) ||
        (rc = nd_alloc(c, up, sizeof(int64_t) * std::max<int64_t>(m, 1))) ||
        (rc = nd_alloc(c, tmp, nd_scan_tmp_bytes(m))) || (rc = nd_alloc(c, g->et_rp, sizeof(int64_t) * (m + 1))) ||
        (rc = nd_alloc(c, g->tbase, sizeof(int64_t) * (m + 1)))) {
        nd_free(c, sigma);
        nd_free(c, up);
        nd_free(c, tmp);
        return rc;
    }
    GraphView v = nd_view(g);
    nd_edge_support(v, (int64_t*)sigma.p, (int64_t*)up.p, st);
    nd_scan_i64((const int64_t*)sigma.p, (int64_t*)g->et_rp.p, m, tmp.p, st);
    nd_scan_i64((const int64_t*)up.p, (int64_t*)g->tbase.p, m, tmp.p, st);
    int64_t tot[2] = {0, 0};
    rc = nd_check_launch("triangle index");
    if (!rc) rc = read_back(g, (int64_t*)g->et_rp.p + m, &tot[0], "triangle index");
    if (!rc) rc = read_back(g, (int64_t*)g->tbase.p + m, &tot[1], "triangle index");
    nd_free(c, sigma);
    nd_free(c, up);
    nd_free(c, tmp);
    if (rc) return rc;
    int64_t n3 = tot[1];
    if (tot[0] != 3 * n3) return nd_set_error(ND_EINTERNAL, "triangle index: %lld entries for %lld triangles",
                                              (long long)tot[0], (long long)n3);
    if (n3 > INT32_MAX) return nd_set_error(ND_EOVERFLOW, "%lld triangles: more than 2^31-1", (long long)n3);
    if ((rc = nd_alloc(c, g->et_w, sizeof(int32_t) * std::max<int64_t>(3 * n3, 1))) ||
        (rc = nd_alloc(c, g->et_t, sizeof(int32_t) * std::max<int64_t>(3 * n3, 1))) ||
        (rc = nd_alloc(c, g->tri_e, sizeof(int32_t) * std::max<int64_t>(3 * n3, 1))) ||
        (rc = nd_alloc(c, g->tri_pos, sizeof(int32_t) * std::max<int64_t>(3 * n3, 1))))
        return rc;
    g->n3 = n3;
    v = nd_view(g);
    nd_edge_fill(v, (int64_t*)g->et_rp.p, (int64_t*)g->tbase.p, (int32_t*)g->et_w.p, (int32_t*)g->et_t.p,
                 (int32_t*)g->tri_e.p, (int32_t*)g->tri_pos.p, st);
    v = nd_view(g);
    nd_edge_fill_tid(v, (int32_t*)g->et_t.p, (int32_t*)g->tri_pos.p, st);
    ND_TRY(nd_check_launch("triangle index"));
    g->have_tri = true;
    return ND_OK;
}

static bool rs_supported(int r, int s) {
    return (r == 1 && s >= 2 && s <= 4) || (r == 2 && s >= 3 && s <= 5) || (r == 3 && s >= 4 && s <= 6) ||
           (r == 4 && s >= 5 && s <= 6);
}

// 4-clique index (r = 4): children of every triangle (count, scan, fill)
static int ensure_quad(nd_graph* g) {
    if (g->have_quad) return ND_OK;
    nd_ctx* c = g->ctx;
    cudaStream_t st = c->stream;
    int64_t n3 = g->n3;
    DBuf qcnt, tmp;
    int rc = ND_OK;
    if ((rc = nd_alloc(c, qcnt, sizeof(int64_t) * std::max<int64_t>(n3, 1))) ||
        (rc = nd_alloc(c, tmp, nd_scan_tmp_bytes(n3))) || (rc = nd_alloc(c, g->qbase, sizeof(int64_t) * (n3 + 1)))) {
        nd_free(c, qcnt);
        nd_free(c, tmp);
        return rc;
    }
    GraphView v = nd_view(g);
    nd_quad_count(v, (int64_t*)qcnt.p, st);
    nd_scan_i64((const int64_t*)qcnt.p, (int64_t*)g->qbase.p, n3, tmp.p, st);
    int64_t n4 = 0;
    rc = nd_check_launch("4-clique index");
    if (!rc) rc = read_back(g, (int64_t*)g->qbase.p + n3, &n4, "4-clique index");
    nd_free(c, qcnt);
    nd_free(c, tmp);
    if (rc) return rc;
    if (n4 > INT32_MAX) return nd_set_error(ND_EOVERFLOW, "%lld 4-cliques: more than 2^31-1", (long long)n4);
    ND_TRY(nd_alloc(c, g->qval, sizeof(int32_t) * std::max<int64_t>(n4, 1)));
    g->n4 = n4;
    v = nd_view(g);
    nd_quad_fill(v, (const int64_t*)g->qbase.p, (int32_t*)g->qval.p, st);
    ND_TRY(nd_check_launch("4-clique index"));
    g->have_quad = true;
    return ND_OK;
}

static int64_t binom64(int64_t a, int b) {
    if (b < 0 || a < b) return 0;
    long double r = 1;
    for (int i = 1; i <= b; ++i) r = r * (long double)(a - b + i) / i;
    return r > 9.0e18L ? INT64_MAX : (int64_t)r;
}

// Prepares orientation and the index for (r,s); *n_r receives the number of r-cliques.
int nd_prepare(nd_graph* g, int r, int s, int64_t* n_r, double* t_orient, double* t_index) {
    if (!rs_supported(r, s)) return nd_set_error(ND_EINVAL, "(r,s) = (%d,%d) is not supported", r, s);
    nd_ctx* c = g->ctx;
    ND_CUDA(cudaSetDevice(c->device));
    cudaEvent_t e0, e1, e2;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    cudaEventRecord(e0, c->stream);
    int rc = ensure_base(g);
    if (!rc && g->orient < 0) rc = build_dg(g, ND_ORIENT_DEGREE);
    cudaEventRecord(e1, c->stream);
    if (!rc && r >= 3) rc = ensure_tri(g);
    if (!rc && r == 4) rc = ensure_quad(g);
    cudaEventRecord(e2, c->stream);
    if (!rc) rc = nd_sync(c, "prepare");
    float a = 0, b = 0;
    if (!rc) {
        cudaEventElapsedTime(&a, e0, e1);
        cudaEventElapsedTime(&b, e1, e2);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    if (rc) return rc;
    if (t_orient) *t_orient = a;
    if (t_index) *t_index = b;
    *n_r = r == 1 ? g->n : r == 2 ? g->m : r == 3 ? g->n3 : g->n4;
    return ND_OK;
}

// An upper bound on any count: the s-cliques containing R are R plus an (s-r)-clique among
// the common neighbours of R, at most C(maxdeg, s-r) of them.
static int64_t count_bound(const nd_graph* g, int r, int s) { return binom64(g->maxdeg, s - r); }

// Largest count a width-4 count array may hold (nd_ctx_set_limits; INT32_MAX by default).
static int64_t width4_limit(const nd_ctx* c) {
    return (c->count_limit > 0 && c->count_limit < INT32_MAX) ? c->count_limit : INT32_MAX;
}

// Runs the counting kernels into a fresh buffer of width w (4 or 8); *cnt receives it.
int nd_count_into(nd_graph* g, int r, int s, int w, int64_t n_r, DBuf& cnt) {
    nd_ctx* c = g->ctx;
    cudaStream_t st = c->stream;
    GraphView v = nd_view(g);
    ND_TRY(nd_alloc(c, cnt, (size_t)w * std::max<int64_t>(n_r, 1)));
    if (w == 8) {
        nd_count_launch<int64_t>(v, r, s, (int64_t*)cnt.p, n_r, st);
        return nd_check_launch("count");
    }
    int64_t limit = width4_limit(c);
    if (count_bound(g, r, s) <= limit) {
        nd_count_launch<int32_t>(v, r, s, (int32_t*)cnt.p, n_r, st);
        return nd_check_launch("count");
    }
    // width 4 requested but counts may not fit: count in int64, then narrow with a check
    DBuf wide;
    ND_TRY(nd_alloc(c, wide, 8 * std::max<int64_t>(n_r, 1)));
    nd_count_launch<int64_t>(v, r, s, (int64_t*)wide.p, n_r, st);
    scalar_zero(g);
    nd_narrow_i64((const int64_t*)wide.p, (int32_t*)cnt.p, n_r, limit, (int*)g->scal.p, st);
    int err = 0;
    int rc = nd_check_launch("count");
    if (!rc) rc = read_back(g, g->scal.p, &err, "count");
    nd_free(c, wide);
    if (rc) return rc;
    if (err) return nd_set_error(ND_EOVERFLOW, "an s-clique count exceeds %lld, the width-4 limit; use count_width 8",
                                 (long long)limit);
    return ND_OK;
}

int nd_pick_width(const nd_graph* g, int r, int s, int count_width, int* w) {
    if (count_width != 0 && count_width != 4 && count_width != 8)
        return nd_set_error(ND_EINVAL, "count_width must be 0, 4 or 8");
    *w = count_width ? count_width : (count_bound(g, r, s) <= width4_limit(g->ctx) ? 4 : 8);
    return ND_OK;
}

static int sum_counts(nd_graph* g, const DBuf& cnt, int w, int64_t n_r, unsigned long long* out) {
    ND_TRY(scalar_zero(g));
    if (w == 8)
        nd_sum_i64((const int64_t*)cnt.p, n_r, (unsigned long long*)g->scal.p, g->ctx->stream);
    else
        nd_sum_i32((const int32_t*)cnt.p, n_r, (unsigned long long*)g->scal.p, g->ctx->stream);
    ND_TRY(nd_check_launch("sum"));
    return read_back(g, g->scal.p, out, "sum");
}

extern "C" int nd_count(nd_graph* g, int r, int s, int count_width, void* counts_out, int flags, int64_t* n_r_out,
                        int64_t* n_s_out) {
    if (!g) return nd_set_error(ND_EINVAL, "nd_count: NULL graph");
    int64_t n_r = 0;
    ND_TRY(nd_prepare(g, r, s, &n_r, nullptr, nullptr));
    if (n_r_out) *n_r_out = n_r;
    int w = 0;
    ND_TRY(nd_pick_width(g, r, s, count_width, &w));
    if (!counts_out && !n_s_out) return ND_OK;
    DBuf cnt;
    int rc = nd_count_into(g, r, s, w, n_r, cnt);
    unsigned long long tot = 0;
    if (!rc && n_s_out) rc = sum_counts(g, cnt, w, n_r, &tot);
    if (!rc && counts_out && n_r > 0) {
        cudaError_t e = cudaMemcpyAsync(counts_out, cnt.p, (size_t)w * n_r,
                                        (flags & ND_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                        g->ctx->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = nd_set_error(ND_ECUDA, "nd_count: copy out: %s", cudaGetErrorString(e));
        }
    }
    if (!rc) rc = nd_sync(g->ctx, "nd_count");
    nd_free(g->ctx, cnt);
    if (!rc && n_s_out) *n_s_out = (int64_t)(tot / (unsigned long long)binom64(s, r));
    return rc;
}

// ------------------------------------------------------------------------------------
// peeling

// Hash directory of the triangle lists for the (3,4) Update: table offsets per edge (an exclusive
// scan of the per-list slot counts) and the tables, filled from the index.
static int build_tri_hash(nd_graph* g, DBuf& hoff, DBuf& htab, DBuf& hpos) {
    nd_ctx* c = g->ctx;
    cudaStream_t st = c->stream;
    int64_t m = g->m;
    DBuf slots, tmp;
    int rc = ND_OK;
    if ((rc = nd_alloc(c, slots, sizeof(int64_t) * std::max<int64_t>(m, 1))) ||
        (rc = nd_alloc(c, tmp, nd_scan_tmp_bytes(m))) || (rc = nd_alloc(c, hoff, sizeof(int64_t) * (m + 1)))) {
        nd_free(c, slots);
        nd_free(c, tmp);
        return rc;
    }
    GraphView v = nd_view(g);
    nd_tri_hash_sizes(v, (int64_t*)slots.p, st);
    nd_scan_i64((const int64_t*)slots.p, (int64_t*)hoff.p, m, tmp.p, st);
    int64_t total = 0;
    rc = nd_check_launch("triangle hash");
    if (!rc) rc = read_back(g, (int64_t*)hoff.p + m, &total, "triangle hash");
    nd_free(c, slots);
    nd_free(c, tmp);
    if (!rc) rc = nd_alloc(c, htab, sizeof(NdHashSlot) * std::max<int64_t>(total, 1));
    if (!rc) rc = nd_alloc(c, hpos, sizeof(int32_t) * std::max<int64_t>(3 * g->n3, 1));
    if (rc) return rc;
    // every table is written whole by the fill kernels (free slots all ones): no clearing pass
    ND_CUDA(cudaMemsetAsync(hpos.p, 0xff, hpos.bytes, st));
    nd_tri_hash_fill(v, (const int64_t*)hoff.p, (NdHashSlot*)htab.p, (int32_t*)hpos.p, st);
    return nd_check_launch("triangle hash");
}

template <typename CT>
static int run_peel(nd_graph* g, int r, int s, DBuf& cnt, int64_t n_r, int flags, PeelOut& po) {
    nd_ctx* c = g->ctx;
    cudaStream_t st = c->stream;
    int64_t cap = std::max<int64_t>(n_r, 1);
    int64_t rcap = std::min<int64_t>(n_r, (int64_t)1 << 22) + 1;
    // (2,4) stages N(u) ∩ N(v) of every heavy edge: its heavy list holds every edge (the light
    // path cannot take one back) and each heavy-phase block gets a slice of 5 * (hstage + 1) int32
    bool staged = r == 2 && s == 4;
    int64_t hcap = staged ? cap : std::min<int64_t>(cap, (int64_t)1 << 20);
    int64_t hstage = 0, hslices = 0;
    int rc = ND_OK;
    if (staged) {
        if (g->edge_mindeg < 0) {
            unsigned long long md = 0;
            ND_TRY(scalar_zero(g));
            nd_max_edge_mindeg(nd_view(g), (unsigned long long*)g->scal.p, st);
            ND_TRY(nd_check_launch("peel setup"));
            ND_TRY(read_back(g, g->scal.p, &md, "peel setup"));
            g->edge_mindeg = (int64_t)md;
        }
        hstage = g->edge_mindeg;
        hslices = nd_peel_heavy_slices();
    }
    // (2,3) graph contraction (Section 5.6): compacted copies of the rows and their lengths
    bool contract = r == 2 && s == 3 && !(flags & ND_CONTRACT_OFF);
    // (3,4): the same for the triangle lists (compacted copies of the lists and entry offsets)
    bool contract34 = r == 3 && s == 4 && !(flags & ND_CONTRACT_OFF);
    // dense buckets (Section 4.2 Discussion): one bucket per count value up to the largest count
    bool dense = flags & ND_DENSE_BUCKETS;
    int64_t bmax = 0;
    if (dense) {
        unsigned long long mx = 0;
        ND_TRY(scalar_zero(g));
        if (sizeof(CT) == 8)
            nd_max_i64((const int64_t*)cnt.p, n_r, (unsigned long long*)g->scal.p, st);
        else
            nd_max_i32((const int32_t*)cnt.p, n_r, (unsigned long long*)g->scal.p, st);
        ND_TRY(nd_check_launch("peel setup"));
        ND_TRY(read_back(g, g->scal.p, &mx, "peel setup"));
        bmax = (int64_t)mx + 1;
    }
    DBuf ctl, A0, A1, N0, N1, L0, L1, H, rs, rl, rt, etr, hsc, abits, ccol, cpos, clen, cprev, bcnt, hcnt, hpre, lw, lt,
        ltp, llen, lprev;
    const int64_t nent = std::max<int64_t>(3 * g->n3, 1);
    if ((rc = nd_alloc(c, ctl, sizeof(PeelCtl))) || (rc = nd_alloc(c, A0, 4 * cap)) || (rc = nd_alloc(c, A1, 4 * cap)) ||
        (rc = nd_alloc(c, N0, 4 * cap)) || (rc = nd_alloc(c, N1, 4 * cap)) || (rc = nd_alloc(c, L0, 4 * cap)) ||
        (rc = nd_alloc(c, L1, 4 * cap)) || (rc = nd_alloc(c, H, 4 * hcap)) || (rc = nd_alloc(c, rs, 8 * rcap)) ||
        (rc = nd_alloc(c, rl, 8 * rcap)) || (rc = nd_alloc(c, rt, 8 * rcap)) || (r == 3 && s == 4 && (rc = nd_alloc(c, etr, 4 * std::max<int64_t>(3 * g->n3, 1)))) ||
        (staged && (rc = nd_alloc(c, hsc, 4 * 5 * (hstage + 1) * hslices))) ||
        (rc = nd_alloc(c, abits, r == 3 ? 4 * ((cap + 31) / 32) : 4)) ||
        (contract && ((rc = nd_alloc(c, ccol, 4 * std::max<int64_t>(g->nnz, 1))) ||
                      (rc = nd_alloc(c, cpos, 4 * std::max<int64_t>(g->nnz, 1))) ||
                      (rc = nd_alloc(c, clen, 4 * std::max<int64_t>(g->n, 1))) ||
                      (rc = nd_alloc(c, cprev, 4 * std::max<int64_t>(g->n, 1))))) ||
        (dense && (rc = nd_alloc(c, bcnt, 4 * std::max<int64_t>(bmax, 1)))) ||
        (staged && ((rc = nd_alloc(c, hcnt, 4 * (hslices + 1))) || (rc = nd_alloc(c, hpre, 8 * (hslices + 1))))) ||
        (contract34 && ((rc = nd_alloc(c, lw, 4 * nent)) || (rc = nd_alloc(c, lt, 4 * nent)) ||
                        (rc = nd_alloc(c, ltp, 4 * nent)) || (rc = nd_alloc(c, llen, 4 * std::max<int64_t>(g->m, 1))) ||
                        (rc = nd_alloc(c, lprev, 4 * std::max<int64_t>(g->m, 1)))))) {
        for (DBuf* b : {&ctl, &A0, &A1, &N0, &N1, &L0, &L1, &H, &rs, &rl, &rt, &etr, &hsc, &abits, &ccol, &cpos, &clen,
                        &cprev, &bcnt, &hcnt, &hpre, &lw, &lt, &ltp, &llen, &lprev})
            nd_free(c, *b);
        return rc;
    }
    PeelView<CT> P;
    P.cnt = (CT*)cnt.p;
    P.rnd = (int32_t*)po.rnd.p;
    P.core = (int32_t*)po.core.p;
    P.A[0] = (int32_t*)A0.p;
    P.A[1] = (int32_t*)A1.p;
    P.N[0] = (int32_t*)N0.p;
    P.N[1] = (int32_t*)N1.p;
    P.L[0] = (int32_t*)L0.p;
    P.L[1] = (int32_t*)L1.p;
    P.H = (int32_t*)H.p;
    P.hcap = (uint32_t)hcap;
    P.hscratch = (int32_t*)hsc.p;
    P.hcnt = staged ? (int32_t*)hcnt.p : nullptr;
    P.hpre = staged ? (int64_t*)hpre.p : nullptr;
    P.hstage = hstage;
    P.hslices = (int32_t)hslices;
    // id-order rebuilds of A pay off for triangles (their lists are long); edges and vertices
    // skip them
    P.abits = r == 3 ? (uint32_t*)abits.p : nullptr;
    // a round sorts A when it holds at least 1/8192 of the r-cliques (and 2048): then the two
    // passes over the bitmap cost little next to the Update they make cache-friendly
    P.sort_min = (uint32_t)std::max<int64_t>(n_r / 8192, 2048);
    cudaMemsetAsync(abits.p, 0, abits.bytes, st);  // a failure surfaces at the launch check below
    P.cap = (uint32_t)cap;
    P.ctl = (PeelCtl*)ctl.p;
    P.round_size = (int64_t*)rs.p;
    P.round_level = (int64_t*)rl.p;
    P.round_ns = (int64_t*)rt.p;
    cudaMemsetAsync(rt.p, 0, rt.bytes, st);
    P.round_cap = rcap;
    P.et_rnd = nullptr;
    P.tri_e = nullptr;
    P.tri_pos = nullptr;
    P.et_rp = nullptr;
    P.hoff = nullptr;
    P.htab = nullptr;
    P.hpos = nullptr;
    if (r == 3 && s == 4) {
        // the hash directory, when the decomposition built one (nd_decompose_dev, (3,4))
        P.hoff = (const int64_t*)g->hoff.p;
        P.htab = (NdHashSlot*)g->htab.p;
        P.hpos = (const int32_t*)g->hpos.p;
        P.et_rnd = (int32_t*)etr.p;
        P.tri_e = (const int32_t*)g->tri_e.p;
        P.tri_pos = (const int32_t*)g->tri_pos.p;
        P.et_rp = (const int64_t*)g->et_rp.p;
        nd_fill_i32(P.et_rnd, ND_UNPEELED, 3 * g->n3, st);
    }
    nd_fill_i32(P.rnd, ND_UNPEELED, n_r, st);
    nd_fill_i32(P.core, 0, n_r, st);
    int64_t max_rounds = c->max_rounds > 0 ? std::min<int64_t>(c->max_rounds, n_r + 2) : n_r + 2;
    GraphView v = nd_view(g);
    P.ccol = P.cpos = P.clen = P.cprev = nullptr;
    P.bcnt = nullptr;
    P.bmax = 0;
    P.heavy_work = c->tune_heavy[r * 8 + s];
    if (dense) {
        P.bcnt = (unsigned int*)bcnt.p;
        P.bmax = bmax;
        cudaMemsetAsync(bcnt.p, 0, bcnt.bytes, st);  // a failure surfaces at the launch check below
        nd_bucket_fill<CT>((const CT*)cnt.p, n_r, P.bcnt, bmax, st);
    }
    int64_t contract_every = 0;
    int contract_shift = 2;
    if (contract) {
        // the paper's schedule: after at least 2n peeled edges, rows that lost a quarter of their
        // entries; ND_CONTRACT_ALWAYS: before every round, every row that lost an entry
        P.ccol = (int32_t*)ccol.p;
        P.cpos = (int32_t*)cpos.p;
        P.clen = (int32_t*)clen.p;
        P.cprev = (int32_t*)cprev.p;
        if (g->nnz) {
            cudaMemcpyAsync(P.ccol, g->col.p, 4 * g->nnz, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(P.cpos, g->pos2e.p, 4 * g->nnz, cudaMemcpyDeviceToDevice, st);
        }
        nd_row_len((const int64_t*)g->rp.p, g->n, P.clen, P.cprev, st);
        v.col = P.ccol;
        v.pos2e = P.cpos;
        v.rlen = P.clen;
        bool always = flags & ND_CONTRACT_ALWAYS;
        contract_every = always ? 1 : std::max<int64_t>(2 * (int64_t)g->n, 1);
        contract_shift = always ? 0 : 2;
    }
    P.lw = P.lt = P.ltp = P.llen = P.lprev = nullptr;
    if (contract34) {
        // lists that lost a quarter of their entries, once 2m triangles (two per list) were peeled
        // since the previous contraction; ND_CONTRACT_ALWAYS: before every round, every list that
        // lost an entry
        P.lw = (int32_t*)lw.p;
        P.lt = (int32_t*)lt.p;
        P.ltp = (int32_t*)ltp.p;
        P.llen = (int32_t*)llen.p;
        P.lprev = (int32_t*)lprev.p;
        if (g->n3) {
            cudaMemcpyAsync(P.lw, g->et_w.p, 4 * 3 * g->n3, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(P.lt, g->et_t.p, 4 * 3 * g->n3, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(P.ltp, g->tri_pos.p, 4 * 3 * g->n3, cudaMemcpyDeviceToDevice, st);
        }
        nd_row_len((const int64_t*)g->et_rp.p, (int32_t)g->m, P.llen, P.lprev, st);
        v.et_w = P.lw;
        v.et_t = P.lt;
        v.llen = P.llen;
        P.tri_pos = P.ltp;
        bool always = flags & ND_CONTRACT_ALWAYS;
        contract_every = always ? 1 : std::max<int64_t>(2 * g->m, 1);
        contract_shift = always ? 0 : 2;
    }
    nd_peel_init(P.ctl, n_r, max_rounds, st, (uint64_t)c->barrier_ns, (c->limit_flags & ND_LIMIT_DROP_BLOCK) ? 1 : 0,
                 contract_every, contract_shift);
    bool looped = false;
    int persistent_launches = 0;
    bool want_persistent = (flags & ND_PEEL_PERSISTENT) || !(flags & (ND_NO_GRAPH | ND_PEEL_LOOP_GRAPH));
    if (want_persistent) {
        // preferred: the whole loop in one cooperative kernel
        cudaError_t e = nd_peel_persistent<CT>(v, r, s, P, st);
        if (e == cudaSuccess) {
            looped = true;
            persistent_launches = 1;
            rc = nd_sync(c, "peel (persistent)");
        } else {
            cudaGetLastError();
            if (flags & ND_PEEL_PERSISTENT)
                rc = nd_set_error(ND_ECUDA, "cooperative launch of the peel loop failed: %s", cudaGetErrorString(e));
        }
    }
    if (!looped && !rc && !(flags & ND_NO_GRAPH)) {
        // preferred: the whole loop in one graph launch (WHILE / IF conditional nodes)
        for (int i = 0; i < 2; ++i)
            if (!c->cap_st[i] && cudaStreamCreateWithFlags(&c->cap_st[i], cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                c->cap_st[i] = nullptr;
            }
        cudaGraph_t lg = nullptr;
        cudaGraphExec_t lx = nullptr;
        if (c->cap_st[0] && c->cap_st[1] &&
            nd_peel_loop_graph<CT>(v, r, s, P, st, c->cap_st[0], c->cap_st[1], &lg) == cudaSuccess &&
            cudaGraphInstantiate(&lx, lg, 0) == cudaSuccess) {
            looped = true;
            rc = (cudaGraphLaunch(lx, st) == cudaSuccess) ? ND_OK : nd_check_launch("peel loop graph");
            if (!rc) rc = nd_sync(c, "peel loop graph");
        }
        cudaGetLastError();
        if (lx) cudaGraphExecDestroy(lx);
        if (lg) cudaGraphDestroy(lg);
    }
    const int kChunk = 32;
    int64_t max_chunks = (n_r + 2) / kChunk + 4;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t graph_nodes = 0;
    bool use_graph = !(flags & ND_NO_GRAPH) && !looped && !rc;
    if (use_graph) {
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            nd_set_capturing(true);
            for (int i = 0; i < kChunk; ++i) nd_peel_round<CT>(v, r, s, P, st);
            nd_set_capturing(false);
            e = cudaStreamEndCapture(st, &graph);
        }
        if (e == cudaSuccess) e = cudaGraphGetNodes(graph, nullptr, &graph_nodes);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (graph) cudaGraphDestroy(graph);
            graph = nullptr;
            exec = nullptr;
            use_graph = false;
        }
    }
    int32_t* hdone = (int32_t*)c->pinned;
    int64_t chunks = 0;
    if (looped) use_graph = false;
    for (; !looped && !rc;) {
        if (use_graph) {
            cudaGraphLaunch(exec, st);
            nd_note_launches((int64_t)graph_nodes);
        } else {
            for (int i = 0; i < kChunk; ++i) nd_peel_round<CT>(v, r, s, P, st);
        }
        if ((rc = nd_check_launch("peel round"))) break;
        cudaMemcpyAsync(hdone, &P.ctl->done, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if ((rc = nd_sync(c, "peel round"))) break;
        if (*hdone) break;
        if (++chunks > max_chunks) {
            rc = nd_set_error(ND_ETIMEOUT, "peeling did not finish within %lld rounds", (long long)(chunks * kChunk));
            break;
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (!rc) {
        PeelCtl h;
        cudaMemcpyAsync(c->pinned, P.ctl, std::min<size_t>(sizeof(PeelCtl), 4096), cudaMemcpyDeviceToHost, st);
        rc = nd_sync(c, "peel stats");
        if (!rc) {
            memcpy(&h, c->pinned, std::min<size_t>(sizeof(PeelCtl), 4096));
            if (h.err & 8) rc = nd_set_error(ND_ETIMEOUT, "peel: a grid barrier of the persistent kernel timed out");
            else if (h.err & 1) rc = nd_set_error(ND_EINTERNAL, "peel: a work list overflowed");
            else if (h.err & 2) rc = nd_set_error(ND_ETIMEOUT, "peel: round cap reached");
            else if (h.err & 4) rc = nd_set_error(ND_EINTERNAL, "peel: empty round (inconsistent state)");
            else if (h.err & 16) rc = nd_set_error(ND_EINTERNAL, "peel: an r-subset of a listed s-clique is not in the index");
            else if (h.finished != n_r) rc = nd_set_error(ND_EINTERNAL, "peel: finished %lld of %lld",
                                                          (long long)h.finished, (long long)n_r);
            po.rho = h.t;
            po.max_core = n_r ? h.k : 0;
            if (looped && !persistent_launches)  // graph nodes executed: every iteration (rho + 1), plus advance and refill phases
                nd_note_launches((int64_t)(h.t + 1) * nd_peel_nodes_per_round(r, s, contract) +
                                 3 * (int64_t)h.advances + 4 * (int64_t)h.refills);
            po.listed = (int64_t)h.listed;
            po.decs = (int64_t)h.decs;
            for (int i = 0; i < 7; ++i) po.phase_ms[i] = persistent_launches ? 1e-6 * (double)h.ph_ns[i] : 0.0;
            po.contractions = h.contractions;
            po.advances = h.advances;
            po.refills = h.refills;
            if (h.k > INT32_MAX && !rc) rc = nd_set_error(ND_EOVERFLOW, "a core number exceeds 2^31-1");
        }
    }
    if (!rc) {
        int64_t nrec = std::min<int64_t>(po.rho, rcap);
        po.sizes.resize(nrec);
        po.levels.resize(nrec);
        po.round_ns.resize(nrec);
        if (nrec) {
            cudaMemcpyAsync(po.sizes.data(), rs.p, 8 * nrec, cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(po.levels.data(), rl.p, 8 * nrec, cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(po.round_ns.data(), rt.p, 8 * nrec, cudaMemcpyDeviceToHost, st);
            rc = nd_sync(c, "peel record");
        }
    }
    for (DBuf* b : {&ctl, &A0, &A1, &N0, &N1, &L0, &L1, &H, &rs, &rl, &rt, &etr, &hsc, &abits, &ccol, &cpos, &clen,
                    &cprev, &bcnt, &hcnt, &hpre, &lw, &lt, &ltp, &llen, &lprev})
        nd_free(c, *b);
    return rc;
}

int nd_decompose_dev(nd_graph* g, int r, int s, int count_width, int flags, PeelOut& po, nd_stats* st) {
    nd_ctx* c = g->ctx;
    if (rs_supported(r, s)) flags |= c->tune_flags[r * 8 + s];
    nd_stats S;
    memset(&S, 0, sizeof(S));
    int64_t n_r = 0;
    double t_or = 0, t_ix = 0;
    ND_TRY(nd_prepare(g, r, s, &n_r, &t_or, &t_ix));
    int w = 0;
    ND_TRY(nd_pick_width(g, r, s, count_width, &w));
    cudaEvent_t e0, e1, e2, e3, eh;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    cudaEventCreate(&e3);
    cudaEventCreate(&eh);
    DBuf cnt;
    int rc = nd_alloc(c, po.core, 4 * std::max<int64_t>(n_r, 1));
    if (!rc) rc = nd_alloc(c, po.rnd, 4 * std::max<int64_t>(n_r, 1));
    cudaEventRecord(e0, c->stream);
    // (3,4): the hash directory of the long triangle lists serves the count's searches and the
    // peel's lookups; it is built inside the counting interval and freed with the decomposition
    if (!rc && r == 3 && s == 4) {
        rc = build_tri_hash(g, g->hoff, g->htab, g->hpos);
        if (rc == ND_ENOMEM) {
            // the directory is an accelerator: without room for it the lists are bisected
            for (DBuf* b : {&g->hoff, &g->htab, &g->hpos}) nd_free(c, *b);
            rc = ND_OK;
        }
    }
    cudaEventRecord(eh, c->stream);
    if (!rc) rc = nd_count_into(g, r, s, w, n_r, cnt);
    cudaEventRecord(e1, c->stream);
    unsigned long long tot = 0;
    if (!rc) rc = sum_counts(g, cnt, w, n_r, &tot);
    cudaEventRecord(e3, c->stream);
    if (!rc) rc = (w == 8) ? run_peel<int64_t>(g, r, s, cnt, n_r, flags, po) : run_peel<int32_t>(g, r, s, cnt, n_r, flags, po);
    cudaEventRecord(e2, c->stream);
    if (!rc) rc = nd_sync(c, "nd_decompose");
    float tc = 0, tp = 0, th = 0;
    if (!rc) {
        cudaEventElapsedTime(&tc, e0, e1);
        cudaEventElapsedTime(&tp, e3, e2);
        cudaEventElapsedTime(&th, e0, eh);
    }
    cudaEventDestroy(eh);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    cudaEventDestroy(e3);
    nd_free(c, cnt);
    for (DBuf* b : {&g->hoff, &g->htab, &g->hpos}) nd_free(c, *b);
    if (rc) return rc;
    S.n_r = n_r;
    S.n_s = (int64_t)(tot / (unsigned long long)binom64(s, r));
    S.rho = po.rho;
    S.max_core = po.max_core;
    S.listed = po.listed;
    S.decrements = po.decs;
    for (int i = 0; i < 6; ++i) S.t_phase_ms[i] = po.phase_ms[i];
    S.t_contract_ms = po.phase_ms[6];
    S.contractions = po.contractions;
    S.advances = po.advances;
    S.refills = po.refills;
    S.count_width = w;
    S.orient_mode = g->orient;
    S.t_orient_ms = t_or;
    S.t_index_ms = t_ix;
    S.t_count_ms = tc;
    S.t_hash_ms = (r == 3 && s == 4) ? th : 0.0;
    S.t_peel_ms = tp;
    S.t_total_ms = t_or + t_ix + tc + tp;
    if (st) *st = S;
    return ND_OK;
}

extern "C" int nd_decompose(nd_graph* g, int r, int s, int count_width, int32_t* core_out, int32_t* round_out,
                            int flags, nd_stats* st) {
    if (!g) return nd_set_error(ND_EINVAL, "nd_decompose: NULL graph");
    PeelOut po;
    int rc = nd_decompose_dev(g, r, s, count_width, flags, po, st);
    nd_ctx* c = g->ctx;
    if (!rc) {
        int64_t n_r = (r == 1) ? g->n : (r == 2) ? g->m : (r == 3) ? g->n3 : g->n4;
        cudaMemcpyKind kind = (flags & ND_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        cudaError_t e = cudaSuccess;
        if (core_out && n_r) e = cudaMemcpyAsync(core_out, po.core.p, 4 * n_r, kind, c->stream);
        if (e == cudaSuccess && round_out && n_r) e = cudaMemcpyAsync(round_out, po.rnd.p, 4 * n_r, kind, c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = nd_set_error(ND_ECUDA, "nd_decompose: copy out: %s", cudaGetErrorString(e));
        }
        if (!rc) rc = nd_sync(c, "nd_decompose");
        g->last_sizes = po.sizes;
        g->last_levels = po.levels;
        g->last_round_ns = po.round_ns;
        g->last_rho = po.rho;
        g->have_last = true;
    }
    nd_free(c, po.core);
    nd_free(c, po.rnd);
    return rc;
}

extern "C" int nd_rounds(nd_graph* g, int64_t* sizes_out, int64_t* levels_out, int64_t cap, int64_t* rho_out) {
    if (!g) return nd_set_error(ND_EINVAL, "nd_rounds: NULL graph");
    if (!g->have_last) return nd_set_error(ND_EINVAL, "nd_rounds: no decomposition has run on this graph");
    int64_t k = std::min<int64_t>(cap, (int64_t)g->last_sizes.size());
    for (int64_t i = 0; i < k; ++i) {
        if (sizes_out) sizes_out[i] = g->last_sizes[i];
        if (levels_out) levels_out[i] = g->last_levels[i];
    }
    if (rho_out) *rho_out = g->last_rho;
    return ND_OK;
}

extern "C" int nd_round_times(nd_graph* g, int64_t* ns_out, int64_t cap) {
    if (!g) return nd_set_error(ND_EINVAL, "nd_round_times: NULL graph");
    if (!g->have_last) return nd_set_error(ND_EINVAL, "nd_round_times: no decomposition has run on this graph");
    int64_t k = std::min<int64_t>(cap, (int64_t)g->last_round_ns.size());
    for (int64_t i = 0; i < k; ++i)
        if (ns_out) ns_out[i] = g->last_round_ns[i];
    return ND_OK;
}

extern "C" int nd_rcliques(nd_graph* g, int r, int32_t* tuples_out, int flags, int64_t* n_r_out) {
    if (!g) return nd_set_error(ND_EINVAL, "nd_rcliques: NULL graph");
    if (r < 1 || r > 4) return nd_set_error(ND_EINVAL, "nd_rcliques: r must be 1, 2, 3 or 4");
    int64_t n_r = 0;
    ND_TRY(nd_prepare(g, r, r + 1, &n_r, nullptr, nullptr));
    if (n_r_out) *n_r_out = n_r;
    if (!tuples_out || n_r == 0) return ND_OK;
    nd_ctx* c = g->ctx;
    DBuf out;
    ND_TRY(nd_alloc(c, out, sizeof(int32_t) * r * n_r));
    GraphView v = nd_view(g);
    if (r == 1)
        nd_iota_i32((int32_t*)out.p, n_r, c->stream);
    else if (r == 2)
        nd_edge_tuples(v, (int32_t*)out.p, c->stream);
    else if (r == 3)
        nd_tri_tuples(v, (int32_t*)out.p, c->stream);
    else
        nd_quad_tuples(v, (int32_t*)out.p, c->stream);
    int rc = nd_check_launch("rcliques");
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(tuples_out, out.p, sizeof(int32_t) * r * n_r,
                                        (flags & ND_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                        c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = nd_set_error(ND_ECUDA, "nd_rcliques: %s", cudaGetErrorString(e));
        }
    }
    if (!rc) rc = nd_sync(c, "nd_rcliques");
    nd_free(c, out);
    return rc;
}

// Degeneracy ranking for ND_ORIENT_DEGENERACY: the round in which each vertex leaves the
// k-core peeling ((1,2) decomposition); ties inside a round are broken by vertex id.
int nd_kcore_rounds(nd_graph* g, DBuf& rnd_out) {
    nd_ctx* c = g->ctx;
    int64_t n = g->n;
    DBuf cnt;
    PeelOut po;
    int rc = nd_alloc(c, po.core, 4 * std::max<int64_t>(n, 1));
    if (!rc) rc = nd_alloc(c, po.rnd, 4 * std::max<int64_t>(n, 1));
    if (!rc) rc = nd_count_into(g, 1, 2, 4, n, cnt);
    if (!rc) rc = run_peel<int32_t>(g, 1, 2, cnt, n, 0, po);
    nd_free(c, cnt);
    nd_free(c, po.core);
    if (rc) {
        nd_free(c, po.rnd);
        return rc;
    }
    rnd_out = po.rnd;
    po.rnd.p = nullptr;
    po.rnd.bytes = 0;
    return ND_OK;
}
