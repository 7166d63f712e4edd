/*
 * nd.h -- C ABI of the GB300 (sm_103a) (r,s) nucleus decomposition library (libnd.so).
 *
 * The library computes, for every r-clique R of a simple undirected graph, its
 * (r,s)-clique core number: the largest c such that R lies in a c-(r,s) nucleus, i.e. in a
 * maximal set of r-cliques each of which is contained in at least c s-cliques whose
 * r-subsets all belong to the set (Shi, Dhulipala, Shun, "Theoretically and Practically
 * Efficient Parallel Nucleus Decomposition", Section 2, definition of the (r,s) nucleus
 * decomposition problem; the connectivity condition of the original definition is not
 * imposed, as in the paper). (1,2) is k-core coreness; (2,3) is k-truss trussness minus 2.
 *
 * Every step runs in hand-written CUDA kernels on one GPU: degree orientation (Section 3,
 * O(alpha)-orientation), the r-clique index (Section 5.2-5.3), s-clique counting
 * (Algorithm 1 with Count-Func of Algorithm 2), and the peeling loop of Algorithm 2 (bucket
 * extraction, Update/Update-Func with exact integer decrements). There is no CPU fallback.
 *
 * Conventions shared by all calls
 *   - Every call returns an int status (ND_OK on success). On failure nothing visible to the
 *     caller has been written except where stated, and nd_last_error() describes the error.
 *   - Graph input is a symmetric CSR: rowptr int64[n+1] (rowptr[0] = 0), col int32[rowptr[n]],
 *     every neighbour list sorted ascending, no self-loops, no duplicate entries, and (u,v)
 *     present iff (v,u) is. ND_VALIDATE checks all of this on the GPU (ND_EINVAL otherwise).
 *   - Pointer arguments are host memory unless ND_PTR_DEVICE is passed in flags, in which
 *     case they are device memory on the context's device. The library never keeps a
 *     caller's pointer after a call returns (except nd_submit, see there); it copies inputs.
 *   - Canonical r-clique order (the id space of all per-r-clique outputs): r-cliques sorted
 *     lexicographically by their ascending tuple of vertex ids. r = 1: vertex id; r = 2:
 *     edges (u < v) in CSR order; r = 3: triangles (a < b < c) by (a, b, c).
 *   - Supported (r, s): (1,2), (1,3), (2,3), (2,4), (3,4) with kernels of their own, and (1,4),
 *     (2,5), (3,5), (3,6), (4,5), (4,6) through the generic listing of the (s-r)-cliques of each
 *     r-clique's common neighbourhood (r = 4 adds a 4-clique index: per triangle (a<b<c), the
 *     vertices d > c adjacent to all three, ascending). Others return ND_EINVAL.
 *   - All work is issued on the context's stream; synchronous calls synchronise that stream
 *     before returning.
 */
#ifndef ND_H
#define ND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ND_API __attribute__((visibility("default")))
#else
#define ND_API
#endif

/* ---- status codes ------------------------------------------------------------------- */
#define ND_OK 0
#define ND_EINVAL 1     /* bad argument, unsupported (r,s), or malformed CSR (ND_VALIDATE) */
#define ND_ENOMEM 2     /* device allocation failed or the context's memory budget is exceeded */
#define ND_EOVERFLOW 3  /* a count exceeds the chosen width, or an id space exceeds int32 */
#define ND_ETIMEOUT 4   /* the peeling loop hit its round cap, or a bounded device-side wait ran out */
#define ND_EBUSY 5      /* server has no free slot / request queue full */
#define ND_PENDING 6    /* nd_poll: the request is still running */
#define ND_EINTERNAL 7  /* internal inconsistency detected on the device */
#define ND_ECUDA 8      /* a CUDA runtime call failed */

/* ---- flags --------------------------------------------------------------------------- */
#define ND_PTR_DEVICE 0x1 /* pointer arguments are device memory (default: host memory) */
#define ND_VALIDATE 0x2   /* nd_load_csr: check the CSR invariants on the GPU */
#define ND_NO_GRAPH 0x4   /* nd_decompose: launch every phase of every peeling round separately */
#define ND_PEEL_LOOP_GRAPH 0x8  /* nd_decompose: run the peeling loop as one CUDA graph (WHILE/IF nodes) */
#define ND_PEEL_PERSISTENT 0x10 /* nd_decompose: run the peeling loop as one cooperative kernel (default
                                   when none of these three flags is given and the launch is possible) */
#define ND_CONTRACT_OFF 0x20    /* nd_decompose (2,3): no graph contraction (Section 5.6); (3,4): no
                                   contraction of the triangle lists (entries of peeled triangles stay) */
#define ND_CONTRACT_ALWAYS 0x40 /* nd_decompose (2,3), (3,4): contract before every round, every row or list
                                   that lost an entry (exercises the contraction; slower than the default) */
#define ND_DENSE_BUCKETS 0x80   /* nd_decompose: find each new level with the dense bucket array and its
                                   doubling search (Section 4.2 Discussion) instead of a scan of the
                                   bucket window; pays off when the range of counts is small */

/* ---- orientation modes (nd_orient) --------------------------------------------------- */
#define ND_ORIENT_DEGREE 0     /* rank by (degree, id); out-degree <= sqrt(2m) */
#define ND_ORIENT_DEGENERACY 1 /* rank by (k-core peeling round, id); out-degree <= degeneracy */

typedef struct nd_ctx nd_ctx;
typedef struct nd_graph nd_graph;

/* Device allocator hooks: alloc returns device memory of at least `bytes` bytes usable on
 * `stream` (NULL on failure); free releases it. `user` is passed through. */
typedef void *(*nd_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*nd_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

/* Statistics of one decomposition (all times in milliseconds, measured with CUDA events on
 * the context's stream). */
typedef struct nd_stats {
    int64_t n_r;        /* number of r-cliques */
    int64_t n_s;        /* number of s-cliques */
    int64_t rho;        /* peeling rounds: each round peels every unpeeled r-clique whose count
                           is <= k, after k = max(k, minimum unpeeled count) */
    int64_t max_core;   /* largest core number */
    int64_t listed;     /* s-cliques destroyed by Update over the run (each exactly once, by the
                           smallest member of A it contains): equals n_s */
    int64_t advances;   /* rounds that moved to a new level k */
    int64_t refills;    /* bucket-window rebuilds */
    int32_t count_width;/* 4 or 8: bytes per count used on the device */
    int32_t orient_mode;
    double t_orient_ms; /* orientation (and the r = 1, 2 index) */
    double t_index_ms;  /* r = 3 index */
    double t_count_ms;  /* s-clique counting */
    double t_peel_ms;   /* the peeling loop */
    double t_total_ms;
    int64_t decrements; /* count decrements applied by Update over the run */
    double t_phase_ms[6];/* persistent peel kernel only (zeros otherwise): wall time per phase as seen
                            by block 0, barrier waits included: [0] level advance (minimum over the
                            bucket window), [1] window refill, [2] selection of A, [3] id-order
                            rebuild of A, [4] Update, [5] Update of the heavy r-cliques */
    double t_contract_ms;/* persistent peel kernel only: wall time of the graph contractions (block 0) */
    int64_t contractions;/* contractions run: (2,3) graph contraction (Section 5.6), by default one
                            whenever at least 2n edges were peeled since the previous one, compacting
                            the adjacency rows that lost at least a quarter of their entries since
                            then; (3,4) the same for the triangle lists, once 2m triangles were peeled */
    double t_hash_ms;   /* (3,4): the part of t_count_ms spent building the hash directory of the
                           triangle lists (0 otherwise); the counting kernel itself took
                           t_count_ms - t_hash_ms */
} nd_stats;

/* ---- context ------------------------------------------------------------------------- */

/* Create a context on CUDA device `device`. `stream` is a cudaStream_t to issue all work on
 * (NULL: the library creates and owns a non-blocking stream). `mem_budget` caps the device
 * bytes the context may hold at once (0: no cap). *out receives the handle.
 * Errors: ND_EINVAL (out NULL, bad device), ND_ECUDA. */
ND_API int nd_ctx_create(int device, void *stream, size_t mem_budget, nd_ctx **out);

/* Route the context's device allocations through caller hooks (e.g. a framework's caching
 * allocator). Must be called before any graph is loaded. Pass NULLs to restore the default
 * (cudaMallocAsync on the context's stream). Errors: ND_EINVAL, ND_EBUSY (graphs exist). */
ND_API int nd_ctx_set_allocator(nd_ctx *ctx, nd_alloc_fn alloc, nd_free_fn free_fn, void *user);

/* Limits of a context's decompositions (no counterpart in the paper; for callers that bound
 * the work of one call, and for tests of the failure paths). Each value 0 keeps the default.
 *   max_rounds          peeling rounds after which nd_decompose gives up with ND_ETIMEOUT
 *                       (default n_r + 2, which no graph reaches: every round peels >= 1 r-clique)
 *   barrier_timeout_ns  longest wait of a block of the persistent peel kernel at one grid barrier;
 *                       a block that waits longer, and every block that sees it gave up, leaves
 *                       the kernel and nd_decompose returns ND_ETIMEOUT (default 60 s)
 *   count_limit         largest s-clique count a width-4 count array may hold; a larger count
 *                       makes nd_count / nd_decompose with count_width 4 return ND_EOVERFLOW
 *                       (default 2^31 - 1; values above it are clamped to it)
 *   flags               ND_LIMIT_DROP_BLOCK: the last block of the persistent peel kernel leaves
 *                       before its first grid barrier, so the other blocks wait for an arrival that
 *                       never comes until barrier_timeout_ns runs out (a test of that bound)
 * Applies to calls that start after it returns. Errors: ND_EINVAL (NULL context, negative value). */
#define ND_LIMIT_DROP_BLOCK 0x1
ND_API int nd_ctx_set_limits(nd_ctx *ctx, int64_t max_rounds, int64_t barrier_timeout_ns, int64_t count_limit,
                             int32_t flags);

/* Per-(r,s) tuning of a context's decompositions (no counterpart in the paper), as chosen for
 * a device and a workload by an autotuner:
 *   heavy_work  length of an r-clique's driving list above which its Update runs on a whole block
 *               in the heavy phase instead of one warp (0: the built-in threshold: 4096 for most
 *               (r,s), 256 for (2,3), 96 for (2,4); (2,4) stages the common neighbourhood of a
 *               warp's edge in shared memory and takes at most 96)
 *   flags       ND_DENSE_BUCKETS and/or ND_CONTRACT_OFF, added to every nd_decompose of this (r,s)
 *               on the context (also inside batches and the server)
 * Errors: ND_EINVAL (NULL context, unsupported (r,s), negative threshold, other flags). */
ND_API int nd_ctx_set_tuning(nd_ctx *ctx, int r, int s, int64_t heavy_work, int32_t flags);

/* Destroy a context. All graphs created from it must have been freed (ND_EBUSY otherwise). */
ND_API int nd_ctx_destroy(nd_ctx *ctx);

/* Device bytes currently held by the context (0 for a NULL context). */
ND_API size_t nd_ctx_bytes_in_use(const nd_ctx *ctx);

/* Number of CUDA kernels this process has launched through the library so far (every node of
 * a replayed CUDA graph counts once per replay). */
ND_API int64_t nd_kernel_launches(void);

/* Human-readable description of the last error raised on the calling thread ("" if none).
 * The string stays valid until the next nd_* call on the same thread. */
ND_API const char *nd_last_error(void);

/* ---- graphs -------------------------------------------------------------------------- */

/* Copy a symmetric CSR graph (see conventions) to the device. n >= 0; rowptr int64[n+1];
 * col int32[rowptr[n]]. flags: ND_PTR_DEVICE, ND_VALIDATE. The caller keeps ownership of
 * its arrays. Errors: ND_EINVAL (bad sizes; malformed CSR with ND_VALIDATE), ND_ENOMEM,
 * ND_EOVERFLOW (more than 2^31 - 1 undirected edges). */
ND_API int nd_load_csr(nd_ctx *ctx, int32_t n, const int64_t *rowptr, const int32_t *col, int flags, nd_graph **out);

/* Free a graph and every device structure derived from it. NULL is accepted. */
ND_API int nd_graph_free(nd_graph *g);

/* Number of vertices and undirected edges of a loaded graph. */
ND_API int nd_graph_size(const nd_graph *g, int32_t *n, int64_t *m);

/* Orient the graph (Section 3, O(alpha)-orientation; Algorithm 2 line "Orient"): every edge
 * is directed from the lower to the higher vertex in a total order; mode selects the order
 * (ND_ORIENT_DEGREE or ND_ORIENT_DEGENERACY). Also builds the canonical edge index. Calling
 * it again with the same mode does nothing; another mode rebuilds the orientation. Vertex
 * ids are never changed: all outputs use the caller's ids. nd_count / nd_decompose orient
 * with ND_ORIENT_DEGREE if the graph is not oriented yet. Errors: ND_EINVAL, ND_ENOMEM. */
ND_API int nd_orient(nd_graph *g, int mode);

/* Discard the orientation and every derived index (the next call rebuilds them). */
ND_API int nd_graph_reset(nd_graph *g);

/* s-clique counts per r-clique (Algorithm 2, Count-Func over all s-cliques listed by
 * Algorithm 1). count_width: 4 (int32), 8 (int64) or 0 (4 if no count can exceed 2^31-1,
 * else 8). counts_out: NULL, or n_r values of count_width bytes in canonical order (host,
 * or device with ND_PTR_DEVICE). n_r_out / n_s_out (nullable, host) receive the numbers
 * of r- and s-cliques. To size counts_out, call first with counts_out = NULL.
 * Errors: ND_EINVAL, ND_ENOMEM, ND_EOVERFLOW (a count exceeds width 4 when width 4 was
 * asked for, or n_r >= 2^31). */
ND_API int nd_count(nd_graph *g, int r, int s, int count_width, void *counts_out, int flags, int64_t *n_r_out,
             int64_t *n_s_out);

/* (r,s) nucleus decomposition (Algorithm 2): core_out receives the core number of every
 * r-clique (int32[n_r], canonical order); round_out (nullable) the peeling round in which
 * each r-clique was removed (int32[n_r], rounds numbered from 0); st (nullable, host) the
 * statistics. Pointers are host memory unless flags has ND_PTR_DEVICE. core_out may be NULL
 * (only the statistics are produced). count_width as in nd_count.
 * Errors: ND_EINVAL, ND_ENOMEM, ND_EOVERFLOW, ND_ETIMEOUT (round cap), ND_EINTERNAL. */
ND_API int nd_decompose(nd_graph *g, int r, int s, int count_width, int32_t *core_out, int32_t *round_out, int flags,
                 nd_stats *st);

/* Per-round record of the last nd_decompose on this graph: sizes_out[t] = |A| peeled in
 * round t, levels_out[t] = level k of round t, for t < min(rho, cap). Host pointers.
 * *rho_out receives rho. Rounds past the device-side record limit (2^22) are not recorded.
 * Errors: ND_EINVAL (no decomposition yet). */
ND_API int nd_rounds(nd_graph *g, int64_t *sizes_out, int64_t *levels_out, int64_t cap, int64_t *rho_out);

/* Profiling aid (no counterpart in the paper): wall time in nanoseconds that the Update of each
 * round of the last nd_decompose on this graph took, as block 0 of the persistent peel kernel saw
 * it (barrier wait included): ns_out[t] for t < min(rho, cap). Zeros when the peel ran in another
 * launch mode. Host pointer. Errors: ND_EINVAL (no decomposition yet). */
ND_API int nd_round_times(nd_graph *g, int64_t *ns_out, int64_t cap);

/* The r-cliques themselves (the inverse index map, Section 5.3): tuples_out receives n_r
 * ascending tuples of r int32 vertex ids in canonical order (host, or device with
 * ND_PTR_DEVICE; NULL to query n_r only). r in {1, 2, 3, 4}. Errors: ND_EINVAL, ND_ENOMEM. */
ND_API int nd_rcliques(nd_graph *g, int r, int32_t *tuples_out, int flags, int64_t *n_r_out);

/* Connected nuclei at one level (Section 2, footnote: the definition of a c-(r,s) nucleus in
 * the nucleus literature also asks that its r-cliques be connected through s-cliques; the
 * paper's core numbers leave this out, and the nucleus hierarchy is built from it). core is
 * the r-clique core number array of an nd_decompose(g, r, s) (n_r int32, canonical order, host
 * or device with ND_PTR_DEVICE). X = the r-cliques with core >= level; two r-cliques of X are
 * joined when some s-clique contains both and has all C(s,r) of its r-subsets in X.
 * comp_out (n_r int32, same memory kind as core; nullable) receives, for each r-clique of X,
 * the smallest canonical id in its component, and -1 for the r-cliques outside X;
 * *n_comp_out (host, nullable) the number of components. Any core array is accepted (the
 * relation is then taken over the X it defines). Errors: ND_EINVAL (NULL graph or core,
 * unsupported (r,s)), ND_ENOMEM, ND_EOVERFLOW (more than INT32_MAX r-cliques), ND_EINTERNAL
 * (a bounded union-find retry loop ran out, or an r-subset is missing from the index). */
ND_API int nd_nuclei(nd_graph *g, int r, int s, const int32_t *core, int32_t level, int32_t *comp_out,
                     int flags, int64_t *n_comp_out);

/* The nucleus hierarchy (Section 2, footnote: the nested connected nuclei of all levels). For
 * each distinct core number c, the connected nuclei at level c are the components of X_c as in
 * nd_nuclei; a node of the hierarchy is such a component that holds an r-clique of core exactly
 * c, and every r-clique belongs to the node of its own core number. The parent of node (c, C) is
 * the node (c', C') at the largest distinct level c' < c whose component C' (of X_c') contains C;
 * nodes without one are roots (the hierarchy is a forest). core: as for nd_nuclei (values in
 * [0, 2^26)). Outputs, n_r int32 each, canonical order, same memory kind as core: comp_out[R] =
 * the smallest r-clique id of the component of R's node; parent_level_out[R] and
 * parent_comp_out[R] = the level and smallest id of the parent node of R's node, -1 and -1 for a
 * root. With host pointers any output may be NULL; with ND_PTR_DEVICE all three are required.
 * *n_nodes_out (host, nullable): the number of nodes. Cost: every s-clique is listed once over all
 * levels (one union-find over the r-cliques, levels taken in decreasing order). Errors:
 * ND_EINVAL (NULL graph or core, unsupported (r,s), a core value outside [0, 2^26)),
 * ND_ENOMEM, ND_EOVERFLOW (more than INT32_MAX r-cliques), ND_EINTERNAL (as for nd_nuclei). */
ND_API int nd_hierarchy(nd_graph *g, int r, int s, const int32_t *core, int32_t *comp_out, int32_t *parent_level_out,
                        int32_t *parent_comp_out, int flags, int64_t *n_nodes_out);

/* ---- batches and serving --------------------------------------------------------------
 * Many independent graphs, each with its own (r,s). A batch merges the graphs that share an
 * (r,s) into one disjoint union and runs a single decomposition on it: the core number of an
 * r-clique depends only on its own connected component, so every graph gets exactly the
 * numbers it would get alone, and the union's canonical order is the graphs' canonical orders
 * one after another. All graphs of a batch are peeled in the same device-resident rounds. */

typedef struct nd_request {
    int32_t n;             /* vertices */
    int32_t r, s;          /* a supported (r,s) */
    const int64_t *rowptr; /* host int64[n+1]: symmetric CSR as in nd_load_csr */
    const int32_t *col;    /* host int32[rowptr[n]] */
    int32_t *core_out;     /* host int32[n_r] receiving the core numbers in canonical order, or
                              NULL (only n_r is reported); caller-owned */
    int64_t core_cap;      /* capacity of core_out in elements (checked; ND_EINVAL if too small) */
    int64_t n_r;           /* out: number of r-cliques */
    int32_t status;        /* out: ND_OK or this request's error */
    int32_t pad;
} nd_request;

typedef struct nd_batch_stats {
    int32_t groups;        /* distinct (r,s) in the batch = union decompositions run */
    int32_t requests;
    int64_t n_r_total, n_s_total;
    int64_t rho_max;       /* most rounds of one union decomposition */
    double t_total_ms;     /* wall time of the whole call, copies included */
} nd_batch_stats;

/* Decompose count requests (host CSRs, host outputs) as one batch per distinct (r,s) on the
 * context's stream. Every request's status is set; the call returns ND_OK if all succeeded,
 * else the first failing request's status (the others still complete). st may be NULL. */
ND_API int nd_batch_run(nd_ctx *ctx, nd_request *reqs, int32_t count, nd_batch_stats *st);

typedef struct nd_server nd_server;

typedef struct nd_server_cfg {
    size_t mem_budget;     /* device bytes that admitted requests may hold at once (0: no cap);
                              admission uses a per-request estimate made before counting */
    int32_t workers;       /* batches running on the device at once, each on its own stream (>= 1) */
    int32_t max_batch;     /* most requests merged into one batch (>= 1) */
    int32_t queue_cap;     /* most requests waiting for admission; nd_submit returns ND_EBUSY beyond */
    int32_t flags;         /* how a worker launches a batch's peeling loop: 0 or ND_PEEL_LOOP_GRAPH (a CUDA
                              graph per batch; the workers' batches share the SMs), ND_PEEL_PERSISTENT
                              (one cooperative kernel per batch, holding every SM; batches take turns) */
} nd_server_cfg;

typedef struct nd_result {
    int32_t status;        /* ND_PENDING while queued or running, else the request's final status */
    int32_t batch_size;    /* requests in the batch that served it */
    int64_t n_r;
    double queue_ms;       /* nd_submit -> start of its batch */
    double run_ms;         /* start -> results written */
    double latency_ms;     /* nd_submit -> results written */
} nd_result;

/* Start a server on ctx's device: worker threads form batches from the queue (oldest request
 * first, merging waiting requests with the same (r,s)), admit them while the memory budget
 * allows, and run up to cfg->workers batches concurrently. Requests that arrive while batches
 * are on the GPU join the next batch a worker forms. Errors: ND_EINVAL, ND_ECUDA. */
ND_API int nd_server_create(nd_ctx *ctx, const nd_server_cfg *cfg, nd_server **out);

/* Queue a request. Its arrays (rowptr, col, core_out) must stay valid and untouched until
 * nd_poll reports a final status. *ticket identifies it. Errors: ND_EINVAL, ND_EBUSY (queue
 * full), ND_ENOMEM (its estimate alone exceeds the budget). */
ND_API int nd_submit(nd_server *sv, const nd_request *req, uint64_t *ticket);

/* Status of a ticket: returns ND_PENDING while it is queued or running, else its final status
 * (also in res->status) and, once final, forgets the ticket. res may be NULL.
 * Errors: ND_EINVAL (unknown ticket). */
ND_API int nd_poll(nd_server *sv, uint64_t ticket, nd_result *res);

/* Block until every submitted request has finished (their results stay pollable). */
ND_API int nd_server_drain(nd_server *sv);

/* Finish all queued and running requests, stop the workers and free the server. */
ND_API int nd_server_destroy(nd_server *sv);

/* ---- allocation-free entry point ----------------------------------------------------- */

/* Largest graph (in vertices) that nd_kcore_noalloc accepts. */
#define ND_NOALLOC_MAX_VERTICES 262144

/* k-core coreness ((1,2) nucleus numbers) of a graph already in device memory, without any
 * device or pinned-host allocation. The paper has no counterpart: this exists for callers that
 * cannot let a library allocate -- a framework that has reserved the GPU's memory in its own
 * caching pool (an allocation outside the pool can fail, or fragment memory, even though the
 * pool has room), or a latency-critical loop where cudaMalloc/cudaFree may synchronise the
 * device. It runs the same counting and peeling kernels as nd_decompose(g, 1, 2, ...), with all
 * scratch in one fixed static device array (about 8.4 MB, held by every GPU that loads the
 * library until the process exits).
 *   n        number of vertices, 0 <= n <= ND_NOALLOC_MAX_VERTICES (ND_EINVAL otherwise)
 *   rowptr   device int64[n+1], col device int32[rowptr[n]]: a symmetric CSR as in nd_load_csr
 *            (sorted rows, no loops, no duplicates; not validated here)
 *   core_out device int32[n], receives the coreness of every vertex
 *   stream   cudaStream_t to run on (NULL: the legacy default stream); the call returns after
 *            the work has finished on that stream. Runs on the calling thread's current device.
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress); make that first call before any stream capture. Every call shares
 * the array: calls whose work overlaps on the GPU
 * race and corrupt each other's results, so serialise them. Errors: ND_EINVAL, ND_ECUDA,
 * ND_ETIMEOUT, ND_EINTERNAL. */
ND_API int nd_kcore_noalloc(int32_t n, const int64_t *rowptr, const int32_t *col, int32_t *core_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ND_H */
