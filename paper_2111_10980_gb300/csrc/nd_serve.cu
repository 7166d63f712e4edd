// Batches and serving: many independent graphs per device-resident run.
//
// A batch merges the requests that share an (r,s) into one disjoint union (vertex ids shifted
// by the sizes of the graphs before it) and runs one decomposition on it. The (r,s) core number
// of an r-clique depends only on its connected component, so each graph receives exactly the
// numbers it gets alone; and because ids are shifted in request order, the union's canonical
// r-clique order is the requests' canonical orders concatenated, so each request's result is
// one contiguous slice. All graphs of a batch share the same peeling rounds, launches and CUDA
// graphs instead of one launch sequence per graph.
//
// The server keeps a FIFO queue. Each of cfg.workers threads owns a stream (its own context on
// the same device) and repeatedly forms a batch: the oldest waiting request plus later waiting
// requests with the same (r,s), up to cfg.max_batch, admitted while the sum of their memory
// estimates fits the budget next to the batches already running. Requests that arrive while
// batches run are picked up by the next worker that frees up, so their work overlaps with the
// batches already on the device (continuous batching at batch granularity).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nd.h"
#include "nd_common.cuh"
#include "nd_host.h"

namespace {

bool rs_ok(int r, int s) {
    return (r == 1 && s >= 2 && s <= 4) || (r == 2 && s >= 3 && s <= 5) || (r == 3 && s >= 4 && s <= 6) ||
           (r == 4 && s >= 5 && s <= 6);
}

__global__ void k_gather_offsets(const int64_t* __restrict__ ebase, const int64_t* __restrict__ tbase,
                                 const int64_t* __restrict__ qbase, const int64_t* __restrict__ voff, int64_t count,
                                 int r, int64_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= count; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = voff[i];
        int64_t o = v;
        if (r >= 2) o = ebase[v];
        if (r >= 3) o = tbase[o];
        if (r >= 4) o = qbase[o];
        out[i] = o;
    }
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Checks of a request's CSR on the host.
//  * check_cheap, O(n + nnz), run while a batch copies the request into its union: rowptr starts
//    at 0, never decreases and ends on an even count; every id lies in [0, n). After it, the
//    union (ids shifted request by request) only ever points inside the request's own range, so
//    the GPU validation of the union (ND_VALIDATE: sorted rows, no loops, symmetry) cannot read
//    outside any array and any violation it finds lies inside one request.
//  * check_request, O(nnz log d), everything the GPU validation checks; run only when the union
//    of a batch fails validation, to find the requests at fault, which then fail alone with
//    ND_EINVAL while the others run.
int check_args(const nd_request& q) {
    if (q.n < 0 || !q.rowptr || !rs_ok(q.r, q.s)) return ND_EINVAL;
    const int64_t* rp = q.rowptr;
    if (rp[0] != 0 || rp[q.n] < 0 || (rp[q.n] > 0 && !q.col) || (rp[q.n] & 1)) return ND_EINVAL;
    return ND_OK;
}

int check_cheap(const nd_request& q) {
    if (check_args(q)) return ND_EINVAL;
    const int64_t* rp = q.rowptr;
    for (int32_t u = 0; u < q.n; ++u)
        if (rp[u + 1] < rp[u]) return ND_EINVAL;
    const int64_t nnz = rp[q.n];
    uint32_t bad = 0;
    for (int64_t p = 0; p < nnz; ++p) bad |= (uint32_t)q.col[p] >= (uint32_t)q.n;
    return bad ? ND_EINVAL : ND_OK;
}

int check_request(const nd_request& q) {
    if (check_cheap(q)) return ND_EINVAL;
    const int64_t* rp = q.rowptr;
    for (int32_t u = 0; u < q.n; ++u) {
        for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
            int32_t v = q.col[p];
            if (v == u) return ND_EINVAL;
            if (p > rp[u] && q.col[p - 1] >= v) return ND_EINVAL;
            const int32_t* row = q.col + rp[v];
            int64_t lo = 0, hi = rp[v + 1] - rp[v];
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                if (row[mid] < u)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            if (lo >= rp[v + 1] - rp[v] || row[lo] != u) return ND_EINVAL;
        }
    }
    return ND_OK;
}

// Union of the requests' CSRs on the device: the staged rows and neighbour lists are copied as
// they are, then request k's row pointers are shifted by its first entry and its neighbour ids by
// its first vertex (offsets voff / eoff, one block per request).
__global__ void k_union_shift(int64_t* __restrict__ rp, int32_t* __restrict__ col, const int64_t* __restrict__ voff,
                              const int64_t* __restrict__ eoff, int64_t count) {
    for (int64_t k = blockIdx.x; k < count; k += gridDim.x) {
        const int64_t v0 = voff[k], v1 = voff[k + 1], e0 = eoff[k], e1 = eoff[k + 1];
        for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) rp[v] += e0;
        const int32_t sh = (int32_t)v0;
        for (int64_t p = e0 + threadIdx.x; p < e1; p += blockDim.x) col[p] += sh;
    }
}

// Pinned staging memory of a context (grown on demand, freed with the context).
void* stage_bytes(nd_ctx* ctx, size_t bytes) {
    if (ctx->stage_bytes < bytes) {
        if (ctx->stage) cudaFreeHost(ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_bytes = 0;
        size_t want = std::max(bytes, (size_t)1 << 20);
        if (cudaMallocHost(&ctx->stage, want) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ctx->stage_bytes = want;
    }
    return ctx->stage;
}

// Runs fn(i) for i in [0, count) on up to `threads` host threads (contiguous ranges).
template <typename F>
void parallel_for(int64_t count, int threads, F fn) {
    if (count <= 0) return;
    int t = (int)std::min<int64_t>(threads, count);
    if (t <= 1) {
        for (int64_t i = 0; i < count; ++i) fn(i);
        return;
    }
    std::vector<std::thread> th;
    for (int j = 0; j < t; ++j)
        th.emplace_back([=] {
            for (int64_t i = count * j / t; i < count * (j + 1) / t; ++i) fn(i);
        });
    for (auto& x : th) x.join();
}

int host_threads() {
    unsigned h = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(8u, h ? h : 1u));
}

// Runs one union decomposition for the requests in idx (all with the same (r,s)). A request whose
// CSR fails a check gets ND_EINVAL and is left out; the others run. peel_flags chooses how the
// peeling loop is launched: nd_batch_run takes the cooperative persistent kernel (one launch for
// the whole loop), the server's workers the loop graph, so that their batches share the SMs.
int run_group(nd_ctx* ctx, nd_request* const* reqs, std::vector<int> idx, nd_batch_stats* st, int peel_flags) {
    int r = reqs[idx[0]]->r, s = reqs[idx[0]]->s;
    cudaStream_t stream = ctx->stream;
    bool full_checks = false;  // set once the union of this group failed validation
    // every pass either removes at least one request, switches to the full checks (once), or runs
    // the decomposition and returns
    while (!idx.empty()) {
        const int64_t K = (int64_t)idx.size();
        std::vector<int64_t> voff(K + 1), eoff(K + 1);
        for (int64_t k = 0; k < K; ++k) {
            voff[k + 1] = voff[k] + reqs[idx[k]]->n;
            eoff[k + 1] = eoff[k] + reqs[idx[k]]->rowptr[reqs[idx[k]]->n];
        }
        const int64_t total_n = voff[K], total_nnz = eoff[K];
        if (total_n > INT32_MAX) return nd_set_error(ND_EOVERFLOW, "batch: more than 2^31-1 vertices in one (r,s) group");
        // stage rows and lists (pinned), checking each request on the way
        size_t rp_bytes = sizeof(int64_t) * (total_n + 1), col_bytes = sizeof(int32_t) * total_nnz;
        size_t col_at = (rp_bytes + 15) & ~(size_t)15;
        char* stg = (char*)stage_bytes(ctx, col_at + col_bytes + 16);
        if (!stg) return nd_set_error(ND_ENOMEM, "batch: pinned staging of %zu bytes failed", col_at + col_bytes);
        int64_t* hrp = (int64_t*)stg;
        int32_t* hcol = (int32_t*)(stg + col_at);
        std::vector<int> bad(K, 0);
        parallel_for(K, host_threads(), [&](int64_t k) {
            const nd_request& q = *reqs[idx[k]];
            bad[k] = full_checks ? check_request(q) : check_cheap(q);
            if (bad[k]) return;
            memcpy(hrp + voff[k], q.rowptr, sizeof(int64_t) * q.n);
            int64_t nnz = q.rowptr[q.n];
            if (nnz) memcpy(hcol + eoff[k], q.col, sizeof(int32_t) * nnz);
        });
        bool any_bad = false;
        for (int64_t k = 0; k < K; ++k) any_bad |= bad[k] != 0;
        if (any_bad) {
            std::vector<int> keep;
            for (int64_t k = 0; k < K; ++k) {
                if (bad[k])
                    reqs[idx[k]]->status = ND_EINVAL;
                else
                    keep.push_back(idx[k]);
            }
            idx.swap(keep);
            continue;  // restage the others
        }
        hrp[total_n] = total_nnz;
        DBuf drp, dcol, doffs;
        int rc = nd_alloc(ctx, drp, rp_bytes);
        if (!rc) rc = nd_alloc(ctx, dcol, std::max<size_t>(col_bytes, 4));
        if (!rc) rc = nd_alloc(ctx, doffs, sizeof(int64_t) * 2 * (K + 1));
        if (!rc) {
            cudaMemcpyAsync(drp.p, hrp, rp_bytes, cudaMemcpyHostToDevice, stream);
            if (col_bytes) cudaMemcpyAsync(dcol.p, hcol, col_bytes, cudaMemcpyHostToDevice, stream);
            cudaMemcpyAsync(doffs.p, voff.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, stream);
            cudaMemcpyAsync((int64_t*)doffs.p + (K + 1), eoff.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice,
                            stream);
            int blocks = (int)std::min<int64_t>(K, (int64_t)nd_sm_count() * 8);
            ND_K(k_union_shift<<<blocks, 256, 0, stream>>>((int64_t*)drp.p, (int32_t*)dcol.p, (const int64_t*)doffs.p,
                                                          (const int64_t*)doffs.p + (K + 1), K));
            rc = nd_check_launch("batch union");
        }
        nd_graph* g = nullptr;
        if (!rc)
            rc = nd_load_csr(ctx, (int32_t)total_n, (const int64_t*)drp.p, (const int32_t*)dcol.p,
                             ND_PTR_DEVICE | ND_VALIDATE, &g);
        nd_free(ctx, drp);
        nd_free(ctx, dcol);
        if (rc == ND_EINVAL && !full_checks) {
            // the union is malformed inside some request: find it with the full host check
            nd_free(ctx, doffs);
            full_checks = true;
            continue;
        }
        if (rc) {
            nd_free(ctx, doffs);
            return rc;
        }
        PeelOut po;
        nd_stats S;
        rc = nd_decompose_dev(g, r, s, 0, peel_flags, po, &S);
        std::vector<int64_t> off(K + 1);
        if (!rc) {
            // canonical offset of each request's first r-clique: r = 1 its first vertex, r = 2 the
            // edge base there, r = 3 the triangle base at that edge, r = 4 the 4-clique base at that
            // triangle
            GraphView v = nd_view(g);
            ND_K(k_gather_offsets<<<std::max<int64_t>(1, (K + 1 + 255) / 256), 256, 0, stream>>>(
                v.ebase, v.tbase, v.qbase, (const int64_t*)doffs.p, K, r, (int64_t*)doffs.p + (K + 1)));
            rc = nd_check_launch("batch offsets");
            if (!rc) {
                cudaMemcpyAsync(off.data(), (int64_t*)doffs.p + (K + 1), sizeof(int64_t) * (K + 1),
                                cudaMemcpyDeviceToHost, stream);
                rc = nd_sync(ctx, "batch offsets");
            }
        }
        nd_free(ctx, doffs);
        if (!rc) {
            int32_t* hcore = S.n_r ? (int32_t*)stage_bytes(ctx, sizeof(int32_t) * S.n_r) : nullptr;
            if (S.n_r && !hcore) rc = nd_set_error(ND_ENOMEM, "batch: pinned staging of the results failed");
            if (!rc && S.n_r) {
                cudaMemcpyAsync(hcore, po.core.p, sizeof(int32_t) * S.n_r, cudaMemcpyDeviceToHost, stream);
                rc = nd_sync(ctx, "batch results");
            }
            if (!rc) {
                parallel_for(K, host_threads(), [&](int64_t k) {
                    nd_request& q = *reqs[idx[k]];
                    int64_t a = off[k], b = off[k + 1];
                    q.n_r = b - a;
                    if (q.core_out) {
                        if (q.core_cap < q.n_r) {
                            q.status = ND_EINVAL;
                            return;
                        }
                        if (b > a) memcpy(q.core_out, hcore + a, sizeof(int32_t) * (b - a));
                    }
                    q.status = ND_OK;
                });
                if (st) {
                    st->n_r_total += S.n_r;
                    st->n_s_total += S.n_s;
                    st->rho_max = std::max<int64_t>(st->rho_max, S.rho);
                }
            }
        }
        nd_free(ctx, po.core);
        nd_free(ctx, po.rnd);
        nd_graph_free(g);
        return rc;
    }
    return ND_OK;
}

int batch_impl(nd_ctx* ctx, nd_request* const* reqs, int count, nd_batch_stats* st, int peel_flags) {
    double t0 = now_ms();
    if (st) {
        memset(st, 0, sizeof(*st));
        st->requests = count;
    }
    std::vector<std::pair<int, int>> keys;
    std::vector<std::vector<int>> groups;
    int first_err = ND_OK;
    for (int i = 0; i < count; ++i) {
        nd_request& q = *reqs[i];
        q.n_r = 0;
        q.status = check_args(q);
        if (q.status) {
            if (!first_err) first_err = q.status;
            continue;
        }
        std::pair<int, int> key(q.r, q.s);
        size_t gi = std::find(keys.begin(), keys.end(), key) - keys.begin();
        if (gi == keys.size()) {
            keys.push_back(key);
            groups.emplace_back();
        }
        groups[gi].push_back(i);
    }
    for (auto& grp : groups) {
        int rc = run_group(ctx, reqs, grp, st, peel_flags);
        if (rc) {
            for (int i : grp) reqs[i]->status = rc;
            if (!first_err) first_err = rc;
        }
        if (st) st->groups++;
    }
    for (int i = 0; i < count; ++i)
        if (reqs[i]->status && !first_err) first_err = reqs[i]->status;
    if (st) st->t_total_ms = now_ms() - t0;
    if (first_err) return nd_set_error(first_err, "batch: %s", nd_last_error());
    return ND_OK;
}

// A memory estimate for one request made before anything is counted: CSR, edge index and
// orientation, plus per r-clique state; for r = 3 the triangle count is bounded by the wedge
// count / 3 and by m sqrt(2m) / 3.
size_t estimate_bytes(const nd_request& q) {
    double n = q.n, m = (double)q.rowptr[q.n] / 2.0;
    double bytes = 16 * (n + 1) + 8 * 2 * m + 16 * n + 4 * 2 * m + 8 * m + 8 * (n + 1) + 8 * m;
    double nr = q.r == 1 ? n : m;
    if (q.r == 3) {
        double w = 0;
        for (int32_t v = 0; v < q.n; ++v) {
            double d = (double)(q.rowptr[v + 1] - q.rowptr[v]);
            w += d * (d - 1) / 2;
        }
        nr = std::min(w / 3.0, m * std::sqrt(2.0 * m) / 3.0);
        // per-edge table bounds + three entries per triangle; the peel adds the lists' hash
        // directory (at most 4 slots of 16 bytes per entry, a slot index per entry) and an offset
        // per edge
        bytes += 16 * m + 48 * nr + 8 * m + 204 * nr;
    }
    bytes += 40 * nr + 64 * 1024;  // counts, rounds, cores, work lists, control block
    return (size_t)bytes;
}

}  // namespace

extern "C" int nd_batch_run(nd_ctx* ctx, nd_request* reqs, int32_t count, nd_batch_stats* st) {
    if (!ctx || (count > 0 && !reqs) || count < 0) return nd_set_error(ND_EINVAL, "nd_batch_run: bad arguments");
    cudaSetDevice(ctx->device);
    std::vector<nd_request*> ptrs(count);
    for (int i = 0; i < count; ++i) ptrs[i] = &reqs[i];
    return batch_impl(ctx, ptrs.data(), count, st, 0);
}

// ------------------------------------------------------------------------------------
// server

struct Ticket {
    nd_request req;
    uint64_t id = 0;
    int32_t status = ND_PENDING;
    int32_t batch_size = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    size_t est = 0;
};

struct nd_server {
    nd_ctx* ctx = nullptr;
    nd_server_cfg cfg;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Ticket*> queue;
    std::unordered_map<uint64_t, Ticket*> tickets;
    uint64_t next_id = 1;
    size_t used = 0;
    int running = 0;
    int64_t unfinished = 0;
    bool stop = false;
    std::vector<std::thread> threads;
    std::vector<nd_ctx*> wctx;
};

static void worker_loop(nd_server* sv, int w) {
    cudaSetDevice(sv->ctx->device);
    nd_ctx* ctx = sv->wctx[w];
    for (;;) {
        std::vector<Ticket*> batch;
        size_t est = 0;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] {
                if (sv->stop && sv->queue.empty()) return true;
                if (sv->queue.empty()) return false;
                size_t need = sv->queue.front()->est;
                return sv->cfg.mem_budget == 0 || sv->used + need <= sv->cfg.mem_budget || sv->running == 0;
            });
            if (sv->queue.empty()) return;  // stopping
            Ticket* head = sv->queue.front();
            int r = head->req.r, s = head->req.s;
            for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)batch.size() < sv->cfg.max_batch;) {
                Ticket* t = *it;
                bool fits = sv->cfg.mem_budget == 0 || sv->used + est + t->est <= sv->cfg.mem_budget ||
                            (batch.empty() && sv->running == 0);
                if (t->req.r == r && t->req.s == s && fits) {
                    batch.push_back(t);
                    est += t->est;
                    it = sv->queue.erase(it);
                } else if (t == head) {
                    break;  // the oldest request does not fit yet
                } else {
                    ++it;
                }
            }
            sv->used += est;
            sv->running++;
        }
        double t0 = now_ms();
        std::vector<nd_request*> reqs(batch.size());
        for (size_t i = 0; i < batch.size(); ++i) reqs[i] = &batch[i]->req;
        batch_impl(ctx, reqs.data(), (int)reqs.size(), nullptr,
                   sv->cfg.flags == ND_PEEL_PERSISTENT ? ND_PEEL_PERSISTENT : ND_PEEL_LOOP_GRAPH);
        double t1 = now_ms();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (Ticket* t : batch) {
                t->t_start = t0;
                t->t_done = t1;
                t->batch_size = (int32_t)batch.size();
                t->status = t->req.status;
                sv->unfinished--;
            }
            sv->used -= est;
            sv->running--;
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

extern "C" int nd_server_create(nd_ctx* ctx, const nd_server_cfg* cfg, nd_server** out) {
    if (!ctx || !cfg || !out) return nd_set_error(ND_EINVAL, "nd_server_create: NULL argument");
    if (cfg->workers < 1 || cfg->max_batch < 1 || cfg->queue_cap < 1)
        return nd_set_error(ND_EINVAL, "nd_server_create: workers, max_batch and queue_cap must be >= 1");
    if (cfg->flags != 0 && cfg->flags != ND_PEEL_LOOP_GRAPH && cfg->flags != ND_PEEL_PERSISTENT)
        return nd_set_error(ND_EINVAL, "nd_server_create: flags must be 0, ND_PEEL_LOOP_GRAPH or ND_PEEL_PERSISTENT");
    nd_server* sv = new nd_server();
    sv->ctx = ctx;
    sv->cfg = *cfg;
    for (int w = 0; w < cfg->workers; ++w) {
        nd_ctx* c = nullptr;
        int rc = nd_ctx_create(ctx->device, nullptr, 0, &c);
        if (rc) {
            for (nd_ctx* x : sv->wctx) nd_ctx_destroy(x);
            delete sv;
            return rc;
        }
        nd_ctx_set_allocator(c, ctx->af, ctx->ff, ctx->user);
        // the workers decompose with the server context's limits and tuning
        c->max_rounds = ctx->max_rounds;
        c->barrier_ns = ctx->barrier_ns;
        c->count_limit = ctx->count_limit;
        for (int i = 0; i < 64; ++i) {
            c->tune_heavy[i] = ctx->tune_heavy[i];
            c->tune_flags[i] = ctx->tune_flags[i];
        }
        sv->wctx.push_back(c);
    }
    for (int w = 0; w < cfg->workers; ++w) sv->threads.emplace_back(worker_loop, sv, w);
    *out = sv;
    return ND_OK;
}

extern "C" int nd_submit(nd_server* sv, const nd_request* req, uint64_t* ticket) {
    if (!sv || !req || !ticket) return nd_set_error(ND_EINVAL, "nd_submit: NULL argument");
    if (check_args(*req)) return nd_set_error(ND_EINVAL, "nd_submit: malformed request");
    Ticket* t = new Ticket();
    t->req = *req;
    t->req.status = ND_PENDING;
    t->est = estimate_bytes(*req);
    t->t_submit = now_ms();
    if (sv->cfg.mem_budget && t->est > sv->cfg.mem_budget) {
        size_t e = t->est;
        delete t;
        return nd_set_error(ND_ENOMEM, "nd_submit: request needs about %zu bytes, budget is %zu", e,
                            sv->cfg.mem_budget);
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            delete t;
            return nd_set_error(ND_EINVAL, "nd_submit: server is stopping");
        }
        if ((int)sv->queue.size() >= sv->cfg.queue_cap) {
            delete t;
            return nd_set_error(ND_EBUSY, "nd_submit: queue full (%d requests)", sv->cfg.queue_cap);
        }
        t->id = sv->next_id++;
        sv->tickets[t->id] = t;
        sv->queue.push_back(t);
        sv->unfinished++;
        *ticket = t->id;
    }
    sv->cv_work.notify_one();
    return ND_OK;
}

extern "C" int nd_poll(nd_server* sv, uint64_t ticket, nd_result* res) {
    if (!sv) return nd_set_error(ND_EINVAL, "nd_poll: NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return nd_set_error(ND_EINVAL, "nd_poll: unknown ticket %llu", (unsigned long long)ticket);
    Ticket* t = it->second;
    if (res) {
        memset(res, 0, sizeof(*res));
        res->status = t->status;
        res->batch_size = t->batch_size;
        res->n_r = t->req.n_r;
        if (t->status != ND_PENDING) {
            res->queue_ms = t->t_start - t->t_submit;
            res->run_ms = t->t_done - t->t_start;
            res->latency_ms = t->t_done - t->t_submit;
        }
    }
    int st = t->status;
    if (st != ND_PENDING) {
        sv->tickets.erase(it);
        delete t;
    }
    return st;
}

extern "C" int nd_server_drain(nd_server* sv) {
    if (!sv) return nd_set_error(ND_EINVAL, "nd_server_drain: NULL server");
    std::unique_lock<std::mutex> lk(sv->mu);
    sv->cv_done.wait(lk, [&] { return sv->unfinished == 0; });
    return ND_OK;
}

extern "C" int nd_server_destroy(nd_server* sv) {
    if (!sv) return ND_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto& th : sv->threads) th.join();
    for (nd_ctx* c : sv->wctx) nd_ctx_destroy(c);
    for (auto& kv : sv->tickets) delete kv.second;
    delete sv;
    return ND_OK;
}
