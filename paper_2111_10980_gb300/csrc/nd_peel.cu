// The peeling loop of Algorithm 2 on the device: bucket extraction (the "next bucket"), the
// Update subroutine with Update-Func, and the bookkeeping of "finished".
//
// Rounds. Each round t peels A_t = every unpeeled r-clique with count <= k, after
// k = max(k, minimum unpeeled count) (the bucketing structure keeps r-cliques whose count
// falls below the current bucket in that bucket; core numbers never decrease). All state
// lives in device memory and every decision is taken on the device, so a round is a fixed
// sequence of launches (k_ctl, k_adv_min, four refill kernels, k_adv_select, k_update_rs)
// that can be captured once in a CUDA graph and replayed until the done flag is set.
//
// Bucketing without scanning every r-clique each round (Section 3, "Parallel Bucketing": only
// the lowest buckets are materialised and empty ranges are skipped):
//   * same-level rounds: an r-clique whose count crosses from > k to <= k during round t's
//     update is appended to the next round's A (it is exactly A_{t+1} when k does not move);
//     its round and core number are written at that moment;
//   * level advances: N is a window list holding every unpeeled r-clique with count < hi;
//     the new level is the minimum count over N and the new A is selected from N, which is
//     compacted at the same time; an r-clique whose count crosses hi from above is appended
//     to N by the update that decrements it;
//   * refill: when N has no unpeeled member, the alive list L is compacted, a 4096-bin
//     histogram of counts above the global minimum picks hi so that N holds about 1/16 of
//     the unpeeled r-cliques (at least 16384), and N is rebuilt.
//
// Update / Update-Func (Algorithm 2) with exact integers. For every R in A, the warp assigned
// to R lists every s-clique S containing R. With round[] = the round in which each r-clique
// was peeled (UNPEELED if alive; t for members of A; t+1 for r-cliques already queued for the
// next round, which are still alive now):
//   * if some r-subset of S has round < t, S was destroyed earlier: skip (the "previously
//     peeled" test of Update-Func);
//   * otherwise the owner of S is its smallest r-subset id with round == t; only the owner's
//     warp applies S's effect, subtracting exactly 1 from every r-subset not in A. The paper
//     has each of the a members of A subtract 1/a; the owner rule gives the same total (1 per
//     live S and surviving member) with integer atomics and without double counting.
// Warps take A in dynamic chunks; r-cliques with long driving lists go to a heavy phase that
// gives each a block ((2,4) in the persistent kernel: stage per block, then the pairs of all
// heavy edges over the whole grid).
//
// Also here: the (2,3) graph contraction of Section 5.6 (rows that lost a quarter of their entries
// are compacted once 2n edges were peeled since the previous contraction), the dense buckets with
// the doubling search of Section 4.2 (Discussion) as an alternative way to find the next level,
// and the three launch modes of the loop: one cooperative persistent kernel (default), one CUDA
// graph with WHILE / IF nodes, or every phase launched.
#include "nd_common.cuh"
#include "nd_gen.cuh"

#include <climits>
#include <cstring>

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int64_t gwarp() { return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int64_t nwarps() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }
__device__ __forceinline__ int64_t gthread() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t nthreads() { return (int64_t)gridDim.x * blockDim.x; }

__device__ __forceinline__ int64_t knew_of(const PeelCtl* c) {
    unsigned long long mn = c->minN != ULLONG_MAX ? c->minN : c->gmin;
    int64_t m = mn == ULLONG_MAX ? c->k : (int64_t)mn;
    return m > c->k ? m : c->k;
}

// a[i] for a two-entry pointer array without dynamic indexing (which would copy the kernel
// parameter block to local memory)
__device__ __forceinline__ int32_t* pick(int32_t* const (&a)[2], int i) { return i ? a[1] : a[0]; }

// (3,4): tag the three index entries of triangle R (and its hash-directory slots) with the round
// in which it is peeled. Out of line with plain pointer arguments: it runs once per triangle, and
// inlined into Update's decrement path it would cost registers there.
__device__ __noinline__ void tri_round_write(const int32_t* tri_e, const int64_t* et_rp, const int32_t* tri_pos,
                                             int32_t* et_rnd, const int32_t* hpos, const int64_t* hoff,
                                             NdHashSlot* htab, int64_t R, int32_t round) {
    for (int x = 0; x < 3; ++x) {
        int32_t e = tri_e[3 * R + x];
        et_rnd[et_rp[e] + tri_pos[3 * R + x]] = round;
        if (hpos) {
            int32_t s = hpos[3 * R + x];
            if (s >= 0) htab[hoff[e] + s].rnd = round;
        }
    }
}

template <typename CT>
__device__ __forceinline__ void set_tri_round(const PeelView<CT>& P, int64_t R, int32_t round) {
    tri_round_write(P.tri_e, P.et_rp, P.tri_pos, P.et_rnd, P.hpos, P.hoff, P.htab, R, round);
}

// Membership bitmap of the next / current A (bit x set while x is scheduled and not yet updated):
// large rounds rebuild A from it in ascending id order, so that warps running side by side work
// on triangles (edges) that share lists and the lists' lines are reused from L2.
template <typename CT>
__device__ __forceinline__ void mark_a(const PeelView<CT>& P, int32_t x) {
    if (P.abits) atomicOr(&P.abits[x >> 5], 1u << (x & 31));
}
template <typename CT>
__device__ __forceinline__ void unmark_a(const PeelView<CT>& P, int32_t x) {
    if (P.abits) atomicAnd(&P.abits[x >> 5], ~(1u << (x & 31)));
}

// list sizes read back from the control block never exceed the list capacity (an overflow sets
// ctl->err and is reported by the host)
__device__ __forceinline__ unsigned clampn(unsigned v, uint32_t cap) { return v < cap ? v : cap; }

__device__ __forceinline__ bool need_refill(const PeelCtl* c) {
    return !c->done && (c->mode & ND_MODE_ADV) && c->minN == ULLONG_MAX;
}

__device__ __forceinline__ unsigned long long block_min(unsigned long long v) {
    __shared__ unsigned long long sm[32];
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_down_sync(0xffffffffu, v, o);
        v = y < v ? y : v;
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sm[lane] : ULLONG_MAX;
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long y = __shfl_down_sync(0xffffffffu, v, o);
            v = y < v ? y : v;
        }
    }
    return v;  // valid in thread 0
}

__global__ void k_init(PeelCtl* c, int64_t n_r, int64_t max_rounds, unsigned long long barrier_ns, int drop_block,
                       int64_t contract_every, int contract_shift) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c->bar_timeout_ns = barrier_ns;
        c->drop_block = drop_block;
        c->contract = 0;
        c->contract_every = contract_every;
        c->contract_shift = contract_shift;
        c->peeled_since = 0;
        c->contractions = 0;
        c->t = 0;
        c->mode = 0;
        c->done = 0;
        c->err = 0;
        c->started = 0;
        c->wa = c->wn = c->wl = 0;
        c->lmat = 0;
        c->heavy = 0;
        c->sorta = 0;
        for (int i = 0; i < 7; ++i) c->ph_ns[i] = 0;
        c->ph_last = 0;
        c->k = 0;
        c->hi = 0;
        c->finished = 0;
        c->n_r = n_r;
        c->max_rounds = max_rounds;
        c->nA = c->cntA = c->nNext = c->nN = c->nN2 = c->nL = c->nL2 = c->nH = 0;
        c->upd_next = 0;
        c->minN = c->gmin = ULLONG_MAX;
        c->listed = 0;
        c->decs = 0;
        c->bar_arrive = 0;
        c->bar_gen = 0;
        c->advances = c->refills = 0;
    }
}

// Finishes round t-1 and sets up round t (one thread). When the rounds run inside a CUDA graph
// WHILE node, it also sets the loop condition (continue while not done) and the IF condition of
// the level-advance phase.
__device__ void ctl_step(PeelCtl* c, int64_t* round_size, int64_t* round_level, int64_t round_cap);

__global__ void k_ctl(PeelCtl* c, int64_t* round_size, int64_t* round_level, int64_t round_cap, int use_cond,
                      cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_adv) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    ctl_step(c, round_size, round_level, round_cap);
    if (use_cond) {
        cudaGraphSetConditional(h_loop, c->done ? 0u : 1u);
        cudaGraphSetConditional(h_adv, (!c->done && (c->mode & ND_MODE_ADV)) ? 1u : 0u);
    }
}

// IF condition of the refill phase: the window N holds no unpeeled r-clique
__global__ void k_set_refill(PeelCtl* c, cudaGraphConditionalHandle h_refill) {
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h_refill, need_refill(c) ? 1u : 0u);
}

__device__ void ctl_step(PeelCtl* c, int64_t* round_size, int64_t* round_level, int64_t round_cap) {
    if (c->done) return;
    if (c->started) {
        bool adv = c->mode & ND_MODE_ADV;
        unsigned nA = adv ? c->cntA : c->nA;
        if (adv) {
            c->k = knew_of(c);
            c->nN = c->nN2;
            c->wn ^= 1;
            c->advances++;
        }
        if (c->t < round_cap) {
            round_size[c->t] = nA;
            round_level[c->t] = c->k;
        }
        c->finished += nA;
        c->peeled_since += nA;
        c->t += 1;
        if (c->finished >= c->n_r) {
            c->done = 1;
            return;
        }
        if (nA == 0) {  // an empty round cannot happen in a consistent state
            c->err |= 4;
            c->done = 1;
            return;
        }
        if (c->t >= c->max_rounds) {
            c->err |= 2;
            c->done = 1;
            return;
        }
    } else {
        c->started = 1;
        if (c->n_r == 0) {
            c->done = 1;
            return;
        }
    }
    c->nH = 0;
    c->upd_next = 0;
    // graph contraction (Section 5.6) once enough r-cliques were peeled since the previous one
    c->contract = c->contract_every > 0 && c->peeled_since >= c->contract_every;
    if (c->contract) {
        c->peeled_since = 0;
        c->contractions++;
    }
    if (c->nNext > 0) {
        c->wa ^= 1;
        c->nA = c->nNext;
        c->nNext = 0;
        c->mode = 0;
    } else {
        c->mode = ND_MODE_ADV;
        c->nA = 0;
        c->cntA = 0;
        c->nN2 = 0;
        c->minN = ULLONG_MAX;
        c->gmin = ULLONG_MAX;
    }
}

// Dense buckets: the new level is the first non-empty bucket at or above k, found by the
// doubling search of Section 4.2 (Discussion): regions [k, k+1), [k+1, k+3), [k+3, k+7), ... of
// sizes 1, 2, 4, ... are searched in turn, each by all threads of block 0 at once, until one holds
// a non-empty bucket. Work O(distance to the next bucket), O(log) steps. Every unpeeled r-clique
// not yet scheduled has a count above k after the first round, so nothing below k is missed. If
// that bucket lies inside the window (count < hi) it is the window's minimum; else the window
// has no unpeeled member and is refilled as usual.
template <typename CT>
__device__ void dense_min(const PeelView<CT>& P) {
    PeelCtl* c = P.ctl;
    if (blockIdx.x != 0) return;
    __shared__ unsigned long long s_found;
    if (threadIdx.x == 0) s_found = ULLONG_MAX;
    __syncthreads();
    int64_t lo = c->k, span = 1;
    unsigned long long got = ULLONG_MAX;
    while (lo < P.bmax) {
        int64_t hi = lo + span < P.bmax ? lo + span : P.bmax;
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
            if (P.bcnt[i]) {
                atomicMin(&s_found, (unsigned long long)i);
                break;
            }
        __syncthreads();
        got = s_found;
        __syncthreads();
        if (got != ULLONG_MAX) break;
        lo = hi;
        span *= 2;
    }
    if (threadIdx.x == 0 && got != ULLONG_MAX && (int64_t)got < c->hi) c->minN = got;
}

template <typename CT>
__device__ void phase_adv_min(const PeelView<CT>& P) {
    PeelCtl* c = P.ctl;
    if (c->done || !(c->mode & ND_MODE_ADV)) return;
    if (P.bcnt) {
        dense_min(P);
        return;
    }
    const int32_t* N = pick(P.N, c->wn);
    unsigned n = clampn(c->nN, P.cap);
    unsigned long long mn = ULLONG_MAX;
    for (int64_t i = gthread(); i < n; i += nthreads()) {
        int32_t R = N[i];
        if (P.rnd[R] == ND_UNPEELED) {
            unsigned long long v = (unsigned long long)P.cnt[R];
            mn = v < mn ? v : mn;
        }
    }
    mn = block_min(mn);
    if (threadIdx.x == 0 && mn != ULLONG_MAX) atomicMin(&c->minN, mn);
}

// refill 1/4: compact L into L' (alive only), global minimum count, clear the histogram
template <typename CT>
__device__ void phase_refill_scan(const PeelView<CT>& P) {
    PeelCtl* c = P.ctl;
    if (!need_refill(c)) return;
    for (int64_t i = gthread(); i < ND_HBINS; i += nthreads()) c->hist[i] = 0;
    const int32_t* L = pick(P.L, c->wl);
    int32_t* L2 = pick(P.L, c->wl ^ 1);
    int64_t n = c->lmat ? (int64_t)clampn(c->nL, P.cap) : c->n_r;
    unsigned long long mn = ULLONG_MAX;
    // grid-stride in whole-warp steps so that appends aggregate per warp
    for (int64_t base = gthread() - (threadIdx.x & 31); base < n; base += nthreads()) {
        int64_t i = base + (threadIdx.x & 31);
        if (i < n) {
            int32_t R = c->lmat ? L[i] : (int32_t)i;
            if (P.rnd[R] == ND_UNPEELED) {
                unsigned long long v = (unsigned long long)P.cnt[R];
                mn = v < mn ? v : mn;
                nd_append(&c->nL2, L2, P.cap, R, &c->err);
            }
        }
    }
    mn = block_min(mn);
    if (threadIdx.x == 0 && mn != ULLONG_MAX) atomicMin(&c->gmin, mn);
}

// refill 2/4: histogram of count - gmin over L'
template <typename CT>
__device__ void phase_refill_hist(const PeelView<CT>& P) {
    PeelCtl* c = P.ctl;
    if (!need_refill(c)) return;
    __shared__ unsigned int h[ND_HBINS];
    for (int i = threadIdx.x; i < ND_HBINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int32_t* L2 = pick(P.L, c->wl ^ 1);
    unsigned n = clampn(c->nL2, P.cap);
    unsigned long long g0 = c->gmin;
    for (int64_t i = gthread(); i < n; i += nthreads()) {
        unsigned long long d = (unsigned long long)P.cnt[L2[i]] - g0;
        atomicAdd(&h[d < ND_HBINS - 1 ? d : ND_HBINS - 1], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ND_HBINS; i += blockDim.x)
        if (h[i]) atomicAdd(&c->hist[i], (unsigned long long)h[i]);
}

// refill 3/4 (one block; any multiple of 32 threads dividing ND_HBINS): choose hi so that the
// window holds about 1/16 of the unpeeled r-cliques (at least 16384), swap L <- L', clear N
__device__ void phase_refill_pick(PeelCtl* c) {
    if (!need_refill(c)) return;
    __shared__ unsigned long long part[1024];
    __shared__ int best;
    const int nt = blockDim.x;
    const int per = ND_HBINS / nt;
    unsigned long long s = 0;
    for (int j = 0; j < per; ++j) s += c->hist[threadIdx.x * per + j];
    part[threadIdx.x] = s;
    if (threadIdx.x == 0) best = ND_HBINS - 1;
    __syncthreads();
    // inclusive scan of part[0..nt) (Hillis-Steele)
    for (int o = 1; o < nt; o <<= 1) {
        unsigned long long y = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += y;
        __syncthreads();
    }
    unsigned long long alive = c->nL2;
    unsigned long long target = alive / 16;
    if (target < 16384) target = 16384;
    unsigned long long run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int j = 0; j < per; ++j) {
        run += c->hist[threadIdx.x * per + j];
        if (run >= target) {
            atomicMin(&best, threadIdx.x * per + j);
            break;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int b = best;
        c->hi = (b >= ND_HBINS - 1) ? LLONG_MAX : (int64_t)c->gmin + b + 1;
        c->wl ^= 1;
        c->nL = c->nL2;
        c->nL2 = 0;
        c->lmat = 1;
        c->nN = 0;
        c->refills++;
    }
    __syncthreads();
}

__global__ void k_refill_pick(PeelCtl* c) { phase_refill_pick(c); }

// The same choice made by one thread (the serial part of a grid barrier).
__device__ void refill_pick_serial(PeelCtl* c) {
    unsigned long long alive = c->nL2;
    unsigned long long target = alive / 16;
    if (target < 16384) target = 16384;
    unsigned long long run = 0;
    int b = ND_HBINS - 1;
    for (int i = 0; i < ND_HBINS; ++i) {
        run += c->hist[i];
        if (run >= target) {
            b = i;
            break;
        }
    }
    c->hi = (b >= ND_HBINS - 1) ? LLONG_MAX : (int64_t)c->gmin + b + 1;
    c->wl ^= 1;
    c->nL = c->nL2;
    c->nL2 = 0;
    c->lmat = 1;
    c->nN = 0;
    c->refills++;
}

// refill 4/4: N = { R in L : count < hi }
template <typename CT>
__device__ void phase_refill_select(const PeelView<CT>& P) {
    PeelCtl* c = P.ctl;
    if (!need_refill(c)) return;
    const int32_t* L = pick(P.L, c->wl);
    int32_t* N = pick(P.N, c->wn);
    unsigned n = clampn(c->nL, P.cap);
    int64_t hi = c->hi;
    for (int64_t base = gthread() - (threadIdx.x & 31); base < n; base += nthreads()) {
        int64_t i = base + (threadIdx.x & 31);
        if (i < n) {
            int32_t R = L[i];
            if ((int64_t)P.cnt[R] < hi) nd_append(&c->nN, N, P.cap, R, &c->err);
        }
    }
}

// advance: k' = max(k, min over N); A = { R in N alive : count <= k' }; N' = the other alive
template <typename CT>
__device__ void phase_adv_select(const PeelView<CT>& P) {
    PeelCtl* c = P.ctl;
    if (c->done || !(c->mode & ND_MODE_ADV)) return;
    int64_t kn = knew_of(c);
    const int32_t* N = pick(P.N, c->wn);
    int32_t* N2 = pick(P.N, c->wn ^ 1);
    int32_t* A = pick(P.A, c->wa);
    unsigned n = clampn(c->nN, P.cap);
    int32_t t = c->t;
    for (int64_t base = gthread() - (threadIdx.x & 31); base < n; base += nthreads()) {
        int64_t i = base + (threadIdx.x & 31);
        if (i < n) {
            int32_t R = N[i];
            if (P.rnd[R] == ND_UNPEELED) {
                if ((int64_t)P.cnt[R] <= kn) {
                    if (P.bcnt) atomicSub(&P.bcnt[(int64_t)P.cnt[R]], 1u);
                    P.rnd[R] = t;
                    P.core[R] = (int32_t)kn;
                    if (P.et_rnd) set_tri_round(P, R, t);
                    mark_a(P, R);
                    nd_append(&c->cntA, A, P.cap, R, &c->err);
                } else {
                    nd_append(&c->nN2, N2, P.cap, R, &c->err);
                }
            }
        }
    }
}

// Graph contraction for (2,3) (Section 5.6): every adjacency row that lost at least
// len_prev >> contract_shift entries since the previous contraction (an entry is lost when its edge
// was peeled in an earlier round) is filtered in place, keeping the order of the other entries;
// one warp per vertex, 32 entries at a time, each kept entry written at (entries kept so far)
// <= its own position. Edges of the current round stay: the owner rule needs them. Runs at the
// start of a round, between barriers, so no Update reads the rows meanwhile.
template <typename CT>
__device__ void phase_contract(const GraphView& g, const PeelView<CT>& P) {
    PeelCtl* c = P.ctl;
    if (c->done || !c->contract) return;
    const int32_t t = c->t, shift = c->contract_shift;
    const int lane = threadIdx.x & 31;
    for (int64_t v = gwarp(); v < g.n; v += nwarps()) {
        const int64_t b = g.rp[v];
        const int32_t len = P.clen[v], prev = P.cprev[v];
        int32_t alive = 0;
        for (int32_t i = lane; i < len; i += 32) alive += P.rnd[P.cpos[b + i]] >= t;
        for (int o = 16; o > 0; o >>= 1) alive += __shfl_xor_sync(0xffffffffu, alive, o);
        // the row is compacted when it lost at least prev >> shift entries (shift 0: any entry)
        const int32_t lost = prev - alive;
        const int32_t need = shift ? (prev >> shift) : 1;
        if (alive == len || lost < need) continue;
        int32_t out = 0;
        for (int32_t i0 = 0; i0 < len; i0 += 32) {
            const int32_t i = i0 + lane;
            int32_t w = 0, e = 0;
            bool keep = false;
            if (i < len) {
                w = P.ccol[b + i];
                e = P.cpos[b + i];
                keep = P.rnd[e] >= t;
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int32_t at = out + __popc(m & nd_lanemask_lt());
                P.ccol[b + at] = w;
                P.cpos[b + at] = e;
            }
            out += __popc(m);
        }
        if (lane == 0) {
            P.clen[v] = out;
            P.cprev[v] = out;
        }
    }
}

template <typename CT>
__global__ void k_contract(GraphView g, PeelView<CT> P) { phase_contract(g, P); }

// The same for the (3,4) triangle lists L(e): an entry is lost when its triangle was peeled in an
// earlier round (its tag); a list that lost at least len_prev >> contract_shift entries since the
// previous contraction is filtered in place, one warp per edge, moving each kept entry's vertex,
// triangle id and tag together and recording its new offset in the triangle's entry table (the
// slot of the entry among its triangle's three lists follows from the vertex order: for the edge
// (a, c) and entry w, the triangle's edges are (xy, xz, yz) for x < y < z and e is xy when w > c, xz
// when a < w < c, yz when w < a). The hash tables keep every entry: a lookup of a removed entry
// finds its earlier tag, so the candidate is dropped as before.
template <typename CT>
__device__ void phase_contract34(const GraphView& g, const PeelView<CT>& P) {
    PeelCtl* c = P.ctl;
    if (c->done || !c->contract) return;
    const int32_t t = c->t, shift = c->contract_shift;
    const int lane = threadIdx.x & 31;
    for (int64_t e = gwarp(); e < g.m; e += nwarps()) {
        const int64_t b = g.et_rp[e];
        const int32_t len = P.llen[e], prev = P.lprev[e];
        int32_t alive = 0;
        for (int32_t i = lane; i < len; i += 32) alive += P.et_rnd[b + i] >= t;
        for (int o = 16; o > 0; o >>= 1) alive += __shfl_xor_sync(0xffffffffu, alive, o);
        const int32_t lost = prev - alive;
        const int32_t need = shift ? (prev >> shift) : 1;
        if (alive == len || lost < need) continue;
        const int32_t a = g.eu[e], cv = g.ev[e];
        int32_t out = 0;
        for (int32_t i0 = 0; i0 < len; i0 += 32) {
            const int32_t i = i0 + lane;
            int32_t w = 0, id = 0, r = 0;
            bool keep = false;
            if (i < len) {
                w = P.lw[b + i];
                id = P.lt[b + i];
                r = P.et_rnd[b + i];
                keep = r >= t;
            }
            const unsigned mk = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int32_t at = out + __popc(mk & nd_lanemask_lt());
                P.lw[b + at] = w;
                P.lt[b + at] = id;
                P.et_rnd[b + at] = r;
                const int x = w > cv ? 0 : (w > a ? 1 : 2);
                P.ltp[3 * (int64_t)id + x] = at;
            }
            out += __popc(mk);
        }
        if (lane == 0) {
            P.llen[e] = out;
            P.lprev[e] = out;
        }
    }
}

template <typename CT>
__global__ void k_contract34(GraphView g, PeelView<CT> P) { phase_contract34(g, P); }

template <typename CT>
__global__ void k_adv_min(PeelView<CT> P) { phase_adv_min(P); }
template <typename CT>
__global__ void k_refill_scan(PeelView<CT> P) { phase_refill_scan(P); }
template <typename CT>
__global__ void k_refill_hist(PeelView<CT> P) { phase_refill_hist(P); }
template <typename CT>
__global__ void k_refill_select(PeelView<CT> P) { phase_refill_select(P); }
template <typename CT>
__global__ void k_adv_select(PeelView<CT> P) { phase_adv_select(P); }

// Rebuild A in ascending id order from the membership bitmap (persistent kernel, large rounds):
// each block owns a fixed range of bitmap words; pass 1 counts its members, the serial step of the
// barrier turns the per-block counts (hist[0 .. gridDim)) into offsets, pass 2 writes the ids.
__device__ __forceinline__ void sort_range(const PeelCtl* c, int64_t& w0, int64_t& w1) {
    int64_t nwords = (c->n_r + 31) >> 5;
    int64_t per = (nwords + gridDim.x - 1) / gridDim.x;
    w0 = (int64_t)blockIdx.x * per;
    w1 = w0 + per < nwords ? w0 + per : nwords;
    if (w0 > w1) w0 = w1;
}

// exclusive prefix over the block (every thread calls it); returns the block total
__device__ unsigned block_excl_sum(unsigned v, unsigned& excl) {
    __shared__ unsigned s_warp[32];
    __shared__ unsigned s_total;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        unsigned x = lane < nw ? s_warp[lane] : 0, xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        if (lane < nw) s_warp[lane] = xi - x;
        if (lane == 31) s_total = xi;
    }
    __syncthreads();
    excl = s_warp[wid] + inc - v;
    unsigned total = s_total;
    __syncthreads();
    return total;
}

template <typename CT>
__device__ void phase_sort_count(const PeelView<CT>& P) {
    PeelCtl* c = P.ctl;
    int64_t w0, w1;
    sort_range(c, w0, w1);
    unsigned cnt = 0, excl;
    for (int64_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) cnt += __popc(P.abits[w]);
    unsigned total = block_excl_sum(cnt, excl);
    if (threadIdx.x == 0) c->hist[blockIdx.x] = total;
}

// Each warp writes the ids of its own slice of the block's words in order: its offset is the
// members of the blocks before (their counts, summed by the whole block) plus those of the warps
// before it in this block (recounted from the bitmap, which the count pass left in L2); inside the
// slice a warp scan places 32 words at a time, with no block-wide barrier per step.
template <typename CT>
__device__ void phase_sort_write(const PeelView<CT>& P) {
    PeelCtl* c = P.ctl;
    int64_t w0, w1;
    sort_range(c, w0, w1);
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t per = (w1 - w0 + nw - 1) / nw;
    int64_t a = w0 + wid * per, b = a + per < w1 ? a + per : w1;
    if (a > b) a = b;
    unsigned cnt = 0;
    for (int64_t w = a + lane; w < b; w += 32) cnt += __popc(P.abits[w]);
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(full, cnt, o);
    unsigned prior = 0;
    for (unsigned x = threadIdx.x; x < blockIdx.x; x += blockDim.x) prior += (unsigned)c->hist[x];
    unsigned excl;
    const unsigned blocks_before = block_excl_sum(prior, excl);
    block_excl_sum(lane == 0 ? cnt : 0u, excl);
    unsigned long long at = (unsigned long long)blocks_before + __shfl_sync(full, excl, 0);
    int32_t* A = pick(P.A, c->wa);
    for (int64_t base = a; base < b; base += 32) {
        const int64_t w = base + lane;
        uint32_t bits = w < b ? P.abits[w] : 0u;
        const unsigned pc = __popc(bits);
        unsigned inc = pc;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(full, inc, o);
            if (lane >= o) inc += y;
        }
        unsigned long long o = at + inc - pc;
        while (bits) {
            int bit = __ffs(bits) - 1;
            bits &= bits - 1;
            if (o < P.cap) A[o] = (int32_t)(w * 32 + bit);
            ++o;
        }
        at += __shfl_sync(full, inc, 31);
    }
}


// ------------------------------------------------------------------------------------
// Update

template <typename CT>
struct RoundEnv {
    PeelView<CT> P;
    int32_t t;
    int64_t k, hi;
    const int32_t* A;
    unsigned nA;
    int32_t* next;
    int32_t* Ncur;
    unsigned int* ncnt;
};

template <typename CT>
__device__ __forceinline__ RoundEnv<CT> round_env(const PeelView<CT>& P) {
    PeelCtl* c = P.ctl;
    RoundEnv<CT> E;
    E.P = P;
    bool adv = c->mode & ND_MODE_ADV;
    E.t = c->t;
    E.k = adv ? knew_of(c) : c->k;
    E.hi = c->hi;
    E.A = pick(P.A, c->wa);
    E.nA = clampn(adv ? c->cntA : c->nA, P.cap);
    E.next = pick(P.A, c->wa ^ 1);
    E.Ncur = adv ? pick(P.N, c->wn ^ 1) : pick(P.N, c->wn);
    E.ncnt = adv ? &c->nN2 : &c->nN;
    return E;
}

// per-thread statistics of one Update phase
struct UpdCounters {
    unsigned long long listed = 0;  // s-cliques destroyed (counted once, by the owner)
    unsigned long long decs = 0;    // count decrements applied
};

// What a decrement of r-clique x from o to o - 1 implies: x falls to <= k (it is the next
// round's A: its round, core number and index tags are written now) and/or below the bucket
// window (it joins N).
template <typename CT>
__device__ __forceinline__ void after_dec(const RoundEnv<CT>& E, int32_t x, int64_t o) {
    // dense buckets: a count above k + 1 moves down one bucket; at k + 1 the r-clique is scheduled
    // now and leaves the buckets; at or below k it was scheduled already
    if (E.P.bcnt && o > E.k) {
        atomicSub(&E.P.bcnt[o], 1u);
        if (o > E.k + 1) atomicAdd(&E.P.bcnt[o - 1], 1u);
    }
    if (o > E.k && o - 1 <= E.k) {
        E.P.rnd[x] = E.t + 1;
        E.P.core[x] = (int32_t)E.k;
        if (E.P.et_rnd) set_tri_round(E.P, x, E.t + 1);
        mark_a(E.P, x);
        nd_append(&E.P.ctl->nNext, E.next, E.P.cap, x, &E.P.ctl->err);
    }
    if (o >= E.hi && o - 1 < E.hi) nd_append(E.ncnt, E.Ncur, E.P.cap, x, &E.P.ctl->err);
}


// Whether a member of a destroyed S with round tag r has its count decremented on the device: not
// if it is in A (r = t), and not if it was already pushed into the next round's A during this
// round (r = t + 1): its core number is fixed and its count is never read again (every later
// reader of counts takes unpeeled r-cliques only). Both still count as decrements of Algorithm 2.
__device__ __forceinline__ bool dec_live(int32_t r, int32_t t) { return r != t && r != t + 1; }

// Update-Func for the s-clique S made of R and the other r-subsets o[0..M). Returns whether S
// was live (no r-subset peeled in an earlier round).
template <typename CT, int M>
__device__ __forceinline__ void update_func(const RoundEnv<CT>& E, int32_t R, const int32_t (&o)[M], UpdCounters& k) {
    int32_t ro[M];
    int32_t owner = R;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        ro[i] = E.P.rnd[o[i]];
        if (ro[i] < E.t) return;  // an r-subset was peeled in an earlier round
        if (ro[i] == E.t && o[i] < owner) owner = o[i];
    }
    if (owner != R) return;
    k.listed++;
    // issue every decrement before looking at any result (the atomics overlap in flight)
    int64_t old[M];
#pragma unroll
    for (int i = 0; i < M; ++i) old[i] = dec_live(ro[i], E.t) ? nd_atomic_dec(&E.P.cnt[o[i]]) : 0;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        k.decs += ro[i] != E.t;
        if (dec_live(ro[i], E.t)) after_dec(E, o[i], old[i]);
    }
}

__device__ __forceinline__ void add_counters(PeelCtl* c, UpdCounters k) {
    for (int o = 16; o > 0; o >>= 1) {
        k.listed += __shfl_down_sync(0xffffffffu, k.listed, o);
        k.decs += __shfl_down_sync(0xffffffffu, k.decs, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (k.listed) atomicAdd(&c->listed, k.listed);
        if (k.decs) atomicAdd(&c->decs, k.decs);
    }
}

// Each Update variant is a functor. (1,2), (1,3), (2,3), (3,4) have
//   prep(g, P, R, q): fills q with R's driving list (b[0], n[0]) -- its entries are the
//                     candidates -- and the lists they are searched in; returns n[0];
//   cand(g, E, R, q, j, k): lists the s-cliques of candidate j and applies Update-Func.
// (2,4) stages N(u) ∩ N(v) instead (run_warp / run_block, below).
struct Prep {
    int64_t b[3];
    int64_t n[3];
    int64_t h[3];  // (3,4): hash-table offset of the list, -1 when it is searched by bisection
    int32_t v[4];  // generic (r,s): the vertices of R
    const int32_t* lp;  // generic (r,s): the driving list
    int32_t hk[3];      // (3,4): log2 of the slots of each list's hash table (from its original length)
};

// The light Update phase gives each warp one R at a time: its lanes share the R's lists and read
// the driving list coalesced. R with more candidates than the variant's threshold go to a list
// that the heavy phase gives one block each, so a few hub r-cliques do not serialise on single
// warps.
constexpr int64_t kHeavy = 4096;

template <typename U, typename CT>
__device__ __forceinline__ void run_all(const GraphView& g, const RoundEnv<CT>& E, int32_t R, int64_t j0,
                                        int64_t dj, UpdCounters& k) {
    Prep q;
    int64_t n0 = U::prep(g, E.P, R, q);
    for (int64_t j = j0; j < n0; j += dj) U::cand(g, E, R, q, j, k);
}


// (1,2): R = v; S = {v, w} for every neighbour w.
template <typename CT>
struct Upd12 {
    __device__ static int64_t prep(const GraphView& g, const PeelView<CT>&, int32_t v, Prep& q) {
        q.b[0] = g.rp[v];
        q.n[0] = g.rp[v + 1] - q.b[0];
        return q.n[0];
    }
    template <typename Q>
    __device__ static void cand(const GraphView& g, const RoundEnv<CT>& E, int32_t v, const Q& q, int64_t j,
                                UpdCounters& k) {
        int32_t o[1] = {g.col[q.b[0] + j]};
        update_func<CT, 1>(E, v, o, k);
    }
};

// (1,3): R = v; S = {v, w, x} for every edge w -> x of DG inside N(v).
template <typename CT>
struct Upd13 {
    __device__ static int64_t prep(const GraphView& g, const PeelView<CT>&, int32_t v, Prep& q) {
        q.b[0] = g.rp[v];
        q.n[0] = g.rp[v + 1] - q.b[0];
        return q.n[0];
    }
    template <typename Q>
    __device__ static void cand(const GraphView& g, const RoundEnv<CT>& E, int32_t v, const Q& q, int64_t j,
                                UpdCounters& k) {
        int32_t w = g.col[q.b[0] + j];
        for (int64_t jx = g.dg_rp[w]; jx < g.dg_rp[w + 1]; ++jx) {
            int32_t x = g.dg_col[jx];
            if (nd_find(g.col + q.b[0], q.n[0], x) < 0) continue;
            int32_t o[2] = {w, x};
            update_func<CT, 2>(E, v, o, k);
        }
    }
};

// (2,3): R = (u,v); S = {u, v, w} for w in N(u) ∩ N(v); the shorter row drives.
// length of row v: the contracted length during a (2,3) peel with contraction, else the degree
__device__ __forceinline__ int64_t row_len(const GraphView& g, int32_t v) {
    return g.rlen ? (int64_t)g.rlen[v] : g.rp[v + 1] - g.rp[v];
}

template <typename CT>
struct Upd23 {
    static constexpr int64_t kHeavyWork = 256;  // a block, not a warp, for rows longer than this
    __device__ static int64_t work(const GraphView& g, int32_t R) {
        int32_t u = g.eu[R], v = g.ev[R];
        int64_t du = row_len(g, u), dv = row_len(g, v);
        return du < dv ? du : dv;
    }
    __device__ static int64_t prep(const GraphView& g, const PeelView<CT>&, int32_t R, Prep& q) {
        int32_t u = g.eu[R], v = g.ev[R];
        int64_t ub = g.rp[u], un = row_len(g, u), vb = g.rp[v], vn = row_len(g, v);
        bool u_drives = un <= vn;
        q.b[0] = u_drives ? ub : vb;
        q.n[0] = u_drives ? un : vn;
        q.b[1] = u_drives ? vb : ub;
        q.n[1] = u_drives ? vn : un;
        return q.n[0];
    }
    template <typename Q>
    __device__ static void cand(const GraphView& g, const RoundEnv<CT>& E, int32_t R, const Q& q, int64_t j,
                                UpdCounters& k) {
        // the edge to the candidate, peeled in an earlier round: every S through it is dead
        int64_t p = q.b[0] + j;
        int32_t e_xw = g.pos2e[p];
        if (E.P.rnd[e_xw] < E.t) return;
        int64_t r = nd_find(g.col + q.b[1], q.n[1], g.col[p]);
        if (r < 0) return;
        int32_t o[2] = {e_xw, g.pos2e[q.b[1] + r]};
        update_func<CT, 2>(E, R, o, k);
    }
};

// (2,4): R = (u,v); S = {u, v, w, x} for w in N(u) ∩ N(v) and x in N_DG(w) ∩ N(u) ∩ N(v).
// (2,4) works on I = N(u) ∩ N(v) staged with its edge ids (to u and to v) and the out-lists of
// its vertices; every DG edge w -> x with w, x in I is a 4-clique S = {u, v, w, x}. The candidate
// pairs (w, x in N_DG(w)) are expanded flat over the threads through a prefix sum of the
// out-degrees, and x is looked up in the staged I, so no thread walks a long list serially.
// An edge whose smaller endpoint degree is at most kI24 is staged in one warp's shared memory;
// larger ones go to the heavy phase, where one block stages I in a global scratch slice.
constexpr int kI24 = 96;
constexpr int kMaxWarpsPerBlock = 16;

struct Stage24 {
    int32_t* w;     // I, ascending
    int32_t* ex;    // edge id (driver endpoint, w)
    int32_t* ey;    // edge id (other endpoint, w)
    int32_t* base;  // DG out-list start of w (fits int32: at most m < 2^31)
    int32_t* pre;   // exclusive prefix of the out-degrees, pre[cnt] = total
};

__device__ __forceinline__ int stage_find(const int32_t* a, int n, int32_t x) {
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

// index i with pre[i] <= p < pre[i+1]
__device__ __forceinline__ int stage_owner(const int32_t* pre, int n, int32_t p) {
    int lo = 0, hi = n;  // invariant: pre[lo] <= p
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (pre[mid] <= p)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

template <typename CT>
struct Upd24 {
    static constexpr int64_t kHeavyWork = kI24;
    static constexpr bool kStaged = true;
    __device__ static int64_t work(const GraphView& g, int32_t R) { return Upd23<CT>::work(g, R); }

    // the 4-cliques of candidate pair number p (0 <= p < pre[cnt]) of the staged I
    __device__ static void pair(const GraphView& g, const RoundEnv<CT>& E, int32_t R, const Stage24& st, int cnt,
                                int32_t p, UpdCounters& k) {
        int i = stage_owner(st.pre, cnt, p);
        int64_t jx = (int64_t)st.base[i] + (p - st.pre[i]);
        int j = stage_find(st.w, cnt, g.dg_col[jx]);
        if (j < 0) return;
        int32_t o[5] = {st.ex[i], st.ey[i], st.ex[j], st.ey[j], g.dg_eid[jx]};
        update_func<CT, 5>(E, R, o, k);
    }

    // One warp; the stage is this warp's shared memory (capacity kI24).
    __device__ static void run_warp(const GraphView& g, const RoundEnv<CT>& E, int32_t R, UpdCounters& k,
                                    const Stage24& st) {
        int lane = threadIdx.x & 31;
        int32_t u = g.eu[R], v = g.ev[R];
        int64_t ub = g.rp[u], un = g.rp[u + 1] - ub, vb = g.rp[v], vn = g.rp[v + 1] - vb;
        bool u_drives = un <= vn;
        int64_t xb = u_drives ? ub : vb, xn = u_drives ? un : vn;
        int64_t yb = u_drives ? vb : ub, yn = u_drives ? vn : un;
        int cnt = 0;
        for (int64_t p0 = 0; p0 < xn; p0 += 32) {
            int64_t p = p0 + lane;
            int64_t q = -1;
            // w joins I only with both edges to R unpeeled before this round: every S through an
            // edge peeled earlier is dead already
            if (p < xn && E.P.rnd[g.pos2e[xb + p]] >= E.t) {
                q = nd_find(g.col + yb, yn, g.col[xb + p]);
                if (q >= 0 && E.P.rnd[g.pos2e[yb + q]] < E.t) q = -1;
            }
            unsigned m = __ballot_sync(0xffffffffu, q >= 0);
            if (q >= 0) {
                int at = cnt + __popc(m & nd_lanemask_lt());
                int32_t w = g.col[xb + p];
                st.w[at] = w;
                st.ex[at] = g.pos2e[xb + p];
                st.ey[at] = g.pos2e[yb + q];
                st.base[at] = (int32_t)g.dg_rp[w];
                st.pre[at] = (int32_t)(g.dg_rp[w + 1] - g.dg_rp[w]);
            }
            cnt += __popc(m);
        }
        __syncwarp();
        // exclusive prefix of the out-degrees (cnt <= kI24 < 128: at most four 32-wide chunks)
        int32_t carry = 0;
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            int i = c0 + lane;
            int32_t d = i < cnt ? st.pre[i] : 0, inc = d;
            for (int o = 1; o < 32; o <<= 1) {
                int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (i < cnt) st.pre[i] = carry + inc - d;
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) st.pre[cnt] = carry;
        __syncwarp();
        for (int32_t p = lane; p < carry; p += 32) pair(g, E, R, st, cnt, p, k);
        __syncwarp();
    }

    // One block stages I of edge R in its global scratch slice and turns the out-degrees into the
    // exclusive prefix of the candidate pairs; returns the number of pairs (the same in every
    // thread) and sets cnt_out to |I|. Every thread of the block calls it.
    __device__ static int32_t stage_block(const GraphView& g, const RoundEnv<CT>& E, int32_t R, const Stage24& st,
                                          int& cnt_out) {
        __shared__ int32_t s_tot[kMaxWarpsPerBlock];
        __shared__ int32_t s_cnt, s_carry;
        int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        int32_t u = g.eu[R], v = g.ev[R];
        int64_t ub = g.rp[u], un = g.rp[u + 1] - ub, vb = g.rp[v], vn = g.rp[v + 1] - vb;
        bool u_drives = un <= vn;
        int64_t xb = u_drives ? ub : vb, xn = u_drives ? un : vn;
        int64_t yb = u_drives ? vb : ub, yn = u_drives ? vn : un;
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        // stage I in ascending order: block-wide ordered compaction, blockDim elements at a time
        for (int64_t p0 = 0; p0 < xn; p0 += blockDim.x) {
            int64_t p = p0 + threadIdx.x;
            int64_t q = -1;
            if (p < xn && E.P.rnd[g.pos2e[xb + p]] >= E.t) {
                q = nd_find(g.col + yb, yn, g.col[xb + p]);
                if (q >= 0 && E.P.rnd[g.pos2e[yb + q]] < E.t) q = -1;
            }
            unsigned m = __ballot_sync(0xffffffffu, q >= 0);
            if (lane == 0) s_tot[wid] = __popc(m);
            __syncthreads();
            int before = 0, tot = 0;
            for (int x = 0; x < nw; ++x) {
                before += x < wid ? s_tot[x] : 0;
                tot += s_tot[x];
            }
            if (q >= 0) {
                int at = s_cnt + before + __popc(m & nd_lanemask_lt());
                int32_t w = g.col[xb + p];
                st.w[at] = w;
                st.ex[at] = g.pos2e[xb + p];
                st.ey[at] = g.pos2e[yb + q];
                st.base[at] = (int32_t)g.dg_rp[w];
                st.pre[at] = (int32_t)(g.dg_rp[w + 1] - g.dg_rp[w]);
            }
            __syncthreads();
            if (threadIdx.x == 0) s_cnt += tot;
            __syncthreads();
        }
        int cnt = s_cnt;
        // exclusive prefix of the out-degrees (one warp; the totals fit int32: at most m)
        if (wid == 0) {
            int32_t carry = 0;
            for (int c0 = 0; c0 < cnt; c0 += 32) {
                int i = c0 + lane;
                int32_t d = i < cnt ? st.pre[i] : 0, inc = d;
                for (int o = 1; o < 32; o <<= 1) {
                    int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                if (i < cnt) st.pre[i] = carry + inc - d;
                carry += __shfl_sync(0xffffffffu, inc, 31);
            }
            if (lane == 0) {
                st.pre[cnt] = carry;
                s_carry = carry;
            }
        }
        __syncthreads();
        int32_t total = s_carry;
        cnt_out = cnt;
        __syncthreads();
        return total;
    }

    // One block (the heavy phase); the stage is the block's global scratch slice. Every thread of
    // the block calls it.
    __device__ static void run_block(const GraphView& g, const RoundEnv<CT>& E, int32_t R, UpdCounters& k,
                                     const Stage24& st) {
        int cnt = 0;
        int32_t total = stage_block(g, E, R, st, cnt);
        for (int32_t p = threadIdx.x; p < total; p += blockDim.x) pair(g, E, R, st, cnt, p, k);
        __syncthreads();
    }
};

// (3,4): R = triangle (a,b,c) with edges ab, ac, bc; S = R + w for w in L(ab) ∩ L(ac) ∩ L(bc);
// the three other triangles of S are the table entries of w in the three lists. Every entry
// carries the round tag of its triangle (et_rnd, written when the triangle is scheduled): a
// tag below the current round means that triangle was peeled earlier, so every S through it is
// dead and the candidate is dropped before any further search; a tag equal to the round marks a
// member of A for the owner rule. No per-triangle state is read at random.
template <typename CT>
__device__ __forceinline__ void lists34(const GraphView& g, const PeelView<CT>& P, int32_t R, Prep& q) {
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        int32_t e = g.tri_e[3 * (int64_t)R + x];
        q.b[x] = g.et_rp[e];
        const int64_t n0 = g.et_rp[e + 1] - q.b[x];  // original length: it sizes the hash table
        q.n[x] = g.llen ? (int64_t)g.llen[e] : n0;   // current length (after list contraction)
        q.h[x] = P.htab && nd_hashed(n0) ? P.hoff[e] : -1;
        q.hk[x] = q.h[x] >= 0 ? nd_hash_bits(n0) : 0;
    }
    // sort the three lists by current length
#pragma unroll
    for (int pass = 0; pass < 3; ++pass) {
        int i = pass == 2 ? 1 : 0, j = pass == 0 ? 1 : 2;  // compare-exchange (0,1), (0,2), (1,2)
        if (q.n[j] < q.n[i]) {
            int64_t tb = q.b[i], tn = q.n[i], th = q.h[i];
            int32_t tk = q.hk[i];
            q.b[i] = q.b[j], q.n[i] = q.n[j], q.h[i] = q.h[j], q.hk[i] = q.hk[j];
            q.b[j] = tb, q.n[j] = tn, q.h[j] = th, q.hk[j] = tk;
        }
    }
}

template <typename CT>
struct Upd34 {
    __device__ static int64_t prep(const GraphView& g, const PeelView<CT>& P, int32_t R, Prep& q) {
        lists34(g, P, R, q);
        return q.n[0];
    }
    // the triangle R + w of list x (w's entry in L(e_x)) and its round; false when w is not there
    template <typename Q>
    __device__ static bool look(const GraphView& g, const RoundEnv<CT>& E, const Q& q, int x, int32_t w,
                                int32_t& id, int32_t& r) {
        if (q.h[x] >= 0) {
            if (!nd_hash_find(E.P.htab + q.h[x], q.hk[x], w, id, r)) return false;
        } else {
            int64_t i = nd_find(g.et_w + q.b[x], q.n[x], w);
            if (i < 0) return false;
            r = E.P.et_rnd[q.b[x] + i];
            id = g.et_t[q.b[x] + i];
        }
        return true;
    }
    // S = R + w, w = entry j of list 0. Only the owner (smallest id of S's members in A) applies
    // S, so R stops as soon as a member in A with a smaller id is known: first the entry's own
    // triangle (read along the list), then the ones found in lists 1 and 2.
    template <typename Q>
    __device__ static void cand(const GraphView& g, const RoundEnv<CT>& E, int32_t R, const Q& q, int64_t j,
                                UpdCounters& k) {
        int32_t r0 = E.P.et_rnd[q.b[0] + j];
        if (r0 < E.t) return;
        int32_t id0 = g.et_t[q.b[0] + j];
        if (r0 == E.t && id0 < R) return;
        int32_t w = g.et_w[q.b[0] + j], id1, r1, id2, r2;
        if (!look(g, E, q, 1, w, id1, r1) || r1 < E.t || (r1 == E.t && id1 < R)) return;
        if (!look(g, E, q, 2, w, id2, r2) || r2 < E.t || (r2 == E.t && id2 < R)) return;
        k.listed++;
        // issue the decrements before looking at any result (the atomics overlap in flight)
        int64_t o0 = dec_live(r0, E.t) ? nd_atomic_dec(&E.P.cnt[id0]) : 0;
        int64_t o1 = dec_live(r1, E.t) ? nd_atomic_dec(&E.P.cnt[id1]) : 0;
        int64_t o2 = dec_live(r2, E.t) ? nd_atomic_dec(&E.P.cnt[id2]) : 0;
        k.decs += (r0 != E.t) + (r1 != E.t) + (r2 != E.t);
        if (dec_live(r0, E.t)) after_dec(E, id0, o0);
        if (dec_live(r1, E.t)) after_dec(E, id1, o1);
        if (dec_live(r2, E.t)) after_dec(E, id2, o2);
    }

    // Light Update over a group of at most 32 triangles of A, with a queue of candidates per warp.
    // Lane l sets up triangle l of the group (its three lists, in parallel with the other lanes,
    // instead of one dependent setup chain per triangle). The warp then reads the driving lists of
    // the group's triangles one after another, coalesced, and drops the dead entries (triangle
    // peeled in an earlier round, or a member of A with a smaller id than R) with one read each; the
    // surviving candidates of any triangle of the group go to a shared-memory queue as (w, id, slot
    // and state of the list-0 triangle). Whenever 32 kIlp are queued, every lane probes lists 1 and 2
    // for kIlp of them and applies the decrements, so the probes and atomics run on full warps
    // whatever mix of short and long lists the group has. A triangle whose lists 1
    // and 2 are not both hashed is listed the per-candidate way after the queue is drained.
    static constexpr bool kQueued = true;
    static constexpr int kIlp = 1;                // queued candidates per lane and drain
    static constexpr int kQueue = 32 * kIlp + 32;  // < 32 kIlp entries before an append of at most 32
    __device__ static void run_group(const GraphView& g, const RoundEnv<CT>& E, const int32_t* Ag, int nG,
                                     int64_t heavy, UpdCounters& k, int32_t* qw, int32_t* qi, int32_t* qm) {
        const unsigned full = 0xffffffffu;
        const int lane = threadIdx.x & 31;
        int32_t R = -1;
        int64_t b0 = 0, h1 = 0, h2 = 0, n0 = 0;
        int32_t hk = 0;
        bool paired = false;
        if (lane < nG) {
            R = Ag[lane];
            unmark_a(E.P, R);
            Prep q;
            lists34(g, E.P, R, q);
            n0 = q.n[0];
            b0 = q.b[0];
            h1 = q.h[1];
            h2 = q.h[2];
            hk = q.hk[1] | (q.hk[2] << 8);
            paired = h1 >= 0 && h2 >= 0;
            if (n0 > heavy) {
                unsigned slot = atomicAdd(&E.P.ctl->nH, 1u);
                if (slot < E.P.hcap) {
                    E.P.H[slot] = R;
                    n0 = 0;  // the heavy phase lists it
                }
            }
        }
        int qn = 0;
        unsigned todo = __ballot_sync(full, paired && n0 > 0);
        while (todo) {
            const int sl = __ffs(todo) - 1;
            todo &= todo - 1;
            const int32_t Rs = __shfl_sync(full, R, sl);
            const int64_t bs = __shfl_sync(full, b0, sl), ns = __shfl_sync(full, n0, sl);
            // entries of the next 32-wide chunk are loaded before the current one is filtered
            int64_t j = lane;
            int32_t r0 = -1, i0 = 0, w0 = 0;
            if (j < ns) {
                r0 = E.P.et_rnd[bs + j];
                i0 = g.et_t[bs + j];
                w0 = g.et_w[bs + j];
            }
            for (int64_t off = 0; off < ns; off += 32) {
                const int64_t jn = off + 32 + lane;
                int32_t r1 = -1, i1 = 0, w1 = 0;
                if (jn < ns) {
                    r1 = E.P.et_rnd[bs + jn];
                    i1 = g.et_t[bs + jn];
                    w1 = g.et_w[bs + jn];
                }
                const bool keep = r0 >= E.t && !(r0 == E.t && i0 < Rs);
                const unsigned m = __ballot_sync(full, keep);
                if (keep) {
                    const int at = qn + __popc(m & nd_lanemask_lt());
                    qw[at] = w0;
                    qi[at] = i0;
                    qm[at] = sl | (r0 == E.t ? 32 : 0) | (dec_live(r0, E.t) ? 64 : 0);
                }
                qn += __popc(m);
                if (qn >= 32 * kIlp) {
                    __syncwarp();
                    const int d = qn - 32 * kIlp;
                    drain(E, R, h1, h2, hk, qw + d, qi + d, qm + d, 32 * kIlp, k);
                    qn = d;
                    __syncwarp();
                }
                r0 = r1, i0 = i1, w0 = w1;
            }
        }
        if (qn > 0) {
            __syncwarp();
            drain(E, R, h1, h2, hk, qw, qi, qm, qn, k);
            __syncwarp();
        }
        // triangles with a list that is not hashed: one at a time, per candidate
        unsigned rest = __ballot_sync(full, !paired && n0 > 0);
        while (rest) {
            const int sl = __ffs(rest) - 1;
            rest &= rest - 1;
            const int32_t Rs = __shfl_sync(full, R, sl);
            Prep q;
            lists34(g, E.P, Rs, q);
            for (int64_t jj = lane; jj < q.n[0]; jj += 32) cand(g, E, Rs, q, jj, k);
        }
    }

    // Probes and decrements of nq <= 32 kIlp queued candidates: lane l takes entries l, l + 32, ...
    // (kIlp chains in flight per lane: every load of a step is issued before any result is used).
    // The group's per-triangle state (R, hash offsets and sizes of lists 1 and 2) is read from the
    // lane that set the triangle up.
    __device__ static void drain(const RoundEnv<CT>& E, int32_t R, int64_t h1, int64_t h2, int32_t hk,
                                 const int32_t* qw, const int32_t* qi, const int32_t* qm, int nq, UpdCounters& k) {
        constexpr int N = kIlp;
        const unsigned full = 0xffffffffu;
        const int lane = threadIdx.x & 31;
        bool live[N];
        int32_t w[N], id0[N], me[N], Rx[N], k1[N], k2[N], i1[N], r1[N], i2[N], r2[N];
        const NdHashSlot* t1[N];
        const NdHashSlot* t2[N];
        uint32_t s1[N], s2[N];
        int4 p1[N], p2[N];
#pragma unroll
        for (int x = 0; x < N; ++x) {
            const int e = lane + 32 * x;
            live[x] = e < nq;
            w[x] = live[x] ? qw[e] : 0;
            id0[x] = live[x] ? qi[e] : 0;
            me[x] = live[x] ? qm[e] : 0;
            const int sl = me[x] & 31;
            Rx[x] = __shfl_sync(full, R, sl);
            t1[x] = E.P.htab + __shfl_sync(full, h1, sl);
            t2[x] = E.P.htab + __shfl_sync(full, h2, sl);
            const int32_t kk = __shfl_sync(full, hk, sl);
            k1[x] = kk & 255;
            k2[x] = kk >> 8;
            s1[x] = nd_hash_slot(w[x], k1[x]);
            s2[x] = nd_hash_slot(w[x], k2[x]);
        }
#pragma unroll
        for (int x = 0; x < N; ++x) {
            p1[x] = make_int4(-1, 0, 0, 0);
            p2[x] = p1[x];
            if (live[x]) {
                p1[x] = *reinterpret_cast<const int4*>(t1[x] + s1[x]);
                p2[x] = *reinterpret_cast<const int4*>(t2[x] + s2[x]);
            }
        }
        int64_t o0[N], o1[N], o2[N];
#pragma unroll
        for (int x = 0; x < N; ++x) {
            i1[x] = r1[x] = i2[x] = r2[x] = 0;
            live[x] = live[x] && nd_hash_resolve(t1[x], k1[x], w[x], s1[x], p1[x], i1[x], r1[x]) &&
                      nd_hash_resolve(t2[x], k2[x], w[x], s2[x], p2[x], i2[x], r2[x]);
            live[x] = live[x] && r1[x] >= E.t && !(r1[x] == E.t && i1[x] < Rx[x]) && r2[x] >= E.t &&
                      !(r2[x] == E.t && i2[x] < Rx[x]);
        }
        // the decrements of every 4-clique go out before any result is looked at
#pragma unroll
        for (int x = 0; x < N; ++x) {
            o0[x] = live[x] && (me[x] & 64) ? nd_atomic_dec(&E.P.cnt[id0[x]]) : 0;
            o1[x] = live[x] && dec_live(r1[x], E.t) ? nd_atomic_dec(&E.P.cnt[i1[x]]) : 0;
            o2[x] = live[x] && dec_live(r2[x], E.t) ? nd_atomic_dec(&E.P.cnt[i2[x]]) : 0;
        }
#pragma unroll
        for (int x = 0; x < N; ++x) {
            if (!live[x]) continue;
            k.listed++;
            k.decs += !(me[x] & 32) + (r1[x] != E.t) + (r2[x] != E.t);
            if (me[x] & 64) after_dec(E, id0[x], o0[x]);
            if (dec_live(r1[x], E.t)) after_dec(E, i1[x], o1[x]);
            if (dec_live(r2[x], E.t)) after_dec(E, i2[x], o2[x]);
        }
    }
};

// Any other (r,s) with r <= 4 and s - r <= 3 ((1,4), (2,5), (3,5), (3,6), (4,5), (4,6)): the candidates are
// the entries of R's driving list; each lists the (s-r)-cliques of R's common neighbourhood that
// start at it (nd_gen.cuh), looks up the ids of the other r-subsets of every S = R + C and applies
// Update-Func. A lookup that fails means an inconsistent index (ctl->err bit 16).
template <typename CT, int R_, int S_>
struct UpdGen {
    static constexpr int M = gen_binom(S_, R_) - 1;
    __device__ static int64_t prep(const GraphView& g, const PeelView<CT>&, int32_t R, Prep& q) {
        gen_verts<R_>(g, R, q.v);
        int64_t len = 0;
        gen_drive<R_>(g, R, q.v, q.lp, len);
        q.n[0] = len;
        return len;
    }
    template <typename Q>
    __device__ static void cand(const GraphView& g, const RoundEnv<CT>& E, int32_t R, const Q& q, int64_t j,
                                UpdCounters& k) {
        gen_cand<R_, S_>(g, q.v, q.lp[j], [&](const int32_t* C) {
            int32_t Sv[S_], o[M];
            gen_merge<R_, S_>(q.v, C, Sv);
            if (!gen_others<R_, S_>(g, q.v, Sv, o)) {
                atomicOr(&E.P.ctl->err, 16);
                return;
            }
            update_func<CT, M>(E, R, o, k);
        });
    }
};

template <typename U, typename = void>
struct is_staged {
    static constexpr bool value = false;
};
template <typename U>
struct is_staged<U, decltype((void)U::kStaged)> {
    static constexpr bool value = U::kStaged;
};


template <typename U, typename = void>
struct is_queued {
    static constexpr bool value = false;
};
template <typename U>
struct is_queued<U, decltype((void)U::kQueued)> {
    static constexpr bool value = U::kQueued;
};

template <typename U, typename = void>
struct heavy_work {
    static constexpr int64_t value = kHeavy;
};
template <typename U>
struct heavy_work<U, decltype((void)U::kHeavyWork)> {
    static constexpr int64_t value = U::kHeavyWork;
};

// Update hands out A to warps in chunks taken from a counter that the round's control step resets:
// a warp that finishes early takes more, so the round ends when the work ends rather than when the
// unluckiest warp of a static assignment does. A chunk holds about nA / (16 warps) r-cliques (at
// least 1), so a round costs about 16 counter updates per warp however large A is.
__device__ __forceinline__ unsigned update_chunk(unsigned nA) {
    unsigned long long w = (unsigned long long)nwarps() * 16ull;
    unsigned long long c = nA / w;
    return c ? (unsigned)c : 1u;
}

__device__ __forceinline__ unsigned take_chunk(PeelCtl* c, unsigned chunk) {
    unsigned i0 = 0;
    if ((threadIdx.x & 31) == 0) i0 = atomicAdd(&c->upd_next, chunk);
    return __shfl_sync(0xffffffffu, i0, 0);
}

// the heavy-phase threshold of this decomposition: a tuned value if given (capped by what a warp's
// stage holds for staged variants), else the variant's own
template <typename U, typename CT>
__device__ __forceinline__ int64_t heavy_limit(const PeelView<CT>& P) {
    int64_t h = P.heavy_work > 0 ? P.heavy_work : heavy_work<U>::value;
    if (is_staged<U>::value && h > heavy_work<U>::value) h = heavy_work<U>::value;
    return h;
}

template <typename CT, typename U>
__device__ void phase_update(const GraphView& g, const PeelView<CT>& P) {
    if (P.ctl->done) return;
    RoundEnv<CT> E = round_env(P);
    const unsigned full = 0xffffffffu;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    UpdCounters k;
    if constexpr (is_staged<U>::value) {
        // one warp per r-clique, I staged in the warp's shared memory
        __shared__ int32_t s_w[kMaxWarpsPerBlock][kI24], s_x[kMaxWarpsPerBlock][kI24],
            s_y[kMaxWarpsPerBlock][kI24], s_b[kMaxWarpsPerBlock][kI24], s_p[kMaxWarpsPerBlock][kI24 + 1];
        const unsigned chunk = update_chunk(E.nA);
        for (unsigned i0 = take_chunk(P.ctl, chunk); i0 < E.nA; i0 = take_chunk(P.ctl, chunk))
        for (unsigned i = i0; i < i0 + chunk && i < E.nA; ++i) {
            int32_t R = E.A[i];
            if (lane == 0) unmark_a(P, R);
            if (U::work(g, R) > heavy_limit<U>(P)) {
                int queued = 0;
                if (lane == 0) {
                    unsigned slot = atomicAdd(&P.ctl->nH, 1u);
                    if (slot < P.hcap) {
                        P.H[slot] = R;
                        queued = 1;
                    }
                }
                if (__shfl_sync(full, queued, 0)) continue;
                // the staged warp path holds at most kI24 entries; the list is sized to hold every
                // r-clique for staged functors, so this is unreachable
                if (lane == 0) atomicOr(&P.ctl->err, 1);
                continue;
            }
            Stage24 stg{s_w[wid], s_x[wid], s_y[wid], s_b[wid], s_p[wid]};
            U::run_warp(g, E, R, k, stg);
        }
    } else if constexpr (is_queued<U>::value) {
        // groups of up to 32 r-cliques per warp with a queue of live candidates (Upd34::run_group);
        // chunks of at most 32, about nA / (4 warps) each, so that small rounds still spread
        __shared__ int32_t s_qw[kMaxWarpsPerBlock][U::kQueue], s_qi[kMaxWarpsPerBlock][U::kQueue],
            s_qm[kMaxWarpsPerBlock][U::kQueue];
        unsigned long long per = (unsigned long long)nwarps() * 4ull;
        unsigned chunk = (unsigned)(E.nA / per);
        chunk = chunk < 1u ? 1u : (chunk > 32u ? 32u : chunk);
        const int64_t heavy = heavy_limit<U>(P);
        for (unsigned i0 = take_chunk(P.ctl, chunk); i0 < E.nA; i0 = take_chunk(P.ctl, chunk)) {
            int nG = (int)(E.nA - i0 < chunk ? E.nA - i0 : chunk);
            U::run_group(g, E, E.A + i0, nG, heavy, k, s_qw[wid], s_qi[wid], s_qm[wid]);
        }
    } else {
        // one warp per r-clique: its lanes read the driving list coalesced
        const unsigned chunk = update_chunk(E.nA);
        for (unsigned i0 = take_chunk(P.ctl, chunk); i0 < E.nA; i0 = take_chunk(P.ctl, chunk))
        for (unsigned i = i0; i < i0 + chunk && i < E.nA; ++i) {
            int32_t R = E.A[i];
            if (lane == 0) unmark_a(P, R);
            Prep q;
            int64_t n0 = U::prep(g, P, R, q);
            if (n0 > heavy_limit<U>(P)) {
                int queued = 0;
                if (lane == 0) {
                    unsigned slot = atomicAdd(&P.ctl->nH, 1u);
                    if (slot < P.hcap) {
                        P.H[slot] = R;
                        queued = 1;
                    }
                }
                if (__shfl_sync(full, queued, 0)) continue;
            }
            for (int64_t j = lane; j < n0; j += 32) U::cand(g, E, R, q, j, k);
        }
    }
    add_counters(P.ctl, k);
}

template <typename CT, typename U>
__device__ void phase_update_heavy(const GraphView& g, const PeelView<CT>& P) {
    if (P.ctl->done) return;
    unsigned nH = clampn(P.ctl->nH, P.hcap);
    if (nH == 0) return;
    RoundEnv<CT> E = round_env(P);
    UpdCounters k;
    // one block per heavy r-clique, its threads striding the driving list: heavy r-cliques run
    // side by side, each over many threads
    if constexpr (is_staged<U>::value) {
        // blocks below hslices own a scratch slice of 5 * (hstage + 1) int32 and share the list
        unsigned ns = (unsigned)P.hslices < gridDim.x ? (unsigned)P.hslices : gridDim.x;
        if (blockIdx.x < ns) {
            int64_t c = P.hstage + 1;
            int32_t* base = P.hscratch + (int64_t)blockIdx.x * 5 * c;
            Stage24 stg{base, base + c, base + 2 * c, base + 3 * c, base + 4 * c};
            for (unsigned h = blockIdx.x; h < nH; h += ns) U::run_block(g, E, P.H[h], k, stg);
        }
    } else {
        for (unsigned h = blockIdx.x; h < nH; h += gridDim.x) run_all<U>(g, E, P.H[h], threadIdx.x, blockDim.x, k);
    }
    add_counters(P.ctl, k);
}

// (2,4) heavy phase split over the grid (persistent kernel, when the round's heavy edges fit the
// scratch slices): first every heavy edge is staged by one block into its own slice (I, its edge
// ids and out-list bounds, the prefix of the candidate pairs); then, after a barrier whose serial
// step turns the per-edge pair totals into offsets, every thread of the grid takes candidate pairs
// of any heavy edge. A round whose few heavy edges used to occupy a few blocks spreads them over
// all of them.
template <typename CT, typename U>
__device__ void phase_heavy_stage(const GraphView& g, const PeelView<CT>& P) {
    if (P.ctl->done) return;
    unsigned nH = clampn(P.ctl->nH, P.hcap);
    RoundEnv<CT> E = round_env(P);
    const int64_t c = P.hstage + 1;
    for (unsigned b = blockIdx.x; b < nH; b += gridDim.x) {
        int32_t* base = P.hscratch + (int64_t)b * 5 * c;
        Stage24 stg{base, base + c, base + 2 * c, base + 3 * c, base + 4 * c};
        int cnt = 0;
        int32_t total = U::stage_block(g, E, P.H[b], stg, cnt);
        if (threadIdx.x == 0) {
            P.hcnt[b] = cnt;
            P.hpre[b] = total;
        }
    }
}

template <typename CT, typename U>
__device__ void phase_heavy_pairs(const GraphView& g, const PeelView<CT>& P) {
    if (P.ctl->done) return;
    unsigned nH = clampn(P.ctl->nH, P.hcap);
    RoundEnv<CT> E = round_env(P);
    UpdCounters k;
    const int64_t c = P.hstage + 1, T = P.hpre[nH];
    for (int64_t p = gthread(); p < T; p += nthreads()) {
        unsigned lo = 0, hi = nH;  // the last edge whose offset is <= p
        while (hi - lo > 1) {
            unsigned mid = (lo + hi) >> 1;
            if (P.hpre[mid] <= p)
                lo = mid;
            else
                hi = mid;
        }
        int32_t* base = P.hscratch + (int64_t)lo * 5 * c;
        Stage24 stg{base, base + c, base + 2 * c, base + 3 * c, base + 4 * c};
        U::pair(g, E, P.H[lo], stg, P.hcnt[lo], (int32_t)(p - P.hpre[lo]), k);
    }
    add_counters(P.ctl, k);
}

template <typename CT, typename U>
__global__ void k_update(GraphView g, PeelView<CT> P) { phase_update<CT, U>(g, P); }
template <typename CT, typename U>
__global__ void k_update_heavy(GraphView g, PeelView<CT> P) { phase_update_heavy<CT, U>(g, P); }

// ------------------------------------------------------------------------------------
// The whole peeling loop in one cooperative launch (every block resident at once), with a grid
// barrier between phases. The barrier's arrive is a release and its poll an acquire at GPU
// scope, so every write before the barrier is visible to every load after it. Its wait is
// bounded by the global timer: after kBarrierTimeoutNs, or once another block has given up, a
// block sets ctl->err bit 8 and returns, so an inconsistent state ends the kernel instead of
// hanging it.
constexpr unsigned long long kBarrierTimeoutNs = 60ull * 1000 * 1000 * 1000;

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_acquire_i32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}


__device__ __forceinline__ unsigned long long atom_add_acq_rel_u64(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid barrier. The block that arrives last runs serial() in its thread 0 (it sees every write
// made before the barrier) and then releases the others, so a control step costs no extra
// barrier. Arrival is an acquire-release RMW and the release a release store; waiting blocks poll
// with an acquire load, so all writes before the barrier are visible after it. The wait is
// bounded by the global timer: after ctl->bar_timeout_ns (kBarrierTimeoutNs by default), or once
// another block gave up, a block sets ctl->err bit 8 and the function returns false.
template <typename F>
__device__ bool grid_barrier(PeelCtl* c, unsigned long long& target, F serial) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        unsigned long long old = atom_add_acq_rel_u64(&c->bar_arrive, 1ull);
        int good = 1;
        if (old + 1 == target) {
            serial();
            st_release_u64(&c->bar_gen, target);
        } else {
            unsigned long long t0 = globaltimer();
            const unsigned long long limit = c->bar_timeout_ns;
            while (ld_acquire_u64(&c->bar_gen) < target) {
                if ((ld_acquire_i32(&c->err) & 8) || globaltimer() - t0 > limit) {
                    atomicOr(&c->err, 8);
                    good = 0;
                    break;
                }
                __nanosleep(20);
            }
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

struct NoSerial {
    __device__ void operator()() const {}
};

// whether the round about to run its Update sorts A first (decided only in serial steps, so every
// block reads the same value after the barrier)
template <typename CT>
__device__ __forceinline__ void decide_sort(PeelCtl* c, const PeelView<CT>* P) {
    unsigned nA = (c->mode & ND_MODE_ADV) ? c->cntA : c->nA;
    c->sorta = P->abits && !c->done && nA >= P->sort_min && nA <= P->cap;
}

template <typename CT>
struct CtlSerial {
    PeelCtl* c;
    const PeelView<CT>* P;
    __device__ void operator()() const {
        ctl_step(c, P->round_size, P->round_level, P->round_cap);
        decide_sort(c, P);  // same-level rounds; advance rounds decide after selecting A
    }
};

template <typename CT>
struct SortDecide {
    PeelCtl* c;
    const PeelView<CT>* P;
    __device__ void operator()() const { decide_sort(c, P); }
};

// after the light Update: finish the round now unless heavy r-cliques are waiting
template <typename CT>
struct CtlUnlessHeavy {
    PeelCtl* c;
    const PeelView<CT>* P;
    __device__ void operator()() const {
        // the blocks branch on `heavy`, which only serial steps write: nH itself may already be
        // growing in the next round's update by the time a slow block looks
        c->heavy = c->nH != 0;
        c->heavy_split = c->heavy && P->hpre && c->nH <= (unsigned)P->hslices;
        if (!c->heavy) {
            ctl_step(c, P->round_size, P->round_level, P->round_cap);
            decide_sort(c, P);
        }
    }
};

struct PickSerial {
    PeelCtl* c;
    __device__ void operator()() const { refill_pick_serial(c); }
};

// (2,4) heavy phase split over the grid: the pair totals of the staged heavy edges become offsets
template <typename CT>
struct HeavyScan {
    PeelCtl* c;
    const PeelView<CT>* P;
    __device__ void operator()() const {
        unsigned nH = c->nH;
        long long run = 0;
        for (unsigned b = 0; b < nH; ++b) {
            long long v = P->hpre[b];
            P->hpre[b] = run;
            run += v;
        }
        P->hpre[nH] = run;
    }
};

// One round: [advance: min over N; (refill: compact + min, histogram, pick, select); select A]
// Update (light, one warp per r-clique), then the heavy r-cliques if any. The control step runs
// as the serial part of the round's last barrier; a same-level round costs one barrier.
template <typename CT, typename U, bool k34>
__global__ void __launch_bounds__(512, 2) k_peel_loop(GraphView g, PeelView<CT> P) {
    PeelCtl* c = P.ctl;
    unsigned long long target = 0;
    bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    int32_t tr = 0;  // the round being run
    // block 0 books the time since the previous barrier to the phase that just ended (and the
    // Update phases also to the round)
    auto book = [&](int ph) {
        if (timer) {
            unsigned long long now = globaltimer(), d = now - c->ph_last;
            c->ph_ns[ph] += d;
            c->ph_last = now;
            if ((ph == 4 || ph == 5) && P.round_ns && tr < P.round_cap) P.round_ns[tr] += (int64_t)d;
        }
    };
    // test of the barrier bound (ND_LIMIT_DROP_BLOCK): one block never arrives, so the others give
    // up after bar_timeout_ns and the call reports ND_ETIMEOUT
    if (c->drop_block && blockIdx.x == gridDim.x - 1) return;
    if (!grid_barrier(c, target, CtlSerial<CT>{c, &P})) return;  // set up round 0
    if (timer) c->ph_last = globaltimer();
    for (;;) {
        if (c->done) return;  // every block reads the same value after the barrier
        tr = c->t;
        if (c->contract) {  // written only by serial steps
            if constexpr (k34)
                phase_contract34(g, P);
            else
                phase_contract(g, P);
            if (!grid_barrier(c, target, NoSerial{})) return;
            book(6);
        }
        if (c->mode & ND_MODE_ADV) {
            phase_adv_min(P);
            if (!grid_barrier(c, target, NoSerial{})) return;
            book(0);
            if (need_refill(c)) {
                phase_refill_scan(P);
                if (!grid_barrier(c, target, NoSerial{})) return;
                phase_refill_hist(P);
                if (!grid_barrier(c, target, PickSerial{c})) return;
                phase_refill_select(P);
                if (!grid_barrier(c, target, NoSerial{})) return;
                book(1);
            }
            phase_adv_select(P);
            if (!grid_barrier(c, target, SortDecide<CT>{c, &P})) return;
            book(2);
        }
        if (c->sorta) {
            phase_sort_count(P);
            if (!grid_barrier(c, target, NoSerial{})) return;
            phase_sort_write(P);
            if (!grid_barrier(c, target, NoSerial{})) return;
            book(3);
        }
        phase_update<CT, U>(g, P);
        if (!grid_barrier(c, target, CtlUnlessHeavy<CT>{c, &P})) return;
        book(4);
        if (c->heavy) {
            if constexpr (is_staged<U>::value) {
                if (c->heavy_split) {  // written only by serial steps
                    phase_heavy_stage<CT, U>(g, P);
                    if (!grid_barrier(c, target, HeavyScan<CT>{c, &P})) return;
                    phase_heavy_pairs<CT, U>(g, P);
                    if (!grid_barrier(c, target, CtlSerial<CT>{c, &P})) return;
                    book(5);
                    continue;
                }
            }
            phase_update_heavy<CT, U>(g, P);
            if (!grid_barrier(c, target, CtlSerial<CT>{c, &P})) return;
            book(5);
        }
    }
}

template <typename CT, typename U, bool k34>
cudaError_t launch_peel_loop(const GraphView& g, const PeelView<CT>& P, cudaStream_t st) {
    auto kern = k_peel_loop<CT, U, k34>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    int blocks = nd_sm_count() * (per_sm < 2 ? per_sm : 2);
    GraphView gv = g;
    PeelView<CT> pv = P;
    void* args[] = {&gv, &pv};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(512), args, 0, st);
    if (e == cudaSuccess) nd_note_launches(1);
    return e;
}

int peel_blocks() { return nd_sm_count() * 4; }

}  // namespace

int nd_peel_heavy_slices() { return nd_sm_count() * 2; }

void nd_peel_init(PeelCtl* ctl, int64_t n_r, int64_t max_rounds, cudaStream_t st, uint64_t barrier_ns,
                  int drop_block, int64_t contract_every, int contract_shift) {
    ND_K(k_init<<<1, 32, 0, st>>>(ctl, n_r, max_rounds, barrier_ns ? barrier_ns : kBarrierTimeoutNs, drop_block,
                                  contract_every, contract_shift));
}

template <typename CT>
void nd_peel_contract(const GraphView& g, const PeelView<CT>& P, cudaStream_t st) {
    if (P.ccol) ND_K(k_contract<CT><<<peel_blocks(), kThreads, 0, st>>>(g, P));
    if (P.lw) ND_K(k_contract34<CT><<<peel_blocks(), kThreads, 0, st>>>(g, P));
}

template <typename CT>
void nd_peel_ctl(const PeelView<CT>& P, cudaStream_t st, int use_cond, cudaGraphConditionalHandle h_loop,
                 cudaGraphConditionalHandle h_adv) {
    ND_K(k_ctl<<<1, 32, 0, st>>>(P.ctl, P.round_size, P.round_level, P.round_cap, use_cond, h_loop, h_adv));
}

template <typename CT>
void nd_peel_adv_min(const PeelView<CT>& P, cudaStream_t st) {
    ND_K(k_adv_min<CT><<<peel_blocks(), kThreads, 0, st>>>(P));
}

void nd_peel_set_refill(PeelCtl* ctl, cudaStream_t st, cudaGraphConditionalHandle h_refill) {
    ND_K(k_set_refill<<<1, 32, 0, st>>>(ctl, h_refill));
}

template <typename CT>
void nd_peel_refill(const PeelView<CT>& P, cudaStream_t st) {
    int nb = peel_blocks();
    ND_K(k_refill_scan<CT><<<nb, kThreads, 0, st>>>(P));
    ND_K(k_refill_hist<CT><<<nb, kThreads, 0, st>>>(P));
    ND_K(k_refill_pick<<<1, 1024, 0, st>>>(P.ctl));
    ND_K(k_refill_select<CT><<<nb, kThreads, 0, st>>>(P));
}

template <typename CT>
void nd_peel_adv_select(const PeelView<CT>& P, cudaStream_t st) {
    ND_K(k_adv_select<CT><<<peel_blocks(), kThreads, 0, st>>>(P));
}

template <typename CT>
void nd_peel_update(const GraphView& g, int r, int s, const PeelView<CT>& P, cudaStream_t st) {
    int nb = peel_blocks();
    if (r == 1 && s == 2) {
        ND_K(k_update<CT, Upd12<CT>><<<nb, kThreads, 0, st>>>(g, P));
        ND_K(k_update_heavy<CT, Upd12<CT>><<<nb, kThreads, 0, st>>>(g, P));
    } else if (r == 1 && s == 3) {
        ND_K(k_update<CT, Upd13<CT>><<<nb, kThreads, 0, st>>>(g, P));
        ND_K(k_update_heavy<CT, Upd13<CT>><<<nb, kThreads, 0, st>>>(g, P));
    } else if (r == 2 && s == 3) {
        ND_K(k_update<CT, Upd23<CT>><<<nb, kThreads, 0, st>>>(g, P));
        ND_K(k_update_heavy<CT, Upd23<CT>><<<nb, kThreads, 0, st>>>(g, P));
    } else if (r == 2 && s == 4) {
        ND_K(k_update<CT, Upd24<CT>><<<nb, kThreads, 0, st>>>(g, P));
        ND_K(k_update_heavy<CT, Upd24<CT>><<<nb, kThreads, 0, st>>>(g, P));
    } else if (r == 3 && s == 4) {
        ND_K(k_update<CT, Upd34<CT>><<<nb, kThreads, 0, st>>>(g, P));
        ND_K(k_update_heavy<CT, Upd34<CT>><<<nb, kThreads, 0, st>>>(g, P));
    } else if (r == 1 && s == 4) {
        ND_K(k_update<CT, UpdGen<CT, 1, 4>><<<nb, kThreads, 0, st>>>(g, P));
        ND_K(k_update_heavy<CT, UpdGen<CT, 1, 4>><<<nb, kThreads, 0, st>>>(g, P));
    } else if (r == 2 && s == 5) {
        ND_K(k_update<CT, UpdGen<CT, 2, 5>><<<nb, kThreads, 0, st>>>(g, P));
        ND_K(k_update_heavy<CT, UpdGen<CT, 2, 5>><<<nb, kThreads, 0, st>>>(g, P));
    } else if (r == 3 && s == 5) {
        ND_K(k_update<CT, UpdGen<CT, 3, 5>><<<nb, kThreads, 0, st>>>(g, P));
        ND_K(k_update_heavy<CT, UpdGen<CT, 3, 5>><<<nb, kThreads, 0, st>>>(g, P));
    } else if (r == 3 && s == 6) {
        ND_K(k_update<CT, UpdGen<CT, 3, 6>><<<nb, kThreads, 0, st>>>(g, P));
        ND_K(k_update_heavy<CT, UpdGen<CT, 3, 6>><<<nb, kThreads, 0, st>>>(g, P));
    } else if (r == 4 && s == 5) {
        ND_K(k_update<CT, UpdGen<CT, 4, 5>><<<nb, kThreads, 0, st>>>(g, P));
        ND_K(k_update_heavy<CT, UpdGen<CT, 4, 5>><<<nb, kThreads, 0, st>>>(g, P));
    } else if (r == 4 && s == 6) {
        ND_K(k_update<CT, UpdGen<CT, 4, 6>><<<nb, kThreads, 0, st>>>(g, P));
        ND_K(k_update_heavy<CT, UpdGen<CT, 4, 6>><<<nb, kThreads, 0, st>>>(g, P));
    }
}

// One round as a plain launch sequence (every phase launched; inactive ones return at once).
template <typename CT>
void nd_peel_round(const GraphView& g, int r, int s, const PeelView<CT>& P, cudaStream_t st) {
    nd_peel_ctl<CT>(P, st, 0, 0, 0);
    nd_peel_contract<CT>(g, P, st);
    nd_peel_adv_min<CT>(P, st);
    nd_peel_refill<CT>(P, st);
    nd_peel_adv_select<CT>(P, st);
    nd_peel_update<CT>(g, r, s, P, st);
}

// Adds a conditional node of the given type after the current capture point of st and returns
// its body graph; the capture continues after the node.
static cudaError_t capture_conditional(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                       cudaGraph_t* body) {
    cudaStreamCaptureStatus status;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(st, &status, nullptr, &graph, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return e;
    if (status != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &p);
    if (e != cudaSuccess) return e;
    *body = p.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// The whole peeling loop as one CUDA graph:
//   WHILE (not done) { k_ctl; IF (advance) { k_adv_min; k_set_refill; IF (refill) { refill x4 };
//                      k_adv_select }; Update kernels }
// st, st2, st3 are three distinct streams used only for capture. On failure nothing is left
// capturing and *out is NULL.
template <typename CT>
cudaError_t nd_peel_loop_graph(const GraphView& g, int r, int s, const PeelView<CT>& P, cudaStream_t st,
                               cudaStream_t st2, cudaStream_t st3, cudaGraph_t* out) {
    *out = nullptr;
    cudaGraph_t graph = nullptr, body = nullptr, adv_body = nullptr, ref_body = nullptr, tmp = nullptr;
    cudaGraphConditionalHandle h_loop, h_adv, h_refill;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    auto fail = [&](cudaError_t err) {
        cudaStreamCaptureStatus cs;
        for (cudaStream_t x : {st3, st2, st}) {
            if (cudaStreamIsCapturing(x, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                cudaGraph_t junk = nullptr;
                cudaStreamEndCapture(x, &junk);
            }
        }
        nd_set_capturing(false);
        cudaGraphDestroy(graph);
        cudaGetLastError();
        return err;
    };
    if ((e = cudaGraphConditionalHandleCreate(&h_loop, graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess ||
        (e = cudaGraphConditionalHandleCreate(&h_adv, graph, 0, cudaGraphCondAssignDefault)) != cudaSuccess ||
        (e = cudaGraphConditionalHandleCreate(&h_refill, graph, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
        return fail(e);
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if ((e = cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &wp)) != cudaSuccess) return fail(e);
    body = wp.conditional.phGraph_out[0];
    nd_set_capturing(true);
    if ((e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return fail(e);
    nd_peel_ctl<CT>(P, st, 1, h_loop, h_adv);
    nd_peel_contract<CT>(g, P, st);
    if ((e = capture_conditional(st, h_adv, cudaGraphCondTypeIf, &adv_body)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamBeginCaptureToGraph(st2, adv_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return fail(e);
    nd_peel_adv_min<CT>(P, st2);
    nd_peel_set_refill(P.ctl, st2, h_refill);
    if ((e = capture_conditional(st2, h_refill, cudaGraphCondTypeIf, &ref_body)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamBeginCaptureToGraph(st3, ref_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return fail(e);
    nd_peel_refill<CT>(P, st3);
    if ((e = cudaStreamEndCapture(st3, &tmp)) != cudaSuccess) return fail(e);
    nd_peel_adv_select<CT>(P, st2);
    if ((e = cudaStreamEndCapture(st2, &tmp)) != cudaSuccess) return fail(e);
    nd_peel_update<CT>(g, r, s, P, st);
    if ((e = cudaStreamEndCapture(st, &tmp)) != cudaSuccess) return fail(e);
    nd_set_capturing(false);
    *out = graph;
    return cudaSuccess;
}

// The whole loop as one cooperative kernel (see k_peel_loop). Fails without side effects if a
// cooperative launch is not possible.
template <typename CT>
cudaError_t nd_peel_persistent(const GraphView& g, int r, int s, const PeelView<CT>& P, cudaStream_t st) {
    if (r == 1 && s == 2) return launch_peel_loop<CT, Upd12<CT>, false>(g, P, st);
    if (r == 1 && s == 3) return launch_peel_loop<CT, Upd13<CT>, false>(g, P, st);
    if (r == 2 && s == 3) return launch_peel_loop<CT, Upd23<CT>, false>(g, P, st);
    if (r == 2 && s == 4) return launch_peel_loop<CT, Upd24<CT>, false>(g, P, st);
    if (r == 3 && s == 4) return launch_peel_loop<CT, Upd34<CT>, true>(g, P, st);
    if (r == 1 && s == 4) return launch_peel_loop<CT, UpdGen<CT, 1, 4>, false>(g, P, st);
    if (r == 2 && s == 5) return launch_peel_loop<CT, UpdGen<CT, 2, 5>, false>(g, P, st);
    if (r == 3 && s == 5) return launch_peel_loop<CT, UpdGen<CT, 3, 5>, false>(g, P, st);
    if (r == 3 && s == 6) return launch_peel_loop<CT, UpdGen<CT, 3, 6>, false>(g, P, st);
    if (r == 4 && s == 5) return launch_peel_loop<CT, UpdGen<CT, 4, 5>, false>(g, P, st);
    if (r == 4 && s == 6) return launch_peel_loop<CT, UpdGen<CT, 4, 6>, false>(g, P, st);
    return cudaErrorInvalidValue;
}

// kernels launched per round by the loop graph (for the launch counter): the nodes executed in
// a same-level round and the extra ones of an advance round
int nd_peel_nodes_per_round(int r, int s, bool contract) { return contract ? 4 : 3; }

template void nd_peel_round<int32_t>(const GraphView&, int, int, const PeelView<int32_t>&, cudaStream_t);
template void nd_peel_round<int64_t>(const GraphView&, int, int, const PeelView<int64_t>&, cudaStream_t);
template cudaError_t nd_peel_persistent<int32_t>(const GraphView&, int, int, const PeelView<int32_t>&, cudaStream_t);
template cudaError_t nd_peel_persistent<int64_t>(const GraphView&, int, int, const PeelView<int64_t>&, cudaStream_t);
template cudaError_t nd_peel_loop_graph<int32_t>(const GraphView&, int, int, const PeelView<int32_t>&, cudaStream_t,
                                                 cudaStream_t, cudaStream_t, cudaGraph_t*);
template cudaError_t nd_peel_loop_graph<int64_t>(const GraphView&, int, int, const PeelView<int64_t>&, cudaStream_t,
                                                 cudaStream_t, cudaStream_t, cudaGraph_t*);

// ------------------------------------------------------------------------------------
// dense buckets: initial occupancy (a shared-memory histogram of the low buckets per block, global
// atomics above it)

namespace {
constexpr int kBinShared = 8192;

template <typename CT>
__global__ void k_bucket_fill(const CT* __restrict__ cnt, int64_t n_r, unsigned int* __restrict__ bcnt, int64_t bmax) {
    __shared__ unsigned int h[kBinShared];
    const int64_t nb = bmax < kBinShared ? bmax : kBinShared;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t R = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; R < n_r; R += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = (int64_t)cnt[R];
        if (v < nb)
            atomicAdd(&h[v], 1u);
        else if (v < bmax)
            atomicAdd(&bcnt[v], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (h[i]) atomicAdd(&bcnt[i], h[i]);
}
}  // namespace

template <typename CT>
void nd_bucket_fill(const CT* cnt, int64_t n_r, unsigned int* bcnt, int64_t bmax, cudaStream_t st) {
    if (n_r <= 0) return;
    int64_t want = (n_r + 255) / 256, cap = (int64_t)nd_sm_count() * 4;
    ND_K(k_bucket_fill<CT><<<(int)(want < cap ? want : cap), 256, 0, st>>>(cnt, n_r, bcnt, bmax));
}

template void nd_bucket_fill<int32_t>(const int32_t*, int64_t, unsigned int*, int64_t, cudaStream_t);
template void nd_bucket_fill<int64_t>(const int64_t*, int64_t, unsigned int*, int64_t, cudaStream_t);
