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
#include "nd_common.cuh"

#include <climits>

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

__global__ void k_init(PeelCtl* c, int64_t n_r, int64_t max_rounds) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c->t = 0;
        c->mode = 0;
        c->done = 0;
        c->err = 0;
        c->started = 0;
        c->wa = c->wn = c->wl = 0;
        c->lmat = 0;
        c->k = 0;
        c->hi = 0;
        c->finished = 0;
        c->n_r = n_r;
        c->max_rounds = max_rounds;
        c->nA = c->cntA = c->nNext = c->nN = c->nN2 = c->nL = c->nL2 = 0;
        c->minN = c->gmin = ULLONG_MAX;
        c->listed = 0;
        c->advances = c->refills = 0;
    }
}

// Finishes round t-1 and sets up round t (one thread).
__global__ void k_ctl(PeelCtl* c, int64_t* round_size, int64_t* round_level, int64_t round_cap) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
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

template <typename CT>
__global__ void k_adv_min(PeelView<CT> P) {
    PeelCtl* c = P.ctl;
    if (c->done || !(c->mode & ND_MODE_ADV)) return;
    const int32_t* N = P.N[c->wn];
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
__global__ void k_refill_scan(PeelView<CT> P) {
    PeelCtl* c = P.ctl;
    if (!need_refill(c)) return;
    for (int64_t i = gthread(); i < ND_HBINS; i += nthreads()) c->hist[i] = 0;
    const int32_t* L = P.L[c->wl];
    int32_t* L2 = P.L[c->wl ^ 1];
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
__global__ void k_refill_hist(PeelView<CT> P) {
    PeelCtl* c = P.ctl;
    if (!need_refill(c)) return;
    __shared__ unsigned int h[ND_HBINS];
    for (int i = threadIdx.x; i < ND_HBINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int32_t* L2 = P.L[c->wl ^ 1];
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

// refill 3/4 (one block of 1024): choose hi, swap L <- L', clear N
__global__ void k_refill_pick(PeelCtl* c) {
    if (!need_refill(c)) return;
    __shared__ unsigned long long part[1024];
    __shared__ int best;
    constexpr int per = ND_HBINS / 1024;
    unsigned long long s = 0;
    for (int j = 0; j < per; ++j) s += c->hist[threadIdx.x * per + j];
    part[threadIdx.x] = s;
    if (threadIdx.x == 0) best = ND_HBINS - 1;
    __syncthreads();
    // inclusive scan of part (Hillis-Steele; 1024 entries)
    for (int o = 1; o < 1024; o <<= 1) {
        unsigned long long y = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += y;
        __syncthreads();
    }
    unsigned long long alive = c->nL2;
    unsigned long long target = alive / 16;
    if (target < 16384) target = 16384;
    unsigned long long before = threadIdx.x ? part[threadIdx.x - 1] : 0;
    unsigned long long run = before;
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
}

// refill 4/4: N = { R in L : count < hi }
template <typename CT>
__global__ void k_refill_select(PeelView<CT> P) {
    PeelCtl* c = P.ctl;
    if (!need_refill(c)) return;
    const int32_t* L = P.L[c->wl];
    int32_t* N = P.N[c->wn];
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
__global__ void k_adv_select(PeelView<CT> P) {
    PeelCtl* c = P.ctl;
    if (c->done || !(c->mode & ND_MODE_ADV)) return;
    int64_t kn = knew_of(c);
    const int32_t* N = P.N[c->wn];
    int32_t* N2 = P.N[c->wn ^ 1];
    int32_t* A = P.A[c->wa];
    unsigned n = clampn(c->nN, P.cap);
    int32_t t = c->t;
    for (int64_t base = gthread() - (threadIdx.x & 31); base < n; base += nthreads()) {
        int64_t i = base + (threadIdx.x & 31);
        if (i < n) {
            int32_t R = N[i];
            if (P.rnd[R] == ND_UNPEELED) {
                if ((int64_t)P.cnt[R] <= kn) {
                    P.rnd[R] = t;
                    P.core[R] = (int32_t)kn;
                    nd_append(&c->cntA, A, P.cap, R, &c->err);
                } else {
                    nd_append(&c->nN2, N2, P.cap, R, &c->err);
                }
            }
        }
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
    E.A = P.A[c->wa];
    E.nA = clampn(adv ? c->cntA : c->nA, P.cap);
    E.next = P.A[c->wa ^ 1];
    E.Ncur = adv ? P.N[c->wn ^ 1] : P.N[c->wn];
    E.ncnt = adv ? &c->nN2 : &c->nN;
    return E;
}

template <typename CT>
__device__ __forceinline__ void dec_one(const RoundEnv<CT>& E, int32_t x) {
    int64_t o = nd_atomic_dec(&E.P.cnt[x]);
    if (o > E.k && o - 1 <= E.k) {
        E.P.rnd[x] = E.t + 1;
        E.P.core[x] = (int32_t)E.k;
        nd_append(&E.P.ctl->nNext, E.next, E.P.cap, x, &E.P.ctl->err);
    }
    if (o >= E.hi && o - 1 < E.hi) nd_append(E.ncnt, E.Ncur, E.P.cap, x, &E.P.ctl->err);
}

// Update-Func for the s-clique S made of R and the other r-subsets o[0..M).
template <typename CT, int M>
__device__ __forceinline__ void update_func(const RoundEnv<CT>& E, int32_t R, const int32_t (&o)[M]) {
    int32_t ro[M];
    int32_t owner = R;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        ro[i] = E.P.rnd[o[i]];
        if (ro[i] < E.t) return;  // an r-subset was peeled in an earlier round
        if (ro[i] == E.t && o[i] < owner) owner = o[i];
    }
    if (owner != R) return;
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (ro[i] != E.t) dec_one(E, o[i]);
}

__device__ __forceinline__ void add_listed(PeelCtl* c, unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&c->listed, v);
}

// (1,2): R = v; S = {v, w} for every neighbour w.
template <typename CT>
__global__ void k_update12(GraphView g, PeelView<CT> P) {
    if (P.ctl->done) return;
    RoundEnv<CT> E = round_env(P);
    int lane = threadIdx.x & 31;
    unsigned long long listed = 0;
    for (int64_t i = gwarp(); i < E.nA; i += nwarps()) {
        int32_t v = E.A[i];
        int64_t b = g.rp[v], e = g.rp[v + 1];
        for (int64_t p = b + lane; p < e; p += 32) {
            int32_t o[1] = {g.col[p]};
            listed++;
            update_func<CT, 1>(E, v, o);
        }
    }
    add_listed(P.ctl, listed);
}

// (1,3): R = v; S = {v, w, x} for every edge w -> x of DG inside N(v).
template <typename CT>
__global__ void k_update13(GraphView g, PeelView<CT> P) {
    if (P.ctl->done) return;
    RoundEnv<CT> E = round_env(P);
    int lane = threadIdx.x & 31;
    unsigned long long listed = 0;
    for (int64_t i = gwarp(); i < E.nA; i += nwarps()) {
        int32_t v = E.A[i];
        int64_t b = g.rp[v], e = g.rp[v + 1];
        for (int64_t p = b + lane; p < e; p += 32) {
            int32_t w = g.col[p];
            for (int64_t jx = g.dg_rp[w]; jx < g.dg_rp[w + 1]; ++jx) {
                int32_t x = g.dg_col[jx];
                if (nd_find(g.col + b, e - b, x) < 0) continue;
                int32_t o[2] = {w, x};
                listed++;
                update_func<CT, 2>(E, v, o);
            }
        }
    }
    add_listed(P.ctl, listed);
}

// (2,3): R = (u,v); S = {u, v, w} for w in N(u) ∩ N(v).
template <typename CT>
__global__ void k_update23(GraphView g, PeelView<CT> P) {
    if (P.ctl->done) return;
    RoundEnv<CT> E = round_env(P);
    int lane = threadIdx.x & 31;
    unsigned long long listed = 0;
    for (int64_t i = gwarp(); i < E.nA; i += nwarps()) {
        int32_t R = E.A[i];
        int32_t u = g.eu[R], v = g.ev[R];
        int64_t xb = g.rp[u], xe = g.rp[u + 1], yb = g.rp[v], ye = g.rp[v + 1];
        if (xe - xb > ye - yb) {
            int64_t t0 = xb, t1 = xe;
            xb = yb, xe = ye, yb = t0, ye = t1;
        }
        for (int64_t p = xb + lane; p < xe; p += 32) {
            int32_t w = g.col[p];
            int64_t q = nd_find(g.col + yb, ye - yb, w);
            if (q < 0) continue;
            int32_t o[2] = {g.pos2e[p], g.pos2e[yb + q]};
            listed++;
            update_func<CT, 2>(E, R, o);
        }
    }
    add_listed(P.ctl, listed);
}

// (2,4): R = (u,v); S = {u, v, w, x} for w in N(u) ∩ N(v) and x in N_DG(w) ∩ N(u) ∩ N(v).
template <typename CT>
__global__ void k_update24(GraphView g, PeelView<CT> P) {
    if (P.ctl->done) return;
    RoundEnv<CT> E = round_env(P);
    int lane = threadIdx.x & 31;
    unsigned long long listed = 0;
    for (int64_t i = gwarp(); i < E.nA; i += nwarps()) {
        int32_t R = E.A[i];
        int32_t u = g.eu[R], v = g.ev[R];
        int64_t ub = g.rp[u], un = g.rp[u + 1] - ub, vb = g.rp[v], vn = g.rp[v + 1] - vb;
        bool u_drives = un <= vn;
        int64_t xb = u_drives ? ub : vb, xn = u_drives ? un : vn;
        int64_t yb = u_drives ? vb : ub, yn = u_drives ? vn : un;
        for (int64_t p = lane; p < xn; p += 32) {
            int32_t w = g.col[xb + p];
            int64_t q = nd_find(g.col + yb, yn, w);
            if (q < 0) continue;
            int32_t e_xw = g.pos2e[xb + p], e_yw = g.pos2e[yb + q];
            for (int64_t jx = g.dg_rp[w]; jx < g.dg_rp[w + 1]; ++jx) {
                int32_t x = g.dg_col[jx];
                int64_t px = nd_find(g.col + xb, xn, x);
                if (px < 0) continue;
                int64_t py = nd_find(g.col + yb, yn, x);
                if (py < 0) continue;
                int32_t o[5] = {e_xw, e_yw, g.pos2e[xb + px], g.pos2e[yb + py], g.dg_eid[jx]};
                listed++;
                update_func<CT, 5>(E, R, o);
            }
        }
    }
    add_listed(P.ctl, listed);
}

// (3,4): R = triangle (a,b,c) with edges ab, ac, bc; S = R + w for w in L(ab) ∩ L(ac) ∩ L(bc);
// the three other triangles of S are read from the same table entries.
template <typename CT>
__global__ void k_update34(GraphView g, PeelView<CT> P) {
    if (P.ctl->done) return;
    RoundEnv<CT> E = round_env(P);
    int lane = threadIdx.x & 31;
    unsigned long long listed = 0;
    for (int64_t i = gwarp(); i < E.nA; i += nwarps()) {
        int32_t R = E.A[i];
        int32_t e0 = g.tri_e[3 * (int64_t)R], e1 = g.tri_e[3 * (int64_t)R + 1], e2 = g.tri_e[3 * (int64_t)R + 2];
        int64_t b0 = g.et_rp[e0], n0 = g.et_rp[e0 + 1] - b0;
        int64_t b1 = g.et_rp[e1], n1 = g.et_rp[e1 + 1] - b1;
        int64_t b2 = g.et_rp[e2], n2 = g.et_rp[e2 + 1] - b2;
        if (n1 < n0) {
            int64_t tb = b0, tn = n0;
            b0 = b1, n0 = n1, b1 = tb, n1 = tn;
        }
        if (n2 < n0) {
            int64_t tb = b0, tn = n0;
            b0 = b2, n0 = n2, b2 = tb, n2 = tn;
        }
        for (int64_t j = lane; j < n0; j += 32) {
            int32_t w = g.et_w[b0 + j];
            int64_t q1 = nd_find(g.et_w + b1, n1, w);
            if (q1 < 0) continue;
            int64_t q2 = nd_find(g.et_w + b2, n2, w);
            if (q2 < 0) continue;
            int32_t o[3] = {g.et_t[b0 + j], g.et_t[b1 + q1], g.et_t[b2 + q2]};
            listed++;
            update_func<CT, 3>(E, R, o);
        }
    }
    add_listed(P.ctl, listed);
}

int peel_blocks() { return nd_sm_count() * 4; }

}  // namespace

void nd_peel_init(PeelCtl* ctl, int64_t n_r, int64_t max_rounds, cudaStream_t st) {
    ND_K(k_init<<<1, 32, 0, st>>>(ctl, n_r, max_rounds));
}

template <typename CT>
void nd_peel_round(const GraphView& g, int r, int s, const PeelView<CT>& P, cudaStream_t st) {
    int nb = peel_blocks();
    ND_K(k_ctl<<<1, 32, 0, st>>>(P.ctl, P.round_size, P.round_level, P.round_cap));
    ND_K(k_adv_min<CT><<<nb, kThreads, 0, st>>>(P));
    ND_K(k_refill_scan<CT><<<nb, kThreads, 0, st>>>(P));
    ND_K(k_refill_hist<CT><<<nb, kThreads, 0, st>>>(P));
    ND_K(k_refill_pick<<<1, 1024, 0, st>>>(P.ctl));
    ND_K(k_refill_select<CT><<<nb, kThreads, 0, st>>>(P));
    ND_K(k_adv_select<CT><<<nb, kThreads, 0, st>>>(P));
    if (r == 1 && s == 2)
        ND_K(k_update12<CT><<<nb, kThreads, 0, st>>>(g, P));
    else if (r == 1 && s == 3)
        ND_K(k_update13<CT><<<nb, kThreads, 0, st>>>(g, P));
    else if (r == 2 && s == 3)
        ND_K(k_update23<CT><<<nb, kThreads, 0, st>>>(g, P));
    else if (r == 2 && s == 4)
        ND_K(k_update24<CT><<<nb, kThreads, 0, st>>>(g, P));
    else if (r == 3 && s == 4)
        ND_K(k_update34<CT><<<nb, kThreads, 0, st>>>(g, P));
}

template void nd_peel_round<int32_t>(const GraphView&, int, int, const PeelView<int32_t>&, cudaStream_t);
template void nd_peel_round<int64_t>(const GraphView&, int, int, const PeelView<int64_t>&, cudaStream_t);
