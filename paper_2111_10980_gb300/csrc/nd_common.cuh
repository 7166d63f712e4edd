// Internal declarations shared by the CUDA translation units of libnd.so.
//
// Data layout in HBM (all arrays are plain device buffers owned by an nd_graph):
//   undirected CSR       rp int64[n+1], col int32[2m]          (caller's ids, rows ascending)
//   canonical edge index split int64[n]   first row position with col > row
//                        ebase int64[n+1]  exclusive scan of upper degrees
//                        pos2e int32[2m]   canonical edge id of every CSR entry
//                        eu, ev int32[m]   endpoints (eu < ev) of every canonical edge
//   oriented graph DG    dg_rp int64[n+1], dg_col int32[m], dg_eid int32[m]
//                        (out-lists keep the ascending-id order of the CSR rows)
//   triangle index       et_rp int64[m+1]  per canonical edge (a,b): start of L(a,b)
//     (r = 3)            et_w int32[3 n3]  L(a,b) = N(a) ∩ N(b), ascending
//                        et_t int32[3 n3]  canonical id of triangle {a,b,w} per entry
//                        tbase int64[m+1]  exclusive scan of |{w in L(a,b) : w > b}|
//                        tri_e int32[3 n3] edges (ab, ac, bc) of triangle (a<b<c)
//                        tri_pos int32[3 n3] offset of the triangle's entry in L(ab), L(ac), L(bc)
//   During a (3,4) peel, et_rnd int32[3 n3] (beside et_t) holds, per entry, the round in which
//   the entry's triangle is peeled (INT32_MAX while unscheduled).
//   4-clique index       qbase int64[n3+1], qval int32[n4]: per triangle (a<b<c) the vertices d > c
//     (r = 4)            adjacent to a, b and c, ascending; a 4-clique's id is its position in qval
//   Peel state (per decomposition): counts, rounds, cores, the A / N / L work lists, the control
//   block PeelCtl, and when enabled the (2,3) contraction's row copies, the dense bucket array,
//   the (2,4) heavy-phase scratch slices.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define ND_UNPEELED 0x7fffffff
#define ND_WARP 32

// ------------------------------------------------------------------------------------
// device helpers

// first index i in [0, n) with a[i] >= x (n if none)
__device__ __forceinline__ int64_t nd_lower_bound(const int32_t* __restrict__ a, int64_t n, int32_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// index of x in the ascending list a[0, n), or -1
__device__ __forceinline__ int64_t nd_find(const int32_t* __restrict__ a, int64_t n, int32_t x) {
    int64_t i = nd_lower_bound(a, n, x);
    return (i < n && __ldg(a + i) == x) ? i : -1;
}

__device__ __forceinline__ unsigned nd_lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Warp-aggregated append: every active lane gets its own slot in list[] (capacity cap);
// one atomicAdd per converged group of lanes. Returns the slot, or -1 if the list is full.
__device__ __forceinline__ int64_t nd_append(unsigned int* counter, int32_t* list, uint32_t cap, int32_t value,
                                             int* err) {
    unsigned mask = __activemask();
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    unsigned slot = base + __popc(mask & nd_lanemask_lt());
    if (slot >= cap) {
        atomicExch(err, 1);
        return -1;
    }
    list[slot] = value;
    return slot;
}

// Merge path over two ascending lists of distinct ids, A before B on ties: the warp splits the
// merged order into 32 runs of equal length, one per lane. nd_merge_run finds where the lane's run
// starts by bisecting its diagonal; nd_merge_walk walks the run one element per step and calls
// visit(i, j, w) for every common element w = A[i] = B[j], in ascending order within the lane.
// Each common element is met in exactly one run (the one that consumes its copy in A: B's next
// element is then the smallest not below it). About (na + nb) / 32 steps per lane, one load each.
// Indices are 32-bit (list lengths are below 2^31).
struct NdMergeRun {
    int i, j, steps;
};

__device__ __forceinline__ NdMergeRun nd_merge_run(const int32_t* __restrict__ A, int na, const int32_t* __restrict__ B,
                                                   int nb) {
    const int lane = threadIdx.x & 31;
    const int total = na + nb, per = (total + 31) >> 5;
    int d = lane * per;
    if (d > total) d = total;
    const int dend = d + per < total ? d + per : total;
    // i = how many of the first d merged elements come from A
    int lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(A + mid) <= __ldg(B + d - 1 - mid))
            lo = mid + 1;
        else
            hi = mid;
    }
    return NdMergeRun{lo, d - lo, dend - d};
}

template <typename Visit>
__device__ __forceinline__ void nd_merge_walk(const int32_t* __restrict__ A, int na, const int32_t* __restrict__ B,
                                              int nb, NdMergeRun r, Visit visit) {
    constexpr int32_t kEnd = 0x7fffffff;  // past a list's end (no vertex id)
    int i = r.i, j = r.j;
    int32_t av = i < na ? __ldg(A + i) : kEnd, bv = j < nb ? __ldg(B + j) : kEnd;
    for (int step = 0; step < r.steps; ++step) {
        const bool ta = av <= bv;
        if (ta && av == bv) visit(i, j, av);
        if (ta)
            ++i;
        else
            ++j;
        const int idx = ta ? i : j, lim = ta ? na : nb;
        const int32_t nv = idx < lim ? __ldg((ta ? A : B) + idx) : kEnd;
        if (ta)
            av = nv;
        else
            bv = nv;
    }
}

// |A ∩ B| counted by this lane's run (sum over the warp for the whole intersection)
__device__ __forceinline__ int nd_merge_count(const int32_t* __restrict__ A, int na, const int32_t* __restrict__ B,
                                              int nb) {
    int c = 0;
    nd_merge_walk(A, na, B, nb, nd_merge_run(A, na, B, nb), [&](int, int, int32_t) { ++c; });
    return c;
}

// Hash directory of the triangle lists (built for a (3,4) peel): list L(e) with more than
// ND_HASH_MIN entries gets an open-addressing table of 2^k >= 2 |L(e)| slots (load <= 1/2),
// linear probing. A slot holds the entry's vertex w, its triangle's id and the triangle's peel
// round (kept current by the peel, like the list tags), so one 16-byte load answers a lookup.
#define ND_HASH_MIN 32

struct __align__(16) NdHashSlot {
    int32_t w;    // -1: free
    int32_t id;
    int32_t rnd;
    int32_t pad;
};

__host__ __device__ __forceinline__ bool nd_hashed(int64_t n) { return n > ND_HASH_MIN && n <= ((int64_t)1 << 30); }

__host__ __device__ __forceinline__ int nd_hash_bits(int64_t n) {
    int k = 0;
    while (((int64_t)1 << k) < 2 * n) ++k;
    return k;
}

__device__ __forceinline__ uint32_t nd_hash_slot(int32_t w, int k) {
    return ((uint32_t)w * 0x9E3779B1u) >> (32 - k);  // multiplicative hashing (Knuth), top k bits
}

// Continue a lookup whose first probe (slot s, contents v) was loaded by the caller.
__device__ __forceinline__ bool nd_hash_resolve(const NdHashSlot* tab, int k, int32_t w, uint32_t s, int4 v,
                                                int32_t& id, int32_t& rnd) {
    uint32_t mask = (1u << k) - 1u;
    for (uint32_t probes = 0; probes <= mask; ++probes) {
        if (v.x == w) {
            id = v.y;
            rnd = v.z;
            return true;
        }
        if (v.x == -1) return false;
        s = (s + 1) & mask;
        v = *reinterpret_cast<const int4*>(tab + s);
    }
    return false;
}

// The slot of w in the table of 2^k slots: id and round of its triangle; false if w is absent.
// Plain (coherent) loads: the round field changes while the peel runs.
__device__ __forceinline__ bool nd_hash_find(const NdHashSlot* tab, int k, int32_t w, int32_t& id, int32_t& rnd) {
    uint32_t mask = (1u << k) - 1u, s = nd_hash_slot(w, k);
    for (uint32_t probes = 0; probes <= mask; ++probes) {
        int4 v = *reinterpret_cast<const int4*>(tab + s);
        if (v.x == w) {
            id = v.y;
            rnd = v.z;
            return true;
        }
        if (v.x == -1) return false;
        s = (s + 1) & mask;
    }
    return false;
}

// Use the warp merge when the longer list is at most this many times the shorter one (plus a
// constant), else per-lane binary searches of the shorter list's elements in the longer one.
__device__ __forceinline__ bool nd_prefer_merge(int64_t n_short, int64_t n_long) {
    return n_long <= 8 * n_short + 64;
}

__device__ __forceinline__ int64_t nd_atomic_dec(int32_t* p) { return (int64_t)atomicSub(p, 1); }
__device__ __forceinline__ int64_t nd_atomic_dec(int64_t* p) {
    return (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(p), 0xffffffffffffffffull);
}
__device__ __forceinline__ void nd_atomic_add(int32_t* p, int64_t v) { atomicAdd(p, (int)v); }
__device__ __forceinline__ void nd_atomic_add(int64_t* p, int64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// ------------------------------------------------------------------------------------
// device views

struct GraphView {
    int32_t n;
    int64_t m;  // undirected edges
    const int64_t* rp;
    const int32_t* col;
    const int64_t* split;
    const int64_t* ebase;
    const int32_t* pos2e;
    const int32_t* eu;
    const int32_t* ev;
    const int64_t* dg_rp;
    const int32_t* dg_col;
    const int32_t* dg_eid;
    const int64_t* et_rp;
    const int32_t* et_w;
    const int32_t* et_t;
    const int64_t* tbase;
    const int32_t* tri_e;
    const int32_t* tri_pos;
    int64_t n3;
    // hash directory of the long triangle lists (during a (3,4) decomposition), else NULL
    const int64_t* hoff;
    const NdHashSlot* htab;
    // (2,3) peel with graph contraction: current length of each adjacency row (rows start at rp[v]
    // and col / pos2e point to the peel's compacted copies), else NULL
    const int32_t* rlen;
    // (3,4) peel with list contraction: current length of each triangle list L(e) (the lists start
    // at et_rp[e]; et_w / et_t point to the peel's compacted copies), else NULL
    const int32_t* llen;
    // 4-clique index (r = 4): per triangle t = (a<b<c) the vertices d > c adjacent to a, b and c,
    // ascending, in qval[qbase[t] .. qbase[t+1]); a 4-clique's id is its position in qval
    const int64_t* qbase;
    const int32_t* qval;
    int64_t n4;
};

// Control block of the device-resident peeling loop (one per decomposition).
// A round t runs: ctl -> adv_min -> refill (4 kernels) -> adv_select -> update. Only ctl is
// a one-thread kernel; the others early-exit when their phase is not needed this round.
#define ND_HBINS 4096
#define ND_MODE_ADV 1

struct PeelCtl {
    // loop state
    int32_t t;          // current round
    int32_t mode;       // ND_MODE_ADV when this round moves to a new level
    int32_t done;       // 1 once every r-clique is peeled
    int32_t err;        // list overflow / inconsistency
    int32_t started;    // 0 before the first round
    int32_t wa, wn, wl; // ping-pong selectors of the A, N and L lists
    int32_t lmat;       // 0: L is implicitly 0..n_r-1
    int32_t heavy;      // persistent kernel: this round has a heavy phase (set by a serial step)
    int32_t sorta;      // persistent kernel: this round rebuilds A in id order (set by a serial step)
    int32_t heavy_split;// persistent kernel, (2,4): this round's heavy phase is split over the grid
    int64_t k;          // current level
    int64_t hi;         // bucket window: N holds every unpeeled r-clique with count < hi
    int64_t finished;   // r-cliques peeled so far
    int64_t n_r;
    int64_t max_rounds; // round cap (ND_ETIMEOUT)
    unsigned long long bar_timeout_ns;  // persistent kernel: longest wait at one grid barrier
    int32_t drop_block; // persistent kernel, test of the barrier bound: the last block leaves at once
    int32_t contract;   // graph contraction before this round's phases (set by the serial control step)
    int64_t contract_every;  // contract once this many r-cliques were peeled since the last one (0: never)
    int64_t peeled_since;    // r-cliques peeled since the last contraction
    int64_t contractions;    // contractions run
    int32_t contract_shift;  // compact a row that lost at least len >> shift entries (0: any loss)
    int32_t pad3;
    // list sizes
    unsigned int nA;    // |A| of a same-level round
    unsigned int cntA;  // |A| written by adv_select
    unsigned int nNext; // next round's A (r-cliques that fell to <= k during this round)
    unsigned int nN;    // |N| (current)
    unsigned int nN2;   // |N'| being written this round (advance rounds)
    unsigned int nL;    // |L|
    unsigned int nL2;   // |L'| being written by refill
    unsigned int nH;    // r-cliques of this round's A deferred to the heavy Update kernel
    unsigned int upd_next;  // next unassigned position of A in this round's Update (dynamic chunks)
    unsigned int upd_pad;
    unsigned long long minN;  // min count over unpeeled members of N (adv_min)
    unsigned long long gmin;  // min count over unpeeled r-cliques (refill)
    // grid barrier of the persistent peel kernel: arrivals since the launch, and the arrival
    // count up to which blocks have been released
    unsigned long long bar_arrive;
    unsigned long long bar_gen;
    // statistics
    unsigned long long listed;
    unsigned long long decs;
    long long advances, refills;
    // persistent kernel: nanoseconds per phase between barriers, as seen by block 0
    unsigned long long ph_ns[7];  // [6]: graph contraction
    unsigned long long ph_last;
    unsigned long long hist[ND_HBINS];
};

template <typename CT>
struct PeelView {
    CT* cnt;
    int32_t* rnd;
    int32_t* core;
    int32_t* A[2];
    int32_t* N[2];
    int32_t* L[2];
    int32_t* H;      // heavy r-cliques of the current round (capacity hcap)
    uint32_t hcap;
    // (2,4) heavy phase: hslices scratch slices of 5 * (hstage + 1) int32, one per block
    int32_t* hscratch;
    int64_t hstage;
    int32_t hslices;
    // (2,4) heavy phase split over the grid (persistent kernel): per slice the number of staged
    // vertices, and the candidate pairs of each heavy edge turned into offsets (hslices + 1)
    int32_t* hcnt;
    int64_t* hpre;
    // membership bitmap of A (NULL: never sorted) and the |A| from which a round sorts A
    uint32_t* abits;
    uint32_t sort_min;
    // (3,4): hash directory of the triangle lists (table offset per edge, tables, and for each
    // triangle and each of its three lists the slot holding it, -1 in a list without a table)
    const int64_t* hoff;
    NdHashSlot* htab;
    const int32_t* hpos;
    // (3,4) only: the round tag of every triangle-index entry, and what is needed to find the
    // three entries of a triangle (NULL for other (r,s))
    int32_t* et_rnd;
    const int32_t* tri_e;
    const int32_t* tri_pos;
    const int64_t* et_rp;
    uint32_t cap;
    PeelCtl* ctl;
    int64_t* round_size;
    int64_t* round_level;
    int64_t* round_ns;      // persistent kernel: Update wall time per round (block 0), or NULL
    int64_t round_cap;
    // (2,3) graph contraction (Section 5.6): the compacted copies of the adjacency rows (neighbour
    // and edge id), their current lengths and their lengths after the previous contraction; NULL
    // when off
    int32_t* ccol;
    int32_t* cpos;
    int32_t* clen;
    int32_t* cprev;
    // dense buckets (Section 4.2 Discussion): bcnt[c] = unpeeled r-cliques not yet scheduled whose
    // count is c, for c < bmax (the largest initial count + 1); NULL when off
    unsigned int* bcnt;
    int64_t bmax;
    // (3,4) list contraction: compacted copies of the triangle lists (vertex, triangle id), of the
    // entry offsets of every triangle (tri_pos), the lists' current lengths and their lengths at the
    // previous contraction; NULL when off (et_rnd is compacted along with them)
    int32_t* lw;
    int32_t* lt;
    int32_t* ltp;
    int32_t* llen;
    int32_t* lprev;
    // driving-list length above which Update defers an r-clique to the heavy phase (0: the
    // variant's built-in threshold)
    int64_t heavy_work;
};

// ------------------------------------------------------------------------------------
// launch accounting: every kernel launch goes through ND_K, which adds one to a process-wide
// counter (launches recorded while a stream is being captured into a CUDA graph are not
// counted; graph replays add their node count instead)
void nd_note_launches(int64_t k);
int64_t nd_total_launches();
void nd_set_capturing(bool on);
#define ND_K(...) (nd_note_launches(1), __VA_ARGS__)

// ------------------------------------------------------------------------------------
// host launchers (all enqueue on `st`, none synchronises)

// out[0..n] = exclusive scan of in[0..n), out[n] = total. tmp: nd_scan_tmp_bytes(n) bytes.
size_t nd_scan_tmp_bytes(int64_t n);
void nd_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t st);
void nd_fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t st);
void nd_iota_i32(int32_t* p, int64_t n, cudaStream_t st);
// *out = max over a[0..n) (int64 device scalar, must be pre-set to 0)
void nd_max_i64(const int64_t* a, int64_t n, unsigned long long* out, cudaStream_t st);
void nd_max_deg(const int64_t* rp, int32_t n, unsigned long long* out, cudaStream_t st);
void nd_sum_i64(const int64_t* a, int64_t n, unsigned long long* out, cudaStream_t st);
void nd_sum_i32(const int32_t* a, int64_t n, unsigned long long* out, cudaStream_t st);
void nd_max_i32(const int32_t* a, int64_t n, unsigned long long* out, cudaStream_t st);
// narrow int64 counts to int32; *err set to 1 if a value exceeds limit (<= INT32_MAX)
void nd_narrow_i64(const int64_t* in, int32_t* out, int64_t n, int64_t limit, int* err, cudaStream_t st);

// graph structure (nd_graph.cu)
void nd_validate_csr(const int64_t* rp, const int32_t* col, int32_t n, int64_t nnz, int* err, cudaStream_t st);
void nd_build_split(const int64_t* rp, const int32_t* col, int32_t n, int64_t* split, int64_t* updeg,
                    cudaStream_t st);
void nd_build_pos2e(const GraphView& g, int32_t* pos2e, int32_t* eu, int32_t* ev, int* err, cudaStream_t st);
// key(v) = (key_hi[v] or degree, v); key_hi NULL means degree
void nd_dg_count(const GraphView& g, const int32_t* key_hi, int64_t* outdeg, cudaStream_t st);
void nd_dg_fill(const GraphView& g, const int32_t* key_hi, int64_t* dg_rp_in, int32_t* dg_col, int32_t* dg_eid,
                cudaStream_t st);
// per canonical edge: sigma = |N(a) ∩ N(b)|, up = |{w in N(a) ∩ N(b) : w > b}|
void nd_edge_support(const GraphView& g, int64_t* sigma, int64_t* up, cudaStream_t st);
void nd_edge_fill(const GraphView& g, int64_t* et_rp, int64_t* tbase, int32_t* et_w, int32_t* et_t,
                  int32_t* tri_e, int32_t* tri_pos, cudaStream_t st);
void nd_edge_fill_tid(const GraphView& g, int32_t* et_t, int32_t* tri_pos, cudaStream_t st);
void nd_tri_tuples(const GraphView& g, int32_t* out, cudaStream_t st);
// 4-clique index: qcnt[t] = children of triangle t; then the children themselves
void nd_quad_count(const GraphView& g, int64_t* qcnt, cudaStream_t st);
void nd_quad_fill(const GraphView& g, const int64_t* qbase, int32_t* qval, cudaStream_t st);
void nd_quad_tuples(const GraphView& g, int32_t* out, cudaStream_t st);
void nd_edge_tuples(const GraphView& g, int32_t* out, cudaStream_t st);
void nd_max_edge_mindeg(const GraphView& g, unsigned long long* out, cudaStream_t st);
// hash directory of the triangle lists: slots per edge (0 for short lists), then the tables
void nd_tri_hash_sizes(const GraphView& g, int64_t* slots, cudaStream_t st);
void nd_tri_hash_fill(const GraphView& g, const int64_t* hoff, NdHashSlot* tab, int32_t* hpos, cudaStream_t st);
// blocks of the (2,4) heavy phase that hold a scratch slice; the others skip the phase
int nd_peel_heavy_slices();

// counting (nd_count.cu): counts into cnt (CT = int32_t or int64_t), zero-initialised
template <typename CT>
void nd_count_launch(const GraphView& g, int r, int s, CT* cnt, int64_t n_r, cudaStream_t st);

// peeling (nd_peel.cu)
template <typename CT>
void nd_peel_round(const GraphView& g, int r, int s, const PeelView<CT>& P, cudaStream_t st);
// the whole loop as one graph (WHILE node over rounds, IF nodes for the advance and refill
// phases); st2 and st3 are extra streams used only while capturing
template <typename CT>
cudaError_t nd_peel_loop_graph(const GraphView& g, int r, int s, const PeelView<CT>& P, cudaStream_t st,
                               cudaStream_t st2, cudaStream_t st3, cudaGraph_t* out);
int nd_peel_nodes_per_round(int r, int s, bool contract);
// the whole loop as one cooperative kernel launch
template <typename CT>
cudaError_t nd_peel_persistent(const GraphView& g, int r, int s, const PeelView<CT>& P, cudaStream_t st);
// barrier_ns 0: the default bound (60 s); drop_block: see ND_LIMIT_DROP_BLOCK; contract_every /
// contract_shift: graph contraction schedule (0: off)
void nd_peel_init(PeelCtl* ctl, int64_t n_r, int64_t max_rounds, cudaStream_t st, uint64_t barrier_ns = 0,
                  int drop_block = 0, int64_t contract_every = 0, int contract_shift = 2);
// row lengths len[v] = rp[v+1] - rp[v] (int32) into two arrays
void nd_row_len(const int64_t* rp, int32_t n, int32_t* a, int32_t* b, cudaStream_t st);
// dense buckets: bcnt[cnt[R]] += 1 for every R < n_r (bcnt zeroed by the caller)
template <typename CT>
void nd_bucket_fill(const CT* cnt, int64_t n_r, unsigned int* bcnt, int64_t bmax, cudaStream_t st);

int nd_sm_count();
