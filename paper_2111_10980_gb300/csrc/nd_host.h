// Host-side structures behind the opaque handles of nd.h.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <vector>

#include "nd.h"
#include "nd_common.cuh"

struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct nd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;
    std::atomic<size_t> in_use{0};
    std::atomic<int> ngraphs{0};
    nd_alloc_fn af = nullptr;
    nd_free_fn ff = nullptr;
    void* user = nullptr;
    void* pinned = nullptr;  // 4 KiB of pinned host memory for scalar read-backs
    cudaStream_t cap_st[2] = {nullptr, nullptr};  // extra streams used only to capture graph bodies
    // nd_ctx_set_limits (0: default)
    int64_t max_rounds = 0;
    int64_t barrier_ns = 0;
    int64_t count_limit = 0;
    int32_t limit_flags = 0;
    void* stage = nullptr;  // pinned staging of batches (grown on demand)
    size_t stage_bytes = 0;
    // nd_ctx_set_tuning, indexed by r * 8 + s
    int64_t tune_heavy[64] = {0};
    int32_t tune_flags[64] = {0};
};

struct nd_graph {
    nd_ctx* ctx = nullptr;
    int32_t n = 0;
    int64_t m = 0;    // undirected edges
    int64_t nnz = 0;  // 2m
    DBuf rp, col, scal;
    // canonical edge index
    bool have_base = false;
    DBuf split, ebase, pos2e, eu, ev;
    int64_t maxdeg = 0;
    int64_t edge_mindeg = -1;  // max over edges of min(deg u, deg v); -1 until needed
    // orientation
    int orient = -1;
    DBuf dg_rp, dg_col, dg_eid;
    int64_t maxout = 0;
    // triangle index
    bool have_tri = false;
    int64_t n3 = 0;
    // 4-clique index
    bool have_quad = false;
    int64_t n4 = 0;
    DBuf qbase, qval;
    DBuf et_rp, et_w, et_t, tbase, tri_e, tri_pos;
    // hash directory of the long triangle lists, held only while a (3,4) decomposition runs
    DBuf hoff, htab, hpos;
    // record of the last decomposition
    bool have_last = false;
    int64_t last_rho = 0;
    std::vector<int64_t> last_sizes, last_levels, last_round_ns;
};

struct PeelOut {
    DBuf core, rnd;
    int64_t rho = 0, max_core = 0, listed = 0, decs = 0, advances = 0, refills = 0;
    double phase_ms[7] = {0, 0, 0, 0, 0, 0, 0};  // [6]: graph contraction
    int64_t contractions = 0;
    std::vector<int64_t> sizes, levels, round_ns;
};

int nd_set_error(int code, const char* fmt, ...);
int nd_alloc(nd_ctx* ctx, DBuf& b, size_t bytes);
void nd_free(nd_ctx* ctx, DBuf& b);
int nd_sync(nd_ctx* ctx, const char* what);
int nd_check_launch(const char* what);
GraphView nd_view(const nd_graph* g);
int nd_prepare(nd_graph* g, int r, int s, int64_t* n_r, double* t_orient, double* t_index);
int nd_pick_width(const nd_graph* g, int r, int s, int count_width, int* w);
int nd_count_into(nd_graph* g, int r, int s, int w, int64_t n_r, DBuf& cnt);
int nd_decompose_dev(nd_graph* g, int r, int s, int count_width, int flags, PeelOut& po, nd_stats* st);
