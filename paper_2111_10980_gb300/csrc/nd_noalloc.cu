// nd_kcore_noalloc: the (1,2) decomposition (k-core coreness) of a graph that is already in
// device memory, for callers that must not allocate.
//
// Some callers cannot let a library allocate device memory: a framework that has reserved the
// GPU's memory in its own caching pool (a cudaMalloc outside the pool can fail even though the
// pool has free space, and fragments the device), or a latency-critical loop in which a
// cudaMalloc / cudaFree may synchronise the device. This entry point serves them: it runs the
// same counting and peeling kernels as nd_decompose(r = 1, s = 2), but every scratch buffer lives
// in one file-scope __device__ array of fixed size, so the call itself allocates nothing.
//
// Limits and sharing:
//   * at most ND_NOALLOC_MAX_VERTICES vertices (larger graphs are rejected with ND_EINVAL);
//   * the array (about 8.4 MB) is part of the library image: every GPU that loads libnd.so holds
//     it until the process exits;
//   * all calls share it and it keeps the last call's contents; every call re-initialises the
//     parts it reads before reading them, so nothing has to be cleared by the caller;
//   * calls whose work overlaps on the GPU (two host threads, or two streams, at once) race on
//     the array and corrupt each other's results; serialise them;
//   * the first call on a device looks up the device address of the array with
//     cudaGetSymbolAddress (the host-side name of a __device__ array is not a device address);
//     that first call should come before any stream capture.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "nd.h"
#include "nd_common.cuh"
#include "nd_host.h"

namespace {

constexpr int64_t kMaxN = ND_NOALLOC_MAX_VERTICES;
constexpr size_t kCtlBytes = (sizeof(PeelCtl) + 255) & ~(size_t)255;
constexpr size_t kArr = (size_t)kMaxN * sizeof(int32_t);
// ctl | cnt | rnd | A0 | A1 | N0 | N1 | L0 | L1
constexpr size_t kScratchBytes = kCtlBytes + 8 * kArr;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (looked up once per device)
int scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return nd_set_error(ND_ECUDA, "nd_kcore_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        }
        g_scratch_dev[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_dev[dev]);
    return ND_OK;
}

}  // namespace

extern "C" int nd_kcore_noalloc(int32_t n, const int64_t* rowptr, const int32_t* col, int32_t* core_out,
                                void* stream) {
    if (n < 0 || n > kMaxN)
        return nd_set_error(ND_EINVAL, "nd_kcore_noalloc: n = %d is outside [0, %lld] (the size of the static scratch)",
                            n, (long long)kMaxN);
    if (!rowptr || (n > 0 && (!col || !core_out)))
        return nd_set_error(ND_EINVAL, "nd_kcore_noalloc: NULL rowptr, col or core_out");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nd_set_error(ND_ECUDA, "nd_kcore_noalloc: no current CUDA device");
    }
    unsigned char* base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    if (n == 0) return ND_OK;
    cudaStream_t st = (cudaStream_t)stream;

    PeelView<int32_t> P;
    memset(&P, 0, sizeof(P));
    P.ctl = reinterpret_cast<PeelCtl*>(base);
    int32_t* arr = reinterpret_cast<int32_t*>(base + kCtlBytes);
    P.cnt = arr + 0 * kMaxN;
    P.rnd = arr + 1 * kMaxN;
    P.A[0] = arr + 2 * kMaxN;
    P.A[1] = arr + 3 * kMaxN;
    P.N[0] = arr + 4 * kMaxN;
    P.N[1] = arr + 5 * kMaxN;
    P.L[0] = arr + 6 * kMaxN;
    P.L[1] = arr + 7 * kMaxN;
    P.core = core_out;
    P.cap = (uint32_t)n;
    P.round_size = nullptr;
    P.round_level = nullptr;
    P.round_cap = 0;  // no per-round record

    GraphView v;
    memset(&v, 0, sizeof(v));
    v.n = n;
    v.rp = rowptr;
    v.col = col;

    // count (degrees), then the same peeling rounds as nd_decompose(1, 2), launched one by one
    nd_count_launch<int32_t>(v, 1, 2, P.cnt, n, st);
    nd_fill_i32(P.rnd, ND_UNPEELED, n, st);
    nd_fill_i32(P.core, 0, n, st);
    nd_peel_init(P.ctl, n, (int64_t)n + 2, st);
    if ((rc = nd_check_launch("nd_kcore_noalloc"))) return rc;
    const int kChunk = 32;
    int64_t max_chunks = ((int64_t)n + 2) / kChunk + 4;
    // the head of the control block up to `finished` (pageable host memory: no pinned allocation)
    constexpr size_t kHead = offsetof(PeelCtl, finished) + sizeof(int64_t);
    alignas(8) unsigned char head[kHead];
    PeelCtl* h = reinterpret_cast<PeelCtl*>(head);
    for (int64_t chunk = 0;; ++chunk) {
        for (int i = 0; i < kChunk; ++i) nd_peel_round<int32_t>(v, 1, 2, P, st);
        if ((rc = nd_check_launch("nd_kcore_noalloc"))) return rc;
        e = cudaMemcpyAsync(head, P.ctl, kHead, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return nd_set_error(ND_ECUDA, "nd_kcore_noalloc: %s", cudaGetErrorString(e));
        }
        if (h->done) break;
        if (chunk + 1 > max_chunks)
            return nd_set_error(ND_ETIMEOUT, "nd_kcore_noalloc: peeling did not finish");
    }
    if (h->err & 1) return nd_set_error(ND_EINTERNAL, "nd_kcore_noalloc: a work list overflowed");
    if (h->err & 2) return nd_set_error(ND_ETIMEOUT, "nd_kcore_noalloc: round cap reached");
    if (h->err & 4) return nd_set_error(ND_EINTERNAL, "nd_kcore_noalloc: inconsistent peeling state");
    if (h->finished != n)
        return nd_set_error(ND_EINTERNAL, "nd_kcore_noalloc: peeled %lld of %d vertices", (long long)h->finished, n);
    return ND_OK;
}
