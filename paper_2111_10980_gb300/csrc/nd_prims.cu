// Parallel primitives (Section 3: prefix sum and filter in O(n) work), written for the GPU:
// a three-phase exclusive scan (tile sums, scan of tile sums, tile scan with offsets),
// grid-stride fills and reductions sized to the SM count.
#include "nd_common.cuh"

#include <atomic>
#include <climits>

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// exclusive block scan (blockDim.x a multiple of 32, <= 1024); returns the thread's prefix,
// *total = block sum. Ends with a barrier so the shared scratch can be reused.
__device__ int64_t block_excl_scan(int64_t v, int64_t* total) {
    __shared__ int64_t wsum[33];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int nw = blockDim.x >> 5;
    int64_t inc = warp_incl_scan(v);
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < nw ? wsum[lane] : 0;
        int64_t wi = warp_incl_scan(w);
        if (lane < nw) wsum[lane] = wi - w;
        if (lane == 31) wsum[32] = wi;
    }
    __syncthreads();
    int64_t res = wsum[wid] + inc - v;
    *total = wsum[32];
    __syncthreads();
    return res;
}

__global__ void k_scan_tiles(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ bsum) {
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    int64_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int64_t* bsum, int64_t nb) {
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanThreads) {
        int64_t idx = base + threadIdx.x;
        int64_t v = idx < nb ? bsum[idx] : 0;
        int64_t tot;
        int64_t pre = block_excl_scan(v, &tot);
        if (idx < nb) bsum[idx] = carry + pre;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_scan_apply(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                             const int64_t* __restrict__ bsum, int64_t nb) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        s += v[i];
    }
    int64_t tot;
    int64_t pre = block_excl_scan(s, &tot) + bsum[blockIdx.x];
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = pre;
        pre += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = bsum[nb];
}

__global__ void k_fill_i32(int32_t* p, int32_t v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_iota_i32(int32_t* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

template <typename T, bool kMax, bool kDiff>
__global__ void k_reduce(const T* __restrict__ a, int64_t n, unsigned long long* out) {
    unsigned long long acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        long long v = kDiff ? (long long)(a[i + 1] - a[i]) : (long long)a[i];
        unsigned long long u = v < 0 ? 0ull : (unsigned long long)v;
        acc = kMax ? (u > acc ? u : acc) : acc + u;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_down_sync(0xffffffffu, acc, o);
        acc = kMax ? (y > acc ? y : acc) : acc + y;
    }
    if ((threadIdx.x & 31) == 0) {
        if (kMax)
            atomicMax(out, acc);
        else
            atomicAdd(out, acc);
    }
}

__global__ void k_narrow(const int64_t* __restrict__ in, int32_t* __restrict__ out, int64_t n, int64_t limit,
                         int* err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = in[i];
        if (v > limit || v < 0) {
            atomicExch(err, 1);
            v = limit;
        }
        out[i] = (int32_t)v;
    }
}

int grid_for(int64_t n, int threads) {
    int64_t want = (n + threads - 1) / threads;
    int64_t cap = (int64_t)nd_sm_count() * 8;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

}  // namespace

static std::atomic<int64_t> g_launches{0};
static thread_local bool g_capturing = false;

void nd_note_launches(int64_t k) {
    if (!g_capturing) g_launches += k;
}
int64_t nd_total_launches() { return g_launches.load(); }
void nd_set_capturing(bool on) { g_capturing = on; }

int nd_sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

size_t nd_scan_tmp_bytes(int64_t n) {
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    return (size_t)(nb + 1) * sizeof(int64_t);
}

void nd_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t st) {
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    int64_t* bsum = static_cast<int64_t*>(tmp);
    ND_K(k_scan_tiles<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, bsum));
    ND_K(k_scan_sums<<<1, kScanThreads, 0, st>>>(bsum, nb));
    ND_K(k_scan_apply<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, bsum, nb));
}

void nd_fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    ND_K(k_fill_i32<<<grid_for(n, 256), 256, 0, st>>>(p, v, n));
}

void nd_iota_i32(int32_t* p, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    ND_K(k_iota_i32<<<grid_for(n, 256), 256, 0, st>>>(p, n));
}

void nd_max_i64(const int64_t* a, int64_t n, unsigned long long* out, cudaStream_t st) {
    if (n <= 0) return;
    ND_K(k_reduce<int64_t, true, false><<<grid_for(n, 256), 256, 0, st>>>(a, n, out));
}

void nd_max_deg(const int64_t* rp, int32_t n, unsigned long long* out, cudaStream_t st) {
    if (n <= 0) return;
    ND_K(k_reduce<int64_t, true, true><<<grid_for(n, 256), 256, 0, st>>>(rp, n, out));
}

void nd_sum_i64(const int64_t* a, int64_t n, unsigned long long* out, cudaStream_t st) {
    if (n <= 0) return;
    ND_K(k_reduce<int64_t, false, false><<<grid_for(n, 256), 256, 0, st>>>(a, n, out));
}

void nd_sum_i32(const int32_t* a, int64_t n, unsigned long long* out, cudaStream_t st) {
    if (n <= 0) return;
    ND_K(k_reduce<int32_t, false, false><<<grid_for(n, 256), 256, 0, st>>>(a, n, out));
}

void nd_max_i32(const int32_t* a, int64_t n, unsigned long long* out, cudaStream_t st) {
    if (n <= 0) return;
    ND_K(k_reduce<int32_t, true, false><<<grid_for(n, 256), 256, 0, st>>>(a, n, out));
}

void nd_narrow_i64(const int64_t* in, int32_t* out, int64_t n, int64_t limit, int* err, cudaStream_t st) {
    if (n <= 0) return;
    ND_K(k_narrow<<<grid_for(n, 256), 256, 0, st>>>(in, out, n, limit < INT_MAX ? limit : INT_MAX, err));
}

namespace {
__global__ void k_row_len(const int64_t* __restrict__ rp, int32_t n, int32_t* __restrict__ a,
                          int32_t* __restrict__ b) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t d = (int32_t)(rp[v + 1] - rp[v]);
        a[v] = d;
        b[v] = d;
    }
}
}  // namespace

void nd_row_len(const int64_t* rp, int32_t n, int32_t* a, int32_t* b, cudaStream_t st) {
    if (n <= 0) return;
    ND_K(k_row_len<<<grid_for(n, 256), 256, 0, st>>>(rp, n, a, b));
}
