// dl_sort_unique_noalloc: sort + deduplicate rows held in caller-owned device columns
// without allocating any memory.  For callers that cannot call cudaMalloc (see dl.h).
//
// All scratch lives in one file-scope device array.  Host code never dereferences the
// array's name (in host code it names a host-side stand-in, not device memory): the device
// address is obtained once per device with cudaGetSymbolAddress and passed to the kernels.
#include <mutex>

#include "common.cuh"

namespace {

constexpr uint32_t kMaxRows = DL_NOALLOC_MAX_ROWS;
constexpr uint32_t kMaxArity = DL_NOALLOC_MAX_ARITY;
constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr uint32_t kTile = kThreads * kItems;                 // rows per tile
constexpr uint32_t kMaxTiles = (kMaxRows + kTile - 1) / kTile;
constexpr int kRadix = 256;
constexpr unsigned kFullMask = 0xffffffffu;

// scratch layout, in uint32 words
constexpr size_t kBufWords = (size_t)kMaxArity * kMaxRows;   // one ping-pong buffer
constexpr size_t kOffA = 0;
constexpr size_t kOffB = kOffA + kBufWords;
constexpr size_t kOffHist = kOffB + kBufWords;                // kRadix * kMaxTiles counters + total
constexpr size_t kOffTile = kOffHist + (size_t)kRadix * kMaxTiles + 1;  // kMaxTiles + 1 counters
constexpr size_t kScratchWords = kOffTile + kMaxTiles + 64;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
uint32_t* g_scratch_addr[kMaxDevices] = {nullptr};

struct Cols {
    uint32_t* c[kMaxArity];
};

__global__ void k_na_hist(const uint32_t* __restrict__ key, uint32_t n, uint32_t shift, uint32_t* __restrict__ hist,
                          uint32_t ntiles) {
    __shared__ uint32_t h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * kTile;
    for (uint32_t j = threadIdx.x; j < kTile; j += blockDim.x) {
        const uint32_t i = base + j;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[d * ntiles + blockIdx.x] = h[d];
}

// Exclusive scan of `count` words in place by one CTA of 1024 threads; data[count] = total.
__global__ void k_na_scan(uint32_t* data, uint32_t count) {
    __shared__ uint32_t warp_sums[32];
    const uint32_t per = (count + blockDim.x - 1) / blockDim.x;
    const uint32_t b = threadIdx.x * per, e = min(b + per, count);
    uint32_t s = 0;
    for (uint32_t i = b; i < e; i++) s += data[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFullMask, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_sums[lane];
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFullMask, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    uint32_t run = (warp ? warp_sums[warp - 1] : 0) + x - s;
    for (uint32_t i = b; i < e; i++) {
        const uint32_t v = data[i];
        data[i] = run;
        run += v;
    }
    if (threadIdx.x == blockDim.x - 1) data[count] = run;
}

// Stable scatter by one 8-bit digit: warp w of a tile owns rows [base + w*32*kItems, +32*kItems)
// and visits them in order, so equal digits keep their input order.
__global__ void __launch_bounds__(kThreads) k_na_scatter(Cols src, Cols dst, uint32_t arity, uint32_t n,
                                                         uint32_t keycol, uint32_t shift,
                                                         const uint32_t* __restrict__ offs, uint32_t ntiles) {
    __shared__ uint32_t wcnt[kThreads / 32][kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kThreads / 32) * kRadix; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint32_t wbase = blockIdx.x * kTile + warp * 32 * kItems;
    const unsigned lt = (1u << lane) - 1;
    uint32_t rank[kItems], dig[kItems];
    const uint32_t* key = src.c[keycol];
    for (int j = 0; j < kItems; j++) {
        const uint32_t i = wbase + j * 32 + lane;
        const bool valid = i < n;
        const uint32_t d = valid ? (key[i] >> shift) & (kRadix - 1) : 0xffffffffu;
        const unsigned peers = __match_any_sync(kFullMask, d);
        const uint32_t before = valid ? wcnt[warp][d] : 0;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[j] = before + __popc(peers & lt);
        dig[j] = d;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
        uint32_t run = offs[d * ntiles + blockIdx.x];
        for (int w = 0; w < kThreads / 32; w++) {
            const uint32_t c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int j = 0; j < kItems; j++) {
        const uint32_t i = wbase + j * 32 + lane;
        if (i < n) {
            const uint32_t to = wcnt[warp][dig[j]] + rank[j];
            for (uint32_t c = 0; c < arity; c++) dst.c[c][to] = src.c[c][i];
        }
    }
}

__device__ __forceinline__ bool first_of_run(const Cols& t, uint32_t arity, uint32_t i) {
    if (i == 0) return true;
    for (uint32_t c = 0; c < arity; c++)
        if (t.c[c][i] != t.c[c][i - 1]) return true;
    return false;
}

__global__ void k_na_count(Cols t, uint32_t arity, uint32_t n, uint32_t* __restrict__ tile_count) {
    __shared__ uint32_t total;
    if (threadIdx.x == 0) total = 0;
    __syncthreads();
    uint32_t c = 0;
    const uint32_t base = blockIdx.x * kTile;
    for (uint32_t j = threadIdx.x; j < kTile; j += blockDim.x) {
        const uint32_t i = base + j;
        if (i < n && first_of_run(t, arity, i)) c++;
    }
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(kFullMask, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&total, c);
    __syncthreads();
    if (threadIdx.x == 0) tile_count[blockIdx.x] = total;
}

__global__ void k_na_write(Cols t, uint32_t arity, uint32_t n, const uint32_t* __restrict__ tile_off, Cols out) {
    __shared__ uint32_t warp_sums[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t run = tile_off[blockIdx.x];
    const uint32_t base = blockIdx.x * kTile;
    for (int j = 0; j < kItems; j++) {
        const uint32_t i = base + j * kThreads + threadIdx.x;
        const bool f = i < n && first_of_run(t, arity, i);
        const unsigned ball = __ballot_sync(kFullMask, f);
        if (lane == 0) warp_sums[warp] = __popc(ball);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < kThreads / 32; w++) {
            if (w < warp) before += warp_sums[w];
            total += warp_sums[w];
        }
        if (f) {
            const uint32_t o = run + before + __popc(ball & ((1u << lane) - 1));
            for (uint32_t c = 0; c < arity; c++) out.c[c][o] = t.c[c][i];
        }
        run += total;
        __syncthreads();
    }
}

// Device address of the scratch array on the current device (set up once per device).
int scratch_address(uint32_t** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DL_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return DL_ERR_CUDA;
        }
        g_scratch_addr[dev] = (uint32_t*)p;
    }
    *out = g_scratch_addr[dev];
    return DL_OK;
}

}  // namespace

extern "C" int dl_sort_unique_noalloc(const uint32_t* const* dcols_in, uint32_t arity, uint64_t nrows,
                                      uint32_t* const* dcols_out, uint64_t* nrows_out, void* stream) {
    if (!dcols_in || !dcols_out || !nrows_out || arity < 1) return DL_ERR_ARG;
    if (arity > kMaxArity || nrows > kMaxRows) return DL_ERR_CAPACITY;
    for (uint32_t c = 0; c < arity; c++)
        if (!dcols_in[c] || !dcols_out[c]) return DL_ERR_ARG;
    uint32_t* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != DL_OK) return rc;
    if (nrows == 0) {
        *nrows_out = 0;
        return DL_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n = (uint32_t)nrows;
    const uint32_t ntiles = (n + kTile - 1) / kTile;
    // A launch error left pending on this thread by earlier, unrelated work would otherwise
    // be reported below as this call's: take it off first.
    (void)cudaGetLastError();
    Cols a, b, out;
    for (uint32_t c = 0; c < kMaxArity; c++) {
        a.c[c] = scratch + kOffA + (size_t)c * kMaxRows;
        b.c[c] = scratch + kOffB + (size_t)c * kMaxRows;
        out.c[c] = c < arity ? dcols_out[c] : nullptr;
    }
    uint32_t* hist = scratch + kOffHist;
    uint32_t* tiles = scratch + kOffTile;
    for (uint32_t c = 0; c < arity; c++)
        if (cudaMemcpyAsync(a.c[c], dcols_in[c], sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return DL_ERR_CUDA;
    // LSD radix sort: last column first, 8-bit digits from low to high; every digit pass
    // rewrites all counters it reads, so nothing left by an earlier call is used.
    for (int c = (int)arity - 1; c >= 0; c--) {
        for (uint32_t shift = 0; shift < 32; shift += 8) {
            k_na_hist<<<ntiles, kThreads, 0, s>>>(a.c[c], n, shift, hist, ntiles);
            k_na_scan<<<1, 1024, 0, s>>>(hist, kRadix * ntiles);
            k_na_scatter<<<ntiles, kThreads, 0, s>>>(a, b, arity, n, (uint32_t)c, shift, hist, ntiles);
            Cols t = a;
            a = b;
            b = t;
        }
    }
    k_na_count<<<ntiles, kThreads, 0, s>>>(a, arity, n, tiles);
    k_na_scan<<<1, 1024, 0, s>>>(tiles, ntiles);
    k_na_write<<<ntiles, kThreads, 0, s>>>(a, arity, n, tiles, out);
    if (cudaGetLastError() != cudaSuccess) return DL_ERR_CUDA;
    uint32_t total = 0;
    if (cudaMemcpyAsync(&total, tiles + ntiles, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return DL_ERR_CUDA;
    *nrows_out = total;
    return DL_OK;
}
