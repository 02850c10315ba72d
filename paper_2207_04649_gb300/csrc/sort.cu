// Device primitives: exclusive prefix sum and a stable LSD radix sort of
// (key, value) pairs. Both are written here from scratch (no CUB): the grid
// build sorts points by cell key, and the rank sort orders points by
// (rho desc, index asc), the order Ex-DPC processes points in (Section 3,
// "Dependent point computation", steps 2-4).
#include "dpc_internal.cuh"

#include <algorithm>
#include <atomic>

namespace dpc {

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;                                  // per thread
constexpr int kScanTile = kScanThreads * kScanItems;           // 2048


inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Each warp owns 32 * kScanItems consecutive values, loaded lane-striped
// (coalesced); value (i, lane) sits at warp offset i * 32 + lane.
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_sums(const uint32_t* __restrict__ in, int64_t n,
                                                                  uint32_t* __restrict__ sums) {
    __shared__ uint32_t wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)w * 32 * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i * 32 + lane;
        if (idx < n) s += in[idx];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) wsum[w] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < kScanThreads / 32; ++i) t += wsum[i];
        sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                              int64_t n, const uint32_t* __restrict__ tile_off,
                                                              uint32_t* __restrict__ total) {
    __shared__ uint32_t wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)w * 32 * kScanItems;
    uint32_t v[kScanItems];
    uint32_t carry = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i * 32 + lane;
        uint32_t x = idx < n ? in[idx] : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        v[i] = carry + incl - x;  // exclusive within the warp's run
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) wsum[w] = carry;
    __syncthreads();
    uint32_t woff = tile_off ? tile_off[blockIdx.x] : 0u;
    for (int i = 0; i < w; ++i) woff += wsum[i];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i * 32 + lane;
        if (idx < n) {
            out[idx] = woff + v[i];
            if (idx == n - 1 && total) *total = woff + v[i] + in[idx];
        }
    }
}

__global__ void k_set_zero(uint32_t* p) { *p = 0u; }

// ------------------------------------------------------------ radix sort
//
// LSD radix sort, 8-bit digits, three steps per pass: per-tile digit counts
// (k_rs_up), one exclusive scan of the counts in digit-major order (every
// tile's first slot for every digit), and the scatter (k_rs_down), which
// ranks a tile's keys stably by digit (warp-private digit counters in index
// order, then the warps' offsets per digit) and writes each key and value to
// its slot. A histogram of every pass's digits over all keys, taken once
// before the first pass, marks passes in which all keys share a digit: such
// a pass keeps the order and is a copy.

constexpr int kRsThreads = 256;
constexpr int kRsMaxPasses = 8;
// keys per thread and per tile: 16 and 4096 for 32-bit keys, 8 and 2048 for
// 64-bit keys (the tile's keys and values are staged in shared memory)
template <typename K>
constexpr int rs_items() { return sizeof(K) == 8 ? 8 : 16; }
template <typename K>
constexpr int rs_tile() { return kRsThreads * rs_items<K>(); }
constexpr int kRsMinTile = kRsThreads * 8;

// Global digit histograms of every pass, [pass][256].
template <typename K>
__global__ void __launch_bounds__(256) k_rs_hist_all(const K* __restrict__ keys, int64_t n, int passes,
                                                      uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kRsMaxPasses][256];
    for (int i = threadIdx.x; i < kRsMaxPasses * 256; i += blockDim.x) (&h[0][0])[i] = 0u;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const K k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(uint32_t)(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

__device__ __forceinline__ bool trivial_pass(const uint32_t* hist, int pass, int64_t n) {
    return __syncthreads_or(hist[pass * 256 + threadIdx.x] == (uint32_t)n) != 0;
}

// Digit counts of one tile: counts[digit * tiles + tile].
template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_rs_up(const K* __restrict__ kin, int64_t n, int pass,
                                                       const uint32_t* __restrict__ hist, uint32_t* __restrict__ counts,
                                                       int64_t tiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0u;
    if (trivial_pass(hist, pass, n)) return;  // also orders the clear before the counts
    constexpr int kRsItems = rs_items<K>(), kRsTile = rs_tile<K>();
    const int shift = 8 * pass;
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
    for (int i = 0; i < kRsItems; ++i) {
        const int64_t idx = base + i * kRsThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(uint32_t)(kin[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile: element order inside the tile is (warp, item,
// lane), which is index order. The tile's keys and values are first placed
// in shared memory in digit order, then written out so that consecutive
// threads write consecutive slots of a digit's run.
template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_rs_down(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                         K* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                                                         int pass, const uint32_t* __restrict__ hist,
                                                         const uint32_t* __restrict__ offs, int64_t tiles) {
    constexpr int kRsItems = rs_items<K>(), kRsTile = rs_tile<K>();
    __shared__ uint32_t wcnt[kRsThreads / 32][256];
    __shared__ uint32_t sbase[256];   // the digit's first global slot for this tile
    __shared__ uint32_t tbase[256];   // the digit's first slot inside the tile
    __shared__ uint32_t wsum[kRsThreads / 32];
    __shared__ K skey[kRsTile];
    __shared__ uint32_t sval[kRsTile];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int ww = 0; ww < kRsThreads / 32; ++ww) wcnt[ww][t] = 0u;
    sbase[t] = offs[(int64_t)t * tiles + blockIdx.x];
    const int64_t tile0 = (int64_t)blockIdx.x * kRsTile;
    if (trivial_pass(hist, pass, n)) {  // every key has the same digit: the order stays
        for (int64_t i = tile0 + t; i < min(n, tile0 + kRsTile); i += kRsThreads) {
            kout[i] = kin[i];
            vout[i] = vin[i];
        }
        return;
    }
    const int64_t base = tile0 + (int64_t)w * 32 * kRsItems;
    const int shift = 8 * pass;
    K key[kRsItems];
    uint32_t val[kRsItems], dig[kRsItems], rnk[kRsItems];
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        const int64_t idx = base + i * 32 + lane;
        const bool valid = idx < n;
        key[i] = valid ? kin[idx] : K(0);
        val[i] = valid ? vin[idx] : 0u;
        dig[i] = valid ? ((uint32_t)(key[i] >> shift) & 255u) : 256u;
    }
    // stable ranks within the warp's run of 32 * kRsItems keys: the lanes of
    // one step sharing a digit take consecutive ranks after the warp's count
    // of that digit so far, which the step's lowest such lane advances with
    // one shared-memory atomic. Every lane waits in the step's shuffle for
    // the value of that atomic, so the steps' atomics take effect in step
    // order. The matches of all steps go out first.
    unsigned peers[kRsItems];
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) peers[i] = __match_any_sync(0xffffffffu, dig[i]);
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        const int leader = __ffs(peers[i]) - 1;
        uint32_t before = 0u;
        if (lane == leader && dig[i] < 256u) before = atomicAdd(&wcnt[w][dig[i]], (uint32_t)__popc(peers[i]));
        before = __shfl_sync(0xffffffffu, before, leader);
        rnk[i] = before + (uint32_t)__popc(peers[i] & lt);
    }
    __syncthreads();
    // thread t = digit t: the warps' exclusive offsets, and the digit's first
    // slot in the tile (an exclusive scan of the tile's counts over digits)
    uint32_t cnt = 0;
#pragma unroll
    for (int ww = 0; ww < kRsThreads / 32; ++ww) {
        const uint32_t c = wcnt[ww][t];
        wcnt[ww][t] = cnt;
        cnt += c;
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    uint32_t wo = 0;
    for (int ww = 0; ww < w; ++ww) wo += wsum[ww];
    tbase[t] = wo + incl - cnt;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        if (dig[i] < 256u) {
            const uint32_t lp = tbase[dig[i]] + wcnt[w][dig[i]] + rnk[i];
            skey[lp] = key[i];
            sval[lp] = val[i];
        }
    }
    __syncthreads();
    const int nvalid = (int)min((int64_t)kRsTile, n - tile0);
    for (int j = t; j < nvalid; j += kRsThreads) {
        const K k = skey[j];
        const uint32_t d = (uint32_t)(k >> shift) & 255u;
        const uint32_t pos = sbase[d] + (uint32_t)j - tbase[d];
        kout[pos] = k;
        vout[pos] = sval[j];
    }
}

template <typename K>
cudaError_t radix_sort_impl(const K* k_in, const uint32_t* v_in, K* k_out, uint32_t* v_out, K* k_tmp,
                            uint32_t* v_tmp, int64_t n, int nbits, void* temp, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int passes = (nbits + 7) / 8;
    if (passes == 0) {
        cudaError_t e = cudaMemcpyAsync(k_out, k_in, n * sizeof(K), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(v_out, v_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    }
    const int64_t tiles = ceil_div(n, rs_tile<K>());
    // temp: hist [8][256], counts [256][tiles], offsets [256][tiles], scan scratch
    uint32_t* hist = reinterpret_cast<uint32_t*>(temp);
    uint32_t* counts = hist + kRsMaxPasses * 256;
    uint32_t* offs = counts + align256(256 * tiles * sizeof(uint32_t)) / sizeof(uint32_t);
    void* stemp = offs + align256(256 * tiles * sizeof(uint32_t)) / sizeof(uint32_t);
    cudaError_t e = cudaMemsetAsync(hist, 0, kRsMaxPasses * 256 * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const unsigned hb = (unsigned)std::min<int64_t>(ceil_div(n, 256 * 16), 152 * 8);
    (k_rs_hist_all<K><<<hb, 256, 0, st>>>(k_in, n, passes, hist), note_launch());
    const K* src_k = k_in;
    const uint32_t* src_v = v_in;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        K* dk = to_out ? k_out : k_tmp;
        uint32_t* dv = to_out ? v_out : v_tmp;
        (k_rs_up<K><<<(unsigned)tiles, kRsThreads, 0, st>>>(src_k, n, p, hist, counts, tiles), note_launch());
        e = exclusive_scan_u32(counts, offs, 256 * tiles, nullptr, stemp, st);
        if (e != cudaSuccess) return e;
        (k_rs_down<K><<<(unsigned)tiles, kRsThreads, 0, st>>>(src_k, src_v, dk, dv, n, p, hist, offs, tiles),
         note_launch());
        src_k = dk;
        src_v = dv;
    }
    return cudaGetLastError();
}

}  // namespace

size_t scan_temp_bytes(int64_t n) {
    size_t b = 0;
    while (n > kScanTile) {
        n = ceil_div(n, kScanTile);
        b += 2 * align256((size_t)n * sizeof(uint32_t));
    }
    return b + 256;
}

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, void* temp,
                               cudaStream_t st) {
    if (n <= 0) {
        if (total) (k_set_zero<<<1, 1, 0, st>>>(total), note_launch());
        return cudaGetLastError();
    }
    const int64_t nblk = ceil_div(n, kScanTile);
    if (nblk == 1) {
        (k_scan_tiles<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr, total), note_launch());
        return cudaGetLastError();
    }
    uint32_t* sums = reinterpret_cast<uint32_t*>(temp);
    uint32_t* sums_scan = sums + align256(nblk * sizeof(uint32_t)) / sizeof(uint32_t);
    void* next = reinterpret_cast<char*>(temp) + 2 * align256(nblk * sizeof(uint32_t));
    (k_scan_tile_sums<<<(unsigned)nblk, kScanThreads, 0, st>>>(in, n, sums), note_launch());
    cudaError_t e = exclusive_scan_u32(sums, sums_scan, nblk, nullptr, next, st);
    if (e != cudaSuccess) return e;
    (k_scan_tiles<<<(unsigned)nblk, kScanThreads, 0, st>>>(in, out, n, sums_scan, total), note_launch());
    return cudaGetLastError();
}

size_t radix_sort_temp_bytes(int64_t n) {
    const int64_t tiles = ceil_div(n > 0 ? n : 1, kRsMinTile);
    return kRsMaxPasses * 256 * sizeof(uint32_t) + 2 * align256(256 * tiles * sizeof(uint32_t)) +
           scan_temp_bytes(256 * tiles) + 256;
}

cudaError_t radix_sort_u64(const uint64_t* k_in, const uint32_t* v_in, uint64_t* k_out, uint32_t* v_out,
                           uint64_t* k_tmp, uint32_t* v_tmp, int64_t n, int nbits, void* temp,
                           cudaStream_t st) {
    return radix_sort_impl<uint64_t>(k_in, v_in, k_out, v_out, k_tmp, v_tmp, n, nbits, temp, st);
}

cudaError_t radix_sort_u32(const uint32_t* k_in, const uint32_t* v_in, uint32_t* k_out, uint32_t* v_out,
                           uint32_t* k_tmp, uint32_t* v_tmp, int64_t n, int nbits, void* temp,
                           cudaStream_t st) {
    return radix_sort_impl<uint32_t>(k_in, v_in, k_out, v_out, k_tmp, v_tmp, n, nbits, temp, st);
}

}  // namespace dpc
