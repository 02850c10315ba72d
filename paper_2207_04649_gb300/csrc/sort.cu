// Device primitives: exclusive prefix sum and a stable LSD radix sort of
// (key, value) pairs. Both are written here from scratch (no CUB): the grid
// build sorts points by cell key, and the rank sort orders points by
// (rho desc, index asc), the order Ex-DPC processes points in (Section 3,
// "Dependent point computation", steps 2-4).
#include "dpc_internal.cuh"

#include <atomic>

namespace dpc {

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;                                  // per thread
constexpr int kScanTile = kScanThreads * kScanItems;           // 2048

constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;                 // 2048 (8 items measured faster than 4, 16 and 32)

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

// Warp-aggregated digit histogram of one tile.
template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const K* __restrict__ keys, int64_t n, int shift,
                                                         uint32_t* __restrict__ hist, int nblk) {
    __shared__ uint32_t h[256];
    const int t = threadIdx.x, lane = t & 31;
    h[t] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int i = 0; i < kRsItems; ++i) {
        int64_t idx = base + i * kRsThreads + t;
        uint32_t dig = idx < n ? ((uint32_t)(keys[idx] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, dig);
        if (dig < 256u && (peers & lt) == 0u) atomicAdd(&h[dig], (uint32_t)__popc(peers));
    }
    __syncthreads();
    hist[(int64_t)t * nblk + blockIdx.x] = h[t];
}

// Stable scatter: element order inside a tile is (iteration, warp, lane),
// which is index order; offsets are digit-major over tiles.
template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                            K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                            int64_t n, int shift, const uint32_t* __restrict__ offs,
                                                            int nblk) {
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[kRsThreads / 32][256];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    run[t] = offs[(int64_t)t * nblk + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int it = 0; it < kRsItems; ++it) {
        const int64_t first = base + (int64_t)it * kRsThreads;
        if (first >= n) break;  // uniform across the block
#pragma unroll
        for (int ww = 0; ww < kRsThreads / 32; ++ww) wcnt[ww][t] = 0u;
        __syncthreads();
        const int64_t idx = first + t;
        const bool valid = idx < n;
        K key = valid ? kin[idx] : K(0);
        uint32_t dig = valid ? ((uint32_t)(key >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, dig);
        uint32_t my = __popc(peers & lt);
        if (valid && my == 0u) wcnt[w][dig] = __popc(peers);
        __syncthreads();
        {
            uint32_t r = run[t];
#pragma unroll
            for (int ww = 0; ww < kRsThreads / 32; ++ww) {
                uint32_t c = wcnt[ww][t];
                wcnt[ww][t] = r;
                r += c;
            }
            run[t] = r;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = wcnt[w][dig] + my;
            kout[pos] = key;
            vout[pos] = vin[idx];
        }
        __syncthreads();
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
    const int nblk = (int)ceil_div(n, kRsTile);
    const int64_t nh = (int64_t)256 * nblk;
    uint32_t* hist = reinterpret_cast<uint32_t*>(temp);
    uint32_t* offs = hist + nh;
    void* stemp = reinterpret_cast<char*>(temp) + align256(2 * nh * sizeof(uint32_t));
    const K* src_k = k_in;
    const uint32_t* src_v = v_in;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        K* dk = to_out ? k_out : k_tmp;
        uint32_t* dv = to_out ? v_out : v_tmp;
        (k_rs_hist<K><<<nblk, kRsThreads, 0, st>>>(src_k, n, 8 * p, hist, nblk), note_launch());
        cudaError_t e = exclusive_scan_u32(hist, offs, nh, nullptr, stemp, st);
        if (e != cudaSuccess) return e;
        (k_rs_scatter<K><<<nblk, kRsThreads, 0, st>>>(src_k, src_v, dk, dv, n, 8 * p, offs, nblk), note_launch());
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
    const int64_t nblk = ceil_div(n > 0 ? n : 1, kRsTile);
    const int64_t nh = 256 * nblk;
    return align256(2 * nh * sizeof(uint32_t)) + scan_temp_bytes(nh);
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
