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

// ------------------------------------------------ one-sweep radix sort
//
// Each 8-bit pass is one kernel: a block takes the next tile of kOsTile keys
// (tiles numbered in the order blocks start, from an atomic counter), ranks
// its keys stably by digit (warp-private digit counters, in index order),
// publishes its digit counts, and finds the counts of all earlier tiles by
// looking back through their published words (decoupled look-back: a tile
// whose inclusive prefix is published ends the walk). Every earlier tile
// belongs to a block that has already started, so a walk only waits for
// blocks that are running; the waits are bounded (kOsSpin polls), after
// which the block sets the error word and stops waiting. The digit offsets
// of every pass come from one histogram pass over the keys before the
// first pass.

constexpr int kOsThreads = 256;
constexpr int kOsItems = 8;
constexpr int kOsTile = kOsThreads * kOsItems;   // 2048 keys
constexpr int kOsMaxPasses = 8;
constexpr int kOsSpin = 1 << 22;                 // look-back polls before a wait gives up
constexpr int kOsWin = 16;                       // earlier tiles read per look-back round

// Global digit histograms of every pass, [pass][256].
template <typename K>
__global__ void __launch_bounds__(256) k_os_hist(const K* __restrict__ keys, int64_t n, int passes,
                                                  uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kOsMaxPasses][256];
    for (int i = threadIdx.x; i < kOsMaxPasses * 256; i += blockDim.x) (&h[0][0])[i] = 0u;
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

__device__ __forceinline__ unsigned long long os_load(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void os_store(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// One pass over bits [8 pass, 8 pass + 8). status: [tiles][256] words
// (flag << 32 | count), flags 2 pass + 1 (the tile's own count) and
// 2 pass + 2 (the count of this and every earlier tile); words of earlier
// passes read as "not yet".
template <typename K>
__global__ void __launch_bounds__(kOsThreads) k_os_pass(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                         K* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                                                         int pass, const uint32_t* __restrict__ hist,
                                                         unsigned long long* __restrict__ status,
                                                         uint32_t* __restrict__ tile_ctr, unsigned int* __restrict__ err) {
    __shared__ uint32_t wcnt[kOsThreads / 32][256];
    __shared__ uint32_t sbase[256];
    __shared__ uint32_t s_tile;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const unsigned lt = (1u << lane) - 1u;
    if (t == 0) s_tile = atomicAdd(&tile_ctr[pass], 1u);
#pragma unroll
    for (int ww = 0; ww < kOsThreads / 32; ++ww) wcnt[ww][t] = 0u;
    // exclusive scan of this pass's global histogram: the digit's first slot
    {
        const uint32_t c = hist[pass * 256 + t];
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) sbase[w] = incl;
        __syncthreads();
        uint32_t off = 0;
        for (int ww = 0; ww < w; ++ww) off += sbase[ww];
        __syncthreads();
        sbase[t] = off + incl - c;
    }
    // a pass in which every key has the same digit keeps the order: copy
    const int trivial = __syncthreads_or(hist[pass * 256 + t] == (uint32_t)n);
    const uint32_t tile = s_tile;
    if (trivial) {
        for (int64_t i = (int64_t)tile * kOsTile + t; i < min(n, (int64_t)(tile + 1) * kOsTile); i += kOsThreads) {
            kout[i] = kin[i];
            vout[i] = vin[i];
        }
        return;
    }
    const int64_t base = (int64_t)tile * kOsTile + (int64_t)w * 32 * kOsItems;
    const int shift = 8 * pass;
    K key[kOsItems];
    uint32_t val[kOsItems], dig[kOsItems], rnk[kOsItems];
#pragma unroll
    for (int i = 0; i < kOsItems; ++i) {
        const int64_t idx = base + i * 32 + lane;
        const bool valid = idx < n;
        key[i] = valid ? kin[idx] : K(0);
        val[i] = valid ? vin[idx] : 0u;
        dig[i] = valid ? ((uint32_t)(key[i] >> shift) & 255u) : 256u;
    }
    // stable ranks within the warp's run of 32 * kOsItems keys
#pragma unroll
    for (int i = 0; i < kOsItems; ++i) {
        const unsigned peers = __match_any_sync(0xffffffffu, dig[i]);
        const uint32_t before = dig[i] < 256u ? wcnt[w][dig[i]] : 0u;
        rnk[i] = before + (uint32_t)__popc(peers & lt);
        __syncwarp();
        if (dig[i] < 256u && (peers & lt) == 0u) wcnt[w][dig[i]] = before + (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread t = digit t: warps' exclusive offsets, the tile's count, look-back
    uint32_t cnt = 0;
#pragma unroll
    for (int ww = 0; ww < kOsThreads / 32; ++ww) {
        const uint32_t c = wcnt[ww][t];
        wcnt[ww][t] = cnt;
        cnt += c;
    }
    const unsigned long long agg = (unsigned long long)(2 * pass + 1) << 32;
    const unsigned long long inc = (unsigned long long)(2 * pass + 2) << 32;
    unsigned long long* my = status + (int64_t)tile * 256 + t;
    uint32_t prefix = 0;
    if (tile == 0) {
        os_store(my, inc | cnt);
    } else {
        os_store(my, agg | cnt);
        // the walk reads kOsWin earlier tiles' words per round trip: their
        // own counts are summed down to the first tile with an inclusive count
        int64_t j = (int64_t)tile - 1;
        int spins = 0;
        bool done = false;
        while (!done) {
            unsigned long long wv[kOsWin];
#pragma unroll
            for (int u = 0; u < kOsWin; ++u) wv[u] = j - u >= 0 ? os_load(status + (j - u) * 256 + t) : inc;
            bool stop = false;
            int adv = 0;
#pragma unroll
            for (int u = 0; u < kOsWin; ++u) {
                if (stop) continue;
                const unsigned long long f = wv[u] & 0xffffffff00000000ull;
                if (f == inc) {
                    prefix += (uint32_t)wv[u];
                    done = stop = true;
                } else if (f == agg) {
                    prefix += (uint32_t)wv[u];
                    ++adv;
                } else {
                    stop = true;  // not published yet: read it again next round
                }
            }
            if (done) break;
            j -= adv;
            if (adv == 0) {
                if (++spins > kOsSpin) {
                    atomicOr(err, kErrSortWait);
                    break;
                }
                __nanosleep(32);
            }
        }
        os_store(my, inc | (prefix + cnt));
    }
    sbase[t] += prefix;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kOsItems; ++i) {
        if (dig[i] < 256u) {
            const uint32_t pos = sbase[dig[i]] + wcnt[w][dig[i]] + rnk[i];
            kout[pos] = key[i];
            vout[pos] = val[i];
        }
    }
}

template <typename K>
cudaError_t radix_sort_impl(const K* k_in, const uint32_t* v_in, K* k_out, uint32_t* v_out, K* k_tmp,
                            uint32_t* v_tmp, int64_t n, int nbits, void* temp, cudaStream_t st, unsigned int* err) {
    if (n <= 0) return cudaSuccess;
    const int passes = (nbits + 7) / 8;
    if (passes == 0) {
        cudaError_t e = cudaMemcpyAsync(k_out, k_in, n * sizeof(K), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(v_out, v_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    }
    const int64_t tiles = ceil_div(n, kOsTile);
    // temp: hist [8][256], tile counters [8], error word, pad, status [tiles][256]
    uint32_t* hist = reinterpret_cast<uint32_t*>(temp);
    uint32_t* tile_ctr = hist + kOsMaxPasses * 256;
    unsigned int* own_err = tile_ctr + kOsMaxPasses;
    unsigned long long* status = reinterpret_cast<unsigned long long*>(hist + kOsMaxPasses * 256 + 64);
    const size_t clear = (kOsMaxPasses * 256 + 64) * sizeof(uint32_t) + (size_t)tiles * 256 * sizeof(unsigned long long);
    cudaError_t e = cudaMemsetAsync(temp, 0, clear, st);
    if (e != cudaSuccess) return e;
    if (!err) err = own_err;
    const unsigned hb = (unsigned)std::min<int64_t>(ceil_div(n, 256 * 16), 152 * 8);
    (k_os_hist<K><<<hb, 256, 0, st>>>(k_in, n, passes, hist), note_launch());
    const K* src_k = k_in;
    const uint32_t* src_v = v_in;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        K* dk = to_out ? k_out : k_tmp;
        uint32_t* dv = to_out ? v_out : v_tmp;
        (k_os_pass<K><<<(unsigned)tiles, kOsThreads, 0, st>>>(src_k, src_v, dk, dv, n, p, hist, status, tile_ctr, err),
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
    const int64_t tiles = ceil_div(n > 0 ? n : 1, kOsTile);
    return (kOsMaxPasses * 256 + 64) * sizeof(uint32_t) + (size_t)tiles * 256 * sizeof(unsigned long long) + 256;
}

cudaError_t radix_sort_u64(const uint64_t* k_in, const uint32_t* v_in, uint64_t* k_out, uint32_t* v_out,
                           uint64_t* k_tmp, uint32_t* v_tmp, int64_t n, int nbits, void* temp,
                           cudaStream_t st, unsigned int* err) {
    return radix_sort_impl<uint64_t>(k_in, v_in, k_out, v_out, k_tmp, v_tmp, n, nbits, temp, st, err);
}

cudaError_t radix_sort_u32(const uint32_t* k_in, const uint32_t* v_in, uint32_t* k_out, uint32_t* v_out,
                           uint32_t* k_tmp, uint32_t* v_tmp, int64_t n, int nbits, void* temp,
                           cudaStream_t st, unsigned int* err) {
    return radix_sort_impl<uint32_t>(k_in, v_in, k_out, v_out, k_tmp, v_tmp, n, nbits, temp, st, err);
}

}  // namespace dpc
