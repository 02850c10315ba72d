// Internal declarations shared by the CUDA translation units of libdpc.
//
// Exact Density-Peaks Clustering (the paper's Section 2.1, Definitions 1-6)
// on one GPU. Every stage works on a *batch* of independent datasets laid
// out back to back; the plain one-dataset path is a batch of one.
//
// Index spaces of a batch with N = sum of n_b points:
//   g  "original" global index: dataset b owns [pt_off_b, pt_off_b + n_b)
//      in the caller's point order.
//   p  "sorted" global index: the same range of dataset b after the points
//      are sorted by grid cell (Morton order of the cells).
// perm[p] = g and pos_of[g] = p map between them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dpc {

constexpr int kMaxDims = 8;
constexpr int kMaxGridDims = 4;
constexpr uint64_t kEmptyKey = ~0ull;

// Per-dataset description, shared by host and device.
struct DsDesc {
    int64_t pt_off;       // first global index (both index spaces)
    int64_t rec_off;      // first int4 record of the sorted points
    int64_t in_off;       // first int32 of the input points (row-major n x d)
    int64_t d_cut;
    int64_t d_cut2;       // d_cut^2
    int64_t s;            // grid cell side
    uint64_t cbase;       // cell-key base of this dataset
    int64_t rho_min;      // label query
    int64_t delta_min2;   // delta_min^2
    int32_t n, d;
    int32_t dp;           // int4 records per point: 1 (d <= 4) or 2 (d <= 8)
    int32_t k;            // gridded dims
    int32_t gdim[kMaxGridDims];    // coordinate of each gridded dim
    int32_t origin[kMaxGridDims];  // smallest coordinate per gridded dim
    int32_t ext[kMaxGridDims];     // cells per gridded dim
    int32_t mbits;        // Morton bits per gridded dim
    int32_t R;            // neighbour reach in cells
    int32_t w32;          // all candidate pair sums fit 31 bits
    int32_t mode;         // density pair test: 0 direct 32-bit, 1 direct 64-bit,
                          // 2 expanded 32-bit, |c|^2 + |q|^2 - T - 2 q.c wrapping mod 2^32 (d <= 4)
    int32_t lo[kMaxDims]; // smallest coordinate per dim
    int32_t rbits;        // bits of the density key in the rank sort
    uint64_t dmask[kMaxGridDims];  // Morton bits of each gridded dim
    int32_t a_side;       // Approx-DPC grid: integer side max(1, floor(d_cut / sqrt(d)));
                          // S-Approx-DPC grid: max(1, floor(eps d_cut / sqrt(d))), at most 2^30
    int32_t a_shift[kMaxDims];  // Approx-DPC grid: bit offset of each dim's cell coordinate in the key
    int32_t prune;        // 1: the neighbour runs may leave out in-reach cells whose box is at least
                          // d_cut away (no point there counts in rho, but one may be nearer than the
                          // searched block's outside for the dependent-point search)
    int32_t span[kMaxDims];  // largest - smallest coordinate + 1 per dim
    int32_t sbits;        // bits of a block's local Morton code in the block table (a block is 2^(sbits / k)
                          // cells per gridded dim); 0: this dataset's neighbour runs use the cell hash
};

// Device views of a batch's buffers (all device pointers).
struct BatchView {
    int32_t B;
    int64_t N;
    const DsDesc* desc;        // [B]
    const int64_t* pt_off;     // [B+1]
    // input and sorted points
    const int32_t* in;         // input points, row-major per dataset
    int4* rec;                 // sorted records (dp int4 per point)
    uint32_t* perm;            // p -> g
    uint32_t* pos_of;          // g -> p (S-Approx-DPC only, else null)
    // grid
    uint64_t* key;             // cell key per sorted point
    uint32_t* cell_start;      // [ncells + 1]
    uint32_t* cell_of;         // sorted: cell of each point
    uint32_t* ncells;          // device scalar
    int4* hash;                // open addressing: {key lo, key hi, start, count}
    uint64_t hmask;
    // block table: aligned blocks of 2^(sbits / k) cells per gridded dim,
    // open addressing over the non-empty blocks; slot = two int4:
    // {key lo, key hi, first cell, 0}, {occupancy lo, occupancy hi, 0, 0}
    int4* sbhash;
    uint64_t sbmask;
    // rho
    int32_t* rho_s;            // sorted
    int32_t* rho;              // original
    // rank
    uint32_t* rank;            // original: position in (rho desc, index asc) within its dataset
    uint32_t* order;           // global rank order: order[pt_off_b + r] = g
    uint2* ro_s;               // sorted: (rank, original local index)
    // delta
    unsigned long long* best_s;  // sorted: packed (min(D, 2^32-1) << 32 | orig local)
    int32_t* dep;              // original: dependent point (local index), -1 top
    int64_t* delta2;           // original
    // labels
    int32_t* parent;           // original, global
    int32_t* label;            // original, local
    uint8_t* exact;            // original: 1 when the dependent point is exact (Approx-DPC)
    uint8_t* pick;             // original: 1 for the picked points of S-Approx-DPC; NULL on other paths
    unsigned long long* ncent; // [B]
    unsigned int* err;         // device error word: kErr* bits set by guarded kernels
};

// Bits of BatchView::err. A guard that trips leaves its output wrong but
// bounded; the host turns a nonzero word into DPC_ERR_CUDA.
constexpr unsigned kErrStaging = 1u;   // candidate runs shorter than counted
constexpr unsigned kErrTreeStack = 2u; // tree search stack full
constexpr unsigned kErrChain = 4u;     // label chain longer than the dataset
constexpr unsigned kErrBulkWait = 8u;  // a bulk copy into shared memory did not complete in time

// ---------------------------------------------------------------- helpers

__host__ __device__ inline uint64_t mix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// Morton code of k cell coordinates with mbits bits each: bit i of dim j
// lands at position i * k + j.
__host__ __device__ inline uint64_t morton(const int32_t* c, int k, int mbits) {
    uint64_t code = 0;
    for (int i = 0; i < mbits; ++i)
        for (int j = 0; j < k; ++j)
            code |= (uint64_t)((c[j] >> i) & 1) << (i * k + j);
    return code;
}

// The same Morton code by bit spreading, for k <= 4 gridded dims whose
// codes fit 40 bits (at most 40, 20, 13 and 10 bits per dim for k = 1..4).
__host__ __device__ inline uint64_t spread2(uint64_t x) {
    x &= 0xffffffffull;
    x = (x | (x << 16)) & 0x0000ffff0000ffffull;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    return (x | (x << 1)) & 0x5555555555555555ull;
}
__host__ __device__ inline uint64_t spread3(uint64_t x) {
    x &= 0x1fffffull;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    return (x | (x << 2)) & 0x1249249249249249ull;
}
__host__ __device__ inline uint64_t spread4(uint64_t x) {
    x &= 0xffffull;
    x = (x | (x << 24)) & 0x000000ff000000ffull;
    x = (x | (x << 12)) & 0x000f000f000f000full;
    x = (x | (x << 6)) & 0x0303030303030303ull;
    return (x | (x << 3)) & 0x1111111111111111ull;
}
__host__ __device__ inline uint64_t morton_k(const int32_t* c, int k) {
    switch (k) {
        case 1: return (uint64_t)(uint32_t)c[0];
        case 2: return spread2((uint32_t)c[0]) | (spread2((uint32_t)c[1]) << 1);
        case 3: return spread3((uint32_t)c[0]) | (spread3((uint32_t)c[1]) << 1) | (spread3((uint32_t)c[2]) << 2);
        case 4:
            return spread4((uint32_t)c[0]) | (spread4((uint32_t)c[1]) << 1) | (spread4((uint32_t)c[2]) << 2) |
                   (spread4((uint32_t)c[3]) << 3);
        default: return 0;
    }
}

__device__ inline int find_ds(const int64_t* pt_off, int B, int64_t g) {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pt_off[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Key of the block of cell key `key` of dataset b in the block table.
__host__ __device__ inline uint64_t block_key(int b, uint64_t key, uint64_t cbase, int sbits) {
    return ((uint64_t)b << 40) | ((key - cbase) >> sbits);
}

// Block table lookup: the block's first cell (in the sorted cell order) and
// its occupancy bitmap (bit i: the cell with local Morton code i is not
// empty); occupancy 0 when the block is empty.
__device__ inline uint32_t block_find(const int4* __restrict__ table, uint64_t mask, uint64_t key,
                                      unsigned long long& occ) {
    uint64_t h = mix64(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        const int4 e = __ldg(&table[2 * h]);
        const int4 m = __ldg(&table[2 * h + 1]);  // same 32-byte sector
        const uint64_t k = (uint64_t)(uint32_t)e.x | ((uint64_t)(uint32_t)e.y << 32);
        if (k == key) {
            occ = (unsigned long long)(uint32_t)m.x | ((unsigned long long)(uint32_t)m.y << 32);
            return (uint32_t)e.z;
        }
        if (k == kEmptyKey) break;
        h = (h + 1) & mask;
    }
    occ = 0ull;
    return 0u;
}

// Hash lookup of a cell key: returns (start, count) or count 0.
__device__ inline uint2 hash_find(const int4* __restrict__ table, uint64_t mask, uint64_t key) {
    uint64_t h = mix64(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        int4 e = __ldg(&table[h]);
        uint64_t k = (uint64_t)(uint32_t)e.x | ((uint64_t)(uint32_t)e.y << 32);
        if (k == key) return make_uint2((uint32_t)e.z, (uint32_t)e.w);
        if (k == kEmptyKey) break;
        h = (h + 1) & mask;
    }
    return make_uint2(0u, 0u);
}

// --------------------------------------------------------- launch helpers

// Count of kernel launches made by this library (all threads).
void note_launch();
long long launch_count();

// sort.cu
size_t radix_sort_temp_bytes(int64_t n);
// Stable LSD radix sort of (key, value) pairs on bits [0, nbits), 8-bit
// digits (per pass: tile counts, a scan, a stable scatter). On return the
// sorted data is in (k_out, v_out).
cudaError_t radix_sort_u64(const uint64_t* k_in, const uint32_t* v_in, uint64_t* k_out, uint32_t* v_out,
                           uint64_t* k_tmp, uint32_t* v_tmp, int64_t n, int nbits, void* temp,
                           cudaStream_t st);
cudaError_t radix_sort_u32(const uint32_t* k_in, const uint32_t* v_in, uint32_t* k_out, uint32_t* v_out,
                           uint32_t* k_tmp, uint32_t* v_tmp, int64_t n, int nbits, void* temp,
                           cudaStream_t st);
size_t scan_temp_bytes(int64_t n);
// Exclusive prefix sum of n uint32 values; writes the total to *total (device) if non-null.
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, void* temp,
                               cudaStream_t st);

}  // namespace dpc
