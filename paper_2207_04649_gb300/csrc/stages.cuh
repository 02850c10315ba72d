// Device helpers and launchers shared by the rho, delta and label stages.
#pragma once
#include "dpc_internal.cuh"

namespace dpc {

constexpr int kSparseMax = 4;     // cells with at most this many points take the thread-per-cell path
constexpr int kQch = 128;         // queries per dense work item (4 per lane)
constexpr int kMaxNb = 81;        // neighbour cells per cell for R = 1, k <= 4

// Dense-cell work description produced by the cell preparation kernels.
struct CellWork {
    const uint32_t* dense;      // dense cell ids
    const uint32_t* ndense;     // device scalar
    const uint32_t* sparse;     // sparse cell ids
    const uint32_t* nsparse;    // device scalar
    const uint2* runs;          // [ndense * kMaxNb] (start, count) of non-empty neighbour cells
    const uint32_t* nruns;      // [ndense]
    const uint32_t* cand;       // [ndense] candidate points per dense cell
    const uint4* items;         // (dense index, query chunk, candidate chunk, 0)
    const uint32_t* nitems;     // device scalar
    int kch;                    // candidates per dense work item
    unsigned long long* stats;  // [0] dense, [1] sparse candidate pairs
};

// Cell coordinate of a point along gridded dim j.
__device__ __forceinline__ int32_t cell_coord(const DsDesc& ds, int j, int32_t x) {
    return (int32_t)(((int64_t)x - ds.origin[j]) / ds.s);
}

// Coordinate k of the point whose first record is r.
__device__ __forceinline__ int32_t rec_coord(const int4* r, int k) {
    const int4 v = r[k >> 2];
    switch (k & 3) {
        case 0: return v.x;
        case 1: return v.y;
        case 2: return v.z;
        default: return v.w;
    }
}

// Neighbour number t in [0, (2R+1)^k) of cell c: writes its coordinates
// and returns false when it falls outside the grid or when its box is at
// least d_cut away from c's box (it can hold no point within d_cut).
__device__ __forceinline__ bool neighbour(const DsDesc& ds, const int32_t* c, int t, int32_t* nc) {
    const int w = 2 * ds.R + 1;
    int64_t gap2 = 0;
    for (int j = 0; j < ds.k; ++j) {
        const int o = t % w - ds.R;
        t /= w;
        nc[j] = c[j] + o;
        if (nc[j] < 0 || nc[j] >= ds.ext[j]) return false;
        const int ao = o < 0 ? -o : o;
        if (ao > 0) {
            const int64_t gap = (int64_t)(ao - 1) * ds.s + 1;
            gap2 += gap * gap;
        }
    }
    return gap2 < ds.d_cut2;
}

__device__ __forceinline__ int num_neighbours(const DsDesc& ds) {
    int w = 2 * ds.R + 1, t = 1;
    for (int j = 0; j < ds.k; ++j) t *= w;
    return t;
}

// ------------------------------------------------------------- launchers

// grid.cu
cudaError_t launch_minmax(const BatchView& v, int32_t* mm, cudaStream_t st);
cudaError_t launch_cell_keys(const BatchView& v, bool key32, void* keys, uint32_t* vals, cudaStream_t st);
cudaError_t launch_gather_cells(const BatchView& v, bool key32, const void* skeys, uint32_t* flag, uint32_t* cidx,
                                void* scan_temp, cudaStream_t st);
cudaError_t launch_hash_insert(const BatchView& v, int64_t ncells_bound, cudaStream_t st);

// rho.cu
struct CellPrepBufs {
    uint32_t* dflag;      // [ncells_bound] temp
    uint32_t* sflag;      // [ncells_bound] temp
    uint32_t* didx;       // [ncells_bound] temp
    uint32_t* sidx;       // [ncells_bound] temp
    uint32_t* dense;      // [ncells_bound]
    uint32_t* sparse;     // [ncells_bound]
    uint32_t* ndense;     // scalar
    uint32_t* nsparse;    // scalar
    uint2* runs;          // [ndense_bound * kMaxNb]
    uint32_t* nruns;      // [ndense_bound]
    uint32_t* cand;       // [ndense_bound]
    uint32_t* nitem_c;    // [ndense_bound] items per dense cell
    uint32_t* item_off;   // [ndense_bound]
    uint4* items;         // [nitems_bound]
    uint32_t* nitems;     // scalar
    unsigned long long* stats;  // [0] += dense candidate pairs
};
cudaError_t launch_classify_cells(const BatchView& v, const CellPrepBufs& cb, int64_t ncells_bound, void* scan_temp,
                                  cudaStream_t st);
cudaError_t launch_dense_prep(const BatchView& v, const CellPrepBufs& cb, int64_t ndense_bound, int kch,
                              void* scan_temp, cudaStream_t st);
cudaError_t launch_fill_items(const BatchView& v, const CellPrepBufs& cb, int64_t ndense_bound, int kch,
                              cudaStream_t st);
// class_mask bit 2*(d-1) + wide: a dataset of dimension d with 32-bit (wide = 0)
// or 64-bit (wide = 1) pair arithmetic is in the batch. counters: [16], zeroed.
cudaError_t launch_rho(const BatchView& v, const CellWork& w, uint32_t class_mask, int64_t nitems_bound,
                       int64_t nsparse_bound, uint32_t* counters, cudaStream_t st);
cudaError_t launch_rho_scatter(const BatchView& v, cudaStream_t st);

// delta.cu
struct DeltaBufs {
    uint32_t* rkeys;      // rank sort keys [N] (u32 or u64 storage)
    uint32_t* rvals;      // [N]
    uint32_t* ucount;     // [2] device counters: tree list, brute list
    uint32_t* tree_list;  // [N]
    uint32_t* bf_list;    // [N]
    uint32_t* bf_keys;    // [N]
    uint32_t* bf_sorted;  // [N]
    int4* rrec;           // [N * 2] records in rank order (prefix only)
    uint32_t* rorig;      // [N]
    int4* node_box;       // [nodes * 4] lo[2], hi[2]
    uint32_t* node_minrank;  // [nodes]
    uint32_t* node_flag;  // [nodes]
    int64_t nodes;
    int64_t leaf_slots;
    const int64_t* slot_off;   // [B+1] leaf-slot prefix per dataset (device)
    uint32_t bf_rank;     // points with rank below this go to the brute-force pass
};
cudaError_t launch_rank(const BatchView& v, const DeltaBufs& db, int key_bits, void* sort_temp, cudaStream_t st);
cudaError_t launch_ring(const BatchView& v, const CellWork& w, uint32_t class_mask, int64_t nitems_bound,
                        int64_t nsparse_bound, uint32_t* counters, cudaStream_t st);
cudaError_t launch_finalize(const BatchView& v, const DeltaBufs& db, cudaStream_t st);
cudaError_t launch_tree_build(const BatchView& v, const DeltaBufs& db, cudaStream_t st);
cudaError_t launch_tree_search(const BatchView& v, const DeltaBufs& db, uint32_t dim_mask, int64_t bound,
                               cudaStream_t st);
cudaError_t launch_bruteforce(const BatchView& v, const DeltaBufs& db, uint32_t dim_mask, int64_t bound,
                              void* sort_temp, cudaStream_t st);

// label.cu
cudaError_t launch_labels(const BatchView& v, cudaStream_t st);

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace dpc
