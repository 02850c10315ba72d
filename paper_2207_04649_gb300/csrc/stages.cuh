// Device helpers and launchers shared by the rho, delta and label stages.
#pragma once
#include "dpc_internal.cuh"

namespace dpc {

constexpr int kSparseMax = 4;     // cells with at most this many points take the thread-per-cell path
constexpr int kQch = 128;         // queries per dense work item at most (4 per lane)
constexpr int kMaxNb = 81;        // neighbour cells per cell for R = 1, k <= 4

// Dense-cell work description produced by the cell preparation kernels.
struct CellWork {
    const uint32_t* dense;      // dense cell ids
    const uint32_t* ndense;     // device scalar
    const uint32_t* sparse;     // sparse cell ids
    const uint32_t* nsparse;    // device scalar
    const uint2* runs;          // [ncells * nbs] (start, count) of the non-empty neighbour cells of each cell
    const uint32_t* nruns;      // [ncells]
    const uint32_t* cand;       // [ncells] candidate points of each cell (sum of its runs)
    const uint4* items;         // (dense index, query chunk, candidate chunk, 0)
    const uint32_t* nitems;     // device scalar
    int kch;                    // candidates per dense work item
    int qch;                    // queries per dense work item (32, 64 or 128): a cell of m points is
                                // ceil(m / qch) query chunks, each its own warp's items
    int nbs;                    // run slots per cell: max over the batch of (2R+1)^k
    unsigned long long* stats;  // [0] candidate pairs of all cells
};

// Cell coordinate of a point along gridded dim j.
__device__ __forceinline__ int32_t cell_coord(const DsDesc& ds, int j, int32_t x) {
    // x >= origin (the dataset's minimum) and s < 2^31: unsigned 32-bit division
    return (int32_t)((uint32_t)(x - ds.origin[j]) / (uint32_t)ds.s);
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

// Bits of gridded dim j inside a Morton code of k dims x mbits bits.
__device__ __forceinline__ uint64_t morton_mask(int k, int mbits, int j) {
    uint64_t m = 0;
    for (int i = 0; i < mbits; ++i) m |= 1ull << (i * k + j);
    return m;
}

// Morton code with the coordinate held in the bits `mask` moved by delta in
// {-1, 0, +1} (the caller keeps the coordinate inside the grid): the carry or
// borrow runs through the dim's bits only.
__device__ __forceinline__ uint64_t morton_step(uint64_t code, uint64_t mask, int delta) {
    if (delta > 0) return (((code | ~mask) + 1) & mask) | (code & ~mask);
    if (delta < 0) return (((code & mask) - 1) & mask) | (code & ~mask);
    return code;
}

__device__ __forceinline__ int num_neighbours(const DsDesc& ds) {
    int w = 2 * ds.R + 1, t = 1;
    for (int j = 0; j < ds.k; ++j) t *= w;
    return t;
}

// Lane layout of a chunk of nq <= 128 queries: Q queries per lane, G groups
// of Mq lanes (Mq a power of two, Mq * G = 32), group g taking candidates
// g, g + G, ...; the layout wasting the fewest query slots, larger Q first.
__device__ __forceinline__ void lane_layout(int nq, int& Q, int& Mq) {
    int best = 1 << 30;
    Q = 1;
    Mq = 32;
    for (int q = 4; q >= 1; --q) {
        int m = 1;
        while (m * q < nq) m <<= 1;
        if (m > 32) continue;
        const int waste = m * q - nq;
        if (waste < best) {
            best = waste;
            Q = q;
            Mq = m;
        }
    }
}

// Candidate stream of one dense work item: the flat range [k0, k1) of the
// concatenated runs of a cell, delivered kChunk candidates at a time. prep()
// issues the loads of the next chunk into registers (lane l holds chunk
// slots l, l + 32, l + 64, l + 96), so that they are in flight while the
// warp works on the previous chunk; the caller then stores them to shared
// memory. All lanes call every method (warp-uniform control flow).
constexpr int kChunk = 128;

template <int DP, bool RO>
struct CandStream {
    const uint2* runs;   // the cell's runs, in shared memory
    uint32_t nr, ri, roff, remaining, cnt;
    int4 r[4][DP];
    uint2 ro[4];

    __device__ __forceinline__ void init(const uint2* runs_, uint32_t nr_, uint32_t k0, uint32_t k1) {
        runs = runs_;
        nr = nr_;
        ri = 0;
        roff = k0;
        remaining = k1 - k0;
        while (ri < nr) {
            const uint32_t len = runs[ri].y;
            if (roff < len) break;
            roff -= len;
            ++ri;
        }
    }

    // Returns false when the stream is exhausted; sets *bad when the runs end
    // before the counted candidates do (cannot happen when counts agree).
    __device__ __forceinline__ bool prep(int lane, const int4* __restrict__ recb, const uint2* __restrict__ ro_s,
                                         bool* bad) {
        if (remaining == 0u) return false;
        const uint32_t total = min((uint32_t)kChunk, remaining);
        int64_t src[4] = {-1, -1, -1, -1};
        uint32_t o = 0;
        while (o < total) {
            if (ri >= nr) {
                *bad = true;
                break;
            }
            const uint2 run = runs[ri];
            const uint32_t piece = min(run.y - roff, total - o);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t f = (uint32_t)lane + 32u * u;
                if (f >= o && f < o + piece) src[u] = (int64_t)run.x + roff + (f - o);
            }
            o += piece;
            roff += piece;
            if (roff == run.y) {
                ++ri;
                roff = 0;
            }
        }
        cnt = o;
        remaining -= total;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (src[u] >= 0) {
#pragma unroll
                for (int q = 0; q < DP; ++q) r[u][q] = __ldg(recb + src[u] * DP + q);
                if (RO) ro[u] = __ldg(ro_s + src[u]);
            }
        }
        return true;
    }
};

// Walk of a sparse cell's concatenated runs in steps of `step`: a lane that
// starts at offset `first` takes candidates first, first + step, ... of the
// flat list. The current run is held in registers; the walk loads a run
// only when it crosses into it, so a lane can find its next few candidates
// before any of their records arrive.
struct RunCursor {
    const uint2* runs;
    uint32_t nr, r, off;
    uint2 cur;

    __device__ __forceinline__ void init(const uint2* runs_, uint32_t nr_, uint32_t first) {
        runs = runs_;
        nr = nr_;
        r = 0;
        off = first;
        cur = nr_ > 0u ? runs_[0] : make_uint2(0u, 0u);
        settle();
    }
    __device__ __forceinline__ void settle() {
        while (r < nr && off >= cur.y) {
            off -= cur.y;
            if (++r < nr) cur = runs[r];
        }
    }
    // The sorted position of the lane's next candidate; false when none is left.
    __device__ __forceinline__ bool next(uint32_t step, uint32_t& p) {
        if (r >= nr) return false;
        p = cur.x + off;
        off += step;
        settle();
        return true;
    }
};

// ------------------------------------------------------------- launchers

// grid.cu
cudaError_t launch_minmax(const BatchView& v, int32_t* mm, cudaStream_t st);
cudaError_t launch_cell_keys(const BatchView& v, bool key32, void* keys, uint32_t* vals, cudaStream_t st);
// bflag, bidx, nblocks: null, or the block-start flags, their exclusive scan
// and the block count (device scalar) for the block table
cudaError_t launch_gather_cells(const BatchView& v, bool key32, const void* skeys, uint32_t* flag, uint32_t* cidx,
                                uint32_t* bflag, uint32_t* bidx, uint32_t* nblocks, void* scan_temp, cudaStream_t st);
// v.pos_of from v.perm (only the passes that need it allocate v.pos_of)
cudaError_t launch_pos_of(const BatchView& v, cudaStream_t st);
// The block table of the datasets with sbits > 0 (after k_cells; v.sbhash
// cleared to 0xff): keys, first cells and occupancy of every block, then
// the hash over them. bocc must be zeroed.
cudaError_t launch_blocks(const BatchView& v, const uint32_t* flag, const uint32_t* bflag, const uint32_t* bidx,
                          const uint32_t* nblocks, int64_t nblocks_bound, uint64_t* bkey, uint32_t* bfirst,
                          unsigned long long* bocc, cudaStream_t st);
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
    uint2* runs;          // [ncells * nbs]
    uint32_t* nruns;      // [ncells]
    uint32_t* cand;       // [ncells]
    uint32_t* nitem_c;    // [ndense_bound] items per dense cell
    uint32_t* item_off;   // [ndense_bound]
    uint4* items;         // [nitems_bound]
    uint32_t* nitems;     // scalar
    int nbs;
    int qch;              // queries per dense work item (CellWork::qch)
    unsigned long long* stats;  // [0] += candidate pairs
};
// Neighbour runs and candidate counts of every cell.
// kmask: bit K (1..4) = a dataset gridded in K dims with reach 1 that uses
// the cell hash is in the batch, bit 8 + K = one that uses the block table;
// bit 0 = one with another reach or no gridded dim.
cudaError_t launch_cell_runs(const BatchView& v, const CellPrepBufs& cb, int64_t ncells, uint32_t kmask,
                            cudaStream_t st);
// Dense and sparse cells (after the runs: a cell with more than sparse_cand
// candidates is dense whatever its size) and their candidate pairs.
cudaError_t launch_classify_cells(const BatchView& v, const CellPrepBufs& cb, int64_t ncells_bound,
                                  uint32_t sparse_cand, void* scan_temp, cudaStream_t st);
// Work items per dense cell and their offsets.
cudaError_t launch_item_prep(const BatchView& v, const CellPrepBufs& cb, int64_t ndense_bound, int kch,
                             void* scan_temp, cudaStream_t st);
cudaError_t launch_fill_items(const BatchView& v, const CellPrepBufs& cb, int64_t ndense_bound, int kch,
                              cudaStream_t st);
// class_mask bit 3*(d-1) + mode: a dataset of dimension d with density test
// mode `mode` (DsDesc::mode) is in the batch. counters: [24], zeroed.
cudaError_t launch_rho(const BatchView& v, const CellWork& w, uint32_t class_mask, int64_t nitems_bound,
                       int64_t nsparse_bound, uint32_t* counters, int parts, cudaStream_t st);
cudaError_t launch_rho_scatter(const BatchView& v, cudaStream_t st);
// the dense density kernels with the picks of each cell as its queries
// (plist[pstart[c] .. pstart[c + 1]), the points of cell c); w.items holds
// (cell, pick chunk, candidate chunk) items
cudaError_t launch_rho_picks(const BatchView& v, const CellWork& w, uint32_t class_mask, int64_t nitems_bound,
                             uint32_t* counters, const uint32_t* plist, const uint32_t* pstart, cudaStream_t st);

// delta.cu
struct DeltaBufs {
    uint32_t* rkeys;      // rank sort keys [N] (u32 or u64 storage)
    uint32_t* rvals;      // [N]
    uint32_t* ucount;     // [2] device counters: open list, brute-force list
    uint32_t* tree_list;  // [N] points open after the ring search
    uint8_t* ocode;       // ordered open lists: per point 0 resolved, 1 tree, 2 brute force (else null)
    uint32_t* ocnt;       // their per-block counts [2][blocks] (tree, brute force)
    uint32_t* oofs;       // and exclusive scans of those
    int lists_sorted;     // 1: tree_list is in position order already
    uint32_t* tclass;     // [9] or null: tree_list grouped by dimension, group d at [tclass[d-1], tclass[d])
    const uint32_t* tcount;  // count of the list the tree search reads
    uint32_t* bf_list;    // [N]
    int4* rrec;           // [N * 2] records in rank order (prefix only)
    uint32_t* rorig;      // [N]
    uint32_t bf_rank;     // points with rank below this go to the brute-force pass
    // Radix tree over the cells of every dataset (tree.cu). Leaf c is cell c;
    // internal node i (i in [first cell, last cell) of its dataset) is
    // indexed by global cell index too. Boxes: 2 * dpb int4 (lo, then hi).
    int dpb;              // int4 per box corner: 1 (all d <= 4) or 2
    int compact;          // 1 (all d <= 3): records of two int4, {lo, smallest rank}, {hi, link}; see tree.cu
    int64_t ncells;
    int64_t* cell_off;    // [B+1] first cell of each dataset
    uint64_t* ckey;       // [ncells] cell key
    int2* child;          // [ncells] children of internal node i: >= 0 internal, < 0 leaf ~c
    int32_t* iparent;     // [ncells] parent of internal node (-1: root)
    int32_t* lparent;     // [ncells] parent of leaf (-1: single-cell dataset)
    // Node records: internal node i at record i, leaf c at record ncells + c;
    // each 2 * dpb + 1 int4: box lo, box hi, then {smallest rank, left, right,
    // parent} for an internal node or {smallest rank, first point, end point,
    // parent} for a leaf (with leaf point lists: first and end list entry).
    // One record is one memory round trip in the search.
    int4* nodes;
    // Leaf point lists (null: a leaf holds its cell's points, a run of sorted
    // positions). S-Approx-DPC's pick path: leaf c holds the picks
    // lplist[lpstart[c] .. lpstart[c + 1]), the only points that can rank
    // above a pick.
    const uint32_t* lplist;
    const uint32_t* lpstart;
    uint32_t* flag;       // [ncells] refit arrival counters
    unsigned long long* stats;  // [0] tree nodes visited, [1] point pairs tested in leaves
    int key_bits;         // widest cell key of the batch's trees (bits; a tree is at most key_bits + 1 deep)
};
cudaError_t launch_rank(const BatchView& v, const DeltaBufs& db, int key_bits, void* sort_temp, cudaStream_t st);
cudaError_t launch_ring(const BatchView& v, const CellWork& w, uint32_t class_mask, int64_t nitems_bound,
                        int64_t nsparse_bound, uint32_t* counters, cudaStream_t st);
// ordered_temp (finalize_temp_bytes(N), or null): the open lists come out in
// position order (then the caller need not sort them)
size_t finalize_temp_bytes(int64_t n);
cudaError_t launch_finalize(const BatchView& v, DeltaBufs db, void* ordered_temp, cudaStream_t st);
// tree.cu: build (cell ranges, keys, radix tree, refit) and search
cudaError_t launch_tree_build(const BatchView& v, const DeltaBufs& db, cudaStream_t st);
// warp: 1 the warp-cooperative search, 0 one lane per open point, 2 the
// warp-cooperative search for d >= 5 only
cudaError_t launch_tree_search(const BatchView& v, const DeltaBufs& db, uint32_t dim_mask, int64_t bound,
                               int warp, cudaStream_t st);
cudaError_t launch_bruteforce(const BatchView& v, const DeltaBufs& db, uint32_t dim_mask, int64_t bound,
                              cudaStream_t st);

// approx.cu: Approx-DPC's dependent points (Section 4.3) on the grid of side
// d_cut / sqrt(d). The points are sorted again by that grid's keys; per cell
// the highest point (p*) and the lowest rank; rule 1 links every other point
// to its cell's p*; rule 2 links a p* to the highest p* of the neighbouring
// cells all of whose points rank higher; the rest go to the exact lists.
struct ApproxBufs {
    uint32_t* ord;        // [N] sorted positions in grid-key order
    uint32_t* flag;       // [N] temp: first point of a cell
    uint32_t* cidx;       // [N] temp: exclusive scan of flag
    uint32_t* cell_of;    // [N] grid cell of every sorted position
    uint32_t* start;      // [ncells + 1] first index (in ord) of every cell
    uint32_t* top;        // [ncells] sorted position of the cell's highest point
    uint32_t* maxrank;    // [ncells] the cell's lowest rank
    uint32_t* ncells;     // device scalar
    uint32_t* light;      // [ncells] cells whose p* has few candidates (one thread each)
    uint32_t* heavy;      // [ncells] the others (one warp each)
    uint32_t* nlh;        // [2] device counts of light, heavy
};
// Sorts the sorted positions by grid key (key_bits wide, the dataset index at
// bshift; keys [3N], ords [3N] scratch); *ord_out receives the key order.
cudaError_t launch_approx_keys(const BatchView& v, int key_bits, int bshift, uint64_t* keys, uint32_t* ords,
                               void* temp, uint32_t** ord_out, cudaStream_t st);
cudaError_t launch_approx_cells(const BatchView& v, const CellWork& w, const ApproxBufs& ab, int key_bits,
                                int bshift, void* scan_temp, cudaStream_t st);
cudaError_t launch_approx_rules(const BatchView& v, const CellWork& w, const ApproxBufs& ab, const DeltaBufs& db,
                                uint32_t dim_mask, int64_t ncells_bound, cudaStream_t st);

// sapprox.cu: S-Approx-DPC (Section 5). Keys, orders and flags are over the
// cells of the finer grid G' (side max(1, floor(eps d_cut / sqrt(d)))).
struct SapproxBufs {
    uint64_t* keys;       // [3N] one 64-bit word of the key of G' per pass; sort input, output, scratch
    uint32_t* ord;        // [3N] original global indices in key order (three rotating buffers)
    uint32_t* flag;       // [N] first point of a cell of G' in key order
    uint32_t* cidx;       // [N] exclusive scan of flag
    uint32_t* picks;      // [N] sorted position of the pick of every cell of G'
    uint32_t* pick_s;     // [N] sorted position -> sorted position of its cell's pick
    uint32_t* npicks;     // device scalar: cells of G'
    uint32_t* pflag;      // [N] pick path: 1 at the sorted position of a pick
    uint32_t* ppos;       // [N] pick path: exclusive scan of pflag
    uint32_t* plist;      // [N] pick path: the picks in sorted order (each cell's together)
    uint32_t* pstart;     // [ncells + 1] pick path: first entry of every exact-grid cell in plist
    uint32_t* scan;       // [N] picks that scan their neighbourhood for the first phase
    uint32_t* nscan;      // device scalar: their count
    unsigned long long* stats;  // [3] pairs the pick-only density pass evaluates; picks reaching the second
                                //     phase; candidate pairs of the picks (before choosing the path)
};
// key_bits: width of the key of G'; bshift: bit offset of the dataset index
cudaError_t launch_sapprox_grid(const BatchView& v, const SapproxBufs& sb, int key_bits, int bshift, void* temp,
                                cudaStream_t st);
// The picks of every exact-grid cell (plist, pstart), for the pick path
cudaError_t launch_sapprox_plist(const BatchView& v, const SapproxBufs& sb, int64_t ncells, void* temp,
                                 cudaStream_t st);
// sb.stats[2] += the candidate pairs of the picks' exact-grid cells
cudaError_t launch_sapprox_pick_pairs(const BatchView& v, const CellWork& w, const SapproxBufs& sb,
                                     int64_t picks_bound, cudaStream_t st);
// by_cell: one warp per exact-grid cell over its picks (needs plist, pstart),
// else one warp per pick
// items of launch_rho_picks for every cell holding picks; cap bounds their number
cudaError_t launch_sapprox_items(const BatchView& v, const CellWork& w, const SapproxBufs& sb, int64_t ncells, int kch,
                                 uint32_t* nitem_c, uint32_t* item_off, uint4* items, uint32_t* nitems, int64_t cap,
                                 void* temp, cudaStream_t st);
cudaError_t launch_sapprox_rho(const BatchView& v, const CellWork& w, const SapproxBufs& sb, uint32_t dim_mask,
                               int64_t picks_bound, int64_t ncells, bool by_cell, cudaStream_t st);
// rho 0 for the points that are not picked (they rank after every pick)
cudaError_t launch_sapprox_mask(const BatchView& v, cudaStream_t st);
// after the rank and the ring search: the points that are not picked, then
// the picks (resolved from the ring result or queued), then the first-phase scan
// near_pass: the pick path's pass over the picks of each block (no ring search
// ran), one thread (near_threads) or one warp per pick
cudaError_t launch_sapprox_first(const BatchView& v, const CellWork& w, const SapproxBufs& sb, const DeltaBufs& db,
                                 uint32_t dim_mask, int64_t picks_bound, int64_t scan_bound, bool near_pass,
                                 bool near_threads, cudaStream_t st);
cudaError_t launch_sapprox_rho_out(const BatchView& v, int32_t* out, cudaStream_t st);

// label.cu
cudaError_t launch_labels(const BatchView& v, cudaStream_t st);
// labels of dataset b only (its points [g0, g0 + n)); the other datasets'
// labels and center counts are left as they are
cudaError_t launch_labels_one(const BatchView& v, int b, int64_t g0, int64_t n, cudaStream_t st);
// The outputs of the device-resident jobs of a batch (null pointers skipped):
// job j's n points are the batch's [src_off, src_off + n) and the
// concatenation's [dst_off, dst_off + n) (dst_off ascending)
struct OutJob {
    int64_t src_off, dst_off, n;
    int32_t* rho;
    int32_t* dep;
    int64_t* delta2;
    uint8_t* aux;
    int32_t* label;  // [nq * n], query-major
    int32_t nq;
};
cudaError_t launch_job_outputs(const OutJob* jobs, int J, int64_t total, const int32_t* rho, const int32_t* dep,
                               const int64_t* delta2, const uint8_t* aux, const int32_t* label, int what, int q,
                               cudaStream_t st);
// The inputs the device can read (device or page-locked host memory): job j's
// points (len = n d ints at src) into dst[dst_off .. dst_off + len) (dst_off
// ascending; the ints of dst in no job's range, of total, are not written)
struct InJob {
    const int32_t* src;
    int64_t dst_off, len;
};
cudaError_t launch_job_inputs(const InJob* jobs, int J, int64_t total, int32_t* dst, cudaStream_t st);

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace dpc
