// Uniform grid over the points of every dataset in a batch.
//
// The grid is the filter behind the local density (Definition 1): a point
// within d_cut of p_i lies in p_i's cell or in a cell at most R cells away
// in every gridded dimension (R = 1 when the cell side is d_cut). It plays
// the role of the paper's grid G of Approx-DPC (Section 4.1: non-empty cells
// only, built online from the data), with cell side d_cut instead of
// d_cut / sqrt(d), and replaces Ex-DPC's kd-tree range search (Section 3).
//
// Build: per-dataset bounding box -> cell key per point (Morton code of the
// cell coordinates, offset by the dataset's key base) -> stable radix sort
// of (key, index) -> gather of the int32 coordinates into sorted, padded
// int4 records -> run boundaries -> cell table -> hash of key -> (start, count).
#include "dpc_internal.cuh"
#include <algorithm>

namespace dpc {

namespace {

__global__ void k_minmax_init(int32_t* mm, int B) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B * kMaxDims) {
        mm[2 * i] = INT32_MAX;
        mm[2 * i + 1] = INT32_MIN;
    }
}

constexpr int kMmItems = 8;  // points per thread in the bounding-box pass

// Per-dataset, per-dimension min and max of the input coordinates. Each
// block reduces its points of the dataset its first point belongs to in
// registers, then warp shuffles, then shared memory, and issues one global
// atomic per dimension; points of a following dataset (blocks straddling a
// boundary) go to global atomics directly.
__global__ void __launch_bounds__(256) k_minmax(BatchView v, int32_t* __restrict__ mm) {
    __shared__ int smin[kMaxDims], smax[kMaxDims];
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * kMmItems;
    if (base >= v.N) return;  // uniform across the block
    const int b0 = find_ds(v.pt_off, v.B, base);
    const DsDesc& d0 = v.desc[b0];
    const int64_t end0 = v.pt_off[b0 + 1];
    if (threadIdx.x < kMaxDims) {
        smin[threadIdx.x] = INT32_MAX;
        smax[threadIdx.x] = INT32_MIN;
    }
    __syncthreads();
    int lo[kMaxDims], hi[kMaxDims];
#pragma unroll
    for (int k = 0; k < kMaxDims; ++k) {
        lo[k] = INT32_MAX;
        hi[k] = INT32_MIN;
    }
    for (int it = 0; it < kMmItems; ++it) {
        const int64_t g = base + (int64_t)it * blockDim.x + threadIdx.x;
        if (g >= v.N) break;
        if (g < end0) {
            const int32_t* x = v.in + d0.in_off + (g - d0.pt_off) * d0.d;
#pragma unroll
            for (int k = 0; k < kMaxDims; ++k)
                if (k < d0.d) {
                    lo[k] = min(lo[k], x[k]);
                    hi[k] = max(hi[k], x[k]);
                }
        } else {
            const int b = find_ds(v.pt_off, v.B, g);
            const DsDesc& ds = v.desc[b];
            const int32_t* x = v.in + ds.in_off + (g - ds.pt_off) * ds.d;
            for (int k = 0; k < ds.d; ++k) {
                atomicMin(&mm[(b * kMaxDims + k) * 2], x[k]);
                atomicMax(&mm[(b * kMaxDims + k) * 2 + 1], x[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kMaxDims; ++k) {
        if (k >= d0.d) break;
        int l = lo[k], h = hi[k];
        for (int o = 16; o > 0; o >>= 1) {
            l = min(l, __shfl_xor_sync(0xffffffffu, l, o));
            h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&smin[k], l);
            atomicMax(&smax[k], h);
        }
    }
    __syncthreads();
    if (threadIdx.x < d0.d) {
        atomicMin(&mm[(b0 * kMaxDims + threadIdx.x) * 2], smin[threadIdx.x]);
        atomicMax(&mm[(b0 * kMaxDims + threadIdx.x) * 2 + 1], smax[threadIdx.x]);
    }
}

// Cell key of every input point: key base of its dataset + Morton code of
// its cell coordinates in the gridded dimensions.
template <typename K>
__global__ void k_cell_keys(BatchView v, K* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= v.N) return;
    const int b = find_ds(v.pt_off, v.B, g);
    const DsDesc& ds = v.desc[b];
    const int32_t* x = v.in + ds.in_off + (g - ds.pt_off) * ds.d;
    int32_t c[kMaxGridDims] = {0, 0, 0, 0};
    const int k = ds.k;
    const uint32_t sd = (uint32_t)ds.s;
#pragma unroll
    for (int j = 0; j < kMaxGridDims; ++j)
        if (j < k) c[j] = (int32_t)((uint32_t)(x[ds.gdim[j]] - ds.origin[j]) / sd);
    keys[g] = (K)(ds.cbase + morton_k(c, k));
    vals[g] = (uint32_t)g;
}

// Sorted records (dp int4 per point, zero-padded), inverse permutation,
// cell-start flags and (bflag non-null) block-start flags of the datasets
// that use the block table.
template <typename K>
__global__ void k_gather(BatchView v, const K* __restrict__ skeys, uint32_t* __restrict__ flag,
                         uint32_t* __restrict__ bflag) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const int b = find_ds(v.pt_off, v.B, p);
    const DsDesc& ds = v.desc[b];
    const uint32_t g = v.perm[p];
    const int32_t* x = v.in + ds.in_off + ((int64_t)g - ds.pt_off) * ds.d;
    int32_t c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = k < ds.d ? x[k] : 0;
    int4* r = v.rec + ds.rec_off + (p - ds.pt_off) * ds.dp;
    // the expanded pair form keeps |x|^2 mod 2^32 in the w lane for d <= 3
    // (4-d records have no spare lane: the kernels compute it when staging)
    if (ds.mode == 2 && ds.d <= 3)
        c[3] = (int32_t)((uint32_t)c[0] * (uint32_t)c[0] + (uint32_t)c[1] * (uint32_t)c[1] +
                         (uint32_t)c[2] * (uint32_t)c[2]);
    r[0] = make_int4(c[0], c[1], c[2], c[3]);
    if (ds.dp == 2) r[1] = make_int4(c[4], c[5], c[6], c[7]);
    v.key[p] = (uint64_t)skeys[p];
    const bool first = p == 0 || p == ds.pt_off;
    flag[p] = (first || skeys[p] != skeys[p - 1]) ? 1u : 0u;
    if (bflag)
        bflag[p] = ds.sbits > 0 && (first || (((uint64_t)skeys[p] - ds.cbase) >> ds.sbits) !=
                                                 (((uint64_t)skeys[p - 1] - ds.cbase) >> ds.sbits))
                       ? 1u
                       : 0u;
}

__global__ void k_cells(BatchView v, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ cidx) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    if (flag[p]) v.cell_start[cidx[p]] = (uint32_t)p;
    v.cell_of[p] = cidx[p] + flag[p] - 1u;
    if (p == v.N - 1) {
        const uint32_t nc = cidx[p] + flag[p];
        v.cell_start[nc] = (uint32_t)v.N;
        *v.ncells = nc;
    }
}

// Blocks of the block table (after k_cells): every block's key and first
// cell, and its occupancy bitmap (one bit per non-empty cell, at the cell's
// local Morton code).
__global__ void k_blocks_fill(BatchView v, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ bflag,
                              const uint32_t* __restrict__ bidx, uint64_t* __restrict__ bkey,
                              uint32_t* __restrict__ bfirst, unsigned long long* __restrict__ bocc) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N || !flag[p]) return;  // one thread per non-empty cell
    const int b = find_ds(v.pt_off, v.B, p);
    const DsDesc& ds = v.desc[b];
    if (ds.sbits == 0) return;
    const uint64_t key = v.key[p];
    const uint32_t s = bidx[p] + bflag[p] - 1u;  // the block holding p
    if (bflag[p]) {
        bkey[s] = block_key(b, key, ds.cbase, ds.sbits);
        bfirst[s] = v.cell_of[p];
    }
    atomicOr(&bocc[s], 1ull << ((key - ds.cbase) & ((1ull << ds.sbits) - 1ull)));
}

__global__ void k_blocks_insert(BatchView v, const uint32_t* __restrict__ nblocks, const uint64_t* __restrict__ bkey,
                                const uint32_t* __restrict__ bfirst, const unsigned long long* __restrict__ bocc) {
    const uint32_t nb = *nblocks;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nb; s += gridDim.x * blockDim.x) {
        const uint64_t key = bkey[s];
        uint64_t h = mix64(key) & v.sbmask;
        for (uint64_t probe = 0; probe <= v.sbmask; ++probe) {
            unsigned long long* slot = reinterpret_cast<unsigned long long*>(&v.sbhash[2 * h]);
            if (atomicCAS(slot, (unsigned long long)kEmptyKey, (unsigned long long)key) == kEmptyKey) {
                v.sbhash[2 * h].z = (int)bfirst[s];
                const unsigned long long o = bocc[s];
                v.sbhash[2 * h + 1] = make_int4((int)(uint32_t)o, (int)(uint32_t)(o >> 32), 0, 0);
                break;
            }
            h = (h + 1) & v.sbmask;
        }
    }
}

__global__ void k_hash_insert(BatchView v) {
    const uint32_t nc = *v.ncells;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const uint32_t st = v.cell_start[c], cnt = v.cell_start[c + 1] - st;
        const uint64_t key = v.key[st];
        uint64_t h = mix64(key) & v.hmask;
        for (uint64_t probe = 0; probe <= v.hmask; ++probe) {
            unsigned long long* slot = reinterpret_cast<unsigned long long*>(&v.hash[h]);
            unsigned long long old = atomicCAS(slot, (unsigned long long)kEmptyKey, (unsigned long long)key);
            if (old == kEmptyKey) {
                v.hash[h].z = (int)st;
                v.hash[h].w = (int)cnt;
                break;
            }
            h = (h + 1) & v.hmask;
        }
    }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_minmax(const BatchView& v, int32_t* mm, cudaStream_t st) {
    (k_minmax_init<<<blocks_for((int64_t)v.B * kMaxDims, 256), 256, 0, st>>>(mm, v.B), note_launch());
    if (v.N > 0) (k_minmax<<<blocks_for(v.N, 256 * kMmItems), 256, 0, st>>>(v, mm), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_cell_keys(const BatchView& v, bool key32, void* keys, uint32_t* vals, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    if (key32)
        (k_cell_keys<uint32_t><<<blocks_for(v.N, 256), 256, 0, st>>>(v, (uint32_t*)keys, vals), note_launch());
    else
        (k_cell_keys<uint64_t><<<blocks_for(v.N, 256), 256, 0, st>>>(v, (uint64_t*)keys, vals), note_launch());
    return cudaGetLastError();
}

// Inverse of the sort permutation (pos_of[perm[p]] = p), for the passes
// that start from original indices (S-Approx-DPC's grid G').
__global__ void k_pos_of(BatchView v) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    v.pos_of[v.perm[p]] = (uint32_t)p;
}

cudaError_t launch_pos_of(const BatchView& v, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    (k_pos_of<<<blocks_for(v.N, 256), 256, 0, st>>>(v), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_gather_cells(const BatchView& v, bool key32, const void* skeys, uint32_t* flag, uint32_t* cidx,
                                uint32_t* bflag, uint32_t* bidx, uint32_t* nblocks, void* scan_temp, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    if (key32)
        (k_gather<uint32_t><<<blocks_for(v.N, 256), 256, 0, st>>>(v, (const uint32_t*)skeys, flag, bflag), note_launch());
    else
        (k_gather<uint64_t><<<blocks_for(v.N, 256), 256, 0, st>>>(v, (const uint64_t*)skeys, flag, bflag), note_launch());
    cudaError_t e = exclusive_scan_u32(flag, cidx, v.N, nullptr, scan_temp, st);
    if (e != cudaSuccess) return e;
    if (bflag) {
        e = exclusive_scan_u32(bflag, bidx, v.N, nblocks, scan_temp, st);
        if (e != cudaSuccess) return e;
    }
    (k_cells<<<blocks_for(v.N, 256), 256, 0, st>>>(v, flag, cidx), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_blocks(const BatchView& v, const uint32_t* flag, const uint32_t* bflag, const uint32_t* bidx,
                          const uint32_t* nblocks, int64_t nblocks_bound, uint64_t* bkey, uint32_t* bfirst,
                          unsigned long long* bocc, cudaStream_t st) {
    if (v.N == 0 || nblocks_bound == 0) return cudaSuccess;
    (k_blocks_fill<<<blocks_for(v.N, 256), 256, 0, st>>>(v, flag, bflag, bidx, bkey, bfirst, bocc), note_launch());
    const unsigned blocks = (unsigned)std::min<int64_t>(blocks_for(nblocks_bound, 256), 152 * 16);
    (k_blocks_insert<<<blocks, 256, 0, st>>>(v, nblocks, bkey, bfirst, bocc), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_hash_insert(const BatchView& v, int64_t ncells_bound, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(blocks_for(ncells_bound, 256), 152 * 16);
    (k_hash_insert<<<blocks, 256, 0, st>>>(v), note_launch());
    return cudaGetLastError();
}

}  // namespace dpc
