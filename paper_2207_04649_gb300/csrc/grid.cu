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

// Per-dataset, per-dimension min and max of the input coordinates.
__global__ void k_minmax(BatchView v, int32_t* __restrict__ mm) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = g < v.N;
    const int b = valid ? find_ds(v.pt_off, v.B, g) : -1;
    const unsigned same = __match_any_sync(0xffffffffu, b);
    if (!valid) return;
    const DsDesc& ds = v.desc[b];
    const int32_t* x = v.in + ds.in_off + (g - ds.pt_off) * ds.d;
    const int lane = threadIdx.x & 31;
    const bool full = same == 0xffffffffu;  // all 32 lanes valid and in one dataset
    for (int k = 0; k < ds.d; ++k) {
        int lo = x[k], hi = x[k];
        if (full) {
            for (int o = 16; o > 0; o >>= 1) {
                lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
        }
        if (!full || lane == 0) {
            atomicMin(&mm[(b * kMaxDims + k) * 2], lo);
            atomicMax(&mm[(b * kMaxDims + k) * 2 + 1], hi);
        }
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
    int32_t c[kMaxGridDims];
    for (int j = 0; j < ds.k; ++j) c[j] = (int32_t)(((int64_t)x[ds.gdim[j]] - ds.origin[j]) / ds.s);
    keys[g] = (K)(ds.cbase + morton(c, ds.k, ds.mbits));
    vals[g] = (uint32_t)g;
}

// Sorted records (dp int4 per point, zero-padded), inverse permutation and
// cell-start flags.
template <typename K>
__global__ void k_gather(BatchView v, const K* __restrict__ skeys, uint32_t* __restrict__ flag) {
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
    r[0] = make_int4(c[0], c[1], c[2], c[3]);
    if (ds.dp == 2) r[1] = make_int4(c[4], c[5], c[6], c[7]);
    v.pos_of[g] = (uint32_t)p;
    v.key[p] = (uint64_t)skeys[p];
    flag[p] = (p == 0 || skeys[p] != skeys[p - 1]) ? 1u : 0u;
}

__global__ void k_cells(BatchView v, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ cidx) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    if (flag[p]) v.cell_start[cidx[p]] = (uint32_t)p;
    if (p == v.N - 1) {
        const uint32_t nc = cidx[p] + flag[p];
        v.cell_start[nc] = (uint32_t)v.N;
        *v.ncells = nc;
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
    if (v.N > 0) (k_minmax<<<blocks_for(v.N, 256), 256, 0, st>>>(v, mm), note_launch());
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

cudaError_t launch_gather_cells(const BatchView& v, bool key32, const void* skeys, uint32_t* flag, uint32_t* cidx,
                                void* scan_temp, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    if (key32)
        (k_gather<uint32_t><<<blocks_for(v.N, 256), 256, 0, st>>>(v, (const uint32_t*)skeys, flag), note_launch());
    else
        (k_gather<uint64_t><<<blocks_for(v.N, 256), 256, 0, st>>>(v, (const uint64_t*)skeys, flag), note_launch());
    cudaError_t e = exclusive_scan_u32(flag, cidx, v.N, nullptr, scan_temp, st);
    if (e != cudaSuccess) return e;
    (k_cells<<<blocks_for(v.N, 256), 256, 0, st>>>(v, flag, cidx), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_hash_insert(const BatchView& v, int64_t ncells_bound, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(blocks_for(ncells_bound, 256), 152 * 16);
    (k_hash_insert<<<blocks, 256, 0, st>>>(v), note_launch());
    return cudaGetLastError();
}

}  // namespace dpc
