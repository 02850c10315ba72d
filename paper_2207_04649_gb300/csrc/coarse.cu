// Coarse ring: the second ring of the expanding search for dependent points.
//
// A point left open by the ring search over its 3^k neighbouring grid cells
// is searched again over the 3^k neighbouring cells of a coarser grid: aligned
// blocks of 2^L x ... x 2^L grid cells. Because the points are sorted by the
// Morton code of their grid cell, a coarse cell is a contiguous run of sorted
// points, found through its own hash table. The point is resolved when the
// best higher point found lies strictly closer than the outside of the 3^k
// coarse block around it (at least 2^L cells away); otherwise, or when one
// of the coarse cells holds more than `ccap` points (dense regions, where a
// coarse scan would be expensive), it stays open for the tree search.
// Distances are exact in 64-bit integers; ties go to the smaller original
// index (Definitions 2-3).
#include "stages.cuh"
#include <algorithm>

namespace dpc {

namespace {

constexpr int kCoarseBits = 44;  // coarse key: dataset << 44 | coarse Morton code

__device__ __forceinline__ uint64_t coarse_key(int b, uint64_t code) {
    return ((uint64_t)b << kCoarseBits) | code;
}

// A fine cell starts a coarse cell when its dataset or its coarse code
// differs from the previous cell's.
__global__ void k_coarse_flag(BatchView v, DeltaBufs db) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= db.ncells) return;
    const uint32_t p = v.cell_start[c];
    const int b = find_ds(v.pt_off, v.B, p);
    const DsDesc& ds = v.desc[b];
    const uint64_t ck = (v.key[p] - ds.cbase) >> (ds.k * db.clevel);
    uint32_t f = 1u;
    if (c > 0) {
        const uint32_t q = v.cell_start[c - 1];
        const int bq = find_ds(v.pt_off, v.B, q);
        const uint64_t cq = (v.key[q] - v.desc[bq].cbase) >> (v.desc[bq].k * db.clevel);
        f = (bq != b || cq != ck) ? 1u : 0u;
    }
    db.cflag[c] = f;
}

__global__ void k_coarse_first(DeltaBufs db) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= db.ncells) return;
    const uint32_t ex = db.cidx[c], f = db.cflag[c];
    if (f) db.cfirst[ex] = (uint32_t)c;
    db.cidx[c] = ex + f - 1u;
    if (c == db.ncells - 1) db.cfirst[ex + f] = (uint32_t)db.ncells;
}

__global__ void k_coarse_insert(BatchView v, DeltaBufs db) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= db.ncoarse) return;
    const uint32_t c = db.cfirst[j], ce = db.cfirst[j + 1];
    const uint32_t st = v.cell_start[c], cnt = v.cell_start[ce] - st;
    const int b = find_ds(v.pt_off, v.B, st);
    const DsDesc& ds = v.desc[b];
    const uint64_t key = coarse_key(b, (v.key[st] - ds.cbase) >> (ds.k * db.clevel));
    uint64_t h = mix64(key) & db.chmask;
    for (uint64_t probe = 0; probe <= db.chmask; ++probe) {
        unsigned long long* slot = reinterpret_cast<unsigned long long*>(&db.chash[h]);
        if (atomicCAS(slot, (unsigned long long)kEmptyKey, (unsigned long long)key) == kEmptyKey) {
            db.chash[h].z = (int)st;
            db.chash[h].w = (int)cnt;
            break;
        }
        h = (h + 1) & db.chmask;
    }
}

template <int D>
__device__ __forceinline__ void c_load(const int4* r, int32_t (&x)[D]) {
    const int4 a = r[0];
    int32_t t[8] = {a.x, a.y, a.z, a.w, 0, 0, 0, 0};
    if (D > 4) {
        const int4 bq = r[1];
        t[4] = bq.x; t[5] = bq.y; t[6] = bq.z; t[7] = bq.w;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = t[k];
}

constexpr int kCoarseBatch = 9;  // hash probes issued together per thread

template <int D>
__global__ void __launch_bounds__(128) k_coarse_ring(BatchView v, DeltaBufs db) {
    constexpr int DP = D <= 4 ? 1 : 2;
    const uint32_t cnt = db.ucount[0];
    const int L = db.clevel;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = db.tree_list[i];
        const int b = find_ds(v.pt_off, v.B, p);
        const DsDesc& ds = v.desc[b];
        if (ds.d != D) continue;
        bool keep_open = ds.R != 1 || ds.k == 0;
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        int32_t x[D];
        c_load<D>(recb + (int64_t)p * DP, x);
        const uint2 ro = v.ro_s[p];
        long long bestD = INT64_MAX;
        uint32_t bestJ = 0xffffffffu;
        const unsigned long long bk = v.best_s[p];
        if (bk != ~0ull && (uint32_t)(bk >> 32) != 0xffffffffu) {
            bestD = (long long)(bk >> 32);
            bestJ = (uint32_t)bk;
        }
        int32_t cc[kMaxGridDims], ce[kMaxGridDims];
        uint64_t cm[kMaxGridDims];
        const int4* rp = recb + (int64_t)p * DP;
        for (int j = 0; j < ds.k; ++j) {
            cc[j] = cell_coord(ds, j, rec_coord(rp, ds.gdim[j])) >> L;
            ce[j] = ((ds.ext[j] - 1) >> L) + 1;
            cm[j] = ds.dmask[j] >> (ds.k * L);
        }
        const uint64_t own = (v.key[p] - ds.cbase) >> (ds.k * L);
        int nnb = 1;
        for (int j = 0; j < ds.k; ++j) nnb *= 3;
        for (int base = 0; base < nnb && !keep_open; base += kCoarseBatch) {
            uint64_t key[kCoarseBatch];
            int4 e[kCoarseBatch];
#pragma unroll
            for (int q = 0; q < kCoarseBatch; ++q) {
                const int t = base + q;
                key[q] = kEmptyKey;
                if (t < nnb) {
                    bool ok = true;
                    uint64_t code = own;
                    int tt = t;
                    for (int j = 0; j < ds.k; ++j) {
                        const int o = tt % 3 - 1;
                        tt /= 3;
                        if (o != 0) {
                            ok = ok && cc[j] + o >= 0 && cc[j] + o < ce[j];
                            code = morton_step(code, cm[j], o);
                        }
                    }
                    if (ok) key[q] = coarse_key(b, code);
                }
                e[q] = key[q] != kEmptyKey ? __ldg(&db.chash[mix64(key[q]) & db.chmask]) : make_int4(-1, -1, 0, 0);
            }
            for (int q = 0; q < kCoarseBatch && !keep_open; ++q) {
                if (key[q] == kEmptyKey) continue;
                const uint64_t k0 = (uint64_t)(uint32_t)e[q].x | ((uint64_t)(uint32_t)e[q].y << 32);
                uint2 r = make_uint2(0u, 0u);
                if (k0 == key[q]) r = make_uint2((uint32_t)e[q].z, (uint32_t)e[q].w);
                else if (k0 != kEmptyKey) r = hash_find(db.chash, db.chmask, key[q]);
                if (r.y > db.ccap) {
                    keep_open = true;
                    break;
                }
                for (uint32_t qq = r.x, q1 = r.x + r.y; qq < q1; ++qq) {
                    const uint2 cr = v.ro_s[qq];
                    if (cr.x >= ro.x) continue;
                    int32_t cx[D];
                    c_load<D>(recb + (int64_t)qq * DP, cx);
                    long long dd = 0;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const long long f = (long long)x[k] - cx[k];
                        dd += f * f;
                    }
                    if (dd < bestD || (dd == bestD && cr.y < bestJ)) {
                        bestD = dd;
                        bestJ = cr.y;
                    }
                }
            }
        }
        bool resolved = false;
        if (!keep_open && bestD != INT64_MAX) {
            // distance to the outside of the 3^k coarse block around the point
            long long bound = INT64_MAX;
            for (int j = 0; j < ds.k; ++j) {
                const long long xj = rec_coord(rp, ds.gdim[j]);
                if (cc[j] - 1 > 0)
                    bound = min(bound, xj - (ds.origin[j] + ((long long)(cc[j] - 1) << L) * ds.s) + 1);
                if (cc[j] + 2 < ce[j])
                    bound = min(bound, ds.origin[j] + ((long long)(cc[j] + 2) << L) * ds.s - xj);
            }
            resolved = bound == INT64_MAX || bestD < bound * bound;
        }
        if (resolved) {
            const int64_t g = ds.pt_off + ro.y;
            v.dep[g] = (int32_t)bestJ;
            v.delta2[g] = bestD;
        } else {
            db.open2[atomicAdd(&db.ucount[2], 1u)] = p;
        }
    }
}

}  // namespace

cudaError_t launch_coarse_cells(const BatchView& v, const DeltaBufs& db, void* scan_temp, cudaStream_t st) {
    if (db.ncells == 0) return cudaSuccess;
    (k_coarse_flag<<<grid_for(db.ncells, 256), 256, 0, st>>>(v, db), note_launch());
    cudaError_t e = exclusive_scan_u32(db.cflag, db.cidx, db.ncells, nullptr, scan_temp, st);
    if (e != cudaSuccess) return e;
    (k_coarse_first<<<grid_for(db.ncells, 256), 256, 0, st>>>(db), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_coarse_hash(const BatchView& v, const DeltaBufs& db, cudaStream_t st) {
    if (db.ncoarse == 0) return cudaSuccess;
    (k_coarse_insert<<<grid_for(db.ncoarse, 256), 256, 0, st>>>(v, db), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_coarse_ring(const BatchView& v, const DeltaBufs& db, uint32_t dim_mask, int64_t bound,
                               cudaStream_t st) {
    if (bound <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(bound, 128));
#define DPC_COARSE_CLASS(D) \
    if (dim_mask & (1u << (D - 1))) (k_coarse_ring<D><<<blocks, 128, 0, st>>>(v, db), note_launch());
    DPC_COARSE_CLASS(1) DPC_COARSE_CLASS(2) DPC_COARSE_CLASS(3) DPC_COARSE_CLASS(4)
    DPC_COARSE_CLASS(5) DPC_COARSE_CLASS(6) DPC_COARSE_CLASS(7) DPC_COARSE_CLASS(8)
#undef DPC_COARSE_CLASS
    return cudaGetLastError();
}

}  // namespace dpc

// ------------------------------------------------------------------ ring 2
//
// The second ring of the expanding search, on the fine grid itself: a point
// the first ring left open (its nearest higher point among the 3^k
// neighbouring cells, if any, is not proven) scans the shell of cells at
// distance 2 (the 5^k block minus the 3^k one), one warp per point, lanes
// taking shell cells, skipping those whose box is farther than the best
// distance so far. It is resolved when the best higher point over both
// rings lies strictly closer than the outside of the 5^k block; otherwise it
// stays open for the tree search. Only datasets with cell side d_cut (reach
// 1) take it.
namespace dpc {
namespace {

template <int D>
__device__ __forceinline__ void r2_load(const int4* r, int32_t (&x)[D]) {
    const int4 a = r[0];
    int32_t t[8] = {a.x, a.y, a.z, a.w, 0, 0, 0, 0};
    if (D > 4) {
        const int4 b = r[1];
        t[4] = b.x; t[5] = b.y; t[6] = b.z; t[7] = b.w;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = t[k];
}

template <int D>
__global__ void __launch_bounds__(128) k_ring2(BatchView v, DeltaBufs db) {
    constexpr int DP = D <= 4 ? 1 : 2;
    const uint32_t cnt = db.ucount[0];
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < cnt; i += nwarps) {
        const uint32_t p = db.tree_list[i];
        const int b = find_ds(v.pt_off, v.B, p);
        const DsDesc& ds = v.desc[b];
        if (ds.d != D) continue;
        bool keep = ds.R != 1 || ds.k == 0;
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        const int4* rp = recb + (int64_t)p * DP;
        int32_t x[D];
        r2_load<D>(rp, x);
        const uint2 ro = v.ro_s[p];
        // the first ring's best (unproven); a saturated distance is no candidate
        long long bd = INT64_MAX;
        uint32_t bj = 0xffffffffu;
        const unsigned long long bk = v.best_s[p];
        if (bk != ~0ull && (uint32_t)(bk >> 32) != 0xffffffffu) {
            bd = (long long)(bk >> 32);
            bj = (uint32_t)bk;
        }
        // a saturated first-ring distance lost its result: scan those cells again
        const bool lost = bk != ~0ull && (uint32_t)(bk >> 32) == 0xffffffffu;
        int32_t cc[kMaxGridDims];
        int nsh = 1;
        for (int j = 0; j < ds.k; ++j) {
            cc[j] = cell_coord(ds, j, rec_coord(rp, ds.gdim[j]));
            nsh *= 5;
        }
        const uint64_t own = v.key[p] - ds.cbase;
        // lanes take the 5^k offsets; the inner 3^k were the first ring
        for (int base = 0; base < nsh && !keep; base += 32) {
            const int t = base + lane;
            if (t < nsh) {
                int tt = t;
                bool inner = true, ok = true;
                int nz = 0;
                uint64_t code = own;
                long long gap2 = 0;
                for (int j = 0; j < ds.k; ++j) {
                    const int o = tt % 5 - 2;
                    tt /= 5;
                    if (o < -1 || o > 1) inner = false;
                    if (o != 0) {
                        ++nz;
                        ok = ok && cc[j] + o >= 0 && cc[j] + o < ds.ext[j];
                        const int ao = o < 0 ? -o : o;
                        for (int u = 0; u < ao; ++u) code = morton_step(code, ds.dmask[j], o);
                        // distance from x to that cell's slab in this dim
                        const int32_t xj = rec_coord(rp, ds.gdim[j]);
                        const long long lo = ds.origin[j] + (long long)(cc[j] + o) * ds.s;
                        const long long g = o > 0 ? lo - xj : xj - (lo + ds.s - 1);
                        if (g > 0) gap2 += g * g;
                    }
                }
                // an inner cell was the first ring's, unless its runs left it out
                // (off in nz >= d_cut^2 dims: no point of it is within d_cut)
                const bool todo = !inner || lost || (long long)nz >= ds.d_cut2;
                if (todo && ok && gap2 <= bd) {
                    const uint2 r = hash_find(v.hash, v.hmask, ds.cbase + code);
                    for (uint32_t q = r.x; q < r.x + r.y; ++q) {
                        const uint2 cr = v.ro_s[q];
                        if (cr.x >= ro.x) continue;
                        int32_t y[D];
                        r2_load<D>(recb + (int64_t)q * DP, y);
                        long long dd = 0;
#pragma unroll
                        for (int k = 0; k < D; ++k) {
                            const long long e = (long long)x[k] - y[k];
                            dd += e * e;
                        }
                        if (dd < bd || (dd == bd && cr.y < bj)) {
                            bd = dd;
                            bj = cr.y;
                        }
                    }
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const long long d2 = __shfl_xor_sync(0xffffffffu, bd, o);
            const uint32_t j2 = __shfl_xor_sync(0xffffffffu, bj, o);
            if (d2 < bd || (d2 == bd && j2 < bj)) {
                bd = d2;
                bj = j2;
            }
        }
        if (lane == 0) {
            bool resolved = false;
            if (!keep && bd != INT64_MAX) {
                // distance to the outside of the 5^k block around the point
                long long bound = INT64_MAX;
                for (int j = 0; j < ds.k; ++j) {
                    const long long xj = rec_coord(rp, ds.gdim[j]);
                    if (cc[j] - 2 > 0) bound = min(bound, xj - (ds.origin[j] + (long long)(cc[j] - 2) * ds.s) + 1);
                    if (cc[j] + 3 < ds.ext[j]) bound = min(bound, ds.origin[j] + (long long)(cc[j] + 3) * ds.s - xj);
                }
                resolved = bound == INT64_MAX || (bound < 3037000499ll && bd < bound * bound);
            }
            if (resolved) {
                const int64_t g = ds.pt_off + ro.y;
                v.dep[g] = (int32_t)bj;
                v.delta2[g] = bd;
            } else {
                db.open2[atomicAdd(&db.ucount[2], 1u)] = p;
            }
        }
    }
}

}  // namespace

cudaError_t launch_ring2(const BatchView& v, const DeltaBufs& db, uint32_t dim_mask, int64_t bound, cudaStream_t st) {
    if (bound <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(bound, 4));
#define DPC_RING2_CLASS(D) \
    if (dim_mask & (1u << (D - 1))) (k_ring2<D><<<blocks, 128, 0, st>>>(v, db), note_launch());
    DPC_RING2_CLASS(1) DPC_RING2_CLASS(2) DPC_RING2_CLASS(3) DPC_RING2_CLASS(4)
    DPC_RING2_CLASS(5) DPC_RING2_CLASS(6) DPC_RING2_CLASS(7) DPC_RING2_CLASS(8)
#undef DPC_RING2_CLASS
    return cudaGetLastError();
}

}  // namespace dpc
