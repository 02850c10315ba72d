// Approx-DPC's dependent points (Section 4.3), on exact local densities.
//
// The grid G of Section 4.1 has cells of side d_cut / sqrt(d) in every
// dimension, here the integer side max(1, floor(d_cut / sqrt(d))) anchored at
// the dataset's per-dimension minimum, so that two points of one cell are
// strictly closer than d_cut. Per cell: p*(c), its highest point in the
// order (rho desc, index asc), and the lowest rank among its points. Then:
//  - rule 1: a point that is not its cell's p* gets dependent point p*(c)
//    and dependent distance d_cut;
//  - rule 2: a p* looks at the cells other than its own that hold a point
//    strictly within d_cut of it (N(c)); among those whose points all rank
//    higher than p*, the one whose own p* ranks highest gives the dependent
//    point, again with dependent distance d_cut;
//  - every other point (a p* with no such cell) is computed exactly, by the
//    same tree search and brute-force passes the exact path uses.
// The cells of N(c) are found through the exact grid of side d_cut: every
// point within d_cut of p* lies in the neighbour runs of p*'s d_cut-cell.
#include "stages.cuh"
#include <algorithm>

namespace dpc {

namespace {

// Grid key of every sorted position: dataset key base + the cell
// coordinates packed at their per-dimension bit offsets.
__global__ void k_approx_keys(BatchView v, ApproxBufs ab) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const int b = find_ds(v.pt_off, v.B, p);
    const DsDesc& ds = v.desc[b];
    const int4* r = v.rec + ds.rec_off + (p - ds.pt_off) * ds.dp;
    uint64_t key = ds.a_base;
    for (int k = 0; k < ds.d; ++k) {
        const uint32_t c = (uint32_t)(rec_coord(r, k) - ds.lo[k]) / (uint32_t)ds.a_side;
        key |= (uint64_t)c << ds.a_shift[k];
    }
    ab.keys[p] = key;
    ab.ord[p] = (uint32_t)p;
}

__global__ void k_approx_flags(const uint64_t* __restrict__ skeys, uint32_t* __restrict__ flag, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    flag[t] = (t == 0 || skeys[t] != skeys[t - 1]) ? 1u : 0u;
}

__global__ void k_approx_cells(ApproxBufs ab, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint32_t f = ab.flag[t], c = ab.cidx[t] + f - 1u;
    ab.cell_of[ab.ord[t]] = c;
    if (f) ab.start[c] = (uint32_t)t;
    if (t == n - 1) {
        ab.start[c + 1] = (uint32_t)n;
        *ab.ncells = c + 1;
    }
}

// Per cell: the highest point (smallest rank) and the lowest rank.
__global__ void k_approx_tops(BatchView v, ApproxBufs ab, int64_t bound) {
    const uint32_t nc = *ab.ncells;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < bound && c < nc;
         c += (int64_t)gridDim.x * blockDim.x) {
        uint32_t best = 0xffffffffu, top = 0, lo = 0;
        for (uint32_t t = ab.start[c], e = ab.start[c + 1]; t < e; ++t) {
            const uint32_t p = ab.ord[t], r = v.ro_s[p].x;
            if (r < best) {
                best = r;
                top = p;
            }
            lo = max(lo, r);
        }
        ab.top[c] = top;
        ab.maxrank[c] = lo;
    }
}

// Rule 1 for every point that is not its cell's p*.
__global__ void k_approx_rule1(BatchView v, ApproxBufs ab) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const uint32_t top = ab.top[ab.cell_of[p]];
    if (top == (uint32_t)p) return;
    const int b = find_ds(v.pt_off, v.B, p);
    const DsDesc& ds = v.desc[b];
    const int64_t g = ds.pt_off + v.ro_s[p].y;
    v.dep[g] = (int32_t)v.ro_s[top].y;
    v.delta2[g] = ds.d_cut2;
    v.exact[g] = 0;
}

template <int D>
__device__ __forceinline__ void ax_load(const int4* r, int32_t (&x)[D]) {
    const int4 a = r[0];
    int32_t t[8] = {a.x, a.y, a.z, a.w, 0, 0, 0, 0};
    if (D > 4) {
        const int4 e = r[1];
        t[4] = e.x; t[5] = e.y; t[6] = e.z; t[7] = e.w;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = t[k];
}

// Rule 2 for every cell's p*, one thread per cell; p* without a qualifying
// cell go to the exact lists (brute force for ranks below bf_rank, else the
// tree search).
template <int D>
__global__ void __launch_bounds__(128) k_approx_rule2(BatchView v, CellWork w, ApproxBufs ab, DeltaBufs db,
                                                      int64_t bound) {
    constexpr int DP = D <= 4 ? 1 : 2;
    const uint32_t nc = *ab.ncells;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < bound; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = base + threadIdx.x;
        bool to_tree = false, to_bf = false;
        uint32_t p = 0;
        if (c < nc) {
            p = ab.top[c];
            const int b = find_ds(v.pt_off, v.B, p);
            const DsDesc& ds = v.desc[b];
            if (ds.d == D) {
                const uint32_t rk = v.ro_s[p].x;
                const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
                int32_t x[D];
                ax_load<D>(recb + (int64_t)p * DP, x);
                const uint32_t e = v.cell_of[p];  // the point's cell of side d_cut
                const uint2* runs = w.runs + (int64_t)e * w.nbs;
                const uint32_t nr = w.nruns[e];
                uint32_t best = 0xffffffffu, best_rank = 0xffffffffu;
                for (uint32_t ri = 0; ri < nr; ++ri) {
                    const uint2 run = runs[ri];
                    for (uint32_t q = run.x; q < run.x + run.y; ++q) {
                        int32_t y[D];
                        ax_load<D>(recb + (int64_t)q * DP, y);
                        long long dd = 0;
#pragma unroll
                        for (int k = 0; k < D; ++k) {
                            const long long t = (long long)x[k] - y[k];
                            dd += t * t;
                        }
                        if (dd >= ds.d_cut2) continue;
                        const uint32_t cq = ab.cell_of[q];
                        if (cq == (uint32_t)c || ab.maxrank[cq] >= rk) continue;
                        const uint32_t tq = ab.top[cq], rq = v.ro_s[tq].x;
                        if (rq < best_rank) {
                            best_rank = rq;
                            best = tq;
                        }
                    }
                }
                const int64_t g = ds.pt_off + v.ro_s[p].y;
                if (best != 0xffffffffu) {
                    v.dep[g] = (int32_t)v.ro_s[best].y;
                    v.delta2[g] = ds.d_cut2;
                    v.exact[g] = 0;
                } else {
                    v.exact[g] = 1;
                    if (rk < db.bf_rank) to_bf = true;
                    else to_tree = true;
                }
            }
        }
        const unsigned mt = __ballot_sync(0xffffffffu, to_tree), mb = __ballot_sync(0xffffffffu, to_bf);
        uint32_t bt = 0, bb = 0;
        if (lane == 0) {
            if (mt) bt = atomicAdd(&db.ucount[0], (uint32_t)__popc(mt));
            if (mb) bb = atomicAdd(&db.ucount[1], (uint32_t)__popc(mb));
        }
        bt = __shfl_sync(0xffffffffu, bt, 0);
        bb = __shfl_sync(0xffffffffu, bb, 0);
        if (to_tree) db.tree_list[bt + __popc(mt & lt)] = p;
        if (to_bf) db.bf_list[bb + __popc(mb & lt)] = p;
    }
}

}  // namespace

cudaError_t launch_approx_keys(const BatchView& v, const ApproxBufs& ab, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    (k_approx_keys<<<grid_for(v.N, 256), 256, 0, st>>>(v, ab), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_approx_cells(const BatchView& v, const ApproxBufs& ab, void* scan_temp, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    (k_approx_flags<<<grid_for(v.N, 256), 256, 0, st>>>(ab.keys, ab.flag, v.N), note_launch());
    cudaError_t e = exclusive_scan_u32(ab.flag, ab.cidx, v.N, nullptr, scan_temp, st);
    if (e != cudaSuccess) return e;
    (k_approx_cells<<<grid_for(v.N, 256), 256, 0, st>>>(ab, v.N), note_launch());
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(v.N, 256));
    (k_approx_tops<<<blocks, 256, 0, st>>>(v, ab, v.N), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_approx_rules(const BatchView& v, const CellWork& w, const ApproxBufs& ab, const DeltaBufs& db,
                                uint32_t dim_mask, int64_t ncells_bound, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    (k_approx_rule1<<<grid_for(v.N, 256), 256, 0, st>>>(v, ab), note_launch());
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(152 * 16, grid_for(ncells_bound, 128)));
#define DPC_APPROX_CLASS(D)        \
    if (dim_mask & (1u << (D - 1))) \
        (k_approx_rule2<D><<<blocks, 128, 0, st>>>(v, w, ab, db, ncells_bound), note_launch());
    DPC_APPROX_CLASS(1) DPC_APPROX_CLASS(2) DPC_APPROX_CLASS(3) DPC_APPROX_CLASS(4)
    DPC_APPROX_CLASS(5) DPC_APPROX_CLASS(6) DPC_APPROX_CLASS(7) DPC_APPROX_CLASS(8)
#undef DPC_APPROX_CLASS
    return cudaGetLastError();
}

}  // namespace dpc
