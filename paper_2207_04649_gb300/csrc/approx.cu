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

// Word w (bits [64 w, 64 w + 64)) of the grid key of sorted position p:
// each cell coordinate at its per-dimension bit offset, the dataset's index
// above them all at bshift (keys of any width, sorted 64 bits at a time).
__device__ __forceinline__ uint64_t a_word(const BatchView& v, int64_t p, int w, int bshift) {
    const int b = find_ds(v.pt_off, v.B, p);
    const DsDesc& ds = v.desc[b];
    const int4* r = v.rec + ds.rec_off + (p - ds.pt_off) * ds.dp;
    const int lo = 64 * w;
    uint64_t word = 0;
    auto put = [&](uint64_t c, int pos) {  // c < 2^31: bits [pos, pos + 31) of the key
        if (pos >= lo + 64 || pos + 31 <= lo) return;
        word |= pos >= lo ? c << (pos - lo) : c >> (lo - pos);
    };
    for (int k = 0; k < ds.d; ++k)
        put((uint32_t)(rec_coord(r, k) - ds.lo[k]) / (uint32_t)ds.a_side, ds.a_shift[k]);
    put((uint64_t)b, bshift);
    return word;
}

// Word w of the key of the position at key-order index t (the first pass
// takes the sorted positions in order).
__global__ void k_approx_keys(BatchView v, const uint32_t* __restrict__ prev, uint64_t* __restrict__ keys,
                              uint32_t* __restrict__ vals, int w, int bshift) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= v.N) return;
    const uint32_t p = prev ? prev[t] : (uint32_t)t;
    keys[t] = a_word(v, p, w, bshift);
    vals[t] = p;
}

__global__ void k_approx_flags(BatchView v, const uint32_t* __restrict__ ord, uint32_t* __restrict__ flag, int words,
                               int bshift) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= v.N) return;
    bool first = t == 0;
    for (int w = 0; w < words && !first; ++w) first = a_word(v, ord[t], w, bshift) != a_word(v, ord[t - 1], w, bshift);
    flag[t] = first ? 1u : 0u;
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

constexpr uint32_t kHeavyCand = 96;  // a p* with more candidates than this gets a whole warp

// Per cell: the highest point (smallest rank) and the lowest rank; the cell
// joins the light or the heavy list by its p*'s candidate count.
__global__ void k_approx_tops(BatchView v, CellWork w, ApproxBufs ab, int64_t bound) {
    const uint32_t nc = *ab.ncells;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < bound; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = base + threadIdx.x;
        bool light = false, heavy = false;
        if (c < nc) {
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
            heavy = w.cand[v.cell_of[top]] > kHeavyCand;
            light = !heavy;
        }
        const unsigned ml = __ballot_sync(0xffffffffu, light), mh = __ballot_sync(0xffffffffu, heavy);
        uint32_t bl = 0, bh = 0;
        if (lane == 0) {
            if (ml) bl = atomicAdd(&ab.nlh[0], (uint32_t)__popc(ml));
            if (mh) bh = atomicAdd(&ab.nlh[1], (uint32_t)__popc(mh));
        }
        bl = __shfl_sync(0xffffffffu, bl, 0);
        bh = __shfl_sync(0xffffffffu, bh, 0);
        if (light) ab.light[bl + __popc(ml & lt)] = (uint32_t)c;
        if (heavy) ab.heavy[bh + __popc(mh & lt)] = (uint32_t)c;
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

// Rule 2 for the p* of cell c: scan the candidates of its d_cut-cell
// neighbourhood, lane `lane` of `step` lanes taking every step-th one of
// each run. Besides the qualifying cell with the highest top, the scan finds
// the nearest higher candidate, which is the exact dependent point when it
// lies strictly closer than the outside of the scanned box of cells (the
// exact path's ring-search argument).
struct Rule2Part {
    uint32_t brq, bq;  // qualifying cell: its top's rank, the top
    long long bd;      // nearest higher candidate: distance, original index
    uint32_t bj;
};

template <int D>
__device__ __forceinline__ Rule2Part rule2_scan(const BatchView& v, const CellWork& w, const ApproxBufs& ab,
                                                const DsDesc& ds, const int4* recb, uint32_t c, uint32_t p,
                                                uint32_t rk, const int32_t (&x)[D], int lane, int step) {
    constexpr int DP = D <= 4 ? 1 : 2;
    Rule2Part r{0xffffffffu, 0u, INT64_MAX, 0xffffffffu};
    const uint32_t e = v.cell_of[p];  // the point's cell of side d_cut
    const uint2* runs = w.runs + (int64_t)e * w.nbs;
    const uint32_t nr = w.nruns[e];
    for (uint32_t ri = 0; ri < nr; ++ri) {
        const uint2 run = runs[ri];
        for (uint32_t q = run.x + lane; q < run.x + run.y; q += step) {
            int32_t y[D];
            ax_load<D>(recb + (int64_t)q * DP, y);
            long long dd = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const long long t = (long long)x[k] - y[k];
                dd += t * t;
            }
            const uint2 cr = v.ro_s[q];
            if (cr.x < rk && (dd < r.bd || (dd == r.bd && cr.y < r.bj))) {
                r.bd = dd;
                r.bj = cr.y;
            }
            if (dd >= ds.d_cut2) continue;
            const uint32_t cq = ab.cell_of[q];
            if (cq == c || ab.maxrank[cq] >= rk) continue;
            const uint32_t tq = ab.top[cq], rq = v.ro_s[tq].x;
            if (rq < r.brq) {
                r.brq = rq;
                r.bq = tq;
            }
        }
    }
    return r;
}

// Writes the outcome for p (or queues it for the exact passes).
template <int D>
__device__ __forceinline__ void rule2_finish(const BatchView& v, const DeltaBufs& db, const DsDesc& ds,
                                             const int4* recb, uint32_t p, uint32_t rk, const Rule2Part& r) {
    constexpr int DP = D <= 4 ? 1 : 2;
    const int64_t g = ds.pt_off + v.ro_s[p].y;
    if (r.brq != 0xffffffffu) {
        v.dep[g] = (int32_t)v.ro_s[r.bq].y;
        v.delta2[g] = ds.d_cut2;
        v.exact[g] = 0;
        return;
    }
    v.exact[g] = 1;
    // distance from the point to the outside of the scanned box of cells
    int64_t bound = INT64_MAX;
    for (int j = 0; j < ds.k; ++j) {
        const int32_t xi = rec_coord(recb + (int64_t)p * DP, ds.gdim[j]);
        const int64_t cj = cell_coord(ds, j, xi);
        if (cj - ds.R > 0) bound = min(bound, (int64_t)xi - (ds.origin[j] + (cj - ds.R) * ds.s) + 1);
        if (cj + ds.R + 1 < ds.ext[j]) bound = min(bound, ds.origin[j] + (cj + ds.R + 1) * ds.s - (int64_t)xi);
    }
    // cells the runs left out (at least d_cut away) were not scanned
    if (ds.prune) bound = min(bound, ds.d_cut);
    const bool proven = r.bd != INT64_MAX && (bound == INT64_MAX || (bound < 3037000499ll && r.bd < bound * bound));
    if (proven) {
        v.dep[g] = (int32_t)r.bj;
        v.delta2[g] = r.bd;
    } else if (rk < db.bf_rank) {
        db.bf_list[atomicAdd(&db.ucount[1], 1u)] = p;
    } else {
        db.tree_list[atomicAdd(&db.ucount[0], 1u)] = p;
    }
}

// Light cells: one thread each.
template <int D>
__global__ void __launch_bounds__(128) k_approx_rule2_light(BatchView v, CellWork w, ApproxBufs ab, DeltaBufs db) {
    constexpr int DP = D <= 4 ? 1 : 2;
    const uint32_t n = ab.nlh[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = ab.light[i], p = ab.top[c];
        const DsDesc& ds = v.desc[find_ds(v.pt_off, v.B, p)];
        if (ds.d != D) continue;
        const uint32_t rk = v.ro_s[p].x;
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        int32_t x[D];
        ax_load<D>(recb + (int64_t)p * DP, x);
        const Rule2Part r = rule2_scan<D>(v, w, ab, ds, recb, c, p, rk, x, 0, 1);
        rule2_finish<D>(v, db, ds, recb, p, rk, r);
    }
}

// Heavy cells: one warp each, the lanes splitting every run.
template <int D>
__global__ void __launch_bounds__(128) k_approx_rule2_heavy(BatchView v, CellWork w, ApproxBufs ab, DeltaBufs db) {
    constexpr int DP = D <= 4 ? 1 : 2;
    const uint32_t n = ab.nlh[1];
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nwarps) {
        const uint32_t c = ab.heavy[i], p = ab.top[c];
        const DsDesc& ds = v.desc[find_ds(v.pt_off, v.B, p)];
        if (ds.d != D) continue;
        const uint32_t rk = v.ro_s[p].x;
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        int32_t x[D];
        ax_load<D>(recb + (int64_t)p * DP, x);
        Rule2Part r = rule2_scan<D>(v, w, ab, ds, recb, c, p, rk, x, lane, 32);
        for (int o = 16; o > 0; o >>= 1) {
            const uint32_t r2 = __shfl_xor_sync(0xffffffffu, r.brq, o), q2 = __shfl_xor_sync(0xffffffffu, r.bq, o);
            if (r2 < r.brq) {
                r.brq = r2;
                r.bq = q2;
            }
            const long long d2 = __shfl_xor_sync(0xffffffffu, r.bd, o);
            const uint32_t j2 = __shfl_xor_sync(0xffffffffu, r.bj, o);
            if (d2 < r.bd || (d2 == r.bd && j2 < r.bj)) {
                r.bd = d2;
                r.bj = j2;
            }
        }
        if (lane == 0) rule2_finish<D>(v, db, ds, recb, p, rk, r);
    }
}

}  // namespace

cudaError_t launch_approx_keys(const BatchView& v, int key_bits, int bshift, uint64_t* keys, uint32_t* ords,
                               void* temp, uint32_t** ord_out, cudaStream_t st) {
    *ord_out = ords;
    if (v.N == 0) return cudaSuccess;
    // LSD over 64-bit words: each pass sorts the previous order stably by
    // the next more significant word; the three value buffers rotate
    const int words = std::max(1, (key_bits + 63) / 64);
    const int64_t N = v.N;
    uint64_t *kin = keys, *kout = keys + N, *ktmp = keys + 2 * N;
    uint32_t *vin = ords + N, *vout = ords, *vtmp = ords + 2 * N;
    const uint32_t* prev = nullptr;
    for (int w = 0; w < words; ++w) {
        const int nbits = std::max(1, std::min(64, key_bits - 64 * w));
        (k_approx_keys<<<grid_for(N, 256), 256, 0, st>>>(v, prev, kin, vin, w, bshift), note_launch());
        cudaError_t e = radix_sort_u64(kin, vin, kout, vout, ktmp, vtmp, N, nbits, temp, st);
        if (e != cudaSuccess) return e;
        prev = vout;
        std::swap(vin, vout);
        std::swap(vin, vtmp);
    }
    *ord_out = const_cast<uint32_t*>(prev);
    return cudaGetLastError();
}

cudaError_t launch_approx_cells(const BatchView& v, const CellWork& w, const ApproxBufs& ab, int key_bits,
                                int bshift, void* scan_temp, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    const int words = std::max(1, (key_bits + 63) / 64);
    (k_approx_flags<<<grid_for(v.N, 256), 256, 0, st>>>(v, ab.ord, ab.flag, words, bshift), note_launch());
    cudaError_t e = exclusive_scan_u32(ab.flag, ab.cidx, v.N, nullptr, scan_temp, st);
    if (e != cudaSuccess) return e;
    (k_approx_cells<<<grid_for(v.N, 256), 256, 0, st>>>(ab, v.N), note_launch());
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(v.N, 256));
    (k_approx_tops<<<blocks, 256, 0, st>>>(v, w, ab, v.N), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_approx_rules(const BatchView& v, const CellWork& w, const ApproxBufs& ab, const DeltaBufs& db,
                                uint32_t dim_mask, int64_t ncells_bound, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    (k_approx_rule1<<<grid_for(v.N, 256), 256, 0, st>>>(v, ab), note_launch());
    const unsigned bl = (unsigned)std::max<int64_t>(1, std::min<int64_t>(152 * 16, grid_for(ncells_bound, 128)));
    const unsigned bh = (unsigned)std::max<int64_t>(1, std::min<int64_t>(152 * 16, grid_for(ncells_bound, 4)));
#define DPC_APPROX_CLASS(D)                                                                   \
    if (dim_mask & (1u << (D - 1))) {                                                          \
        (k_approx_rule2_light<D><<<bl, 128, 0, st>>>(v, w, ab, db), note_launch());            \
        (k_approx_rule2_heavy<D><<<bh, 128, 0, st>>>(v, w, ab, db), note_launch());            \
    }
    DPC_APPROX_CLASS(1) DPC_APPROX_CLASS(2) DPC_APPROX_CLASS(3) DPC_APPROX_CLASS(4)
    DPC_APPROX_CLASS(5) DPC_APPROX_CLASS(6) DPC_APPROX_CLASS(7) DPC_APPROX_CLASS(8)
#undef DPC_APPROX_CLASS
    return cudaGetLastError();
}

}  // namespace dpc
