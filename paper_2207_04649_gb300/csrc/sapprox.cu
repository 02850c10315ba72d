// S-Approx-DPC (Section 5): local densities and dependent points of one
// picked point per cell of a finer grid G'.
//
// G' has cells of side eps * d_cut / sqrt(d) in every dimension, here the
// integer side max(1, floor(eps * d_cut / sqrt(d))) anchored at the
// dataset's per-dimension minimum. The picked point of a cell is its point
// with the smallest original index. Then:
//  - every pick gets its local density (Definition 1). When picks are a
//    large share of the points, the exact path's density kernels count every
//    point (cheaper per pair than a pick-only pass); otherwise one warp per
//    pick counts over the neighbour runs of its cell of the exact grid (side
//    d_cut, reach R), which hold every point within d_cut of it;
//  - picks are ordered by (rho desc, index asc); the other points rank
//    after all of them (their rho is set to 0), so the exact path's ring,
//    tree and brute-force searches, which look for the nearest point of
//    lower rank, only ever return picks;
//  - first phase: the cells of G' (other than its own) holding a point
//    strictly within d_cut of a pick form N(c); among their picks that rank
//    higher, the nearest (ties to the smaller index) is the dependent point,
//    at its exact distance. With picks a quarter of the points or more, the
//    exact ring search over pick ranks runs first: when the nearest higher
//    pick of a pick's searched block of exact-grid cells lies strictly
//    within d_cut, it is the nearest higher pick overall and belongs to
//    N(c), so it is the first-phase answer, and only the other picks scan
//    their neighbourhood for N(c). With fewer picks a pass over the picks of
//    each pick's block (no other points' records read) gives the same
//    nearest higher pick of the block, and the cost follows the picks, not
//    the points;
//  - second phase, for a pick without a first-phase candidate: its nearest
//    higher pick over all picks: the nearest higher pick of the searched
//    block (kept by the scan, or the ring's) when it lies strictly closer
//    than the outside of the block, else the tree search or the brute force;
//  - a point that is not picked depends on its cell's pick, at its exact
//    distance.
#include "stages.cuh"
#include <algorithm>

namespace dpc {

namespace {

// Word w (bits [64 w, 64 w + 64)) of the key of G' of original point g: each
// cell coordinate at its bit offset, the dataset's index above them all at
// bshift. Words are recomputed from the coordinates wherever they are needed.
__device__ __forceinline__ uint64_t sap_word(const BatchView& v, int64_t g, int w, int bshift) {
    const int b = find_ds(v.pt_off, v.B, g);
    const DsDesc& ds = v.desc[b];
    const int4* r = v.rec + ds.rec_off + ((int64_t)v.pos_of[g] - ds.pt_off) * ds.dp;
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

// Word w of the key of the point at key-order position t (the first pass
// takes the points in original order).
__global__ void k_sap_keys(BatchView v, const uint32_t* __restrict__ ord, uint64_t* __restrict__ keys,
                           uint32_t* __restrict__ vals, int w, int bshift) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= v.N) return;
    const uint32_t g = ord ? ord[t] : (uint32_t)t;
    keys[t] = sap_word(v, g, w, bshift);
    vals[t] = g;
}

__global__ void k_sap_flags(BatchView v, SapproxBufs sb, int words, int bshift) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= v.N) return;
    bool first = t == 0;
    for (int w = 0; w < words && !first; ++w)
        first = sap_word(v, sb.ord[t], w, bshift) != sap_word(v, sb.ord[t - 1], w, bshift);
    sb.flag[t] = first ? 1u : 0u;
}

// The first point of every cell of G' (in key order) is its pick.
__global__ void k_sap_picks(BatchView v, SapproxBufs sb, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint32_t f = sb.flag[t], c = sb.cidx[t] + f - 1u;
    if (f) sb.picks[c] = v.pos_of[sb.ord[t]];
    if (t == n - 1) *sb.npicks = c + 1;
}

// Every point learns its cell's pick (sorted positions) and whether it is one.
__global__ void k_sap_pick_of(BatchView v, SapproxBufs sb, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint32_t f = sb.flag[t], c = sb.cidx[t] + f - 1u;
    const uint32_t g = sb.ord[t];
    sb.pick_s[v.pos_of[g]] = sb.picks[c];
    v.pick[g] = (uint8_t)f;
}

// Picks of every exact-grid cell, contiguous: plist holds the picks in
// sorted order, pstart[c] .. pstart[c + 1] those of cell c (pos is the
// exclusive count of picks before each sorted position).
__global__ void k_sap_pflag(BatchView v, SapproxBufs sb) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < v.N) sb.pflag[p] = sb.pick_s[p] == (uint32_t)p ? 1u : 0u;
}

__global__ void k_sap_plist(BatchView v, SapproxBufs sb, int64_t ncells) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < v.N && sb.pflag[p]) sb.plist[sb.ppos[p]] = (uint32_t)p;
    if (p < ncells) sb.pstart[p] = sb.ppos[v.cell_start[p]];
    if (p == 0) sb.pstart[ncells] = *sb.npicks;
}

// Candidate pairs a pass over the picks alone would evaluate: the sum over
// picks of their exact-grid cell's candidates.
__global__ void k_sap_pick_pairs(BatchView v, CellWork w, SapproxBufs sb) {
    const uint32_t m = *sb.npicks;
    unsigned long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        s += w.cand[v.cell_of[sb.picks[i]]];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(&sb.stats[2], s);
}

template <int D>
__device__ __forceinline__ void sx_load(const int4* r, int32_t (&x)[D]) {
    const int4 a = r[0];
    int32_t t[8] = {a.x, a.y, a.z, a.w, 0, 0, 0, 0};
    if (D > 4) {
        const int4 e = r[1];
        t[4] = e.x; t[5] = e.y; t[6] = e.z; t[7] = e.w;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = t[k];
}

template <int D>
__device__ __forceinline__ long long sx_dist(const int32_t (&x)[D], const int32_t (&y)[D]) {
    long long dd = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const long long t = (long long)x[k] - y[k];
        dd += t * t;
    }
    return dd;
}

// Local density of every pick: one warp per pick, the lanes splitting every
// neighbour run of its exact-grid cell.
template <int D>
__global__ void __launch_bounds__(128) k_sap_rho(BatchView v, CellWork w, SapproxBufs sb) {
    constexpr int DP = D <= 4 ? 1 : 2;
    const uint32_t m = *sb.npicks;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long pairs = 0;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += nwarps) {
        const uint32_t p = sb.picks[i];
        const DsDesc& ds = v.desc[find_ds(v.pt_off, v.B, p)];
        if (ds.d != D) continue;
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        int32_t x[D];
        sx_load<D>(recb + (int64_t)p * DP, x);
        const uint32_t e = v.cell_of[p];
        const uint2* runs = w.runs + (int64_t)e * w.nbs;
        const uint32_t nr = w.nruns[e];
        uint32_t cnt = 0;
        for (uint32_t ri = 0; ri < nr; ++ri) {
            const uint2 run = runs[ri];
            for (uint32_t q = run.x + lane; q < run.x + run.y; q += 32) {
                int32_t y[D];
                sx_load<D>(recb + (int64_t)q * DP, y);
                cnt += sx_dist<D>(x, y) < ds.d_cut2 ? 1u : 0u;
            }
            pairs += run.y;
        }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) {
            v.rho_s[p] = (int32_t)cnt;
            v.rho[v.perm[p]] = (int32_t)cnt;
        }
    }
    if (lane == 0 && pairs) atomicAdd(&sb.stats[0], pairs);
}

// Pick path, local density of every pick, one warp per exact-grid cell that
// holds picks: the cell's neighbour runs are staged once per chunk in shared
// memory and shared by all its picks. The lanes form S pick slots times
// 32 / S candidate groups (S the smallest power of two at least the number
// of picks, at most 32); each group takes every (32 / S)-th candidate of a
// chunk and the groups' counts are added with shuffles.
template <int D>
__global__ void __launch_bounds__(128) k_sap_rho_cells(BatchView v, CellWork w, SapproxBufs sb, int64_t ncells) {
    constexpr int DP = D <= 4 ? 1 : 2;
    __shared__ int4 sbuf[128 / 32][kChunk * DP];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int4* buf = sbuf[wid];
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long pairs = 0;
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; c < ncells; c += nwarps) {
        const uint32_t k0 = sb.pstart[c], k1 = sb.pstart[c + 1];
        if (k0 == k1) continue;
        const uint32_t cs = v.cell_start[c];
        const DsDesc& ds = v.desc[find_ds(v.pt_off, v.B, cs)];
        if (ds.d != D) continue;
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        const uint2* runs = w.runs + c * w.nbs;
        const uint32_t nr = w.nruns[c], ctot = w.cand[c];
        for (uint32_t g0 = k0; g0 < k1; g0 += 32) {
            const uint32_t np = min(32u, k1 - g0);
            int S = 1;
            while (S < (int)np) S <<= 1;
            const int G = 32 / S, slot = lane & (S - 1), grp = lane / S;
            const bool mine = (uint32_t)slot < np;
            const uint32_t p = sb.plist[g0 + (mine ? slot : 0)];
            int32_t x[D];
            sx_load<D>(recb + (int64_t)p * DP, x);
            uint32_t cnt = 0;
            CandStream<DP, false> cst;
            cst.init(runs, nr, 0, ctot);
            bool bad = false;
            while (cst.prep(lane, recb, nullptr, &bad)) {
                const int nb = (int)cst.cnt;
                __syncwarp();  // every lane is done with the previous chunk
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int f = lane + 32 * u;
                    if (f < nb) {
#pragma unroll
                        for (int q = 0; q < DP; ++q) buf[f * DP + q] = cst.r[u][q];
                    }
                }
                __syncwarp();
                for (int j = grp; j < nb; j += G) {
                    int32_t y[D];
                    sx_load<D>(buf + j * DP, y);
                    cnt += sx_dist<D>(x, y) < ds.d_cut2 ? 1u : 0u;
                }
            }
            for (int o = S; o < 32; o <<= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            if (bad && lane == 0) atomicOr(v.err, kErrStaging);
            if (mine && grp == 0) {
                v.rho_s[p] = (int32_t)cnt;
                v.rho[v.perm[p]] = (int32_t)cnt;
                pairs += ctot;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    if (lane == 0 && pairs) atomicAdd(&sb.stats[0], pairs);
}

// Work items of the pick path's density in the dense kernels: for every
// exact-grid cell holding picks, (cell, chunk of kQch picks, chunk of kch
// candidates).
__global__ void k_sap_item_count(CellWork w, SapproxBufs sb, int64_t ncells, int kch, uint32_t* nitem_c) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t np = sb.pstart[c + 1] - sb.pstart[c];
        const uint32_t cand = w.cand[c];
        const uint32_t nk = cand == 0u ? 1u : (cand + kch - 1) / kch;
        nitem_c[c] = np == 0u ? 0u : (np + kQch - 1) / kQch * nk;
    }
}

// Writes the items; a total above cap (which the host's bound rules out)
// raises the consistency flag and leaves no item to run.
__global__ void k_sap_fill_items(BatchView v, CellWork w, SapproxBufs sb, int64_t ncells, int kch,
                                 const uint32_t* item_off, uint4* items, uint32_t* nitems, int64_t cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && (int64_t)*nitems > cap) {
        *nitems = 0u;
        atomicOr(v.err, kErrStaging);
    }
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t np = sb.pstart[c + 1] - sb.pstart[c];
        if (np == 0u) continue;
        const uint32_t cand = w.cand[c];
        const uint32_t nq = (np + kQch - 1) / kQch, nk = cand == 0u ? 1u : (cand + kch - 1) / kch;
        if ((int64_t)item_off[c] + (int64_t)nq * nk > cap) continue;
        uint4* out = items + item_off[c];
        for (uint32_t q = 0; q < nq; ++q)
            for (uint32_t k = 0; k < nk; ++k) out[q * nk + k] = make_uint4((uint32_t)c, q, k, 0u);
    }
}

// A point that is not picked depends on its cell's pick.
__global__ void k_sap_follow(BatchView v, SapproxBufs sb) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const uint32_t k = sb.pick_s[p];
    if (k == (uint32_t)p) return;
    const int b = find_ds(v.pt_off, v.B, p);
    const DsDesc& ds = v.desc[b];
    const int4* rp = v.rec + ds.rec_off + (p - ds.pt_off) * ds.dp;
    const int4* rk = v.rec + ds.rec_off + ((int64_t)k - ds.pt_off) * ds.dp;
    long long dd = 0;
    for (int c = 0; c < ds.d; ++c) {
        const long long t = (long long)rec_coord(rp, c) - rec_coord(rk, c);
        dd += t * t;
    }
    const int64_t g = ds.pt_off + v.ro_s[p].y;
    v.dep[g] = (int32_t)v.ro_s[k].y;
    v.delta2[g] = dd;
}

__device__ __forceinline__ void keep_min(long long& d, uint32_t& j, long long d2, uint32_t j2) {
    if (d2 < d || (d2 == d && j2 < j)) {
        d = d2;
        j = j2;
    }
}

// Points that are not picked get rho 0, so that they rank after every pick.
__global__ void k_sap_mask(BatchView v) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const uint32_t g = v.perm[p];
    if (!v.pick[g]) {
        v.rho_s[p] = 0;
        v.rho[g] = 0;
    }
}

// Distance from the point to the outside of its searched block of
// exact-grid cells (capped at d_cut when the runs leave cells out).
__device__ __forceinline__ int64_t block_bound(const DsDesc& ds, const int4* r) {
    int64_t bound = INT64_MAX;
    for (int j = 0; j < ds.k; ++j) {
        const int32_t xi = rec_coord(r, ds.gdim[j]);
        const int64_t cj = cell_coord(ds, j, xi);
        if (cj - ds.R > 0) bound = min(bound, (int64_t)xi - (ds.origin[j] + (cj - ds.R) * ds.s) + 1);
        if (cj + ds.R + 1 < ds.ext[j]) bound = min(bound, ds.origin[j] + (cj + ds.R + 1) * ds.s - (int64_t)xi);
    }
    if (ds.prune) bound = min(bound, ds.d_cut);
    return bound;
}

// Every pick, one thread each: the densest pick; picks whose ring result
// (nearest higher pick of the searched block) lies strictly within d_cut;
// the others queue for the first-phase scan.
__global__ void k_sap_resolve(BatchView v, SapproxBufs sb) {
    const uint32_t m = *sb.npicks;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint32_t p = sb.picks[i];
    const DsDesc& ds = v.desc[find_ds(v.pt_off, v.B, p)];
    const uint2 ro = v.ro_s[p];
    const int64_t g = ds.pt_off + ro.y;
    if (ro.x == 0u) {
        v.dep[g] = -1;
        v.delta2[g] = INT64_MAX;
        return;
    }
    const unsigned long long bk = v.best_s[p];
    const long long dd = (long long)(bk >> 32);
    if (bk != ~0ull && dd < 0xffffffffll && dd < ds.d_cut2) {
        v.dep[g] = (int32_t)(uint32_t)bk;
        v.delta2[g] = dd;
        return;
    }
    sb.scan[atomicAdd(&sb.nscan[0], 1u)] = p;
}

// Both near-pass forms take a lane's candidate picks kNearBatch at a time:
// their list entries first, then their ranks and records together (a record
// is read whether or not its pick ranks higher), so that a lane waits for two
// memory round trips per batch instead of three per candidate.
constexpr int kNearBatch = 4;

// Pick path, every pick, one warp each: the nearest higher pick among the
// picks of its searched block (through the cells' pick lists: only the
// picks' own records are read). When
// it lies strictly within d_cut it is the nearest higher pick overall and
// belongs to N(c): the first-phase answer. Otherwise it is kept for the
// second phase and the pick queues for the full first-phase scan.
template <int D>
__global__ void __launch_bounds__(128) k_sap_near(BatchView v, CellWork w, SapproxBufs sb) {
    constexpr int DP = D <= 4 ? 1 : 2;
    const uint32_t m = *sb.npicks;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += nwarps) {
        const uint32_t p = sb.picks[i];
        const DsDesc& ds = v.desc[find_ds(v.pt_off, v.B, p)];
        if (ds.d != D) continue;
        const uint2 ro = v.ro_s[p];
        const int64_t g = ds.pt_off + ro.y;
        if (ro.x == 0u) {  // the densest pick
            if (lane == 0) {
                v.dep[g] = -1;
                v.delta2[g] = INT64_MAX;
            }
            continue;
        }
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        int32_t x[D];
        sx_load<D>(recb + (int64_t)p * DP, x);
        const uint32_t e = v.cell_of[p];
        const uint2* runs = w.runs + (int64_t)e * w.nbs;
        const uint32_t nr = w.nruns[e];
        long long bd = INT64_MAX;
        uint32_t bj = 0xffffffffu;
        for (uint32_t ri = 0; ri < nr; ++ri) {
            // the picks of the run's cells (a run is one or more whole cells,
            // consecutive in the sorted order, whose picks are consecutive too)
            const uint2 run = runs[ri];
            const uint32_t t0 = sb.pstart[v.cell_of[run.x]];
            const uint32_t t1 = sb.pstart[v.cell_of[run.x + run.y - 1] + 1];
            // kNearBatch candidates per lane in flight (lane + 32 u); past
            // the run's last pick a lane repeats it, which changes nothing
            for (uint32_t t = t0 + lane; t < t1; t += 32 * kNearBatch) {
                uint32_t q[kNearBatch];
#pragma unroll
                for (int u = 0; u < kNearBatch; ++u) q[u] = sb.plist[min(t + 32u * u, t1 - 1u)];
                uint2 cr[kNearBatch];
                int32_t y[kNearBatch][D];
#pragma unroll
                for (int u = 0; u < kNearBatch; ++u) {
                    cr[u] = v.ro_s[q[u]];
                    sx_load<D>(recb + (int64_t)q[u] * DP, y[u]);
                }
#pragma unroll
                for (int u = 0; u < kNearBatch; ++u)
                    if (cr[u].x < ro.x) keep_min(bd, bj, sx_dist<D>(x, y[u]), cr[u].y);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const long long b2 = __shfl_xor_sync(0xffffffffu, bd, o);
            const uint32_t bj2 = __shfl_xor_sync(0xffffffffu, bj, o);
            keep_min(bd, bj, b2, bj2);
        }
        if (lane != 0) continue;
        if (bj != 0xffffffffu && bd < ds.d_cut2) {
            v.dep[g] = (int32_t)bj;
            v.delta2[g] = bd;
            continue;
        }
        if (bd < 0xffffffffll) v.best_s[p] = ((unsigned long long)bd << 32) | bj;
        sb.scan[atomicAdd(&sb.nscan[0], 1u)] = p;
    }
}

// The same near pass with one thread per pick (a pick's block holds few
// picks on dense data: tens, against thousands of points), its candidates
// kNearBatch at a time as in the warp form.

template <int D>
__global__ void __launch_bounds__(128) k_sap_near_t(BatchView v, CellWork w, SapproxBufs sb) {
    constexpr int DP = D <= 4 ? 1 : 2;
    const uint32_t m = *sb.npicks;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = sb.picks[i];
        const DsDesc& ds = v.desc[find_ds(v.pt_off, v.B, p)];
        if (ds.d != D) continue;
        const uint2 ro = v.ro_s[p];
        const int64_t g = ds.pt_off + ro.y;
        if (ro.x == 0u) {  // the densest pick
            v.dep[g] = -1;
            v.delta2[g] = INT64_MAX;
            continue;
        }
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        int32_t x[D];
        sx_load<D>(recb + (int64_t)p * DP, x);
        const uint32_t e = v.cell_of[p];
        const uint2* runs = w.runs + (int64_t)e * w.nbs;
        const uint32_t nr = w.nruns[e];
        long long bd = INT64_MAX;
        uint32_t bj = 0xffffffffu;
        for (uint32_t ri = 0; ri < nr; ++ri) {
            const uint2 run = runs[ri];  // one or more whole cells
            const uint32_t t1 = sb.pstart[v.cell_of[run.x + run.y - 1] + 1];
            for (uint32_t t = sb.pstart[v.cell_of[run.x]]; t < t1; t += kNearBatch) {
                // past the run's last pick the batch repeats it, and a
                // repeated candidate changes nothing
                uint32_t q[kNearBatch];
#pragma unroll
                for (int u = 0; u < kNearBatch; ++u) q[u] = sb.plist[min(t + (uint32_t)u, t1 - 1u)];
                uint2 cr[kNearBatch];
                int32_t y[kNearBatch][D];
#pragma unroll
                for (int u = 0; u < kNearBatch; ++u) {
                    cr[u] = v.ro_s[q[u]];
                    sx_load<D>(recb + (int64_t)q[u] * DP, y[u]);
                }
#pragma unroll
                for (int u = 0; u < kNearBatch; ++u)
                    if (cr[u].x < ro.x) keep_min(bd, bj, sx_dist<D>(x, y[u]), cr[u].y);
            }
        }
        if (bj != 0xffffffffu && bd < ds.d_cut2) {
            v.dep[g] = (int32_t)bj;
            v.delta2[g] = bd;
            continue;
        }
        if (bd < 0xffffffffll) v.best_s[p] = ((unsigned long long)bd << 32) | bj;
        sb.scan[atomicAdd(&sb.nscan[0], 1u)] = p;
    }
}

// First phase for the queued picks: one warp per pick scans the neighbour
// runs of its exact-grid cell for points strictly within d_cut in other
// cells of G', and keeps the nearest of their cells' picks that rank
// higher. A pick without one goes to the second phase.
template <int D>
__global__ void __launch_bounds__(128) k_sap_first(BatchView v, CellWork w, SapproxBufs sb, DeltaBufs db) {
    constexpr int DP = D <= 4 ? 1 : 2;
    const uint32_t m = sb.nscan[0];
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += nwarps) {
        const uint32_t p = sb.scan[i];
        const DsDesc& ds = v.desc[find_ds(v.pt_off, v.B, p)];
        if (ds.d != D) continue;
        const uint2 ro = v.ro_s[p];
        const int64_t g = ds.pt_off + ro.y;
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        int32_t x[D];
        sx_load<D>(recb + (int64_t)p * DP, x);
        const uint32_t e = v.cell_of[p];
        const uint2* runs = w.runs + (int64_t)e * w.nbs;
        const uint32_t nr = w.nruns[e];
        long long fd = INT64_MAX, bd = INT64_MAX;
        uint32_t fj = 0xffffffffu, bj = 0xffffffffu;
        for (uint32_t ri = 0; ri < nr; ++ri) {
            const uint2 run = runs[ri];
            for (uint32_t q = run.x + lane; q < run.x + run.y; q += 32) {
                // only a point whose cell of G' has a higher pick matters
                // (its rank first: the pick's record is shared by its cell)
                const uint32_t k = sb.pick_s[q];
                if (k == p) continue;
                const uint2 kr = v.ro_s[k];
                if (kr.x >= ro.x) continue;
                int32_t y[D];
                sx_load<D>(recb + (int64_t)q * DP, y);
                const long long dq = sx_dist<D>(x, y);
                // a higher pick: the nearest of the block, for the second phase
                if (k == q) keep_min(bd, bj, dq, kr.y);
                if (dq >= ds.d_cut2) continue;
                int32_t z[D];
                sx_load<D>(recb + (int64_t)k * DP, z);
                keep_min(fd, fj, sx_dist<D>(x, z), kr.y);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const long long f2 = __shfl_xor_sync(0xffffffffu, fd, o);
            const uint32_t fj2 = __shfl_xor_sync(0xffffffffu, fj, o);
            keep_min(fd, fj, f2, fj2);
            const long long b2 = __shfl_xor_sync(0xffffffffu, bd, o);
            const uint32_t bj2 = __shfl_xor_sync(0xffffffffu, bj, o);
            keep_min(bd, bj, b2, bj2);
        }
        if (lane != 0) continue;
        if (fj != 0xffffffffu) {
            v.dep[g] = (int32_t)fj;
            v.delta2[g] = fd;
            continue;
        }
        // second phase: the nearest higher pick of the searched block (this
        // scan's, or the ring search's when it ran), when proven, else the
        // exact passes
        atomicAdd(&sb.stats[1], 1ull);
        const unsigned long long bk = v.best_s[p];
        if (bk != ~0ull && (uint32_t)(bk >> 32) != 0xffffffffu)
            keep_min(bd, bj, (long long)(bk >> 32), (uint32_t)bk);
        const int64_t bound = block_bound(ds, recb + (int64_t)p * DP);
        const bool proven = bj != 0xffffffffu &&
                            (bound == INT64_MAX || (bound < 3037000499ll && bd < bound * bound));
        if (proven) {
            v.dep[g] = (int32_t)bj;
            v.delta2[g] = bd;
            continue;
        }
        // the unproven best is a valid start for the tree search
        if (bd < 0xffffffffll) v.best_s[p] = ((unsigned long long)bd << 32) | bj;
        if (ro.x < db.bf_rank) {
            db.bf_list[atomicAdd(&db.ucount[1], 1u)] = p;
        } else {
            db.tree_list[atomicAdd(&db.ucount[0], 1u)] = p;
        }
    }
}

// rho as reported: -1 for the points that are not picked.
__global__ void k_sap_rho_out(BatchView v, int32_t* out) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= v.N) return;
    out[g] = v.pick[g] ? v.rho[g] : -1;
}

unsigned warp_blocks(int64_t bound) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(152 * 16, grid_for(bound, 4)));
}

}  // namespace

cudaError_t launch_sapprox_grid(const BatchView& v, const SapproxBufs& sb, int key_bits, int bshift, void* temp,
                                cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    // LSD over 64-bit words: each pass sorts the previous order stably by
    // the next more significant word
    const int words = std::max(1, (key_bits + 63) / 64);
    const int64_t N = v.N;
    uint64_t *kin = sb.keys, *kout = sb.keys + N, *ktmp = sb.keys + 2 * N;
    uint32_t *vin = sb.ord + N, *vout = sb.ord, *vtmp = sb.ord + 2 * N;
    const uint32_t* prev = nullptr;
    for (int w = 0; w < words; ++w) {
        const int nbits = std::max(1, std::min(64, key_bits - 64 * w));
        (k_sap_keys<<<grid_for(N, 256), 256, 0, st>>>(v, prev, kin, vin, w, bshift), note_launch());
        cudaError_t e = radix_sort_u64(kin, vin, kout, vout, ktmp, vtmp, N, nbits, temp, st);
        if (e != cudaSuccess) return e;
        // the sorted order (vout) feeds the next pass; its values go to vin
        prev = vout;
        std::swap(vin, vout);
        std::swap(vin, vtmp);
    }
    SapproxBufs s2 = sb;
    s2.ord = const_cast<uint32_t*>(prev);
    (k_sap_flags<<<grid_for(N, 256), 256, 0, st>>>(v, s2, words, bshift), note_launch());
    cudaError_t e = exclusive_scan_u32(s2.flag, s2.cidx, N, nullptr, temp, st);
    if (e != cudaSuccess) return e;
    (k_sap_picks<<<grid_for(N, 256), 256, 0, st>>>(v, s2, N), note_launch());
    (k_sap_pick_of<<<grid_for(N, 256), 256, 0, st>>>(v, s2, N), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_sapprox_plist(const BatchView& v, const SapproxBufs& sb, int64_t ncells, void* temp,
                                 cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    (k_sap_pflag<<<grid_for(v.N, 256), 256, 0, st>>>(v, sb), note_launch());
    cudaError_t e = exclusive_scan_u32(sb.pflag, sb.ppos, v.N, nullptr, temp, st);
    if (e != cudaSuccess) return e;
    (k_sap_plist<<<grid_for(std::max<int64_t>(v.N, ncells + 1), 256), 256, 0, st>>>(v, sb, ncells), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_sapprox_items(const BatchView& v, const CellWork& w, const SapproxBufs& sb, int64_t ncells, int kch,
                                 uint32_t* nitem_c, uint32_t* item_off, uint4* items, uint32_t* nitems, int64_t cap,
                                 void* temp, cudaStream_t st) {
    if (ncells <= 0) return cudaMemsetAsync(nitems, 0, sizeof(uint32_t), st);
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(ncells, 256));
    (k_sap_item_count<<<blocks, 256, 0, st>>>(w, sb, ncells, kch, nitem_c), note_launch());
    cudaError_t e = exclusive_scan_u32(nitem_c, item_off, ncells, nitems, temp, st);
    if (e != cudaSuccess) return e;
    (k_sap_fill_items<<<blocks, 256, 0, st>>>(v, w, sb, ncells, kch, item_off, items, nitems, cap), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_sapprox_pick_pairs(const BatchView& v, const CellWork& w, const SapproxBufs& sb,
                                     int64_t picks_bound, cudaStream_t st) {
    if (v.N == 0 || picks_bound <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 8, grid_for(picks_bound, 256));
    (k_sap_pick_pairs<<<blocks, 256, 0, st>>>(v, w, sb), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_sapprox_rho(const BatchView& v, const CellWork& w, const SapproxBufs& sb, uint32_t dim_mask,
                               int64_t picks_bound, int64_t ncells, bool by_cell, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    const unsigned blocks = warp_blocks(by_cell ? ncells : picks_bound);
#define DPC_SAP_RHO(D)                                                                          \
    if (dim_mask & (1u << (D - 1))) {                                                           \
        if (by_cell) (k_sap_rho_cells<D><<<blocks, 128, 0, st>>>(v, w, sb, ncells), note_launch()); \
        else (k_sap_rho<D><<<blocks, 128, 0, st>>>(v, w, sb), note_launch());                   \
    }
    DPC_SAP_RHO(1) DPC_SAP_RHO(2) DPC_SAP_RHO(3) DPC_SAP_RHO(4)
    DPC_SAP_RHO(5) DPC_SAP_RHO(6) DPC_SAP_RHO(7) DPC_SAP_RHO(8)
#undef DPC_SAP_RHO
    return cudaGetLastError();
}

cudaError_t launch_sapprox_mask(const BatchView& v, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    (k_sap_mask<<<grid_for(v.N, 256), 256, 0, st>>>(v), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_sapprox_first(const BatchView& v, const CellWork& w, const SapproxBufs& sb, const DeltaBufs& db,
                                 uint32_t dim_mask, int64_t picks_bound, int64_t scan_bound, bool near_pass,
                                 bool near_threads, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    (k_sap_follow<<<grid_for(v.N, 256), 256, 0, st>>>(v, sb), note_launch());
    if (near_pass) {
        const unsigned nb = near_threads ? (unsigned)std::max<int64_t>(1, std::min<int64_t>(152 * 32, grid_for(picks_bound, 128)))
                                         : warp_blocks(picks_bound);
#define DPC_SAP_NEAR(D)                                                                            \
    if (dim_mask & (1u << (D - 1))) {                                                              \
        if (near_threads) (k_sap_near_t<D><<<nb, 128, 0, st>>>(v, w, sb), note_launch());          \
        else (k_sap_near<D><<<nb, 128, 0, st>>>(v, w, sb), note_launch());                        \
    }
        DPC_SAP_NEAR(1) DPC_SAP_NEAR(2) DPC_SAP_NEAR(3) DPC_SAP_NEAR(4)
        DPC_SAP_NEAR(5) DPC_SAP_NEAR(6) DPC_SAP_NEAR(7) DPC_SAP_NEAR(8)
#undef DPC_SAP_NEAR
    } else {
        (k_sap_resolve<<<grid_for(std::max<int64_t>(picks_bound, 1), 256), 256, 0, st>>>(v, sb), note_launch());
    }
    const unsigned blocks = warp_blocks(scan_bound);
#define DPC_SAP_FIRST(D) \
    if (dim_mask & (1u << (D - 1))) (k_sap_first<D><<<blocks, 128, 0, st>>>(v, w, sb, db), note_launch());
    DPC_SAP_FIRST(1) DPC_SAP_FIRST(2) DPC_SAP_FIRST(3) DPC_SAP_FIRST(4)
    DPC_SAP_FIRST(5) DPC_SAP_FIRST(6) DPC_SAP_FIRST(7) DPC_SAP_FIRST(8)
#undef DPC_SAP_FIRST
    return cudaGetLastError();
}

cudaError_t launch_sapprox_rho_out(const BatchView& v, int32_t* out, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    (k_sap_rho_out<<<grid_for(v.N, 256), 256, 0, st>>>(v, out), note_launch());
    return cudaGetLastError();
}

}  // namespace dpc
