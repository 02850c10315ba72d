// Dependent point and dependent distance (Definitions 2 and 3).
//
// "Higher" is the total order (rho desc, index asc): Ex-DPC sorts the points
// by density and gives each one the nearest neighbour among the points ahead
// of it (Section 3, "Dependent point computation", steps 2-4); with a stable
// sort the points ahead of p_i are exactly those of smaller rank. The
// dependent point is the lexicographic minimum of (squared distance,
// original index) over them; the rank-0 point has none (delta = infinity).
//
// Ex-DPC's one-by-one kd-tree insertion is sequential (Section 3,
// "Implementation for parallel processing"). Here every point searches in
// parallel, in three passes:
//  1. ring search: the cell of p_i and its neighbours (rings 0..R of the
//     grid), same work split as the density stage, keeping the packed key
//     (min(D, 2^32-1) << 32 | index) of the best higher point. When the best
//     distance is below the distance from p_i to the outside of the searched
//     box, no unseen point can beat it and p_i is resolved.
//  2. points still open with a small rank (the density peaks) go to a tiled
//     brute-force pass over the higher-ranked prefix of their dataset, staged
//     through shared memory (cf. the exact step of Approx-DPC, Section 4.3,
//     which scans only the subsets of higher density);
//  3. the other open points continue the expanding search over a tree of
//     boxes over the Morton-ordered points; each node keeps its box and the
//     smallest rank inside it, so a node is skipped when nothing in it ranks
//     higher or when its box is farther than the best distance so far.
#include "stages.cuh"
#include <algorithm>

namespace dpc {

namespace {

constexpr int kThreads = 256;
constexpr int kCb = 128;
constexpr unsigned long long kNoBest = ~0ull;
constexpr uint32_t kSat = 0xffffffffu;

template <int D>
__device__ __forceinline__ void load_pt(const int4* r, int32_t (&x)[D]) {
    const int4 a = r[0];
    int32_t t[8] = {a.x, a.y, a.z, a.w, 0, 0, 0, 0};
    if (D > 4) {
        const int4 bq = r[1];
        t[4] = bq.x; t[5] = bq.y; t[6] = bq.z; t[7] = bq.w;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = t[k];
}

// Squared distance, saturated to 2^32 - 1 (exact below it).
template <int D, bool W64>
__device__ __forceinline__ uint32_t dist_sat(const int32_t (&q)[D], const int32_t (&c)[D]) {
    if (W64) {
        unsigned long long s = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const long long dd = (long long)q[k] - c[k];
            s += (unsigned long long)(dd * dd);
        }
        return s >= kSat ? kSat : (uint32_t)s;
    } else {
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int dd = q[k] - c[k];
            s += (uint32_t)(dd * dd);
        }
        return s;
    }
}

template <int D>
__device__ __forceinline__ long long dist64(const int32_t (&q)[D], const int32_t (&c)[D]) {
    long long s = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const long long dd = (long long)q[k] - c[k];
        s += dd * dd;
    }
    return s;
}

// ------------------------------------------------------------- rank sort

__global__ void k_rank_keys(BatchView v, int rbits, bool key64, void* keys, uint32_t* vals) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= v.N) return;
    const int b = find_ds(v.pt_off, v.B, g);
    const uint64_t k = ((uint64_t)b << rbits) | (((1ull << rbits) - 1ull) - (uint64_t)v.rho[g]);
    if (key64) reinterpret_cast<uint64_t*>(keys)[g] = k;
    else reinterpret_cast<uint32_t*>(keys)[g] = (uint32_t)k;
    vals[g] = (uint32_t)g;
}

__global__ void k_rank_from_order(BatchView v) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= v.N) return;
    const int b = find_ds(v.pt_off, v.B, r);
    v.rank[v.order[r]] = (uint32_t)(r - v.pt_off[b]);
}

__global__ void k_ro(BatchView v) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const int b = find_ds(v.pt_off, v.B, p);
    const uint32_t g = v.perm[p];
    v.ro_s[p] = make_uint2(v.rank[g], (uint32_t)(g - v.pt_off[b]));
}

// ----------------------------------------------------------- ring search

template <int D, bool W64, int Q>
__device__ __forceinline__ void eval_ring(const int4* buf, const uint2* rbuf, int nb, const int32_t (&qx)[4][D],
                                          const uint32_t (&qr)[4], unsigned long long (&best)[4]) {
    constexpr int DP = D <= 4 ? 1 : 2;
#pragma unroll 2
    for (int j = 0; j < nb; ++j) {
        int32_t c[D];
        load_pt<D>(buf + j * DP, c);
        const uint2 ro = rbuf[j];
#pragma unroll
        for (int t = 0; t < Q; ++t) {
            const uint32_t dd = dist_sat<D, W64>(qx[t], c);
            const unsigned long long key = ((unsigned long long)dd << 32) | ro.y;
            if (ro.x < qr[t] && key < best[t]) best[t] = key;
        }
    }
}

template <int D, bool W64>
__global__ void __launch_bounds__(kThreads) k_ring_dense(BatchView v, CellWork w, uint32_t* counter) {
    constexpr int DP = D <= 4 ? 1 : 2;
    __shared__ int4 sbuf[kThreads / 32][kCb * DP];
    __shared__ uint2 srb[kThreads / 32][kCb];
    const int lane = threadIdx.x & 31;
    int4* buf = sbuf[threadIdx.x >> 5];
    uint2* rbuf = srb[threadIdx.x >> 5];
    const uint32_t nitems = *w.nitems;
    while (true) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(counter, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nitems) break;
        const uint4 item = w.items[it];
        const uint32_t dc = item.x, qc = item.y, kc = item.z;
        const uint32_t c = w.dense[dc];
        const uint32_t cs = v.cell_start[c], m = v.cell_start[c + 1] - cs;
        const int b = find_ds(v.pt_off, v.B, cs);
        const DsDesc& ds = v.desc[b];
        if (ds.d != D || (ds.w32 == 0) != W64) continue;
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        const int q0 = (int)qc * kQch;
        const int nq = min(kQch, (int)m - q0);
        const int Q = (nq + 31) >> 5;
        int32_t qx[4][D];
        uint32_t qr[4];
        unsigned long long best[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int qi = min(lane + 32 * t, nq - 1);
            load_pt<D>(recb + ((int64_t)cs + q0 + qi) * DP, qx[t]);
            qr[t] = v.ro_s[cs + q0 + qi].x;
            best[t] = kNoBest;
        }
        const uint2* runs = w.runs + (int64_t)dc * kMaxNb;
        const uint32_t nr = w.nruns[dc], ctot = w.cand[dc];
        const uint32_t k0 = kc * (uint32_t)w.kch;
        uint32_t remaining = min(ctot, k0 + (uint32_t)w.kch) - k0;
        uint32_t ri = 0, roff = k0;
        while (ri < nr) {
            const uint32_t len = runs[ri].y;
            if (roff < len) break;
            roff -= len;
            ++ri;
        }
        while (remaining > 0u) {
            int nb = 0;
            while (nb < kCb && remaining > 0u) {
                const uint2 run = ri < nr ? runs[ri] : make_uint2(0u, 0u);
                const uint32_t take = ri < nr ? min(min(run.y - roff, (uint32_t)(kCb - nb)), remaining) : 0u;
                if (take == 0u) {  // runs exhausted early: cannot happen when counts agree
                    if (lane == 0) atomicOr(v.err, kErrStaging);
                    remaining = 0u;
                    break;
                }
                const int4* src = recb + ((int64_t)run.x + roff) * DP;
                for (uint32_t t = lane; t < take * DP; t += 32) buf[nb * DP + t] = __ldg(src + t);
                for (uint32_t t = lane; t < take; t += 32) rbuf[nb + t] = v.ro_s[run.x + roff + t];
                nb += (int)take;
                roff += take;
                remaining -= take;
                if (roff == run.y) {
                    ++ri;
                    roff = 0;
                }
            }
            __syncwarp();
            switch (Q) {
                case 1: eval_ring<D, W64, 1>(buf, rbuf, nb, qx, qr, best); break;
                case 2: eval_ring<D, W64, 2>(buf, rbuf, nb, qx, qr, best); break;
                case 3: eval_ring<D, W64, 3>(buf, rbuf, nb, qx, qr, best); break;
                default: eval_ring<D, W64, 4>(buf, rbuf, nb, qx, qr, best); break;
            }
            __syncwarp();
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (lane + 32 * t < nq && best[t] != kNoBest) atomicMin(&v.best_s[cs + q0 + lane + 32 * t], best[t]);
    }
}

template <int D, bool W64>
__global__ void __launch_bounds__(256) k_ring_sparse(BatchView v, CellWork w) {
    constexpr int DP = D <= 4 ? 1 : 2;
    const uint32_t ns = *w.nsparse;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = w.sparse[i];
        const uint32_t cs = v.cell_start[c], m = v.cell_start[c + 1] - cs;
        const int b = find_ds(v.pt_off, v.B, cs);
        const DsDesc& ds = v.desc[b];
        if (ds.d != D || (ds.w32 == 0) != W64) continue;
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        int32_t qx[kSparseMax][D];
        uint32_t qr[kSparseMax];
        unsigned long long best[kSparseMax];
#pragma unroll
        for (int t = 0; t < kSparseMax; ++t) {
            const uint32_t qi = min((uint32_t)t, m - 1);
            load_pt<D>(recb + ((int64_t)cs + qi) * DP, qx[t]);
            qr[t] = v.ro_s[cs + qi].x;
            best[t] = kNoBest;
        }
        int32_t cc[kMaxGridDims];
        for (int j = 0; j < ds.k; ++j) cc[j] = cell_coord(ds, j, rec_coord(recb + (int64_t)cs * DP, ds.gdim[j]));
        const int nnb = num_neighbours(ds);
        for (int t = 0; t < nnb; ++t) {
            int32_t nc[kMaxGridDims];
            if (!neighbour(ds, cc, t, nc)) continue;
            const uint2 e = hash_find(v.hash, v.hmask, ds.cbase + morton(nc, ds.k, ds.mbits));
            for (uint32_t j = 0; j < e.y; ++j) {
                int32_t cj[D];
                load_pt<D>(recb + ((int64_t)e.x + j) * DP, cj);
                const uint2 ro = v.ro_s[e.x + j];
#pragma unroll
                for (int q = 0; q < kSparseMax; ++q) {
                    const uint32_t dd = dist_sat<D, W64>(qx[q], cj);
                    const unsigned long long key = ((unsigned long long)dd << 32) | ro.y;
                    if (ro.x < qr[q] && key < best[q]) best[q] = key;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kSparseMax; ++q)
            if ((uint32_t)q < m) v.best_s[cs + q] = best[q];
    }
}

// Resolve the points whose ring-search result is provably final; queue the
// others for the brute-force pass (rank < bf_rank) or the tree search.
__global__ void k_finalize(BatchView v, DeltaBufs db) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const int b = find_ds(v.pt_off, v.B, p);
    const DsDesc& ds = v.desc[b];
    const uint2 ro = v.ro_s[p];
    const int64_t g = ds.pt_off + ro.y;
    if (ro.x == 0u) {  // the densest point: no dependent point, delta = infinity
        v.dep[g] = -1;
        v.delta2[g] = INT64_MAX;
        return;
    }
    const unsigned long long bk = v.best_s[p];
    const uint32_t dd = (uint32_t)(bk >> 32);
    // distance from the point to the outside of the searched box of cells
    const int4* r = v.rec + ds.rec_off + (p - ds.pt_off) * ds.dp;
    int64_t bound = INT64_MAX;
    for (int j = 0; j < ds.k; ++j) {
        const int64_t x = rec_coord(r, ds.gdim[j]);
        const int64_t cj = (x - ds.origin[j]) / ds.s;
        if (cj - ds.R > 0) bound = min(bound, x - (ds.origin[j] + (cj - ds.R) * ds.s) + 1);
        if (cj + ds.R + 1 < ds.ext[j]) bound = min(bound, ds.origin[j] + (cj + ds.R + 1) * ds.s - x);
    }
    const bool found = bk != kNoBest && dd != kSat;
    const bool resolved = found && (bound == INT64_MAX || (int64_t)dd < bound * bound);
    if (resolved) {
        v.dep[g] = (int32_t)(uint32_t)bk;
        v.delta2[g] = (int64_t)dd;
    } else if (ro.x < db.bf_rank) {
        db.bf_list[atomicAdd(&db.ucount[1], 1u)] = (uint32_t)p;
    } else {
        db.tree_list[atomicAdd(&db.ucount[0], 1u)] = (uint32_t)p;
    }
}

// ---------------------------------------------------------------- tree

__device__ __forceinline__ int find_slot_ds(const int64_t* slot_off, int B, int64_t s) {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (slot_off[mid] <= s) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Leaf boxes and smallest ranks, then a bottom-up refit: the second child
// to finish computes its parent.
__global__ void k_tree_build(BatchView v, DeltaBufs db) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= db.leaf_slots) return;
    const int b = find_slot_ds(db.slot_off, v.B, s);
    const DsDesc& ds = v.desc[b];
    const int64_t leaf = s - db.slot_off[b];
    int64_t node = (1ll << ds.h) + leaf;
    int32_t lo[8], hi[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        lo[k] = INT32_MAX;
        hi[k] = INT32_MIN;
    }
    uint32_t mr = 0xffffffffu;
    const int64_t p0 = ds.pt_off + leaf * kLeaf;
    const int64_t p1 = min(p0 + kLeaf, ds.pt_off + (int64_t)ds.n);
    for (int64_t p = p0; p < p1; ++p) {
        const int4* r = v.rec + ds.rec_off + (p - ds.pt_off) * ds.dp;
        const int4 a = r[0];
        const int4 c = ds.dp == 2 ? r[1] : make_int4(0, 0, 0, 0);
        const int32_t x[8] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            lo[k] = min(lo[k], x[k]);
            hi[k] = max(hi[k], x[k]);
        }
        mr = min(mr, v.ro_s[p].x);
    }
    int4* nb = db.node_box + (ds.node_off + node) * 4;
    nb[0] = make_int4(lo[0], lo[1], lo[2], lo[3]);
    nb[1] = make_int4(lo[4], lo[5], lo[6], lo[7]);
    nb[2] = make_int4(hi[0], hi[1], hi[2], hi[3]);
    nb[3] = make_int4(hi[4], hi[5], hi[6], hi[7]);
    db.node_minrank[ds.node_off + node] = mr;
    while (node > 1) {
        __threadfence();
        const int64_t parent = node >> 1;
        if (atomicAdd(&db.node_flag[ds.node_off + parent], 1u) == 0u) return;
        __threadfence();
        const int4* cl = db.node_box + (ds.node_off + 2 * parent) * 4;
        const int4* cr = cl + 4;
        int4 q[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int4 x = __ldcg(cl + i), y = __ldcg(cr + i);
            q[i] = i < 2 ? make_int4(min(x.x, y.x), min(x.y, y.y), min(x.z, y.z), min(x.w, y.w))
                         : make_int4(max(x.x, y.x), max(x.y, y.y), max(x.z, y.z), max(x.w, y.w));
        }
        int4* pb = db.node_box + (ds.node_off + parent) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) pb[i] = q[i];
        db.node_minrank[ds.node_off + parent] = min(__ldcg(&db.node_minrank[ds.node_off + 2 * parent]),
                                                    __ldcg(&db.node_minrank[ds.node_off + 2 * parent + 1]));
        node = parent;
    }
}

template <int D>
__device__ __forceinline__ long long box_dist(const int4* nb, const int32_t (&x)[D]) {
    const int4 l0 = nb[0], h0 = nb[2];
    int32_t lo[8] = {l0.x, l0.y, l0.z, l0.w, 0, 0, 0, 0};
    int32_t hi[8] = {h0.x, h0.y, h0.z, h0.w, 0, 0, 0, 0};
    if (D > 4) {
        const int4 l1 = nb[1], h1 = nb[3];
        lo[4] = l1.x; lo[5] = l1.y; lo[6] = l1.z; lo[7] = l1.w;
        hi[4] = h1.x; hi[5] = h1.y; hi[6] = h1.z; hi[7] = h1.w;
    }
    long long s = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const long long dd = x[k] < lo[k] ? (long long)lo[k] - x[k] : (x[k] > hi[k] ? (long long)x[k] - hi[k] : 0);
        s += dd * dd;
    }
    return s;
}

template <int D>
__global__ void __launch_bounds__(128) k_tree_search(BatchView v, DeltaBufs db) {
    constexpr int DP = D <= 4 ? 1 : 2;
    const uint32_t cnt = db.ucount[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = db.tree_list[i];
        const int b = find_ds(v.pt_off, v.B, p);
        const DsDesc& ds = v.desc[b];
        if (ds.d != D) continue;
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        int32_t x[D];
        load_pt<D>(recb + (int64_t)p * DP, x);
        const uint2 ro = v.ro_s[p];
        long long bestD = INT64_MAX;
        uint32_t bestJ = 0xffffffffu;
        const unsigned long long bk = v.best_s[p];
        if (bk != kNoBest && (uint32_t)(bk >> 32) != kSat) {
            bestD = (long long)(bk >> 32);
            bestJ = (uint32_t)bk;
        }
        const int4* boxes = db.node_box + ds.node_off * 4;
        const uint32_t* minrank = db.node_minrank + ds.node_off;
        const int64_t first_leaf = 1ll << ds.h;
        constexpr int kStack = 64;
        int64_t stack[kStack];
        int sp = 0;
        stack[sp++] = 1;
        while (sp > 0) {
            const int64_t nd = stack[--sp];
            if (minrank[nd] >= ro.x) continue;
            if (box_dist<D>(boxes + nd * 4, x) > bestD) continue;
            if (nd >= first_leaf) {
                const int64_t q0 = ds.pt_off + (nd - first_leaf) * kLeaf;
                const int64_t q1 = min(q0 + kLeaf, ds.pt_off + (int64_t)ds.n);
                for (int64_t q = q0; q < q1; ++q) {
                    const uint2 cr = v.ro_s[q];
                    if (cr.x >= ro.x) continue;
                    int32_t c[D];
                    load_pt<D>(recb + q * DP, c);
                    const long long dd = dist64<D>(x, c);
                    if (dd < bestD || (dd == bestD && cr.y < bestJ)) {
                        bestD = dd;
                        bestJ = cr.y;
                    }
                }
            } else if (sp + 2 > kStack) {
                atomicOr(v.err, kErrTreeStack);
            } else {
                const int64_t l = 2 * nd, r = l + 1;
                const long long dl = minrank[l] < ro.x ? box_dist<D>(boxes + l * 4, x) : INT64_MAX;
                const long long dr = minrank[r] < ro.x ? box_dist<D>(boxes + r * 4, x) : INT64_MAX;
                // push the farther child first so the nearer one is searched first
                if (dl <= dr) {
                    if (dr <= bestD) stack[sp++] = r;
                    if (dl <= bestD) stack[sp++] = l;
                } else {
                    if (dl <= bestD) stack[sp++] = l;
                    if (dr <= bestD) stack[sp++] = r;
                }
            }
        }
        const int64_t g = ds.pt_off + ro.y;
        v.dep[g] = (int32_t)bestJ;
        v.delta2[g] = bestD;
    }
}

// --------------------------------------------------------- brute force

__global__ void k_bf_prefix(BatchView v, DeltaBufs db) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= v.N) return;
    const uint32_t r = v.rank[g];
    if (r >= db.bf_rank) return;
    const int b = find_ds(v.pt_off, v.B, g);
    const DsDesc& ds = v.desc[b];
    const int64_t pos = ds.pt_off + r;
    const int4* src = v.rec + ds.rec_off + ((int64_t)v.pos_of[g] - ds.pt_off) * ds.dp;
    db.rrec[pos * 2] = src[0];
    db.rrec[pos * 2 + 1] = ds.dp == 2 ? src[1] : make_int4(0, 0, 0, 0);
    db.rorig[pos] = (uint32_t)(g - ds.pt_off);
}

__global__ void k_bf_keys(BatchView v, DeltaBufs db) {
    const uint32_t cnt = db.ucount[1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = db.bf_list[i];
        const int b = find_ds(v.pt_off, v.B, p);
        db.bf_keys[i] = (uint32_t)(v.pt_off[b] + v.ro_s[p].x);
    }
}

constexpr int kBfThreads = 128;
constexpr int kBfTile = 256;

// One thread per open point, the block's points consecutive in global rank
// order; the union of their higher-ranked prefixes streams through shared
// memory in tiles and every thread keeps the candidates of its own prefix.
template <int D>
__global__ void __launch_bounds__(kBfThreads) k_bruteforce(BatchView v, DeltaBufs db) {
    __shared__ int4 tile[kBfTile * 2];
    __shared__ uint32_t torig[kBfTile];
    __shared__ int64_t s_lo, s_hi;
    const uint32_t cnt = db.ucount[1];
    const int64_t i = (int64_t)blockIdx.x * kBfThreads + threadIdx.x;
    if ((int64_t)blockIdx.x * kBfThreads >= cnt) return;
    if (threadIdx.x == 0) {
        s_lo = INT64_MAX;
        s_hi = 0;
    }
    __syncthreads();
    const bool valid = i < cnt;
    uint32_t p = 0;
    int b = 0;
    int64_t my_lo = 0, my_hi = 0;  // candidate positions [my_lo, my_hi) in global rank order
    bool mine = false;
    if (valid) {
        p = db.bf_sorted[i];
        b = find_ds(v.pt_off, v.B, p);
        my_lo = v.pt_off[b];
        my_hi = my_lo + v.ro_s[p].x;
        mine = v.desc[b].d == D;
        atomicMin((unsigned long long*)&s_lo, (unsigned long long)my_lo);
        atomicMax((unsigned long long*)&s_hi, (unsigned long long)my_hi);
    }
    __syncthreads();
    int32_t x[D];
    if (valid) {
        const DsDesc& ds = v.desc[b];
        const int4* r = v.rec + ds.rec_off + ((int64_t)p - ds.pt_off) * ds.dp;
        load_pt<D>(r, x);
    }
    long long bestD = INT64_MAX;
    uint32_t bestJ = 0xffffffffu;
    for (int64_t base = s_lo; base < s_hi; base += kBfTile) {
        const int64_t nt = min((int64_t)kBfTile, s_hi - base);
        for (int t = threadIdx.x; t < nt * 2; t += kBfThreads) tile[t] = db.rrec[base * 2 + t];
        for (int t = threadIdx.x; t < nt; t += kBfThreads) torig[t] = db.rorig[base + t];
        __syncthreads();
        if (mine) {
            const int64_t j0 = max((int64_t)0, my_lo - base), j1 = min(nt, my_hi - base);
            for (int64_t j = j0; j < j1; ++j) {
                int32_t c[D];
                load_pt<D>(tile + 2 * j, c);
                const long long dd = dist64<D>(x, c);
                const uint32_t o = torig[j];
                if (dd < bestD || (dd == bestD && o < bestJ)) {
                    bestD = dd;
                    bestJ = o;
                }
            }
        }
        __syncthreads();
    }
    if (mine) {
        const int64_t g = v.pt_off[b] + v.ro_s[p].y;
        v.dep[g] = (int32_t)bestJ;
        v.delta2[g] = bestD;
    }
}

template <int D, bool W64>
void launch_ring_class(const BatchView& v, const CellWork& w, int64_t nitems_bound, int64_t nsparse_bound,
                       uint32_t* counter, cudaStream_t st) {
    if (nitems_bound > 0) {
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(152 * 8, (nitems_bound + 7) / 8));
        (k_ring_dense<D, W64><<<blocks, kThreads, 0, st>>>(v, w, counter), note_launch());
    }
    if (nsparse_bound > 0) {
        const unsigned blocks = (unsigned)std::min<int64_t>(152 * 32, grid_for(nsparse_bound, 256));
        (k_ring_sparse<D, W64><<<blocks, 256, 0, st>>>(v, w), note_launch());
    }
}

}  // namespace

cudaError_t launch_rank(const BatchView& v, const DeltaBufs& db, int rbits, void* sort_temp, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    int bbits = 0;
    while ((1ll << bbits) < v.B) ++bbits;
    const int nbits = bbits + rbits;
    const bool key64 = nbits > 32;
    // key and value buffers: rkeys holds 3 key arrays (in, tmp, out) of the
    // chosen width; rvals holds in + tmp, v.order receives the result
    char* kb = reinterpret_cast<char*>(db.rkeys);
    const size_t ks = (key64 ? 8 : 4) * (size_t)v.N;
    void* kin = kb;
    void* ktmp = kb + ((ks + 255) & ~size_t(255));
    void* kout = kb + 2 * ((ks + 255) & ~size_t(255));
    uint32_t* vin = db.rvals;
    uint32_t* vtmp = db.rvals + ((v.N + 63) & ~int64_t(63));
    (k_rank_keys<<<grid_for(v.N, 256), 256, 0, st>>>(v, rbits, key64, kin, vin), note_launch());
    cudaError_t e;
    if (key64)
        e = radix_sort_u64((uint64_t*)kin, vin, (uint64_t*)kout, v.order, (uint64_t*)ktmp, vtmp, v.N, nbits, sort_temp, st);
    else
        e = radix_sort_u32((uint32_t*)kin, vin, (uint32_t*)kout, v.order, (uint32_t*)ktmp, vtmp, v.N, nbits, sort_temp, st);
    if (e != cudaSuccess) return e;
    (k_rank_from_order<<<grid_for(v.N, 256), 256, 0, st>>>(v), note_launch());
    (k_ro<<<grid_for(v.N, 256), 256, 0, st>>>(v), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_ring(const BatchView& v, const CellWork& w, uint32_t class_mask, int64_t nitems_bound,
                        int64_t nsparse_bound, uint32_t* counters, cudaStream_t st) {
#define DPC_RING_CLASS(D)                                                                             \
    if (class_mask & (1u << (2 * (D - 1))))                                                           \
        launch_ring_class<D, false>(v, w, nitems_bound, nsparse_bound, counters + 2 * (D - 1), st);   \
    if (class_mask & (1u << (2 * (D - 1) + 1)))                                                       \
        launch_ring_class<D, true>(v, w, nitems_bound, nsparse_bound, counters + 2 * (D - 1) + 1, st);
    DPC_RING_CLASS(1) DPC_RING_CLASS(2) DPC_RING_CLASS(3) DPC_RING_CLASS(4)
    DPC_RING_CLASS(5) DPC_RING_CLASS(6) DPC_RING_CLASS(7) DPC_RING_CLASS(8)
#undef DPC_RING_CLASS
    return cudaGetLastError();
}

cudaError_t launch_finalize(const BatchView& v, const DeltaBufs& db, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    (k_finalize<<<grid_for(v.N, 256), 256, 0, st>>>(v, db), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_tree_build(const BatchView& v, const DeltaBufs& db, cudaStream_t st) {
    if (db.leaf_slots == 0) return cudaSuccess;
    (k_tree_build<<<grid_for(db.leaf_slots, 128), 128, 0, st>>>(v, db), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_tree_search(const BatchView& v, const DeltaBufs& db, uint32_t dim_mask, int64_t bound,
                               cudaStream_t st) {
    if (bound <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(bound, 128));
#define DPC_TREE_CLASS(D) \
    if (dim_mask & (1u << (D - 1))) (k_tree_search<D><<<blocks, 128, 0, st>>>(v, db), note_launch());
    DPC_TREE_CLASS(1) DPC_TREE_CLASS(2) DPC_TREE_CLASS(3) DPC_TREE_CLASS(4)
    DPC_TREE_CLASS(5) DPC_TREE_CLASS(6) DPC_TREE_CLASS(7) DPC_TREE_CLASS(8)
#undef DPC_TREE_CLASS
    return cudaGetLastError();
}

cudaError_t launch_bruteforce(const BatchView& v, const DeltaBufs& db, uint32_t dim_mask, int64_t bound,
                              void* sort_temp, cudaStream_t st) {
    if (bound <= 0 || v.N == 0) return cudaSuccess;
    (k_bf_prefix<<<grid_for(v.N, 256), 256, 0, st>>>(v, db), note_launch());
    const unsigned kblocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(bound, 256));
    (k_bf_keys<<<kblocks, 256, 0, st>>>(v, db), note_launch());
    int nbits = 0;
    while ((1ll << nbits) < v.N) ++nbits;
    // sort the open points by global rank position; the list length lives on
    // the device, so sort the bound and let the padding (key ~0) sink last
    cudaError_t e = radix_sort_u32(db.bf_keys, db.bf_list, db.bf_keys + bound, db.bf_sorted, db.bf_keys + 2 * bound,
                                   db.bf_sorted + bound, bound, nbits > 0 ? nbits : 1, sort_temp, st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = grid_for(bound, kBfThreads);
#define DPC_BF_CLASS(D) \
    if (dim_mask & (1u << (D - 1))) (k_bruteforce<D><<<blocks, kBfThreads, 0, st>>>(v, db), note_launch());
    DPC_BF_CLASS(1) DPC_BF_CLASS(2) DPC_BF_CLASS(3) DPC_BF_CLASS(4)
    DPC_BF_CLASS(5) DPC_BF_CLASS(6) DPC_BF_CLASS(7) DPC_BF_CLASS(8)
#undef DPC_BF_CLASS
    return cudaGetLastError();
}

}  // namespace dpc
