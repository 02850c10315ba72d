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

constexpr int kRingThreads = 128;  // 4 warps per block, double-buffered chunks each
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

// Q queries per lane against staged candidates grp, grp + G, ...: keeps the
// least packed key (min(D, 2^32-1) << 32 | original index) of a higher point.
// Forms: direct 32-bit (MODE 0), direct 64-bit saturated (MODE 1), and
// expanded (MODE 2, d <= 3: a record is (c, |c|^2 mod 2^32), a query keeps
// -2 q and |q|^2; D = |c|^2 + |q|^2 - 2 q.c in wrapping 32-bit arithmetic,
// exact because every candidate lies in the 3^k cells around the query's,
// so 0 <= D < 4 d s^2 < 2^31).
template <int D, int MODE, int Q>
__device__ __forceinline__ void eval_ring(const int4* buf, const uint32_t* nrm, const uint2* rbuf, int nb, int grp,
                                          int G, const int32_t (&qx)[4][D], const uint32_t (&qa)[4][4],
                                          const uint32_t (&qn)[4], const uint32_t (&qr)[4],
                                          unsigned long long (&best)[4]) {
    constexpr int DP = D <= 4 ? 1 : 2;
#pragma unroll 2
    for (int j = grp; j < nb; j += G) {
        const uint2 ro = rbuf[j];
        if (MODE == 2) {
            const int4 c = buf[j];
            const uint32_t cn = D == 4 ? nrm[j] : (uint32_t)c.w;  // 4 dims: staged beside the record
#pragma unroll
            for (int t = 0; t < Q; ++t) {
                uint32_t s = cn + qn[t];
                s += (uint32_t)c.x * qa[t][0];
                if (D > 1) s += (uint32_t)c.y * qa[t][1];
                if (D > 2) s += (uint32_t)c.z * qa[t][2];
                if (D > 3) s += (uint32_t)c.w * qa[t][3];
                const unsigned long long key = ((unsigned long long)s << 32) | ro.y;
                if (ro.x < qr[t] && key < best[t]) best[t] = key;
            }
        } else {
            int32_t c[D];
            load_pt<D>(buf + j * DP, c);
#pragma unroll
            for (int t = 0; t < Q; ++t) {
                const uint32_t dd = dist_sat<D, MODE == 1>(qx[t], c);
                const unsigned long long key = ((unsigned long long)dd << 32) | ro.y;
                if (ro.x < qr[t] && key < best[t]) best[t] = key;
            }
        }
    }
}

template <int D, int MODE>
__global__ void __launch_bounds__(kRingThreads) k_ring_dense(BatchView v, CellWork w, uint32_t* counter) {
    constexpr int DP = D <= 4 ? 1 : 2;
    constexpr bool EXP = MODE == 2;
    __shared__ int4 sbuf[kRingThreads / 32][2][kChunk * DP];
    __shared__ uint32_t snrm[kRingThreads / 32][2][EXP && D == 4 ? kChunk : 1];  // 4-d expanded form: |c|^2
    __shared__ uint2 srb[kRingThreads / 32][2][kChunk];
    __shared__ uint2 sruns[kRingThreads / 32][kMaxNb];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint2* srun = sruns[wid];
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
        if (ds.d != D || ds.mode != MODE) continue;
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        const int q0 = (int)qc * w.qch;
        const int nq = min(w.qch, (int)m - q0);
        int Q, Mq;
        lane_layout(nq, Q, Mq);
        const int G = 32 / Mq;
        const int grp = lane / Mq, ql = lane & (Mq - 1);
        int32_t qx[4][D];
        uint32_t qr[4];
        unsigned long long best[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int qi = min(ql * Q + t, nq - 1);
            load_pt<D>(recb + ((int64_t)cs + q0 + qi) * DP, qx[t]);
            qr[t] = v.ro_s[cs + q0 + qi].x;
            best[t] = kNoBest;
        }
        uint32_t qa[4][4], qn[4];
        if (EXP) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                uint32_t nrm = 0u;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t x = k < D ? (uint32_t)qx[t][k < D ? k : 0] : 0u;
                    qa[t][k] = 0u - 2u * x;
                    nrm += x * x;
                }
                qn[t] = nrm;
            }
        }
        const uint32_t nr = w.nruns[c], ctot = w.cand[c];
        // the runs in shared memory when they fit (reach 1), else read in place
        const uint2* runs_c = w.runs + (int64_t)c * w.nbs;
        if (nr <= (uint32_t)kMaxNb) {
            for (uint32_t t = lane; t < nr; t += 32) srun[t] = runs_c[t];
            runs_c = srun;
        }
        __syncwarp();
        const uint32_t k0 = kc * (uint32_t)w.kch;
        CandStream<DP, true> cst;
        cst.init(runs_c, nr, k0, min(ctot, k0 + (uint32_t)w.kch));
        bool bad = false;
        bool have = cst.prep(lane, recb, v.ro_s, &bad);
        int sb = 0;
        while (have) {
            int4* buf = sbuf[wid][sb];
            uint32_t* nbuf = snrm[wid][EXP && D == 4 ? sb : 0];
            uint2* rbuf = srb[wid][sb];
            const int nb = (int)cst.cnt;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int f = lane + 32 * u;
                if (f < nb) {
#pragma unroll
                    for (int q = 0; q < DP; ++q) buf[f * DP + q] = cst.r[u][q];
                    if (EXP && D == 4) {
                        const int4 r = cst.r[u][0];
                        nbuf[f] = (uint32_t)r.x * (uint32_t)r.x + (uint32_t)r.y * (uint32_t)r.y +
                                  (uint32_t)r.z * (uint32_t)r.z + (uint32_t)r.w * (uint32_t)r.w;
                    }
                    rbuf[f] = cst.ro[u];
                }
            }
            __syncwarp();
            have = cst.prep(lane, recb, v.ro_s, &bad);
            sb ^= 1;
            switch (Q) {
                case 1: eval_ring<D, MODE, 1>(buf, nbuf, rbuf, nb, grp, G, qx, qa, qn, qr, best); break;
                case 2: eval_ring<D, MODE, 2>(buf, nbuf, rbuf, nb, grp, G, qx, qa, qn, qr, best); break;
                case 3: eval_ring<D, MODE, 3>(buf, nbuf, rbuf, nb, grp, G, qx, qa, qn, qr, best); break;
                default: eval_ring<D, MODE, 4>(buf, nbuf, rbuf, nb, grp, G, qx, qa, qn, qr, best); break;
            }
        }
        if (bad && lane == 0) atomicOr(v.err, kErrStaging);
        __syncwarp();
        // least key over the groups, then one lane per query writes
#pragma unroll
        for (int t = 0; t < 4; ++t)
            for (int o = Mq; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, best[t], o);
                if (y < best[t]) best[t] = y;
            }
        if (grp == 0) {
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (t < Q && ql * Q + t < nq && best[t] != kNoBest) atomicMin(&v.best_s[cs + q0 + ql * Q + t], best[t]);
        }
    }
}

// Sparse cells: kRingSparseLanes lanes per cell, each with all of the
// cell's queries, take every kRingSparseLanes-th candidate of the cell's
// concatenated runs, kRingSparseBatch of them found before their records
// and ranks are loaded together (overlapping latencies, as in the sparse
// density pass); the least keys are combined with warp shuffles (the cell
// loop is warp-uniform).
constexpr int kRingSparseLanes = 2;
constexpr int kRingSparseBatch = 4;

template <int D, bool W64>
__global__ void __launch_bounds__(256) k_ring_sparse(BatchView v, CellWork w) {
    constexpr int DP = D <= 4 ? 1 : 2;
    constexpr int G = kRingSparseLanes, CPW = 32 / G;
    const uint32_t ns = *w.nsparse;
    const int lane = threadIdx.x & 31, sl = lane & (G - 1), grp = lane / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * CPW; base < ns; base += nwarps * CPW) {
        const int64_t i = base + grp;
        unsigned long long best[kSparseMax];
#pragma unroll
        for (int t = 0; t < kSparseMax; ++t) best[t] = kNoBest;
        uint32_t cs = 0, m = 0;
        bool mine = false;
        if (i < ns) {
            const uint32_t c = w.sparse[i];
            cs = v.cell_start[c];
            m = v.cell_start[c + 1] - cs;
            const DsDesc& ds = v.desc[find_ds(v.pt_off, v.B, cs)];
            mine = ds.d == D && (ds.w32 == 0) == W64;
            if (mine) {
                const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
                int32_t qx[kSparseMax][D];
                uint32_t qr[kSparseMax];
#pragma unroll
                for (int t = 0; t < kSparseMax; ++t) {
                    const uint32_t qi = min((uint32_t)t, m - 1);
                    load_pt<D>(recb + ((int64_t)cs + qi) * DP, qx[t]);
                    qr[t] = v.ro_s[cs + qi].x;
                }
                RunCursor rc;
                rc.init(w.runs + (int64_t)c * w.nbs, w.nruns[c], (uint32_t)sl);
                bool more = true;
                while (more) {
                    // positions first (a lane past its last candidate reads
                    // the cell's own first point and keeps nothing from it)
                    uint32_t p[kRingSparseBatch];
                    bool ok[kRingSparseBatch];
#pragma unroll
                    for (int u = 0; u < kRingSparseBatch; ++u) {
                        ok[u] = rc.next((uint32_t)G, p[u]);
                        if (!ok[u]) p[u] = cs;
                    }
                    more = ok[kRingSparseBatch - 1];
                    int32_t cj[kRingSparseBatch][D];
                    uint2 ro[kRingSparseBatch];
#pragma unroll
                    for (int u = 0; u < kRingSparseBatch; ++u) {
                        load_pt<D>(recb + (int64_t)p[u] * DP, cj[u]);
                        ro[u] = v.ro_s[p[u]];
                    }
#pragma unroll
                    for (int u = 0; u < kRingSparseBatch; ++u)
#pragma unroll
                        for (int q = 0; q < kSparseMax; ++q) {
                            const uint32_t dd = dist_sat<D, W64>(qx[q], cj[u]);
                            const unsigned long long key = ((unsigned long long)dd << 32) | ro[u].y;
                            if (ok[u] && ro[u].x < qr[q] && key < best[q]) best[q] = key;
                        }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kSparseMax; ++q)
#pragma unroll
            for (int o = 1; o < G; o <<= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, best[q], o);
                if (y < best[q]) best[q] = y;
            }
        if (mine && sl == 0) {
#pragma unroll
            for (int q = 0; q < kSparseMax; ++q)
                if ((uint32_t)q < m) v.best_s[cs + q] = best[q];
        }
    }
}

// Resolve the points whose ring-search result is provably final; queue the
// others for the brute-force pass (rank < bf_rank) or the tree search: in
// position (Morton) order when db.ocode is set (codes, block counts, scan,
// k_emit_open), else in position order within each warp.
constexpr int kFinThreads = 256;
constexpr int kOpenCodes = kMaxDims + 2;  // 0 resolved, 1..8 tree search in that many dims, 9 brute force

__global__ void __launch_bounds__(kFinThreads) k_finalize(BatchView v, DeltaBufs db) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = p < v.N;
    bool to_tree = false, to_bf = false;
    if (valid) {
        const int b = find_ds(v.pt_off, v.B, p);
        const DsDesc& ds = v.desc[b];
        const uint2 ro = v.ro_s[p];
        const int64_t g = ds.pt_off + ro.y;
        if (ro.x == 0u) {  // the densest point: no dependent point, delta = infinity
            v.dep[g] = -1;
            v.delta2[g] = INT64_MAX;
        } else {
            const unsigned long long bk = v.best_s[p];
            const uint32_t dd = (uint32_t)(bk >> 32);
            // distance from the point to the outside of the searched box of cells
            const int4* r = v.rec + ds.rec_off + (p - ds.pt_off) * ds.dp;
            int64_t bound = INT64_MAX;
            for (int j = 0; j < ds.k; ++j) {
                const int32_t xi = rec_coord(r, ds.gdim[j]);
                const int64_t x = xi;
                const int64_t cj = cell_coord(ds, j, xi);
                if (cj - ds.R > 0) bound = min(bound, x - (ds.origin[j] + (cj - ds.R) * ds.s) + 1);
                if (cj + ds.R + 1 < ds.ext[j]) bound = min(bound, ds.origin[j] + (cj + ds.R + 1) * ds.s - x);
            }
            // cells the runs left out (at least d_cut away) were not searched
            if (ds.prune) bound = min(bound, ds.d_cut);
            const bool found = bk != kNoBest && dd != kSat;
            if (found && (bound == INT64_MAX || (int64_t)dd < bound * bound)) {
                v.dep[g] = (int32_t)(uint32_t)bk;
                v.delta2[g] = (int64_t)dd;
            } else if (ro.x < db.bf_rank) {
                to_bf = true;
            } else {
                to_tree = true;
            }
        }
    }
    const int lane = threadIdx.x & 31;
    const unsigned mt = __ballot_sync(0xffffffffu, to_tree), mb = __ballot_sync(0xffffffffu, to_bf);
    if (db.ocode) {
        // ordered lists: a code per point (0 resolved, d: tree search in d
        // dims, 9: brute force) and the block's counts per code; the lists
        // are written by k_emit_open after a scan, the tree list grouped by
        // dimension and in position order within each group
        __shared__ uint32_t cc[kFinThreads / 32][kOpenCodes];
        int code = 0;
        if (to_tree) code = v.desc[find_ds(v.pt_off, v.B, p)].d;
        else if (to_bf) code = kOpenCodes - 1;
        if (valid) db.ocode[p] = (uint8_t)code;
#pragma unroll
        for (int c = 1; c < kOpenCodes; ++c) {
            const unsigned m = __ballot_sync(0xffffffffu, code == c);
            if (lane == 0) cc[threadIdx.x >> 5][c] = (uint32_t)__popc(m);
        }
        __syncthreads();
        if (threadIdx.x >= 1 && threadIdx.x < kOpenCodes) {
            uint32_t a = 0;
            for (int w = 0; w < kFinThreads / 32; ++w) a += cc[w][threadIdx.x];
            db.ocnt[(int64_t)(threadIdx.x - 1) * gridDim.x + blockIdx.x] = a;
        }
        return;
    }
    const unsigned lt = (1u << lane) - 1u;
    uint32_t bt = 0, bb = 0;
    if (lane == 0) {
        if (mt) bt = atomicAdd(&db.ucount[0], (uint32_t)__popc(mt));
        if (mb) bb = atomicAdd(&db.ucount[1], (uint32_t)__popc(mb));
    }
    bt = __shfl_sync(0xffffffffu, bt, 0);
    bb = __shfl_sync(0xffffffffu, bb, 0);
    if (to_tree) db.tree_list[bt + __popc(mt & lt)] = (uint32_t)p;
    if (to_bf) db.bf_list[bb + __popc(mb & lt)] = (uint32_t)p;
}

// The open lists from the codes of k_finalize: a point of code c of block b
// goes to the exclusive scan of the (code, block) counts (code-major) plus
// the warps before its own and the lanes before it with the same code.
__global__ void __launch_bounds__(kFinThreads) k_emit_open(BatchView v, DeltaBufs db) {
    __shared__ uint32_t cc[kFinThreads / 32][kOpenCodes];
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int code = p < v.N ? db.ocode[p] : 0;
    const unsigned peers = __match_any_sync(0xffffffffu, code);
#pragma unroll
    for (int c = 1; c < kOpenCodes; ++c) {
        const unsigned m = __ballot_sync(0xffffffffu, code == c);
        if (lane == 0) cc[w][c] = (uint32_t)__popc(m);
    }
    __syncthreads();
    if (code == 0) return;
    uint32_t off = db.oofs[(int64_t)(code - 1) * gridDim.x + blockIdx.x];
    for (int u = 0; u < w; ++u) off += cc[u][code];
    off += (uint32_t)__popc(peers & ((1u << lane) - 1u));
    if (code < kOpenCodes - 1) db.tree_list[off] = (uint32_t)p;
    else db.bf_list[off] = (uint32_t)p;
}

// Where the tree list's group of each dimension starts: tclass[d - 1], and
// tclass[8] = the list's length.
__global__ void k_open_classes(DeltaBufs db, int64_t nb) {
    const int c = threadIdx.x;
    if (c < kMaxDims) db.tclass[c] = db.oofs[(int64_t)c * nb];
    if (c == kMaxDims) db.tclass[c] = db.ucount[0];
}

// --------------------------------------------------------- brute force

// The records of every dataset's bf_rank highest-ranked points, in rank
// order, with their original indices (one thread per sorted position).
__global__ void k_bf_prefix(BatchView v, DeltaBufs db) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const uint2 ro = v.ro_s[p];  // (rank, original local index)
    if (ro.x >= db.bf_rank) return;
    const int b = find_ds(v.pt_off, v.B, p);
    const DsDesc& ds = v.desc[b];
    const int64_t pos = ds.pt_off + ro.x;
    const int4* src = v.rec + ds.rec_off + (p - ds.pt_off) * ds.dp;
    db.rrec[pos * 2] = src[0];
    db.rrec[pos * 2 + 1] = ds.dp == 2 ? src[1] : make_int4(0, 0, 0, 0);
    db.rorig[pos] = ro.y;
}

constexpr int kBfThreads = 128;

// One warp per open point of the list: the lanes stride through the point's
// higher-ranked prefix of its dataset in rank order (the records rrec[pt_off
// .. pt_off + rank), gathered by k_bf_prefix), each keeping the least
// (distance, original index), then a warp reduction.
template <int D>
__global__ void __launch_bounds__(kBfThreads) k_bruteforce(BatchView v, DeltaBufs db) {
    const uint32_t cnt = db.ucount[1];
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < cnt; i += nwarps) {
        const uint32_t p = db.bf_list[i];
        const int b = find_ds(v.pt_off, v.B, p);
        const DsDesc& ds = v.desc[b];
        if (ds.d != D) continue;  // warp-uniform
        int32_t x[D];
        load_pt<D>(v.rec + ds.rec_off + ((int64_t)p - ds.pt_off) * ds.dp, x);
        const uint2 ro = v.ro_s[p];
        const int64_t lo = v.pt_off[b], hi = lo + ro.x;
        long long bestD = INT64_MAX;
        uint32_t bestJ = 0xffffffffu;
        for (int64_t j = lo + lane; j < hi; j += 32) {
            int32_t c[D];
            load_pt<D>(db.rrec + 2 * j, c);
            const long long dd = dist64<D>(x, c);
            const uint32_t o = db.rorig[j];
            if (dd < bestD || (dd == bestD && o < bestJ)) {
                bestD = dd;
                bestJ = o;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const long long d2 = __shfl_xor_sync(0xffffffffu, bestD, o);
            const uint32_t j2 = __shfl_xor_sync(0xffffffffu, bestJ, o);
            if (d2 < bestD || (d2 == bestD && j2 < bestJ)) {
                bestD = d2;
                bestJ = j2;
            }
        }
        if (lane == 0) {
            const int64_t g = ds.pt_off + ro.y;
            v.dep[g] = (int32_t)bestJ;
            v.delta2[g] = bestD;
        }
    }
}

template <int D, int MODE>
void launch_ring_dense(const BatchView& v, const CellWork& w, int64_t nitems_bound, uint32_t* counter,
                       cudaStream_t st) {
    if (nitems_bound <= 0) return;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(152 * 16, (nitems_bound + 3) / 4));
    (k_ring_dense<D, MODE><<<blocks, kRingThreads, 0, st>>>(v, w, counter), note_launch());
}

template <int D, bool W64>
void launch_ring_sparse(const BatchView& v, const CellWork& w, int64_t nsparse_bound, cudaStream_t st) {
    if (nsparse_bound <= 0) return;
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 32, grid_for(nsparse_bound * kRingSparseLanes, 256));
    (k_ring_sparse<D, W64><<<blocks, 256, 0, st>>>(v, w), note_launch());
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
    // dense: one launch per (dimension, mode) class; sparse: modes 0 and 2
    // share the 32-bit kernel, mode 1 is 64-bit
#define DPC_BIT(D, M) (class_mask & (1u << (3 * ((D) - 1) + (M))))
#define DPC_RING_CLASS(D)                                                                                 \
    if (DPC_BIT(D, 0)) launch_ring_dense<D, 0>(v, w, nitems_bound, counters + 3 * (D - 1), st);           \
    if (DPC_BIT(D, 1)) launch_ring_dense<D, 1>(v, w, nitems_bound, counters + 3 * (D - 1) + 1, st);       \
    if (DPC_BIT(D, 0) || DPC_BIT(D, 2)) launch_ring_sparse<D, false>(v, w, nsparse_bound, st);            \
    if (DPC_BIT(D, 1)) launch_ring_sparse<D, true>(v, w, nsparse_bound, st);
#define DPC_RING_X(D) \
    if (DPC_BIT(D, 2)) launch_ring_dense<D, 2>(v, w, nitems_bound, counters + 3 * (D - 1) + 2, st);
    DPC_RING_CLASS(1) DPC_RING_CLASS(2) DPC_RING_CLASS(3) DPC_RING_CLASS(4)
    DPC_RING_CLASS(5) DPC_RING_CLASS(6) DPC_RING_CLASS(7) DPC_RING_CLASS(8)
    DPC_RING_X(1) DPC_RING_X(2) DPC_RING_X(3) DPC_RING_X(4)
#undef DPC_RING_X
#undef DPC_RING_CLASS
#undef DPC_BIT
    return cudaGetLastError();
}

size_t finalize_temp_bytes(int64_t n) {
    const int64_t nb = (n + kFinThreads - 1) / kFinThreads;
    return (size_t)n + 2 * (kOpenCodes - 1) * sizeof(uint32_t) * (size_t)nb + scan_temp_bytes(kMaxDims * nb) +
           1024;
}

cudaError_t launch_finalize(const BatchView& v, DeltaBufs db, void* ordered_temp, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    const int64_t nb = grid_for(v.N, kFinThreads);
    if (ordered_temp) {
        char* t = static_cast<char*>(ordered_temp);
        db.ocnt = reinterpret_cast<uint32_t*>(t);
        db.oofs = db.ocnt + (kOpenCodes - 1) * nb;
        void* stemp = db.oofs + (kOpenCodes - 1) * nb;
        db.ocode = reinterpret_cast<uint8_t*>(static_cast<char*>(stemp) +
                                              ((scan_temp_bytes(kMaxDims * nb) + 255) & ~(size_t)255));
        (k_finalize<<<(unsigned)nb, kFinThreads, 0, st>>>(v, db), note_launch());
        // offsets in the tree list (code-major over the dims), then in the
        // brute-force list
        cudaError_t e = exclusive_scan_u32(db.ocnt, db.oofs, kMaxDims * nb, db.ucount, stemp, st);
        if (e != cudaSuccess) return e;
        e = exclusive_scan_u32(db.ocnt + kMaxDims * nb, db.oofs + kMaxDims * nb, nb, db.ucount + 1, stemp, st);
        if (e != cudaSuccess) return e;
        (k_emit_open<<<(unsigned)nb, kFinThreads, 0, st>>>(v, db), note_launch());
        if (db.tclass) (k_open_classes<<<1, 32, 0, st>>>(db, nb), note_launch());
        return cudaGetLastError();
    }
    db.ocode = nullptr;
    (k_finalize<<<(unsigned)nb, kFinThreads, 0, st>>>(v, db), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_bruteforce(const BatchView& v, const DeltaBufs& db, uint32_t dim_mask, int64_t bound,
                              cudaStream_t st) {
    if (bound <= 0 || v.N == 0) return cudaSuccess;
    (k_bf_prefix<<<grid_for(v.N, 256), 256, 0, st>>>(v, db), note_launch());
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(bound * 32, kBfThreads));
#define DPC_BF_CLASS(D) \
    if (dim_mask & (1u << (D - 1))) (k_bruteforce<D><<<blocks, kBfThreads, 0, st>>>(v, db), note_launch());
    DPC_BF_CLASS(1) DPC_BF_CLASS(2) DPC_BF_CLASS(3) DPC_BF_CLASS(4)
    DPC_BF_CLASS(5) DPC_BF_CLASS(6) DPC_BF_CLASS(7) DPC_BF_CLASS(8)
#undef DPC_BF_CLASS
    return cudaGetLastError();
}

}  // namespace dpc
