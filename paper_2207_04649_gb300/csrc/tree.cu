// Expanding search for the dependent points the ring searches left open.
//
// A binary radix tree over the Morton-ordered cells of each dataset: leaf c
// is grid cell c (a contiguous run of sorted points), and every internal
// node covers the cells sharing a longest common key prefix, i.e. an
// axis-aligned box of cells. It is built in one parallel pass from the
// sorted unique cell keys (each internal node finds its key range and split
// point by binary searches on common-prefix lengths, the construction of
// Karras, "Maximizing parallelism in the construction of BVHs, octrees, and
// k-d trees", HPG 2012), then refitted bottom-up: every node record holds
// the bounding box of its points, the smallest rank (highest density) among
// them, and its children (or, for a leaf, its run of points), so that one
// node costs one memory round trip in the search.
//
// The search is the nearest-neighbour search among higher-ranked points that
// Ex-DPC runs on its incrementally built kd-tree (Section 3, steps 3-4),
// done here for all open points in parallel, depth first from the root of
// the point's dataset: a subtree is skipped when no point in it ranks higher
// or when its box is farther than the best distance so far, and the nearer
// child is searched first. Ties in distance go to the smaller original index.
#include "stages.cuh"
#include <algorithm>

namespace dpc {

namespace {

template <int D>
__device__ __forceinline__ void t_load(const int4* r, int32_t (&x)[D]) {
    const int4 a = r[0];
    int32_t t[8] = {a.x, a.y, a.z, a.w, 0, 0, 0, 0};
    if (D > 4) {
        const int4 bq = r[1];
        t[4] = bq.x; t[5] = bq.y; t[6] = bq.z; t[7] = bq.w;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = t[k];
}

__device__ __forceinline__ int find_off(const int64_t* off, int B, int64_t x) {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// First cell of every dataset: lower bound of pt_off_b in cell_start.
__global__ void k_cell_ranges(BatchView v, DeltaBufs db) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > v.B) return;
    if (b == v.B) {
        db.cell_off[b] = db.ncells;
        return;
    }
    const uint32_t target = (uint32_t)v.pt_off[b];
    int64_t lo = 0, hi = db.ncells;  // first c with cell_start[c] >= target
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (v.cell_start[mid] < target) lo = mid + 1; else hi = mid;
    }
    db.cell_off[b] = lo;
}

// The Morton code of every cell within its dataset (the dataset's key base
// removed), so that every internal node is a Morton-prefix box of cells.
__global__ void k_cell_key(BatchView v, DeltaBufs db) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= db.ncells) return;
    const int b = find_off(db.cell_off, v.B, c);
    db.ckey[c] = v.key[v.cell_start[c]] - v.desc[b].cbase;
}

// Common-prefix length of the keys of cells i and j, -1 outside [c0, c1).
__device__ __forceinline__ int prefix(const uint64_t* __restrict__ key, int64_t c0, int64_t c1, int64_t i,
                                      int64_t j) {
    if (j < c0 || j >= c1) return -1;
    return __clzll((long long)(key[i] ^ key[j]));
}

__global__ void k_radix_tree(BatchView v, DeltaBufs db) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= db.ncells) return;
    const int b = find_off(db.cell_off, v.B, i);
    const int64_t c0 = db.cell_off[b], c1 = db.cell_off[b + 1];
    if (i == c0 && c1 - c0 == 1) db.lparent[i] = -1;  // a dataset with one cell: the leaf is the root
    if (i >= c1 - 1) return;                           // internal nodes are c0 .. c1-2
    const uint64_t* key = db.ckey;
    const int d = prefix(key, c0, c1, i, i + 1) > prefix(key, c0, c1, i, i - 1) ? 1 : -1;
    const int dmin = prefix(key, c0, c1, i, i - d);
    int64_t lmax = 2;
    while (prefix(key, c0, c1, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (prefix(key, c0, c1, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = prefix(key, c0, c1, i, j);
    int64_t s = 0, t = l;
    while (true) {
        t = (t + 1) >> 1;
        if (prefix(key, c0, c1, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
    }
    const int64_t g = i + s * d + min(d, 0);
    const int64_t lo = min(i, j), hi = max(i, j);
    const int32_t left = lo == g ? ~(int32_t)g : (int32_t)g;
    const int32_t right = hi == g + 1 ? ~(int32_t)(g + 1) : (int32_t)(g + 1);
    db.child[i] = make_int2(left, right);
    if (left < 0) db.lparent[g] = (int32_t)i; else db.iparent[g] = (int32_t)i;
    if (right < 0) db.lparent[g + 1] = (int32_t)i; else db.iparent[g + 1] = (int32_t)i;
    if (i == c0) db.iparent[i] = -1;
}

// Record index of a node reference: internal i >= 0, leaf ~c.
__device__ __forceinline__ int64_t rec_of(const DeltaBufs& db, int32_t ref) {
    return ref >= 0 ? (int64_t)ref : db.ncells + (int64_t)(~ref);
}

// Leaf records: every cell's box, smallest rank and point run (or its range
// of the leaf point list). A lane takes a cell of at most kLeafLane points;
// larger cells (dense data) are taken by the whole warp, the lanes striding
// the points.
constexpr uint32_t kLeafLane = 64;

__device__ __forceinline__ void write_leaf(const DeltaBufs& db, int64_t c, const int32_t (&lo)[8],
                                           const int32_t (&hi)[8], uint32_t mr, uint32_t p0, uint32_t p1) {
    if (db.compact) {  // {lo, smallest rank}, {hi, 0}: the points come from the cell starts
        int4* lr = db.nodes + (db.ncells + c) * 2;
        lr[0] = make_int4(lo[0], lo[1], lo[2], (int)mr);
        lr[1] = make_int4(hi[0], hi[1], hi[2], 0);
        return;
    }
    const int dpb = db.dpb, ns = 2 * dpb + 1;
    int4* lr = db.nodes + (db.ncells + c) * ns;
    lr[0] = make_int4(lo[0], lo[1], lo[2], lo[3]);
    if (dpb == 2) lr[1] = make_int4(lo[4], lo[5], lo[6], lo[7]);
    lr[dpb] = make_int4(hi[0], hi[1], hi[2], hi[3]);
    if (dpb == 2) lr[dpb + 1] = make_int4(hi[4], hi[5], hi[6], hi[7]);
    lr[2 * dpb] = make_int4((int)mr, (int)p0, (int)p1, db.lparent[c]);
}

__device__ __forceinline__ void leaf_add(const BatchView& v, const DsDesc& ds, uint32_t p, int32_t (&lo)[8],
                                         int32_t (&hi)[8], uint32_t& mr) {
    const int4* r = v.rec + ds.rec_off + ((int64_t)p - ds.pt_off) * ds.dp;
    const int4 a = r[0];
    const int4 e = ds.dp == 2 ? r[1] : make_int4(0, 0, 0, 0);
    const int32_t x[8] = {a.x, a.y, a.z, a.w, e.x, e.y, e.z, e.w};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        lo[k] = min(lo[k], x[k]);
        hi[k] = max(hi[k], x[k]);
    }
    mr = min(mr, v.ro_s[p].x);
}

__global__ void k_leaves(BatchView v, DeltaBufs db) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < db.ncells;
         base += nwarps * 32) {
        const int64_t c = base + lane;
        const bool valid = c < db.ncells;
        int b = 0;
        uint32_t p0 = 0, p1 = 0;
        bool big = false;
        if (valid) {
            b = find_off(db.cell_off, v.B, c);
            p0 = db.lplist ? db.lpstart[c] : v.cell_start[c];
            p1 = db.lplist ? db.lpstart[c + 1] : v.cell_start[c + 1];
            big = p1 - p0 > kLeafLane;
        }
        if (valid && !big) {
            const DsDesc& ds = v.desc[b];
            int32_t lo[8], hi[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                lo[k] = INT32_MAX;
                hi[k] = INT32_MIN;
            }
            uint32_t mr = 0xffffffffu;
            // four points in flight at a time; past the cell's end the last
            // point is read again (min and max are unchanged by a repeat)
            for (uint32_t p = p0; p < p1; p += 4) {
                int4 ra[4], rb[4];
                uint32_t rk[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t pu = min(p + (uint32_t)u, p1 - 1u);
                    const uint32_t q = db.lplist ? db.lplist[pu] : pu;
                    const int4* r = v.rec + ds.rec_off + ((int64_t)q - ds.pt_off) * ds.dp;
                    ra[u] = r[0];
                    rb[u] = ds.dp == 2 ? r[1] : make_int4(0, 0, 0, 0);
                    rk[u] = v.ro_s[q].x;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int32_t x[8] = {ra[u].x, ra[u].y, ra[u].z, ra[u].w, rb[u].x, rb[u].y, rb[u].z, rb[u].w};
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        lo[k] = min(lo[k], x[k]);
                        hi[k] = max(hi[k], x[k]);
                    }
                    mr = min(mr, rk[u]);
                }
            }
            write_leaf(db, c, lo, hi, mr, p0, p1);
        }
        unsigned bigm = __ballot_sync(0xffffffffu, big);
        while (bigm) {
            const int src = __ffs(bigm) - 1;
            bigm &= bigm - 1u;
            const int64_t cc = __shfl_sync(0xffffffffu, c, src);
            const int bb = __shfl_sync(0xffffffffu, b, src);
            const uint32_t q0 = __shfl_sync(0xffffffffu, p0, src), q1 = __shfl_sync(0xffffffffu, p1, src);
            const DsDesc& ds = v.desc[bb];
            int32_t lo[8], hi[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                lo[k] = INT32_MAX;
                hi[k] = INT32_MIN;
            }
            uint32_t mr = 0xffffffffu;
            for (uint32_t p = q0 + lane; p < q1; p += 32) leaf_add(v, ds, db.lplist ? db.lplist[p] : p, lo, hi, mr);
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
                    hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
                }
                mr = min(mr, __shfl_xor_sync(0xffffffffu, mr, o));
            }
            if (lane == 0) write_leaf(db, cc, lo, hi, mr, q0, q1);
        }
    }
}

// Compact records (every dataset of the batch in at most 3 dims): two int4,
// {lo, smallest rank} and {hi, link}. An internal node's children are cells
// g and g + 1 of the radix tree (Karras), each an internal node or a leaf:
// link = g << 2 | (left is a leaf) << 1 | (right is a leaf).
__device__ __forceinline__ uint32_t compact_link(int2 ch) {
    const uint32_t g = (uint32_t)(ch.x >= 0 ? ch.x : ~ch.x);
    return (g << 2) | (ch.x < 0 ? 2u : 0u) | (ch.y < 0 ? 1u : 0u);
}

__device__ __forceinline__ int32_t link_left(uint32_t link) {
    const int32_t g = (int32_t)(link >> 2);
    return (link & 2u) ? ~g : g;
}

__device__ __forceinline__ int32_t link_right(uint32_t link) {
    const int32_t g = (int32_t)(link >> 2) + 1;
    return (link & 1u) ? ~g : g;
}

// Bottom-up refit from the leaf records: the second child to arrive at a
// node writes the node's record.
__global__ void k_refit(BatchView v, DeltaBufs db) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= db.ncells) return;
    const int dpb = db.dpb, ns = 2 * dpb + 1;
    int32_t node = db.lparent[c];
    while (node >= 0) {
        __threadfence();
        if (atomicAdd(&db.flag[node], 1u) == 0u) return;
        __threadfence();
        const int2 ch = __ldcg(&db.child[node]);
        if (db.compact) {
            const int4* ca = db.nodes + rec_of(db, ch.x) * 2;
            const int4* cb = db.nodes + rec_of(db, ch.y) * 2;
            const int4 a0 = __ldcg(ca), a1 = __ldcg(ca + 1), b0 = __ldcg(cb), b1 = __ldcg(cb + 1);
            int4* nr = db.nodes + (int64_t)node * 2;
            nr[0] = make_int4(min(a0.x, b0.x), min(a0.y, b0.y), min(a0.z, b0.z),
                              (int)min((uint32_t)a0.w, (uint32_t)b0.w));
            nr[1] = make_int4(max(a1.x, b1.x), max(a1.y, b1.y), max(a1.z, b1.z), (int)compact_link(ch));
            node = __ldcg(&db.iparent[node]);
            continue;
        }
        const int4* ca = db.nodes + rec_of(db, ch.x) * ns;
        const int4* cb = db.nodes + rec_of(db, ch.y) * ns;
        int4* nr = db.nodes + (int64_t)node * ns;
        for (int q = 0; q < 2 * dpb; ++q) {
            const int4 x = __ldcg(ca + q), y = __ldcg(cb + q);
            nr[q] = q < dpb ? make_int4(min(x.x, y.x), min(x.y, y.y), min(x.z, y.z), min(x.w, y.w))
                            : make_int4(max(x.x, y.x), max(x.y, y.y), max(x.z, y.z), max(x.w, y.w));
        }
        const uint32_t m0 = (uint32_t)__ldcg(ca + 2 * dpb).x, m1 = (uint32_t)__ldcg(cb + 2 * dpb).x;
        const int32_t par = __ldcg(&db.iparent[node]);
        nr[2 * dpb] = make_int4((int)min(m0, m1), ch.x, ch.y, par);
        node = par;
    }
}

// Loads a node record: squared distance from x to its box (INT64_MAX when
// nothing in it ranks above `rank`) and its meta word.
template <int D>
__device__ __forceinline__ long long node_test(const int4* rec, int dpb, const int32_t (&x)[D], uint32_t rank,
                                               int4& meta) {
    const int4 l0 = rec[0], h0 = rec[dpb];
    int32_t lo[8] = {l0.x, l0.y, l0.z, l0.w, 0, 0, 0, 0};
    int32_t hi[8] = {h0.x, h0.y, h0.z, h0.w, 0, 0, 0, 0};
    if (D > 4) {
        const int4 l1 = rec[1], h1 = rec[dpb + 1];
        lo[4] = l1.x; lo[5] = l1.y; lo[6] = l1.z; lo[7] = l1.w;
        hi[4] = h1.x; hi[5] = h1.y; hi[6] = h1.z; hi[7] = h1.w;
    }
    meta = rec[2 * dpb];
    if ((uint32_t)meta.x >= rank) return INT64_MAX;
    long long s = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const long long dd = x[k] < lo[k] ? (long long)lo[k] - x[k] : (x[k] > hi[k] ? (long long)x[k] - hi[k] : 0);
        s += dd * dd;
    }
    return s;
}

// A node is skipped when nothing in it ranks higher (INT64_MAX from
// node_test; real squared distances stay below it for coordinates under
// 2^30) or when its box is farther than the best distance so far.
__device__ __forceinline__ bool out_of_reach(long long d, long long best) {
    return d == INT64_MAX || d > best;
}

// A stack entry keeps a lower bound of its node's squared distance (32
// bits, saturated), so that a node the best distance has overtaken since it
// was pushed is dropped without loading its record. The radix tree over
// cell keys of at most 40 bits is at most 41 levels deep, and the search
// holds at most one more entry than the depth.
constexpr int kStack = 64;

__device__ __forceinline__ uint32_t lb32(long long d) {
    return d >= 0xffffffffll ? 0xffffffffu : (uint32_t)d;
}

// Squared distance from x to a compact record's box (INT64_MAX when nothing
// in it ranks above `rank`); link receives the record's link word.
template <int D>
__device__ __forceinline__ long long node_test_c(const int4* rec, const int32_t (&x)[D], uint32_t rank,
                                                 uint32_t& link) {
    const int4 a = rec[0], h = rec[1];
    link = (uint32_t)h.w;
    if ((uint32_t)a.w >= rank) return INT64_MAX;
    const int32_t lo[3] = {a.x, a.y, a.z}, hi[3] = {h.x, h.y, h.z};
    long long s = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const long long dd = x[k] < lo[k] ? (long long)lo[k] - x[k] : (x[k] > hi[k] ? (long long)x[k] - hi[k] : 0);
        s += dd * dd;
    }
    return s;
}

// The points of a cell (or of its range of the leaf point list) against the
// best so far, kLeafBatch points at a time: their ranks and records are all
// loaded before any is tested (a record is read whether or not its point
// ranks higher), so that a long scan waits for one memory round trip per
// kLeafBatch points instead of two per point.
constexpr int kLeafBatch = 2;

template <int D>
__device__ __forceinline__ void leaf_point(const int32_t (&x)[D], const int32_t (&cx)[D], uint2 cr, uint32_t rank,
                                           long long& bestD, uint32_t& bestJ, unsigned long long& tests) {
    if (cr.x >= rank) return;
    ++tests;
    long long dd = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const long long e = (long long)x[k] - cx[k];
        dd += e * e;
    }
    if (dd < bestD || (dd == bestD && cr.y < bestJ)) {
        bestD = dd;
        bestJ = cr.y;
    }
}

template <int D>
__device__ __forceinline__ void scan_leaf(const BatchView& v, const DeltaBufs& db, const int4* recb, int64_t c,
                                          int32_t t0, int32_t t1, const int32_t (&x)[D], uint32_t rank,
                                          long long& bestD, uint32_t& bestJ, unsigned long long& tests) {
    constexpr int DP = D <= 4 ? 1 : 2;
    int32_t t = t0;
    for (; t + kLeafBatch <= t1; t += kLeafBatch) {
        uint32_t q[kLeafBatch];
        uint2 cr[kLeafBatch];
        int32_t cx[kLeafBatch][D];
#pragma unroll
        for (int u = 0; u < kLeafBatch; ++u) q[u] = db.lplist ? db.lplist[t + u] : (uint32_t)(t + u);
#pragma unroll
        for (int u = 0; u < kLeafBatch; ++u) {
            cr[u] = v.ro_s[q[u]];
            t_load<D>(recb + (int64_t)q[u] * DP, cx[u]);
        }
#pragma unroll
        for (int u = 0; u < kLeafBatch; ++u) leaf_point<D>(x, cx[u], cr[u], rank, bestD, bestJ, tests);
    }
    if (t < t1) {  // the last t1 - t < kLeafBatch points, loaded together as well
        uint32_t q[kLeafBatch - 1];
        uint2 cr[kLeafBatch - 1];
        int32_t cx[kLeafBatch - 1][D];
#pragma unroll
        for (int u = 0; u < kLeafBatch - 1; ++u) {
            const int32_t tu = min(t + u, t1 - 1);
            q[u] = db.lplist ? db.lplist[tu] : (uint32_t)tu;
            cr[u] = v.ro_s[q[u]];
            t_load<D>(recb + (int64_t)q[u] * DP, cx[u]);
        }
#pragma unroll
        for (int u = 0; u < kLeafBatch - 1; ++u)
            if (t + u < t1) leaf_point<D>(x, cx[u], cr[u], rank, bestD, bestJ, tests);
    }
}

// S stack entries per lane (local memory): 32 when every tree is at most 31
// levels deep (cell keys of at most 30 bits), else 64. Bounded to 11 blocks
// per SM: more warps to hide the pointer chasing' latency, at the cost of a
// few spilled registers (5.8M x 3: open points 2.39 -> 2.28 ms).
template <int D, int S>
__global__ void __launch_bounds__(128, 11) k_tree_search(BatchView v, DeltaBufs db) {
    constexpr int DP = D <= 4 ? 1 : 2;
    constexpr bool CMP = D <= 3;  // compact records possible
    // the list's group of dimension D when it is grouped, else all of it
    const uint32_t i0 = db.tclass ? db.tclass[D - 1] : 0u;
    const uint32_t cnt = db.tclass ? db.tclass[D] : *db.tcount;
    const int dpb = db.dpb, ns = 2 * dpb + 1;
    const bool compact = CMP && db.compact;
    unsigned long long visits = 0, tests = 0;
    for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = db.tree_list[i];
        const int b = find_ds(v.pt_off, v.B, p);
        const DsDesc& ds = v.desc[b];
        if (ds.d != D) continue;
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;
        int32_t x[D];
        t_load<D>(recb + (int64_t)p * DP, x);
        const uint2 ro = v.ro_s[p];
        long long bestD = INT64_MAX;
        uint32_t bestJ = 0xffffffffu;
        const unsigned long long bk = v.best_s[p];  // unproven ring-search result: a valid start
        if (bk != ~0ull && (uint32_t)(bk >> 32) != 0xffffffffu) {
            bestD = (long long)(bk >> 32);
            bestJ = (uint32_t)bk;
        }
        int32_t stack[S];
        uint32_t slb[S];
        const int64_t c0 = db.cell_off[b], c1 = db.cell_off[b + 1];
        const int32_t root = c1 - c0 >= 2 ? (int32_t)c0 : ~(int32_t)c0;
        if (compact) {
            // the current node (tested, in reach) walks to its nearer child
            // in reach; the farther child in reach is stacked as (entry,
            // distance bound), the entry being a cell's reference (~c < 0)
            // or an internal node's link word (its children, >= 0: fewer
            // than 2^29 cells); a node whose children are both out of reach,
            // or a scanned cell, takes the next stacked node still in reach
            uint32_t cur_link;
            int32_t cur = root;
            int sp = 0;
            bool have = !out_of_reach(node_test_c<D>(db.nodes + rec_of(db, root) * 2, x, ro.x, cur_link), bestD);
            while (have) {
                ++visits;
                bool next = false;
                if (cur < 0) {  // a cell: scan its points
                    const int64_t c = ~cur;
                    const uint32_t t0 = db.lplist ? db.lpstart[c] : v.cell_start[c];
                    const uint32_t t1 = db.lplist ? db.lpstart[c + 1] : v.cell_start[c + 1];
                    scan_leaf<D>(v, db, recb, c, (int32_t)t0, (int32_t)t1, x, ro.x, bestD, bestJ, tests);
                } else {
                    const int32_t l = link_left(cur_link), r = link_right(cur_link);
                    uint32_t ll, rl;
                    const long long d0 = node_test_c<D>(db.nodes + rec_of(db, l) * 2, x, ro.x, ll);
                    const long long d1 = node_test_c<D>(db.nodes + rec_of(db, r) * 2, x, ro.x, rl);
                    const bool swap = d1 < d0;
                    const long long dn = swap ? d1 : d0, df = swap ? d0 : d1;
                    if (!out_of_reach(df, bestD)) {
                        if (sp < S) {
                            const int32_t fr = swap ? l : r;
                            stack[sp] = fr < 0 ? fr : (int32_t)(swap ? ll : rl);
                            slb[sp] = lb32(df);
                            ++sp;
                        } else {
                            atomicOr(v.err, kErrTreeStack);
                        }
                    }
                    if (!out_of_reach(dn, bestD)) {
                        cur = swap ? r : l;
                        cur_link = swap ? rl : ll;
                        next = true;
                    }
                }
                while (!next && sp > 0) {
                    --sp;
                    if ((long long)slb[sp] > bestD) continue;  // overtaken since it was stacked
                    const int32_t e = stack[sp];
                    cur = e < 0 ? e : 0;  // an internal node is known by its link word
                    cur_link = (uint32_t)e;
                    next = true;
                }
                have = next;
            }
        } else {
            // as above; the current node's meta word comes with it (the
            // nearer child's from its test); a stacked node keeps its
            // children as a link word (a cell's points come from the cell
            // starts), so that a pop loads nothing
            int4 meta;
            uint32_t slink[S];
            int32_t cur = root;
            int sp = 0;
            bool have = !out_of_reach(node_test<D>(db.nodes + rec_of(db, root) * ns, dpb, x, ro.x, meta), bestD);
            while (have) {
                ++visits;
                bool next = false;
                if (cur < 0) {  // a cell: scan its points
                    scan_leaf<D>(v, db, recb, ~cur, meta.y, meta.z, x, ro.x, bestD, bestJ, tests);
                } else {
                    // both children's records in one round; the nearer is searched first
                    int4 m0, m1;
                    const long long d0 = node_test<D>(db.nodes + rec_of(db, meta.y) * ns, dpb, x, ro.x, m0);
                    const long long d1 = node_test<D>(db.nodes + rec_of(db, meta.z) * ns, dpb, x, ro.x, m1);
                    const bool swap = d1 < d0;
                    const long long dn = swap ? d1 : d0, df = swap ? d0 : d1;
                    const int32_t nn = swap ? meta.z : meta.y, nf = swap ? meta.y : meta.z;
                    if (!out_of_reach(df, bestD)) {
                        if (sp < S) {
                            const int4 mf = swap ? m0 : m1;
                            stack[sp] = nf;
                            slb[sp] = lb32(df);
                            slink[sp] = nf >= 0 ? compact_link(make_int2(mf.y, mf.z)) : 0u;
                            ++sp;
                        } else {
                            atomicOr(v.err, kErrTreeStack);
                        }
                    }
                    if (!out_of_reach(dn, bestD)) {
                        cur = nn;
                        meta = swap ? m1 : m0;
                        next = true;
                    }
                }
                while (!next && sp > 0) {
                    --sp;
                    if ((long long)slb[sp] > bestD) continue;  // overtaken since it was stacked
                    cur = stack[sp];
                    if (cur >= 0) {
                        meta.y = link_left(slink[sp]);
                        meta.z = link_right(slink[sp]);
                    } else {
                        const int64_t c = ~cur;
                        meta.y = (int)(db.lplist ? db.lpstart[c] : v.cell_start[c]);
                        meta.z = (int)(db.lplist ? db.lpstart[c + 1] : v.cell_start[c + 1]);
                    }
                    next = true;
                }
                have = next;
            }
        }
        const int64_t g = ds.pt_off + ro.y;
        v.dep[g] = (int32_t)bestJ;
        v.delta2[g] = bestD;
    }
    for (int o = 16; o > 0; o >>= 1) {
        visits += __shfl_xor_sync(0xffffffffu, visits, o);
        tests += __shfl_xor_sync(0xffffffffu, tests, o);
    }
    if ((threadIdx.x & 31) == 0 && db.stats) {
        atomicAdd(&db.stats[0], visits);
        atomicAdd(&db.stats[1], tests);
    }
}

// Warp-cooperative form of the same search. The 32 lanes of a warp take 32
// consecutive entries of the open list (in position order, so mostly
// neighbouring points) and walk their dataset's tree together: a node record
// is loaded once for the warp (every lane reads the same address) and every
// lane tests it against its own point, rank and best distance; the warp
// enters a subtree when any lane has it in reach, and a lane takes part only
// in the subtrees in its own reach, so every lane's result is that of its own
// pruned search. Of two children both in reach, the one nearer for more of
// the lanes is entered first; the other is stacked with the lanes' mask and
// each lane's distance bound (shared memory). A leaf's points are loaded by
// the lanes together and broadcast by shuffles.
constexpr int kWStack = 42;  // cell keys have at most 40 bits: at most 40 internal levels
constexpr int kWWarps = 4;   // warps per block

template <int D>
__device__ __forceinline__ long long w_test(const DeltaBufs& db, bool compact, int dpb, int32_t ref,
                                            const int32_t (&x)[D], uint32_t rank, int4& meta) {
    if (compact) {
        uint32_t link;
        const long long d = node_test_c<D>(db.nodes + rec_of(db, ref) * 2, x, rank, link);
        meta = make_int4(0, (int)link, 0, 0);
        return d;
    }
    return node_test<D>(db.nodes + rec_of(db, ref) * (2 * dpb + 1), dpb, x, rank, meta);
}

template <int D>
__global__ void __launch_bounds__(kWWarps * 32) k_tree_search_warp(BatchView v, DeltaBufs db) {
    constexpr int DP = D <= 4 ? 1 : 2;
    constexpr bool CMP = D <= 3;
    constexpr unsigned kAll = 0xffffffffu;
    __shared__ uint32_t s_lb[kWWarps][kWStack][32];
    __shared__ int4 s_ent[kWWarps][kWStack];  // {node, meta y, meta z, lane mask}
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t i0 = db.tclass ? db.tclass[D - 1] : 0u;
    const uint32_t cnt = db.tclass ? db.tclass[D] : *db.tcount;
    const int dpb = db.dpb;
    const bool compact = CMP && db.compact;
    unsigned long long visits = 0, tests = 0;
    for (int64_t base = i0 + ((int64_t)blockIdx.x * kWWarps + wi) * 32; base < cnt;
         base += (int64_t)gridDim.x * kWWarps * 32) {
        const int64_t i = base + lane;
        int b = -1;
        uint32_t p = 0;
        int32_t x[D];
#pragma unroll
        for (int k = 0; k < D; ++k) x[k] = 0;
        uint2 ro = make_uint2(0u, 0u);
        long long bestD = INT64_MAX;
        uint32_t bestJ = 0xffffffffu;
        if (i < cnt) {
            p = db.tree_list[i];
            b = find_ds(v.pt_off, v.B, p);
            const DsDesc& ds = v.desc[b];
            if (ds.d == D) {
                t_load<D>(v.rec + ds.rec_off + ((int64_t)p - ds.pt_off) * DP, x);
                ro = v.ro_s[p];
                const unsigned long long bk = v.best_s[p];  // unproven ring-search result: a valid start
                if (bk != ~0ull && (uint32_t)(bk >> 32) != 0xffffffffu) {
                    bestD = (long long)(bk >> 32);
                    bestJ = (uint32_t)bk;
                }
            } else {
                b = -1;
            }
        }
        // the lanes of one dataset search its tree together
        unsigned todo = __ballot_sync(kAll, b >= 0);
        while (todo) {
            const int bl = __shfl_sync(kAll, b, __ffs(todo) - 1);
            const unsigned grp = __ballot_sync(kAll, b == bl) & todo;
            todo &= ~grp;
            const bool mine = (grp >> lane) & 1u;
            const DsDesc& ds = v.desc[bl];
            const int4* recg = v.rec + ds.rec_off - ds.pt_off * DP;
            const int64_t c0 = db.cell_off[bl], c1 = db.cell_off[bl + 1];
            int32_t cur = c1 - c0 >= 2 ? (int32_t)c0 : ~(int32_t)c0;
            int4 cm;
            const long long dr = w_test<D>(db, compact, dpb, cur, x, ro.x, cm);
            unsigned m = __ballot_sync(kAll, mine && !out_of_reach(dr, bestD));
            int sp = 0;
            while (m) {
                ++visits;
                const bool act = (m >> lane) & 1u;
                bool next = false;
                if (cur < 0) {  // a cell: its points, 32 at a time, broadcast to the lanes
                    const int64_t c = ~cur;
                    uint32_t t0, t1;
                    if (compact) {
                        t0 = db.lplist ? db.lpstart[c] : v.cell_start[c];
                        t1 = db.lplist ? db.lpstart[c + 1] : v.cell_start[c + 1];
                    } else {
                        t0 = (uint32_t)cm.y;
                        t1 = (uint32_t)cm.z;
                    }
                    for (uint32_t j = t0; j < t1; j += 32) {
                        const uint32_t t = j + lane;
                        int32_t cx[D];
#pragma unroll
                        for (int k = 0; k < D; ++k) cx[k] = 0;
                        uint2 cr = make_uint2(0xffffffffu, 0u);
                        if (t < t1) {
                            const uint32_t q = db.lplist ? db.lplist[t] : t;
                            cr = v.ro_s[q];
                            t_load<D>(recg + (int64_t)q * DP, cx);
                        }
                        const int nk = (int)min(32u, t1 - j);
                        for (int k = 0; k < nk; ++k) {
                            const uint32_t rk = __shfl_sync(kAll, cr.x, k);
                            const uint32_t ok = __shfl_sync(kAll, cr.y, k);
                            long long dd = 0;
#pragma unroll
                            for (int e = 0; e < D; ++e) {
                                const long long f = (long long)x[e] - __shfl_sync(kAll, cx[e], k);
                                dd += f * f;
                            }
                            if (act && rk < ro.x) {
                                ++tests;
                                if (dd < bestD || (dd == bestD && ok < bestJ)) {
                                    bestD = dd;
                                    bestJ = ok;
                                }
                            }
                        }
                    }
                } else {
                    const int32_t l = compact ? link_left((uint32_t)cm.y) : cm.y;
                    const int32_t r = compact ? link_right((uint32_t)cm.y) : cm.z;
                    int4 ml, mr;
                    const long long dl = w_test<D>(db, compact, dpb, l, x, ro.x, ml);
                    const long long dr2 = w_test<D>(db, compact, dpb, r, x, ro.x, mr);
                    const bool inl = act && !out_of_reach(dl, bestD), inr = act && !out_of_reach(dr2, bestD);
                    const unsigned bl_ = __ballot_sync(kAll, inl), br_ = __ballot_sync(kAll, inr);
                    if (bl_ && br_) {
                        const unsigned pr = __ballot_sync(kAll, inl && inr && dr2 < dl);
                        const unsigned pl = __ballot_sync(kAll, inl && inr && !(dr2 < dl));
                        const bool rfirst = __popc(pr) > __popc(pl);
                        if (sp < kWStack) {
                            s_lb[wi][sp][lane] = lb32(rfirst ? dl : dr2);
                            if (lane == 0) {
                                const int4 fm = rfirst ? ml : mr;
                                s_ent[wi][sp] = make_int4(rfirst ? l : r, fm.y, fm.z, (int)(rfirst ? bl_ : br_));
                            }
                            ++sp;
                        } else if (lane == 0) {
                            atomicOr(v.err, kErrTreeStack);
                        }
                        cur = rfirst ? r : l;
                        cm = rfirst ? mr : ml;
                        m = rfirst ? br_ : bl_;
                        next = true;
                    } else if (bl_) {
                        cur = l;
                        cm = ml;
                        m = bl_;
                        next = true;
                    } else if (br_) {
                        cur = r;
                        cm = mr;
                        m = br_;
                        next = true;
                    }
                }
                while (!next && sp > 0) {
                    --sp;
                    __syncwarp();
                    const int4 e = s_ent[wi][sp];
                    const uint32_t lb = s_lb[wi][sp][lane];
                    const unsigned mm = __ballot_sync(kAll, (((unsigned)e.w >> lane) & 1u) && (long long)lb <= bestD);
                    if (mm) {
                        cur = e.x;
                        cm = make_int4(0, e.y, e.z, 0);
                        m = mm;
                        next = true;
                    }
                }
                if (!next) m = 0;
                __syncwarp();
            }
        }
        if (b >= 0) {
            const int64_t g = v.desc[b].pt_off + ro.y;
            v.dep[g] = (int32_t)bestJ;
            v.delta2[g] = bestD;
        }
    }
    for (int o = 16; o > 0; o >>= 1) tests += __shfl_xor_sync(kAll, tests, o);
    if (lane == 0 && db.stats) {
        atomicAdd(&db.stats[0], visits);
        atomicAdd(&db.stats[1], tests);
    }
}

}  // namespace

cudaError_t launch_tree_build(const BatchView& v, const DeltaBufs& db, cudaStream_t st) {
    if (db.ncells == 0) return cudaSuccess;
    (k_cell_ranges<<<grid_for(v.B + 1, 128), 128, 0, st>>>(v, db), note_launch());
    (k_cell_key<<<grid_for(db.ncells, 256), 256, 0, st>>>(v, db), note_launch());
    (k_radix_tree<<<grid_for(db.ncells, 256), 256, 0, st>>>(v, db), note_launch());
    (k_leaves<<<(unsigned)std::min<int64_t>(152 * 16, grid_for(db.ncells, 256)), 256, 0, st>>>(v, db), note_launch());
    (k_refit<<<grid_for(db.ncells, 256), 256, 0, st>>>(v, db), note_launch());
    return cudaGetLastError();
}

template <int D>
static void k_tree_search_launch(const BatchView& v, const DeltaBufs& db, unsigned blocks, cudaStream_t st) {
    if (db.key_bits <= 30) (k_tree_search<D, 32><<<blocks, 128, 0, st>>>(v, db), note_launch());
    else (k_tree_search<D, kStack><<<blocks, 128, 0, st>>>(v, db), note_launch());
}

cudaError_t launch_tree_search(const BatchView& v, const DeltaBufs& db, uint32_t dim_mask, int64_t bound,
                               int warp, cudaStream_t st) {
    if (bound <= 0) return cudaSuccess;
    // one lane per point: 32 blocks per SM of grid-stride threads (16 and 64
    // measured slower); warp-cooperative: 8 blocks of 4 warps per SM
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 32, grid_for(bound, 128));
    const unsigned wblocks = (unsigned)std::min<int64_t>(152 * 8, grid_for(bound, kWWarps * 32));
#define DPC_TREE_CLASS(D)                                                                  \
    if (dim_mask & (1u << (D - 1))) {                                                      \
        if (warp == 1 || (warp == 2 && D >= 5))                                            \
            (k_tree_search_warp<D><<<wblocks, kWWarps * 32, 0, st>>>(v, db), note_launch()); \
        else                                                                               \
            k_tree_search_launch<D>(v, db, blocks, st);                                    \
    }
    DPC_TREE_CLASS(1) DPC_TREE_CLASS(2) DPC_TREE_CLASS(3) DPC_TREE_CLASS(4)
    DPC_TREE_CLASS(5) DPC_TREE_CLASS(6) DPC_TREE_CLASS(7) DPC_TREE_CLASS(8)
#undef DPC_TREE_CLASS
    return cudaGetLastError();
}

}  // namespace dpc
