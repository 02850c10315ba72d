// Expanding search for the dependent points the ring search left open.
//
// A binary radix tree over the Morton-ordered cells of each dataset: leaf c
// is grid cell c (a contiguous run of sorted points), and every internal
// node covers the cells sharing a longest common key prefix, i.e. an
// axis-aligned box of cells. It is built in one parallel pass from the
// sorted unique cell keys (each internal node finds its key range and split
// point by binary searches on common-prefix lengths, the construction of
// Karras, "Maximizing parallelism in the construction of BVHs, octrees, and
// k-d trees", HPG 2012), then refitted bottom-up: every node stores the
// bounding box of its points and the smallest rank (highest density) among
// them.
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

// Leaf boxes and smallest ranks, then a bottom-up refit: the second child to
// arrive at a node computes it.
__global__ void k_refit(BatchView v, DeltaBufs db) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= db.ncells) return;
    const int dpb = db.dpb;
    const int b = find_off(db.cell_off, v.B, c);
    const DsDesc& ds = v.desc[b];
    int32_t lo[8], hi[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        lo[k] = INT32_MAX;
        hi[k] = INT32_MIN;
    }
    uint32_t mr = 0xffffffffu;
    const uint32_t p0 = v.cell_start[c], p1 = v.cell_start[c + 1];
    for (uint32_t p = p0; p < p1; ++p) {
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
    int4* lb = db.lbox + c * 2 * dpb;
    lb[0] = make_int4(lo[0], lo[1], lo[2], lo[3]);
    if (dpb == 2) lb[1] = make_int4(lo[4], lo[5], lo[6], lo[7]);
    lb[dpb] = make_int4(hi[0], hi[1], hi[2], hi[3]);
    if (dpb == 2) lb[dpb + 1] = make_int4(hi[4], hi[5], hi[6], hi[7]);
    db.lmin[c] = mr;
    int32_t node = db.lparent[c];
    while (node >= 0) {
        __threadfence();
        if (atomicAdd(&db.flag[node], 1u) == 0u) return;
        __threadfence();
        const int2 ch = __ldcg(&db.child[node]);
        const int4* cb[2];
        uint32_t cm[2];
        const int32_t kids[2] = {ch.x, ch.y};
        for (int q = 0; q < 2; ++q) {
            if (kids[q] < 0) {
                cb[q] = db.lbox + (int64_t)(~kids[q]) * 2 * dpb;
                cm[q] = __ldcg(&db.lmin[~kids[q]]);
            } else {
                cb[q] = db.ibox + (int64_t)kids[q] * 2 * dpb;
                cm[q] = __ldcg(&db.imin[kids[q]]);
            }
        }
        int4* nb = db.ibox + (int64_t)node * 2 * dpb;
        for (int q = 0; q < 2 * dpb; ++q) {
            const int4 x = __ldcg(cb[0] + q), y = __ldcg(cb[1] + q);
            nb[q] = q < dpb ? make_int4(min(x.x, y.x), min(x.y, y.y), min(x.z, y.z), min(x.w, y.w))
                            : make_int4(max(x.x, y.x), max(x.y, y.y), max(x.z, y.z), max(x.w, y.w));
        }
        db.imin[node] = min(cm[0], cm[1]);
        node = __ldcg(&db.iparent[node]);
    }
}

template <int D>
__device__ __forceinline__ void load_box(const int4* box, int dpb, int32_t (&lo)[D], int32_t (&hi)[D]) {
    const int4 l0 = box[0], h0 = box[dpb];
    int32_t a[8] = {l0.x, l0.y, l0.z, l0.w, 0, 0, 0, 0};
    int32_t z[8] = {h0.x, h0.y, h0.z, h0.w, 0, 0, 0, 0};
    if (D > 4) {
        const int4 l1 = box[1], h1 = box[dpb + 1];
        a[4] = l1.x; a[5] = l1.y; a[6] = l1.z; a[7] = l1.w;
        z[4] = h1.x; z[5] = h1.y; z[6] = h1.z; z[7] = h1.w;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
        lo[k] = a[k];
        hi[k] = z[k];
    }
}

template <int D>
__device__ __forceinline__ long long box_dist(const int4* box, int dpb, const int32_t (&x)[D]) {
    int32_t lo[D], hi[D];
    load_box<D>(box, dpb, lo, hi);
    long long s = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const long long dd = x[k] < lo[k] ? (long long)lo[k] - x[k] : (x[k] > hi[k] ? (long long)x[k] - hi[k] : 0);
        s += dd * dd;
    }
    return s;
}

// The ball of squared radius r2 around x lies inside the box in every
// gridded dimension (bit k of gmask).
template <int D>
__device__ __forceinline__ bool ball_inside(const int4* box, int dpb, const int32_t (&x)[D], uint32_t gmask,
                                            long long r2) {
    int32_t lo[D], hi[D];
    load_box<D>(box, dpb, lo, hi);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        if (!((gmask >> k) & 1u)) continue;
        const long long a = (long long)x[k] - lo[k], b = (long long)hi[k] - x[k];
        if (a < 0 || b < 0 || a * a < r2 || b * b < r2) return false;
    }
    return true;
}

constexpr int kStack = 96;

template <int D>
__global__ void __launch_bounds__(128) k_tree_search(BatchView v, DeltaBufs db) {
    constexpr int DP = D <= 4 ? 1 : 2;
    const uint32_t cnt = db.ucount[0];
    const int dpb = db.dpb;
    unsigned long long visits = 0, tests = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
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
        int32_t stack[kStack];
        const int64_t c0 = db.cell_off[b], c1 = db.cell_off[b + 1];
        {
            int sp = 0;
            stack[sp++] = c1 - c0 >= 2 ? (int32_t)c0 : ~(int32_t)c0;  // the dataset's root
            while (sp > 0) {
                const int32_t nd = stack[--sp];
                ++visits;
                if (nd < 0) {
                    const int32_t c = ~nd;
                    if (db.lmin[c] >= ro.x) continue;
                    if (box_dist<D>(db.lbox + (int64_t)c * 2 * dpb, dpb, x) > bestD) continue;
                    const uint32_t q1 = v.cell_start[c + 1];
                    for (uint32_t q = v.cell_start[c]; q < q1; ++q) {
                        const uint2 cr = v.ro_s[q];
                        if (cr.x >= ro.x) continue;
                        ++tests;
                        int32_t cx[D];
                        t_load<D>(recb + (int64_t)q * DP, cx);
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
                    continue;
                }
                if (db.imin[nd] >= ro.x) continue;
                if (box_dist<D>(db.ibox + (int64_t)nd * 2 * dpb, dpb, x) > bestD) continue;
                if (sp + 2 > kStack) {
                    atomicOr(v.err, kErrTreeStack);
                    continue;
                }
                const int2 cc = db.child[nd];
                long long dk[2];
                const int32_t kid[2] = {cc.x, cc.y};
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const bool leaf = kid[q] < 0;
                    const int64_t id = leaf ? ~kid[q] : kid[q];
                    const uint32_t mr = leaf ? db.lmin[id] : db.imin[id];
                    dk[q] = mr < ro.x ? box_dist<D>((leaf ? db.lbox : db.ibox) + id * 2 * dpb, dpb, x) : INT64_MAX;
                }
                // push the farther child first so the nearer one is searched first
                const int nearer = dk[1] < dk[0] ? 1 : 0;
                if (dk[1 - nearer] <= bestD) stack[sp++] = kid[1 - nearer];
                if (dk[nearer] <= bestD) stack[sp++] = kid[nearer];
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

}  // namespace

cudaError_t launch_tree_build(const BatchView& v, const DeltaBufs& db, cudaStream_t st) {
    if (db.ncells == 0) return cudaSuccess;
    (k_cell_ranges<<<grid_for(v.B + 1, 128), 128, 0, st>>>(v, db), note_launch());
    (k_cell_key<<<grid_for(db.ncells, 256), 256, 0, st>>>(v, db), note_launch());
    (k_radix_tree<<<grid_for(db.ncells, 256), 256, 0, st>>>(v, db), note_launch());
    (k_refit<<<grid_for(db.ncells, 256), 256, 0, st>>>(v, db), note_launch());
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

}  // namespace dpc
