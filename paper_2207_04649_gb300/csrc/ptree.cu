// Point tree: local density and dependent points for datasets with more
// dimensions than the grid covers.
//
// The paper's exact algorithm (Ex-DPC, Section 3) answers both questions on
// a kd-tree: the local density of a point is a range count of the open ball
// of radius d_cut around it (Definition 1), and its dependent point is the
// nearest point of higher density (Definitions 2-3), found by a nearest-
// neighbour search over the points inserted so far, i.e. the higher ones.
// Here the tree is built once, without insertions: the dataset's points are
// sorted by the Morton code of all their coordinates (each quantized to tb
// bits of its span), every kLeaf consecutive sorted points form a leaf, and
// a complete binary tree over the leaves (heap order) carries each node's
// bounding box, point count and, once ranks exist, smallest rank. A subtree
// whose smallest rank is not above the point's holds no candidate, which
// stands in for the paper's incremental insertion. The rank order is
// (rho desc, index asc), distances are exact squared 64-bit integers, and
// ties in distance go to the smaller original index.
#include "stages.cuh"
#include <algorithm>

namespace dpc {

namespace {

constexpr int kPtStack = 40;  // the heap is at most 28 levels deep (n < 2^31, kLeaf = 16)

// Last j in [0, m) with off[j] <= x (off strictly increasing).
__device__ __forceinline__ int pt_find(const int64_t* off, int m, int64_t x) {
    int lo = 0, hi = m - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Leaf boxes and counts, then a bottom-up merge: the second child to arrive
// at a node writes the node's record.
__global__ void k_pt_leaves(BatchView v, PtBufs pb) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= pb.nslots) return;
    const int j = pt_find(pb.leaf_off, pb.m, s);
    const DsDesc& ds = v.desc[pb.ds_idx[j]];
    const int64_t leaf = s - pb.leaf_off[j];
    const int64_t first_leaf = (1ll << ds.h) - 1;
    int4* nodes = pb.nodes + ds.node_off * kPtRec;
    int32_t lo[8], hi[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        lo[k] = INT32_MAX;
        hi[k] = INT32_MIN;
    }
    const int64_t q0 = min(leaf * kLeaf, (int64_t)ds.n), q1 = min(q0 + kLeaf, (int64_t)ds.n);
    for (int64_t q = q0; q < q1; ++q) {
        const int4* r = v.rec + ds.rec_off + q * ds.dp;
        const int4 a = r[0];
        const int4 e = ds.dp == 2 ? r[1] : make_int4(0, 0, 0, 0);
        const int32_t x[8] = {a.x, a.y, a.z, a.w, e.x, e.y, e.z, e.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            lo[k] = min(lo[k], x[k]);
            hi[k] = max(hi[k], x[k]);
        }
    }
    int64_t node = first_leaf + leaf;
    int4* rec = nodes + node * kPtRec;
    rec[0] = make_int4(lo[0], lo[1], lo[2], lo[3]);
    rec[1] = make_int4(lo[4], lo[5], lo[6], lo[7]);
    rec[2] = make_int4(hi[0], hi[1], hi[2], hi[3]);
    rec[3] = make_int4(hi[4], hi[5], hi[6], hi[7]);
    rec[4] = make_int4(-1, (int)(q1 - q0), (int)(ds.pt_off + q0), 0);
    while (node > 0) {
        const int64_t par = (node - 1) >> 1;
        __threadfence();
        if (atomicAdd(&pb.flag[ds.leaf_off + par], 1u) == 0u) return;
        __threadfence();
        const int4* a = nodes + (2 * par + 1) * kPtRec;
        const int4* c = a + kPtRec;
        int4* o = nodes + par * kPtRec;
        for (int q = 0; q < 4; ++q) {
            const int4 x = __ldcg(a + q), y = __ldcg(c + q);
            o[q] = q < 2 ? make_int4(min(x.x, y.x), min(x.y, y.y), min(x.z, y.z), min(x.w, y.w))
                         : make_int4(max(x.x, y.x), max(x.y, y.y), max(x.z, y.z), max(x.w, y.w));
        }
        const int4 ma = __ldcg(a + 4), mc = __ldcg(c + 4);
        o[4] = make_int4(-1, ma.y + mc.y, ma.z, 0);  // leaves fill from the left: the left child starts the range
        node = par;
    }
}

// Smallest rank of every node, bottom-up the same way.
__global__ void k_pt_minrank(BatchView v, PtBufs pb) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= pb.nslots) return;
    const int j = pt_find(pb.leaf_off, pb.m, s);
    const DsDesc& ds = v.desc[pb.ds_idx[j]];
    const int64_t leaf = s - pb.leaf_off[j];
    const int64_t first_leaf = (1ll << ds.h) - 1;
    int4* nodes = pb.nodes + ds.node_off * kPtRec;
    const int64_t q0 = min(leaf * kLeaf, (int64_t)ds.n), q1 = min(q0 + kLeaf, (int64_t)ds.n);
    uint32_t mr = 0xffffffffu;
    for (int64_t q = q0; q < q1; ++q) mr = min(mr, v.ro_s[ds.pt_off + q].x);
    int64_t node = first_leaf + leaf;
    nodes[node * kPtRec + 4].x = (int)mr;
    while (node > 0) {
        const int64_t par = (node - 1) >> 1;
        __threadfence();
        if (atomicAdd(&pb.flag[ds.leaf_off + par], 1u) == 0u) return;
        __threadfence();
        const uint32_t ma = (uint32_t)__ldcg(&nodes[(2 * par + 1) * kPtRec + 4].x);
        const uint32_t mc = (uint32_t)__ldcg(&nodes[(2 * par + 2) * kPtRec + 4].x);
        nodes[par * kPtRec + 4].x = (int)min(ma, mc);
        node = par;
    }
}

template <int D>
__device__ __forceinline__ void pt_load(const int4* r, int32_t (&x)[D]) {
    const int4 a = r[0];
    int32_t t[8] = {a.x, a.y, a.z, a.w, 0, 0, 0, 0};
    if (D > 4) {
        const int4 e = r[1];
        t[4] = e.x; t[5] = e.y; t[6] = e.z; t[7] = e.w;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = t[k];
}

// Squared distances from x to the nearest and to the farthest point of a
// node's (non-empty) box.
template <int D>
__device__ __forceinline__ void box_range(const int4* r, const int32_t (&x)[D], long long& mn, long long& mx) {
    int32_t lo[D], hi[D];
    pt_load<D>(r, lo);
    pt_load<D>(r + 2, hi);
    mn = 0;
    mx = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const long long a = (long long)x[k] - lo[k], c = (long long)hi[k] - x[k];
        const long long near = a < 0 ? -a : (c < 0 ? -c : 0);
        const long long far = max(a < 0 ? -a : a, c < 0 ? -c : c);
        mn += near * near;
        mx += far * far;
    }
}

template <int D>
__device__ __forceinline__ long long box_min(const int4* r, const int32_t (&x)[D]) {
    int32_t lo[D], hi[D];
    pt_load<D>(r, lo);
    pt_load<D>(r + 2, hi);
    long long mn = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const long long a = (long long)lo[k] - x[k], c = (long long)x[k] - hi[k];
        const long long near = a > 0 ? a : (c > 0 ? c : 0);
        mn += near * near;
    }
    return mn;
}

template <int D>
__device__ __forceinline__ long long sq_dist(const int32_t (&x)[D], const int32_t (&y)[D]) {
    long long s = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const long long e = (long long)x[k] - y[k];
        s += e * e;
    }
    return s;
}

// Local density (Definition 1, self included): a node entirely inside the
// ball adds its count, a node entirely outside is skipped, leaves in
// between test their points.
template <int D>
__global__ void __launch_bounds__(128) k_rho_ptree(BatchView v, PtBufs pb, int64_t t0, int64_t t1) {
    constexpr int DP = D <= 4 ? 1 : 2;
    unsigned long long visits = 0, tests = 0;
    for (int64_t t = t0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < t1;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int j = pt_find(pb.pt_off, pb.m, t);
        const DsDesc& ds = v.desc[pb.ds_idx[j]];
        const int64_t q = t - pb.pt_off[j];
        const int4* recs = v.rec + ds.rec_off - ds.pt_off * DP;  // indexed by global sorted position
        int32_t x[D];
        pt_load<D>(recs + (ds.pt_off + q) * DP, x);
        const int4* nodes = pb.nodes + ds.node_off * kPtRec;
        const int64_t first_leaf = (1ll << ds.h) - 1;
        const long long dc2 = ds.d_cut2;
        int32_t stack[kPtStack];
        int sp = 0;
        stack[sp++] = 0;
        int32_t rho = 0;
        while (sp > 0) {
            const int32_t i = stack[--sp];
            ++visits;
            const int4* r = nodes + (int64_t)i * kPtRec;
            const int4 meta = r[4];
            if (meta.y == 0) continue;
            long long mn, mx;
            box_range<D>(r, x, mn, mx);
            if (mn >= dc2) continue;
            if (mx < dc2) {
                rho += meta.y;
                continue;
            }
            if (i >= first_leaf) {
                for (int32_t u = 0; u < meta.y; ++u) {
                    int32_t y[D];
                    pt_load<D>(recs + ((int64_t)meta.z + u) * DP, y);
                    rho += sq_dist<D>(x, y) < dc2 ? 1 : 0;
                }
                tests += (unsigned long long)meta.y;
            } else if (sp + 2 > kPtStack) {
                atomicOr(v.err, kErrTreeStack);
            } else {
                stack[sp++] = 2 * i + 2;
                stack[sp++] = 2 * i + 1;
            }
        }
        v.rho_s[ds.pt_off + q] = rho;
    }
    for (int o = 16; o > 0; o >>= 1) {
        visits += __shfl_xor_sync(0xffffffffu, visits, o);
        tests += __shfl_xor_sync(0xffffffffu, tests, o);
    }
    if ((threadIdx.x & 31) == 0 && pb.stats) {
        atomicAdd(&pb.stats[0], visits);
        atomicAdd(&pb.stats[1], tests);
    }
}

// Dependent point (Definitions 2-3): depth first, nearer child first; a
// subtree is skipped when nothing in it ranks higher or when its box is
// farther than the best distance so far (equal distances are kept: a
// smaller index may win the tie).
template <int D>
__global__ void __launch_bounds__(128) k_delta_ptree(BatchView v, PtBufs pb, int64_t t0, int64_t t1) {
    constexpr int DP = D <= 4 ? 1 : 2;
    unsigned long long visits = 0, tests = 0;
    for (int64_t t = t0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < t1;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int j = pt_find(pb.pt_off, pb.m, t);
        const DsDesc& ds = v.desc[pb.ds_idx[j]];
        const int64_t p = ds.pt_off + (t - pb.pt_off[j]);
        const int4* recs = v.rec + ds.rec_off - ds.pt_off * DP;
        int32_t x[D];
        pt_load<D>(recs + p * DP, x);
        const uint2 ro = v.ro_s[p];
        const int4* nodes = pb.nodes + ds.node_off * kPtRec;
        const int64_t first_leaf = (1ll << ds.h) - 1;
        long long best = INT64_MAX;
        uint32_t bestJ = 0xffffffffu;
        int32_t sn[kPtStack];
        long long sd[kPtStack];
        int sp = 0;
        {
            const int4 meta = nodes[4];
            if (meta.y > 0 && (uint32_t)meta.x < ro.x) {
                sn[0] = 0;
                sd[0] = box_min<D>(nodes, x);
                sp = 1;
            }
        }
        while (sp > 0) {
            --sp;
            const int32_t i = sn[sp];
            if (sd[sp] > best) continue;
            ++visits;
            if (i >= first_leaf) {
                const int4 meta = nodes[(int64_t)i * kPtRec + 4];
                for (int32_t u = 0; u < meta.y; ++u) {
                    const uint2 cr = v.ro_s[meta.z + u];
                    if (cr.x >= ro.x) continue;
                    ++tests;
                    int32_t y[D];
                    pt_load<D>(recs + ((int64_t)meta.z + u) * DP, y);
                    const long long dd = sq_dist<D>(x, y);
                    if (dd < best || (dd == best && cr.y < bestJ)) {
                        best = dd;
                        bestJ = cr.y;
                    }
                }
                continue;
            }
            const int4* ra = nodes + (int64_t)(2 * i + 1) * kPtRec;
            const int4* rc = ra + kPtRec;
            const int4 ma = ra[4], mc = rc[4];
            const long long da = (ma.y > 0 && (uint32_t)ma.x < ro.x) ? box_min<D>(ra, x) : INT64_MAX;
            const long long dc = (mc.y > 0 && (uint32_t)mc.x < ro.x) ? box_min<D>(rc, x) : INT64_MAX;
            if (sp + 2 > kPtStack) {
                atomicOr(v.err, kErrTreeStack);
                continue;
            }
            const bool a_first = da <= dc;
            const int32_t nn = a_first ? 2 * i + 1 : 2 * i + 2, fn = a_first ? 2 * i + 2 : 2 * i + 1;
            const long long dn = a_first ? da : dc, df = a_first ? dc : da;
            if (df != INT64_MAX && df <= best) {
                sn[sp] = fn;
                sd[sp++] = df;
            }
            if (dn != INT64_MAX && dn <= best) {
                sn[sp] = nn;
                sd[sp++] = dn;
            }
        }
        const int64_t g = ds.pt_off + ro.y;
        v.dep[g] = (int32_t)bestJ;  // -1 for the densest point
        v.delta2[g] = best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        visits += __shfl_xor_sync(0xffffffffu, visits, o);
        tests += __shfl_xor_sync(0xffffffffu, tests, o);
    }
    if ((threadIdx.x & 31) == 0 && pb.stats) {
        atomicAdd(&pb.stats[2], visits);
        atomicAdd(&pb.stats[3], tests);
    }
}

}  // namespace

cudaError_t launch_pt_build(const BatchView& v, const PtBufs& pb, cudaStream_t st) {
    if (pb.m == 0 || pb.nslots == 0) return cudaSuccess;
    (k_pt_leaves<<<grid_for(pb.nslots, 256), 256, 0, st>>>(v, pb), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_pt_minrank(const BatchView& v, const PtBufs& pb, cudaStream_t st) {
    if (pb.m == 0 || pb.nslots == 0) return cudaSuccess;
    (k_pt_minrank<<<grid_for(pb.nslots, 256), 256, 0, st>>>(v, pb), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_rho_ptree(const BatchView& v, const PtBufs& pb, int d, int64_t t0, int64_t t1, cudaStream_t st) {
    if (t1 <= t0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(t1 - t0, 128));
    switch (d) {
#define DPC_PT_RHO(D) \
    case D: (k_rho_ptree<D><<<blocks, 128, 0, st>>>(v, pb, t0, t1), note_launch()); break;
        DPC_PT_RHO(1) DPC_PT_RHO(2) DPC_PT_RHO(3) DPC_PT_RHO(4)
        DPC_PT_RHO(5) DPC_PT_RHO(6) DPC_PT_RHO(7) DPC_PT_RHO(8)
#undef DPC_PT_RHO
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_delta_ptree(const BatchView& v, const PtBufs& pb, int d, int64_t t0, int64_t t1,
                               cudaStream_t st) {
    if (t1 <= t0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(t1 - t0, 128));
    switch (d) {
#define DPC_PT_DELTA(D) \
    case D: (k_delta_ptree<D><<<blocks, 128, 0, st>>>(v, pb, t0, t1), note_launch()); break;
        DPC_PT_DELTA(1) DPC_PT_DELTA(2) DPC_PT_DELTA(3) DPC_PT_DELTA(4)
        DPC_PT_DELTA(5) DPC_PT_DELTA(6) DPC_PT_DELTA(7) DPC_PT_DELTA(8)
#undef DPC_PT_DELTA
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dpc
