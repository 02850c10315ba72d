// Local density (Definition 1): rho_i = #{ j : dist(p_i, p_j) < d_cut },
// p_i itself included, compared exactly as sum_k (x_ik - x_jk)^2 < d_cut^2
// in integers.
//
// Candidates for the points of a cell are the points of its neighbour cells
// (the cell itself included). Handling all points of a cell against one
// candidate list is the paper's joint range search (Section 4.2: one range
// query per cell, then a scan of the result for every member), with the
// neighbour cells of the grid in place of the kd-tree query.
//
// Preparation: one warp per cell looks up the cell's (2R+1)^k neighbours in
// the hash table in parallel (one lane each) and stores the non-empty ones as
// runs (start, count) of sorted points, with the candidate count. The hot
// kernels then read runs only; the ring search of the delta stage reuses them.
//
// Two kernels share the pair work:
//  * dense cells (more than kSparseMax points): one warp per work item
//    (cell, chunk of up to 128 queries, chunk of candidates). Candidates are
//    staged in shared memory from the runs with 128-bit loads. A chunk of 32
//    or more queries keeps 1-4 queries per lane; a smaller one is split over
//    the lanes in 2 or 4 groups, each group taking every 2nd or 4th
//    candidate, and the groups' counts are added with warp shuffles. Items
//    are claimed from an atomic counter by persistent warps.
//  * sparse cells: one thread per cell, its few queries in registers,
//    candidates read from the runs with unrolled 128-bit loads.
//
// Pair arithmetic: when every candidate difference is small enough
// (DsDesc::w32) the test runs in 32-bit integers as the sign of
// sum_k dx_k^2 - d_cut^2; otherwise in 64-bit integers.
#include "stages.cuh"
#include <algorithm>

namespace dpc {

namespace {

constexpr int kRhoThreads = 128;  // 4 warps per block, double-buffered chunks each

// A cell is dense (one warp per work item) when it holds more than
// kSparseMax points or has more than sparse_cand candidates (a few points
// facing many candidates, as in high dimensions, would leave one thread
// walking them all); the others take one thread each. Counts the candidate
// pairs of both classes.
__global__ void k_classify(BatchView v, CellPrepBufs cb, int64_t bound, uint32_t sparse_cand) {
    const uint32_t nc = *v.ncells;
    unsigned long long pairs = 0, spairs = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < bound; c += (int64_t)gridDim.x * blockDim.x) {
        uint32_t dense = 0, sparse = 0;
        if (c < nc) {
            const uint32_t m = v.cell_start[c + 1] - v.cell_start[c];
            const uint32_t cand = cb.cand[c];
            dense = m > (uint32_t)kSparseMax || cand > sparse_cand;
            sparse = !dense;
            if (dense) pairs += (unsigned long long)m * cand;
            else spairs += (unsigned long long)m * cand;
        }
        cb.dflag[c] = dense;
        cb.sflag[c] = sparse;
    }
    for (int o = 16; o > 0; o >>= 1) {
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        spairs += __shfl_xor_sync(0xffffffffu, spairs, o);
    }
    if ((threadIdx.x & 31) == 0 && pairs) atomicAdd(&cb.stats[0], pairs);
    if ((threadIdx.x & 31) == 0 && spairs) atomicAdd(&cb.stats[1], spairs);
}

__global__ void k_compact_cells(BatchView v, CellPrepBufs cb, int64_t bound) {
    const uint32_t nc = *v.ncells;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < bound; c += (int64_t)gridDim.x * blockDim.x) {
        if (c >= nc) break;
        if (cb.dflag[c]) cb.dense[cb.didx[c]] = (uint32_t)c;
        else if (cb.sflag[c]) cb.sparse[cb.sidx[c]] = (uint32_t)c;
    }
}

constexpr int kProbeBatch = 3;  // hash probes issued together per thread (3 to 6 measured alike, 9 and more slower)

__device__ __forceinline__ uint2 resolve_probe(const BatchView& v, uint64_t key, int4 e) {
    const uint64_t k0 = (uint64_t)(uint32_t)e.x | ((uint64_t)(uint32_t)e.y << 32);
    if (k0 == key) return make_uint2((uint32_t)e.z, (uint32_t)e.w);
    if (k0 == kEmptyKey) return make_uint2(0u, 0u);
    return hash_find(v.hash, v.hmask, key);  // collision: keep probing
}

// One thread per cell of a dataset gridded in K dims with reach R = 1. The
// 3^K neighbour offsets are compile-time constants; a neighbour's key comes
// from the cell's own key by carry/borrow steps inside each dim's Morton
// bits; first hash probes are issued kProbeBatch at a time as independent
// loads, then resolved. Non-empty neighbours become the cell's runs, in
// neighbour order.
template <int K>
__global__ void __launch_bounds__(256) k_cell_runs(BatchView v, CellPrepBufs cb, int64_t ncells) {
    constexpr int NNB = K == 1 ? 3 : (K == 2 ? 9 : (K == 3 ? 27 : 81));
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t cs = v.cell_start[c];
        const int b = find_ds(v.pt_off, v.B, cs);
        const DsDesc& ds = v.desc[b];
        if (ds.k != K || ds.R != 1 || ds.sbits != 0) continue;
        const int4* r0 = v.rec + ds.rec_off + ((int64_t)cs - ds.pt_off) * ds.dp;
        int32_t cc[K];
#pragma unroll
        for (int j = 0; j < K; ++j)
            cc[j] = (int32_t)((uint32_t)(rec_coord(r0, ds.gdim[j]) - ds.origin[j]) / (uint32_t)ds.s);
        const uint64_t own = v.key[cs] - ds.cbase;
        uint32_t nr = 0, cand = 0;
        uint2* runs = cb.runs + c * cb.nbs;
#pragma unroll
        for (int base = 0; base < NNB; base += kProbeBatch) {
            uint64_t key[kProbeBatch];
            int4 e[kProbeBatch];
#pragma unroll
            for (int q = 0; q < kProbeBatch; ++q) {
                const int t = base + q;
                key[q] = kEmptyKey;
                if (t < NNB) {
                    bool ok = true;
                    int nz = 0;
                    uint64_t code = own;
                    int tt = t;
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        const int o = tt % 3 - 1;
                        tt /= 3;
                        if (o != 0) {
                            ++nz;
                            ok = ok && cc[j] + o >= 0 && cc[j] + o < ds.ext[j];
                            code = morton_step(code, ds.dmask[j], o);
                        }
                    }
                    // offsets in nz dims: boxes at least sqrt(nz) apart
                    if (ok && nz < ds.d_cut2) key[q] = ds.cbase + code;
                }
                e[q] = key[q] != kEmptyKey ? __ldg(&v.hash[mix64(key[q]) & v.hmask]) : make_int4(-1, -1, 0, 0);
            }
#pragma unroll
            for (int q = 0; q < kProbeBatch; ++q) {
                if (key[q] == kEmptyKey) continue;
                const uint2 r = resolve_probe(v, key[q], e[q]);
                if (r.y > 0u) {
                    runs[nr++] = r;
                    cand += r.y;
                }
            }
        }
        cb.nruns[c] = nr;
        cb.cand[c] = cand;
    }
}

// Local Morton codes of a block (K dims, L bits per dim, K * L <= 6) whose
// coordinate along dim j is c: bit i of dim j sits at code bit i * K + j.
__device__ __forceinline__ unsigned long long code_bit(int q) {
    switch (q) {
        case 0: return 0xAAAAAAAAAAAAAAAAull;
        case 1: return 0xCCCCCCCCCCCCCCCCull;
        case 2: return 0xF0F0F0F0F0F0F0F0ull;
        case 3: return 0xFF00FF00FF00FF00ull;
        case 4: return 0xFFFF0000FFFF0000ull;
        default: return 0xFFFFFFFF00000000ull;
    }
}

template <int K, int L>
__device__ __forceinline__ unsigned long long coord_codes(int j, int c) {
    unsigned long long m = K * L >= 6 ? ~0ull : ((1ull << (1 << (K * L))) - 1ull);  // 2^(K L) codes
#pragma unroll
    for (int i = 0; i < L; ++i) {
        const unsigned long long p = code_bit(i * K + j);
        m &= ((c >> i) & 1) ? p : ~p;
    }
    return m;
}

// Codes whose coordinate along dim j lies in [a, e] (e - a <= 2).
template <int K, int L>
__device__ __forceinline__ unsigned long long range_codes(int j, int a, int e) {
    unsigned long long m = coord_codes<K, L>(j, a);
    if (e > a) m |= coord_codes<K, L>(j, a + 1);
    if (e > a + 1) m |= coord_codes<K, L>(j, a + 2);
    return m;
}

// Neighbour runs from the block table, one thread per cell of a dataset
// gridded in K dims with reach 1: the 3^K neighbourhood meets at most 2^K
// aligned blocks of W = 2^L cells per dim; each is one table probe, whose
// occupancy bitmap masked by the neighbourhood's box gives the non-empty
// neighbour cells, and a cell's index in the sorted cell order is the
// block's first cell plus the occupied codes below it. Neighbour cells whose
// indices follow one another hold consecutive points and become one run.
// The cell-index runs wait in shared memory (K <= 3: at most 3^K of them per
// cell, one column per thread) until their point ranges are looked up, so
// each run is written to global memory once.
constexpr int kRunsBlkThreads = 128;

template <int K>
__global__ void __launch_bounds__(kRunsBlkThreads) k_cell_runs_blk(BatchView v, CellPrepBufs cb, int64_t ncells) {
    constexpr int L = K == 1 ? 6 : (K == 2 ? 3 : (K == 3 ? 2 : 1));
    constexpr int W = 1 << L;
    constexpr int NB = 1 << K;  // blocks the neighbourhood can meet
    constexpr bool SM = K <= 3;
    constexpr int MAXR = K == 1 ? 3 : (K == 2 ? 9 : 27);
    __shared__ uint2 sruns[SM ? MAXR : 1][kRunsBlkThreads];
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t cs = v.cell_start[c];
        const int b = find_ds(v.pt_off, v.B, cs);
        const DsDesc& ds = v.desc[b];
        if (ds.k != K || ds.sbits == 0) continue;
        const int4* r0 = v.rec + ds.rec_off + ((int64_t)cs - ds.pt_off) * ds.dp;
        int32_t lo[K], hi[K], cbk[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int32_t cc = (int32_t)((uint32_t)(rec_coord(r0, ds.gdim[j]) - ds.origin[j]) / (uint32_t)ds.s);
            lo[j] = max(cc - 1, 0);
            hi[j] = min(cc + 1, ds.ext[j] - 1);
            cbk[j] = cc >> L;
        }
        const uint64_t own = (v.key[cs] - ds.cbase) >> (K * L);
        uint2* runs = cb.runs + c * cb.nbs;
        uint32_t nr = 0;
        uint32_t first_ci = 0, last_ci = 0;
        bool open = false;
        // per dim: the one or two blocks the neighbourhood meets, the codes
        // of its cells in each, and the step from the cell's own block
        unsigned long long dmask_codes[K][2];
        int dstep[K][2], nb[K];
        uint64_t bmask[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int blo = lo[j] >> L, bhi = hi[j] >> L;
            nb[j] = bhi != blo ? 2 : 1;
            dstep[j][0] = blo - cbk[j];
            dstep[j][1] = bhi - cbk[j];
            dmask_codes[j][0] = range_codes<K, L>(j, lo[j] - blo * W, min(hi[j], blo * W + W - 1) - blo * W);
            dmask_codes[j][1] = range_codes<K, L>(j, max(lo[j], bhi * W) - bhi * W, hi[j] - bhi * W);
            bmask[j] = ds.dmask[j] >> (K * L);
        }
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            bool ok = true;
            uint64_t code = own;
            unsigned long long box = ~0ull;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const int up = (t >> j) & 1;
                if (up >= nb[j]) ok = false;
                code = morton_step(code, bmask[j], dstep[j][up]);
                box &= dmask_codes[j][up];
            }
            if (!ok) continue;
            unsigned long long occ;
            const uint32_t f = block_find(v.sbhash, v.sbmask, ((uint64_t)b << 40) | code, occ);
            // the selected cells a piece at a time: a piece runs from the
            // lowest selected code up to the next occupied code outside the
            // box, so its cells have consecutive indices
            unsigned long long sel = occ & box;
            const unsigned long long gaps = occ & ~box;
            while (sel) {
                const int a = __ffsll((long long)sel) - 1;
                const unsigned long long above = ~0ull << a;
                const unsigned long long g = gaps & above;
                const unsigned long long seg = g ? (((g & (0ull - g)) - 1ull) & above) : above;
                sel &= ~seg;
                const uint32_t ci = f + (uint32_t)__popcll(occ & ~above);
                const uint32_t ce = ci + (uint32_t)__popcll(occ & box & seg) - 1u;
                if (open && ci == last_ci + 1u) {
                    last_ci = ce;
                } else {
                    if (open) {
                        if (SM) sruns[nr][threadIdx.x] = make_uint2(first_ci, last_ci);
                        else runs[nr] = make_uint2(first_ci, last_ci);
                        ++nr;
                    }
                    first_ci = ci;
                    last_ci = ce;
                    open = true;
                }
            }
        }
        if (open) {
            if (SM) sruns[nr][threadIdx.x] = make_uint2(first_ci, last_ci);
            else runs[nr] = make_uint2(first_ci, last_ci);
            ++nr;
        }
        // cell index ranges -> point runs (independent loads)
        uint32_t cand = 0;
#pragma unroll 4
        for (uint32_t r = 0; r < nr; ++r) {
            const uint2 e = SM ? sruns[r][threadIdx.x] : runs[r];
            const uint32_t p0 = v.cell_start[e.x], p1 = v.cell_start[e.y + 1];
            runs[r] = make_uint2(p0, p1 - p0);
            cand += p1 - p0;
        }
        cb.nruns[c] = nr;
        cb.cand[c] = cand;
    }
}

// Any k, any reach R (used when R != 1).
__global__ void __launch_bounds__(256) k_cell_runs_any(BatchView v, CellPrepBufs cb, int64_t ncells) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t cs = v.cell_start[c];
        const int b = find_ds(v.pt_off, v.B, cs);
        const DsDesc& ds = v.desc[b];
        if (ds.R == 1 && ds.k >= 1) continue;
        const int4* r0 = v.rec + ds.rec_off + ((int64_t)cs - ds.pt_off) * ds.dp;
        int32_t cc[kMaxGridDims];
        for (int j = 0; j < ds.k; ++j) cc[j] = cell_coord(ds, j, rec_coord(r0, ds.gdim[j]));
        const int nnb = num_neighbours(ds);
        uint32_t nr = 0, cand = 0;
        uint2* runs = cb.runs + c * cb.nbs;
        for (int t = 0; t < nnb; ++t) {
            int32_t nc[kMaxGridDims];
            if (!neighbour(ds, cc, t, nc)) continue;
            const uint2 r = hash_find(v.hash, v.hmask, ds.cbase + morton(nc, ds.k, ds.mbits));
            if (r.y > 0u) {
                runs[nr++] = r;
                cand += r.y;
            }
        }
        cb.nruns[c] = nr;
        cb.cand[c] = cand;
    }
}

// Work items per dense cell; zero for the slots in [ndense, bound) that the
// scan after it also reads.
__global__ void k_item_count(BatchView v, CellPrepBufs cb, int kch, int64_t bound) {
    const uint32_t nd = *cb.ndense;
    for (int64_t dc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; dc < bound; dc += (int64_t)gridDim.x * blockDim.x) {
        if (dc >= nd) {
            cb.nitem_c[dc] = 0u;
            continue;
        }
        const uint32_t c = cb.dense[dc];
        const uint32_t m = v.cell_start[c + 1] - v.cell_start[c];
        const uint32_t cand = cb.cand[c];
        const uint32_t qch = (uint32_t)cb.qch;
        const uint32_t nq = (m + qch - 1) / qch, nk = cand == 0u ? 1u : (cand + kch - 1) / kch;
        cb.nitem_c[dc] = nq * nk;
    }
}

// Work items of every dense cell: (query chunk) x (candidate chunk).
__global__ void k_fill_items(BatchView v, CellPrepBufs cb, int kch) {
    const uint32_t nd = *cb.ndense;
    for (int64_t dc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; dc < nd; dc += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = cb.dense[dc];
        const uint32_t m = v.cell_start[c + 1] - v.cell_start[c];
        const uint32_t nq = (m + (uint32_t)cb.qch - 1) / (uint32_t)cb.qch;
        const uint32_t cand = cb.cand[c];
        const uint32_t nk = cand == 0u ? 1u : (cand + kch - 1) / kch;
        uint4* out = cb.items + cb.item_off[dc];
        for (uint32_t q = 0; q < nq; ++q)
            for (uint32_t k = 0; k < nk; ++k) out[q * nk + k] = make_uint4((uint32_t)dc, q, k, 0u);
    }
}

template <int D>
__device__ __forceinline__ void load_point(const int4* r, int32_t (&x)[D]) {
    const int4 a = r[0];
    int32_t t[8] = {a.x, a.y, a.z, a.w, 0, 0, 0, 0};
    if (D > 4) {
        const int4 bq = r[1];
        t[4] = bq.x; t[5] = bq.y; t[6] = bq.z; t[7] = bq.w;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = t[k];
}

template <int D, bool W64>
__device__ __forceinline__ uint32_t inside(const int32_t (&q)[D], const int32_t (&c)[D], int64_t T) {
    if (W64) {
        long long s = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int dd = q[k] - c[k];
            s += (long long)dd * dd;
        }
        return s < T ? 1u : 0u;
    } else {
        int s = -(int)T;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int dd = q[k] - c[k];
            s += dd * dd;
        }
        return (uint32_t)s >> 31;
    }
}

// Q queries per lane against staged candidates grp, grp + G, ... (direct
// test: sum of squared differences against d_cut^2).
template <int D, bool W64, int Q>
__device__ __forceinline__ void eval_rho(const int4* buf, int nb, int grp, int G, const int32_t (&qx)[4][D],
                                         uint32_t (&cnt)[4], int64_t T) {
    constexpr int DP = D <= 4 ? 1 : 2;
#pragma unroll 4
    for (int j = grp; j < nb; j += G) {
        int32_t c[D];
        load_point<D>(buf + j * DP, c);
#pragma unroll
        for (int t = 0; t < Q; ++t) cnt[t] += inside<D, W64>(qx[t], c, T);
    }
}

// Expanded test (d <= 3). A record is (c_0, c_1, c_2, |c|^2 mod 2^32) and a
// query keeps a_k = -2 q_k and b = |q|^2 - d_cut^2 (mod 2^32), so that
//   |q - c|^2 - d_cut^2 = |c|^2 + b + sum_k c_k a_k   (mod 2^32):
// one add and d multiply-adds in wrapping 32-bit arithmetic. Candidates come
// from the 3^k cells around the query's, so |q - c|^2 < 4 d s^2 <= 2^31 (the
// form is chosen only when 9 d s^2 < 2^31): the true value lies in
// [-2^31, 2^31), and the sign bit of the wrapped sum is the pair test.
// In 4 dims the record's spare lane is taken: |c|^2 is computed when the
// candidate is staged and kept beside it (nrm).
template <int D, int Q>
__device__ __forceinline__ void eval_rho_x(const int4* buf, const uint32_t* nrm, int nb, int grp, int G,
                                           const uint32_t (&qa)[4][4], const uint32_t (&qb)[4], uint32_t (&cnt)[4]) {
#pragma unroll 4
    for (int j = grp; j < nb; j += G) {
        const int4 c = buf[j];
        const uint32_t cn = D == 4 ? nrm[j] : (uint32_t)c.w;
#pragma unroll
        for (int t = 0; t < Q; ++t) {
            uint32_t s = cn + qb[t];
            s += (uint32_t)c.x * qa[t][0];
            if (D > 1) s += (uint32_t)c.y * qa[t][1];
            if (D > 2) s += (uint32_t)c.z * qa[t][2];
            if (D > 3) s += (uint32_t)c.w * qa[t][3];
            cnt[t] += s >> 31;
        }
    }
}

// The expanded form's query terms: a_k = -2 q_k, b = |q|^2 - T (mod 2^32).
template <int D>
__device__ __forceinline__ void expand_query(const int32_t (&q)[D], uint32_t T, uint32_t (&a)[4], uint32_t& b) {
    uint32_t n = 0u - T;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t x = k < D ? (uint32_t)q[k < D ? k : 0] : 0u;
        a[k] = 0u - 2u * x;
        n += x * x;
    }
    b = n;
}

// |c|^2 mod 2^32 of a 4-d record (the expanded form's candidate norm).
__device__ __forceinline__ uint32_t norm4(const int4 r) {
    return (uint32_t)r.x * (uint32_t)r.x + (uint32_t)r.y * (uint32_t)r.y + (uint32_t)r.z * (uint32_t)r.z +
           (uint32_t)r.w * (uint32_t)r.w;
}


// QL: the queries of a cell are the points qlist[qstart[c] .. qstart[c + 1])
// (S-Approx-DPC's picks, all of them points of cell c) and an item's first
// field is the cell itself; otherwise the queries are all the cell's points
// and the first field indexes the dense cell list.
template <int D, int MODE, bool QL>
__global__ void __launch_bounds__(kRhoThreads) k_rho_dense(BatchView v, CellWork w, uint32_t* counter,
                                                           const uint32_t* __restrict__ qlist,
                                                           const uint32_t* __restrict__ qstart) {
    constexpr int DP = D <= 4 ? 1 : 2;
    constexpr bool W64 = MODE == 1;
    constexpr bool EXP = MODE == 2;
    __shared__ int4 sbuf[kRhoThreads / 32][2][kChunk * DP];  // double buffer per warp
    __shared__ uint32_t snrm[kRhoThreads / 32][2][EXP && D == 4 ? kChunk : 1];  // 4-d expanded form: |c|^2
    __shared__ uint2 sruns[kRhoThreads / 32][kMaxNb];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint2* srun = sruns[wid];
    const uint32_t nitems = *w.nitems;
    // the next item's index, record and cell are fetched in stages while the
    // current item runs (one stage per candidate chunk)
    uint32_t nx = 0, it_n = 0, c_n = 0, cs_n = 0, ce_n = 0, nr_n = 0, ct_n = 0, qs_n = 0, qe_n = 0;
    uint4 item_n = make_uint4(0u, 0u, 0u, 0u);
    auto stage = [&](int s) {
        if (s == 0) {
            it_n = __shfl_sync(0xffffffffu, nx, 0);
            if (it_n < nitems) item_n = w.items[it_n];
        } else if (s == 1) {
            if (it_n < nitems) c_n = QL ? item_n.x : w.dense[item_n.x];
        } else if (s == 2) {
            if (it_n < nitems) {
                cs_n = v.cell_start[c_n];
                ce_n = v.cell_start[c_n + 1];
                nr_n = w.nruns[c_n];
                ct_n = w.cand[c_n];
                if (QL) {
                    qs_n = qstart[c_n];
                    qe_n = qstart[c_n + 1];
                }
            }
        }
    };
    if (lane == 0) nx = atomicAdd(counter, 1u);
    stage(0);
    stage(1);
    stage(2);
    while (true) {
        const uint32_t it = it_n;
        if (it >= nitems) break;
        const uint4 item = item_n;  // (dense cell, query chunk, candidate chunk)
        const uint32_t qc = item.y, kc = item.z;
        const uint32_t c = c_n;
        const uint32_t cs = cs_n, m = QL ? qe_n - qs_n : ce_n - cs_n, qs = qs_n;
        const uint32_t nr_c = nr_n, ctot_c = ct_n;
        if (lane == 0) nx = atomicAdd(counter, 1u);
        int pf = 0;
        const int b = find_ds(v.pt_off, v.B, cs);
        const DsDesc& ds = v.desc[b];
        if (ds.d != D || ds.mode != MODE) {
            for (; pf < 3; ++pf) stage(pf);
            continue;
        }
        const int4* recb = v.rec + ds.rec_off - ds.pt_off * DP;  // indexed by global sorted position
        const int q0 = (int)qc * w.qch;
        const int nq = min(w.qch, (int)m - q0);
        int Q, Mq;
        lane_layout(nq, Q, Mq);
        const int G = 32 / Mq;
        const int grp = lane / Mq, ql = lane & (Mq - 1);
        // query t of this lane: ql * Q + t (slots at or past nq are dummies),
        // the point at sorted position cs + q0 + ql * Q + t (QL: qpos[t])
        uint32_t qpos[4];
        int32_t qx[4][D];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint32_t i = (uint32_t)(q0 + min(ql * Q + t, nq - 1));
            if (QL) qpos[t] = qlist[qs + i];
            load_point<D>(recb + (int64_t)(QL ? qpos[t] : cs + i) * DP, qx[t]);
        }
        // expanded form: the queries' terms (the records carry |c|^2)
        uint32_t qa[4][4], qb[4];
        if (EXP) {
#pragma unroll
            for (int t = 0; t < 4; ++t) expand_query<D>(qx[t], (uint32_t)ds.d_cut2, qa[t], qb[t]);
        }
        uint32_t cnt[4] = {0u, 0u, 0u, 0u};
        // the cell's runs into shared memory, then the candidate stream
        const uint32_t nr = nr_c, ctot = ctot_c;
        // the runs in shared memory when they fit (reach 1), else read in place
        const uint2* runs_c = w.runs + (int64_t)c * w.nbs;
        if (nr <= (uint32_t)kMaxNb) {
            for (uint32_t t = lane; t < nr; t += 32) srun[t] = runs_c[t];
            runs_c = srun;
        }
        __syncwarp();
        const uint32_t k0 = kc * (uint32_t)w.kch;
        CandStream<DP, false> cst;
        cst.init(runs_c, nr, k0, min(ctot, k0 + (uint32_t)w.kch));
        bool bad = false;
        bool have = cst.prep(lane, recb, nullptr, &bad);
        const int64_t T = ds.d_cut2;
        int sb = 0;
        while (have) {
            // store the loaded chunk (relative to the cell corner in the
            // expanded form), then put the next chunk's loads in flight
            int4* buf = sbuf[wid][sb];
            uint32_t* nbuf = snrm[wid][EXP && D == 4 ? sb : 0];
            const int nb = (int)cst.cnt;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int f = lane + 32 * u;
                if (f < nb) {
#pragma unroll
                    for (int q = 0; q < DP; ++q) buf[f * DP + q] = cst.r[u][q];
                    if (EXP && D == 4) nbuf[f] = norm4(cst.r[u][0]);
                }
            }
            __syncwarp();
            have = cst.prep(lane, recb, nullptr, &bad);
            sb ^= 1;
            if (pf < 3) stage(pf++);
            if (EXP) {
                switch (Q) {
                    case 1: eval_rho_x<D, 1>(buf, nbuf, nb, grp, G, qa, qb, cnt); break;
                    case 2: eval_rho_x<D, 2>(buf, nbuf, nb, grp, G, qa, qb, cnt); break;
                    case 3: eval_rho_x<D, 3>(buf, nbuf, nb, grp, G, qa, qb, cnt); break;
                    default: eval_rho_x<D, 4>(buf, nbuf, nb, grp, G, qa, qb, cnt); break;
                }
            } else {
                switch (Q) {
                    case 1: eval_rho<D, W64, 1>(buf, nb, grp, G, qx, cnt, T); break;
                    case 2: eval_rho<D, W64, 2>(buf, nb, grp, G, qx, cnt, T); break;
                    case 3: eval_rho<D, W64, 3>(buf, nb, grp, G, qx, cnt, T); break;
                    default: eval_rho<D, W64, 4>(buf, nb, grp, G, qx, cnt, T); break;
                }
            }
        }
        for (; pf < 3; ++pf) stage(pf);
        if (bad && lane == 0) atomicOr(v.err, kErrStaging);
        __syncwarp();
        // add the groups' counts, then one lane per query writes
#pragma unroll
        for (int t = 0; t < 4; ++t)
            for (int o = Mq; o < 32; o <<= 1) cnt[t] += __shfl_xor_sync(0xffffffffu, cnt[t], o);
        if (grp == 0) {
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (t < Q && ql * Q + t < nq)
                    atomicAdd(&v.rho_s[QL ? qpos[t] : cs + q0 + ql * Q + t], (int)cnt[t]);
        }
    }
}

// ------------------------------------------------ bulk-copy staging
//
// The same dense pass with its candidates staged by the copy engine: a warp
// walks its runs for the next chunk of up to kChunk records, and every run
// piece (a contiguous range of records, 16 bytes each) goes to shared memory
// as one cp.async.bulk, completed on the chunk buffer's mbarrier by byte
// count (lane 0 announces the chunk's bytes before any piece is issued).
// The copy of chunk i + 1 is in flight while chunk i is evaluated. Waits are
// bounded: a buffer whose bytes do not arrive in time raises kErrBulkWait
// and the warp stops after a bounded wait for its other buffer. Records of
// one int4 only (d <= 4), direct 32-bit (mode 0) or expanded (mode 2) form.

constexpr int kBulkSpin = 1 << 22;                 // try_wait rounds before a wait gives up
constexpr unsigned long long kBulkWaitNs = 1000000000ull;  // or this much wall time (1 s)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One test of the phase of the given parity; a thread left waiting is
// suspended for at most about 1 us.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0u;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase of the given parity: kBulkSpin tests or
// kBulkWaitNs of wall time, whichever ends first.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (int i = 0; i < kBulkSpin; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && global_ns() - t0 > kBulkWaitNs) return false;
    }
    return false;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Orders this thread's earlier generic accesses to shared memory before
// later copy-engine writes to it.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Run walk of one item's candidate range, as CandStream's (warp-uniform).
struct BulkWalk {
    const uint2* runs;
    uint32_t nr, ri, roff, remaining;

    __device__ __forceinline__ void init(const uint2* runs_, uint32_t nr_, uint32_t k0, uint32_t k1) {
        runs = runs_;
        nr = nr_;
        ri = 0;
        roff = k0;
        remaining = k1 - k0;
        while (ri < nr) {
            const uint32_t len = runs[ri].y;
            if (roff < len) break;
            roff -= len;
            ++ri;
        }
    }

    // Announces and issues the copies of the next chunk into buf (bar its
    // mbarrier); returns the records staged (0 when the range is done).
    // Piece t of the chunk is issued by lane t % 32.
    __device__ __forceinline__ uint32_t issue(int lane, const int4* __restrict__ recb, int4* buf, uint64_t* bar,
                                              bool* bad) {
        if (remaining == 0u) return 0u;
        const uint32_t total = min((uint32_t)kChunk, remaining);
        // this lane's pieces (at most 4: a chunk has at most kChunk pieces)
        uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0, d0 = 0, d1 = 0, d2 = 0, d3 = 0, l0 = 0, l1 = 0, l2 = 0, l3 = 0;
        uint32_t o = 0, t = 0;
        while (o < total) {
            if (ri >= nr) {
                *bad = true;
                break;
            }
            const uint2 run = runs[ri];
            const uint32_t piece = min(run.y - roff, total - o);
            if ((t & 31u) == (uint32_t)lane) {
                const uint32_t sx = run.x + roff, u = t >> 5;
                if (u == 0u) { s0 = sx; d0 = o; l0 = piece; }
                else if (u == 1u) { s1 = sx; d1 = o; l1 = piece; }
                else if (u == 2u) { s2 = sx; d2 = o; l2 = piece; }
                else { s3 = sx; d3 = o; l3 = piece; }
            }
            ++t;
            o += piece;
            roff += piece;
            if (roff == run.y) {
                ++ri;
                roff = 0;
            }
        }
        remaining -= total;
        if (o == 0u) return 0u;
        if (lane == 0) mbar_arrive_expect(bar, o * (uint32_t)sizeof(int4));
        __syncwarp();
        if (l0) bulk_copy_g2s(buf + d0, recb + s0, l0 * (uint32_t)sizeof(int4), bar);
        if (l1) bulk_copy_g2s(buf + d1, recb + s1, l1 * (uint32_t)sizeof(int4), bar);
        if (l2) bulk_copy_g2s(buf + d2, recb + s2, l2 * (uint32_t)sizeof(int4), bar);
        if (l3) bulk_copy_g2s(buf + d3, recb + s3, l3 * (uint32_t)sizeof(int4), bar);
        return o;
    }
};

template <int D, int MODE>
__global__ void __launch_bounds__(kRhoThreads) k_rho_dense_bulk(BatchView v, CellWork w, uint32_t* counter) {
    static_assert(D <= 4 && (MODE == 0 || (MODE == 2 && D <= 3)), "one int4 per record, 32-bit forms");
    constexpr bool EXP = MODE == 2;
    __shared__ __align__(128) int4 sbuf[kRhoThreads / 32][2][kChunk];  // double buffer per warp
    __shared__ uint2 sruns[kRhoThreads / 32][kMaxNb];
    __shared__ __align__(8) uint64_t sbar[kRhoThreads / 32][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint2* srun = sruns[wid];
    uint64_t* bar = sbar[wid];
    if (lane == 0) {
        mbar_init(&bar[0], 1u);
        mbar_init(&bar[1], 1u);
    }
    fence_proxy_async();
    __syncwarp();
    uint32_t par = 0u;  // bit b: parity of buffer b's next phase
    const uint32_t nitems = *w.nitems;
    uint32_t nx = 0, it_n = 0, c_n = 0, cs_n = 0, ce_n = 0, nr_n = 0, ct_n = 0;
    uint4 item_n = make_uint4(0u, 0u, 0u, 0u);
    auto stage = [&](int s) {
        if (s == 0) {
            it_n = __shfl_sync(0xffffffffu, nx, 0);
            if (it_n < nitems) item_n = w.items[it_n];
        } else if (s == 1) {
            if (it_n < nitems) c_n = w.dense[item_n.x];
        } else if (s == 2) {
            if (it_n < nitems) {
                cs_n = v.cell_start[c_n];
                ce_n = v.cell_start[c_n + 1];
                nr_n = w.nruns[c_n];
                ct_n = w.cand[c_n];
            }
        }
    };
    if (lane == 0) nx = atomicAdd(counter, 1u);
    stage(0);
    stage(1);
    stage(2);
    bool stop = false;
    while (!stop) {
        const uint32_t it = it_n;
        if (it >= nitems) break;
        const uint4 item = item_n;  // (dense cell, query chunk, candidate chunk)
        const uint32_t qc = item.y, kc = item.z;
        const uint32_t c = c_n;
        const uint32_t cs = cs_n, m = ce_n - cs_n;
        const uint32_t nr_c = nr_n, ctot_c = ct_n;
        if (lane == 0) nx = atomicAdd(counter, 1u);
        int pf = 0;
        const int b = find_ds(v.pt_off, v.B, cs);
        const DsDesc& ds = v.desc[b];
        if (ds.d != D || ds.mode != MODE) {
            for (; pf < 3; ++pf) stage(pf);
            continue;
        }
        const int4* recb = v.rec + ds.rec_off - ds.pt_off;  // indexed by global sorted position
        const int q0 = (int)qc * w.qch;
        const int nq = min(w.qch, (int)m - q0);
        int Q, Mq;
        lane_layout(nq, Q, Mq);
        const int G = 32 / Mq;
        const int grp = lane / Mq, ql = lane & (Mq - 1);
        int32_t qx[4][D];
#pragma unroll
        for (int t = 0; t < 4; ++t) load_point<D>(recb + ((int64_t)cs + q0 + min(ql * Q + t, nq - 1)), qx[t]);
        uint32_t qa[4][4], qb[4];
        if (EXP) {
#pragma unroll
            for (int t = 0; t < 4; ++t) expand_query<D>(qx[t], (uint32_t)ds.d_cut2, qa[t], qb[t]);
        }
        uint32_t cnt[4] = {0u, 0u, 0u, 0u};
        const uint32_t nr = nr_c, ctot = ctot_c;
        const uint2* runs_c = w.runs + (int64_t)c * w.nbs;
        if (nr <= (uint32_t)kMaxNb) {
            for (uint32_t t = lane; t < nr; t += 32) srun[t] = runs_c[t];
            runs_c = srun;
        }
        __syncwarp();
        const uint32_t k0 = kc * (uint32_t)w.kch;
        BulkWalk walk;
        walk.init(runs_c, nr, k0, min(ctot, k0 + (uint32_t)w.kch));
        bool bad = false;
        const int64_t T = ds.d_cut2;
        int sb = 0;
        uint32_t cur = walk.issue(lane, recb, sbuf[wid][sb], &bar[sb], &bad);
        while (cur > 0u) {
            // the next chunk's copies go out before this chunk is used
            const uint32_t nxt = walk.issue(lane, recb, sbuf[wid][sb ^ 1], &bar[sb ^ 1], &bad);
            const bool ok = mbar_wait(&bar[sb], (par >> sb) & 1u);
            par ^= 1u << sb;
            if (!ok) {
                if (lane == 0) atomicOr(v.err, kErrBulkWait);
                if (nxt > 0u) mbar_wait(&bar[sb ^ 1], (par >> (sb ^ 1)) & 1u);
                stop = true;
                break;
            }
            int4* buf = sbuf[wid][sb];
            const uint32_t* nbuf = nullptr;  // the norm is the record's w lane (d <= 3)
            const int nb = (int)cur;
            if (pf < 3) stage(pf++);
            if (EXP) {
                switch (Q) {
                    case 1: eval_rho_x<D, 1>(buf, nbuf, nb, grp, G, qa, qb, cnt); break;
                    case 2: eval_rho_x<D, 2>(buf, nbuf, nb, grp, G, qa, qb, cnt); break;
                    case 3: eval_rho_x<D, 3>(buf, nbuf, nb, grp, G, qa, qb, cnt); break;
                    default: eval_rho_x<D, 4>(buf, nbuf, nb, grp, G, qa, qb, cnt); break;
                }
            } else {
                switch (Q) {
                    case 1: eval_rho<D, false, 1>(buf, nb, grp, G, qx, cnt, T); break;
                    case 2: eval_rho<D, false, 2>(buf, nb, grp, G, qx, cnt, T); break;
                    case 3: eval_rho<D, false, 3>(buf, nb, grp, G, qx, cnt, T); break;
                    default: eval_rho<D, false, 4>(buf, nb, grp, G, qx, cnt, T); break;
                }
            }
            // every lane is done with this buffer before copies refill it
            fence_proxy_async();
            __syncwarp();
            sb ^= 1;
            cur = nxt;
        }
        if (stop) break;
        for (; pf < 3; ++pf) stage(pf);
        if (bad && lane == 0) atomicOr(v.err, kErrStaging);
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 4; ++t)
            for (int o = Mq; o < 32; o <<= 1) cnt[t] += __shfl_xor_sync(0xffffffffu, cnt[t], o);
        if (grp == 0) {
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (t < Q && ql * Q + t < nq) atomicAdd(&v.rho_s[cs + q0 + ql * Q + t], (int)cnt[t]);
        }
    }
}

// Sparse cells (at most kSparseMax points, few candidates): kSparseLanes
// lanes per cell, each with all of the cell's queries, take every
// kSparseLanes-th candidate of the cell's concatenated runs; their counts
// are added with warp shuffles. (One thread per cell left most lanes of a
// warp idle: cells in a warp have very different candidate counts.) A lane
// finds its next kSparseBatch candidates first and then loads their records
// together, so that their latencies overlap (the runs hold 2-3 points each
// in sparse regions: a loop per run kept one load in flight). The loop over
// cells is warp-uniform, so that every lane reaches the shuffles.
constexpr int kSparseLanes = 2;
constexpr int kSparseBatch = 4;
// (5 blocks of 256 threads per SM: density 1.74 -> 1.70 ms at 5.8M x 3; the
// ring search's sparse kernel spills under the same bound and ran slower)

template <int D, bool W64>
__global__ void __launch_bounds__(256, 5) k_rho_sparse(BatchView v, CellWork w) {
    constexpr int DP = D <= 4 ? 1 : 2;
    constexpr int G = kSparseLanes, CPW = 32 / G;  // lanes per cell, cells per warp
    const uint32_t ns = *w.nsparse;
    const int lane = threadIdx.x & 31, sl = lane & (G - 1), grp = lane / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * CPW; base < ns; base += nwarps * CPW) {
        const int64_t i = base + grp;
        uint32_t cnt[kSparseMax] = {0u, 0u, 0u, 0u};
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
#pragma unroll
                for (int t = 0; t < kSparseMax; ++t)
                    load_point<D>(recb + ((int64_t)cs + min((uint32_t)t, m - 1)) * DP, qx[t]);
                const int64_t T = ds.d_cut2;
                RunCursor rc;
                rc.init(w.runs + (int64_t)c * w.nbs, w.nruns[c], (uint32_t)sl);
                bool more = true;
                while (more) {
                    // positions first (a lane past its last candidate reads
                    // the cell's own first record and counts nothing)
                    uint32_t p[kSparseBatch];
                    bool ok[kSparseBatch];
#pragma unroll
                    for (int u = 0; u < kSparseBatch; ++u) {
                        ok[u] = rc.next((uint32_t)G, p[u]);
                        if (!ok[u]) p[u] = cs;
                    }
                    more = ok[kSparseBatch - 1];
                    int32_t cj[kSparseBatch][D];
#pragma unroll
                    for (int u = 0; u < kSparseBatch; ++u) load_point<D>(recb + (int64_t)p[u] * DP, cj[u]);
#pragma unroll
                    for (int u = 0; u < kSparseBatch; ++u)
#pragma unroll
                        for (int q = 0; q < kSparseMax; ++q)
                            cnt[q] += ok[u] ? inside<D, W64>(qx[q], cj[u], T) : 0u;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kSparseMax; ++q)
#pragma unroll
            for (int o = 1; o < G; o <<= 1) cnt[q] += __shfl_xor_sync(0xffffffffu, cnt[q], o);
        if (mine && sl == 0) {
#pragma unroll
            for (int q = 0; q < kSparseMax; ++q)
                if ((uint32_t)q < m) v.rho_s[cs + q] = (int32_t)cnt[q];
        }
    }
}
__global__ void k_rho_scatter(BatchView v) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < v.N) v.rho[v.perm[p]] = v.rho_s[p];
}

template <int D, int MODE, bool QL = false>
void launch_rho_dense(const BatchView& v, const CellWork& w, int64_t nitems_bound, uint32_t* counter,
                      cudaStream_t st, const uint32_t* qlist = nullptr, const uint32_t* qstart = nullptr) {
    if (nitems_bound <= 0) return;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(152 * 16, (nitems_bound + 3) / 4));
    (k_rho_dense<D, MODE, QL><<<blocks, kRhoThreads, 0, st>>>(v, w, counter, qlist, qstart), note_launch());
}

template <int D, int MODE>
void launch_rho_dense_bulk(const BatchView& v, const CellWork& w, int64_t nitems_bound, uint32_t* counter,
                           cudaStream_t st) {
    if (nitems_bound <= 0) return;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(152 * 16, (nitems_bound + 3) / 4));
    (k_rho_dense_bulk<D, MODE><<<blocks, kRhoThreads, 0, st>>>(v, w, counter), note_launch());
}

template <int D, bool W64>
void launch_rho_sparse(const BatchView& v, const CellWork& w, int64_t nsparse_bound, cudaStream_t st) {
    if (nsparse_bound <= 0) return;
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 32, grid_for(nsparse_bound * kSparseLanes, 256));
    (k_rho_sparse<D, W64><<<blocks, 256, 0, st>>>(v, w), note_launch());
}

}  // namespace

cudaError_t launch_cell_runs(const BatchView& v, const CellPrepBufs& cb, int64_t ncells, uint32_t kmask,
                            cudaStream_t st) {
    if (ncells <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(ncells, 256));
    if (kmask & 1u) (k_cell_runs_any<<<blocks, 256, 0, st>>>(v, cb, ncells), note_launch());
    if (kmask & 2u) (k_cell_runs<1><<<blocks, 256, 0, st>>>(v, cb, ncells), note_launch());
    if (kmask & 4u) (k_cell_runs<2><<<blocks, 256, 0, st>>>(v, cb, ncells), note_launch());
    if (kmask & 8u) (k_cell_runs<3><<<blocks, 256, 0, st>>>(v, cb, ncells), note_launch());
    if (kmask & 16u) (k_cell_runs<4><<<blocks, 256, 0, st>>>(v, cb, ncells), note_launch());
    const unsigned bblocks = (unsigned)std::min<int64_t>(152 * 32, grid_for(ncells, kRunsBlkThreads));
    if (kmask & (2u << 8)) (k_cell_runs_blk<1><<<bblocks, kRunsBlkThreads, 0, st>>>(v, cb, ncells), note_launch());
    if (kmask & (4u << 8)) (k_cell_runs_blk<2><<<bblocks, kRunsBlkThreads, 0, st>>>(v, cb, ncells), note_launch());
    if (kmask & (8u << 8)) (k_cell_runs_blk<3><<<bblocks, kRunsBlkThreads, 0, st>>>(v, cb, ncells), note_launch());
    if (kmask & (16u << 8)) (k_cell_runs_blk<4><<<bblocks, kRunsBlkThreads, 0, st>>>(v, cb, ncells), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_classify_cells(const BatchView& v, const CellPrepBufs& cb, int64_t ncells_bound,
                                  uint32_t sparse_cand, void* scan_temp, cudaStream_t st) {
    if (ncells_bound <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(ncells_bound, 256));
    (k_classify<<<blocks, 256, 0, st>>>(v, cb, ncells_bound, sparse_cand), note_launch());
    cudaError_t e = exclusive_scan_u32(cb.dflag, cb.didx, ncells_bound, cb.ndense, scan_temp, st);
    if (e != cudaSuccess) return e;
    e = exclusive_scan_u32(cb.sflag, cb.sidx, ncells_bound, cb.nsparse, scan_temp, st);
    if (e != cudaSuccess) return e;
    (k_compact_cells<<<blocks, 256, 0, st>>>(v, cb, ncells_bound), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_item_prep(const BatchView& v, const CellPrepBufs& cb, int64_t ndense_bound, int kch,
                             void* scan_temp, cudaStream_t st) {
    if (ndense_bound <= 0) return cudaMemsetAsync(cb.nitems, 0, sizeof(uint32_t), st);
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(ndense_bound, 256));
    (k_item_count<<<blocks, 256, 0, st>>>(v, cb, kch, ndense_bound), note_launch());
    return exclusive_scan_u32(cb.nitem_c, cb.item_off, ndense_bound, cb.nitems, scan_temp, st);
}

cudaError_t launch_fill_items(const BatchView& v, const CellPrepBufs& cb, int64_t ndense_bound, int kch,
                              cudaStream_t st) {
    if (ndense_bound <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(ndense_bound, 256));
    (k_fill_items<<<blocks, 256, 0, st>>>(v, cb, kch), note_launch());
    return cudaGetLastError();
}

// The dense kernel of class (D, M): with bulk, the copy-engine staging where
// it exists (one int4 per record, a 32-bit form).
template <int D, int M>
void launch_dense_class(const BatchView& v, const CellWork& w, int64_t nitems_bound, uint32_t* counter, bool bulk,
                        cudaStream_t st) {
    if constexpr (D <= 4 && M != 1 && !(M == 2 && D == 4)) {
        if (bulk) {
            launch_rho_dense_bulk<D, M>(v, w, nitems_bound, counter, st);
            return;
        }
    }
    launch_rho_dense<D, M>(v, w, nitems_bound, counter, st);
}

cudaError_t launch_rho(const BatchView& v, const CellWork& w, uint32_t class_mask, int64_t nitems_bound,
                       int64_t nsparse_bound, uint32_t* counters, int parts, cudaStream_t st) {
    // one dense launch per (dimension, arithmetic mode) class present in the
    // batch and one sparse launch per (dimension, width); each kernel skips
    // the work of the other classes. parts: bit 0 dense kernels, bit 1
    // sparse, bit 2 bulk-copy staging in the dense kernels that have it
    const bool bulk = (parts & 4) != 0;
#define DPC_BIT(D, M) (class_mask & (1u << (3 * ((D) - 1) + (M))))
#define DPC_RHO_CLASS(D)                                                                                  \
    if ((parts & 1) && DPC_BIT(D, 0))                                                                     \
        launch_dense_class<D, 0>(v, w, nitems_bound, counters + 3 * (D - 1), bulk, st);                  \
    if ((parts & 1) && DPC_BIT(D, 1))                                                                     \
        launch_dense_class<D, 1>(v, w, nitems_bound, counters + 3 * (D - 1) + 1, bulk, st);              \
    if ((parts & 2) && (DPC_BIT(D, 0) || DPC_BIT(D, 2))) launch_rho_sparse<D, false>(v, w, nsparse_bound, st); \
    if ((parts & 2) && DPC_BIT(D, 1)) launch_rho_sparse<D, true>(v, w, nsparse_bound, st);
#define DPC_RHO_X(D) \
    if ((parts & 1) && DPC_BIT(D, 2)) launch_dense_class<D, 2>(v, w, nitems_bound, counters + 3 * (D - 1) + 2, bulk, st);
    DPC_RHO_CLASS(1) DPC_RHO_CLASS(2) DPC_RHO_CLASS(3) DPC_RHO_CLASS(4)
    DPC_RHO_CLASS(5) DPC_RHO_CLASS(6) DPC_RHO_CLASS(7) DPC_RHO_CLASS(8)
    DPC_RHO_X(1) DPC_RHO_X(2) DPC_RHO_X(3) DPC_RHO_X(4)
#undef DPC_RHO_X
#undef DPC_RHO_CLASS
#undef DPC_BIT
    return cudaGetLastError();
}

cudaError_t launch_rho_picks(const BatchView& v, const CellWork& w, uint32_t class_mask, int64_t nitems_bound,
                             uint32_t* counters, const uint32_t* plist, const uint32_t* pstart, cudaStream_t st) {
    // the dense kernels of every (dimension, arithmetic mode) class present,
    // over the items of the cells' picks
#define DPC_BIT(D, M) (class_mask & (1u << (3 * ((D) - 1) + (M))))
#define DPC_RHOP(D, M) \
    if (DPC_BIT(D, M)) launch_rho_dense<D, M, true>(v, w, nitems_bound, counters + 3 * (D - 1) + M, st, plist, pstart);
#define DPC_RHOP_CLASS(D) DPC_RHOP(D, 0) DPC_RHOP(D, 1)
    DPC_RHOP_CLASS(1) DPC_RHOP_CLASS(2) DPC_RHOP_CLASS(3) DPC_RHOP_CLASS(4)
    DPC_RHOP_CLASS(5) DPC_RHOP_CLASS(6) DPC_RHOP_CLASS(7) DPC_RHOP_CLASS(8)
    DPC_RHOP(1, 2) DPC_RHOP(2, 2) DPC_RHOP(3, 2) DPC_RHOP(4, 2)
#undef DPC_RHOP_CLASS
#undef DPC_RHOP
#undef DPC_BIT
    return cudaGetLastError();
}

cudaError_t launch_rho_scatter(const BatchView& v, cudaStream_t st) {
    if (v.N == 0) return cudaSuccess;
    (k_rho_scatter<<<grid_for(v.N, 256), 256, 0, st>>>(v), note_launch());
    return cudaGetLastError();
}

}  // namespace dpc
