// Noise, cluster centers and cluster labels (Definitions 4-6).
//
// noise_i  <=> rho_i < rho_min;
// center_i <=> not noise and delta_i >= delta_min (tested as
//              delta2_i >= delta_min^2; the densest point has delta2 =
//              INT64_MAX, so it is a center whenever it is not noise);
// a center is its own parent, noise has none, every other point hangs on its
// dependent point. On S-Approx-DPC's datasets (Section 5) these rules apply
// to the picked points; every other point hangs on its pick. The paper propagates labels depth-first from the centers
// (Section 2.2, step 4); the same forest is labelled here by pointer jumping:
// every thread follows its parent chain to the root and stores the progress
// back into its own parent slot, so chains through it shrink for the other
// threads. Every value ever stored is an ancestor of the slot's point, so the
// roots found are exact, whatever the interleaving.
#include "stages.cuh"
#include <algorithm>

namespace dpc {

namespace {

// Points [g0, g1) of the batch (all of them, or one dataset's).
__global__ void k_parent(BatchView v, int64_t g0, int64_t g1) {
    const int64_t g = g0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = g < g1;
    int b = -1;
    bool center = false;
    if (valid) {
        b = find_ds(v.pt_off, v.B, g);
        const DsDesc& ds = v.desc[b];
        if (v.pick && !v.pick[g]) {
            // S-Approx-DPC: a point that is not picked takes its pick's label
            // (none when the pick is noise)
            const int64_t k = ds.pt_off + v.dep[g];
            v.parent[g] = (int64_t)v.rho[k] < ds.rho_min ? -1 : (int32_t)k;
        } else {
            const bool noise = (int64_t)v.rho[g] < ds.rho_min;
            center = !noise && v.delta2[g] >= ds.delta_min2;
            v.parent[g] = noise ? -1 : (center ? (int32_t)g : (int32_t)(ds.pt_off + v.dep[g]));
        }
    }
    // count centers per dataset, aggregated over the lanes of one dataset
    const unsigned same = __match_any_sync(0xffffffffu, b);
    const unsigned ctr = __ballot_sync(0xffffffffu, center) & same;
    const int lane = threadIdx.x & 31;
    if (valid && ctr != 0u && (same & ((1u << lane) - 1u)) == 0u)
        atomicAdd(&v.ncent[b], (unsigned long long)__popc(ctr));
}

__global__ void k_jump(BatchView v, int64_t g0, int64_t g1) {
    const int64_t g = g0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= g1) return;
    int32_t p = v.parent[g];
    if (p < 0) {
        v.label[g] = -1;
        return;
    }
    // a chain visits distinct points of one dataset, so it is shorter than N
    for (int64_t hop = 0;; ++hop) {
        const int32_t pp = __ldcg(&v.parent[p]);
        if (pp == p) break;
        if (hop > v.N || pp < 0) {
            atomicOr(v.err, kErrChain);
            break;
        }
        p = pp;
        __stcg(&v.parent[g], p);
    }
    const int b = find_ds(v.pt_off, v.B, g);
    v.label[g] = (int32_t)(p - v.pt_off[b]);
}

// Every device-resident job's outputs in one pass: thread t of the
// concatenation of the jobs' points (job j's at [dst_off_j, dst_off_j + n_j))
// copies its point's values from the batch's arrays to the job's buffers.
// what 0: rho, dep, delta2 and aux; 1: the labels of query q into
// label + q n (jobs with q queries or fewer are skipped).
__global__ void k_job_outputs(const OutJob* __restrict__ jobs, int J, int64_t total, const int32_t* __restrict__ rho,
                              const int32_t* __restrict__ dep, const int64_t* __restrict__ delta2,
                              const uint8_t* __restrict__ aux, const int32_t* __restrict__ label, int what, int q) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = J - 1;  // the last job with dst_off <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].dst_off <= t) lo = mid; else hi = mid - 1;
        }
        const OutJob& o = jobs[lo];
        const int64_t i = t - o.dst_off, g = o.src_off + i;
        if (what == 0) {
            if (o.rho) o.rho[i] = rho[g];
            if (o.dep) o.dep[i] = dep[g];
            if (o.delta2) o.delta2[i] = delta2[g];
            if (o.aux) o.aux[i] = aux[g];
        } else if (o.label && q < o.nq) {
            o.label[(int64_t)q * o.n + i] = label[g];
        }
    }
}

// The inputs of a batch's jobs whose points the device can read (device or
// page-locked host memory) into the batch's input buffer, one pass over its
// elements (job j's at [dst_off_j, dst_off_j + len_j); the others are left).
__global__ void k_job_inputs(const InJob* __restrict__ jobs, int J, int64_t total, int32_t* __restrict__ dst) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = J - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].dst_off <= t) lo = mid; else hi = mid - 1;
        }
        const int64_t i = t - jobs[lo].dst_off;
        if (i >= 0 && i < jobs[lo].len) dst[t] = jobs[lo].src[i];
    }
}

}  // namespace

cudaError_t launch_job_inputs(const InJob* jobs, int J, int64_t total, int32_t* dst, cudaStream_t st) {
    if (J <= 0 || total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(total, 256));
    (k_job_inputs<<<blocks, 256, 0, st>>>(jobs, J, total, dst), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_job_outputs(const OutJob* jobs, int J, int64_t total, const int32_t* rho, const int32_t* dep,
                               const int64_t* delta2, const uint8_t* aux, const int32_t* label, int what, int q,
                               cudaStream_t st) {
    if (J <= 0 || total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(152 * 16, grid_for(total, 256));
    (k_job_outputs<<<blocks, 256, 0, st>>>(jobs, J, total, rho, dep, delta2, aux, label, what, q), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_labels(const BatchView& v, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(v.ncent, 0, sizeof(unsigned long long) * v.B, st);
    if (e != cudaSuccess || v.N == 0) return e;
    (k_parent<<<grid_for(v.N, 256), 256, 0, st>>>(v, 0, v.N), note_launch());
    (k_jump<<<grid_for(v.N, 256), 256, 0, st>>>(v, 0, v.N), note_launch());
    return cudaGetLastError();
}

cudaError_t launch_labels_one(const BatchView& v, int b, int64_t g0, int64_t n, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(v.ncent + b, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || n == 0) return e;
    (k_parent<<<grid_for(n, 256), 256, 0, st>>>(v, g0, g0 + n), note_launch());
    (k_jump<<<grid_for(n, 256), 256, 0, st>>>(v, g0, g0 + n), note_launch());
    return cudaGetLastError();
}

}  // namespace dpc
