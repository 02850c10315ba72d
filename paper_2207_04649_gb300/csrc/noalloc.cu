// Labels without any device allocation.
//
// The labels step (noise, centers, pointer jumping to the center) needs one
// scratch array: the parent of every point. dpc_label takes it from the
// dataset's memory; dpc_label_static below takes it from a fixed array
// compiled into the library instead, for callers that cannot allocate device
// memory when they call: code that runs on a device budget reserved up
// front, or in a section that must not allocate (a callback, a real-time
// loop), or under a pool that fails once it is exhausted. The caller passes
// the inputs and the outputs; nothing is allocated or freed.
//
// The array holds at most kStaticMaxPoints parents (16 MiB) and lives on
// every GPU that loads the library until the process exits. All calls share
// it and it keeps the last call's contents, so calls that overlap on the GPU
// (different streams, or different host threads without ordering) race.
#include <mutex>

#include "dpc.h"
#include "dpc_internal.cuh"

namespace dpc {
namespace {

constexpr int64_t kStaticMaxPoints = 1ll << 22;

// The scratch. In host code these names are host-side stand-ins, not device
// addresses: the host takes their device addresses with
// cudaGetSymbolAddress (per device) and passes those to the kernels.
static __device__ __align__(256) int32_t g_parent[kStaticMaxPoints];
static __device__ __align__(256) unsigned long long g_centers;
static __device__ __align__(256) unsigned int g_err;  // nonzero: a dependent link was rejected

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t* g_parent_ptr[kMaxDevices] = {};
unsigned long long* g_centers_ptr[kMaxDevices] = {};
unsigned int* g_err_ptr[kMaxDevices] = {};

// A point that is neither noise nor a center hangs on its dependent point,
// which must lie in [0, n) and be strictly higher in the total order (rho
// desc, index asc): Definitions 2-3 give every point but the densest such a
// link, and links that all go strictly up a total order form a forest, so
// every chain ends at a root. A link that breaks this rule is not followed:
// the point's parent becomes kBadLink and the error word is set.
constexpr int32_t kBadLink = -2;

__global__ void k_parent_static(const int32_t* __restrict__ rho, const int32_t* __restrict__ dep,
                                const int64_t* __restrict__ delta2, int64_t n, int64_t rho_min, int64_t dmin2,
                                int32_t* __restrict__ parent, unsigned long long* __restrict__ centers,
                                unsigned int* __restrict__ err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool center = false;
    if (i < n) {
        const int32_t r = rho[i];
        const bool noise = (int64_t)r < rho_min;
        center = !noise && delta2[i] >= dmin2;
        int32_t p = noise ? -1 : (int32_t)i;
        if (!noise && !center) {
            const int32_t q = dep[i];
            // range first: rho[q] is read only for q inside the array
            const bool ok = q >= 0 && (int64_t)q < n && (rho[q] > r || (rho[q] == r && (int64_t)q < i));
            if (ok) {
                p = q;
            } else {
                p = kBadLink;
                atomicOr(err, 1u);
            }
        }
        parent[i] = p;
    }
    const unsigned m = __ballot_sync(0xffffffffu, center);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(centers, (unsigned long long)__popc(m));
}

// Every parent is -1, kBadLink, the point itself (a root) or a strictly
// higher point, so a chain has fewer than n hops; the bound is a guard only.
__global__ void k_jump_static(int64_t n, int32_t* __restrict__ parent, int32_t* __restrict__ label,
                              unsigned int* __restrict__ err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t p = parent[i];
    if (p < 0) {
        label[i] = p == kBadLink ? kBadLink : -1;
        return;
    }
    for (int64_t hop = 0;; ++hop) {
        const int32_t pp = __ldcg(&parent[p]);
        if (pp == p) break;
        if (pp < 0 || (int64_t)pp >= n || hop > n) {  // the chain runs into a rejected link
            p = kBadLink;
            atomicOr(err, 2u);
            break;
        }
        p = pp;
        __stcg(&parent[i], p);
    }
    label[i] = p;
}

// The center count, or -1 when a link was rejected.
__global__ void k_centers_out(const unsigned long long* centers, const unsigned int* err, int64_t* out) {
    *out = *err ? -1 : (int64_t)*centers;
}

}  // namespace
}  // namespace dpc

extern "C" dpc_status dpc_label_static(const int32_t* rho, const int32_t* dep, const int64_t* delta2, int64_t n,
                                       int64_t rho_min, int64_t delta_min, int32_t* label_out,
                                       int64_t* n_centers_out, void* cuda_stream) {
    using namespace dpc;
    if (n < 0 || n > kStaticMaxPoints) return DPC_ERR_INVALID_ARG;  // beyond the static scratch
    if (n > 0 && (!rho || !dep || !delta2 || !label_out)) return DPC_ERR_INVALID_ARG;
    if (delta_min < 1 || delta_min > 3037000499ll) return DPC_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DPC_ERR_CUDA;
    int32_t* parent = nullptr;
    unsigned long long* centers = nullptr;
    unsigned int* err = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_parent_ptr[dev]) {
            void* a = nullptr;
            void* b = nullptr;
            void* e = nullptr;
            if (cudaGetSymbolAddress(&a, g_parent) != cudaSuccess) return DPC_ERR_CUDA;
            if (cudaGetSymbolAddress(&b, g_centers) != cudaSuccess) return DPC_ERR_CUDA;
            if (cudaGetSymbolAddress(&e, g_err) != cudaSuccess) return DPC_ERR_CUDA;
            g_parent_ptr[dev] = static_cast<int32_t*>(a);
            g_centers_ptr[dev] = static_cast<unsigned long long*>(b);
            g_err_ptr[dev] = static_cast<unsigned int*>(e);
        }
        parent = g_parent_ptr[dev];
        centers = g_centers_ptr[dev];
        err = g_err_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // the counter and the error word keep the last call's values: clear them
    if (cudaMemsetAsync(centers, 0, sizeof(unsigned long long), st) != cudaSuccess) return DPC_ERR_CUDA;
    if (cudaMemsetAsync(err, 0, sizeof(unsigned int), st) != cudaSuccess) return DPC_ERR_CUDA;
    if (n > 0) {
        const unsigned blocks = (unsigned)((n + 255) / 256);
        (k_parent_static<<<blocks, 256, 0, st>>>(rho, dep, delta2, n, rho_min, delta_min * delta_min, parent,
                                                 centers, err), note_launch());
        (k_jump_static<<<blocks, 256, 0, st>>>(n, parent, label_out, err), note_launch());
    }
    if (n_centers_out) (k_centers_out<<<1, 1, 0, st>>>(centers, err, n_centers_out), note_launch());
    return cudaGetLastError() == cudaSuccess ? DPC_OK : DPC_ERR_CUDA;
}
