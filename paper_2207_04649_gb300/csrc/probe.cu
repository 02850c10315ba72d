// Throughput probe for the density stage's pair test.
//
// Every thread keeps 4 queries and 16 candidates in registers and applies the
// density kernel's pair test to all 64 pairs per sweep, on every SM, in one
// of the kernel's three forms:
//   direct   (mode 0): sign of sum_k (q_k - c_k)^2 - d_cut^2 in 32 bits;
//   direct   (mode 1): sum_k (q_k - c_k)^2 < d_cut^2 in 64 bits;
//   expanded (mode 2, d <= 4): sign of |c|^2 + (|q|^2 - d_cut^2) + sum_k c_k (-2 q_k)
//                              in wrapping 32-bit arithmetic (|c|^2 beside the record in 4 dims).
// After each sweep every query operand moves by an amount that depends on
// the counts, so no part of a pair test can be hoisted out of the loop (this
// costs d + 1 adds per query per 16 pairs, charged to the probe). The rate it
// reports is the integer-ALU ceiling of that instruction mix on this GPU at
// its current clock: the denominator of the density kernel's roofline.
#include "dpc.h"
#include "dpc_internal.cuh"

namespace dpc {
namespace {

template <int D, bool W64>
__global__ void __launch_bounds__(256) k_pair_probe(const int32_t* __restrict__ seed, int iters, int T,
                                                   unsigned long long* __restrict__ sink) {
    int32_t q[4][D], c[16][D];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) q[i][k] = seed[(t * 7 + i * D + k) & 1023];
#pragma unroll
    for (int j = 0; j < 16; ++j)
#pragma unroll
        for (int k = 0; k < D; ++k) c[j][k] = seed[(t * 13 + j * D + k + 512) & 1023];
    uint32_t cnt[4] = {0u, 0u, 0u, 0u};
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (W64) {
                    long long s = 0;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const int dd = q[i][k] - c[j][k];
                        s += (long long)dd * dd;
                    }
                    cnt[i] += s < (long long)T ? 1u : 0u;
                } else {
                    int s = -T;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const int dd = q[i][k] - c[j][k];
                        s += dd * dd;
                    }
                    cnt[i] += (uint32_t)s >> 31;
                }
            }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k) q[i][k] += (int)(cnt[i] & 1u);
    }
    if (cnt[0] + cnt[1] + cnt[2] + cnt[3] == 0xdeadbeefu) sink[0] = t;
}

template <int D>
__global__ void __launch_bounds__(256) k_pair_probe_x(const int32_t* __restrict__ seed, int iters, int T,
                                                     unsigned long long* __restrict__ sink) {
    uint32_t qa[4][4], qb[4];
    int4 c[16];
    uint32_t cn[16];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t n = 0u - (uint32_t)T;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t x = k < D ? (uint32_t)seed[(t * 7 + i * 4 + k) & 1023] : 0u;
            qa[i][k] = 0u - 2u * x;
            n += x * x;
        }
        qb[i] = n;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int32_t x = seed[(t * 13 + j * 4 + 512) & 1023];
        const int32_t y = D > 1 ? seed[(t * 13 + j * 4 + 513) & 1023] : 0;
        const int32_t z = D > 2 ? seed[(t * 13 + j * 4 + 514) & 1023] : 0;
        const int32_t u = D > 3 ? seed[(t * 13 + j * 4 + 515) & 1023] : 0;
        cn[j] = (uint32_t)(x * x + y * y + z * z + u * u);
        c[j] = make_int4(x, y, z, D > 3 ? u : (int32_t)cn[j]);
    }
    uint32_t cnt[4] = {0u, 0u, 0u, 0u};
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint32_t nj = D == 4 ? cn[j] : (uint32_t)c[j].w;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t s = nj + qb[i];
                s += (uint32_t)c[j].x * qa[i][0];
                if (D > 1) s += (uint32_t)c[j].y * qa[i][1];
                if (D > 2) s += (uint32_t)c[j].z * qa[i][2];
                if (D > 3) s += (uint32_t)c[j].w * qa[i][3];
                cnt[i] += s >> 31;
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t m = cnt[i] & 1u;
            qb[i] += m;
#pragma unroll
            for (int k = 0; k < D; ++k) qa[i][k] += m;
        }
    }
    if (cnt[0] + cnt[1] + cnt[2] + cnt[3] == 0xdeadbeefu) sink[0] = t;
}

// The dependent-point ring search's pair test in the expanded form: the
// density test's sum, then the candidate counts only when it ranks higher,
// and the packed key (squared distance << 32 | index) keeps the least. Each
// candidate carries (rank, index) beside its coordinates, as the ring
// kernel stages them; after each sweep the queries' operands and ranks move
// by amounts that depend on the keys kept.
template <int D>
__global__ void __launch_bounds__(256) k_ring_probe_x(const int32_t* __restrict__ seed, int iters,
                                                     unsigned long long* __restrict__ sink) {
    uint32_t qa[4][4], qn[4];
    uint32_t qr[4];
    int4 c[16];
    uint32_t cn[16];
    uint2 ro[16];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t n = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t x = k < D ? (uint32_t)seed[(t * 7 + i * 4 + k) & 1023] : 0u;
            qa[i][k] = 0u - 2u * x;
            n += x * x;
        }
        qn[i] = n;
        qr[i] = (uint32_t)seed[(t * 5 + i) & 1023] * 7u;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int32_t x = seed[(t * 13 + j * 4 + 512) & 1023];
        const int32_t y = D > 1 ? seed[(t * 13 + j * 4 + 513) & 1023] : 0;
        const int32_t z = D > 2 ? seed[(t * 13 + j * 4 + 514) & 1023] : 0;
        const int32_t u = D > 3 ? seed[(t * 13 + j * 4 + 515) & 1023] : 0;
        cn[j] = (uint32_t)(x * x + y * y + z * z + u * u);
        c[j] = make_int4(x, y, z, D > 3 ? u : (int32_t)cn[j]);
        ro[j] = make_uint2((uint32_t)seed[(t * 11 + j) & 1023] * 7u, (uint32_t)(t * 16 + j));
    }
    unsigned long long best[4] = {~0ull, ~0ull, ~0ull, ~0ull};
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint32_t nj = D == 4 ? cn[j] : (uint32_t)c[j].w;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t s = nj + qn[i];
                s += (uint32_t)c[j].x * qa[i][0];
                if (D > 1) s += (uint32_t)c[j].y * qa[i][1];
                if (D > 2) s += (uint32_t)c[j].z * qa[i][2];
                if (D > 3) s += (uint32_t)c[j].w * qa[i][3];
                const unsigned long long key = ((unsigned long long)s << 32) | ro[j].y;
                if (ro[j].x < qr[i] && key < best[i]) best[i] = key;
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t m = (uint32_t)(best[i] & 1ull);
            qn[i] += m;
            qr[i] += m;
#pragma unroll
            for (int k = 0; k < D; ++k) qa[i][k] += m;
        }
    }
    if ((best[0] ^ best[1] ^ best[2] ^ best[3]) == 0xdeadbeefull) sink[0] = t;
}

}  // namespace
}  // namespace dpc

extern "C" dpc_status dpc_probe_pair_rate(int device, int d, int mode, double* pairs_per_s, double* ms) {
    using namespace dpc;
    if (!pairs_per_s || d < 1 || d > 8 || mode < 0 || mode > 3 || (mode >= 2 && d > 4))
        return DPC_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return DPC_ERR_CUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int32_t* seed = nullptr;
    unsigned long long* sink = nullptr;
    if (cudaMalloc(&seed, 1024 * sizeof(int32_t)) != cudaSuccess) return DPC_ERR_OOM;
    if (cudaMalloc(&sink, sizeof(unsigned long long)) != cudaSuccess) {
        cudaFree(seed);
        return DPC_ERR_OOM;
    }
    int32_t h[1024];
    for (int i = 0; i < 1024; ++i) h[i] = (int32_t)((i * 2654435761u) % 600u);
    cudaMemcpy(seed, h, sizeof(h), cudaMemcpyHostToDevice);
    const int blocks = sms * 8, threads = 256, iters = 4096;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    auto launch = [&](int it) {
        if (mode == 3) {
            switch (d) {
                case 1: k_ring_probe_x<1><<<blocks, threads>>>(seed, it, sink); break;
                case 2: k_ring_probe_x<2><<<blocks, threads>>>(seed, it, sink); break;
                case 3: k_ring_probe_x<3><<<blocks, threads>>>(seed, it, sink); break;
                default: k_ring_probe_x<4><<<blocks, threads>>>(seed, it, sink); break;
            }
        } else if (mode == 2) {
            switch (d) {
                case 1: k_pair_probe_x<1><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 2: k_pair_probe_x<2><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 3: k_pair_probe_x<3><<<blocks, threads>>>(seed, it, 90000, sink); break;
                default: k_pair_probe_x<4><<<blocks, threads>>>(seed, it, 90000, sink); break;
            }
        } else if (mode == 1) {
            switch (d) {
                case 1: k_pair_probe<1, true><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 2: k_pair_probe<2, true><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 3: k_pair_probe<3, true><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 4: k_pair_probe<4, true><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 5: k_pair_probe<5, true><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 6: k_pair_probe<6, true><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 7: k_pair_probe<7, true><<<blocks, threads>>>(seed, it, 90000, sink); break;
                default: k_pair_probe<8, true><<<blocks, threads>>>(seed, it, 90000, sink); break;
            }
        } else {
            switch (d) {
                case 1: k_pair_probe<1, false><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 2: k_pair_probe<2, false><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 3: k_pair_probe<3, false><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 4: k_pair_probe<4, false><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 5: k_pair_probe<5, false><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 6: k_pair_probe<6, false><<<blocks, threads>>>(seed, it, 90000, sink); break;
                case 7: k_pair_probe<7, false><<<blocks, threads>>>(seed, it, 90000, sink); break;
                default: k_pair_probe<8, false><<<blocks, threads>>>(seed, it, 90000, sink); break;
            }
        }
        note_launch();
    };
    launch(64);  // warm-up
    cudaEventRecord(a);
    launch(iters);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(seed);
    cudaFree(sink);
    if (e != cudaSuccess) return DPC_ERR_CUDA;
    const double pairs = (double)blocks * threads * iters * 64.0;
    *pairs_per_s = pairs / (t * 1e-3);
    if (ms) *ms = t;
    return DPC_OK;
}
