// Block and grid reductions shared by the assembly and the PCG translation units (each gets its
// own copy: internal linkage).
#pragma once
#include "common.cuh"

namespace ttie {
namespace {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ T block_sum(T v) {
    __shared__ T sh[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    T r = T(0);
    if (w == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : T(0);
#pragma unroll
        for (int o = 16; o; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

// Deterministic grid sums of N values; the last block to finish runs `fin` on the totals.
template <int N, typename Fin>
__device__ __forceinline__ void grid_sums(const double (&v)[N], double *partials, unsigned int *ticket, Fin fin) {
    __shared__ bool last;
    double b[N];
#pragma unroll
    for (int i = 0; i < N; ++i) b[i] = block_sum(v[i]);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) partials[(size_t)i * gridDim.x + blockIdx.x] = b[i];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        double tot[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
            for (unsigned j = threadIdx.x; j < gridDim.x; j += blockDim.x) s += __ldcg(&partials[(size_t)i * gridDim.x + j]);
            tot[i] = block_sum(s);
        }
        if (threadIdx.x == 0) {
            fin(tot);
            *ticket = 0u;
        }
    }
}

}  // namespace
}  // namespace ttie
