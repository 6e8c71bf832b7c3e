// Grid-wide reductions with a last-CTA finish: each CTA reduces its threads' values with warp
// shuffles, writes one partial per value, and the last CTA to arrive (atomic ticket) combines
// the partials in CTA order. The combination order depends only on the launch shape, so the
// results are deterministic.
#pragma once

#include "mhd_internal.cuh"

namespace mhd {

struct OpSum {
    static __device__ __forceinline__ double apply(double a, double b) { return a + b; }
    static constexpr double identity = 0.0;
};
struct OpMax {
    static __device__ __forceinline__ double apply(double a, double b) { return fmax(a, b); }
    static constexpr double identity = 0.0;  // used only for non-negative quantities
};

// Returns true in the last CTA; there, thread 0 holds the grid-wide results in out[].
// Works for any block size up to 1024 threads (32 warps).
template <int K, typename Op = OpSum>
__device__ __forceinline__ bool reduce_last(double (&v)[K], double* __restrict__ partials,
                                            unsigned int* count, double (&out)[K]) {
    __shared__ double sm[K][32];
    __shared__ int is_last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] = Op::apply(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) sm[k][w] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double s = Op::identity;
            for (int i = 0; i < nw; i++) s = Op::apply(s, sm[k][i]);
            partials[blockIdx.x * K + k] = s;
        }
        __threadfence();
        const unsigned int t = atomicAdd(count, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < K; k++) {
        double s = Op::identity;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s = Op::apply(s, __ldcg(&partials[b * K + k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = Op::apply(s, __shfl_xor_sync(0xffffffffu, s, o));
        v[k] = s;
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) sm[k][w] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double s = Op::identity;
            for (int i = 0; i < nw; i++) s = Op::apply(s, sm[k][i]);
            out[k] = s;
        }
        *count = 0u;
    }
    return true;
}

}  // namespace mhd
