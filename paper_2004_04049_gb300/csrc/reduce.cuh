// reduce.cuh - deterministic float64 block and grid reductions.
//
// A grid reduction here is: every block reduces its share with a fixed tree and writes
// one partial per block; the last block to finish (found with an atomic ticket) adds
// the partials in block order with the same fixed tree. The result does not depend on
// block scheduling, so repeated runs give identical bits.
#pragma once

#include <cuda_runtime.h>

namespace holo {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; the result is valid in thread 0. `sm` holds >= 32 doubles.
// blockDim.x must be a multiple of 32.
__device__ __forceinline__ double block_sum(double v, double* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();   // sm may still be read by a previous call
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (warp == 0) {
        v = lane < nw ? sm[lane] : 0.0;
        v = warp_sum(v);
    }
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// K float32 per-thread sums -> K float64 block sums, valid in thread 0 (out[k]).
// The 32 values of a warp are added in float32 (a five-level tree); warp results are
// converted to float64 and added across warps in a fixed order. `sm` holds >= 32*K
// doubles. blockDim.x must be a multiple of 32.
template <int K>
__device__ __forceinline__ void block_sums_f32_to_f64(const float (&v)[K], double (&out)[K], double* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = warp_sum_f(v[k]);
    __syncthreads();   // sm may still be read by a previous call
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sm[k * 32 + warp] = double(w[k]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double acc = 0.0;
            for (int i = 0; i < nw; ++i) acc += sm[k * 32 + i];
            out[k] = acc;
        }
    }
}

// float64 sum of x[0..n) by one warp: lane l adds x[l], x[l+32], ... in order, then a
// fixed shuffle tree; the result is valid in every lane of the calling warp.
__device__ __forceinline__ double warp_sum_array(const double* __restrict__ x, int n) {
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    for (int i = lane; i < n; i += 32) v += x[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Writes `v` (valid in thread 0) as this block's partial and returns true in every
// thread of the last block to finish; that block may then read all partials.
__device__ __forceinline__ bool grid_partial_done(double v, double* partials, unsigned int* ticket,
                                                  int* s_last) {
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = v;
        __threadfence();
        const unsigned int n = atomicAdd(ticket, 1u);
        *s_last = (n == gridDim.x - 1);
    }
    __syncthreads();
    const bool last = *s_last != 0;
    if (last) __threadfence();
    return last;
}

// In the last block: fixed-order sum of partials[0..n), valid in thread 0.
__device__ __forceinline__ double sum_partials(const double* partials, int n, double* sm) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += ((volatile const double*)partials)[i];
    return block_sum(v, sm);
}

}  // namespace holo
