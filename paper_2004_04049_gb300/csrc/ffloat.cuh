// ffloat.cuh - float-float ("double-single") arithmetic for the library's error sums.
//
// A value is an unevaluated sum hi + lo of two float32 numbers with |lo| <= ulp(hi)/2,
// about 48 significant bits. Additions use Knuth's error-free TwoSum and products use the
// FMA-based TwoProd (Dekker's splitting is not needed with fmaf), as in Dekker (1971) and
// the double-double literature (e.g. Hida, Li and Bailey, 2001). The reductions that the
// interface reports in float64 (replay error sums, GS error, target energy) run in this
// form on the float32 pipe: on this GPU a dependent float64 operation costs hundreds of
// cycles, so float64 reduction trees, not the bytes per pixel, would bound the kernels.
// Only the final results are converted to float64.
#pragma once

#include <cuda_runtime.h>

namespace holo {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float x) { return ff{x, 0.f}; }

// error-free a + b = s + e (any magnitudes)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// error-free a + b = s + e when |a| >= |b| (or a == 0)
__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    float t, f;
    two_sum(a.lo, b.lo, t, f);
    e = __fadd_rn(e, t);
    quick_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    ff r;
    quick_two_sum(s, e, r.hi, r.lo);
    return r;
}

// a * b: the product of the high parts formed exactly with an FMA (TwoProd), the cross
// terms added in float32 (about 44 bits)
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    ff r;
    quick_two_sum(p, e, r.hi, r.lo);
    return r;
}

// a / b with one Newton-style correction (about 44 bits)
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    // r = a - q1*b, the product q1*b.hi formed exactly with an FMA
    const float p = __fmul_rn(q1, b.hi);
    const float pe = __fmaf_rn(q1, b.hi, -p);
    ff r = ff_add(a, ff{-p, -pe});
    r = ff_add(r, ff{-__fmul_rn(q1, b.lo), 0.f});
    const float q2 = __fdiv_rn(r.hi, b.hi);
    ff q;
    quick_two_sum(q1, q2, q.hi, q.lo);
    return q;
}

__device__ __forceinline__ double ff_to_double(ff a) { return double(a.hi) + double(a.lo); }

__device__ __forceinline__ ff ff_shfl_xor(ff a, int o) {
    return ff{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// sum over the warp (fixed butterfly order); valid in every lane
__device__ __forceinline__ ff warp_sum_ff(ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = ff_add(v, ff_shfl_xor(v, o));
    return v;
}

// K per-thread float-float sums -> K float-float block sums (valid in thread 0). Warps add
// with a fixed butterfly; warp results are added in warp order. `sm` holds >= 32*K ff
// values. blockDim.x must be a multiple of 32.
template <int K>
__device__ __forceinline__ void block_sums_ffv(const ff (&v)[K], ff (&out)[K], ff* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ff w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = warp_sum_ff(v[k]);
    __syncthreads();   // sm may still be read by a previous call
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sm[k * 32 + warp] = w[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            ff acc = ff_make(0.f);
            for (int i = 0; i < nw; ++i) acc = ff_add(acc, sm[k * 32 + i]);
            out[k] = acc;
        }
    }
}

// the same from K per-thread float32 sums
template <int K>
__device__ __forceinline__ void block_sums_ff(const float (&v)[K], ff (&out)[K], ff* sm) {
    ff w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = ff_make(v[k]);
    block_sums_ffv<K>(w, out, sm);
}

// float-float sum of x[0..n) by one warp: lane l adds x[l], x[l+32], ... in order, then
// a fixed butterfly; valid in every lane of the calling warp. Loads are issued in batches
// of 8 per lane before they are added, so the sum costs a few load latencies, not n/32.
__device__ __forceinline__ ff warp_sum_array_ff(const ff* __restrict__ x, int n) {
    const int lane = threadIdx.x & 31;
    ff v = ff_make(0.f);
    for (int base = 0; base < n; base += 32 * 8) {
        ff buf[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = base + 32 * k + lane;
            buf[k] = i < n ? x[i] : ff_make(0.f);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) v = ff_add(v, buf[k]);
    }
    return warp_sum_ff(v);
}

}  // namespace holo
