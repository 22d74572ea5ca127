// error_block.cuh - one block of the one-pass replay error of Section 5.2 / Eq. 3 (the
// reading, the exact identity and the float-float sums are described in error.cu), as a
// device function shared by the replay_error kernel and the persistent batch kernel.
#pragma once

#include "ffloat.cuh"
#include "runtime.h"

namespace holo {

constexpr int kErrThreads = 256;
constexpr int kErrPix = 16;                             // pixels per thread
constexpr int kErrBlockPix = kErrThreads * kErrPix;     // pixels per block
constexpr int kErrParts = 7;                            // partials per block, see below

// blocks of a P-pixel image (at least one)
__host__ __device__ inline int err_blocks(int64_t P) {
    const int64_t nb = (P + kErrBlockPix - 1) / kErrBlockPix;
    return int(nb < 1 ? 1 : nb);
}

// Block b owns pixels [4096 b, 4096 b + 4096). With 16-byte aligned inputs (and a pixel
// count divisible by 4) thread t reads the float4 groups 1024 b + 256 k + t (k < 4), else
// the single pixels 4096 b + 256 k + t (k < 16); both are coalesced. Pixels past P read
// as I = T = 0 with mask 0.
struct ErrPixels {
    float i[kErrPix], t[kErrPix], m[kErrPix];
};

__device__ __forceinline__ void err_gather(const float* __restrict__ I, const float* __restrict__ T,
                                           const uint8_t* __restrict__ mask, int64_t P, bool vec, int64_t b,
                                           bool active, ErrPixels& x) {
    if (!active) {   // threads beyond the block's 256 (a larger CTA running one block): no pixels
#pragma unroll
        for (int k = 0; k < kErrPix; ++k) x.i[k] = x.t[k] = x.m[k] = 0.f;
        return;
    }
    if (vec) {
        const int64_t P4 = P / 4;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t g = b * (kErrBlockPix / 4) + k * kErrThreads + threadIdx.x;
            const bool in = g < P4;
            const float4 iv = in ? __ldg(reinterpret_cast<const float4*>(I) + g) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 tv = in ? __ldg(reinterpret_cast<const float4*>(T) + g) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float w = in ? 1.f : 0.f;
            float4 mv = make_float4(w, w, w, w);
            if (mask && in) {
                const uchar4 m = reinterpret_cast<const uchar4*>(mask)[g];
                mv = make_float4(m.x ? 1.f : 0.f, m.y ? 1.f : 0.f, m.z ? 1.f : 0.f, m.w ? 1.f : 0.f);
            }
            x.i[4 * k] = iv.x; x.i[4 * k + 1] = iv.y; x.i[4 * k + 2] = iv.z; x.i[4 * k + 3] = iv.w;
            x.t[4 * k] = tv.x; x.t[4 * k + 1] = tv.y; x.t[4 * k + 2] = tv.z; x.t[4 * k + 3] = tv.w;
            x.m[4 * k] = mv.x; x.m[4 * k + 1] = mv.y; x.m[4 * k + 2] = mv.z; x.m[4 * k + 3] = mv.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kErrPix; ++k) {
            const int64_t p = b * kErrBlockPix + k * kErrThreads + threadIdx.x;
            const bool in = p < P;
            x.i[k] = in ? I[p] : 0.f;
            x.t[k] = in ? T[p] : 0.f;
            x.m[k] = in ? (mask ? (mask[p] ? 1.f : 0.f) : 1.f) : 0.f;
        }
    }
}

// Block b of nb: partials laid out [k][nb]: k = 0 sum I T^2, 1 sum I^2, 2 sum T^4,
// 3 count, 4 S1, 5 S2, 6 a_b (as {a_b, 0}); *done must be 0 before the first block (the
// host clears it). Threads 0..255 carry the block's pixels; a CTA with more threads runs
// the same block with the others contributing exact zeros (a float-float sum plus zero is
// unchanged), so the results are the same bits. The block that completes the count
// writes d_out and, when `finished` is given, then sets *finished = 1 (release).
__device__ __forceinline__ void replay_error_block(const float* __restrict__ I, const float* __restrict__ T,
                                                   const uint8_t* __restrict__ mask, int64_t P, ff* part,
                                                   unsigned* done, double* __restrict__ d_out, int b, int nb,
                                                   unsigned* finished = nullptr) {
    __shared__ ff sm[32 * 4];
    __shared__ float s_scale;
    __shared__ ff s_alpha;
    __shared__ bool s_last;
    const bool active = threadIdx.x < kErrThreads;
    const bool vec = (P % 4 == 0) && ((reinterpret_cast<uintptr_t>(I) | reinterpret_cast<uintptr_t>(T) |
                                       reinterpret_cast<uintptr_t>(mask)) & 15) == 0;
    ErrPixels x;
    err_gather(I, T, mask, P, vec, b, active, x);
    // this block's sums and its own scale a_b
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < kErrPix; ++k) {
        x.t[k] = x.t[k] * x.t[k] * x.m[k];   // T^2, masked
        x.i[k] = x.i[k] * x.m[k];            // I, masked
        acc[0] = fmaf(x.i[k], x.t[k], acc[0]);
        acc[1] = fmaf(x.i[k], x.i[k], acc[1]);
        acc[2] = fmaf(x.t[k], x.t[k], acc[2]);
        acc[3] += x.m[k];
    }
    ff b4[4];
    block_sums_ff<4>(acc, b4, sm);
    if (threadIdx.x == 0) {
        s_scale = b4[1].hi > 0.f ? ff_div(b4[0], b4[1]).hi : 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) part[size_t(k) * nb + b] = b4[k];
    }
    __syncthreads();
    const float ab = s_scale;
    float acc2[2] = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < kErrPix; ++k) {
        const float d = fmaf(ab, x.i[k], -x.t[k]);
        acc2[0] = fmaf(d, d, acc2[0]);
        acc2[1] = fmaf(x.i[k], d, acc2[1]);
    }
    ff b2[2];
    block_sums_ff<2>(acc2, b2, sm);
    // publish this block's partials; the block whose increment completes the count reduces
    // them (threadfence reduction: every other block fenced its stores before its
    // increment, and the last block reads the partials through L2)
    if (threadIdx.x == 0) {
        part[size_t(4) * nb + b] = b2[0];
        part[size_t(5) * nb + b] = b2[1];
        part[size_t(6) * nb + b] = ff_make(ab);
        __threadfence();
        s_last = atomicAdd(done, 1u) == unsigned(nb - 1);
    }
    __syncthreads();
    if (!s_last) return;   // uniform over the CTA
    __threadfence();
    const float2* p2 = reinterpret_cast<const float2*>(part);
    auto at = [&](int k, int j) {
        const float2 q = __ldcg(p2 + size_t(k) * nb + j);
        return ff{q.x, q.y};
    };
    // global sums: thread t adds blocks t, t + 256, ... in order, then the threads' sums in
    // a fixed order
    ff g[4] = {ff_make(0.f), ff_make(0.f), ff_make(0.f), ff_make(0.f)};
    for (int j = threadIdx.x; active && j < nb; j += kErrThreads)
#pragma unroll
        for (int k = 0; k < 4; ++k) g[k] = ff_add(g[k], at(k, j));
    ff tot[4];
    block_sums_ffv<4>(g, tot, sm);
    if (threadIdx.x == 0) s_alpha = tot[1].hi > 0.f ? ff_div(tot[0], tot[1]) : ff_make(0.f);
    __syncthreads();
    const ff alpha = s_alpha;
    // the squared error at alpha from every block's S1, S2, sum I^2 and a_b
    ff sse[1] = {ff_make(0.f)};
    for (int j = threadIdx.x; active && j < nb; j += kErrThreads) {
        const ff d = ff_add(alpha, ff_make(-at(6, j).hi));
        const ff two_d = ff{2.f * d.hi, 2.f * d.lo};
        ff term = ff_add(at(4, j), ff_mul(two_d, at(5, j)));
        term = ff_add(term, ff_mul(ff_mul(d, d), at(1, j)));
        sse[0] = ff_add(sse[0], term);
    }
    ff s[1];
    block_sums_ffv<1>(sse, s, sm);
    if (threadIdx.x == 0) {
        d_out[0] = ff_to_double(alpha);
        d_out[1] = tot[3].hi > 0.f ? ff_to_double(ff_div(s[0], tot[3])) : 0.0;
        d_out[2] = tot[2].hi > 0.f ? ff_to_double(ff_div(s[0], tot[2])) : 0.0;
        if (finished) {
            __threadfence();
            atomicExch(finished, 1u);
        }
    }
}


}  // namespace holo
