// tc_dft.cuh - DFT-32 stages of a line FFT on the tensor cores (mma.sync.m16n8k16) with
// split hi/lo fp16 or bf16 operands and float32 accumulation.
//
// A radix-32 Stockham stage applies the 32-point DFT matrix F[k][m] = exp(DIR 2 pi i km/32)
// to NSUB = N/32 vectors X[.][j] of the line. In real form that is one GEMM
//     [Yr; Yi] = [[Fr, -Fi], [Fi, Fr]] [Xr; Xi]     (M = 64, K = 64, N = NSUB),
// Fr = cos, Fi = DIR sin. Each operand x is split as x = hi + lo with hi = round16(x),
// lo = round16(x - hi), and the product is accumulated as hi*hi + hi*lo + lo*hi in fp32
// (the lo*lo term is below the fp32 rounding of the sum).
//
// Fragment layouts of mma.m16n8k16 (lane = 4*g + c): A (16x16, row major) holds
// {A[g][2c..2c+1], A[g+8][2c..2c+1], A[g][2c+8..2c+9], A[g+8][2c+8..2c+9]}; B (16x8)
// holds {B[2c..2c+1][g], B[2c+8..2c+9][g]}; C (16x8, fp32) holds
// {C[g][2c], C[g][2c+1], C[g+8][2c], C[g+8][2c+1]}.
//
// The DFT matrix never changes, so each warp keeps its A fragments (cos and sin tiles,
// hi and lo) in registers for the whole line; the line itself is staged in shared memory
// (the padded line buffer of fft_core.cuh) and every stage reads one buffer and writes the
// other.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fft_core.cuh"

namespace holo {

enum TcPrec : int { kTcFp16 = 1, kTcBf16 = 2 };

// Per precision: the A fragments of the 32x32 cos and sin matrices, 4 tiles each (16x16,
// tile = 2*mt + kt), hi and lo, 4 registers per lane: [mat][hilo][tile][lane][4].
struct TcFrags {
    uint32_t v[2][2][4][32][4];
};

template <int PREC>
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    if constexpr (PREC == kTcBf16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 f = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - f.x, b - f.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 f = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - f.x, b - f.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

template <int PREC>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    if constexpr (PREC == kTcBf16) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// A fragments of one warp: cos and sin tiles, hi and lo
struct TcA {
    uint32_t c[2][4][4];   // [hilo][tile][reg]
    uint32_t s[2][4][4];
};

template <int PREC>
__device__ __forceinline__ void tc_load_a(TcA& A, const TcFrags* __restrict__ frags, int lane) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint4 cv = __ldg(reinterpret_cast<const uint4*>(frags->v[0][h][t][lane]));
            const uint4 sv = __ldg(reinterpret_cast<const uint4*>(frags->v[1][h][t][lane]));
            A.c[h][t][0] = cv.x; A.c[h][t][1] = cv.y; A.c[h][t][2] = cv.z; A.c[h][t][3] = cv.w;
            A.s[h][t][0] = sv.x; A.s[h][t][1] = sv.y; A.s[h][t][2] = sv.z; A.s[h][t][3] = sv.w;
        }
}

__device__ __forceinline__ void neg4(const uint32_t (&a)[4], uint32_t (&o)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = a[i] ^ 0x80008000u;
}

// One radix-32 stage of an N-point line (N = 32 * NSUB) by one warp on the NSUB/WPL
// vectors j in [j0, j0 + NSUB/WPL):
//   STAGE 0: X[m][j] = in[j + NSUB*m],                     out[32 j + k] = Y[k][j]
//   STAGE 1: X[m][j] = in[j + NSUB*m] * W_{1024}^{(j%32) m}, out[(j/32)*1024 + j%32 + 32 k]
// `scale` multiplies the operand before the split and `unscale` the result (powers of
// two that keep fp16 operands in range).
template <int N, int DIR, int PREC, int STAGE, int WPL>
__device__ __forceinline__ void tc_stage(const float2* __restrict__ in, float2* __restrict__ out, const TcA& A,
                                         int lane, int j0, const float2* __restrict__ tw, float scale,
                                         float unscale) {
    constexpr int NSUB = N / 32;
    constexpr int NT = NSUB / WPL / 8;        // 8-column tiles of this warp
    const int g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int j = j0 + 8 * nt + g;
        // B fragments: real parts (kt = kt') and imaginary parts (kt = kt' + 2)
        uint32_t bre[2][2][2], bim[2][2][2];   // [kt'][hilo][reg]
#pragma unroll
        for (int kt = 0; kt < 2; ++kt) {
            float2 x[4];
            const int m0 = 16 * kt + 2 * c;
            const int ms[4] = {m0, m0 + 1, m0 + 8, m0 + 9};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 v = in[pad_index<32>(j + NSUB * ms[q])];
                if constexpr (STAGE == 1) {
                    const float2 w = __ldg(tw + stage_offset(N, 32, 1) + ms[q] * 32 + (j & 31));
                    v = cmul_dir<DIR>(v, w);
                }
                x[q] = make_float2(v.x * scale, v.y * scale);
            }
            split2<PREC>(x[0].x, x[1].x, bre[kt][0][0], bre[kt][1][0]);
            split2<PREC>(x[2].x, x[3].x, bre[kt][0][1], bre[kt][1][1]);
            split2<PREC>(x[0].y, x[1].y, bim[kt][0][0], bim[kt][1][0]);
            split2<PREC>(x[2].y, x[3].y, bim[kt][0][1], bim[kt][1][1]);
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < 2; ++kt) {
                const int t = 2 * mt + kt;
                // -DIR*sin for the Re output from Im input, +DIR*sin for Im output from Re input
                uint32_t sp[2][4], sn[2][4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (DIR > 0) {
                        neg4(A.s[h][t], sn[h]);
#pragma unroll
                        for (int i = 0; i < 4; ++i) sp[h][i] = A.s[h][t][i];
                    } else {
                        neg4(A.s[h][t], sp[h]);
#pragma unroll
                        for (int i = 0; i < 4; ++i) sn[h][i] = A.s[h][t][i];
                    }
                }
                // re += Fr*Xr - Fi*Xi ; im += Fi*Xr + Fr*Xi   (hi*hi + hi*lo + lo*hi each)
                mma16816<PREC>(re, A.c[0][t], bre[kt][0][0], bre[kt][0][1]);
                mma16816<PREC>(re, A.c[0][t], bre[kt][1][0], bre[kt][1][1]);
                mma16816<PREC>(re, A.c[1][t], bre[kt][0][0], bre[kt][0][1]);
                mma16816<PREC>(re, sn[0], bim[kt][0][0], bim[kt][0][1]);
                mma16816<PREC>(re, sn[0], bim[kt][1][0], bim[kt][1][1]);
                mma16816<PREC>(re, sn[1], bim[kt][0][0], bim[kt][0][1]);
                mma16816<PREC>(im, sp[0], bre[kt][0][0], bre[kt][0][1]);
                mma16816<PREC>(im, sp[0], bre[kt][1][0], bre[kt][1][1]);
                mma16816<PREC>(im, sp[1], bre[kt][0][0], bre[kt][0][1]);
                mma16816<PREC>(im, A.c[0][t], bim[kt][0][0], bim[kt][0][1]);
                mma16816<PREC>(im, A.c[0][t], bim[kt][1][0], bim[kt][1][1]);
                mma16816<PREC>(im, A.c[1][t], bim[kt][0][0], bim[kt][0][1]);
            }
            // C rows k = 16 mt + g (+8), columns j = j0 + 8 nt + 2c (+1)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = 16 * mt + g + (q >= 2 ? 8 : 0);
                const int jj = j0 + 8 * nt + 2 * c + (q & 1);
                const float2 y = make_float2(re[q] * unscale, im[q] * unscale);
                if constexpr (STAGE == 0) out[pad_index<32>(32 * jj + k)] = y;
                else out[pad_index<32>((jj >> 5) * 1024 + (jj & 31) + 32 * k)] = y;
            }
        }
    }
}

// N-point line FFT (N = 1024 or 2048) of a line held in canonical layout (slot e <-> element
// t + T*e, T = N/32) whose two radix-32 stages run on the tensor cores; `buf` and `buf2`
// are this line's two shared-memory line buffers, `wl` the warp's index within the line's
// WPL = T/32 warps. A 2048-point line finishes with its radix-2 stage on the CUDA cores.
// All threads of the block call it (block-wide barriers).
template <int N, int DIR, int PREC>
__device__ __forceinline__ void line_fft_tc(float2 (&v)[32], float2* buf, float2* buf2, float2* buf_w,
                                            float2* buf2_w, int t, int wl, const TcFrags* __restrict__ frags,
                                            const float2* __restrict__ tw) {
    constexpr int T = N / 32;
    constexpr int WPL = T / 32;
    const int lane = threadIdx.x & 31;
    // fp16 keeps only 5 exponent bits: operands are scaled into range and back (exact)
    const float scale = PREC == kTcFp16 ? 1.f / 256.f : 1.f;
    const float unscale = PREC == kTcFp16 ? 256.f : 1.f;
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 32; ++e) buf[pad_index<32>(t + T * e)] = v[e];
    TcA A;
    tc_load_a<PREC>(A, frags, lane);
    __syncthreads();
    tc_stage<N, DIR, PREC, 0, WPL>(buf_w, buf2_w, A, lane, wl * (T / WPL), tw, scale, unscale);
    __syncthreads();
    tc_stage<N, DIR, PREC, 1, WPL>(buf2_w, buf_w, A, lane, wl * (T / WPL), tw, scale, unscale);
    if constexpr (N == 2048) {
        LineStage<N, 32, DIR, true, 2>::run(v, buf, t, tw);
    } else {
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = buf[pad_index<32>(t + T * e)];
    }
}

}  // namespace holo
