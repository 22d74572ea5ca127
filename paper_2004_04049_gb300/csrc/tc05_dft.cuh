// tc05_dft.cuh - radix-32 DFT stages of a line FFT on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory), for lines of 1024 and 2048 points.
//
// Each thread holds one 32-point sub-line of a Stockham stage in registers (the layout of
// fft_core.cuh). In real form the 32-point DFT is a 64x64 matrix acting on
// [Re x_0..31, Im x_0..31]; 128 threads form one GEMM
//     D[row][j] = sum_i A[row][i] B[j][i]      (M = 128 sub-lines, N = 64, K = 64)
// with A = the sub-lines (each thread writes its own row) and B = the DFT matrix. Every
// operand is split x = hi + lo into two 16-bit floats and D accumulates
// A_hi B_hi + A_lo B_hi + A_hi B_lo in float32 (the lo*lo term is below float32 rounding).
// A and B sit in shared memory in the canonical K-major 128-byte-swizzle layout
// (row r at (r/8)*1024 + (r%8)*128, its 16-byte chunk c at chunk c^(r%8)); one thread per
// group of 128 issues the 12 MMAs and commits them to the group's mbarrier; each thread
// then reads its row back from tensor memory (tcgen05.ld 32x32b: TMEM lane = row).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fft_core.cuh"
#include "runtime.h"

namespace holo {

// the tensor-core precisions (holo.h HOLO_FP16X2, HOLO_BF16X2)
enum TcPrec : int { kTcFp16 = 1, kTcBf16 = 2 };

constexpr int kTc05TileBytes = 128 * 128;   // A tile: 128 rows x 128 bytes
constexpr int kTc05BBytes = 64 * 128;       // B tile: 64 rows x 128 bytes
constexpr uint32_t kTc05WaitLimit = 1u << 22;

// byte offset of element (row, k) of a K-major 128-byte-swizzled tile of 64-element rows
__host__ __device__ constexpr uint32_t sw128_offset(int row, int k) {
    return uint32_t(row >> 3) * 1024u + uint32_t(row & 7) * 128u + (uint32_t(((k >> 3) ^ (row & 7))) << 4) +
           uint32_t(k & 7) * 2u;
}

__device__ __forceinline__ uint64_t tc05_desc(uint32_t addr) {
    return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
           (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

// kind::f16 instruction descriptor: fp16 (0) or bf16 (1) operands, float32 D, M = 128, N = 64
template <int PREC>
__host__ __device__ constexpr uint32_t tc05_idesc() {
    return (1u << 4) | (uint32_t(PREC == kTcBf16 ? 1 : 0) << 7) | (uint32_t(PREC == kTcBf16 ? 1 : 0) << 10) |
           (uint32_t(64 >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

struct Tc05Group {
    uint32_t a_hi, a_lo;   // this group's A tiles (shared addresses, 1024-aligned)
    uint32_t b_hi, b_lo;   // the DFT matrix tiles for the transform direction
    uint32_t bar;          // this group's mbarrier
    uint32_t tmem;         // this group's 64 accumulator columns
    uint32_t phase;        // parity of the next mbarrier phase
    int row;               // this thread's row (threadIdx.x % 128)
    int* fault;            // set when a bounded wait expires
};

template <int PREC>
__device__ __forceinline__ uint32_t pack16(float a, float b, uint32_t& lo) {
    if constexpr (PREC == kTcBf16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 f = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - f.x, b - f.y);
        lo = *reinterpret_cast<const uint32_t*>(&l);
        return *reinterpret_cast<const uint32_t*>(&h);
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 f = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - f.x, b - f.y);
        lo = *reinterpret_cast<const uint32_t*>(&l);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
}

__device__ __forceinline__ void tc05_sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// true once the mbarrier phase of the given parity has completed; false after `limit`
// polls (the caller then records a fault instead of waiting on)
__device__ __forceinline__ bool tc05_wait(uint32_t bar, uint32_t parity, uint32_t limit = kTc05WaitLimit) {
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// u <- DFT_32(u) (unnormalised, direction fixed by the group's B tiles). Every thread of
// the block calls it (three block-wide barriers: the A tiles share memory with the line
// buffers, so they are written only after every thread is done with the buffers, and the
// buffers are released only after every group's MMAs have completed). A variant with a
// named barrier per group (groups owning whole lines) measured slower: it needed more
// registers (spills) and the block barriers were not the limit.
template <int PREC>
__device__ __forceinline__ void dft32_tc05(float2 (&u)[32], Tc05Group& g, float scale, float unscale) {
    __syncthreads();
    const uint32_t rowoff = uint32_t(g.row >> 3) * 1024u + uint32_t(g.row & 7) * 128u;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        // chunk c: K indices 8c .. 8c+7 = Re u[8c..] for c < 4, Im u[8(c-4)..] otherwise
        uint32_t h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int n = 8 * (c & 3) + 2 * q;
            const float a = (c < 4 ? u[n].x : u[n].y) * scale;
            const float b = (c < 4 ? u[n + 1].x : u[n + 1].y) * scale;
            h[q] = pack16<PREC>(a, b, l[q]);
        }
        const uint32_t off = rowoff + (uint32_t(c ^ (g.row & 7)) << 4);
        tc05_sts128(g.a_hi + off, h[0], h[1], h[2], h[3]);
        tc05_sts128(g.a_lo + off, l[0], l[1], l[2], l[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (g.row == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        constexpr uint32_t idesc = tc05_idesc<PREC>();
        const uint32_t as[3] = {g.a_hi, g.a_lo, g.a_hi};
        const uint32_t bs[3] = {g.b_hi, g.b_hi, g.b_lo};
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = tc05_desc(as[p] + 32u * kk), bd = tc05_desc(bs[p] + 32u * kk);
                const uint32_t acc = (p | kk) != 0;
                asm volatile(
                    "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(g.tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(g.bar)
                     : "memory");
    }
    if (!tc05_wait(g.bar, g.phase)) atomicExch(g.fault, 1);
    g.phase ^= 1u;
    // the lanes leave the polling loop independently; tcgen05.ld is .sync.aligned and
    // must be executed by the whole warp together
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t taddr = g.tmem + (uint32_t(32 * ((threadIdx.x >> 5) & 3)) << 16);
    uint32_t r[32];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr + uint32_t(32 * half)));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const float x = __uint_as_float(r[k]) * unscale;
            if (half == 0) u[k].x = x;
            else u[k].y = x;
        }
    }
    // the A tiles share memory with the line buffers the caller writes next
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
}

// N-point line FFT (N = 1024 or 2048) of a line held by its T = N/32 threads in canonical
// layout (slot e <-> element t + T e): the two radix-32 stages on the tensor cores, the
// closing radix-2 stage of a 2048-point line on the CUDA cores. `buf` is the line's padded
// buffer (fft_core.cuh) for the exchanges between the stages. Every thread of the block
// calls it.
template <int N, int DIR, int PREC>
__device__ __forceinline__ void line_fft_tc05(float2 (&v)[32], float2* buf, int t, const float2* __restrict__ tw,
                                             Tc05Group& g) {
    static_assert(N == 1024 || N == 2048, "tcgen05 line FFT: 1024 or 2048 points");
    constexpr int T = N / 32;
    const float scale = PREC == kTcFp16 ? 1.f / 256.f : 1.f;
    const float unscale = PREC == kTcFp16 ? 256.f : 1.f;
    // stage 0 (sub-transform length 1): DFT of elements t + T m, output m to 32 t + m
    dft32_tc05<PREC>(v, g, scale, unscale);
#pragma unroll
    for (int m = 0; m < 32; ++m) buf[pad_index<32>(32 * t + m)] = v[m];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 32; ++e) v[e] = buf[pad_index<32>(t + T * e)];
    // stage 1 (sub-transform length 32): twiddle W_1024^(k m) with k = t mod 32, DFT,
    // output m to element (t / 32) 1024 + k + 32 m
    const int k = t & 31;
    const float2* tws = tw + stage_offset(N, 32, 1) + k;
#pragma unroll
    for (int m = 1; m < 32; ++m) v[m] = cmul_dir<DIR>(v[m], __ldg(tws + 32 * m));
    dft32_tc05<PREC>(v, g, scale, unscale);
    if constexpr (N == 2048) {
        // dft32_tc05 ends with a block barrier, so the buffer is free again
#pragma unroll
        for (int m = 0; m < 32; ++m) buf[pad_index<32>((t >> 5) * 1024 + k + 32 * m)] = v[m];
        LineStage<N, 32, DIR, true, 2>::run(v, buf, t, tw);   // barrier, canonical read, radix 2
    }
}

// ------------------------------------------------- kernel setup of a pass ----
// A pass on tcgen05 runs 256-thread CTAs, two MMA groups of 128 sub-lines: a column pass
// holds 8192 / N columns of N/32 threads, a row pass 8192 / N rows. The A tiles of both
// groups (64 KiB) share memory with the padded line buffers.
constexpr int kTc05Threads = 256;
template <int N>
constexpr int tc05_lpc() { return kTc05Threads / (N / 32); }
template <int N>
constexpr int tc05_col_stride() { return col_line_stride(N, 32, tc05_lpc<N>()); }
template <int N>
constexpr size_t tc05_col_line_bytes() { return sizeof(float2) * tc05_lpc<N>() * tc05_col_stride<N>(); }
template <int N>
constexpr size_t tc05_row_line_bytes() { return sizeof(float2) * tc05_lpc<N>() * line_stride(N, 32); }
static_assert(tc05_col_line_bytes<1024>() >= 4 * kTc05TileBytes && tc05_col_line_bytes<2048>() >= 4 * kTc05TileBytes &&
                  tc05_row_line_bytes<1024>() >= 4 * kTc05TileBytes && tc05_row_line_bytes<2048>() >= 4 * kTc05TileBytes,
              "the A tiles of both groups fit in the line buffers");

// TMEM (128 columns), the B tiles and the mbarriers of a pass, set up by every thread of
// the CTA: `nb` B tiles are copied from `bsrc` to the start of shared memory `bdst`, the
// two mbarriers (one per MMA group) sit at shared address `bars`.
__device__ __forceinline__ void tc05_setup(uint32_t* s_tmem, const uint8_t* bsrc, uint8_t* bdst, int nb,
                                           uint32_t bars) {
    const int tid = threadIdx.x;
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(
                         static_cast<uint32_t>(__cvta_generic_to_shared(s_tmem)))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bars) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bars + 8) : "memory");
    }
    const uint4* src = reinterpret_cast<const uint4*>(bsrc);
    uint4* dst = reinterpret_cast<uint4*>(bdst);
    for (int i = tid; i < nb * kTc05BBytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
}
// after tc05_setup and any other shared-memory fill: the CTA barrier that publishes them
// (the TMEM address that warp 0's allocation wrote included: it is read after the
// barrier), then the MMA group of this thread (A tiles at `atiles`, 2 x kTc05TileBytes
// per group; an expired wait sets *fault)
__device__ __forceinline__ Tc05Group tc05_group(uint32_t atiles, uint32_t bars, const uint32_t* s_tmem, int* fault) {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem_addr = *reinterpret_cast<const volatile uint32_t*>(s_tmem);
    Tc05Group g;
    const int grp = threadIdx.x >> 7;
    g.row = threadIdx.x & 127;
    g.a_hi = atiles + uint32_t(grp) * 2u * kTc05TileBytes;
    g.a_lo = g.a_hi + kTc05TileBytes;
    g.b_hi = g.b_lo = 0;
    g.bar = bars + 8u * grp;
    g.tmem = tmem_addr + 64u * grp;
    g.phase = 0;
    g.fault = fault;
    return g;
}
__device__ __forceinline__ void tc05_teardown(uint32_t tmem_addr) {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(tmem_addr) : "memory");
}
// the 1024-byte aligned start of the dynamic shared memory (generic and shared address)
__device__ __forceinline__ uint8_t* tc05_smem(uint8_t* smraw, uint32_t& base) {
    const uint32_t raw = static_cast<uint32_t>(__cvta_generic_to_shared(smraw));
    base = (raw + 1023u) & ~1023u;
    return smraw + (base - raw);
}

}  // namespace holo
