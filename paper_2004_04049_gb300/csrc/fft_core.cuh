// fft_core.cuh - float32 line FFTs for the 2D DFT of Eq. 1 / Eq. 2 (paper Section 2).
//
// A "line" is one row or one column of length N (a power of two, 64..4096). The T = N/R
// threads of a line each hold R complex values in registers, in the canonical layout
// "slot e holds element t + T*e". The transform is a Stockham autosort FFT: stages of
// radix R (the last one may be smaller) whose butterflies run in registers, with one
// exchange through a padded shared-memory line buffer between stages. Outputs come back
// in natural order and already in the canonical layout, so a pass ends with coalesced
// global stores of the same shape as its loads.
//
// Stage s (sub-transform length Ns before it, radix Rs): butterfly j = t + b*T with
// k = j mod Ns takes elements j + m*N/Rs (m < Rs), multiplies element m by
// W_{Ns*Rs}^{k*m}, applies a Rs-point DFT, and writes output m to
// (j div Ns)*Ns*Rs + k + m*Ns.
//
// Transforms are unnormalised here: DIR = -1 computes sum x e^{-2 pi i nk/N} (Eq. 1
// without its scale), DIR = +1 the inverse sum (Eq. 2 without its scale). Callers apply
// 1/sqrt(H*W) where a unitary result is needed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace holo {

// ------------------------------------------------------------------ complex ----
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * (c + i*DIR*s) where (c, s) = (cos, sin) of a positive angle
template <int DIR>
__device__ __forceinline__ float2 cmul_dir(float2 a, float2 cs) {
    if (DIR > 0) return make_float2(fmaf(a.x, cs.x, -a.y * cs.y), fmaf(a.y, cs.x, a.x * cs.y));
    return make_float2(fmaf(a.x, cs.x, a.y * cs.y), fmaf(a.y, cs.x, -a.x * cs.y));
}

// --------------------------------------------------------------- FFT plans ----
constexpr int kMinLog2 = 6;    // shortest supported line: 64
constexpr int kMaxLog2 = 12;   // longest supported line: 4096

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }

__host__ __device__ constexpr int stage_ns(int N, int R, int s) {
    int ns = 1;
    for (int i = 0; i < s; ++i) ns *= cmin(R, N / ns);
    return ns;
}
__host__ __device__ constexpr int stage_radix(int N, int R, int s) { return cmin(R, N / stage_ns(N, R, s)); }
__host__ __device__ constexpr int stage_count(int N, int R) {
    int s = 0, ns = 1;
    while (ns < N) { ns *= cmin(R, N / ns); ++s; }
    return s;
}
// twiddles of plan (N, R): for every stage s >= 1 a block of Ns*Rs (cos, sin) pairs,
// entry [m*Ns + k] = angle 2*pi*k*m/(Ns*Rs)
__host__ __device__ constexpr int plan_table_size(int N, int R) {
    int sz = 0;
    for (int s = 1; s < stage_count(N, R); ++s) sz += stage_ns(N, R, s) * stage_radix(N, R, s);
    return sz;
}
__host__ __device__ constexpr int plan_base(int N, int R) {
    int off = 0;
    for (int lg = kMinLog2; lg <= kMaxLog2; ++lg)
        for (int lr = 1; lr <= 5; ++lr) {
            if ((1 << lg) == N && (1 << lr) == R) return off;
            off += plan_table_size(1 << lg, 1 << lr);
        }
    return -1;
}
__host__ __device__ constexpr int twiddle_total() {
    int off = 0;
    for (int lg = kMinLog2; lg <= kMaxLog2; ++lg)
        for (int lr = 1; lr <= 5; ++lr) off += plan_table_size(1 << lg, 1 << lr);
    return off;
}
__host__ __device__ constexpr int stage_offset(int N, int R, int s) {
    int off = plan_base(N, R);
    for (int i = 1; i < s; ++i) off += stage_ns(N, R, i) * stage_radix(N, R, i);
    return off;
}
constexpr int kTwiddleTotal = twiddle_total();

// line buffer: one float2 of padding every R entries (bank spread of the stage stores),
// plus an offset so that the line buffers of the lanes sharing a half-warp start on
// different banks: rows use one line per warp (offset 1); a column pass puts LPC
// consecutive columns on consecutive lanes and 16/LPC thread indices t of each column in
// a half-warp, so its line stride is 16/LPC (mod 16) and lane (lc, t) lands on bank
// lc*16/LPC + t.
__host__ __device__ constexpr int line_stride(int N, int R) { return N + N / R + 1; }
__host__ __device__ constexpr int col_line_stride(int N, int R, int LPC) {
    return N + N / R + (LPC >= 16 ? 1 : 16 / LPC);
}
template <int R>
__device__ __forceinline__ int pad_index(int i) { return i + i / R; }

// ------------------------------------------------------ in-register DFT-R ----
// cos(2*pi*j/32), j = 0..8
__device__ __forceinline__ constexpr float cos32(int j) {
    return j == 0 ? 1.0f
         : j == 1 ? 0.98078528040323044913f
         : j == 2 ? 0.92387953251128675613f
         : j == 3 ? 0.83146961230254523708f
         : j == 4 ? 0.70710678118654752440f
         : j == 5 ? 0.55557023301960222474f
         : j == 6 ? 0.38268343236508977173f
         : j == 7 ? 0.19509032201612826785f
         : 0.0f;
}

// a * exp(DIR * 2 pi i * j / 32) for 0 <= j < 16 (j is a compile-time constant after unrolling)
template <int DIR>
__device__ __forceinline__ float2 rot32(float2 a, int j) {
    if (j == 0) return a;
    if (j == 8) return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    const float c = j < 8 ? cos32(j) : -cos32(16 - j);
    const float s = cos32(j < 8 ? 8 - j : j - 8);
    if (DIR > 0) return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.y, c, a.x * s));
    return make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s));
}

__host__ __device__ constexpr int bitrev(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}
__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// In-place R-point DFT (R = 1..32) of registers a[0..R): iterative radix-2 decimation in
// frequency, then the bit-reversal reorder (register renaming after unrolling).
template <int R, int DIR>
__device__ __forceinline__ void dft_reg(float2 (&a)[R]) {
    if constexpr (R == 1) return;
#pragma unroll
    for (int half = R / 2; half >= 1; half /= 2) {
#pragma unroll
        for (int blk = 0; blk < R; blk += 2 * half) {
#pragma unroll
            for (int k = 0; k < half; ++k) {
                const float2 x = a[blk + k];
                const float2 y = a[blk + k + half];
                a[blk + k] = cadd(x, y);
                a[blk + k + half] = rot32<DIR>(csub(x, y), k * (16 / half));
            }
        }
    }
    float2 b[R];
#pragma unroll
    for (int k = 0; k < R; ++k) b[k] = a[bitrev(k, ilog2(R))];
#pragma unroll
    for (int k = 0; k < R; ++k) a[k] = b[k];
}

// ------------------------------------------------------- Stockham line FFT ----
template <bool BLOCK>
__device__ __forceinline__ void line_sync() {
    if (BLOCK) __syncthreads();
    else __syncwarp();
}

template <int N, int R, int DIR, bool BLOCK, int S>
struct LineStage {
    static __device__ __forceinline__ void run(float2 (&v)[R], float2* buf, int t,
                                               const float2* __restrict__ tw) {
        constexpr int T = N / R;
        constexpr int NSTAGE = stage_count(N, R);
        constexpr int Ns = stage_ns(N, R, S);
        constexpr int Rs = stage_radix(N, R, S);
        constexpr int NB = R / Rs;
        constexpr bool last = (S == NSTAGE - 1);
        if constexpr (S > 0) {
            // pick up the canonical layout written by the previous stage
            line_sync<BLOCK>();
#pragma unroll
            for (int e = 0; e < R; ++e) v[e] = buf[pad_index<R>(t + T * e)];
            if constexpr (!last) line_sync<BLOCK>();
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = t + b * T;
            const int k = j & (Ns - 1);
            float2 u[Rs];
#pragma unroll
            for (int m = 0; m < Rs; ++m) u[m] = v[b + m * NB];
            if constexpr (S > 0) {
                const float2* tws = tw + stage_offset(N, R, S) + k;
#pragma unroll
                for (int m = 1; m < Rs; ++m) u[m] = cmul_dir<DIR>(u[m], __ldg(tws + m * Ns));
            }
            dft_reg<Rs, DIR>(u);
            if constexpr (last) {
#pragma unroll
                for (int m = 0; m < Rs; ++m) v[b + m * NB] = u[m];
            } else {
                const int base = (j / Ns) * Ns * Rs + k;
#pragma unroll
                for (int m = 0; m < Rs; ++m) buf[pad_index<R>(base + m * Ns)] = u[m];
            }
        }
        if constexpr (!last) LineStage<N, R, DIR, BLOCK, S + 1>::run(v, buf, t, tw);
    }
};

// N-point DFT of one line held in canonical layout by its T = N/R threads.
// `buf` is this line's shared-memory buffer of line_stride(N, R) float2; `tw` is the
// global twiddle table. Every thread of the block (BLOCK) or warp (!BLOCK) must call it.
template <int N, int R, int DIR, bool BLOCK>
__device__ __forceinline__ void line_fft(float2 (&v)[R], float2* buf, int t,
                                         const float2* __restrict__ tw) {
    static_assert(N % R == 0 && R <= 32, "bad FFT plan");
    if constexpr (stage_count(N, R) > 1) line_sync<BLOCK>();   // buffer may still be read by a previous use
    LineStage<N, R, DIR, BLOCK, 0>::run(v, buf, t, tw);
}

// ------------------------------------------- replicated cos/sin table ----
// The 256-entry (cos, sin) table replicated COPIES times in shared memory: entry c of
// copy k sits at [c*COPIES + k] and lane l reads copy l mod COPIES. With 16 copies the
// 16 lanes of a half-warp hit 16 different banks whatever codes they look up (random
// codes would otherwise collide); a kernel that looks up few codes per table load uses
// one copy.
template <int COPIES>
constexpr int cs_smem_entries() { return 256 * COPIES; }
constexpr int kCsCopies = 16;
constexpr int kCsSmemEntries = 256 * kCsCopies;

template <int COPIES = kCsCopies>
__device__ __forceinline__ void load_cs_table(float2* sm, const float2* __restrict__ cs256) {
    for (int i = threadIdx.x; i < 256 * COPIES; i += blockDim.x) sm[i] = __ldg(cs256 + i / COPIES);
}
// (cos, sin)(2*pi*i/256) for i < 256
template <int COPIES = kCsCopies>
__device__ __forceinline__ float2 cs_lookup(const float2* sm, uint32_t i) {
    return sm[i * COPIES + (threadIdx.x & (COPIES - 1))];
}

// --------------------------------------------------------------- helpers ----
// a mod d for 32-bit a, d >= 1, with M = floor((2^64 - 1)/d) + 1 precomputed
// (Lemire, Kaser and Kurz, "Faster remainder by direct computation", 2019).
__device__ __forceinline__ uint32_t fastmod_u32(uint32_t a, uint64_t M, uint32_t d) {
    const uint64_t low = M * (uint64_t)a;
    return (uint32_t)__umul64hi(low, (uint64_t)d);
}

// SplitMix64 output k of stream `seed` (Steele, Lea and Flood, 2014).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace holo
