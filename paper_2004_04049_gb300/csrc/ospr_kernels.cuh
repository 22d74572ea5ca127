// ospr_kernels.cuh - kernels of binary-phase One-Step Phase-Retrieval (paper Sections 2, 3, 5.2, 6).
//
// Per sub-frame s: E = T*exp(i*theta_s) with theta_s from the LUT draw rule (Fig. 3),
// H_s = IDFT(E) (Eq. 2), h_s = sign(Re H_s) with sign(0) = +1, and the replay
// I = (1/N) sum_s |DFT(h_s)|^2 (Eq. 1).
//
// Only Re H_s is needed and h_s is real, so sub-frames go through the transforms in
// pairs (s0, s1) = (2j, 2j+1):
//   * IDFT of the Hermitian part E^h(k) = E(k) + conj(E(-k)) is real and equals
//     2 Re IDFT(E), so one complex IDFT of Z = E^h_{s0} + i E^h_{s1} gives
//     Re H_{s0} (real part) and Re H_{s1} (imaginary part) at once, up to a positive
//     factor the binarisation ignores;
//   * DFT(h_{s0} + i h_{s1}) = R_{s0} + i R_{s1} with R real-input spectra, and
//     |R_{s0}(k)|^2 + |R_{s1}(k)|^2 = (|Z(k)|^2 + |Z(-k)|^2)/2, so the kernels
//     accumulate S = sum |Z|^2 and the last step symmetrises S(k) + S(-k).
// An odd N leaves one sub-frame that is transformed alone (Z = E, h imaginary part 0).
//
// Three passes per chunk of pairs, each one global round trip of a complex field:
//   col_ifft  columns: build Z from the target and the table, column IDFT
//   row       rows:    row IDFT, binarise (bits out), row DFT of h_{s0} + i h_{s1}
//   col_fft   columns: column DFT, S += |Z|^2 over the pairs of a group
// then finalize: I(k) = (sum_g S_g(k) + S_g(-k)) / (2*N*H*W).
#pragma once

#include "fft_core.cuh"
#include "phase_source.cuh"
#include "runtime.h"

namespace holo {

// Launch shapes per line length and tile variant V (the autotuner picks V per shape).
// Column passes hold LPC columns of T = N/R threads with R elements each; row passes use
// T >= 32 threads per row so that a warp holds 32 consecutive pixels.
template <int N, int V> struct ColCfg;
template <> struct ColCfg<64, 0>   { static constexpr int R = 8,  LPC = 32; };
template <> struct ColCfg<128, 0>  { static constexpr int R = 16, LPC = 32; };
template <> struct ColCfg<256, 0>  { static constexpr int R = 16, LPC = 32; };
template <> struct ColCfg<512, 0>  { static constexpr int R = 16, LPC = 16; };
template <> struct ColCfg<1024, 0> { static constexpr int R = 32, LPC = 16; };
template <> struct ColCfg<2048, 0> { static constexpr int R = 32, LPC = 8; };
template <> struct ColCfg<4096, 0> { static constexpr int R = 32, LPC = 4; };
template <> struct ColCfg<512, 1>  { static constexpr int R = 32, LPC = 16; };
template <> struct ColCfg<1024, 1> { static constexpr int R = 32, LPC = 8; };
template <> struct ColCfg<2048, 1> { static constexpr int R = 32, LPC = 4; };
template <> struct ColCfg<4096, 1> { static constexpr int R = 32, LPC = 2; };
template <> struct ColCfg<512, 2>  { static constexpr int R = 16, LPC = 8; };
template <> struct ColCfg<1024, 2> { static constexpr int R = 16, LPC = 8; };
template <> struct ColCfg<2048, 2> { static constexpr int R = 16, LPC = 4; };
template <> struct ColCfg<4096, 2> { static constexpr int R = 16, LPC = 2; };
template <int N, int V> struct RowCfg;
template <> struct RowCfg<64, 0>   { static constexpr int R = 2,  LPR = 4; };
template <> struct RowCfg<128, 0>  { static constexpr int R = 4,  LPR = 4; };
template <> struct RowCfg<256, 0>  { static constexpr int R = 8,  LPR = 4; };
template <> struct RowCfg<512, 0>  { static constexpr int R = 16, LPR = 4; };
template <> struct RowCfg<1024, 0> { static constexpr int R = 32, LPR = 4; };
template <> struct RowCfg<2048, 0> { static constexpr int R = 32, LPR = 2; };
template <> struct RowCfg<4096, 0> { static constexpr int R = 32, LPR = 1; };
template <> struct RowCfg<512, 1>  { static constexpr int R = 8,  LPR = 4; };
template <> struct RowCfg<1024, 1> { static constexpr int R = 16, LPR = 2; };
template <> struct RowCfg<2048, 1> { static constexpr int R = 16, LPR = 1; };
template <> struct RowCfg<4096, 1> { static constexpr int R = 16, LPR = 1; };
// tile variants of each length (column passes: 0..2, row pass: 0..1 from 512 up)
constexpr int col_variants(int N) { return N >= 512 ? 3 : 1; }
constexpr int row_variants(int N) { return N >= 512 ? 2 : 1; }

constexpr int kMaxChunkPairs = 16;   // pairs whose fields are in flight at once
constexpr int kMaxGroups = 4;        // partial accumulators of the column DFT pass

struct OsprArgs {
    const float* target;
    int H, W, N;
    PhaseSource ps;
    float2* zbuf;         // [chunk pairs][H][W]
    float* sacc;          // [groups][H][W]
    int groups;
    int first_pair;       // global index of the chunk's pair 0
    int pairs;            // pairs in this chunk
    uint32_t* bits;       // [N][H*W/32] or null
    int accumulate;       // add to sacc instead of overwriting
    const float2* tw;
    const float2* cs256;
    const uint8_t* tc05b; // tcgen05 DFT-32 matrices of that precision ([direction][hi, lo])
    // Fresnel propagation: one sub-frame per field slot (no two-for-one packing) and the
    // quadratic phase Q(y, x) = chirp_y[y] * chirp_x[x]; 0 / null for the far field
    int fresnel;
    const float2* chirp_y;   // [H] exp(i*pi*kappa*(y - H/2)^2)
    const float2* chirp_x;   // [W] exp(i*pi*kappa*(x - W/2)^2)
};

// first sub-frame of field slot `slot` and whether the slot holds one sub-frame only
__device__ __forceinline__ int slot_subframe(const OsprArgs& a, int slot, bool& single) {
    const int s0 = (a.fresnel ? 1 : 2) * (a.first_pair + slot);
    single = a.fresnel || s0 + 1 >= a.N;
    return s0;
}

template <int NC, int V>
constexpr int col_stride() { return col_line_stride(NC, ColCfg<NC, V>::R, ColCfg<NC, V>::LPC); }
// pass 1 also holds the replicated cos/sin table
template <int NC, int V>
constexpr size_t col_ifft_smem_bytes() {
    return sizeof(float2) * (kCsSmemEntries + size_t(ColCfg<NC, V>::LPC) * col_stride<NC, V>());
}
template <int NC, int V>
constexpr size_t col_fft_smem_bytes() {
    return sizeof(float2) * size_t(ColCfg<NC, V>::LPC) * col_stride<NC, V>();
}
template <int NR, int V>
constexpr size_t row_smem_bytes() {
    return sizeof(float2) * size_t(RowCfg<NR, V>::LPR) * line_stride(NR, RowCfg<NR, V>::R);
}

// Line FFT of a column pass: line lc of the LPC line buffers at `lines`
template <int NC, int V, int DIR>
__device__ __forceinline__ void col_line_fft(float2 (&v)[ColCfg<NC, V>::R], float2* lines, int lc, int t,
                                             const OsprArgs& a) {
    constexpr int R = ColCfg<NC, V>::R, S = col_stride<NC, V>();
    line_fft<NC, R, DIR, true>(v, lines + lc * S, t, a.tw);
}

// Line FFT of a row pass: line `line` of LPR, T = N/R threads per line.
template <int NR, int V, int DIR>
__device__ __forceinline__ void row_line_fft(float2 (&v)[RowCfg<NR, V>::R], float2* lines, int line, int t,
                                             const OsprArgs& a) {
    constexpr int R = RowCfg<NR, V>::R, T = NR / R;
    constexpr int S = line_stride(NR, R);
    line_fft<NR, R, DIR, (T > 32)>(v, lines + line * S, t, a.tw);
}

// ------------------------------------------------------------------ pass 1 ----
// Z = E^h_{s0} + i E^h_{s1} needs, at pixel p, E_s(p) and E_s(-p) of both sub-frames, and
// Z(-p) = conj(E^h_{s0}(p)) + i conj(E^h_{s1}(p)) needs the same four values. A CTA
// therefore holds mirror columns together: its first LPC/2 lines take columns
// u = blockIdx.x*LPC/2 + j and the last LPC/2 lines their mirrors W - u (for u = 0 the
// self-mirrored columns 0 and W/2), and each element pair {p, -p} is generated once, by
// one of the two threads that own p and -p, which hands the other its value through
// shared memory.
template <int LPC>
__device__ __forceinline__ void mirror_column(int b, int lc, int W, int& col, int& partner) {
    constexpr int HL = LPC / 2;
    static_assert(LPC >= 2 && (LPC & (LPC - 1)) == 0, "mirror pairing needs an even power-of-two LPC");
    const int u = b * HL + (lc & (HL - 1));
    const bool second = lc >= HL;
    if (u == 0) {
        col = second ? W / 2 : 0;
        partner = lc;
    } else {
        col = second ? W - u : u;
        partner = second ? lc - HL : lc + HL;
    }
}

// Element e of thread t is row r = t + T*e; its mirror row (H - r) mod H is row
// (T - t) + T*(R-1-e) of thread T - t for t > 0 and row T*((R - e) mod R) of thread 0 for
// t = 0. Threads with t > 0 generate slots 0..R/2-1 and receive R/2..R-1; thread 0
// generates 0..R/2 (slots 0 and R/2 mirror onto themselves and are not handed over) and
// receives R/2+1..R-1. `xline` is the partner line's buffer.
//
// MODE and SINGLE are compile-time so that the element loops hold no branches: for each
// batch of kBatch elements every load (target, mirror target, four codes) is issued before
// any of them is used. SINGLE (the last sub-frame of an odd N) has no mirror terms and
// builds all R slots itself.
constexpr int kBatch = 16;

template <int NC, int V, int MODE, bool SINGLE>
__device__ __forceinline__ void ospr_build_column(float2 (&v)[ColCfg<NC, V>::R], const OsprArgs& a,
                                                  const float2* cs, float2* xline, int t, int c, int s0) {
    constexpr int R = ColCfg<NC, V>::R, T = NC / R;
    constexpr int EG = SINGLE ? R : R / 2;   // slots generated by every thread
    constexpr int B = EG < kBatch ? EG : kBatch;
    const int W = a.W;
    const int cm = (W - c) & (W - 1);
    const int sh = a.ps.cs_shift;
    const SubframeDraw d0 = subframe_draw(a.ps, s0);
    const SubframeDraw d1 = subframe_draw(a.ps, SINGLE ? s0 : s0 + 1);
    // table mode: indices (start + s*stride + p) mod L advance by D = T*W mod L per element;
    // the mirror pixel of row r = t + T*e is (H - r)*W + cm = q0 - e*T*W, except for row 0
    const uint32_t L = a.ps.L;
    const uint64_t fm = a.ps.fm;
    uint32_t D = 0, i0 = 0, i1 = 0, m0 = 0, m1 = 0, z0 = 0, z1 = 0;
    if constexpr (MODE == kPhaseTable) {
        D = uint32_t((uint64_t(T) * uint64_t(W)) % L);
        const uint32_t p0 = uint32_t(t) * uint32_t(W) + uint32_t(c);
        const uint32_t q0 = uint32_t(NC - t) * uint32_t(W) + uint32_t(cm);
        i0 = fastmod_u32(d0.base_mod + p0, fm, L);
        i1 = fastmod_u32(d1.base_mod + p0, fm, L);
        m0 = fastmod_u32(d0.base_mod + q0, fm, L);
        m1 = fastmod_u32(d1.base_mod + q0, fm, L);
        z0 = fastmod_u32(d0.base_mod + uint32_t(cm), fm, L);
        z1 = fastmod_u32(d1.base_mod + uint32_t(cm), fm, L);
    }
    const int gshift = 64 - a.ps.bits;
    // packed codes of (s0, p), (s0, -p), (s1, p), (s1, -p), one byte each, of row r (slot e)
    auto codes_of = [&](int e, int r, int rm) -> uint32_t {
        if constexpr (MODE == kPhaseTable) {
            const uint32_t jm0 = (e == 0 && t == 0) ? z0 : m0;
            const uint32_t jm1 = (e == 0 && t == 0) ? z1 : m1;
            // ordinary (coherent) loads: the persistent batch kernel builds a frame's table in
            // the same launch that reads it, which the read-only path does not allow
            uint32_t w = a.ps.codes[i0];
            if constexpr (!SINGLE) {
                w |= uint32_t(a.ps.codes[jm0]) << 8;
                w |= uint32_t(a.ps.codes[i1]) << 16;
                w |= uint32_t(a.ps.codes[jm1]) << 24;
            }
            i0 += D; i0 -= (i0 >= L) ? L : 0u;
            i1 += D; i1 -= (i1 >= L) ? L : 0u;
            m0 = (m0 >= D) ? m0 - D : m0 + (L - D);
            m1 = (m1 >= D) ? m1 - D : m1 + (L - D);
            return w;
        } else if constexpr (MODE == kPhaseGenerator) {
            const uint64_t p = uint64_t(r) * uint64_t(W) + uint64_t(c);
            const uint64_t pm = uint64_t(rm) * uint64_t(W) + uint64_t(cm);
            uint32_t w = uint32_t(splitmix64_at(a.ps.seed, d0.base + p) >> gshift);
            if constexpr (!SINGLE) {
                w |= uint32_t(splitmix64_at(a.ps.seed, d0.base + pm) >> gshift) << 8;
                w |= uint32_t(splitmix64_at(a.ps.seed, d1.base + p) >> gshift) << 16;
                w |= uint32_t(splitmix64_at(a.ps.seed, d1.base + pm) >> gshift) << 24;
            }
            return w;
        } else {
            return 0u;   // flat phase
        }
    };
    // Hermitian parts E(k) + conj(E(-k)) of both sub-frames at row r
    auto hermitian = [&](float tp, float tm, uint32_t pk, float2& h0, float2& h1) {
        const float2 c0 = cs_lookup(cs, (pk & 0xffu) << sh);
        const float2 c0m = cs_lookup(cs, ((pk >> 8) & 0xffu) << sh);
        const float2 c1 = cs_lookup(cs, ((pk >> 16) & 0xffu) << sh);
        const float2 c1m = cs_lookup(cs, (pk >> 24) << sh);
        h0 = make_float2(fmaf(tp, c0.x, tm * c0m.x), fmaf(tp, c0.y, -tm * c0m.y));
        h1 = make_float2(fmaf(tp, c1.x, tm * c1m.x), fmaf(tp, c1.y, -tm * c1m.y));
    };
#pragma unroll
    for (int e0 = 0; e0 < EG; e0 += B) {
        float tp[B], tm[B];
        uint32_t pk[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int e = e0 + k;
            const int r = t + T * e;
            const int rm = (NC - r) & (NC - 1);
            tp[k] = __ldg(a.target + r * W + c);
            tm[k] = SINGLE ? 0.f : __ldg(a.target + rm * W + cm);
            pk[k] = codes_of(e, r, rm);
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int e = e0 + k;
            if constexpr (SINGLE) {
                const float2 c0 = cs_lookup(cs, (pk[k] & 0xffu) << sh);
                v[e] = make_float2(tp[k] * c0.x, tp[k] * c0.y);
            } else {
                float2 h0, h1;
                hermitian(tp[k], tm[k], pk[k], h0, h1);
                v[e] = make_float2(h0.x - h1.y, h0.y + h1.x);
                if (t > 0 || e > 0) {
                    const int rm = (NC - (t + T * e)) & (NC - 1);
                    xline[pad_index<R>(rm)] = make_float2(h0.x + h1.y, h1.x - h0.y);
                }
            }
        }
    }
    if constexpr (!SINGLE) {
        if (t == 0) {   // row H/2: its mirror is row H/2 of the partner line, built there
            constexpr int e = R / 2;
            const int r = T * e;
            const float tp = __ldg(a.target + r * W + c);
            const float tm = __ldg(a.target + r * W + cm);
            float2 h0, h1;
            hermitian(tp, tm, codes_of(e, r, r), h0, h1);
            v[e] = make_float2(h0.x - h1.y, h0.y + h1.x);
        }
    }
}

// Pass 1 on column tile `tile` (LPC/2 mirror column pairs) of field slot `slot`; every
// thread of the CTA (ColCfg threads) calls it with the cos/sin table `cs` loaded and the
// line buffers `lines` free (no thread still reading them). `trigger` lets the next kernel
// launch once the tile's transforms are done.
template <int NC, int V>
__device__ __forceinline__ void ospr_col_ifft_tile(const OsprArgs& a, int tile, int slot, const float2* cs,
                                                   float2* lines, bool trigger) {
    constexpr int R = ColCfg<NC, V>::R, LPC = ColCfg<NC, V>::LPC, T = NC / R, S = col_stride<NC, V>();
    static_assert(stage_count(NC, R) > 1, "the line FFT's opening barrier guards the exchange buffer");
    const int lc = threadIdx.x % LPC, t = threadIdx.x / LPC;
    const int W = a.W;
    int c, pl;
    mirror_column<LPC>(tile, lc, W, c, pl);
    bool single;   // uniform over the CTA
    const int s0 = slot_subframe(a, slot, single);
    float2* xline = lines + pl * S;
    float2 v[R];
    if (a.ps.mode == kPhaseTable) {
        if (single) ospr_build_column<NC, V, kPhaseTable, true>(v, a, cs, xline, t, c, s0);
        else ospr_build_column<NC, V, kPhaseTable, false>(v, a, cs, xline, t, c, s0);
    } else if (a.ps.mode == kPhaseGenerator) {
        if (single) ospr_build_column<NC, V, kPhaseGenerator, true>(v, a, cs, xline, t, c, s0);
        else ospr_build_column<NC, V, kPhaseGenerator, false>(v, a, cs, xline, t, c, s0);
    } else {
        if (single) ospr_build_column<NC, V, kPhaseFlat, true>(v, a, cs, xline, t, c, s0);
        else ospr_build_column<NC, V, kPhaseFlat, false>(v, a, cs, xline, t, c, s0);
    }
    if (!single) {
        __syncthreads();
        const float2* own = lines + lc * S;
#pragma unroll
        for (int e = R / 2; e < R; ++e)
            if (t > 0 || e > R / 2) v[e] = own[pad_index<R>(t + T * e)];
    }
    col_line_fft<NC, V, +1>(v, lines, lc, t, a);
    if (trigger) pdl_trigger();
    float2* z = a.zbuf + size_t(slot) * size_t(NC) * size_t(W);
#pragma unroll
    for (int e = 0; e < R; ++e) z[size_t(t + T * e) * W + c] = v[e];
}

// One tile with the table loaded first (the persistent batch kernel's form).
template <int NC, int V>
__device__ __forceinline__ void ospr_col_ifft_body(const OsprArgs& a, int tile, int slot) {
    extern __shared__ float2 sm[];
    load_cs_table(sm, a.cs256);
    pdl_wait();   // the table and target may be written by the previous kernel
    __syncthreads();
    ospr_col_ifft_tile<NC, V>(a, tile, slot, sm, sm + kCsSmemEntries, true);
}

// Pass 1 over the chunk's n = (W/LPC) x pairs tiles, item i being tile i mod (W/LPC) of
// slot i / (W/LPC). Where col_ifft_loops holds the grid has one CTA per resident slot and
// CTA b takes items b, b + G, b + 2G, ...: it loads the cos/sin table once, and the CTAs
// running at one time write neighbouring tiles of one field, as a grid of one CTA per
// tile would (1024-point columns of variant 0: 80.4 against 82.8 us per 12-pair launch at
// 1024^2; longer columns and the other variants ran slower so, and keep one CTA per tile,
// grid (W/LPC, pairs)).
// (256-thread tiles are held to 128 registers, two CTAs per SM)
template <int NC, int V>
constexpr bool col_ifft_loops() { return V == 0 && NC <= 1024; }

template <int NC, int V>
__global__ void __launch_bounds__((NC / ColCfg<NC, V>::R) * ColCfg<NC, V>::LPC,
                                  (NC / ColCfg<NC, V>::R) * ColCfg<NC, V>::LPC <= 256 ? 2 : 1)
k_ospr_col_ifft(OsprArgs a) {
    if constexpr (col_ifft_loops<NC, V>()) {
        extern __shared__ float2 sm[];
        load_cs_table(sm, a.cs256);
        pdl_wait();   // the table and target may be written by the previous kernel
        const int tiles = a.W / ColCfg<NC, V>::LPC;
        const int n = tiles * a.pairs;
        for (int i = blockIdx.x; i < n; i += gridDim.x) {
            __syncthreads();   // the table is in place; the previous tile is done with the line buffers
            ospr_col_ifft_tile<NC, V>(a, i % tiles, i / tiles, sm, sm + kCsSmemEntries, i + int(gridDim.x) >= n);
        }
    } else {
        ospr_col_ifft_body<NC, V>(a, int(blockIdx.x), int(blockIdx.y));
    }
}

// ------------------------------------------------------------------ pass 2 ----
// FRESNEL: the row holds one sub-frame's IDFT(E); the hologram field is conj(Q) * IDFT(E),
// binarised on its real part, and the replay transform takes h * Q.
// Rows row0 + threadIdx.x / T of field slot `slot` (a CTA of any multiple of T threads
// holds that many lines; the kernel below uses RowCfg's LPR lines per CTA).
template <int NR, int V, bool REPLAY, bool FRESNEL>
__device__ __forceinline__ void ospr_row_body(const OsprArgs& a, int row0, int slot) {
    constexpr int R = RowCfg<NR, V>::R, T = NR / R;
    extern __shared__ float2 sm[];
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int lane = threadIdx.x & 31;
    const int r = row0 + line;
    bool single;
    const int s0 = slot_subframe(a, slot, single);
    const size_t P = size_t(a.H) * NR;
    float2* z = a.zbuf + size_t(slot) * P + size_t(r) * NR;
    pdl_wait();
    float2 v[R];
#pragma unroll
    for (int e = 0; e < R; ++e) v[e] = z[t + T * e];
    row_line_fft<NR, V, +1>(v, sm, line, t, a);

    float2 qy = make_float2(1.f, 0.f);
    if constexpr (FRESNEL) qy = __ldg(a.chirp_y + r);
    const size_t words = P / 32;
#pragma unroll
    for (int e = 0; e < R; ++e) {
        float2 q = make_float2(1.f, 0.f);
        if constexpr (FRESNEL) {
            q = cmul(qy, __ldg(a.chirp_x + t + T * e));
            v[e].x = fmaf(v[e].x, q.x, v[e].y * q.y);   // Re(IDFT(E) * conj(Q))
        }
        const bool n0 = v[e].x < 0.f;
        const bool n1 = v[e].y < 0.f;
        if (a.bits) {
            const unsigned b0 = __ballot_sync(0xffffffffu, n0);
            const unsigned b1 = __ballot_sync(0xffffffffu, n1);
            if (lane == 0) {
                const size_t w = (size_t(r) * NR + size_t(t - lane + T * e)) >> 5;
                a.bits[size_t(s0) * words + w] = b0;
                if (!single) a.bits[size_t(s0 + 1) * words + w] = b1;
            }
        }
        if constexpr (FRESNEL) v[e] = n0 ? make_float2(-q.x, -q.y) : q;   // h * Q
        else v[e] = make_float2(n0 ? -1.f : 1.f, single ? 0.f : (n1 ? -1.f : 1.f));
    }
    if constexpr (REPLAY) {
        row_line_fft<NR, V, -1>(v, sm, line, t, a);
        pdl_trigger();
#pragma unroll
        for (int e = 0; e < R; ++e) z[t + T * e] = v[e];
    }
}

template <int NR, int V, bool REPLAY, bool FRESNEL = false>
__global__ void __launch_bounds__((NR / RowCfg<NR, V>::R) * RowCfg<NR, V>::LPR)
k_ospr_row(OsprArgs a) {
    ospr_row_body<NR, V, REPLAY, FRESNEL>(a, int(blockIdx.x) * RowCfg<NR, V>::LPR, int(blockIdx.y));
}


// ------------------------------------------------------------------ pass 3 ----
// Pass 3 on column tile `tile` for accumulator group g (pairs g, g + groups, ...).
// `before_pair(j)` runs (uniformly over the CTA) before pair j is read and `after_read(j)`
// once its field is in registers: the standalone kernel passes no-ops, the persistent
// batch kernel waits for the pair's row pass and reports that its field may be reused.
struct NoHook {
    __device__ __forceinline__ void operator()(int) const {}
};
template <int NC, int V, class Before = NoHook, class After = NoHook>
__device__ __forceinline__ void ospr_col_fft_body(const OsprArgs& a, int tile, int g, Before before_pair = {},
                                                  After after_read = {}) {
    constexpr int R = ColCfg<NC, V>::R, LPC = ColCfg<NC, V>::LPC, T = NC / R;
    extern __shared__ float2 sm[];
    float2* lines = sm;
    const int lc = threadIdx.x % LPC, t = threadIdx.x / LPC;
    const int W = a.W;
    const int c = tile * LPC + lc;
    const size_t P = size_t(NC) * W;
    pdl_wait();
    float acc[R];
#pragma unroll
    for (int e = 0; e < R; ++e) acc[e] = 0.f;
    for (int j = g; j < a.pairs; j += a.groups) {
        before_pair(j);
        const float2* z = a.zbuf + size_t(j) * P;
        float2 v[R];
#pragma unroll
        for (int e = 0; e < R; ++e) v[e] = z[size_t(t + T * e) * W + c];
        after_read(j);
        col_line_fft<NC, V, -1>(v, lines, lc, t, a);
#pragma unroll
        for (int e = 0; e < R; ++e) acc[e] = fmaf(v[e].x, v[e].x, fmaf(v[e].y, v[e].y, acc[e]));
    }
    pdl_trigger();
    float* S = a.sacc + size_t(g) * P;
#pragma unroll
    for (int e = 0; e < R; ++e) {
        const size_t i = size_t(t + T * e) * W + c;
        S[i] = a.accumulate ? S[i] + acc[e] : acc[e];
    }
}

// (256-thread tiles are held to 128 registers, two CTAs per SM)
template <int NC, int V>
__global__ void __launch_bounds__((NC / ColCfg<NC, V>::R) * ColCfg<NC, V>::LPC,
                                  (NC / ColCfg<NC, V>::R) * ColCfg<NC, V>::LPC <= 256 ? 2 : 1)
k_ospr_col_fft(OsprArgs a) {
    ospr_col_fft_body<NC, V>(a, int(blockIdx.x), int(blockIdx.y));
}


// ------------------------------------------------------------------ finalize ----
// I(k) = I(-k) = (sum_g S_g(k) + S_g(-k)) * scale for the pixel pair of thread index p:
// p runs over the first half of the raster (rows 0 .. H/2), and the pair is written by the
// index of the two that comes first
__device__ __forceinline__ void ospr_finalize_pixel(const float* __restrict__ S, int groups, int H, int W,
                                                    float scale, float* __restrict__ I, size_t p) {
    const size_t P = size_t(H) * W;
    const size_t half = P / 2 + W;             // rows 0 .. H/2 inclusive
    if (p >= half) return;
    const int r = int(p / W), c = int(p % W);
    const size_t pm = size_t((H - r) & (H - 1)) * W + size_t((W - c) & (W - 1));
    if (pm < p) return;                        // the pair was taken by its partner
    float s = 0.f;
    for (int g = 0; g < groups; ++g) s += S[size_t(g) * P + p] + S[size_t(g) * P + pm];
    s *= scale;
    I[p] = s;
    I[pm] = s;
}

// pass launchers (ospr_col.cu, ospr_row.cu); `v` selects the tile variant
int ospr_run_col_ifft(const OsprArgs& a, int v, cudaStream_t st);
int ospr_run_col_fft(const OsprArgs& a, int v, cudaStream_t st);
int ospr_run_row(const OsprArgs& a, int v, bool replay, cudaStream_t st);
// tensor-core precisions (ospr_tc.cu, tcgen05): lengths 1024 and 2048, fixed tiles
int ospr_run_col_ifft_tc(const OsprArgs& a, int prec, cudaStream_t st);
int ospr_run_col_fft_tc(const OsprArgs& a, int prec, cudaStream_t st);
int ospr_run_row_tc(const OsprArgs& a, int prec, bool replay, cudaStream_t st);

}  // namespace holo
