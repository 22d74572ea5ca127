// phase_source.cuh - the draw rule of the phase LUT (paper Section 5, Fig. 3): sub-frame s
// of a frame takes draw indices start + s*stride + p, and draw i reads table entry i mod L
// (or, with no table, the generator's output i; or nothing at all for flat phase).
#pragma once

#include "fft_core.cuh"
#include "runtime.h"

namespace holo {

enum PhaseMode : int { kPhaseFlat = 0, kPhaseTable = 1, kPhaseGenerator = 2 };

struct PhaseSource {
    const uint8_t* codes;  // [L] table (kPhaseTable)
    uint64_t start;        // draw index of pixel 0 of sub-frame 0
    uint64_t stride;       // draw-index step between sub-frames
    uint64_t seed;         // generator stream (kPhaseGenerator)
    uint64_t fm;           // fastmod constant of L
    uint32_t L;            // table length
    int mode;              // PhaseMode
    int bits;              // code bits, log2(levels)
    int cs_shift;          // 8 - bits: code -> index into the 256-entry cos/sin table
};

// table entry k: the top `bits` bits of SplitMix64 output k of stream `seed` (Section 4:
// a pool of random phases generated once; 8-bit entries per Section 5.2)
__device__ __forceinline__ uint8_t lut_entry(uint64_t seed, uint64_t k, int bits) {
    return uint8_t(splitmix64_at(seed, k) >> (64 - bits));
}

struct SubframeDraw {
    uint64_t base;   // start + s*stride
    uint32_t base_mod;  // (start + s*stride) mod L (table mode)
};

__device__ __forceinline__ SubframeDraw subframe_draw(const PhaseSource& ps, int s) {
    SubframeDraw d;
    d.base = ps.start + uint64_t(s) * ps.stride;
    d.base_mod = ps.mode == kPhaseTable ? uint32_t(d.base % uint64_t(ps.L)) : 0u;
    return d;
}

// code of draw base + p; p < 2^24 and base_mod < 2^31 keep the table index sum in 32 bits
__device__ __forceinline__ uint32_t draw_code(const PhaseSource& ps, const SubframeDraw& d, uint32_t p) {
    if (ps.mode == kPhaseTable) return ps.codes[fastmod_u32(d.base_mod + p, ps.fm, ps.L)];
    if (ps.mode == kPhaseGenerator) return uint32_t(splitmix64_at(ps.seed, d.base + p) >> (64 - ps.bits));
    return 0u;
}

// Fresnel propagation's separable quadratic phase Q(y, x) = chirp[y] * chirp[H + x] with
// chirp[i] = exp(i*pi*kappa*(i - n/2)^2), n = H for the first H entries and W for the W
// after them; written on the stream (ospr.cu).
int fresnel_chirp_build(int H, int W, double kappa, float2* d_chirp, cudaStream_t st);

// Host: validates the table arguments of a call and fills a PhaseSource.
inline int make_phase_source(const char* who, const uint8_t* d_codes, int64_t L, int levels,
                             uint64_t seed, int64_t start, int64_t stride, PhaseSource* ps) {
    if (!is_pow2(levels) || levels < 2 || levels > 256)
        return fail(HOLO_EINVAL, "%s: levels=%d is not a power of two in [2, 256]", who, levels);
    if (L < HOLO_L_UNREPEATED || L > INT64_C(0x7FFFFFFF))
        return fail(HOLO_EINVAL, "%s: L=%lld out of range", who, (long long)L);
    if (L > 0 && !d_codes) return fail(HOLO_EINVAL, "%s: d_codes is NULL with L=%lld", who, (long long)L);
    if (start < 0 || stride < 0) return fail(HOLO_EINVAL, "%s: negative start or stride", who);
    ps->codes = d_codes;
    ps->start = uint64_t(start);
    ps->stride = uint64_t(stride);
    ps->seed = seed;
    ps->L = L > 0 ? uint32_t(L) : 1u;
    ps->fm = ~uint64_t(0) / uint64_t(ps->L) + 1;
    ps->mode = L > 0 ? kPhaseTable : (L == 0 ? kPhaseFlat : kPhaseGenerator);
    ps->bits = log2i(levels);
    ps->cs_shift = 8 - ps->bits;
    return HOLO_OK;
}

}  // namespace holo
