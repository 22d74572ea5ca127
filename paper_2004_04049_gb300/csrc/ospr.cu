// ospr.cu - binary-phase One-Step Phase-Retrieval (paper Sections 2, 3, 5.2, 6).
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
#include <cmath>
#include <cstdlib>
#include <mutex>

#include "fft_core.cuh"
#include "phase_source.cuh"
#include "runtime.h"

namespace holo {

// launch shapes per line length: column passes hold LPC columns of R-element threads
template <int N> struct ColCfg;
template <> struct ColCfg<64>   { static constexpr int R = 8,  LPC = 32; };
template <> struct ColCfg<128>  { static constexpr int R = 16, LPC = 32; };
template <> struct ColCfg<256>  { static constexpr int R = 16, LPC = 32; };
template <> struct ColCfg<512>  { static constexpr int R = 16, LPC = 16; };
template <> struct ColCfg<1024> { static constexpr int R = 32, LPC = 16; };
template <> struct ColCfg<2048> { static constexpr int R = 32, LPC = 8; };
template <> struct ColCfg<4096> { static constexpr int R = 32, LPC = 4; };
// row passes: T = N/R >= 32 threads per row so that a warp holds 32 consecutive pixels
template <int N> struct RowCfg;
template <> struct RowCfg<64>   { static constexpr int R = 2,  LPR = 4; };
template <> struct RowCfg<128>  { static constexpr int R = 4,  LPR = 4; };
template <> struct RowCfg<256>  { static constexpr int R = 8,  LPR = 4; };
template <> struct RowCfg<512>  { static constexpr int R = 16, LPR = 4; };
template <> struct RowCfg<1024> { static constexpr int R = 32, LPR = 4; };
template <> struct RowCfg<2048> { static constexpr int R = 32, LPR = 2; };
template <> struct RowCfg<4096> { static constexpr int R = 32, LPR = 1; };

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
};

template <int NC>
constexpr int col_stride() { return col_line_stride(NC, ColCfg<NC>::R, ColCfg<NC>::LPC); }
// pass 1 also holds the replicated cos/sin table
template <int NC>
constexpr size_t col_ifft_smem_bytes() {
    return sizeof(float2) * (kCsSmemEntries + size_t(ColCfg<NC>::LPC) * col_stride<NC>());
}
template <int NC>
constexpr size_t col_fft_smem_bytes() {
    return sizeof(float2) * size_t(ColCfg<NC>::LPC) * col_stride<NC>();
}
template <int NR>
constexpr size_t row_smem_bytes() {
    return sizeof(float2) * size_t(RowCfg<NR>::LPR) * line_stride(NR, RowCfg<NR>::R);
}

// ------------------------------------------------------------------ pass 1 ----
// Z for one column of one pair, in canonical layout (slot e <-> row t + T*e). MODE and
// SINGLE are compile-time so that the element loops hold no branches: for each batch of
// kBatch elements every load (target, mirror target, four codes) is issued before any
// of them is used.
constexpr int kBatch = 8;

template <int NC, int MODE, bool SINGLE>
__device__ __forceinline__ void ospr_build_column(float2 (&v)[ColCfg<NC>::R], const OsprArgs& a,
                                                  const float2* cs, int t, int c, int s0) {
    constexpr int R = ColCfg<NC>::R, T = NC / R;
    constexpr int B = R < kBatch ? R : kBatch;
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
#pragma unroll
    for (int e0 = 0; e0 < R; e0 += B) {
        float tp[B], tm[B];
        uint32_t pk[B];   // codes of (s0, p), (s0, -p), (s1, p), (s1, -p), one byte each
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int e = e0 + k;
            const int r = t + T * e;
            const int rm = (NC - r) & (NC - 1);
            tp[k] = __ldg(a.target + r * W + c);
            tm[k] = SINGLE ? 0.f : __ldg(a.target + rm * W + cm);
            if constexpr (MODE == kPhaseTable) {
                const uint32_t jm0 = (e == 0 && t == 0) ? z0 : m0;
                const uint32_t jm1 = (e == 0 && t == 0) ? z1 : m1;
                uint32_t w = __ldg(a.ps.codes + i0);
                if constexpr (!SINGLE) {
                    w |= uint32_t(__ldg(a.ps.codes + jm0)) << 8;
                    w |= uint32_t(__ldg(a.ps.codes + i1)) << 16;
                    w |= uint32_t(__ldg(a.ps.codes + jm1)) << 24;
                }
                pk[k] = w;
                i0 += D; i0 -= (i0 >= L) ? L : 0u;
                i1 += D; i1 -= (i1 >= L) ? L : 0u;
                m0 = (m0 >= D) ? m0 - D : m0 + (L - D);
                m1 = (m1 >= D) ? m1 - D : m1 + (L - D);
            } else if constexpr (MODE == kPhaseGenerator) {
                const uint64_t p = uint64_t(r) * uint64_t(W) + uint64_t(c);
                const uint64_t pm = uint64_t(rm) * uint64_t(W) + uint64_t(cm);
                uint32_t w = uint32_t(splitmix64_at(a.ps.seed, d0.base + p) >> gshift);
                if constexpr (!SINGLE) {
                    w |= uint32_t(splitmix64_at(a.ps.seed, d0.base + pm) >> gshift) << 8;
                    w |= uint32_t(splitmix64_at(a.ps.seed, d1.base + p) >> gshift) << 16;
                    w |= uint32_t(splitmix64_at(a.ps.seed, d1.base + pm) >> gshift) << 24;
                }
                pk[k] = w;
            } else {
                pk[k] = 0u;   // flat phase
            }
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const float2 c0 = cs_lookup(cs, (pk[k] & 0xffu) << sh);
            if constexpr (SINGLE) {
                v[e0 + k] = make_float2(tp[k] * c0.x, tp[k] * c0.y);
            } else {
                const float2 c0m = cs_lookup(cs, ((pk[k] >> 8) & 0xffu) << sh);
                const float2 c1 = cs_lookup(cs, ((pk[k] >> 16) & 0xffu) << sh);
                const float2 c1m = cs_lookup(cs, (pk[k] >> 24) << sh);
                // Hermitian parts E(k) + conj(E(-k)) of both sub-frames, packed as a + i b
                const float2 h0 = make_float2(fmaf(tp[k], c0.x, tm[k] * c0m.x), fmaf(tp[k], c0.y, -tm[k] * c0m.y));
                const float2 h1 = make_float2(fmaf(tp[k], c1.x, tm[k] * c1m.x), fmaf(tp[k], c1.y, -tm[k] * c1m.y));
                v[e0 + k] = make_float2(h0.x - h1.y, h0.y + h1.x);
            }
        }
    }
}

template <int NC>
__global__ void __launch_bounds__((NC / ColCfg<NC>::R) * ColCfg<NC>::LPC)
k_ospr_col_ifft(OsprArgs a) {
    constexpr int R = ColCfg<NC>::R, LPC = ColCfg<NC>::LPC, T = NC / R;
    extern __shared__ float2 sm[];
    float2* cs = sm;
    float2* lines = sm + kCsSmemEntries;
    load_cs_table(cs, a.cs256);
    __syncthreads();

    const int lc = threadIdx.x % LPC, t = threadIdx.x / LPC;
    const int W = a.W;
    const int c = blockIdx.x * LPC + lc;
    const int s0 = 2 * (a.first_pair + int(blockIdx.y));
    const bool single = s0 + 1 >= a.N;
    float2 v[R];
    if (a.ps.mode == kPhaseTable) {
        if (single) ospr_build_column<NC, kPhaseTable, true>(v, a, cs, t, c, s0);
        else ospr_build_column<NC, kPhaseTable, false>(v, a, cs, t, c, s0);
    } else if (a.ps.mode == kPhaseGenerator) {
        if (single) ospr_build_column<NC, kPhaseGenerator, true>(v, a, cs, t, c, s0);
        else ospr_build_column<NC, kPhaseGenerator, false>(v, a, cs, t, c, s0);
    } else {
        if (single) ospr_build_column<NC, kPhaseFlat, true>(v, a, cs, t, c, s0);
        else ospr_build_column<NC, kPhaseFlat, false>(v, a, cs, t, c, s0);
    }
    line_fft<NC, R, +1, true>(v, lines + lc * col_stride<NC>(), t, a.tw);
    float2* z = a.zbuf + size_t(blockIdx.y) * size_t(NC) * size_t(W);
#pragma unroll
    for (int e = 0; e < R; ++e) z[size_t(t + T * e) * W + c] = v[e];
}

// ------------------------------------------------------------------ pass 2 ----
template <int NR, bool REPLAY>
__global__ void __launch_bounds__((NR / RowCfg<NR>::R) * RowCfg<NR>::LPR)
k_ospr_row(OsprArgs a) {
    constexpr int R = RowCfg<NR>::R, T = NR / R;
    constexpr bool BLOCK = T > 32;
    extern __shared__ float2 sm[];
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * RowCfg<NR>::LPR + line;
    const int s0 = 2 * (a.first_pair + int(blockIdx.y));
    const bool single = s0 + 1 >= a.N;
    const size_t P = size_t(a.H) * NR;
    float2* z = a.zbuf + size_t(blockIdx.y) * P + size_t(r) * NR;
    float2* buf = sm + line * line_stride(NR, R);

    float2 v[R];
#pragma unroll
    for (int e = 0; e < R; ++e) v[e] = z[t + T * e];
    line_fft<NR, R, +1, BLOCK>(v, buf, t, a.tw);

    const size_t words = P / 32;
#pragma unroll
    for (int e = 0; e < R; ++e) {
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
        v[e] = make_float2(n0 ? -1.f : 1.f, single ? 0.f : (n1 ? -1.f : 1.f));
    }
    if constexpr (REPLAY) {
        line_fft<NR, R, -1, BLOCK>(v, buf, t, a.tw);
#pragma unroll
        for (int e = 0; e < R; ++e) z[t + T * e] = v[e];
    }
}

// ------------------------------------------------------------------ pass 3 ----
template <int NC>
__global__ void __launch_bounds__((NC / ColCfg<NC>::R) * ColCfg<NC>::LPC)
k_ospr_col_fft(OsprArgs a) {
    constexpr int R = ColCfg<NC>::R, LPC = ColCfg<NC>::LPC, T = NC / R;
    extern __shared__ float2 sm[];
    float2* lines = sm;
    const int lc = threadIdx.x % LPC, t = threadIdx.x / LPC;
    const int W = a.W;
    const int c = blockIdx.x * LPC + lc;
    const size_t P = size_t(NC) * W;
    float acc[R];
#pragma unroll
    for (int e = 0; e < R; ++e) acc[e] = 0.f;
    for (int j = blockIdx.y; j < a.pairs; j += a.groups) {
        const float2* z = a.zbuf + size_t(j) * P;
        float2 v[R];
#pragma unroll
        for (int e = 0; e < R; ++e) v[e] = z[size_t(t + T * e) * W + c];
        line_fft<NC, R, -1, true>(v, lines + lc * col_stride<NC>(), t, a.tw);
#pragma unroll
        for (int e = 0; e < R; ++e) acc[e] = fmaf(v[e].x, v[e].x, fmaf(v[e].y, v[e].y, acc[e]));
    }
    float* S = a.sacc + size_t(blockIdx.y) * P;
#pragma unroll
    for (int e = 0; e < R; ++e) {
        const size_t i = size_t(t + T * e) * W + c;
        S[i] = a.accumulate ? S[i] + acc[e] : acc[e];
    }
}

// ---------------------------------------------------------------- finalize ----
// I(k) = I(-k) = (sum_g S_g(k) + S_g(-k)) * scale: one thread per pixel pair {k, -k}
// reads both accumulators once and writes both outputs. Thread q handles pixel q of the
// first half of the raster (rows 0 .. H/2) whose mirror lies at or after it.
__global__ void k_ospr_finalize(const float* __restrict__ S, int groups, int H, int W,
                                float scale, float* __restrict__ I) {
    const size_t P = size_t(H) * W;
    const size_t half = P / 2 + W;             // rows 0 .. H/2 inclusive
    const size_t p = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
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

// ------------------------------------------------------------------- host ----
template <int NC>
static int launch_col_ifft(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = col_ifft_smem_bytes<NC>();
    int rc = ensure_smem((const void*)k_ospr_col_ifft<NC>, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.W / ColCfg<NC>::LPC, a.pairs);
    Launch ln("ospr_col_ifft", st);
    k_ospr_col_ifft<NC><<<grid, (NC / ColCfg<NC>::R) * ColCfg<NC>::LPC, smem, st>>>(a);
    return ln.done("ospr_col_ifft launch");
}

template <int NR, bool REPLAY>
static int launch_row(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = row_smem_bytes<NR>();
    int rc = ensure_smem((const void*)k_ospr_row<NR, REPLAY>, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.H / RowCfg<NR>::LPR, a.pairs);
    Launch ln("ospr_row", st);
    k_ospr_row<NR, REPLAY><<<grid, (NR / RowCfg<NR>::R) * RowCfg<NR>::LPR, smem, st>>>(a);
    return ln.done("ospr_row launch");
}

template <int NC>
static int launch_col_fft(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = col_fft_smem_bytes<NC>();
    int rc = ensure_smem((const void*)k_ospr_col_fft<NC>, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.W / ColCfg<NC>::LPC, a.groups);
    Launch ln("ospr_col_fft", st);
    k_ospr_col_fft<NC><<<grid, (NC / ColCfg<NC>::R) * ColCfg<NC>::LPC, smem, st>>>(a);
    return ln.done("ospr_col_fft launch");
}

#define HOLO_LEN_SWITCH(n, CALL)                          \
    switch (n) {                                          \
        case 64: return CALL(64);                         \
        case 128: return CALL(128);                       \
        case 256: return CALL(256);                       \
        case 512: return CALL(512);                       \
        case 1024: return CALL(1024);                     \
        case 2048: return CALL(2048);                     \
        case 4096: return CALL(4096);                     \
        default: return fail(HOLO_EUNSUPPORTED, "line length %d", n); \
    }

static int run_col_ifft(const OsprArgs& a, cudaStream_t st) {
#define C(n) launch_col_ifft<n>(a, st)
    HOLO_LEN_SWITCH(a.H, C)
#undef C
}
static int run_row(const OsprArgs& a, bool replay, cudaStream_t st) {
#define C(n) (replay ? launch_row<n, true>(a, st) : launch_row<n, false>(a, st))
    HOLO_LEN_SWITCH(a.W, C)
#undef C
}
static int run_col_fft(const OsprArgs& a, cudaStream_t st) {
#define C(n) launch_col_fft<n>(a, st)
    HOLO_LEN_SWITCH(a.H, C)
#undef C
}

struct OsprPlan {
    int npairs, chunk, groups;
    size_t z_bytes, s_bytes, total;
};

// Tuning override: HOLO_OSPR_CHUNK (pairs in flight, 1..16) and HOLO_OSPR_GROUPS
// (partial accumulators, 1..4) replace the defaults; read once per process.
static int env_int(const char* name, int lo, int hi, int dflt) {
    const char* v = getenv(name);
    if (!v || !*v) return dflt;
    const int x = atoi(v);
    return x < lo ? lo : (x > hi ? hi : x);
}
static int tuned_chunk() {
    static const int v = env_int("HOLO_OSPR_CHUNK", 1, kMaxChunkPairs, kMaxChunkPairs);
    return v;
}
static int tuned_groups() {
    static const int v = env_int("HOLO_OSPR_GROUPS", 1, kMaxGroups, kMaxGroups);
    return v;
}

static OsprPlan ospr_plan(int H, int W, int N) {
    OsprPlan pl;
    const size_t P = size_t(H) * W;
    pl.npairs = (N + 1) / 2;
    const int cmax = tuned_chunk();
    pl.chunk = pl.npairs < cmax ? pl.npairs : cmax;
    const int gmax = tuned_groups();
    pl.groups = pl.chunk < gmax ? pl.chunk : gmax;
    pl.z_bytes = align_up(size_t(pl.chunk) * P * sizeof(float2), 256);
    pl.s_bytes = align_up(size_t(pl.groups) * P * sizeof(float), 256);
    pl.total = pl.z_bytes + pl.s_bytes;
    return pl;
}

static bool is_prime(int64_t n) {
    if (n < 2) return false;
    for (int64_t d = 2; d * d <= n; ++d)
        if (n % d == 0) return false;
    return true;
}

static int check_shape(const char* who, int H, int W) {
    if (!is_pow2(H) || !is_pow2(W) || H < kMinDim || W < kMinDim || H > kMaxDim || W > kMaxDim)
        return fail(HOLO_EUNSUPPORTED, "%s: H=%d W=%d must be powers of two in [%d, %d]", who, H, W,
                    kMinDim, kMaxDim);
    return HOLO_OK;
}

}  // namespace holo

using namespace holo;

extern "C" int ospr_workspace_size(int H, int W, int N, int precision, size_t* bytes) {
    clear_error();
    if (!bytes) return fail(HOLO_EINVAL, "ospr_workspace_size: NULL output");
    int rc = check_shape("ospr_workspace_size", H, W);
    if (rc) return rc;
    if (N < 1 || N > 4096) return fail(HOLO_EINVAL, "ospr_workspace_size: N=%d out of [1, 4096]", N);
    if (precision != HOLO_FP32) return fail(HOLO_EUNSUPPORTED, "ospr_workspace_size: precision %d", precision);
    *bytes = ospr_plan(H, W, N).total;
    return HOLO_OK;
}

extern "C" int ospr_generate(const float* d_target, int H, int W, int N,
                             const uint8_t* d_codes, int64_t L, int levels, uint64_t seed,
                             int64_t start_index, int64_t subframe_stride, int precision,
                             uint32_t* d_holo_bits, float* d_replay,
                             void* d_ws, size_t ws_bytes, holo_stream_t s) {
    clear_error();
    const char* who = "ospr_generate";
    int rc = check_shape(who, H, W);
    if (rc) return rc;
    if (N < 1 || N > 4096) return fail(HOLO_EINVAL, "%s: N=%d out of [1, 4096]", who, N);
    if (precision != HOLO_FP32) return fail(HOLO_EUNSUPPORTED, "%s: precision %d is not built", who, precision);
    if (!d_target) return fail(HOLO_EINVAL, "%s: d_target is NULL", who);
    if (!d_holo_bits && !d_replay) return fail(HOLO_EINVAL, "%s: both outputs are NULL", who);
    const int64_t P = int64_t(H) * W;
    const int64_t stride = subframe_stride == 0 ? P : subframe_stride;
    if (stride > (INT64_C(1) << 40) || start_index > (INT64_C(1) << 61))
        return fail(HOLO_EINVAL, "%s: start or stride too large", who);
    PhaseSource ps;
    rc = make_phase_source(who, d_codes, L, levels, seed, start_index, stride, &ps);
    if (rc) return rc;
    const OsprPlan pl = ospr_plan(H, W, N);
    if (!d_ws || ws_bytes < pl.total)
        return fail(HOLO_EWORKSPACE, "%s: workspace %zu bytes, need %zu", who, ws_bytes, pl.total);
    if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0)
        return fail(HOLO_EWORKSPACE, "%s: workspace is not 256-byte aligned", who);
    Tables tab;
    rc = device_tables(&tab);
    if (rc) return rc;

    OsprArgs a;
    a.target = d_target;
    a.H = H;
    a.W = W;
    a.N = N;
    a.ps = ps;
    a.zbuf = static_cast<float2*>(d_ws);
    a.sacc = reinterpret_cast<float*>(static_cast<char*>(d_ws) + pl.z_bytes);
    a.groups = pl.groups;
    a.bits = d_holo_bits;
    a.tw = tab.twiddles;
    a.cs256 = tab.cs256;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    const bool replay = d_replay != nullptr;
    for (int first = 0; first < pl.npairs; first += pl.chunk) {
        a.first_pair = first;
        a.pairs = pl.npairs - first < pl.chunk ? pl.npairs - first : pl.chunk;
        a.accumulate = first > 0;
        if ((rc = run_col_ifft(a, st))) return rc;
        if ((rc = run_row(a, replay, st))) return rc;
        if (replay && (rc = run_col_fft(a, st))) return rc;
    }
    if (replay) {
        const float scale = float(1.0 / (2.0 * double(N) * double(P)));
        const int threads = 256;
        const int blocks = int((P / 2 + W + threads - 1) / threads);
        Launch ln("ospr_finalize", st);
        k_ospr_finalize<<<blocks, threads, 0, st>>>(a.sacc, pl.groups, H, W, scale, d_replay);
        if ((rc = ln.done("ospr_finalize launch"))) return rc;
    }
    // Section 8 design rules: warnings only
    if (L > 0) {
        if (!is_prime(L)) warn("design rule: L=%lld is not prime", (long long)L);
        if (L <= N) warn("design rule: L=%lld is not greater than N=%d", (long long)L, N);
        if (L <= (H > W ? H : W)) warn("design rule: L=%lld is not greater than max(H, W)", (long long)L);
    }
    return HOLO_OK;
}

// ================================================= fixed-scratch variant ====
// ospr_generate_noalloc: the same computation as ospr_generate for callers that cannot
// allocate device memory. Its scratch is one file-scope device array of a fixed size,
// shared by every call in the process; host code reaches it only through the address
// cudaGetSymbolAddress returns for the current device.
namespace holo {

static __device__ __align__(256) unsigned char g_ospr_noalloc_scratch[HOLO_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64];

// Device address of the scratch array on the current device, looked up once per device.
static int noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "ospr_generate_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(HOLO_EUNSUPPORTED, "ospr_generate_noalloc: device %d", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_ospr_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "ospr_generate_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return HOLO_OK;
}

// One partial accumulator and as many sub-frame pairs per chunk as the scratch holds.
static bool noalloc_plan(int H, int W, int N, OsprPlan* pl) {
    const size_t P = size_t(H) * W;
    pl->npairs = (N + 1) / 2;
    pl->groups = 1;
    pl->s_bytes = align_up(P * sizeof(float), 256);
    if (pl->s_bytes >= size_t(HOLO_NOALLOC_SCRATCH_BYTES)) return false;
    const size_t fit = (size_t(HOLO_NOALLOC_SCRATCH_BYTES) - pl->s_bytes) / align_up(P * sizeof(float2), 256);
    if (fit < 1) return false;
    int chunk = pl->npairs < kMaxChunkPairs ? pl->npairs : kMaxChunkPairs;
    if (size_t(chunk) > fit) chunk = int(fit);
    pl->chunk = chunk;
    pl->z_bytes = align_up(size_t(chunk) * P * sizeof(float2), 256);
    pl->total = pl->z_bytes + pl->s_bytes;
    return pl->total <= size_t(HOLO_NOALLOC_SCRATCH_BYTES);
}

}  // namespace holo

extern "C" int ospr_generate_noalloc(const float* d_target, int H, int W, int N,
                                     const uint8_t* d_codes, int64_t L, int levels, uint64_t seed,
                                     int64_t start_index, int64_t subframe_stride, int precision,
                                     uint32_t* d_holo_bits, float* d_replay, holo_stream_t s) {
    clear_error();
    const char* who = "ospr_generate_noalloc";
    int rc = check_shape(who, H, W);
    if (rc) return rc;
    if (N < 1 || N > 4096) return fail(HOLO_EINVAL, "%s: N=%d out of [1, 4096]", who, N);
    if (precision != HOLO_FP32) return fail(HOLO_EUNSUPPORTED, "%s: precision %d is not built", who, precision);
    if (!d_target) return fail(HOLO_EINVAL, "%s: d_target is NULL", who);
    if (!d_holo_bits && !d_replay) return fail(HOLO_EINVAL, "%s: both outputs are NULL", who);
    OsprPlan pl;
    if (!noalloc_plan(H, W, N, &pl))
        return fail(HOLO_EWORKSPACE,
                    "%s: H=%d W=%d needs more than the fixed %u-byte scratch (one complex64 "
                    "and one float32 H*W field); use ospr_generate with a workspace", who, H, W,
                    unsigned(HOLO_NOALLOC_SCRATCH_BYTES));
    const int64_t P = int64_t(H) * W;
    const int64_t stride = subframe_stride == 0 ? P : subframe_stride;
    if (stride > (INT64_C(1) << 40) || start_index > (INT64_C(1) << 61))
        return fail(HOLO_EINVAL, "%s: start or stride too large", who);
    PhaseSource ps;
    rc = make_phase_source(who, d_codes, L, levels, seed, start_index, stride, &ps);
    if (rc) return rc;
    void* scratch = nullptr;
    if ((rc = noalloc_scratch(&scratch))) return rc;
    Tables tab;
    if ((rc = device_tables(&tab))) return rc;

    OsprArgs a;
    a.target = d_target;
    a.H = H;
    a.W = W;
    a.N = N;
    a.ps = ps;
    a.zbuf = static_cast<float2*>(scratch);
    a.sacc = reinterpret_cast<float*>(static_cast<char*>(scratch) + pl.z_bytes);
    a.groups = pl.groups;
    a.bits = d_holo_bits;
    a.tw = tab.twiddles;
    a.cs256 = tab.cs256;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    const bool replay = d_replay != nullptr;
    // every scratch byte a kernel reads was written earlier in this call (the first chunk
    // overwrites the accumulator), so nothing needs clearing between calls
    for (int first = 0; first < pl.npairs; first += pl.chunk) {
        a.first_pair = first;
        a.pairs = pl.npairs - first < pl.chunk ? pl.npairs - first : pl.chunk;
        a.accumulate = first > 0;
        if ((rc = run_col_ifft(a, st))) return rc;
        if ((rc = run_row(a, replay, st))) return rc;
        if (replay && (rc = run_col_fft(a, st))) return rc;
    }
    if (replay) {
        const float scale = float(1.0 / (2.0 * double(N) * double(P)));
        const int threads = 256;
        const int blocks = int((P / 2 + W + threads - 1) / threads);
        Launch ln("ospr_finalize", st);
        k_ospr_finalize<<<blocks, threads, 0, st>>>(a.sacc, pl.groups, H, W, scale, d_replay);
        if ((rc = ln.done("ospr_finalize launch"))) return rc;
    }
    return HOLO_OK;
}
