// gs.cu - Gerchberg-Saxton with a phase-quantised hologram (paper Section 2; random
// initial phase of Section 3 drawn from the LUT; Section 8's GS design rules).
//
// Replay-plane field E, target scaled to the hologram's energy T_s = T*sqrt(P/sum T^2).
// Iteration: H = IDFT(E); q = quantise(arg H); h = exp(2 pi i q/levels); R = DFT(h);
// eps = sum (|R| - T_s)^2; E = T_s exp(i arg R).
//
// Passes (one global round trip of the complex field each; the field stays resident):
//   prepare    sum T^2 -> scale (float-float block partials, ffloat.cuh)
//   col_init   columns: E_0 from the LUT / a phase / a saved state, column IDFT
//   row        rows: row IDFT, quantise (codes out on the last iteration), row DFT
//   col        columns: column DFT, error partials, amplitude constraint, column IDFT
//              (the next iteration's first half); on the last iteration it writes
//              |R|^2 and the state instead of transforming back
//   finish     per-iteration error sums (float-float, converted to float64 once)
// A batch of B targets of one shape runs through the same launches: blockIdx.y is the
// target, every buffer holds B fields of H*W (gs_iterate is the batch of one).
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>

#include "ffloat.cuh"
#include "fft_core.cuh"
#include "phase_source.cuh"
#include "runtime.h"
#include "tc05_dft.cuh"

namespace holo {

// column passes: small column tiles so that a single field fills the GPU. Lengths 512 to
// 2048 have two more tile variants (fewer values per thread, or fewer lines per CTA),
// chosen per shape with gs_tuning_set; the defaults are the fastest measured on GB300.
template <int N, int V> struct GsColCfg;
template <> struct GsColCfg<64, 0>   { static constexpr int R = 8,  LPC = 8; };
template <> struct GsColCfg<128, 0>  { static constexpr int R = 16, LPC = 8; };
template <> struct GsColCfg<256, 0>  { static constexpr int R = 16, LPC = 8; };
template <> struct GsColCfg<512, 0>  { static constexpr int R = 16, LPC = 4; };
template <> struct GsColCfg<1024, 0> { static constexpr int R = 16, LPC = 4; };
template <> struct GsColCfg<2048, 0> { static constexpr int R = 32, LPC = 4; };
template <> struct GsColCfg<4096, 0> { static constexpr int R = 32, LPC = 2; };
template <> struct GsColCfg<512, 1>  { static constexpr int R = 8,  LPC = 4; };
template <> struct GsColCfg<1024, 1> { static constexpr int R = 8,  LPC = 4; };
template <> struct GsColCfg<2048, 1> { static constexpr int R = 16, LPC = 4; };
template <> struct GsColCfg<512, 2>  { static constexpr int R = 16, LPC = 2; };
template <> struct GsColCfg<1024, 2> { static constexpr int R = 16, LPC = 2; };
template <> struct GsColCfg<2048, 2> { static constexpr int R = 32, LPC = 2; };
template <int N, int V> struct GsRowCfg;
template <> struct GsRowCfg<64, 0>   { static constexpr int R = 2,  LPR = 4; };
template <> struct GsRowCfg<128, 0>  { static constexpr int R = 4,  LPR = 4; };
template <> struct GsRowCfg<256, 0>  { static constexpr int R = 8,  LPR = 4; };
template <> struct GsRowCfg<512, 0>  { static constexpr int R = 16, LPR = 4; };
template <> struct GsRowCfg<1024, 0> { static constexpr int R = 32, LPR = 4; };
template <> struct GsRowCfg<2048, 0> { static constexpr int R = 32, LPR = 2; };
template <> struct GsRowCfg<4096, 0> { static constexpr int R = 32, LPR = 1; };
template <> struct GsRowCfg<512, 1>  { static constexpr int R = 8,  LPR = 4; };
template <> struct GsRowCfg<1024, 1> { static constexpr int R = 16, LPR = 2; };
template <> struct GsRowCfg<2048, 1> { static constexpr int R = 16, LPR = 1; };
template <> struct GsRowCfg<512, 2>  { static constexpr int R = 16, LPR = 2; };
template <> struct GsRowCfg<1024, 2> { static constexpr int R = 8,  LPR = 2; };
template <> struct GsRowCfg<2048, 2> { static constexpr int R = 16, LPR = 2; };
constexpr bool gs_has_variants(int N) { return N >= 512 && N <= 2048; }
constexpr int kGsMinLpc = 2;   // the smallest LPC of any variant (bounds the error partials)

constexpr int kGsPrepThreads = 256;
constexpr int kGsPrepBlocks = 152;

struct GsScalars {
    float scale;        // sqrt(P / sum T^2), written by k_gs_col_init
    float pad[63];
};

struct GsArgs {
    const float* target;
    int H, W, levels_bits;
    PhaseSource ps;              // initial phase from the LUT
    const float* init_phase;     // or a caller phase
    const float2* state_in;      // or a saved field
    float2* y;                   // [H][W] complex work field
    GsScalars* sc;
    const ff* prep_part;         // [kGsPrepBlocks] partial sums of T^2
    ff* err_part;                // [targets][iters][col blocks] partial error sums
    int iter, iters;
    int batch;                   // targets (grid.y of every launch)
    uint8_t* codes_out;
    float* replay_out;
    float2* state_out;
    const float2* tw;
    const float2* cs256;
    const uint8_t* tc05b;        // tcgen05 DFT-32 matrices of the tensor-core precision in use
    float inv_sqrt_p;
    // Fresnel propagation: Q(y, x) = chirp_y[y] * chirp_x[x] (null for the far field)
    const float2* chirp_y;
    const float2* chirp_x;
};

template <int NC, int V>
constexpr int gs_col_stride() { return col_line_stride(NC, GsColCfg<NC, V>::R, GsColCfg<NC, V>::LPC); }
// col_init and row also hold one copy of the cos/sin table (one lookup per pixel)
template <int NC, int V>
constexpr size_t gs_col_smem() {
    return sizeof(float2) * (256 + size_t(GsColCfg<NC, V>::LPC) * gs_col_stride<NC, V>());
}
// The row pass looks up one quantised code per pixel in a 4-way replicated table (8 KiB;
// lane l reads copy l mod 4, so a half-warp's 16 lookups meet about two-way bank conflicts).
// Every 128-thread CTA loads the table for its two rows: 16 copies (32 KiB, conflict-free)
// cost more in loads than they saved (1024^2 row pass 14.4 against 12.4 us; 8 targets of
// 1024^2 62.9 k against 69.2 k iterations/s).
constexpr int kGsRowCopies = 4;
template <int NR, int V>
constexpr size_t gs_row_smem() {
    return sizeof(float2) * (cs_smem_entries<kGsRowCopies>() + size_t(GsRowCfg<NR, V>::LPR) * line_stride(NR, GsRowCfg<NR, V>::R));
}

// Line FFT of a GS column pass (LPC lines of T threads, lane-consecutive columns)
template <int NC, int V, int DIR>
__device__ __forceinline__ void gs_col_line_fft(float2 (&v)[GsColCfg<NC, V>::R], float2* lines, int lc, int t,
                                                const GsArgs& a) {
    constexpr int R = GsColCfg<NC, V>::R, S = gs_col_stride<NC, V>();
    line_fft<NC, R, DIR, true>(v, lines + lc * S, t, a.tw);
}
// Line FFT of the GS row pass: line `line` of LPR, T threads per line
template <int NR, int V, int DIR>
__device__ __forceinline__ void gs_row_line_fft(float2 (&v)[GsRowCfg<NR, V>::R], float2* lines, int line, int t,
                                                const GsArgs& a) {
    constexpr int R = GsRowCfg<NR, V>::R, T = NR / R, S = line_stride(NR, R);
    line_fft<NR, R, DIR, (T > 32)>(v, lines + line * S, t, a.tw);
}

// The arguments of target b of a batch: every per-target buffer advances by b fields;
// the initial phases continue the table draw (target b = sub-frame b of the draw rule)
__device__ __forceinline__ GsArgs gs_target(const GsArgs& a0, int b) {
    GsArgs a = a0;
    const size_t P = size_t(a.H) * a.W;
    const size_t off = size_t(b) * P;
    a.target += off;
    if (a.init_phase) a.init_phase += off;
    if (a.state_in) a.state_in += off;
    a.y += off;
    a.sc += b;
    a.prep_part += size_t(b) * kGsPrepBlocks;
    if (a.codes_out) a.codes_out += off;
    if (a.replay_out) a.replay_out += off;
    if (a.state_out) a.state_out += off;
    return a;
}

// ----------------------------------------------------------------- prepare ----
// per-block float-float partials of sum T^2
__global__ void __launch_bounds__(kGsPrepThreads)
k_gs_prepare(const float* __restrict__ T, int64_t P, ff* __restrict__ partials) {
    __shared__ ff sm[32];
    T += int64_t(blockIdx.y) * P;                  // target blockIdx.y of the batch
    partials += size_t(blockIdx.y) * kGsPrepBlocks;
    float acc[1] = {0.f};
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P; i += int64_t(gridDim.x) * blockDim.x)
        acc[0] = fmaf(T[i], T[i], acc[0]);
    ff b[1];
    block_sums_ff<1>(acc, b, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = b[0];
}

// scale = sqrt(P / sum T^2), reduced by one warp in a fixed order (same bits in every block)
__device__ __forceinline__ float gs_scale(const ff* __restrict__ partials, int64_t P) {
    const ff tot = warp_sum_array_ff(partials, kGsPrepBlocks);
    return tot.hi > 0.f ? sqrtf(ff_div(ff_make(float(P)), tot).hi) : 0.f;
}

// -------------------------------------------------------- per-pixel steps ----
// (shared by the float32 passes and the tcgen05 passes of the tensor-core precisions)

// E_0 at rows t + T e of column c: the saved state, or T_s exp(i phi) with phi from the
// caller or the table draw of target blockIdx.y (looked up in a COPIES-way cos/sin table)
template <int R, int T, int COPIES>
__device__ __forceinline__ void gs_initial_field(float2 (&v)[R], const GsArgs& a, const float2* cs, float scale,
                                                 int t, int c) {
    const int W = a.W;
    const SubframeDraw d0 = subframe_draw(a.ps, blockIdx.y);
#pragma unroll
    for (int e = 0; e < R; ++e) {
        const uint32_t p = uint32_t(t + T * e) * uint32_t(W) + uint32_t(c);
        if (a.state_in) {
            v[e] = a.state_in[p];
        } else {
            const float ts = __ldg(a.target + p) * scale;
            float2 ph;
            if (a.init_phase) sincosf(__ldg(a.init_phase + p), &ph.y, &ph.x);
            else ph = cs_lookup<COPIES>(cs, draw_code(a.ps, d0, p) << a.ps.cs_shift);
            v[e] = make_float2(ts * ph.x, ts * ph.y);
        }
    }
}

// Row r's IDFT at slots t + T e -> the hologram exp(2 pi i q / levels) with q the phase
// quantised to the nearest level (codes written when asked). FRESNEL: the field is first
// multiplied by conj(Q) and the hologram by Q.
template <int R, int T, bool FRESNEL, int COPIES>
__device__ __forceinline__ void gs_quantise_row(float2 (&v)[R], const GsArgs& a, const float2* cs, int r, int t) {
    constexpr int NR = R * T;
    const int levels = 1 << a.levels_bits;
    const float k_code = float(levels) * 0.15915494309189533577f;   // levels / (2 pi)
    const int shift = 8 - a.levels_bits;
    float2 qy = make_float2(1.f, 0.f);
    if constexpr (FRESNEL) qy = __ldg(a.chirp_y + r);
#pragma unroll
    for (int e = 0; e < R; ++e) {
        float2 qc = make_float2(1.f, 0.f);
        if constexpr (FRESNEL) {
            qc = cmul(qy, __ldg(a.chirp_x + t + T * e));
            v[e] = make_float2(fmaf(v[e].x, qc.x, v[e].y * qc.y), fmaf(v[e].y, qc.x, -v[e].x * qc.y));
        }
        const float ang = atan2f(v[e].y, v[e].x);
        const int q = int(floorf(fmaf(ang, k_code, 0.5f))) & (levels - 1);
        if (a.codes_out) a.codes_out[size_t(r) * NR + t + T * e] = uint8_t(q);
        v[e] = cs_lookup<COPIES>(cs, uint32_t(q) << shift);
        if constexpr (FRESNEL) v[e] = cmul(v[e], qc);
    }
}

// Amplitude constraint at pixels p0 + e rs of the column DFT: R = DFT / sqrt(P), the
// error sum of (|R| - T_s)^2 is returned, E = T_s R / |R| (T_s where R = 0) replaces v; the
// last iteration writes |R|^2 and E instead.
template <int R, bool LAST>
__device__ __forceinline__ float gs_constrain(float2 (&v)[R], const float (&tg)[R], const GsArgs& a, float scale,
                                              size_t p0, size_t rs) {
    float err = 0.f;
#pragma unroll
    for (int e = 0; e < R; ++e) {
        const size_t p = p0 + e * rs;
        const float2 Rv = make_float2(v[e].x * a.inv_sqrt_p, v[e].y * a.inv_sqrt_p);
        const float amp = sqrtf(fmaf(Rv.x, Rv.x, Rv.y * Rv.y));
        const float ts = tg[e] * scale;
        const float d = amp - ts;
        err = fmaf(d, d, err);
        float2 En = make_float2(ts, 0.f);
        if (amp > 0.f) {
            const float f = ts / amp;
            En = make_float2(Rv.x * f, Rv.y * f);
        }
        if constexpr (LAST) {
            if (a.replay_out) a.replay_out[p] = amp * amp;
            if (a.state_out) a.state_out[p] = En;
        }
        v[e] = En;
    }
    return err;
}

// --------------------------------------------------------------- col_init ----
template <int NC, int V>
__global__ void __launch_bounds__((NC / GsColCfg<NC, V>::R) * GsColCfg<NC, V>::LPC)
k_gs_col_init(GsArgs a0) {
    constexpr int R = GsColCfg<NC, V>::R, LPC = GsColCfg<NC, V>::LPC, T = NC / R;
    const GsArgs a = gs_target(a0, blockIdx.y);
    extern __shared__ float2 sm[];
    float2* cs = sm;
    float2* lines = sm + 256;
    load_cs_table<1>(cs, a.cs256);
    pdl_wait();
    __syncthreads();
    __shared__ float s_scale;
    if (threadIdx.x < 32) {
        const float sc = gs_scale(a.prep_part, int64_t(a.H) * a.W);
        if (threadIdx.x == 0) {
            s_scale = sc;
            if (blockIdx.x == 0) a.sc->scale = sc;
        }
    }
    __syncthreads();
    const int lc = threadIdx.x % LPC, t = threadIdx.x / LPC;
    const int W = a.W;
    const int c = blockIdx.x * LPC + lc;
    float2 v[R];
    gs_initial_field<R, T, 1>(v, a, cs, s_scale, t, c);
    gs_col_line_fft<NC, V, +1>(v, lines, lc, t, a);
    pdl_trigger();
#pragma unroll
    for (int e = 0; e < R; ++e) a.y[size_t(t + T * e) * W + c] = v[e];
}

// -------------------------------------------------------------------- row ----
// FRESNEL: the hologram field is conj(Q) * IDFT(E) and the replay transform takes h * Q.
template <int NR, int V, bool FRESNEL = false>
__global__ void __launch_bounds__((NR / GsRowCfg<NR, V>::R) * GsRowCfg<NR, V>::LPR)
k_gs_row(GsArgs a0) {
    constexpr int R = GsRowCfg<NR, V>::R, T = NR / R;
    const GsArgs a = gs_target(a0, blockIdx.y);
    extern __shared__ float2 sm[];
    float2* cs = sm;
    float2* lines = sm + cs_smem_entries<kGsRowCopies>();
    load_cs_table<kGsRowCopies>(cs, a.cs256);
    pdl_wait();
    __syncthreads();
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int r = blockIdx.x * GsRowCfg<NR, V>::LPR + line;
    float2* z = a.y + size_t(r) * NR;
    float2 v[R];
#pragma unroll
    for (int e = 0; e < R; ++e) v[e] = z[t + T * e];
    gs_row_line_fft<NR, V, +1>(v, lines, line, t, a);
    gs_quantise_row<R, T, FRESNEL, kGsRowCopies>(v, a, cs, r, t);
    gs_row_line_fft<NR, V, -1>(v, lines, line, t, a);
    pdl_trigger();
#pragma unroll
    for (int e = 0; e < R; ++e) z[t + T * e] = v[e];
}

// -------------------------------------------------------------------- col ----
template <int NC, int V, bool LAST>
__global__ void __launch_bounds__((NC / GsColCfg<NC, V>::R) * GsColCfg<NC, V>::LPC,
                                  (NC / GsColCfg<NC, V>::R) * GsColCfg<NC, V>::LPC <= 256 ? 2 : 1)
k_gs_col(GsArgs a0) {
    constexpr int R = GsColCfg<NC, V>::R, LPC = GsColCfg<NC, V>::LPC, T = NC / R;
    const GsArgs a = gs_target(a0, blockIdx.y);
    extern __shared__ float2 sm[];
    __shared__ ff red[32];
    float2* lines = sm;
    const int lc = threadIdx.x % LPC, t = threadIdx.x / LPC;
    const int W = a.W;
    const int c = blockIdx.x * LPC + lc;
    pdl_wait();
    // the target and the scale do not depend on the transform: load them with the field
    // so that their latency hides behind the column DFT
    const size_t rs = size_t(T) * W;                 // element stride of a thread's slots
    const size_t p0 = size_t(t) * W + c;
    float tg[R];
#pragma unroll
    for (int e = 0; e < R; ++e) tg[e] = __ldg(a.target + p0 + e * rs);
    const float scale = a.sc->scale;
    float2 v[R];
#pragma unroll
    for (int e = 0; e < R; ++e) v[e] = a.y[p0 + e * rs];
    gs_col_line_fft<NC, V, -1>(v, lines, lc, t, a);
    const float errv[1] = {gs_constrain<R, LAST>(v, tg, a, scale, p0, rs)};
    ff b[1];
    block_sums_ff<1>(errv, b, red);
    if (threadIdx.x == 0)
        a.err_part[(size_t(blockIdx.y) * a.iters + size_t(a.iter)) * gridDim.x + blockIdx.x] = b[0];
    if constexpr (!LAST) {
        gs_col_line_fft<NC, V, +1>(v, lines, lc, t, a);
        pdl_trigger();
#pragma unroll
        for (int e = 0; e < R; ++e) a.y[size_t(t + T * e) * W + c] = v[e];
    }
}

// ----------------------------------------------------------------- finish ----
__global__ void __launch_bounds__(32)
k_gs_finish(const ff* __restrict__ err_part, int nb, double* __restrict__ err) {
    pdl_wait();
    const size_t k = size_t(blockIdx.y) * gridDim.x + blockIdx.x;   // target blockIdx.y, iteration blockIdx.x
    const ff v = warp_sum_array_ff(err_part + k * nb, nb);
    if (threadIdx.x == 0) err[k] = ff_to_double(v);
}

// ------------------------------------------------------------------- host ----
// Tile variants per shape. Defaults (GB300, 20 iterations, CUDA events): 1024^2 takes
// column variant 0 and row variant 1 (19.9 us per iteration against 22.4 for 0/0),
// 2048^2 column 1 and row 2 (71.9 against 85.7 us).
struct GsTiles {
    int col_v, row_v;
};
static std::mutex g_gs_mu;
static std::map<std::pair<int, int>, GsTiles> g_gs_tiles;

static GsTiles gs_tiles(int H, int W) {
    {
        std::lock_guard<std::mutex> lk(g_gs_mu);
        auto it = g_gs_tiles.find({H, W});
        if (it != g_gs_tiles.end()) return it->second;
    }
    GsTiles t;
    t.col_v = H == 2048 ? 1 : 0;
    t.row_v = (W == 1024 || W == 2048) ? 1 : 0;
    return t;
}

// every launch after k_gs_prepare may overlap the previous kernel's tail (pdl_wait first)
template <int NC, int V>
static int launch_col_init(const GsArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = gs_col_smem<NC, V>();
    int rc = ensure_smem((const void*)k_gs_col_init<NC, V>, smem, &mask);
    if (rc) return rc;
    Launch ln("gs_col_init", st);
    const cudaError_t le = launch_pdl(k_gs_col_init<NC, V>, dim3(a.W / GsColCfg<NC, V>::LPC, a.batch),
                                      dim3((NC / GsColCfg<NC, V>::R) * GsColCfg<NC, V>::LPC), smem, st, a);
    return ln.done("gs_col_init launch", le);
}
template <int NR, int V, bool FRESNEL>
static int launch_row_kind(const GsArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = gs_row_smem<NR, V>();
    int rc = ensure_smem((const void*)k_gs_row<NR, V, FRESNEL>, smem, &mask);
    if (rc) return rc;
    Launch ln("gs_row", st);
    const cudaError_t le = launch_pdl(k_gs_row<NR, V, FRESNEL>, dim3(a.H / GsRowCfg<NR, V>::LPR, a.batch),
                                      dim3((NR / GsRowCfg<NR, V>::R) * GsRowCfg<NR, V>::LPR), smem, st, a);
    return ln.done("gs_row launch", le);
}
template <int NR, int V>
static int launch_row(const GsArgs& a, cudaStream_t st) {
    return a.chirp_y ? launch_row_kind<NR, V, true>(a, st) : launch_row_kind<NR, V, false>(a, st);
}
template <int NC, int V>
static int launch_col(const GsArgs& a, bool last, cudaStream_t st) {
    static uint64_t mask0 = 0, mask1 = 0;
    constexpr size_t smem = sizeof(float2) * size_t(GsColCfg<NC, V>::LPC) * gs_col_stride<NC, V>();
    const dim3 grid(a.W / GsColCfg<NC, V>::LPC, a.batch), threads((NC / GsColCfg<NC, V>::R) * GsColCfg<NC, V>::LPC);
    int rc = last ? ensure_smem((const void*)k_gs_col<NC, V, true>, smem, &mask1)
                  : ensure_smem((const void*)k_gs_col<NC, V, false>, smem, &mask0);
    if (rc) return rc;
    Launch ln("gs_col", st);
    const cudaError_t le = last ? launch_pdl(k_gs_col<NC, V, true>, grid, threads, smem, st, a)
                                : launch_pdl(k_gs_col<NC, V, false>, grid, threads, smem, st, a);
    return ln.done("gs_col launch", le);
}

// ------------------------------------------------- tensor-core precisions ----
// The three passes with both radix-32 stages of every 1024- or 2048-point line on tcgen05
// (tc05_dft.cuh: split fp16 / bf16 operands, float32 accumulators in tensor memory), far
// field only; the per-pixel steps are those of the float32 passes. 256-thread CTAs:
// 8192 / N columns or rows each. Shared memory from a 1024-byte aligned base: the DFT
// matrices (hi, lo) of the directions the pass needs, the cos/sin table (col_init: one
// copy; row: kGsTc05Copies), the padded line buffers (their first 64 KiB also hold the
// A tiles), two mbarriers.
static __device__ int g_gs_tc05_fault;
constexpr int kGsTc05Copies = 4;   // 4-way replicated table: two row CTAs fit on an SM

template <int NC>
constexpr size_t gs_tc05_col_init_smem() {
    return 1024 + 2 * kTc05BBytes + sizeof(float2) * 256 + tc05_col_line_bytes<NC>() + 16;
}
template <int NR>
constexpr size_t gs_tc05_row_smem() {
    return 1024 + 4 * kTc05BBytes + sizeof(float2) * 256 * kGsTc05Copies + tc05_row_line_bytes<NR>() + 16;
}
template <int NC>
constexpr size_t gs_tc05_col_smem() { return 1024 + 4 * kTc05BBytes + tc05_col_line_bytes<NC>() + 16; }
static_assert((2 * kTc05BBytes + sizeof(float2) * 256) % 1024 == 0 &&
                  (4 * kTc05BBytes + sizeof(float2) * 256 * kGsTc05Copies) % 1024 == 0,
              "the line buffers (A tiles) start 1024-byte aligned");
static_assert(2 * (gs_tc05_row_smem<2048>() + 1024) <= 228 * 1024, "two row CTAs per SM");

template <int NC, int PREC>
__global__ void __launch_bounds__(kTc05Threads, 1) k_gs_col_init_tc05(GsArgs a0) {
    constexpr int R = 32, LPC = tc05_lpc<NC>(), T = NC / R, S = tc05_col_stride<NC>();
    const GsArgs a = gs_target(a0, blockIdx.y);
    extern __shared__ uint8_t smraw[];
    __shared__ uint32_t s_tmem;
    __shared__ float s_scale;
    uint32_t base;
    uint8_t* const sm = tc05_smem(smraw, base);
    float2* cs = reinterpret_cast<float2*>(sm + 2 * kTc05BBytes);
    float2* lines = cs + 256;
    const uint32_t lines_u32 = base + 2 * kTc05BBytes + uint32_t(sizeof(float2) * 256);
    const uint32_t bars = lines_u32 + uint32_t(tc05_col_line_bytes<NC>());
    tc05_setup(&s_tmem, a.tc05b + 2 * kTc05BBytes, sm, 2, bars);   // direction +1
    load_cs_table<1>(cs, a.cs256);
    pdl_wait();
    Tc05Group g = tc05_group(lines_u32, bars, &s_tmem, &g_gs_tc05_fault);
    g.b_hi = base;
    g.b_lo = base + kTc05BBytes;
    if (threadIdx.x < 32) {
        const float sc = gs_scale(a.prep_part, int64_t(a.H) * a.W);
        if (threadIdx.x == 0) {
            s_scale = sc;
            if (blockIdx.x == 0) a.sc->scale = sc;
        }
    }
    __syncthreads();
    const int lc = threadIdx.x % LPC, t = threadIdx.x / LPC;
    const int W = a.W;
    const int c = blockIdx.x * LPC + lc;
    float2 v[R];
    gs_initial_field<R, T, 1>(v, a, cs, s_scale, t, c);
    line_fft_tc05<NC, +1, PREC>(v, lines + lc * S, t, a.tw, g);
    pdl_trigger();
#pragma unroll
    for (int e = 0; e < R; ++e) a.y[size_t(t + T * e) * W + c] = v[e];
    tc05_teardown(s_tmem);
}

template <int NR, int PREC>
__global__ void __launch_bounds__(kTc05Threads, 2) k_gs_row_tc05(GsArgs a0) {
    constexpr int R = 32, T = NR / R, LPR = tc05_lpc<NR>(), S = line_stride(NR, 32);
    const GsArgs a = gs_target(a0, blockIdx.y);
    extern __shared__ uint8_t smraw[];
    __shared__ uint32_t s_tmem;
    uint32_t base;
    uint8_t* const sm = tc05_smem(smraw, base);
    float2* cs = reinterpret_cast<float2*>(sm + 4 * kTc05BBytes);
    float2* lines = cs + 256 * kGsTc05Copies;
    const uint32_t lines_u32 = base + 4 * kTc05BBytes + uint32_t(sizeof(float2) * 256 * kGsTc05Copies);
    const uint32_t bars = lines_u32 + uint32_t(tc05_row_line_bytes<NR>());
    tc05_setup(&s_tmem, a.tc05b, sm, 4, bars);   // [-1 hi, -1 lo, +1 hi, +1 lo]
    load_cs_table<kGsTc05Copies>(cs, a.cs256);
    pdl_wait();
    Tc05Group g = tc05_group(lines_u32, bars, &s_tmem, &g_gs_tc05_fault);
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int r = blockIdx.x * LPR + line;
    float2* z = a.y + size_t(r) * NR;
    float2* buf = lines + line * S;
    float2 v[R];
#pragma unroll
    for (int e = 0; e < R; ++e) v[e] = z[t + T * e];
    g.b_hi = base + 2 * kTc05BBytes;
    g.b_lo = base + 3 * kTc05BBytes;
    line_fft_tc05<NR, +1, PREC>(v, buf, t, a.tw, g);
    gs_quantise_row<R, T, false, kGsTc05Copies>(v, a, cs, r, t);
    g.b_hi = base;
    g.b_lo = base + kTc05BBytes;
    line_fft_tc05<NR, -1, PREC>(v, buf, t, a.tw, g);
    pdl_trigger();
#pragma unroll
    for (int e = 0; e < R; ++e) z[t + T * e] = v[e];
    tc05_teardown(s_tmem);
}

template <int NC, bool LAST, int PREC>
__global__ void __launch_bounds__(kTc05Threads, 1) k_gs_col_tc05(GsArgs a0) {
    constexpr int R = 32, LPC = tc05_lpc<NC>(), T = NC / R, S = tc05_col_stride<NC>();
    const GsArgs a = gs_target(a0, blockIdx.y);
    extern __shared__ uint8_t smraw[];
    __shared__ uint32_t s_tmem;
    __shared__ ff red[32];
    uint32_t base;
    uint8_t* const sm = tc05_smem(smraw, base);
    float2* lines = reinterpret_cast<float2*>(sm + 4 * kTc05BBytes);
    const uint32_t lines_u32 = base + 4 * kTc05BBytes;
    const uint32_t bars = lines_u32 + uint32_t(tc05_col_line_bytes<NC>());
    tc05_setup(&s_tmem, a.tc05b, sm, LAST ? 2 : 4, bars);   // [-1 hi, -1 lo (, +1 hi, +1 lo)]
    Tc05Group g = tc05_group(lines_u32, bars, &s_tmem, &g_gs_tc05_fault);
    const int lc = threadIdx.x % LPC, t = threadIdx.x / LPC;
    const int W = a.W;
    const int c = blockIdx.x * LPC + lc;
    pdl_wait();
    const size_t rs = size_t(T) * W;
    const size_t p0 = size_t(t) * W + c;
    float tg[R];
#pragma unroll
    for (int e = 0; e < R; ++e) tg[e] = __ldg(a.target + p0 + e * rs);
    const float scale = a.sc->scale;
    float2 v[R];
#pragma unroll
    for (int e = 0; e < R; ++e) v[e] = a.y[p0 + e * rs];
    g.b_hi = base;
    g.b_lo = base + kTc05BBytes;
    line_fft_tc05<NC, -1, PREC>(v, lines + lc * S, t, a.tw, g);
    const float errv[1] = {gs_constrain<R, LAST>(v, tg, a, scale, p0, rs)};
    ff b[1];
    block_sums_ff<1>(errv, b, red);
    if (threadIdx.x == 0)
        a.err_part[(size_t(blockIdx.y) * a.iters + size_t(a.iter)) * gridDim.x + blockIdx.x] = b[0];
    if constexpr (!LAST) {
        g.b_hi = base + 2 * kTc05BBytes;
        g.b_lo = base + 3 * kTc05BBytes;
        line_fft_tc05<NC, +1, PREC>(v, lines + lc * S, t, a.tw, g);
        pdl_trigger();
#pragma unroll
        for (int e = 0; e < R; ++e) a.y[size_t(t + T * e) * W + c] = v[e];
    }
    tc05_teardown(s_tmem);
}

template <int NC, int PREC>
static int launch_col_init_tc05(const GsArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = gs_tc05_col_init_smem<NC>();
    int rc = ensure_smem((const void*)k_gs_col_init_tc05<NC, PREC>, smem, &mask);
    if (rc) return rc;
    Launch ln("gs_col_init", st);
    const cudaError_t le = launch_pdl(k_gs_col_init_tc05<NC, PREC>, dim3(a.W / tc05_lpc<NC>(), a.batch),
                                      dim3(kTc05Threads), smem, st, a);
    return ln.done("gs_col_init tcgen05 launch", le);
}
template <int NR, int PREC>
static int launch_row_tc05(const GsArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = gs_tc05_row_smem<NR>();
    int rc = ensure_smem((const void*)k_gs_row_tc05<NR, PREC>, smem, &mask);
    if (rc) return rc;
    Launch ln("gs_row", st);
    const cudaError_t le = launch_pdl(k_gs_row_tc05<NR, PREC>, dim3(a.H / tc05_lpc<NR>(), a.batch),
                                      dim3(kTc05Threads), smem, st, a);
    return ln.done("gs_row tcgen05 launch", le);
}
template <int NC, int PREC>
static int launch_col_tc05(const GsArgs& a, bool last, cudaStream_t st) {
    static uint64_t mask0 = 0, mask1 = 0;
    constexpr size_t smem = gs_tc05_col_smem<NC>();
    const dim3 grid(a.W / tc05_lpc<NC>(), a.batch);
    int rc = last ? ensure_smem((const void*)k_gs_col_tc05<NC, true, PREC>, smem, &mask1)
                  : ensure_smem((const void*)k_gs_col_tc05<NC, false, PREC>, smem, &mask0);
    if (rc) return rc;
    Launch ln("gs_col", st);
    const cudaError_t le = last ? launch_pdl(k_gs_col_tc05<NC, true, PREC>, grid, dim3(kTc05Threads), smem, st, a)
                                : launch_pdl(k_gs_col_tc05<NC, false, PREC>, grid, dim3(kTc05Threads), smem, st, a);
    return ln.done("gs_col tcgen05 launch", le);
}

// tensor-core precisions: lengths 1024 and 2048, far field only
#define HOLO_GS_TC(n, prec, F)                                                              \
    switch (n) {                                                                            \
        case 1024: return prec == HOLO_BF16X2 ? F(1024, kTcBf16) : F(1024, kTcFp16);        \
        case 2048: return prec == HOLO_BF16X2 ? F(2048, kTcBf16) : F(2048, kTcFp16);        \
        default: return fail(HOLO_EUNSUPPORTED, "tensor-core GS: line length %d", n);     \
    }
static int run_col_init_tc(const GsArgs& a, int prec, cudaStream_t st) {
#define C(n, p) launch_col_init_tc05<n, p>(a, st)
    HOLO_GS_TC(a.H, prec, C)
#undef C
}
static int run_row_tc(const GsArgs& a, int prec, cudaStream_t st) {
#define C(n, p) launch_row_tc05<n, p>(a, st)
    HOLO_GS_TC(a.W, prec, C)
#undef C
}
static int run_col_tc(const GsArgs& a, int prec, bool last, cudaStream_t st) {
#define C(n, p) launch_col_tc05<n, p>(a, last, st)
    HOLO_GS_TC(a.H, prec, C)
#undef C
}
static bool gs_tc_shape(int H, int W) { return (H == 1024 || H == 2048) && (W == 1024 || W == 2048); }

#define HOLO_GS_V(n, v, F) (v == 2 ? F(n, 2) : v == 1 ? F(n, 1) : F(n, 0))
#define HOLO_GS_SWITCH(n, v, F)                           \
    switch (n) {                                          \
        case 64: return F(64, 0);                         \
        case 128: return F(128, 0);                       \
        case 256: return F(256, 0);                       \
        case 512: return HOLO_GS_V(512, v, F);            \
        case 1024: return HOLO_GS_V(1024, v, F);          \
        case 2048: return HOLO_GS_V(2048, v, F);          \
        case 4096: return F(4096, 0);                     \
        default: return fail(HOLO_EUNSUPPORTED, "line length %d", n); \
    }

static int run_col_init(const GsArgs& a, int cv, cudaStream_t st) {
#define C(n, v) launch_col_init<n, v>(a, st)
    HOLO_GS_SWITCH(a.H, cv, C)
#undef C
}
static int run_row(const GsArgs& a, int rv, cudaStream_t st) {
#define C(n, v) launch_row<n, v>(a, st)
    HOLO_GS_SWITCH(a.W, rv, C)
#undef C
}
static int run_col(const GsArgs& a, int cv, bool last, cudaStream_t st) {
#define C(n, v) launch_col<n, v>(a, last, st)
    HOLO_GS_SWITCH(a.H, cv, C)
#undef C
}
static int col_blocks(int H, int W, int cv) {
#define C(n, v) W / GsColCfg<n, v>::LPC
    HOLO_GS_SWITCH(H, cv, C)
#undef C
}

struct GsLayout {
    size_t y_off, sc_off, prep_off, err_off, chirp_off, total;
};
// B targets: B complex fields, scalars, T^2 partials and error partials, then the chirp
static GsLayout gs_layout(int H, int W, int iters, int B = 1) {
    GsLayout l;
    const size_t P = size_t(H) * W;
    l.y_off = 0;
    l.sc_off = align_up(size_t(B) * P * sizeof(float2), 256);
    l.prep_off = l.sc_off + align_up(size_t(B) * sizeof(GsScalars), 256);
    l.err_off = l.prep_off + align_up(sizeof(ff) * kGsPrepBlocks * size_t(B), 256);
    // error partials for the column tiles with the fewest lines (any variant fits)
    l.chirp_off = l.err_off + align_up(sizeof(ff) * size_t(B) * size_t(iters) * size_t(W / kGsMinLpc), 256);
    // the chirp factors of Fresnel propagation (gs_iterate_fresnel)
    l.total = l.chirp_off + align_up(sizeof(float2) * size_t(H + W), 256);
    return l;
}

static int gs_check_shape(const char* who, int H, int W) {
    if (!is_pow2(H) || !is_pow2(W) || H < kMinDim || W < kMinDim || H > kMaxDim || W > kMaxDim)
        return fail(HOLO_EUNSUPPORTED, "%s: H=%d W=%d must be powers of two in [%d, %d]", who, H, W,
                    kMinDim, kMaxDim);
    return HOLO_OK;
}

}  // namespace holo

using namespace holo;

extern "C" int gs_workspace_size(int H, int W, int iters, int precision, size_t* bytes) {
    clear_error();
    if (!bytes) return fail(HOLO_EINVAL, "gs_workspace_size: NULL output");
    int rc = gs_check_shape("gs_workspace_size", H, W);
    if (rc) return rc;
    if (iters < 1 || iters > 100000) return fail(HOLO_EINVAL, "gs_workspace_size: iters=%d", iters);
    if (precision != HOLO_FP32 && precision != HOLO_FP16X2 && precision != HOLO_BF16X2)
        return fail(HOLO_EINVAL, "gs_workspace_size: unknown precision %d", precision);
    if (precision != HOLO_FP32 && !gs_tc_shape(H, W))
        return fail(HOLO_EUNSUPPORTED, "gs_workspace_size: tensor-core precisions need H, W in {1024, 2048}");
    *bytes = gs_layout(H, W, iters).total;
    return HOLO_OK;
}

namespace holo {

// gs_iterate, gs_iterate_batch (B targets) and gs_iterate_fresnel; `fresnel` selects the
// propagation pair
static int gs_iterate_impl(const char* who, int B, const float* d_target, int H, int W, int iters, int levels,
                           const float* d_init_phase, const uint8_t* d_codes, int64_t L, int lut_levels,
                           uint64_t seed, int64_t start_index, int precision, bool fresnel, double kappa,
                           uint8_t* d_phase_codes, float* d_replay, double* d_err, const float* d_state_in,
                           float* d_state_out, void* d_ws, size_t ws_bytes, holo_stream_t s) {
    clear_error();
    int rc = gs_check_shape(who, H, W);
    if (rc) return rc;
    if (iters < 1 || iters > 100000) return fail(HOLO_EINVAL, "%s: iters=%d out of [1, 100000]", who, iters);
    if (!is_pow2(levels) || levels < 2 || levels > 256)
        return fail(HOLO_EINVAL, "%s: levels=%d is not a power of two in [2, 256]", who, levels);
    if (precision != HOLO_FP32 && precision != HOLO_FP16X2 && precision != HOLO_BF16X2)
        return fail(HOLO_EINVAL, "%s: unknown precision %d", who, precision);
    if (precision != HOLO_FP32 && (fresnel || !gs_tc_shape(H, W)))
        return fail(HOLO_EUNSUPPORTED, "%s: tensor-core precisions need the far field and H, W in {1024, 2048}", who);
    if (!d_target) return fail(HOLO_EINVAL, "%s: d_target is NULL", who);
    if (B < 1 || B > 65535 || int64_t(B) * H * W > (int64_t(1) << 31))
        return fail(HOLO_EINVAL, "%s: %d targets of %dx%d (B*H*W at most 2^31)", who, B, H, W);
    PhaseSource ps;
    const bool use_lut = !d_init_phase && !d_state_in;
    rc = make_phase_source(who, use_lut ? d_codes : nullptr, use_lut ? L : 0, lut_levels, seed,
                           start_index, int64_t(H) * W, &ps);
    if (rc) return rc;
    const GsLayout lay = gs_layout(H, W, iters, B);
    if (!d_ws || ws_bytes < lay.total)
        return fail(HOLO_EWORKSPACE, "%s: workspace %zu bytes, need %zu", who, ws_bytes, lay.total);
    if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0)
        return fail(HOLO_EWORKSPACE, "%s: workspace is not 256-byte aligned", who);
    Tables tab;
    rc = device_tables(&tab);
    if (rc) return rc;
    char* ws = static_cast<char*>(d_ws);
    GsArgs a;
    a.target = d_target;
    a.H = H;
    a.W = W;
    a.levels_bits = log2i(levels);
    a.ps = ps;
    a.init_phase = d_init_phase;
    a.state_in = reinterpret_cast<const float2*>(d_state_in);
    a.y = reinterpret_cast<float2*>(ws + lay.y_off);
    a.sc = reinterpret_cast<GsScalars*>(ws + lay.sc_off);
    a.err_part = reinterpret_cast<ff*>(ws + lay.err_off);
    a.iter = 0;
    a.iters = iters;
    a.batch = B;
    a.codes_out = nullptr;
    a.replay_out = d_replay;
    a.state_out = reinterpret_cast<float2*>(d_state_out);
    a.tw = tab.twiddles;
    a.cs256 = tab.cs256;
    a.tc05b = tab.tc05b[precision];
    a.inv_sqrt_p = float(1.0 / std::sqrt(double(H) * double(W)));
    a.chirp_y = a.chirp_x = nullptr;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    if (fresnel) {
        if (!std::isfinite(kappa) || std::fabs(kappa) > 1e6) return fail(HOLO_EINVAL, "%s: kappa %g", who, kappa);
        float2* chirp = reinterpret_cast<float2*>(ws + lay.chirp_off);
        if ((rc = fresnel_chirp_build(H, W, kappa, chirp, st))) return rc;
        a.chirp_y = chirp;
        a.chirp_x = chirp + H;
    }

    a.prep_part = reinterpret_cast<const ff*>(ws + lay.prep_off);
    {
        Launch ln("gs_prepare", st);
        k_gs_prepare<<<dim3(kGsPrepBlocks, B), kGsPrepThreads, 0, st>>>(d_target, int64_t(H) * W,
                                                                        reinterpret_cast<ff*>(ws + lay.prep_off));
        if ((rc = ln.done("gs_prepare launch"))) return rc;
    }
    const GsTiles tiles = gs_tiles(H, W);
    const bool tc = precision != HOLO_FP32;
    if ((rc = tc ? run_col_init_tc(a, precision, st) : run_col_init(a, tiles.col_v, st))) return rc;
    for (int k = 0; k < iters; ++k) {
        const bool last = k == iters - 1;
        a.iter = k;
        a.codes_out = last ? d_phase_codes : nullptr;
        if ((rc = tc ? run_row_tc(a, precision, st) : run_row(a, tiles.row_v, st))) return rc;
        if ((rc = tc ? run_col_tc(a, precision, last, st) : run_col(a, tiles.col_v, last, st))) return rc;
    }
    if (d_err) {
        const int nb = tc ? W / (H == 1024 ? tc05_lpc<1024>() : tc05_lpc<2048>())
                          : col_blocks(H, W, tiles.col_v);
        if (nb < 1) return HOLO_EUNSUPPORTED;
        Launch ln("gs_finish", st);
        const cudaError_t le = launch_pdl(k_gs_finish, dim3(iters, B), dim3(32), 0, st,
                                          static_cast<const ff*>(a.err_part), nb, d_err);
        if ((rc = ln.done("gs_finish launch", le))) return rc;
    }
    if (use_lut && L > 0) {
        bool prime = L >= 2;
        for (int64_t d = 2; prime && d * d <= L; ++d) prime = (L % d) != 0;
        if (!prime) warn("design rule: L=%lld is not prime", (long long)L);
        if (L <= (H > W ? H : W)) warn("design rule: L=%lld is not greater than max(H, W)", (long long)L);
    }
    return HOLO_OK;
}

}  // namespace holo

extern "C" int gs_iterate(const float* d_target, int H, int W, int iters, int levels,
                          const float* d_init_phase,
                          const uint8_t* d_codes, int64_t L, int lut_levels, uint64_t seed,
                          int64_t start_index, int precision,
                          uint8_t* d_phase_codes, float* d_replay, double* d_err,
                          const float* d_state_in, float* d_state_out,
                          void* d_ws, size_t ws_bytes, holo_stream_t s) {
    return gs_iterate_impl("gs_iterate", 1, d_target, H, W, iters, levels, d_init_phase, d_codes, L, lut_levels,
                           seed, start_index, precision, false, 0.0, d_phase_codes, d_replay, d_err, d_state_in,
                           d_state_out, d_ws, ws_bytes, s);
}

extern "C" int gs_batch_workspace_size(int B, int H, int W, int iters, int precision, size_t* bytes) {
    clear_error();
    if (!bytes) return fail(HOLO_EINVAL, "gs_batch_workspace_size: NULL output");
    int rc = gs_check_shape("gs_batch_workspace_size", H, W);
    if (rc) return rc;
    if (iters < 1 || iters > 100000) return fail(HOLO_EINVAL, "gs_batch_workspace_size: iters=%d", iters);
    if (B < 1 || B > 65535 || int64_t(B) * H * W > (int64_t(1) << 31))
        return fail(HOLO_EINVAL, "gs_batch_workspace_size: %d targets of %dx%d", B, H, W);
    if (precision != HOLO_FP32 && precision != HOLO_FP16X2 && precision != HOLO_BF16X2)
        return fail(HOLO_EINVAL, "gs_batch_workspace_size: unknown precision %d", precision);
    if (precision != HOLO_FP32 && !gs_tc_shape(H, W))
        return fail(HOLO_EUNSUPPORTED, "gs_batch_workspace_size: tensor-core precisions need H, W in {1024, 2048}");
    *bytes = gs_layout(H, W, iters, B).total;
    return HOLO_OK;
}

extern "C" int gs_iterate_batch(const float* d_targets, int B, int H, int W, int iters, int levels,
                                const float* d_init_phases, const uint8_t* d_codes, int64_t L, int lut_levels,
                                uint64_t seed, int64_t start_index, int precision, uint8_t* d_phase_codes,
                                float* d_replay, double* d_err, const float* d_states_in, float* d_states_out,
                                void* d_ws, size_t ws_bytes, holo_stream_t s) {
    return gs_iterate_impl("gs_iterate_batch", B, d_targets, H, W, iters, levels, d_init_phases, d_codes, L,
                           lut_levels, seed, start_index, precision, false, 0.0, d_phase_codes, d_replay, d_err,
                           d_states_in, d_states_out, d_ws, ws_bytes, s);
}

extern "C" int gs_iterate_fresnel(const float* d_target, int H, int W, int iters, int levels,
                                  const float* d_init_phase, const uint8_t* d_codes, int64_t L, int lut_levels,
                                  uint64_t seed, int64_t start_index, double kappa, uint8_t* d_phase_codes,
                                  float* d_replay, double* d_err, const float* d_state_in, float* d_state_out,
                                  void* d_ws, size_t ws_bytes, holo_stream_t s) {
    return gs_iterate_impl("gs_iterate_fresnel", 1, d_target, H, W, iters, levels, d_init_phase, d_codes, L,
                           lut_levels, seed, start_index, HOLO_FP32, true, kappa, d_phase_codes, d_replay, d_err,
                           d_state_in, d_state_out, d_ws, ws_bytes, s);
}

namespace holo {

int gs_tc05_fault(int* out, bool clear) {
    int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_gs_tc05_fault, sizeof(int));
    if (e != cudaSuccess) return cuda_status(e, "gs_tc05_fault");
    if (clear && v) {
        const int z = 0;
        if ((e = cudaMemcpyToSymbol(g_gs_tc05_fault, &z, sizeof(int))) != cudaSuccess)
            return cuda_status(e, "gs_tc05_fault");
    }
    *out = v;
    return HOLO_OK;
}

// phase[p] = arg(state[p]) in (-pi, pi], with arg(0) = 0 whatever the zeros' signs
__global__ void k_gs_state_phase(const float2* __restrict__ state, int64_t n, float* __restrict__ phase) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const float2 e = state[i];
        phase[i] = (e.x == 0.f && e.y == 0.f) ? 0.f : atan2f(e.y, e.x);
    }
}

}  // namespace holo

extern "C" int gs_state_phase(const float* d_state, int H, int W, float* d_phase, holo_stream_t s) {
    clear_error();
    if (!d_state || !d_phase || H < 1 || W < 1 || int64_t(H) * W > (int64_t(1) << 28))
        return fail(HOLO_EINVAL, "gs_state_phase: bad arguments (%dx%d)", H, W);
    const int64_t n = int64_t(H) * W;
    const int threads = 256;
    const int blocks = int((n + threads - 1) / threads < 152 * 16 ? (n + threads - 1) / threads : 152 * 16);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    Launch ln("gs_state_phase", st);
    k_gs_state_phase<<<blocks, threads, 0, st>>>(reinterpret_cast<const float2*>(d_state), n, d_phase);
    return ln.done("gs_state_phase launch");
}

extern "C" int gs_tuning_set(int H, int W, int col_variant, int row_variant) {
    clear_error();
    int rc = gs_check_shape("gs_tuning_set", H, W);
    if (rc) return rc;
    if (col_variant < -1 || col_variant > 2 || row_variant < -1 || row_variant > 2)
        return fail(HOLO_EINVAL, "gs_tuning_set: variants -1..2 (got %d, %d)", col_variant, row_variant);
    std::lock_guard<std::mutex> lk(g_gs_mu);
    if (col_variant < 0 || row_variant < 0) {
        g_gs_tiles.erase({H, W});
        return HOLO_OK;
    }
    g_gs_tiles[{H, W}] = GsTiles{gs_has_variants(H) ? col_variant : 0, gs_has_variants(W) ? row_variant : 0};
    return HOLO_OK;
}

extern "C" int gs_tuning_get(int H, int W, int* col_variant, int* row_variant) {
    clear_error();
    int rc = gs_check_shape("gs_tuning_get", H, W);
    if (rc) return rc;
    if (!col_variant || !row_variant) return fail(HOLO_EINVAL, "gs_tuning_get: NULL output");
    const GsTiles t = gs_tiles(H, W);
    *col_variant = t.col_v;
    *row_variant = t.row_v;
    return HOLO_OK;
}
