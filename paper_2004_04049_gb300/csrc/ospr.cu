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
constexpr size_t col_smem_bytes() {
    return sizeof(float2) * (256 + size_t(ColCfg<NC>::LPC) * line_stride(NC, ColCfg<NC>::R));
}
template <int NR>
constexpr size_t row_smem_bytes() {
    return sizeof(float2) * size_t(RowCfg<NR>::LPR) * line_stride(NR, RowCfg<NR>::R);
}

// ------------------------------------------------------------------ pass 1 ----
template <int NC>
__global__ void __launch_bounds__((NC / ColCfg<NC>::R) * ColCfg<NC>::LPC)
k_ospr_col_ifft(OsprArgs a) {
    constexpr int R = ColCfg<NC>::R, LPC = ColCfg<NC>::LPC, T = NC / R;
    extern __shared__ float2 sm[];
    float2* cs = sm;
    float2* lines = sm + 256;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) cs[i] = a.cs256[i];
    __syncthreads();

    const int lc = threadIdx.x % LPC, t = threadIdx.x / LPC;
    const int W = a.W;
    const int c = blockIdx.x * LPC + lc;
    const int cm = (W - c) & (W - 1);
    const int s0 = 2 * (a.first_pair + int(blockIdx.y));
    const bool single = s0 + 1 >= a.N;
    const SubframeDraw d0 = subframe_draw(a.ps, s0);
    const SubframeDraw d1 = subframe_draw(a.ps, single ? s0 : s0 + 1);
    const int sh = a.ps.cs_shift;

    float2 v[R];
#pragma unroll
    for (int e = 0; e < R; ++e) {
        const int r = t + T * e;
        const int rm = (NC - r) & (NC - 1);
        const uint32_t p = uint32_t(r) * uint32_t(W) + uint32_t(c);
        const uint32_t pm = uint32_t(rm) * uint32_t(W) + uint32_t(cm);
        const float tp = __ldg(a.target + p);
        const float2 c0 = cs[draw_code(a.ps, d0, p) << sh];
        if (single) {
            v[e] = make_float2(tp * c0.x, tp * c0.y);
        } else {
            const float tm = __ldg(a.target + pm);
            const float2 c0m = cs[draw_code(a.ps, d0, pm) << sh];
            const float2 c1 = cs[draw_code(a.ps, d1, p) << sh];
            const float2 c1m = cs[draw_code(a.ps, d1, pm) << sh];
            // Hermitian parts E(k) + conj(E(-k)) of both sub-frames, packed as a + i b
            const float2 h0 = make_float2(fmaf(tp, c0.x, tm * c0m.x), fmaf(tp, c0.y, -tm * c0m.y));
            const float2 h1 = make_float2(fmaf(tp, c1.x, tm * c1m.x), fmaf(tp, c1.y, -tm * c1m.y));
            v[e] = make_float2(h0.x - h1.y, h0.y + h1.x);
        }
    }
    line_fft<NC, R, +1, true>(v, lines + lc * line_stride(NC, R), t, a.tw);
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
    float2* lines = sm + 256;
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
        line_fft<NC, R, -1, true>(v, lines + lc * line_stride(NC, R), t, a.tw);
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
__global__ void k_ospr_finalize(const float* __restrict__ S, int groups, int H, int W,
                                float scale, float* __restrict__ I) {
    const size_t P = size_t(H) * W;
    const size_t p = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int r = int(p / W), c = int(p % W);
    const size_t pm = size_t((H - r) & (H - 1)) * W + size_t((W - c) & (W - 1));
    float s = 0.f;
    for (int g = 0; g < groups; ++g) s += S[size_t(g) * P + p] + S[size_t(g) * P + pm];
    I[p] = s * scale;
}

// ------------------------------------------------------------------- host ----
template <int NC>
static int launch_col_ifft(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = col_smem_bytes<NC>();
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
    constexpr size_t smem = col_smem_bytes<NC>();
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

static OsprPlan ospr_plan(int H, int W, int N) {
    OsprPlan pl;
    const size_t P = size_t(H) * W;
    pl.npairs = (N + 1) / 2;
    pl.chunk = pl.npairs < kMaxChunkPairs ? pl.npairs : kMaxChunkPairs;
    pl.groups = pl.chunk < kMaxGroups ? pl.chunk : kMaxGroups;
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
        const int blocks = int((P + threads - 1) / threads);
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
        const int blocks = int((P + threads - 1) / threads);
        Launch ln("ospr_finalize", st);
        k_ospr_finalize<<<blocks, threads, 0, st>>>(a.sacc, pl.groups, H, W, scale, d_replay);
        if ((rc = ln.done("ospr_finalize launch"))) return rc;
    }
    return HOLO_OK;
}
