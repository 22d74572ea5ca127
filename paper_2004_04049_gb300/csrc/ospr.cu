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
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>

#include "ospr_kernels.cuh"

namespace holo {

// ---------------------------------------------------------------- finalize ----
// I(k) = I(-k) = (sum_g S_g(k) + S_g(-k)) * scale for the pixel pairs {k, -k}, in the order
// of ospr_finalize_pixel (the same bits). Thread q takes the four pixels 4q .. 4q+3 of the
// first half of the raster (rows 0 .. H/2; W >= 64 keeps them in one row): one float4 load
// per group of their own accumulators, scalar loads of the mirrors (the mirror run is
// descending and one pixel off the float4 grid), a float4 store of their outputs (scalar
// stores into a replay buffer that is not 16-byte aligned) and scalar stores of the
// mirrors' (P < 2^31: 32-bit indices). In rows 0 and H/2 a pixel whose
// mirror lies before it is left to the mirror.
__global__ void k_ospr_finalize(const float* __restrict__ S, int groups, int H, int W, int log2W,
                                float scale, float* __restrict__ I) {
    pdl_wait();
    const uint32_t P = uint32_t(H) * uint32_t(W);
    const uint32_t p0 = 4u * (blockIdx.x * blockDim.x + threadIdx.x);
    if (p0 >= P / 2 + uint32_t(W)) return;
    const uint32_t r = p0 >> log2W, c0 = p0 & uint32_t(W - 1);
    const uint32_t rm = (uint32_t(H) - r) & uint32_t(H - 1);
    uint32_t pm[4];
    float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) pm[k] = rm * uint32_t(W) + ((uint32_t(W) - c0 - uint32_t(k)) & uint32_t(W - 1));
    for (int g = 0; g < groups; ++g) {
        const float* Sg = S + size_t(g) * P;
        const float4 own = __ldg(reinterpret_cast<const float4*>(Sg + p0));
        s[0] += own.x + __ldg(Sg + pm[0]);
        s[1] += own.y + __ldg(Sg + pm[1]);
        s[2] += own.z + __ldg(Sg + pm[2]);
        s[3] += own.w + __ldg(Sg + pm[3]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) s[k] *= scale;
    const bool edge = r == 0 || r == uint32_t(H / 2);   // rows whose mirrors lie in the same row
    if (!edge) {
        if ((reinterpret_cast<uintptr_t>(I) & 15) == 0) {
            *reinterpret_cast<float4*>(I + p0) = make_float4(s[0], s[1], s[2], s[3]);
        } else {   // a caller buffer aligned to its float only
#pragma unroll
            for (int k = 0; k < 4; ++k) I[p0 + k] = s[k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) I[pm[k]] = s[k];
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (pm[k] >= p0 + uint32_t(k)) {
                I[p0 + k] = s[k];
                I[pm[k]] = s[k];
            }
    }
}

// Fresnel replay: no twin symmetry, I(k) = scale * sum_g S_g(k)
__global__ void k_ospr_finalize_fresnel(const float* __restrict__ S, int groups, size_t P, float scale,
                                        float* __restrict__ I) {
    pdl_wait();
    const size_t p = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= P) return;
    float s = 0.f;
    for (int g = 0; g < groups; ++g) s += S[size_t(g) * P + p];
    I[p] = s * scale;
}

// The separable quadratic phase of Fresnel propagation, chirp[i] = exp(i*pi*kappa*(i - n/2)^2)
// for the H rows and then the W columns, evaluated in float64 (sincospi reduces the
// argument exactly) and rounded to float32.
__global__ void k_fresnel_chirp(int H, int W, double kappa, float2* __restrict__ chirp) {
    pdl_wait();   // a previous kernel may still read the table
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H + W) return;
    const int n = i < H ? H : W;
    const double d = double(i < H ? i : i - H) - 0.5 * double(n);
    double sn, cs;
    sincospi(kappa * d * d, &sn, &cs);
    chirp[i] = make_float2(float(cs), float(sn));
}

int fresnel_chirp_build(int H, int W, double kappa, float2* d_chirp, cudaStream_t st) {
    Launch ln("fresnel_chirp", st);
    const cudaError_t le = launch_pdl(k_fresnel_chirp, dim3(unsigned((H + W + 255) / 256)), dim3(256), 0, st, H, W,
                                      kappa, d_chirp);
    return ln.done("fresnel_chirp launch", le);
}

// ------------------------------------------------------------------- host ----
// Per-shape tuning: tile variants of the three passes (column IDFT, row, column DFT;
// the two column passes share only the field layout, so their tiles are independent),
// pairs in flight (chunk) and partial accumulators (groups). Defaults: variant 0, 16
// pairs, 4 groups (overridable with HOLO_OSPR_CHUNK / HOLO_OSPR_GROUPS); ospr_autotune
// replaces them per shape with the fastest measured candidate, and HOLO_TUNE_CACHE names
// a file that keeps the choices across processes. The workspace size follows the tuning
// of the shape.
struct OsprTuning {
    int ci_v, cf_v, row_v, chunk, groups;
};

static OsprTuning clamp_variants(int H, int W, OsprTuning t) {
    if (t.ci_v < 0 || t.ci_v >= col_variants(H)) t.ci_v = 0;
    if (t.cf_v < 0 || t.cf_v >= col_variants(H)) t.cf_v = 0;
    if (t.row_v < 0 || t.row_v >= row_variants(W)) t.row_v = 0;
    return t;
}

static int env_int(const char* name, int lo, int hi, int dflt) {
    const char* v = getenv(name);
    if (!v || !*v) return dflt;
    const int x = atoi(v);
    return x < lo ? lo : (x > hi ? hi : x);
}

static OsprTuning default_tuning() {
    static const OsprTuning t{0, 0, 0, env_int("HOLO_OSPR_CHUNK", 1, kMaxChunkPairs, kMaxChunkPairs),
                              env_int("HOLO_OSPR_GROUPS", 1, kMaxGroups, kMaxGroups)};
    return t;
}

static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, OsprTuning> g_tune;
static bool g_tune_loaded = false;

static void tune_cache_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = getenv("HOLO_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    int H, W, ci, cf, rv, ch, gr;
    while (fscanf(f, " {\"H\": %d, \"W\": %d, \"col_ifft_variant\": %d, \"col_fft_variant\": %d, "
                     "\"row_variant\": %d, \"chunk\": %d, \"groups\": %d}",
                  &H, &W, &ci, &cf, &rv, &ch, &gr) == 7) {
        if (ch < 1 || ch > kMaxChunkPairs || gr < 1 || gr > kMaxGroups) continue;
        g_tune[{H, W}] = clamp_variants(H, W, OsprTuning{ci, cf, rv, ch, gr});
    }
    fclose(f);
}

static void tune_cache_save_locked() {
    const char* path = getenv("HOLO_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "w");
    if (!f) return;
    for (const auto& kv : g_tune)
        fprintf(f, "{\"H\": %d, \"W\": %d, \"col_ifft_variant\": %d, \"col_fft_variant\": %d, "
                   "\"row_variant\": %d, \"chunk\": %d, \"groups\": %d}\n", kv.first.first, kv.first.second,
                kv.second.ci_v, kv.second.cf_v, kv.second.row_v, kv.second.chunk, kv.second.groups);
    fclose(f);
}

static OsprTuning tuning_for(int H, int W) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_load_locked();
    auto it = g_tune.find({H, W});
    return it == g_tune.end() ? default_tuning() : it->second;
}

static void tuning_install(int H, int W, const OsprTuning& t, bool save) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_load_locked();
    g_tune[{H, W}] = t;
    if (save) tune_cache_save_locked();
}

struct OsprPlan {
    int npairs, chunk, groups, ci_v, cf_v, row_v;
    int prec = HOLO_FP32;
    size_t z_bytes, s_bytes, total;
};

static OsprPlan ospr_plan_with(int H, int W, int N, const OsprTuning& t) {
    OsprPlan pl;
    const size_t P = size_t(H) * W;
    pl.npairs = (N + 1) / 2;
    pl.chunk = pl.npairs < t.chunk ? pl.npairs : t.chunk;
    pl.groups = pl.chunk < t.groups ? pl.chunk : t.groups;
    const OsprTuning c = clamp_variants(H, W, t);
    pl.ci_v = c.ci_v;
    pl.cf_v = c.cf_v;
    pl.row_v = c.row_v;
    pl.z_bytes = align_up(size_t(pl.chunk) * P * sizeof(float2), 256);
    pl.s_bytes = align_up(size_t(pl.groups) * P * sizeof(float), 256);
    pl.total = pl.z_bytes + pl.s_bytes;
    return pl;
}

static bool tc_shape(int H, int W) { return (H == 1024 || H == 2048) && (W == 1024 || W == 2048); }

// the tensor-core precisions run the fixed tiles of ospr_tc.cu; the tile variants of the
// plan apply to the float32 passes
static OsprPlan ospr_plan(int H, int W, int N, int precision = HOLO_FP32) {
    OsprPlan pl = ospr_plan_with(H, W, N, tuning_for(H, W));
    pl.prec = precision;
    return pl;
}

static int check_precision(const char* who, int precision, int H, int W) {
    if (precision == HOLO_FP32) return HOLO_OK;
    if (precision != HOLO_FP16X2 && precision != HOLO_BF16X2)
        return fail(HOLO_EINVAL, "%s: unknown precision %d", who, precision);
    if (!tc_shape(H, W))
        return fail(HOLO_EUNSUPPORTED, "%s: tensor-core precisions need H, W in {1024, 2048} (got %dx%d)", who, H, W);
    return HOLO_OK;
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

// chunks of sub-frame pairs through the three passes, then the symmetrising finalize;
// `bits_ready` (optional) is recorded on the stream once the last row pass, which writes
// the last hologram bits, is queued
static int ospr_run(OsprArgs& a, const OsprPlan& pl, bool replay, float* d_replay, cudaStream_t st,
                    cudaEvent_t bits_ready = nullptr) {
    int rc;
    for (int first = 0; first < pl.npairs; first += pl.chunk) {
        a.first_pair = first;
        a.pairs = pl.npairs - first < pl.chunk ? pl.npairs - first : pl.chunk;
        a.accumulate = first > 0;
        const bool last = first + a.pairs >= pl.npairs;
        if (pl.prec == HOLO_FP32) {
            if ((rc = ospr_run_col_ifft(a, pl.ci_v, st))) return rc;
            if ((rc = ospr_run_row(a, pl.row_v, replay, st))) return rc;
        } else {
            if ((rc = ospr_run_col_ifft_tc(a, pl.prec, st))) return rc;
            if ((rc = ospr_run_row_tc(a, pl.prec, replay, st))) return rc;
        }
        if (last && bits_ready) {
            const cudaError_t e = cudaEventRecord(bits_ready, st);
            if (e != cudaSuccess) return cuda_status(e, "ospr: bits event");
        }
        if (replay) {
            if (pl.prec == HOLO_FP32) rc = ospr_run_col_fft(a, pl.cf_v, st);
            else rc = ospr_run_col_fft_tc(a, pl.prec, st);
            if (rc) return rc;
        }
    }
    if (replay && a.fresnel) {
        const size_t P = size_t(a.H) * a.W;
        const float scale = float(1.0 / (double(a.N) * double(P)));
        const int threads = 256;
        Launch ln("ospr_finalize", st);
        const cudaError_t le = launch_pdl(k_ospr_finalize_fresnel, dim3(unsigned((P + threads - 1) / threads)),
                                          dim3(threads), 0, st, static_cast<const float*>(a.sacc), pl.groups, P,
                                          scale, d_replay);
        return ln.done("ospr_finalize launch", le);
    }
    if (replay) {
        const size_t P = size_t(a.H) * a.W;
        const float scale = float(1.0 / (2.0 * double(a.N) * double(P)));
        const int threads = 256;
        const size_t quads = (P / 2 + a.W) / 4;   // W >= 64: the half raster is whole quads
        const int blocks = int((quads + threads - 1) / threads);
        Launch ln("ospr_finalize", st);
        const cudaError_t le = launch_pdl(k_ospr_finalize, dim3(blocks), dim3(threads), 0, st,
                                          static_cast<const float*>(a.sacc), pl.groups, a.H, a.W, log2i(a.W),
                                          scale, d_replay);
        if ((rc = ln.done("ospr_finalize launch", le))) return rc;
    }
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
    if ((rc = check_precision("ospr_workspace_size", precision, H, W))) return rc;
    *bytes = ospr_plan(H, W, N, precision).total;
    return HOLO_OK;
}

namespace holo {

// Section 8 design rules for the table length (prime, longer than the sub-frame count
// and than the largest image dimension): recorded as warnings with HOLO_OK
static void ospr_design_rules(int64_t L, int N, int H, int W) {
    if (L <= 0) return;
    if (!is_prime(L)) warn("design rule: L=%lld is not prime", (long long)L);
    if (L <= N) warn("design rule: L=%lld is not greater than N=%d", (long long)L, N);
    if (L <= (H > W ? H : W)) warn("design rule: L=%lld is not greater than max(H, W)", (long long)L);
}

}  // namespace holo

namespace holo {

// ospr_generate, with an optional event recorded on s once the last hologram bits are
// written (the batch with host buffers starts their copy there)
int ospr_generate_ev(const float* d_target, int H, int W, int N, const uint8_t* d_codes, int64_t L, int levels,
                     uint64_t seed, int64_t start_index, int64_t subframe_stride, int precision,
                     uint32_t* d_holo_bits, float* d_replay, void* d_ws, size_t ws_bytes, holo_stream_t s,
                     cudaEvent_t bits_ready) {
    const char* who = "ospr_generate";
    int rc = check_shape(who, H, W);
    if (rc) return rc;
    if (N < 1 || N > 4096) return fail(HOLO_EINVAL, "%s: N=%d out of [1, 4096]", who, N);
    if ((rc = check_precision(who, precision, H, W))) return rc;
    if (!d_target) return fail(HOLO_EINVAL, "%s: d_target is NULL", who);
    if (!d_holo_bits && !d_replay) return fail(HOLO_EINVAL, "%s: both outputs are NULL", who);
    const int64_t P = int64_t(H) * W;
    const int64_t stride = subframe_stride == 0 ? P : subframe_stride;
    if (stride > (INT64_C(1) << 40) || start_index > (INT64_C(1) << 61))
        return fail(HOLO_EINVAL, "%s: start or stride too large", who);
    PhaseSource ps;
    rc = make_phase_source(who, d_codes, L, levels, seed, start_index, stride, &ps);
    if (rc) return rc;
    const OsprPlan pl = ospr_plan(H, W, N, precision);
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
    a.tc05b = tab.tc05b[precision];
    a.fresnel = 0;
    a.chirp_y = a.chirp_x = nullptr;
    if ((rc = ospr_run(a, pl, d_replay != nullptr, d_replay, reinterpret_cast<cudaStream_t>(s), bits_ready)))
        return rc;
    ospr_design_rules(L, N, H, W);
    return HOLO_OK;
}

}  // namespace holo

extern "C" int ospr_generate(const float* d_target, int H, int W, int N,
                             const uint8_t* d_codes, int64_t L, int levels, uint64_t seed,
                             int64_t start_index, int64_t subframe_stride, int precision,
                             uint32_t* d_holo_bits, float* d_replay,
                             void* d_ws, size_t ws_bytes, holo_stream_t s) {
    clear_error();
    return ospr_generate_ev(d_target, H, W, N, d_codes, L, levels, seed, start_index, subframe_stride, precision,
                            d_holo_bits, d_replay, d_ws, ws_bytes, s, nullptr);
}

// Fresnel propagation: one sub-frame per field slot, so the plan of 2N sub-frames gives N
// slots; the chirp tables (H + W complex64) follow the plan's buffers.
static OsprPlan fresnel_plan(int H, int W, int N, size_t* chirp_off) {
    OsprPlan pl = ospr_plan(H, W, 2 * N, HOLO_FP32);
    *chirp_off = pl.total;
    pl.total += align_up(size_t(H + W) * sizeof(float2), 256);
    return pl;
}

extern "C" int ospr_fresnel_workspace_size(int H, int W, int N, size_t* bytes) {
    clear_error();
    if (!bytes) return fail(HOLO_EINVAL, "ospr_fresnel_workspace_size: NULL output");
    int rc = check_shape("ospr_fresnel_workspace_size", H, W);
    if (rc) return rc;
    if (N < 1 || N > 4096) return fail(HOLO_EINVAL, "ospr_fresnel_workspace_size: N=%d out of [1, 4096]", N);
    size_t off = 0;
    *bytes = fresnel_plan(H, W, N, &off).total;
    return HOLO_OK;
}

extern "C" int ospr_generate_fresnel(const float* d_target, int H, int W, int N, const uint8_t* d_codes, int64_t L,
                                     int levels, uint64_t seed, int64_t start_index, int64_t subframe_stride,
                                     double kappa, uint32_t* d_holo_bits, float* d_replay, void* d_ws,
                                     size_t ws_bytes, holo_stream_t s) {
    clear_error();
    const char* who = "ospr_generate_fresnel";
    int rc = check_shape(who, H, W);
    if (rc) return rc;
    if (N < 1 || N > 4096) return fail(HOLO_EINVAL, "%s: N=%d out of [1, 4096]", who, N);
    if (!std::isfinite(kappa) || std::fabs(kappa) > 1e6) return fail(HOLO_EINVAL, "%s: kappa %g", who, kappa);
    if (!d_target) return fail(HOLO_EINVAL, "%s: d_target is NULL", who);
    if (!d_holo_bits && !d_replay) return fail(HOLO_EINVAL, "%s: both outputs are NULL", who);
    const int64_t P = int64_t(H) * W;
    const int64_t stride = subframe_stride == 0 ? P : subframe_stride;
    if (stride > (INT64_C(1) << 40) || start_index > (INT64_C(1) << 61))
        return fail(HOLO_EINVAL, "%s: start or stride too large", who);
    PhaseSource ps;
    rc = make_phase_source(who, d_codes, L, levels, seed, start_index, stride, &ps);
    if (rc) return rc;
    size_t chirp_off = 0;
    const OsprPlan pl = fresnel_plan(H, W, N, &chirp_off);
    if (!d_ws || ws_bytes < pl.total)
        return fail(HOLO_EWORKSPACE, "%s: workspace %zu bytes, need %zu", who, ws_bytes, pl.total);
    if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0)
        return fail(HOLO_EWORKSPACE, "%s: workspace is not 256-byte aligned", who);
    Tables tab;
    if ((rc = device_tables(&tab))) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    float2* chirp = reinterpret_cast<float2*>(static_cast<char*>(d_ws) + chirp_off);
    if ((rc = fresnel_chirp_build(H, W, kappa, chirp, st))) return rc;
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
    a.tc05b = nullptr;
    a.fresnel = 1;
    a.chirp_y = chirp;
    a.chirp_x = chirp + H;
    return ospr_run(a, pl, d_replay != nullptr, d_replay, st);
}

extern "C" int ospr_tuning_get(int H, int W, int* col_ifft_variant, int* col_fft_variant, int* row_variant,
                               int* chunk, int* groups) {
    clear_error();
    int rc = check_shape("ospr_tuning_get", H, W);
    if (rc) return rc;
    if (!col_ifft_variant || !col_fft_variant || !row_variant || !chunk || !groups)
        return fail(HOLO_EINVAL, "ospr_tuning_get: NULL output");
    const OsprTuning t = clamp_variants(H, W, tuning_for(H, W));
    *col_ifft_variant = t.ci_v;
    *col_fft_variant = t.cf_v;
    *row_variant = t.row_v;
    *chunk = t.chunk;
    *groups = t.groups;
    return HOLO_OK;
}

extern "C" int ospr_tuning_set(int H, int W, int col_ifft_variant, int col_fft_variant, int row_variant,
                               int chunk, int groups) {
    clear_error();
    int rc = check_shape("ospr_tuning_set", H, W);
    if (rc) return rc;
    if (col_ifft_variant < 0 || col_ifft_variant > 2 || col_fft_variant < 0 || col_fft_variant > 2 ||
        row_variant < 0 || row_variant > 1 || chunk < 1 || chunk > kMaxChunkPairs || groups < 1 ||
        groups > kMaxGroups)
        return fail(HOLO_EINVAL, "ospr_tuning_set: column variants 0..2, row variant 0..1, chunk 1..%d, groups 1..%d",
                    kMaxChunkPairs, kMaxGroups);
    tuning_install(H, W, clamp_variants(H, W, OsprTuning{col_ifft_variant, col_fft_variant, row_variant, chunk,
                                                         groups}), false);
    return HOLO_OK;
}

extern "C" int ospr_autotune(int H, int W, int N, int reps, holo_stream_t s, double* best_ms) {
    clear_error();
    const char* who = "ospr_autotune";
    int rc = check_shape(who, H, W);
    if (rc) return rc;
    if (N < 1 || N > 4096 || reps < 1 || reps > 100) return fail(HOLO_EINVAL, "%s: N=%d reps=%d", who, N, reps);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    const size_t P = size_t(H) * W;
    const int64_t L = 10007;
    // the largest candidate plan bounds the workspace
    const size_t ws_bytes = ospr_plan_with(H, W, N, OsprTuning{0, 0, 0, kMaxChunkPairs, kMaxGroups}).total;
    if (fault_injected("alloc")) return fail(HOLO_ENOMEM, "%s: injected allocation failure (HOLO_FAULT_INJECT)", who);
    void *d_t = nullptr, *d_codes = nullptr, *d_bits = nullptr, *d_rep = nullptr, *d_ws = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaMalloc(&d_t, P * sizeof(float));
    if (ce == cudaSuccess) ce = cudaMalloc(&d_codes, size_t(L));
    if (ce == cudaSuccess) ce = cudaMalloc(&d_bits, size_t(N) * P / 8);
    if (ce == cudaSuccess) ce = cudaMalloc(&d_rep, P * sizeof(float));
    if (ce == cudaSuccess) ce = cudaMalloc(&d_ws, ws_bytes);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    auto release = [&]() {
        cudaStreamSynchronize(st);
        cudaFree(d_t); cudaFree(d_codes); cudaFree(d_bits); cudaFree(d_rep); cudaFree(d_ws);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (ce != cudaSuccess) {
        release();
        return fail(HOLO_ENOMEM, "%s: scratch allocation failed: %s", who, cudaGetErrorString(ce));
    }
    rc = cuda_status(cudaMemsetAsync(d_t, 0x3c, P * sizeof(float), st), "ospr_autotune: fill");
    if (!rc) rc = lut_build(7, L, 256, static_cast<uint8_t*>(d_codes), nullptr, s);
    const OsprTuning before = tuning_for(H, W);
    const int npairs = (N + 1) / 2;
    // time one candidate: one warm-up call, then the median of `reps` calls
    auto measure = [&](const OsprTuning& t, float* ms) -> int {
        tuning_install(H, W, t, false);
        int r = ospr_generate(static_cast<const float*>(d_t), H, W, N, static_cast<const uint8_t*>(d_codes), L, 256, 7,
                              0, 0, HOLO_FP32, static_cast<uint32_t*>(d_bits), static_cast<float*>(d_rep), d_ws,
                              ws_bytes, s);
        if (r) return r;
        float v[100];
        for (int i = 0; i < reps; ++i) {
            cudaEventRecord(e0, st);
            r = ospr_generate(static_cast<const float*>(d_t), H, W, N, static_cast<const uint8_t*>(d_codes), L, 256,
                              7, 0, 0, HOLO_FP32, static_cast<uint32_t*>(d_bits), static_cast<float*>(d_rep), d_ws,
                              ws_bytes, s);
            if (r) return r;
            cudaEventRecord(e1, st);
            cudaError_t x = cudaEventSynchronize(e1);
            if (x != cudaSuccess) return cuda_status(x, "ospr_autotune: timing");
            cudaEventElapsedTime(&v[i], e0, e1);
        }
        std::sort(v, v + reps);
        *ms = v[reps / 2];
        return HOLO_OK;
    };
    // the descent starts from the 256-thread column DFT tiles (variant 1, two CTAs per SM):
    // alone a frame times them within about 1% of variant 0, but in a batch they let
    // other frames' CTAs share the SMs (14-frame 1024^2 step: 164.9 k against 160.9 k
    // sub-frames/s), so a tie keeps them
    OsprTuning best{0, col_variants(H) > 1 ? 1 : 0, 0, kMaxChunkPairs < npairs ? kMaxChunkPairs : npairs, kMaxGroups};
    float best_t = 0.f;
    if (!rc) rc = measure(best, &best_t);
    // coordinate descent, two sweeps: column IDFT tiles, row tiles, column DFT tiles,
    // pairs in flight, accumulator groups (a tile choice can change the best chunking).
    // Timings within 1% count as a tie, won by the smaller workspace (fewer fields in
    // flight or accumulators): it leaves more of L2 to frames running beside this one and
    // gives the finalize fewer bytes to read.
    auto consider = [&](OsprTuning t) {
        if (rc) return;
        float ms = 0.f;
        rc = measure(t, &ms);
        if (rc) return;
        const bool tie = ms <= best_t * 1.01f && ms >= best_t * 0.99f;
        const bool smaller = ospr_plan_with(H, W, N, t).total < ospr_plan_with(H, W, N, best).total;
        if ((!tie && ms < best_t) || (tie && smaller)) { best_t = ms; best = t; }
    };
    const int chunks[] = {2, 4, 8, 12, 16};
    const int groups[] = {1, 2, 4};
    for (int sweep = 0; sweep < 2 && !rc; ++sweep) {
        OsprTuning b = best;
        for (int v = 0; v < col_variants(H); ++v)
            if (v != b.ci_v) { OsprTuning t = b; t.ci_v = v; consider(t); }
        b = best;
        for (int v = 0; v < row_variants(W); ++v)
            if (v != b.row_v) { OsprTuning t = b; t.row_v = v; consider(t); }
        b = best;
        for (int v = 0; v < col_variants(H); ++v)
            if (v != b.cf_v) { OsprTuning t = b; t.cf_v = v; consider(t); }
        b = best;
        for (int c : chunks)
            if (c <= npairs && c != b.chunk) { OsprTuning t = b; t.chunk = c; consider(t); }
        b = best;
        for (int g : groups)
            if (g != b.groups && g <= b.chunk) { OsprTuning t = b; t.groups = g; consider(t); }
    }
    release();
    if (rc) {
        tuning_install(H, W, before, false);
        return rc;
    }
    tuning_install(H, W, best, true);
    if (best_ms) *best_ms = best_t;
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
    pl->ci_v = 0;
    pl->cf_v = 0;
    pl->row_v = 0;
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
    a.tc05b = nullptr;
    a.zbuf = static_cast<float2*>(scratch);
    a.sacc = reinterpret_cast<float*>(static_cast<char*>(scratch) + pl.z_bytes);
    a.groups = pl.groups;
    a.bits = d_holo_bits;
    a.tw = tab.twiddles;
    a.cs256 = tab.cs256;
    a.fresnel = 0;
    a.chirp_y = a.chirp_x = nullptr;
    // every scratch byte a kernel reads was written earlier in this call (the first chunk
    // overwrites the accumulator), so nothing needs clearing between calls
    if ((rc = ospr_run(a, pl, d_replay != nullptr, d_replay, reinterpret_cast<cudaStream_t>(s)))) return rc;
    ospr_design_rules(L, N, H, W);
    return HOLO_OK;
}
