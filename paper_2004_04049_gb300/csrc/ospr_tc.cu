// ospr_tc.cu - the OSPR passes whose radix-32 DFT stages run on the 5th-generation tensor
// cores (tcgen05.mma: split fp16 or bf16 operands, float32 accumulators in tensor memory;
// tc05_dft.cuh), for line lengths 1024 and 2048.
//
// Shared memory of a pass, from a 1024-byte aligned base: the DFT matrices (hi, lo) of the
// directions the pass needs, the replicated cos/sin table (build pass only), the padded
// line buffers, whose first 64 KiB also hold the groups' A tiles, and two mbarriers.
#include "ospr_kernels.cuh"
#include "tc05_dft.cuh"

namespace holo {

static __device__ int g_tc05_dft_fault;

template <int N>
constexpr size_t tc05_col_fft_smem() { return 1024 + 2 * kTc05BBytes + tc05_col_line_bytes<N>() + 16; }
template <int N>
constexpr size_t tc05_col_ifft_smem() {
    return 1024 + 2 * kTc05BBytes + sizeof(float2) * kCsSmemEntries + tc05_col_line_bytes<N>() + 16;
}
template <int N>
constexpr size_t tc05_row_smem() { return 1024 + 4 * kTc05BBytes + tc05_row_line_bytes<N>() + 16; }
static_assert(tc05_lpc<1024>() == ColCfg<1024, 1>::LPC && tc05_lpc<2048>() == ColCfg<2048, 1>::LPC &&
                  ColCfg<1024, 1>::R == 32 && ColCfg<2048, 1>::R == 32,
              "the build pass uses the radix-32 column tiles of variant 1");
static_assert(tc05_col_ifft_smem<2048>() <= 227 * 1024 && tc05_row_smem<2048>() <= 227 * 1024, "shared memory");

// Build + column IDFT pass (k_ospr_col_ifft): mirror column pairs as in the float32 pass,
// both radix-32 stages on tcgen05 with the inverse-direction matrix.
template <int NC, int PREC>
__global__ void __launch_bounds__(kTc05Threads, 1) k_ospr_col_ifft_tc05(OsprArgs a) {
    constexpr int R = 32, LPC = tc05_lpc<NC>(), T = NC / R, S = tc05_col_stride<NC>();
    extern __shared__ uint8_t smraw[];
    __shared__ uint32_t s_tmem;
    uint32_t base;
    uint8_t* const sm = tc05_smem(smraw, base);
    float2* cs = reinterpret_cast<float2*>(sm + 2 * kTc05BBytes);
    float2* lines = cs + kCsSmemEntries;
    const uint32_t lines_u32 = base + 2 * kTc05BBytes + uint32_t(sizeof(float2) * kCsSmemEntries);
    const uint32_t bars = lines_u32 + uint32_t(tc05_col_line_bytes<NC>());
    // the inverse direction (+1): the second pair of this precision's matrices
    tc05_setup(&s_tmem, a.tc05b + 2 * kTc05BBytes, sm, 2, bars);
    load_cs_table(cs, a.cs256);
    pdl_wait();   // the table and target may be written by the previous kernel
    Tc05Group g = tc05_group(lines_u32, bars, &s_tmem, &g_tc05_dft_fault);
    g.b_hi = base;
    g.b_lo = base + kTc05BBytes;

    const int tid = threadIdx.x;
    const int lc = tid % LPC, t = tid / LPC;
    const int W = a.W;
    int c, pl;
    mirror_column<LPC>(blockIdx.x, lc, W, c, pl);
    bool single;   // uniform over the CTA
    const int s0 = slot_subframe(a, int(blockIdx.y), single);
    float2* xline = lines + pl * S;
    float2 v[R];
    if (a.ps.mode == kPhaseTable) {
        if (single) ospr_build_column<NC, 1, kPhaseTable, true>(v, a, cs, xline, t, c, s0);
        else ospr_build_column<NC, 1, kPhaseTable, false>(v, a, cs, xline, t, c, s0);
    } else if (a.ps.mode == kPhaseGenerator) {
        if (single) ospr_build_column<NC, 1, kPhaseGenerator, true>(v, a, cs, xline, t, c, s0);
        else ospr_build_column<NC, 1, kPhaseGenerator, false>(v, a, cs, xline, t, c, s0);
    } else {
        if (single) ospr_build_column<NC, 1, kPhaseFlat, true>(v, a, cs, xline, t, c, s0);
        else ospr_build_column<NC, 1, kPhaseFlat, false>(v, a, cs, xline, t, c, s0);
    }
    if (!single) {
        __syncthreads();
        const float2* own = lines + lc * S;
#pragma unroll
        for (int e = R / 2; e < R; ++e)
            if (t > 0 || e > R / 2) v[e] = own[pad_index<R>(t + T * e)];
    }
    // (the line FFT opens with a block barrier before its A tiles overwrite the buffers)
    line_fft_tc05<NC, +1, PREC>(v, lines + lc * S, t, a.tw, g);
    pdl_trigger();
    float2* z = a.zbuf + size_t(blockIdx.y) * size_t(NC) * size_t(W);
#pragma unroll
    for (int e = 0; e < R; ++e) z[size_t(t + T * e) * W + c] = v[e];
    tc05_teardown(s_tmem);
}

// Row pass (row IDFT, binarise, row DFT; k_ospr_row without Fresnel): one row per NR/32
// threads, both directions' matrices resident.
template <int NR, int PREC, bool REPLAY>
__global__ void __launch_bounds__(kTc05Threads, 2) k_ospr_row_tc05(OsprArgs a) {
    constexpr int R = 32, T = NR / R, LPR = tc05_lpc<NR>(), S = line_stride(NR, 32);
    extern __shared__ uint8_t smraw[];
    __shared__ uint32_t s_tmem;
    uint32_t base;
    uint8_t* const sm = tc05_smem(smraw, base);
    float2* lines = reinterpret_cast<float2*>(sm + 4 * kTc05BBytes);
    const uint32_t lines_u32 = base + 4 * kTc05BBytes;
    const uint32_t bars = lines_u32 + uint32_t(tc05_row_line_bytes<NR>());
    tc05_setup(&s_tmem, a.tc05b, sm, 4, bars);   // [-1 hi, -1 lo, +1 hi, +1 lo]
    Tc05Group g = tc05_group(lines_u32, bars, &s_tmem, &g_tc05_dft_fault);

    const int tid = threadIdx.x;
    const int line = tid / T, t = tid % T;
    const int lane = tid & 31;
    const int r = blockIdx.x * LPR + line;
    bool single;
    const int s0 = slot_subframe(a, int(blockIdx.y), single);
    const size_t P = size_t(a.H) * NR;
    float2* z = a.zbuf + size_t(blockIdx.y) * P + size_t(r) * NR;
    float2* buf = lines + line * S;
    pdl_wait();
    float2 v[R];
#pragma unroll
    for (int e = 0; e < R; ++e) v[e] = z[t + T * e];
    g.b_hi = base + 2 * kTc05BBytes;
    g.b_lo = base + 3 * kTc05BBytes;
    line_fft_tc05<NR, +1, PREC>(v, buf, t, a.tw, g);
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
        g.b_hi = base;
        g.b_lo = base + kTc05BBytes;
        line_fft_tc05<NR, -1, PREC>(v, buf, t, a.tw, g);
        pdl_trigger();
#pragma unroll
        for (int e = 0; e < R; ++e) z[t + T * e] = v[e];
    }
    tc05_teardown(s_tmem);
}

// Column DFT + accumulate pass (k_ospr_col_fft): pairs g, g + groups, ... of the chunk,
// S_g += |Z|^2, with the forward-direction matrix.
template <int NC, int PREC>
__global__ void __launch_bounds__(kTc05Threads, 2) k_ospr_col_fft_tc05(OsprArgs a) {
    constexpr int R = 32, LPC = tc05_lpc<NC>(), T = NC / R, S = tc05_col_stride<NC>();
    extern __shared__ uint8_t smraw[];
    __shared__ uint32_t s_tmem;
    uint32_t base;
    uint8_t* const sm = tc05_smem(smraw, base);
    float2* lines = reinterpret_cast<float2*>(sm + 2 * kTc05BBytes);
    const uint32_t lines_u32 = base + 2 * kTc05BBytes;
    const uint32_t bars = lines_u32 + uint32_t(tc05_col_line_bytes<NC>());
    tc05_setup(&s_tmem, a.tc05b, sm, 2, bars);   // direction -1: the first pair
    Tc05Group g = tc05_group(lines_u32, bars, &s_tmem, &g_tc05_dft_fault);
    g.b_hi = base;
    g.b_lo = base + kTc05BBytes;

    const int tid = threadIdx.x;
    const int lc = tid % LPC, t = tid / LPC;
    const int W = a.W;
    const int c = blockIdx.x * LPC + lc;
    const size_t P = size_t(NC) * W;
    pdl_wait();
    float acc[R];
#pragma unroll
    for (int e = 0; e < R; ++e) acc[e] = 0.f;
    for (int j = blockIdx.y; j < a.pairs; j += a.groups) {
        const float2* z = a.zbuf + size_t(j) * P;
        float2 v[R];
#pragma unroll
        for (int e = 0; e < R; ++e) v[e] = z[size_t(t + T * e) * W + c];
        line_fft_tc05<NC, -1, PREC>(v, lines + lc * S, t, a.tw, g);
#pragma unroll
        for (int e = 0; e < R; ++e) acc[e] = fmaf(v[e].x, v[e].x, fmaf(v[e].y, v[e].y, acc[e]));
    }
    pdl_trigger();
    float* Sacc = a.sacc + size_t(blockIdx.y) * P;
#pragma unroll
    for (int e = 0; e < R; ++e) {
        const size_t i = size_t(t + T * e) * W + c;
        Sacc[i] = a.accumulate ? Sacc[i] + acc[e] : acc[e];
    }
    tc05_teardown(s_tmem);
}

template <int NC, int PREC>
static int launch_col_ifft_tc05(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = tc05_col_ifft_smem<NC>();
    int rc = ensure_smem((const void*)k_ospr_col_ifft_tc05<NC, PREC>, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.W / tc05_lpc<NC>(), a.pairs);
    Launch ln("ospr_col_ifft", st);
    const cudaError_t le = launch_pdl(k_ospr_col_ifft_tc05<NC, PREC>, grid, dim3(kTc05Threads), smem, st, a);
    return ln.done("ospr_col_ifft tcgen05 launch", le);
}

template <int NR, int PREC, bool REPLAY>
static int launch_row_tc05(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = tc05_row_smem<NR>();
    int rc = ensure_smem((const void*)k_ospr_row_tc05<NR, PREC, REPLAY>, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.H / tc05_lpc<NR>(), a.pairs);
    Launch ln("ospr_row", st);
    const cudaError_t le = launch_pdl(k_ospr_row_tc05<NR, PREC, REPLAY>, grid, dim3(kTc05Threads), smem, st, a);
    return ln.done("ospr_row tcgen05 launch", le);
}

template <int NC, int PREC>
static int launch_col_fft_tc05(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = tc05_col_fft_smem<NC>();
    int rc = ensure_smem((const void*)k_ospr_col_fft_tc05<NC, PREC>, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.W / tc05_lpc<NC>(), a.groups);
    Launch ln("ospr_col_fft", st);
    const cudaError_t le = launch_pdl(k_ospr_col_fft_tc05<NC, PREC>, grid, dim3(kTc05Threads), smem, st, a);
    return ln.done("ospr_col_fft tcgen05 launch", le);
}

// Self-test of the bounded waits: one warp waits on an mbarrier that nothing arrives at,
// gives up after `limit` polls and records the fault exactly as the tcgen05 kernels do.
__global__ void k_wait_selftest(uint32_t limit) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = static_cast<uint32_t>(__cvta_generic_to_shared(&bar));
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(b) : "memory");
    __syncwarp();
    const bool done = tc05_wait(b, 0u, limit);
    if (!done && threadIdx.x == 0) atomicExch(&g_tc05_dft_fault, 1);
}

int ospr_tc05_fault(int* out, bool clear) {
    int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc05_dft_fault, sizeof(int));
    if (e != cudaSuccess) return cuda_status(e, "ospr_tc05_fault");
    if (clear && v) {
        const int z = 0;
        if ((e = cudaMemcpyToSymbol(g_tc05_dft_fault, &z, sizeof(int))) != cudaSuccess)
            return cuda_status(e, "ospr_tc05_fault");
    }
    *out = v;
    return HOLO_OK;
}

int ospr_run_col_ifft_tc(const OsprArgs& a, int prec, cudaStream_t st) {
    if (a.H == 1024) return prec == kTcBf16 ? launch_col_ifft_tc05<1024, kTcBf16>(a, st) : launch_col_ifft_tc05<1024, kTcFp16>(a, st);
    if (a.H == 2048) return prec == kTcBf16 ? launch_col_ifft_tc05<2048, kTcBf16>(a, st) : launch_col_ifft_tc05<2048, kTcFp16>(a, st);
    return fail(HOLO_EUNSUPPORTED, "tensor-core stages: column length %d", a.H);
}
int ospr_run_col_fft_tc(const OsprArgs& a, int prec, cudaStream_t st) {
    if (a.H == 1024) return prec == kTcBf16 ? launch_col_fft_tc05<1024, kTcBf16>(a, st) : launch_col_fft_tc05<1024, kTcFp16>(a, st);
    if (a.H == 2048) return prec == kTcBf16 ? launch_col_fft_tc05<2048, kTcBf16>(a, st) : launch_col_fft_tc05<2048, kTcFp16>(a, st);
    return fail(HOLO_EUNSUPPORTED, "tensor-core stages: column length %d", a.H);
}
template <int NR>
static int run_row_tc05(const OsprArgs& a, int prec, bool replay, cudaStream_t st) {
    if (prec == kTcBf16) return replay ? launch_row_tc05<NR, kTcBf16, true>(a, st) : launch_row_tc05<NR, kTcBf16, false>(a, st);
    return replay ? launch_row_tc05<NR, kTcFp16, true>(a, st) : launch_row_tc05<NR, kTcFp16, false>(a, st);
}
int ospr_run_row_tc(const OsprArgs& a, int prec, bool replay, cudaStream_t st) {
    if (a.W == 1024) return run_row_tc05<1024>(a, prec, replay, st);
    if (a.W == 2048) return run_row_tc05<2048>(a, prec, replay, st);
    return fail(HOLO_EUNSUPPORTED, "tensor-core stages: row length %d", a.W);
}

}  // namespace holo

using namespace holo;

extern "C" int holo_wait_selftest(int limit, holo_stream_t s) {
    clear_error();
    if (limit < 1 || limit > (1 << 24)) return fail(HOLO_EINVAL, "holo_wait_selftest: limit %d out of [1, 2^24]", limit);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    Launch ln("wait_selftest", st);
    k_wait_selftest<<<1, 32, 0, st>>>(uint32_t(limit));
    int rc = ln.done("wait_selftest launch");
    if (rc) return rc;
    if ((rc = cuda_status(cudaStreamSynchronize(st), "holo_wait_selftest"))) return rc;
    int f = 0;
    if ((rc = ospr_tc05_fault(&f, false))) return rc;
    return f ? fail(HOLO_ETIMEOUT, "holo_wait_selftest: the wait gave up after %d polls", limit) : HOLO_OK;
}
