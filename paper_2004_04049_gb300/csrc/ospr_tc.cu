// ospr_tc.cu - launchers of the OSPR passes whose radix-32 DFT stages run on the tensor
// cores (split fp16 or bf16 operands, float32 accumulation), for line lengths 1024 and 2048:
// every pass of 1024-point lines on tcgen05 (accumulators in tensor memory), the passes of
// 2048-point lines on mma.sync (tc_dft.cuh).
#include "ospr_kernels.cuh"
#include "tc05_dft.cuh"

namespace holo {

// ---------------------------------------------------------------- tcgen05 ----
// Column DFT + accumulate pass (k_ospr_col_fft) for 1024-point columns with both radix-32
// stages on tcgen05 (tc05_dft.cuh). Tile: 8 columns x 32 threads = 256 threads, i.e. two
// MMA groups of 128 sub-lines. Shared memory: the DFT matrix (hi, lo) for the forward
// direction of this pass, then the padded line buffers, whose first 64 KiB also hold the
// groups' A tiles, then two mbarriers.
static __device__ int g_tc05_dft_fault;

constexpr int kTc05Lpc = ColCfg<1024, 1>::LPC;
constexpr int kTc05Threads = (1024 / 32) * kTc05Lpc;
constexpr size_t kTc05LineBytes = sizeof(float2) * kTc05Lpc * col_stride<1024, 1>();
constexpr size_t kTc05Smem = 1024 + 2 * kTc05BBytes + kTc05LineBytes + 16;
static_assert(kTc05Threads == 256 && 2 * 2 * kTc05TileBytes <= kTc05LineBytes, "tcgen05 column tile");

template <int PREC>
__global__ void __launch_bounds__(kTc05Threads, 2) k_ospr_col_fft_tc05(OsprArgs a) {
    constexpr int NC = 1024, R = 32, LPC = kTc05Lpc, T = NC / R, S = col_stride<1024, 1>();
    extern __shared__ uint8_t smraw[];
    __shared__ uint32_t s_tmem;
    const uint32_t raw = static_cast<uint32_t>(__cvta_generic_to_shared(smraw));
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* const sm = smraw + (base - raw);
    float2* lines = reinterpret_cast<float2*>(sm + 2 * kTc05BBytes);
    const uint32_t lines_u32 = base + 2 * kTc05BBytes;
    const uint32_t bar0 = lines_u32 + uint32_t(kTc05LineBytes);
    const int tid = threadIdx.x;
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(
                         static_cast<uint32_t>(__cvta_generic_to_shared(&s_tmem)))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0 + 8) : "memory");
    }
    // the inverse-direction matrix: direction index 0 (-1) of this precision's table
    const uint4* bsrc = reinterpret_cast<const uint4*>(a.tc05b);
    uint4* bdst = reinterpret_cast<uint4*>(sm);
    for (int i = tid; i < 2 * kTc05BBytes / 16; i += kTc05Threads) bdst[i] = __ldg(bsrc + i);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

    Tc05Group g;
    const int grp = tid >> 7;
    g.row = tid & 127;
    g.a_hi = lines_u32 + uint32_t(grp) * 2u * kTc05TileBytes;
    g.a_lo = g.a_hi + kTc05TileBytes;
    g.b_hi = base;
    g.b_lo = base + kTc05BBytes;
    g.bar = bar0 + 8u * grp;
    g.tmem = s_tmem + 64u * grp;
    g.phase = 0;
    g.fault = &g_tc05_dft_fault;

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
        line_fft_1024_tc05<-1, PREC>(v, lines + lc * S, t, a.tw, g);
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
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if ((tid >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(s_tmem) : "memory");
}

template <int PREC>
static int launch_col_fft_tc05(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    int rc = ensure_smem((const void*)k_ospr_col_fft_tc05<PREC>, kTc05Smem, &mask);
    if (rc) return rc;
    dim3 grid(a.W / kTc05Lpc, a.groups);
    Launch ln("ospr_col_fft", st);
    const cudaError_t le = launch_pdl(k_ospr_col_fft_tc05<PREC>, grid, dim3(kTc05Threads), kTc05Smem, st, a);
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

// TMEM, mbarriers and the B tiles of a tcgen05 pass, set up by every thread of a 256-thread
// CTA (two MMA groups of 128): `nb` B tiles (hi/lo pairs of directions) are copied from
// `bsrc` to the start of shared memory; the A tiles of group grp live at `atiles` +
// grp * 2 * kTc05TileBytes and the two mbarriers at `bars`.
__device__ __forceinline__ void tc05_setup(uint32_t* s_tmem, const uint8_t* bsrc, uint8_t* bdst, int nb) {
    const int tid = threadIdx.x;
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(
                         static_cast<uint32_t>(__cvta_generic_to_shared(s_tmem)))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    const uint4* src = reinterpret_cast<const uint4*>(bsrc);
    uint4* dst = reinterpret_cast<uint4*>(bdst);
    for (int i = tid; i < nb * kTc05BBytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
}
__device__ __forceinline__ Tc05Group tc05_group(uint32_t atiles, uint32_t bars, uint32_t tmem) {
    Tc05Group g;
    const int grp = threadIdx.x >> 7;
    g.row = threadIdx.x & 127;
    g.a_hi = atiles + uint32_t(grp) * 2u * kTc05TileBytes;
    g.a_lo = g.a_hi + kTc05TileBytes;
    g.b_hi = g.b_lo = 0;
    g.bar = bars + 8u * grp;
    g.tmem = tmem + 64u * grp;
    g.phase = 0;
    g.fault = &g_tc05_dft_fault;
    return g;
}
__device__ __forceinline__ void tc05_teardown(uint32_t tmem) {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(tmem) : "memory");
}

// Build + column IDFT pass (k_ospr_col_ifft) for 1024-point columns with both radix-32
// stages on tcgen05. Tile: 8 columns (4 mirror pairs) x 32 threads. Shared memory: the
// inverse-direction DFT matrix (hi, lo), the replicated cos/sin table, the padded line
// buffers (whose first 64 KiB also hold the groups' A tiles), two mbarriers.
constexpr size_t kTc05CiSmem = 1024 + 2 * kTc05BBytes + sizeof(float2) * kCsSmemEntries + kTc05LineBytes + 16;

template <int PREC>
__global__ void __launch_bounds__(kTc05Threads, 1) k_ospr_col_ifft_tc05(OsprArgs a) {
    constexpr int NC = 1024, V = 1, R = 32, LPC = kTc05Lpc, T = NC / R, S = col_stride<1024, 1>();
    extern __shared__ uint8_t smraw[];
    __shared__ uint32_t s_tmem;
    const uint32_t raw = static_cast<uint32_t>(__cvta_generic_to_shared(smraw));
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* const sm = smraw + (base - raw);
    float2* cs = reinterpret_cast<float2*>(sm + 2 * kTc05BBytes);
    float2* lines = cs + kCsSmemEntries;
    const uint32_t lines_u32 = base + 2 * kTc05BBytes + uint32_t(sizeof(float2) * kCsSmemEntries);
    const uint32_t bar0 = lines_u32 + uint32_t(kTc05LineBytes);
    const int tid = threadIdx.x;
    // the inverse direction (+1) matrix: the second pair of this precision's table
    tc05_setup(&s_tmem, a.tc05b + 2 * kTc05BBytes, sm, 2);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0 + 8) : "memory");
    }
    load_cs_table(cs, a.cs256);
    pdl_wait();   // the table and target may be written by the previous kernel
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    Tc05Group g = tc05_group(lines_u32, bar0, s_tmem);
    g.b_hi = base;
    g.b_lo = base + kTc05BBytes;

    const int lc = tid % LPC, t = tid / LPC;
    const int W = a.W;
    int c, pl;
    mirror_column<LPC>(blockIdx.x, lc, W, c, pl);
    bool single;   // uniform over the CTA
    const int s0 = slot_subframe(a, int(blockIdx.y), single);
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
    line_fft_1024_tc05<+1, PREC>(v, lines + lc * S, t, a.tw, g);
    pdl_trigger();
    float2* z = a.zbuf + size_t(blockIdx.y) * size_t(NC) * size_t(W);
#pragma unroll
    for (int e = 0; e < R; ++e) z[size_t(t + T * e) * W + c] = v[e];
    tc05_teardown(s_tmem);
}

// Row pass (row IDFT, binarise, row DFT) for 1024-point rows with every radix-32 stage on
// tcgen05. Tile: 8 rows of 32 threads (one warp per row). Shared memory: the DFT matrices
// of both directions (hi, lo), the padded line buffers (whose first 64 KiB also hold the
// groups' A tiles), two mbarriers.
constexpr int kTc05RowLines = 8;
constexpr size_t kTc05RowLineBytes = sizeof(float2) * kTc05RowLines * line_stride(1024, 32);
constexpr size_t kTc05RowSmem = 1024 + 4 * kTc05BBytes + kTc05RowLineBytes + 16;
static_assert(2 * 2 * kTc05TileBytes <= kTc05RowLineBytes && kTc05RowLineBytes % 8 == 0, "tcgen05 row tile");

template <int PREC, bool REPLAY>
__global__ void __launch_bounds__(kTc05Threads, 2) k_ospr_row_tc05(OsprArgs a) {
    constexpr int NR = 1024, R = 32, T = 32, S = line_stride(1024, 32);
    extern __shared__ uint8_t smraw[];
    __shared__ uint32_t s_tmem;
    const uint32_t raw = static_cast<uint32_t>(__cvta_generic_to_shared(smraw));
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* const sm = smraw + (base - raw);
    float2* lines = reinterpret_cast<float2*>(sm + 4 * kTc05BBytes);
    const uint32_t lines_u32 = base + 4 * kTc05BBytes;
    const uint32_t bar0 = lines_u32 + uint32_t(kTc05RowLineBytes);
    const int tid = threadIdx.x;
    tc05_setup(&s_tmem, a.tc05b, sm, 4);   // [-1 hi, -1 lo, +1 hi, +1 lo]
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0 + 8) : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    Tc05Group g = tc05_group(lines_u32, bar0, s_tmem);

    const int line = tid / T, t = tid % T;
    const int lane = tid & 31;
    const int r = blockIdx.x * kTc05RowLines + line;
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
    line_fft_1024_tc05<+1, PREC>(v, buf, t, a.tw, g);
    const size_t words = P / 32;
#pragma unroll
    for (int e = 0; e < R; ++e) {
        const bool n0 = v[e].x < 0.f;
        const bool n1 = v[e].y < 0.f;
        if (a.bits) {
            const unsigned b0 = __ballot_sync(0xffffffffu, n0);
            const unsigned b1 = __ballot_sync(0xffffffffu, n1);
            if (lane == 0) {
                const size_t w = (size_t(r) * NR + size_t(T * e)) >> 5;
                a.bits[size_t(s0) * words + w] = b0;
                if (!single) a.bits[size_t(s0 + 1) * words + w] = b1;
            }
        }
        v[e] = make_float2(n0 ? -1.f : 1.f, single ? 0.f : (n1 ? -1.f : 1.f));
    }
    if constexpr (REPLAY) {
        g.b_hi = base;
        g.b_lo = base + kTc05BBytes;
        line_fft_1024_tc05<-1, PREC>(v, buf, t, a.tw, g);
        pdl_trigger();
#pragma unroll
        for (int e = 0; e < R; ++e) z[t + T * e] = v[e];
    }
    tc05_teardown(s_tmem);
}

template <int PREC>
static int launch_col_ifft_tc05(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    int rc = ensure_smem((const void*)k_ospr_col_ifft_tc05<PREC>, kTc05CiSmem, &mask);
    if (rc) return rc;
    dim3 grid(a.W / kTc05Lpc, a.pairs);
    Launch ln("ospr_col_ifft", st);
    const cudaError_t le = launch_pdl(k_ospr_col_ifft_tc05<PREC>, grid, dim3(kTc05Threads), kTc05CiSmem, st, a);
    return ln.done("ospr_col_ifft tcgen05 launch", le);
}

template <int PREC, bool REPLAY>
static int launch_row_tc05(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    int rc = ensure_smem((const void*)k_ospr_row_tc05<PREC, REPLAY>, kTc05RowSmem, &mask);
    if (rc) return rc;
    dim3 grid(a.H / kTc05RowLines, a.pairs);
    Launch ln("ospr_row", st);
    const cudaError_t le = launch_pdl(k_ospr_row_tc05<PREC, REPLAY>, grid, dim3(kTc05Threads), kTc05RowSmem, st, a);
    return ln.done("ospr_row tcgen05 launch", le);
}

template <int NC, int PREC>
static int launch_col_ifft_tc(const OsprArgs& a, cudaStream_t st) {
    constexpr int V = kTcColVariant;
    static uint64_t mask = 0;
    constexpr size_t smem = col_ifft_smem_bytes<NC, V, PREC>();
    int rc = ensure_smem((const void*)k_ospr_col_ifft<NC, V, PREC>, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.W / ColCfg<NC, V>::LPC, a.pairs);
    Launch ln("ospr_col_ifft", st);
    const cudaError_t le = launch_pdl(k_ospr_col_ifft<NC, V, PREC>, grid, dim3((NC / ColCfg<NC, V>::R) * ColCfg<NC, V>::LPC), smem, st, a);
    return ln.done("ospr_col_ifft launch", le);
}

template <int NC, int PREC>
static int launch_col_fft_tc(const OsprArgs& a, cudaStream_t st) {
    constexpr int V = kTcColVariant;
    static uint64_t mask = 0;
    constexpr size_t smem = col_fft_smem_bytes<NC, V, PREC>();
    int rc = ensure_smem((const void*)k_ospr_col_fft<NC, V, PREC>, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.W / ColCfg<NC, V>::LPC, a.groups);
    Launch ln("ospr_col_fft", st);
    const cudaError_t le = launch_pdl(k_ospr_col_fft<NC, V, PREC>, grid, dim3((NC / ColCfg<NC, V>::R) * ColCfg<NC, V>::LPC), smem, st, a);
    return ln.done("ospr_col_fft launch", le);
}

template <int NR, int PREC, bool REPLAY>
static int launch_row_tc(const OsprArgs& a, cudaStream_t st) {
    constexpr int V = kTcRowVariant;
    static uint64_t mask = 0;
    constexpr size_t smem = row_smem_bytes<NR, V, PREC>();
    int rc = ensure_smem((const void*)k_ospr_row<NR, V, REPLAY, PREC>, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.H / RowCfg<NR, V>::LPR, a.pairs);
    Launch ln("ospr_row", st);
    const cudaError_t le = launch_pdl(k_ospr_row<NR, V, REPLAY, PREC>, grid, dim3((NR / RowCfg<NR, V>::R) * RowCfg<NR, V>::LPR), smem, st, a);
    return ln.done("ospr_row launch", le);
}

int ospr_run_col_ifft_tc(const OsprArgs& a, int prec, cudaStream_t st) {
    if (a.H == 1024) return prec == kTcBf16 ? launch_col_ifft_tc05<kTcBf16>(a, st) : launch_col_ifft_tc05<kTcFp16>(a, st);
    if (a.H == 2048) return prec == kTcBf16 ? launch_col_ifft_tc<2048, kTcBf16>(a, st) : launch_col_ifft_tc<2048, kTcFp16>(a, st);
    return fail(HOLO_EUNSUPPORTED, "tensor-core stages: column length %d", a.H);
}
int ospr_run_col_fft_tc(const OsprArgs& a, int prec, cudaStream_t st) {
    if (a.H == 1024) return prec == kTcBf16 ? launch_col_fft_tc05<kTcBf16>(a, st) : launch_col_fft_tc05<kTcFp16>(a, st);
    if (a.H == 2048) return prec == kTcBf16 ? launch_col_fft_tc<2048, kTcBf16>(a, st) : launch_col_fft_tc<2048, kTcFp16>(a, st);
    return fail(HOLO_EUNSUPPORTED, "tensor-core stages: column length %d", a.H);
}
int ospr_run_row_tc(const OsprArgs& a, int prec, bool replay, cudaStream_t st) {
    if (a.W == 1024) {
        if (prec == kTcBf16) return replay ? launch_row_tc05<kTcBf16, true>(a, st) : launch_row_tc05<kTcBf16, false>(a, st);
        return replay ? launch_row_tc05<kTcFp16, true>(a, st) : launch_row_tc05<kTcFp16, false>(a, st);
    }
    if (a.W == 2048) {
        if (prec == kTcBf16) return replay ? launch_row_tc<2048, kTcBf16, true>(a, st) : launch_row_tc<2048, kTcBf16, false>(a, st);
        return replay ? launch_row_tc<2048, kTcFp16, true>(a, st) : launch_row_tc<2048, kTcFp16, false>(a, st);
    }
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
