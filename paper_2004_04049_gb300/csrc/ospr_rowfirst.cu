// ospr_rowfirst.cu - the row-first pass layout of OSPR (same method as ospr_kernels.cuh:
// paper Sections 2, 3, 5.2; the 2D transforms of Eq. 1 and Eq. 2 are separable, so their
// 1D passes may run in either order).
//
// Every line FFT here is held by the threads of one line with warp-level exchanges only
// (lines of up to 1024 points are one warp); the field changes orientation in shared
// memory once per pass instead of synchronising the block between FFT stages:
//   row_gen   rows:    build Z = E^h_{s0} + i E^h_{s1} from the target and the table
//                      (mirror rows r and H - r share a CTA, so each pixel pair {p, -p}
//                      is drawn once), row IDFT, store the field transposed (Zt[c][r])
//   row       lines of Zt (the image columns): column IDFT, binarise (bit words of 32
//                      consecutive rows of a column), column DFT of h_{s0} + i h_{s1};
//                      the row pass of ospr_kernels.cuh run on the transposed field
//   row_acc   rows:    load the field back from Zt (transposed through shared memory),
//                      row DFT, S += |Z|^2 over the pairs of a group
// then bits_transpose turns the column-oriented bit words into the row-major packing
// (bit j of word w = pixel 32w + j) and the finalize of ospr.cu symmetrises S.
#include "ospr_kernels.cuh"

namespace holo {

// ---------------------------------------------------------------- pass 1 ----
// Row length NR: R values per thread, T = NR/R threads per row, HL mirror row pairs per
// CTA (2*HL rows). HL >= 4 makes each transposed store segment 32 bytes.
template <int NR> struct RowGenCfg;
template <> struct RowGenCfg<64>   { static constexpr int R = 2,  HL = 8; };
template <> struct RowGenCfg<128>  { static constexpr int R = 4,  HL = 8; };
template <> struct RowGenCfg<256>  { static constexpr int R = 8,  HL = 8; };
template <> struct RowGenCfg<512>  { static constexpr int R = 16, HL = 4; };
template <> struct RowGenCfg<1024> { static constexpr int R = 32, HL = 4; };
template <> struct RowGenCfg<2048> { static constexpr int R = 32, HL = 4; };
template <> struct RowGenCfg<4096> { static constexpr int R = 32, HL = 2; };

template <int NR>
constexpr int rowgen_threads() { return 2 * RowGenCfg<NR>::HL * (NR / RowGenCfg<NR>::R); }
// line buffers: a stride of 16/LPR (mod 16) float2 spreads the transposed read of LPR
// lines x (16/LPR) columns of a half-warp over 16 different bank pairs
template <int NR>
constexpr int rowgen_stride() { return col_line_stride(NR, RowGenCfg<NR>::R, 2 * RowGenCfg<NR>::HL); }
template <int NR>
constexpr size_t rowgen_smem_bytes() {
    return sizeof(float2) * (kCsSmemEntries + size_t(2 * RowGenCfg<NR>::HL) * rowgen_stride<NR>());
}

// Rows of CTA b: lines j < HL take rows u = b*HL + j, lines HL + j their mirrors H - u;
// for u = 0 the self-mirrored rows 0 and H/2 (each its own partner).
template <int HL>
__device__ __forceinline__ void mirror_row(int b, int line, int H, int& row, int& partner) {
    const int u = b * HL + (line & (HL - 1));
    const bool second = line >= HL;
    if (u == 0) {
        row = second ? H / 2 : 0;
        partner = line;
    } else {
        row = second ? H - u : u;
        partner = second ? line - HL : line + HL;
    }
}

// Builds slots of v for image row r (element e of thread t = column c = t + T*e). The
// mirror pixel of (r, c) is (H - r mod H, W - c mod W); for thread t > 0 the mirror of
// slot e is slot R-1-e of thread T - t in the partner row, for thread 0 it is slot
// (R - e) mod R of thread 0. Threads with t > 0 generate slots 0..R/2-1 and hand the
// mirror values over through the partner row's line buffer; thread 0 generates slots
// 0..R/2 (slots 0 and R/2 lie on columns 0 and W/2, whose mirrors the partner row's
// thread 0 generates itself). SINGLE (the last sub-frame of an odd N) builds all slots.
template <int NR, int MODE, bool SINGLE>
__device__ __forceinline__ void ospr_build_row(float2 (&v)[RowGenCfg<NR>::R], const OsprArgs& a,
                                               const float2* cs, float2* xline, int t, int r, int s0) {
    constexpr int R = RowGenCfg<NR>::R, T = NR / R;
    constexpr int EG = SINGLE ? R : R / 2;
    constexpr int B = EG < kBatch ? EG : kBatch;
    const int H = a.H;
    const int rm = (H - r) & (H - 1);
    const float* trow = a.target + size_t(r) * NR;
    const float* tmir = a.target + size_t(rm) * NR;
    const int sh = a.ps.cs_shift;
    const SubframeDraw d0 = subframe_draw(a.ps, s0);
    const SubframeDraw d1 = subframe_draw(a.ps, SINGLE ? s0 : s0 + 1);
    // table mode: the index of (r, c) advances by D = T mod L per slot, the mirror's
    // (rm, W - c) falls by D; the mirror of column 0 (t = 0, e = 0) is column 0
    const uint32_t L = a.ps.L;
    const uint64_t fm = a.ps.fm;
    uint32_t D = 0, i0 = 0, i1 = 0, m0 = 0, m1 = 0, z0 = 0, z1 = 0;
    if constexpr (MODE == kPhaseTable) {
        D = uint32_t(T) % L;
        const uint32_t p0 = uint32_t(r) * uint32_t(NR) + uint32_t(t);
        const uint32_t q0 = uint32_t(rm) * uint32_t(NR) + uint32_t(NR - t);
        i0 = fastmod_u32(d0.base_mod + p0, fm, L);
        i1 = fastmod_u32(d1.base_mod + p0, fm, L);
        m0 = fastmod_u32(d0.base_mod + q0, fm, L);
        m1 = fastmod_u32(d1.base_mod + q0, fm, L);
        z0 = fastmod_u32(d0.base_mod + uint32_t(rm) * uint32_t(NR), fm, L);
        z1 = fastmod_u32(d1.base_mod + uint32_t(rm) * uint32_t(NR), fm, L);
    }
    const int gshift = 64 - a.ps.bits;
    // packed codes of (s0, p), (s0, -p), (s1, p), (s1, -p), one byte each, of column c
    auto codes_of = [&](int e, int c, int cm) -> uint32_t {
        if constexpr (MODE == kPhaseTable) {
            const uint32_t jm0 = (e == 0 && t == 0) ? z0 : m0;
            const uint32_t jm1 = (e == 0 && t == 0) ? z1 : m1;
            uint32_t w = __ldg(a.ps.codes + i0);
            if constexpr (!SINGLE) {
                w |= uint32_t(__ldg(a.ps.codes + jm0)) << 8;
                w |= uint32_t(__ldg(a.ps.codes + i1)) << 16;
                w |= uint32_t(__ldg(a.ps.codes + jm1)) << 24;
            }
            i0 += D; i0 -= (i0 >= L) ? L : 0u;
            i1 += D; i1 -= (i1 >= L) ? L : 0u;
            m0 = (m0 >= D) ? m0 - D : m0 + (L - D);
            m1 = (m1 >= D) ? m1 - D : m1 + (L - D);
            return w;
        } else if constexpr (MODE == kPhaseGenerator) {
            const uint64_t p = uint64_t(r) * uint64_t(NR) + uint64_t(c);
            const uint64_t pm = uint64_t(rm) * uint64_t(NR) + uint64_t(cm);
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
    // Hermitian parts E(k) + conj(E(-k)) of both sub-frames at column c
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
            const int c = t + T * e;
            const int cm = (NR - c) & (NR - 1);
            tp[k] = __ldg(trow + c);
            tm[k] = SINGLE ? 0.f : __ldg(tmir + cm);
            pk[k] = codes_of(e, c, cm);
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
                    const int cm = (NR - (t + T * e)) & (NR - 1);
                    xline[pad_index<R>(cm)] = make_float2(h0.x + h1.y, h1.x - h0.y);
                }
            }
        }
    }
    if constexpr (!SINGLE) {
        if (t == 0) {   // column W/2: its mirror is column W/2 of the partner row, built there
            constexpr int e = R / 2;
            const int c = T * e;
            const float tp = __ldg(trow + c);
            const float tm = __ldg(tmir + c);
            float2 h0, h1;
            hermitian(tp, tm, codes_of(e, c, c), h0, h1);
            v[e] = make_float2(h0.x - h1.y, h0.y + h1.x);
        }
    }
}

template <int NR>
__global__ void __launch_bounds__(rowgen_threads<NR>(), rowgen_threads<NR>() <= 256 ? 2 : 1)
k_ospr_row_gen(OsprArgs a) {
    constexpr int R = RowGenCfg<NR>::R, HL = RowGenCfg<NR>::HL, LPR = 2 * HL, T = NR / R;
    constexpr int S = rowgen_stride<NR>();
    constexpr bool BLOCK = T > 32;
    static_assert(stage_count(NR, R) > 1, "the line FFT's opening barrier guards the exchange buffer");
    extern __shared__ float2 sm[];
    float2* cs = sm;
    float2* lines = sm + kCsSmemEntries;
    load_cs_table(cs, a.cs256);
    pdl_wait();   // the table and target may be written by the previous kernel
    __syncthreads();

    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int H = a.H;
    int r, pl;
    mirror_row<HL>(blockIdx.x, line, H, r, pl);
    bool single;   // uniform over the CTA
    const int s0 = slot_subframe(a, int(blockIdx.y), single);
    float2* own = lines + line * S;
    float2* xline = lines + pl * S;
    float2 v[R];
    if (a.ps.mode == kPhaseTable) {
        if (single) ospr_build_row<NR, kPhaseTable, true>(v, a, cs, xline, t, r, s0);
        else ospr_build_row<NR, kPhaseTable, false>(v, a, cs, xline, t, r, s0);
    } else if (a.ps.mode == kPhaseGenerator) {
        if (single) ospr_build_row<NR, kPhaseGenerator, true>(v, a, cs, xline, t, r, s0);
        else ospr_build_row<NR, kPhaseGenerator, false>(v, a, cs, xline, t, r, s0);
    } else {
        if (single) ospr_build_row<NR, kPhaseFlat, true>(v, a, cs, xline, t, r, s0);
        else ospr_build_row<NR, kPhaseFlat, false>(v, a, cs, xline, t, r, s0);
    }
    if (!single) {
        __syncthreads();
#pragma unroll
        for (int e = R / 2; e < R; ++e)
            if (t > 0 || e > R / 2) v[e] = own[pad_index<R>(t + T * e)];
    }
    line_fft<NR, R, +1, BLOCK>(v, own, t, a.tw);

    // transposed store: the rows of the CTA go to Zt[c][row] through the line buffers
    line_sync<BLOCK>();   // the last FFT stage's reads of the buffer are done
#pragma unroll
    for (int e = 0; e < R; ++e) own[pad_index<R>(t + T * e)] = v[e];
    __syncthreads();
    pdl_trigger();
    // element k of this thread: line j = tid mod LPR (fixed), column c = tid / LPR + k*T;
    // a warp covers 32/LPR columns of every line, so each column's rows of the first and of
    // the second half of the CTA land in two contiguous segments
    const int j = int(threadIdx.x) % LPR, cj = int(threadIdx.x) / LPR;
    int row, unused;
    mirror_row<HL>(blockIdx.x, j, H, row, unused);
    const float2* src = lines + j * S;
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = src[pad_index<R>(cj + k * T)];
    float2* zt = a.zbuf + size_t(blockIdx.y) * size_t(H) * NR + size_t(cj) * H + row;
#pragma unroll
    for (int k = 0; k < R; ++k) zt[size_t(k) * T * H] = v[k];
}

// ---------------------------------------------------------------- pass 3 ----
// LPR consecutive rows per CTA (32-byte transposed load segments for LPR >= 4).
template <int NR> struct RowAccCfg;
template <> struct RowAccCfg<64>   { static constexpr int R = 2,  LPR = 16; };
template <> struct RowAccCfg<128>  { static constexpr int R = 4,  LPR = 16; };
template <> struct RowAccCfg<256>  { static constexpr int R = 8,  LPR = 8; };
template <> struct RowAccCfg<512>  { static constexpr int R = 16, LPR = 4; };
template <> struct RowAccCfg<1024> { static constexpr int R = 32, LPR = 4; };
template <> struct RowAccCfg<2048> { static constexpr int R = 32, LPR = 4; };
template <> struct RowAccCfg<4096> { static constexpr int R = 32, LPR = 2; };

template <int NR>
constexpr int rowacc_threads() { return RowAccCfg<NR>::LPR * (NR / RowAccCfg<NR>::R); }
template <int NR>
constexpr int rowacc_stride() { return col_line_stride(NR, RowAccCfg<NR>::R, RowAccCfg<NR>::LPR); }
template <int NR>
constexpr size_t rowacc_smem_bytes() { return sizeof(float2) * size_t(RowAccCfg<NR>::LPR) * rowacc_stride<NR>(); }

// registers: R accumulators and R complex values per thread; capped so that 512 threads
// (four CTAs of 128 at length 1024) share an SM
template <int NR>
__global__ void __launch_bounds__(rowacc_threads<NR>(), 512 / rowacc_threads<NR>() > 0 ? 512 / rowacc_threads<NR>() : 1)
k_ospr_row_acc(OsprArgs a) {
    constexpr int R = RowAccCfg<NR>::R, LPR = RowAccCfg<NR>::LPR, T = NR / R;
    constexpr int S = rowacc_stride<NR>();
    static_assert((LPR * T) % LPR == 0 && 32 % LPR == 0, "a warp covers whole columns of the tile");
    extern __shared__ float2 sm[];
    float2* lines = sm;
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int H = a.H;
    const int r0 = blockIdx.x * LPR;
    const size_t P = size_t(H) * NR;
    float2* own = lines + line * S;
    pdl_wait();
    float acc[R];
#pragma unroll
    for (int e = 0; e < R; ++e) acc[e] = 0.f;
    // transposed load: element k of this thread is line jl = tid mod LPR (fixed), column
    // cl = tid / LPR + k*T (NT/LPR = T), i.e. Zt[cl][r0 + jl]
    const int jl = int(threadIdx.x) % LPR, cl = int(threadIdx.x) / LPR;
    float2* dst = lines + jl * S;
    for (int j = blockIdx.y; j < a.pairs; j += a.groups) {
        const float2* zt = a.zbuf + size_t(j) * P + size_t(cl) * H + r0 + jl;
        float2 v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = zt[size_t(k) * T * H];
        __syncthreads();   // the previous pair's FFT no longer reads the buffers
#pragma unroll
        for (int k = 0; k < R; ++k) dst[pad_index<R>(cl + k * T)] = v[k];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < R; ++e) v[e] = own[pad_index<R>(t + T * e)];
        line_fft<NR, R, -1, (T > 32)>(v, own, t, a.tw);
#pragma unroll
        for (int e = 0; e < R; ++e) acc[e] = fmaf(v[e].x, v[e].x, fmaf(v[e].y, v[e].y, acc[e]));
    }
    pdl_trigger();
    float* Sg = a.sacc + size_t(blockIdx.y) * P + size_t(r0 + line) * NR;
#pragma unroll
    for (int e = 0; e < R; ++e) {
        const int i = t + T * e;
        Sg[i] = a.accumulate ? Sg[i] + acc[e] : acc[e];
    }
}

// ------------------------------------------------------- bit transposition ----
// in: per sub-frame the bits of the transposed image (line c of H bits: word c*H/32 + r/32,
// bit r mod 32 is pixel (r, c)); out: the row-major packing (word r*W/32 + c/32, bit
// c mod 32). One CTA transposes a TB x TB tile through shared memory; each warp turns a
// 32 x 32 block around with 32 ballots.
template <int TB>
__global__ void __launch_bounds__(256)
k_bits_transpose(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int H, int W) {
    constexpr int NW = TB / 32;
    __shared__ uint32_t tin[TB][NW + 1];    // [c][word of r]
    __shared__ uint32_t tout[TB][NW + 1];   // [r][word of c]
    const size_t plane = size_t(H) * W / 32;
    const uint32_t* src = in + size_t(blockIdx.z) * plane;
    uint32_t* dst = out + size_t(blockIdx.z) * plane;
    const int c0 = blockIdx.x * TB, r0 = blockIdx.y * TB;
    const int wl = H / 32, wr = W / 32;
    pdl_wait();
    for (int i = threadIdx.x; i < TB * NW; i += blockDim.x) {
        const int c = i / NW, w = i % NW;
        tin[c][w] = src[size_t(c0 + c) * wl + r0 / 32 + w];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int blk = warp; blk < NW * NW; blk += blockDim.x / 32) {
        const int bc = blk / NW, br = blk % NW;
        const uint32_t x = tin[32 * bc + lane][br];   // column 32bc + lane, rows 32br .. 32br + 31
        uint32_t mine = 0;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const uint32_t b = __ballot_sync(0xffffffffu, (x >> i) & 1u);
            if (lane == i) mine = b;
        }
        tout[32 * br + lane][bc] = mine;              // row 32br + lane, columns 32bc .. 32bc + 31
    }
    __syncthreads();
    pdl_trigger();
    for (int i = threadIdx.x; i < TB * NW; i += blockDim.x) {
        const int r = i / NW, w = i % NW;
        dst[size_t(r0 + r) * wr + c0 / 32 + w] = tout[r][w];
    }
}

// --------------------------------------------------------------- launchers ----
template <int NR>
static int launch_row_gen(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = rowgen_smem_bytes<NR>();
    int rc = ensure_smem((const void*)k_ospr_row_gen<NR>, smem, &mask);
    if (rc) return rc;
    const dim3 grid(a.H / (2 * RowGenCfg<NR>::HL), a.pairs);
    Launch ln("ospr_row_gen", st);
    const cudaError_t le = launch_pdl(k_ospr_row_gen<NR>, grid, dim3(rowgen_threads<NR>()), smem, st, a);
    return ln.done("ospr_row_gen launch", le);
}

template <int NR>
static int launch_row_acc(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = rowacc_smem_bytes<NR>();
    int rc = ensure_smem((const void*)k_ospr_row_acc<NR>, smem, &mask);
    if (rc) return rc;
    const dim3 grid(a.H / RowAccCfg<NR>::LPR, a.groups);
    Launch ln("ospr_row_acc", st);
    const cudaError_t le = launch_pdl(k_ospr_row_acc<NR>, grid, dim3(rowacc_threads<NR>()), smem, st, a);
    return ln.done("ospr_row_acc launch", le);
}

#define HOLO_ROWFIRST_SWITCH(n, F)                                   \
    switch (n) {                                                     \
        case 64: return F<64>(a, st);                                \
        case 128: return F<128>(a, st);                              \
        case 256: return F<256>(a, st);                              \
        case 512: return F<512>(a, st);                              \
        case 1024: return F<1024>(a, st);                            \
        case 2048: return F<2048>(a, st);                            \
        case 4096: return F<4096>(a, st);                            \
        default: return fail(HOLO_EUNSUPPORTED, "row length %d", n); \
    }

int ospr_run_row_gen(const OsprArgs& a, cudaStream_t st) { HOLO_ROWFIRST_SWITCH(a.W, launch_row_gen) }
int ospr_run_row_acc(const OsprArgs& a, cudaStream_t st) { HOLO_ROWFIRST_SWITCH(a.W, launch_row_acc) }

int ospr_run_bits_transpose(const uint32_t* bits_t, uint32_t* bits, int H, int W, int N, cudaStream_t st) {
    Launch ln("ospr_bits_transpose", st);
    cudaError_t le;
    if (H >= 128 && W >= 128)
        le = launch_pdl(k_bits_transpose<128>, dim3(W / 128, H / 128, N), dim3(256), 0, st, bits_t, bits, H, W);
    else
        le = launch_pdl(k_bits_transpose<64>, dim3(W / 64, H / 64, N), dim3(256), 0, st, bits_t, bits, H, W);
    return ln.done("ospr_bits_transpose launch", le);
}

}  // namespace holo
