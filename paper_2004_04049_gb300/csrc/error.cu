// error.cu - replay error of Section 5.2 / Eq. 3 with the intensity-domain,
// optimal-scale reading: alpha = sum(I T^2)/sum(I^2), mse = sum((alpha I - T^2)^2)/P,
// nmse = sum((alpha I - T^2)^2)/sum(T^4).
//
// One pass over the pixels. The squared error at the global alpha needs alpha first, so
// every block b takes its own scale a_b = sum_b(I T^2)/sum_b(I^2) from its 4096 pixels
// (held in registers) and forms, besides its shares of sum I T^2, sum I^2, sum T^4 and the
// pixel count,
//     S1_b = sum_b (a_b I - T^2)^2,   S2_b = sum_b I (a_b I - T^2),
// and the block that finishes last (a completion counter, no waiting) reduces the blocks
// in block order and uses the exact identity
//     sum (alpha I - T^2)^2 = sum_b [S1_b + 2 (alpha - a_b) S2_b + (alpha - a_b)^2 sum_b I^2]
// (expand (a_b I - T^2) + (alpha - a_b) I). Every term is a sum of squares or carries the
// small factor alpha - a_b (S2_b vanishes at a_b up to rounding), so nothing cancels the
// way the one-pass expansion alpha^2 sum I^2 - 2 alpha sum I T^2 + sum T^4 does.
// Each thread forms its terms with single-rounding fmaf in float32 over its 16 pixels;
// every sum across threads, warps and blocks is float-float (about 48 significant bits,
// ffloat.cuh) in a fixed order, so results are bit-reproducible, and only the three
// reported values are converted to float64. Reads 8 bytes per pixel once (+1 with a
// mask); at 1024^2 the block reductions and the last block's combination, not the bytes,
// take most of the time.
#include "ffloat.cuh"
#include "runtime.h"

namespace holo {

constexpr int kErrThreads = 256;
constexpr int kErrPix = 16;                             // pixels per thread
constexpr int kErrBlockPix = kErrThreads * kErrPix;     // pixels per block
constexpr int kErrParts = 7;                            // partials per block, see below

static int err_blocks(int64_t P) {
    const int64_t nb = (P + kErrBlockPix - 1) / kErrBlockPix;
    return int(nb < 1 ? 1 : nb);
}

// Block b owns pixels [4096 b, 4096 b + 4096). With 16-byte aligned inputs (and a pixel
// count divisible by 4) thread t reads the float4 groups 1024 b + 256 k + t (k < 4), else
// the single pixels 4096 b + 256 k + t (k < 16); both are coalesced. Pixels past P read
// as I = T = 0 with mask 0.
struct ErrPixels {
    float i[kErrPix], t[kErrPix], m[kErrPix];
};

__device__ __forceinline__ void err_gather(const float* __restrict__ I, const float* __restrict__ T,
                                           const uint8_t* __restrict__ mask, int64_t P, bool vec, ErrPixels& x) {
    const int64_t b = blockIdx.x;
    if (vec) {
        const int64_t P4 = P / 4;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t g = b * (kErrBlockPix / 4) + k * kErrThreads + threadIdx.x;
            const bool in = g < P4;
            const float4 iv = in ? __ldg(reinterpret_cast<const float4*>(I) + g) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 tv = in ? __ldg(reinterpret_cast<const float4*>(T) + g) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float w = in ? 1.f : 0.f;
            float4 mv = make_float4(w, w, w, w);
            if (mask && in) {
                const uchar4 m = reinterpret_cast<const uchar4*>(mask)[g];
                mv = make_float4(m.x ? 1.f : 0.f, m.y ? 1.f : 0.f, m.z ? 1.f : 0.f, m.w ? 1.f : 0.f);
            }
            x.i[4 * k] = iv.x; x.i[4 * k + 1] = iv.y; x.i[4 * k + 2] = iv.z; x.i[4 * k + 3] = iv.w;
            x.t[4 * k] = tv.x; x.t[4 * k + 1] = tv.y; x.t[4 * k + 2] = tv.z; x.t[4 * k + 3] = tv.w;
            x.m[4 * k] = mv.x; x.m[4 * k + 1] = mv.y; x.m[4 * k + 2] = mv.z; x.m[4 * k + 3] = mv.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kErrPix; ++k) {
            const int64_t p = b * kErrBlockPix + k * kErrThreads + threadIdx.x;
            const bool in = p < P;
            x.i[k] = in ? I[p] : 0.f;
            x.t[k] = in ? T[p] : 0.f;
            x.m[k] = in ? (mask ? (mask[p] ? 1.f : 0.f) : 1.f) : 0.f;
        }
    }
}

// partials laid out [k][nb]: k = 0 sum I T^2, 1 sum I^2, 2 sum T^4, 3 count, 4 S1, 5 S2,
// 6 a_b (as {a_b, 0}); *done must be 0 at launch (the host clears it)
__global__ void __launch_bounds__(kErrThreads)
k_replay_error(const float* __restrict__ I, const float* __restrict__ T, const uint8_t* __restrict__ mask,
               int64_t P, ff* part, unsigned* done, double* __restrict__ d_out) {
    __shared__ ff sm[32 * 4];
    __shared__ float s_scale;
    __shared__ ff s_alpha;
    __shared__ bool s_last;
    const int nb = gridDim.x;
    const bool vec = (P % 4 == 0) && ((reinterpret_cast<uintptr_t>(I) | reinterpret_cast<uintptr_t>(T) |
                                       reinterpret_cast<uintptr_t>(mask)) & 15) == 0;
    ErrPixels x;
    err_gather(I, T, mask, P, vec, x);
    // this block's sums and its own scale a_b
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < kErrPix; ++k) {
        x.t[k] = x.t[k] * x.t[k] * x.m[k];   // T^2, masked
        x.i[k] = x.i[k] * x.m[k];            // I, masked
        acc[0] = fmaf(x.i[k], x.t[k], acc[0]);
        acc[1] = fmaf(x.i[k], x.i[k], acc[1]);
        acc[2] = fmaf(x.t[k], x.t[k], acc[2]);
        acc[3] += x.m[k];
    }
    ff b4[4];
    block_sums_ff<4>(acc, b4, sm);
    if (threadIdx.x == 0) {
        s_scale = b4[1].hi > 0.f ? ff_div(b4[0], b4[1]).hi : 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) part[size_t(k) * nb + blockIdx.x] = b4[k];
    }
    __syncthreads();
    const float ab = s_scale;
    float acc2[2] = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < kErrPix; ++k) {
        const float d = fmaf(ab, x.i[k], -x.t[k]);
        acc2[0] = fmaf(d, d, acc2[0]);
        acc2[1] = fmaf(x.i[k], d, acc2[1]);
    }
    ff b2[2];
    block_sums_ff<2>(acc2, b2, sm);
    // publish this block's partials; the block whose increment completes the count reduces
    // them (threadfence reduction: every other block fenced its stores before its
    // increment, and the last block reads the partials through L2)
    if (threadIdx.x == 0) {
        part[size_t(4) * nb + blockIdx.x] = b2[0];
        part[size_t(5) * nb + blockIdx.x] = b2[1];
        part[size_t(6) * nb + blockIdx.x] = ff_make(ab);
        __threadfence();
        s_last = atomicAdd(done, 1u) == unsigned(nb - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const float2* p2 = reinterpret_cast<const float2*>(part);
    auto at = [&](int k, int j) {
        const float2 q = __ldcg(p2 + size_t(k) * nb + j);
        return ff{q.x, q.y};
    };
    // global sums: thread t adds blocks t, t + 256, ... in order, then the threads' sums in
    // a fixed order
    ff g[4] = {ff_make(0.f), ff_make(0.f), ff_make(0.f), ff_make(0.f)};
    for (int j = threadIdx.x; j < nb; j += kErrThreads)
#pragma unroll
        for (int k = 0; k < 4; ++k) g[k] = ff_add(g[k], at(k, j));
    ff tot[4];
    block_sums_ffv<4>(g, tot, sm);
    if (threadIdx.x == 0) s_alpha = tot[1].hi > 0.f ? ff_div(tot[0], tot[1]) : ff_make(0.f);
    __syncthreads();
    const ff alpha = s_alpha;
    // the squared error at alpha from every block's S1, S2, sum I^2 and a_b
    ff sse[1] = {ff_make(0.f)};
    for (int j = threadIdx.x; j < nb; j += kErrThreads) {
        const ff d = ff_add(alpha, ff_make(-at(6, j).hi));
        const ff two_d = ff{2.f * d.hi, 2.f * d.lo};
        ff term = ff_add(at(4, j), ff_mul(two_d, at(5, j)));
        term = ff_add(term, ff_mul(ff_mul(d, d), at(1, j)));
        sse[0] = ff_add(sse[0], term);
    }
    ff s[1];
    block_sums_ffv<1>(sse, s, sm);
    if (threadIdx.x == 0) {
        d_out[0] = ff_to_double(alpha);
        d_out[1] = tot[3].hi > 0.f ? ff_to_double(ff_div(s[0], tot[3])) : 0.0;
        d_out[2] = tot[2].hi > 0.f ? ff_to_double(ff_div(s[0], tot[2])) : 0.0;
    }
}

static size_t err_part_bytes(int nb) { return align_up(sizeof(ff) * size_t(nb) * kErrParts, 256); }
static size_t err_ws_bytes(int64_t P) { return err_part_bytes(err_blocks(P)) + 256; }

}  // namespace holo

using namespace holo;

extern "C" int replay_error_workspace_size(int H, int W, size_t* bytes) {
    clear_error();
    if (!bytes) return fail(HOLO_EINVAL, "replay_error_workspace_size: NULL output");
    if (H < 1 || W < 1 || int64_t(H) * W > (INT64_C(1) << 28))
        return fail(HOLO_EINVAL, "replay_error_workspace_size: H=%d W=%d", H, W);
    *bytes = err_ws_bytes(int64_t(H) * W);
    return HOLO_OK;
}

extern "C" int replay_error(const float* d_replay, const float* d_target, const uint8_t* d_mask,
                            int H, int W, double* d_out, void* d_ws, size_t ws_bytes,
                            holo_stream_t s) {
    clear_error();
    const char* who = "replay_error";
    if (!d_replay || !d_target || !d_out) return fail(HOLO_EINVAL, "%s: NULL input or output", who);
    if (H < 1 || W < 1 || int64_t(H) * W > (INT64_C(1) << 28))
        return fail(HOLO_EINVAL, "%s: H=%d W=%d out of range", who, H, W);
    const int64_t P = int64_t(H) * W;
    const size_t need = err_ws_bytes(P);
    if (!d_ws || ws_bytes < need) return fail(HOLO_EWORKSPACE, "%s: workspace %zu bytes, need %zu", who, ws_bytes, need);
    if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0) return fail(HOLO_EWORKSPACE, "%s: workspace not 256-byte aligned", who);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    const int nb = err_blocks(P);
    ff* part = static_cast<ff*>(d_ws);
    unsigned* done = reinterpret_cast<unsigned*>(static_cast<char*>(d_ws) + err_part_bytes(nb));
    // the completion counter starts at 0 (cleared on the stream; the kernel is an ordinary
    // launch after it, so nothing of it runs before the clear has landed)
    const cudaError_t e = cudaMemsetAsync(done, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_status(e, "replay_error: counter clear");
    Launch ln("replay_error", st);
    k_replay_error<<<nb, kErrThreads, 0, st>>>(d_replay, d_target, d_mask, P, part, done, d_out);
    return ln.done("replay_error launch");
}
