// error.cu - replay error of Section 5.2 / Eq. 3 with the intensity-domain,
// optimal-scale reading: alpha = sum(I T^2)/sum(I^2), mse = sum((alpha I - T^2)^2)/P,
// nmse = sum((alpha I - T^2)^2)/sum(T^4).
//
// Two launches:
//   partials1  per block: sum I*T^2, sum I^2, sum T^4, count
//   partials2  every warp first reduces partials1 to alpha (fixed order, so every warp of
//              every block gets the same bits), then its share of sum (alpha I - T^2)^2;
//              the block that finishes last (a completion counter, no waiting) adds the
//              shares in block order and writes mse and nmse
// Each thread forms its terms with single-rounding fmaf in float32 over a few pixels;
// every sum across threads, warps and blocks is float-float (about 48 significant bits,
// ffloat.cuh) in a fixed order, so results are bit-reproducible, and only the three
// reported values are converted to float64. HBM-bound: 8 bytes per pixel per pass (+1
// with a mask).
#include "ffloat.cuh"
#include "runtime.h"

namespace holo {

constexpr int kErrThreads = 256;
constexpr int kErrMaxBlocks = 152 * 2;

static int err_blocks(int64_t P) {
    int64_t nb = (P / 16 + kErrThreads - 1) / kErrThreads;
    if (nb < 1) nb = 1;
    return int(nb < kErrMaxBlocks ? nb : kErrMaxBlocks);
}

__device__ __forceinline__ float mask_at(const uint8_t* m, int64_t i) { return m ? (m[i] ? 1.f : 0.f) : 1.f; }

// Every thread owns up to kErrVec float4 groups of pixels (q = tid + k*nth) and issues
// all of their loads before any arithmetic, so a pass costs about one memory latency
// instead of one per grid-stride iteration.
constexpr int kErrVec = 4;

struct ErrTile {
    float4 i[kErrVec], t[kErrVec];
};

__device__ __forceinline__ void err_load(const float* __restrict__ I, const float* __restrict__ T,
                                         int64_t q0, int64_t nth, int64_t P4, ErrTile& x) {
#pragma unroll
    for (int k = 0; k < kErrVec; ++k) {
        const int64_t q = q0 + k * nth;
        x.i[k] = q < P4 ? __ldg(reinterpret_cast<const float4*>(I) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        x.t[k] = q < P4 ? __ldg(reinterpret_cast<const float4*>(T) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__device__ __forceinline__ float4 mask4(const uint8_t* __restrict__ m, int64_t q, int64_t P4) {
    if (!m || q >= P4) return make_float4(q < P4 ? 1.f : 0.f, q < P4 ? 1.f : 0.f, q < P4 ? 1.f : 0.f,
                                          q < P4 ? 1.f : 0.f);
    const uchar4 b = reinterpret_cast<const uchar4*>(m)[q];
    return make_float4(b.x ? 1.f : 0.f, b.y ? 1.f : 0.f, b.z ? 1.f : 0.f, b.w ? 1.f : 0.f);
}

// partials laid out [k][nb]: k = 0 sum I T^2, 1 sum I^2, 2 sum T^4, 3 count. Block 0 also
// clears the completion counter of pass 2 (which runs after this launch on the stream).
__global__ void __launch_bounds__(kErrThreads)
k_err_pass1(const float* __restrict__ I, const float* __restrict__ T, const uint8_t* __restrict__ mask,
            int64_t P, ff* __restrict__ partials, unsigned* __restrict__ done) {
    __shared__ ff sm[32 * 4];
    pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) *done = 0u;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nth = int64_t(gridDim.x) * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(I) | reinterpret_cast<uintptr_t>(T) |
                       reinterpret_cast<uintptr_t>(mask)) & 15) == 0;
    const int64_t P4 = vec ? P / 4 : 0;
    for (int64_t q0 = tid; q0 < P4; q0 += kErrVec * nth) {
        ErrTile x;
        err_load(I, T, q0, nth, P4, x);
#pragma unroll
        for (int k = 0; k < kErrVec; ++k) {
            const float4 m4 = mask4(mask, q0 + k * nth, P4);
            const float iv[4] = {x.i[k].x, x.i[k].y, x.i[k].z, x.i[k].w};
            const float tv[4] = {x.t[k].x, x.t[k].y, x.t[k].z, x.t[k].w};
            const float mv[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float t2 = tv[j] * tv[j] * mv[j], i1 = iv[j] * mv[j];
                acc[0] = fmaf(i1, t2, acc[0]);
                acc[1] = fmaf(i1, i1, acc[1]);
                acc[2] = fmaf(t2, t2, acc[2]);
                acc[3] += mv[j];
            }
        }
    }
    for (int64_t i = 4 * P4 + tid; i < P; i += nth) {
        const float m = mask_at(mask, i);
        const float t2 = T[i] * T[i] * m, i1 = I[i] * m;
        acc[0] = fmaf(i1, t2, acc[0]);
        acc[1] = fmaf(i1, i1, acc[1]);
        acc[2] = fmaf(t2, t2, acc[2]);
        acc[3] += m;
    }
    ff b[4];
    block_sums_ff<4>(acc, b, sm);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) partials[k * gridDim.x + blockIdx.x] = b[k];
    }
}

__global__ void __launch_bounds__(kErrThreads)
k_err_pass2(const float* __restrict__ I, const float* __restrict__ T, const uint8_t* __restrict__ mask,
            int64_t P, const ff* __restrict__ partials1, ff* partials2, unsigned* done,
            double* __restrict__ d_out) {
    __shared__ ff sm[32];
    __shared__ bool s_last;
    pdl_wait();
    const int nb = gridDim.x;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nth = int64_t(gridDim.x) * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(I) | reinterpret_cast<uintptr_t>(T) |
                       reinterpret_cast<uintptr_t>(mask)) & 15) == 0;
    const int64_t P4 = vec ? P / 4 : 0;
    // first tile's loads go out before alpha is formed; every warp reduces the pass-1
    // partials itself (same fixed order, so the same bits everywhere) instead of waiting
    // at a block barrier for one warp to do it
    ErrTile x;
    err_load(I, T, tid, nth, P4, x);
    const ff s_it = warp_sum_array_ff(partials1, nb);
    const ff s_ii = warp_sum_array_ff(partials1 + nb, nb);
    const ff alpha_ff = s_ii.hi > 0.f ? ff_div(s_it, s_ii) : ff_make(0.f);
    if (blockIdx.x == 0 && threadIdx.x == 0) d_out[0] = ff_to_double(alpha_ff);
    const float alpha = alpha_ff.hi;
    float acc[1] = {0.f};
    for (int64_t q0 = tid; q0 < P4; q0 += kErrVec * nth) {
        if (q0 != tid) err_load(I, T, q0, nth, P4, x);
#pragma unroll
        for (int k = 0; k < kErrVec; ++k) {
            const float4 m4 = mask4(mask, q0 + k * nth, P4);
            const float iv[4] = {x.i[k].x, x.i[k].y, x.i[k].z, x.i[k].w};
            const float tv[4] = {x.t[k].x, x.t[k].y, x.t[k].z, x.t[k].w};
            const float mv[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float d = fmaf(alpha, iv[j], -tv[j] * tv[j]) * mv[j];
                acc[0] = fmaf(d, d, acc[0]);
            }
        }
    }
    for (int64_t i = 4 * P4 + tid; i < P; i += nth) {
        const float d = fmaf(alpha, I[i], -T[i] * T[i]) * mask_at(mask, i);
        acc[0] = fmaf(d, d, acc[0]);
    }
    ff b[1];
    block_sums_ff<1>(acc, b, sm);
    // publish this block's share; the block whose increment completes the count reduces
    // all shares (threadfence reduction: every other block fenced its store before its
    // increment, and the last block reads the shares through L2)
    if (threadIdx.x == 0) {
        partials2[blockIdx.x] = b[0];
        __threadfence();
        s_last = atomicAdd(done, 1u) == unsigned(nb - 1);
    }
    __syncthreads();
    if (!s_last || threadIdx.x >= 32) return;
    __threadfence();
    const ff s_tt = warp_sum_array_ff(partials1 + 2 * nb, nb);
    const ff count = warp_sum_array_ff(partials1 + 3 * nb, nb);
    const ff sse = warp_sum_array_ff_cg(partials2, nb);
    if (threadIdx.x == 0) {
        d_out[1] = count.hi > 0.f ? ff_to_double(ff_div(sse, count)) : 0.0;
        d_out[2] = s_tt.hi > 0.f ? ff_to_double(ff_div(sse, s_tt)) : 0.0;
    }
}

static size_t err_part_bytes(int nb) { return align_up(sizeof(ff) * size_t(nb) * 4, 256); }
static size_t err_ws_bytes(int64_t P) {
    const int nb = err_blocks(P);
    return err_part_bytes(nb) + align_up(sizeof(ff) * size_t(nb), 256) + 256;
}

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
    ff* part1 = static_cast<ff*>(d_ws);
    ff* part2 = part1 + err_part_bytes(nb) / sizeof(ff);
    unsigned* done = reinterpret_cast<unsigned*>(static_cast<char*>(d_ws) + err_part_bytes(nb) +
                                                 align_up(sizeof(ff) * size_t(nb), 256));
    int rc;
    {
        Launch ln("err_pass1", st);
        const cudaError_t le = launch_pdl(k_err_pass1, dim3(nb), dim3(kErrThreads), 0, st, d_replay, d_target,
                                          d_mask, P, part1, done);
        if ((rc = ln.done("err_pass1 launch", le))) return rc;
    }
    Launch ln("err_pass2", st);
    const cudaError_t le = launch_pdl(k_err_pass2, dim3(nb), dim3(kErrThreads), 0, st, d_replay, d_target, d_mask,
                                      P, static_cast<const ff*>(part1), part2, done, d_out);
    return ln.done("err_pass2 launch", le);
}
