// error.cu - replay error of Section 5.2 / Eq. 3 with the intensity-domain,
// optimal-scale reading: alpha = sum(I T^2)/sum(I^2), mse = sum((alpha I - T^2)^2)/P,
// nmse = sum((alpha I - T^2)^2)/sum(T^4).
//
// Two passes (alpha must be known before the residual sum). Each thread forms its terms
// with single-rounding fmaf in float32 over a handful of pixels; every sum across threads
// and blocks is float64 with a fixed reduction order, so results are bit-reproducible.
// The kernels are HBM-bound: 8 bytes per pixel per pass (+1 with a mask).
#include "reduce.cuh"
#include "runtime.h"

namespace holo {

constexpr int kErrThreads = 256;
constexpr int kErrMaxBlocks = 152 * 8;

struct ErrWs {
    unsigned int ticket[2];
    unsigned int pad[62];
    double alpha, s_tt, count, pad2[29];
};

static int err_blocks(int64_t P) {
    int64_t nb = (P / 4 + kErrThreads - 1) / kErrThreads;
    if (nb < 1) nb = 1;
    return int(nb < kErrMaxBlocks ? nb : kErrMaxBlocks);
}

__device__ __forceinline__ float mask_at(const uint8_t* m, int64_t i) { return m ? (m[i] ? 1.f : 0.f) : 1.f; }

__global__ void __launch_bounds__(kErrThreads)
k_err_pass1(const float* __restrict__ I, const float* __restrict__ T, const uint8_t* __restrict__ mask,
            int64_t P, ErrWs* ws, double* partials, double* d_out) {
    __shared__ double sm[32];
    __shared__ int s_last;
    float sit = 0.f, sii = 0.f, stt = 0.f, cnt = 0.f;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nth = int64_t(gridDim.x) * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(I) | reinterpret_cast<uintptr_t>(T)) & 15) == 0;
    const int64_t P4 = vec ? P / 4 : 0;
    for (int64_t q = tid; q < P4; q += nth) {
        const float4 i4 = __ldg(reinterpret_cast<const float4*>(I) + q);
        const float4 t4 = __ldg(reinterpret_cast<const float4*>(T) + q);
        const float iv[4] = {i4.x, i4.y, i4.z, i4.w}, tv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float m = mask_at(mask, 4 * q + k);
            const float t2 = tv[k] * tv[k] * m, i1 = iv[k] * m;
            sit = fmaf(i1, t2, sit);
            sii = fmaf(i1, i1, sii);
            stt = fmaf(t2, t2, stt);
            cnt += m;
        }
    }
    for (int64_t i = 4 * P4 + tid; i < P; i += nth) {
        const float m = mask_at(mask, i);
        const float t2 = T[i] * T[i] * m, i1 = I[i] * m;
        sit = fmaf(i1, t2, sit);
        sii = fmaf(i1, i1, sii);
        stt = fmaf(t2, t2, stt);
        cnt += m;
    }
    const int nb = gridDim.x;
    double v[4] = {sit, sii, stt, cnt};
    for (int k = 0; k < 4; ++k) {
        const double b = block_sum(v[k], sm);
        if (threadIdx.x == 0) partials[k * nb + blockIdx.x] = b;
    }
    if (!grid_partial_done(0.0, partials + 4 * nb, &ws->ticket[0], &s_last)) return;
    double tot[4];
    for (int k = 0; k < 4; ++k) tot[k] = sum_partials(partials + k * nb, nb, sm);
    if (threadIdx.x == 0) {
        const double alpha = tot[1] > 0.0 ? tot[0] / tot[1] : 0.0;
        ws->alpha = alpha;
        ws->s_tt = tot[2];
        ws->count = tot[3];
        d_out[0] = alpha;
    }
}

__global__ void __launch_bounds__(kErrThreads)
k_err_pass2(const float* __restrict__ I, const float* __restrict__ T, const uint8_t* __restrict__ mask,
            int64_t P, ErrWs* ws, double* partials, double* d_out) {
    __shared__ double sm[32];
    __shared__ int s_last;
    const float alpha = float(ws->alpha);
    float sse = 0.f;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nth = int64_t(gridDim.x) * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(I) | reinterpret_cast<uintptr_t>(T)) & 15) == 0;
    const int64_t P4 = vec ? P / 4 : 0;
    for (int64_t q = tid; q < P4; q += nth) {
        const float4 i4 = __ldg(reinterpret_cast<const float4*>(I) + q);
        const float4 t4 = __ldg(reinterpret_cast<const float4*>(T) + q);
        const float iv[4] = {i4.x, i4.y, i4.z, i4.w}, tv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float d = fmaf(alpha, iv[k], -tv[k] * tv[k]) * mask_at(mask, 4 * q + k);
            sse = fmaf(d, d, sse);
        }
    }
    for (int64_t i = 4 * P4 + tid; i < P; i += nth) {
        const float d = fmaf(alpha, I[i], -T[i] * T[i]) * mask_at(mask, i);
        sse = fmaf(d, d, sse);
    }
    const int nb = gridDim.x;
    const double b = block_sum(double(sse), sm);
    if (!grid_partial_done(b, partials, &ws->ticket[1], &s_last)) return;
    const double tot = sum_partials(partials, nb, sm);
    if (threadIdx.x == 0) {
        d_out[1] = ws->count > 0.0 ? tot / ws->count : 0.0;
        d_out[2] = ws->s_tt > 0.0 ? tot / ws->s_tt : 0.0;
    }
}

static size_t err_ws_bytes(int64_t P) {
    const int nb = err_blocks(P);
    return align_up(sizeof(ErrWs), 256) + align_up(sizeof(double) * size_t(nb) * 5, 256) +
           align_up(sizeof(double) * size_t(nb), 256);
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
    ErrWs* ws = static_cast<ErrWs*>(d_ws);
    double* part1 = reinterpret_cast<double*>(static_cast<char*>(d_ws) + align_up(sizeof(ErrWs), 256));
    const int nb = err_blocks(P);
    double* part2 = part1 + align_up(sizeof(double) * size_t(nb) * 5, 256) / sizeof(double);
    int rc = cuda_status(cudaMemsetAsync(ws->ticket, 0, sizeof(ws->ticket), st), "replay_error: reset");
    if (rc) return rc;
    {
        Launch ln("err_pass1", st);
        k_err_pass1<<<nb, kErrThreads, 0, st>>>(d_replay, d_target, d_mask, P, ws, part1, d_out);
        if ((rc = ln.done("err_pass1 launch"))) return rc;
    }
    Launch ln("err_pass2", st);
    k_err_pass2<<<nb, kErrThreads, 0, st>>>(d_replay, d_target, d_mask, P, ws, part2, d_out);
    return ln.done("err_pass2 launch");
}
