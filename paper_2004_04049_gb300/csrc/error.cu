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
#include "error_block.cuh"

namespace holo {

__global__ void __launch_bounds__(kErrThreads)
k_replay_error(const float* __restrict__ I, const float* __restrict__ T, const uint8_t* __restrict__ mask,
               int64_t P, ff* part, unsigned* done, double* __restrict__ d_out) {
    replay_error_block(I, T, mask, P, part, done, d_out, int(blockIdx.x), int(gridDim.x));
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
