// runtime.h - host-side runtime shared by the library's translation units: status and
// last-error reporting, kernel-launch accounting, per-kernel CUDA-event timing and the
// per-device constant tables (FFT twiddles, phase cos/sin).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "holo.h"

namespace holo {

// ---- status -----------------------------------------------------------------
// Records a message for holo_last_error() on this thread and returns `code`.
int fail(int code, const char* fmt, ...);
// Records a warning message (returned later with HOLO_OK).
void warn(const char* fmt, ...);
void clear_error();
// Maps a CUDA error to HOLO_ECUDA with a message; returns HOLO_OK for cudaSuccess.
int cuda_status(cudaError_t e, const char* what);

// ---- launches ---------------------------------------------------------------
// Wraps one kernel launch: counts it and, while profiling is on, records CUDA events
// around it on `stream`. Construct immediately before the launch and call done() with
// the launch's cudaGetLastError() right after it.
class Launch {
  public:
    Launch(const char* family, cudaStream_t stream);
    // `launch` is the status a cudaLaunchKernelEx call returned (cudaSuccess for <<<>>>)
    int done(const char* what, cudaError_t launch = cudaSuccess);
  private:
    const char* family_;
    cudaStream_t stream_;
    cudaEvent_t start_ = nullptr;
};

// Sets event profiling on or off and returns the previous setting.
int profiling_swap(int on);
// Adjusts the launch count by n (kernels replayed by a graph, or captured and not run).
void add_launches(int64_t n);

// Host-side fault injection for tests: true when the environment variable
// HOLO_FAULT_INJECT (a comma-separated list) names `kind` ("alloc": scratch allocations
// fail, "timeout": holo_check reports an expired wait, "plan": batch planning fails).
bool fault_injected(const char* kind);

// ---- programmatic dependent launch ------------------------------------------------
// A kernel launched with launch_pdl may be scheduled while the previous kernel on its
// stream is still running, which hides the launch latency between dependent kernels.
// It must execute pdl_wait() before its first access to memory that earlier work on the
// stream writes or reads (griddepcontrol.wait returns once the preceding grid has
// completed and its writes are visible; it returns at once when there is none), and
// may execute pdl_trigger() once its own CTAs no longer need the slots the next
// kernel's CTAs would take (the next kernel launches when every CTA has triggered or
// exited).
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---- constant tables ---------------------------------------------------------
struct Tables {
    const float2* twiddles;   // Stockham stage twiddles, see fft_core.cuh
    const float2* cs256;      // (cos, sin)(2*pi*c/256), c < 256
    // tcgen05 DFT-32 B operand per precision (index 1 fp16, 2 bf16): [direction -1, +1][hi, lo]
    // 64x64 real-form matrices, 8192 bytes each in the K-major 128-byte-swizzle layout
    const uint8_t* tc05b[3];
};
// Fills the tables on the current device the first time and returns their addresses.
int device_tables(Tables* out);

// ---- misc -------------------------------------------------------------------
inline bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
inline int log2i(int64_t x) { int l = 0; while ((int64_t(1) << l) < x) ++l; return l; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
constexpr int kMinDim = 64;
constexpr int kMaxDim = 4096;

// ---- entry points shared between translation units (library-internal) -----
// the bounded-wait flags of the tcgen05 DFT passes (ospr_tc.cu, gs.cu) and of the
// persistent batch kernel (batch_persistent.cu): read, and cleared when `clear`
int ospr_tc05_fault(int* out, bool clear);
int gs_tc05_fault(int* out, bool clear);
int ospr_persistent_fault(int* out, bool clear);
// ospr_generate with an optional event recorded on s once the last hologram bits are
// written (ospr.cu; the host-buffer batch starts their copy there)
int ospr_generate_ev(const float* d_target, int H, int W, int N, const uint8_t* d_codes, int64_t L, int levels,
                     uint64_t seed, int64_t start_index, int64_t subframe_stride, int precision,
                     uint32_t* d_holo_bits, float* d_replay, void* d_ws, size_t ws_bytes, holo_stream_t s,
                     cudaEvent_t bits_ready);
// a holo_graph for a graph built in another translation unit (batch.cu defines the type)
holo_graph* make_holo_graph(cudaGraph_t graph, cudaGraphExec_t exec, int device, int64_t kernels);

// Sets the dynamic shared-memory limit of kernel `fn` on the current device once.
int ensure_smem(const void* fn, size_t bytes, uint64_t* device_mask);
// *ctas = how many CTAs of kernel `fn` (threads, dynamic shared memory `bytes`) the current
// device holds at once (CTAs per SM x SMs), found once per device and kept in cache[64]
// (zero-initialised by the caller).
int resident_ctas(const void* fn, int threads, size_t bytes, int* cache, int* ctas);

}  // namespace holo
