/*
 * holo.h - C ABI of the GB300 library for LUT phase randomisation, One-Step
 * Phase-Retrieval (OSPR) and Gerchberg-Saxton (GS) hologram generation
 * (arXiv 2004.04049, "Lookup tables for phase randomisation in hardware generated
 * holograms").
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Images are row-major float32 [H][W]; pixel p = r*W + c (column index fastest).
 *    H and W are powers of two in [64, 4096] unless a call says otherwise.
 *  - Every pointer named d_* is a device pointer on the current CUDA device. The caller
 *    owns all of them (inputs, outputs and the workspace) and keeps them alive until the
 *    stream has finished the call. The library never frees caller memory. Pointers
 *    named h_* are host pointers, with the same ownership rule.
 *  - Every call is asynchronous on the caller's stream `s` (NULL = the legacy default
 *    stream). The return value reports argument validation and launch errors only;
 *    errors raised while the kernels run surface at the next synchronisation and via
 *    holo_check().
 *  - Return codes: HOLO_OK (0) or a negative holo_status. A message for the last
 *    non-OK return (and for design-rule warnings returned with HOLO_OK) is available
 *    from holo_last_error() on the same host thread.
 *  - There is no CPU fallback: without a usable CUDA device every compute call fails
 *    with HOLO_ECUDA.
 *  - The library sets up per-device state on first use (constant tables, internal
 *    streams, scratch addresses) and keeps it until the process exits; a process that
 *    calls cudaDeviceReset must not call the library on that device afterwards.
 *  - Transforms are the unitary DFT of Eq. 1 (forward, exp(-2 pi i ...)) and Eq. 2
 *    (inverse, exp(+2 pi i ...)), scale 1/sqrt(H*W).
 */
#ifndef HOLO_H
#define HOLO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so this header needs no CUDA headers. */
typedef struct CUstream_st* holo_stream_t;

typedef enum holo_status {
    HOLO_OK = 0,
    HOLO_EINVAL = -1,        /* a pointer, size or count is invalid */
    HOLO_EUNSUPPORTED = -2,  /* a valid value this build does not implement */
    HOLO_ECUDA = -3,         /* a CUDA runtime call failed (no device, launch error) */
    HOLO_ETIMEOUT = -4,      /* a bounded device-side wait gave up */
    HOLO_ENOMEM = -5,        /* the library could not allocate its own small state */
    HOLO_EWORKSPACE = -6     /* the caller's workspace is missing or too small */
} holo_status;

typedef enum holo_precision {
    HOLO_FP32 = 0,     /* all transforms in float32 */
    HOLO_FP16X2 = 1,   /* DFT-32 stages on the tcgen05 tensor cores, fp16 hi+lo operands, fp32 accumulate */
    HOLO_BF16X2 = 2    /* DFT-32 stages on the tcgen05 tensor cores, bf16 hi+lo operands, fp32 accumulate */
} holo_precision;

/* L value selecting the per-pixel generator with no table (the "unrepeated" case). */
#define HOLO_L_UNREPEATED (-1)

/* ---------------------------------------------------------------- utilities ---- */

/* Library version, major*10000 + minor*100 + patch. */
int holo_version(void);

/* Message of the last non-OK return on this host thread (or of a warning returned with
 * HOLO_OK); "" if none. The pointer stays valid until the next call on this thread. */
const char* holo_last_error(void);

/* Synchronises stream s and reports any CUDA error raised by earlier calls, and the
 * library's sticky device status (HOLO_ETIMEOUT if a bounded wait gave up).
 * Host-side fault injection for tests: the environment variable HOLO_FAULT_INJECT, a
 * comma-separated list, makes "timeout" holo_check return HOLO_ETIMEOUT, "alloc"
 * ospr_autotune's scratch allocation fail (HOLO_ENOMEM) and "plan" batch planning fail
 * (HOLO_EINVAL), before any device work. */
int holo_check(holo_stream_t s);

/* Number of kernels this library has launched in this process (all devices). */
int holo_launch_count(uint64_t* out_count);

/* Per-kernel timing with CUDA events recorded on the launching stream around every
 * launch while enabled. holo_profile_read synchronises the recorded events and returns,
 * for the kernel family `name`, the number of launches and their summed duration in
 * milliseconds since the last holo_profile_reset. Families: "lut_build",
 * "ospr_col_ifft", "ospr_row", "ospr_col_fft", "ospr_finalize", "fresnel_chirp", "gs_prepare",
 * "gs_col_init", "gs_row", "gs_col", "gs_finish", "replay_error", "lfsr_build",
 * "nn_conv_fwd", "nn_conv_dgrad", "nn_conv_wgrad", "nn_elementwise",
 * "nn_loss", "nn_adam". */
int holo_profile_enable(int on);
int holo_profile_reset(void);
int holo_profile_read(const char* name, uint64_t* launches, double* total_ms);

/* ------------------------------------------------------------- phase LUT ---- */

/*
 * lut_build - fill the phase lookup table ("pool") of Section 4: L random phase codes
 * generated once and then drawn sequentially (Section 5, Fig. 3). The entries are
 * 8-bit codes (Section 5.2: "over 12 Mb" for 256x256x24 entries).
 *
 *   seed     generator stream; entry k holds the top log2(levels) bits of the k-th
 *            SplitMix64 output, mix(seed + (k+1)*0x9E3779B97F4A7C15).
 *   L        number of entries, 1 <= L <= 2^31 - 1.
 *   levels   phase levels, a power of two in [2, 256]; code c means 2*pi*c/levels.
 *   d_codes  [L] uint8 output.
 *   d_cs     [2L] float32 output (cos, sin of each entry's phase, interleaved), or NULL.
 * Errors: HOLO_EINVAL for L out of range, bad levels or NULL d_codes.
 */
int lut_build(uint64_t seed, int64_t L, int levels, uint8_t* d_codes, float* d_cs,
              holo_stream_t s);

/*
 * lfsr_build - m-sequence phase codes: the PRNG alternative Section 7 weighs against the
 * LUT (an m-sequence generator feeding a cos/sin table). Not part of the paper's method;
 * provided to compare the two on error and speed.
 *
 * Galois LFSR with the primitive polynomial x^31 + x^3 + 1: state s_k = seed_state * x^k
 * mod p, output bit b_k = coefficient of x^30 of s_k (period 2^31 - 1). Writes
 * d_codes[k] = code(start + k), k < count, where code i packs bits b_{m i} ..
 * b_{m i + m - 1} (m = log2(levels)) most significant first. The result is a table for the
 * table mode of ospr_generate / gs_iterate (L = count): with count >= N*H*W every pixel of
 * every sub-frame draws its own m-sequence code (start = the frame's first draw).
 *
 *   seed_state  1 .. 2^31 - 1.   start  0 .. 2^56.   count 1 .. 2^31 - 1.
 *   levels      power of two in [2, 256].   d_codes  [count] uint8, device, caller-owned.
 * Errors: HOLO_EINVAL, HOLO_ECUDA. Asynchronous on s.
 */
int lfsr_build(uint32_t seed_state, int64_t start, int64_t count, int levels, uint8_t* d_codes,
               holo_stream_t s);

/* ------------------------------------------------------------------- OSPR ---- */

/*
 * ospr_workspace_size - bytes of device workspace ospr_generate needs for this shape.
 */
int ospr_workspace_size(int H, int W, int N, int precision, size_t* bytes);

/*
 * ospr_generate - N binary-phase OSPR sub-frames of one target and their time-averaged
 * replay (Section 2: back-propagate, quantise; Section 3: random phase per sub-frame;
 * Section 5.2 / Section 6: binary phase device).
 *
 * Per sub-frame s in [0, N):
 *   draw index of pixel p   i = start_index + s*stride + p     (Fig. 3 continuation)
 *   code                    c = d_codes[i mod L]               (L > 0)
 *                           c = top bits of SplitMix64(seed, i) (L == HOLO_L_UNREPEATED)
 *                           c = 0                               (L == 0: flat phase)
 *   E = T * exp(2*pi*i*c/levels);  H_s = IDFT(E) (Eq. 2)
 *   h_s = +1 where Re H_s >= 0, else -1
 *   I  += |DFT(h_s)|^2 / N  (Eq. 1)
 *
 *   d_target     [H][W] float32 target amplitude (>= 0).
 *   N            sub-frames, 1 <= N <= 4096.
 *   d_codes      [L] uint8 codes (ignored, may be NULL, when L <= 0).
 *   L            table length (>= 0) or HOLO_L_UNREPEATED.
 *   levels       code levels, power of two in [2, 256] (the table's levels).
 *   seed         generator stream for L == HOLO_L_UNREPEATED (ignored otherwise).
 *   start_index  draw index of pixel 0 of sub-frame 0 (>= 0): frames that share one
 *                table continue from the previous frame's end (Fig. 3).
 *   subframe_stride  draw-index step between sub-frames; 0 means H*W.
 *   precision    HOLO_FP32, or HOLO_FP16X2 / HOLO_BF16X2: both radix-32 DFT stages of every
 *                line transform as 64x64 real GEMMs on the tcgen05 tensor cores, operands
 *                split into hi + lo 16-bit halves, float32 accumulators (far field, H and
 *                W in {1024, 2048}; HOLO_EUNSUPPORTED otherwise).
 *   d_holo_bits  [N][H*W/32] uint32 output or NULL: bit j of word w is pixel 32*w + j
 *                of that sub-frame, 1 for -1.
 *   d_replay     [H][W] float32 output or NULL: mean replay intensity over sub-frames.
 *   d_ws         device workspace of at least ospr_workspace_size() bytes, 256-byte
 *                aligned. Sub-frame pairs go through the transforms in chunks of up to
 *                16 pairs; the chunk size, accumulator groups and FFT tile variants come
 *                from the shape's tuning (ospr_autotune / ospr_tuning_set; defaults
 *                overridable with HOLO_OSPR_CHUNK=1..16 and HOLO_OSPR_GROUPS=1..4), and
 *                the workspace size follows the same setting.
 * Design-rule warnings (Section 8: L prime, L > N, L > max(H, W)) are returned with
 * HOLO_OK and a message in holo_last_error(). Errors: HOLO_EINVAL, HOLO_EUNSUPPORTED,
 * HOLO_EWORKSPACE, HOLO_ECUDA.
 */
int ospr_generate(const float* d_target, int H, int W, int N,
                  const uint8_t* d_codes, int64_t L, int levels, uint64_t seed,
                  int64_t start_index, int64_t subframe_stride, int precision,
                  uint32_t* d_holo_bits, float* d_replay,
                  void* d_ws, size_t ws_bytes, holo_stream_t s);

/*
 * OSPR tuning per shape (H, W): the tile variants of the column IDFT pass and of the
 * column DFT pass (0..2 each: radix-32 lines at two widths, radix-16 lines; lengths below
 * 512 have only variant 0), of the row pass (0..1; only 0 below 512), the sub-frame pairs
 * in flight per chunk (1..16) and the partial accumulators of the column DFT pass (1..4).
 * A variant a length does not have falls back to 0. Every setting computes the same
 * values up to float32 rounding order; the workspace size of ospr_workspace_size follows
 * the current setting, so query it after changing it.
 * ospr_autotune times ospr_generate on synthetic data of this shape (a 10007-entry table)
 * for candidate settings (two sweeps of coordinate descent over the column IDFT variant,
 * row variant, column DFT variant, chunk and groups, starting from column DFT variant 1
 * where the length has it, whose two CTAs per SM let batch frames share the SMs; each
 * candidate the median of `reps` runs after one warm-up, CUDA events on stream s; timings
 * within 1% are a tie, kept by the current setting unless the candidate's workspace is
 * smaller), installs the fastest for this process
 * and, when the environment variable HOLO_TUNE_CACHE names a file, writes every installed
 * setting there (one JSON object per line), from where later processes read it. It
 * allocates and frees its own scratch (HOLO_ENOMEM if that fails) and synchronises s.
 * best_ms (nullable) receives the winner's time per call.
 * ospr_tuning_set installs a setting without timing (for tests and reproduction); values
 * outside the ranges above are HOLO_EINVAL.
 */
int ospr_autotune(int H, int W, int N, int reps, holo_stream_t s, double* best_ms);
int ospr_tuning_get(int H, int W, int* col_ifft_variant, int* col_fft_variant, int* row_variant, int* chunk,
                    int* groups);
int ospr_tuning_set(int H, int W, int col_ifft_variant, int col_fft_variant, int row_variant, int chunk,
                    int groups);

/*
 * ospr_generate_noalloc - ospr_generate for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a deployment variant, not part of the method.
 *
 * Some callers can't call cudaMalloc or hand the library a workspace: a display
 * pipeline with a hard per-frame deadline (cudaMalloc and cudaFree may synchronise the
 * device and stall the frame), a plug-in inside a host application that owns every
 * device allocation and exposes none, or firmware-style hosts whose device memory is
 * partitioned once at start-up. This entry point takes the same arguments as
 * ospr_generate minus the workspace and gives the same results (the bits are identical;
 * the replay differs only in the float32 summation order of sub-frame pairs).
 *
 * Scratch: one file-scope device array of HOLO_NOALLOC_SCRATCH_BYTES (32 MiB), which
 * every GPU that loads the library holds until the process exits. It fits one complex64
 * and one float32 H*W field, so H*W <= 2^21 (e.g. 1024x1024 or 1024x2048); larger
 * shapes return HOLO_EWORKSPACE with a message, and nothing is launched.
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 * The first call on each device looks up the array's device address with
 * cudaGetSymbolAddress, with that device current; make that first call before any
 * stream capture.
 * Every call on a device shares the one array and leaves its contents behind; a call
 * writes every scratch byte before reading it, so no clearing is needed, but calls
 * whose kernels overlap on the GPU (different streams, or host threads) race on the
 * array and corrupt each other's results: serialise them.
 * The looked-up address is kept for the life of the process, like the library's other
 * per-device state (constant tables, internal streams): after a cudaDeviceReset the
 * process must not call the library on that device again.
 * Design-rule warnings (Section 8) are recorded as ospr_generate records them.
 * Errors: as ospr_generate, with HOLO_EWORKSPACE for shapes beyond the scratch.
 */
#define HOLO_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int ospr_generate_noalloc(const float* d_target, int H, int W, int N,
                          const uint8_t* d_codes, int64_t L, int levels, uint64_t seed,
                          int64_t start_index, int64_t subframe_stride, int precision,
                          uint32_t* d_holo_bits, float* d_replay, holo_stream_t s);

/* --------------------------------------------------- Fresnel propagation ---- */

/*
 * ospr_fresnel_workspace_size - bytes of device workspace ospr_generate_fresnel needs.
 */
int ospr_fresnel_workspace_size(int H, int W, int N, size_t* bytes);

/*
 * ospr_generate_fresnel - OSPR with Fresnel instead of far-field propagation (Section 2
 * names both regimes; the paper's experiments use the far field). Model: the replay of a
 * hologram h is |DFT(h * Q)|^2 with the separable quadratic phase
 *     Q(y, x) = exp(i*pi*kappa*((x - W/2)^2 + (y - H/2)^2)),  kappa = pitch^2 / (wavelength * z),
 * the replay plane's own quadratic phase being invisible to an intensity replay (the
 * random target phase is drawn relative to it). Per sub-frame s:
 *     E_s = T * exp(i*theta_s)  (the draw rule of ospr_generate),
 *     H_s = conj(Q) * IDFT(E_s), h_s = +1 where Re H_s >= 0 else -1,
 *     I   = (1/N) sum_s |DFT(h_s * Q)|^2  (unitary transforms).
 * kappa = 0 is the far field of ospr_generate. The Fresnel field is not Hermitian, so
 * every sub-frame takes its own transforms (twice the work of ospr_generate per
 * sub-frame) and the replay has no twin symmetry.
 *   d_target ... subframe_stride, d_holo_bits, d_replay, stream: as for ospr_generate.
 *   kappa       finite, |kappa| <= 1e6 (pixel pitch^2 / (wavelength * distance)).
 *   d_ws        device workspace of at least ospr_fresnel_workspace_size() bytes,
 *               256-byte aligned; it also holds the H + W chirp factors of Q, made on the
 *               device at the start of the call (float64 sincospi rounded to float32).
 * Float32 only (tile variants, pairs in flight and accumulators follow the shape's OSPR
 * tuning). Returns HOLO_EINVAL / HOLO_EUNSUPPORTED / HOLO_EWORKSPACE on bad arguments.
 */
int ospr_generate_fresnel(const float* d_target, int H, int W, int N, const uint8_t* d_codes, int64_t L,
                          int levels, uint64_t seed, int64_t start_index, int64_t subframe_stride, double kappa,
                          uint32_t* d_holo_bits, float* d_replay, void* d_ws, size_t ws_bytes, holo_stream_t s);

/* ------------------------------------------------------- batched frames ---- */

/*
 * A batch of independent OSPR frames of mixed shapes, each with its own table and
 * sub-frame count (Section 5, Fig. 3: frames draw from the pool; here each frame may also
 * build its own table first). Field meanings follow ospr_generate and lut_build.
 *   d_codes    [L] uint8: filled by lut_build(seed, L, levels) first when build_lut != 0,
 *              otherwise read as given.
 *   d_err      [3] float64 (alpha, mse, nmse of the replay, as replay_error) or NULL;
 *              needs d_replay.
 */
typedef struct holo_frame_desc {
    const float* d_target;
    int H, W, N;
    uint8_t* d_codes;
    int64_t L;
    int levels;
    uint64_t seed;
    int build_lut;
    int64_t start_index;
    int64_t subframe_stride;
    uint32_t* d_holo_bits;
    float* d_replay;
    double* d_err;
} holo_frame_desc;

/*
 * ospr_batch_workspace_size - bytes of device workspace ospr_generate_batch (and the
 * graph made by ospr_batch_graph_create) needs for these frames.
 */
int ospr_batch_workspace_size(const holo_frame_desc* h_frames, int n_frames, int precision,
                              size_t* bytes);

/*
 * ospr_generate_batch - runs every frame of the batch (lut_build if asked, ospr_generate,
 * replay_error if d_err is given) with frames spread over the library's internal streams
 * so that frames of different shapes share the GPU. Frames are assigned longest first to
 * the least-loaded of S streams (S = 8, environment override HOLO_BATCH_STREAMS=1..32);
 * each stream's frames run in order on that stream's slice of the workspace. The call
 * forks from and joins back to stream `s`: work queued on `s` before the call runs first,
 * work queued after it waits for every frame. Results equal those of per-frame calls.
 * Calls may come from several host threads: a per-device lock is held while a call
 * enqueues its work (fork to join), so concurrent calls queue one after the other on the
 * internal streams, and an eager call made while another thread captures a batch graph
 * waits for the capture to end.
 *   h_frames   host array of n_frames descriptors (read during the call only).
 * Errors: as the per-frame calls, with the index of the offending frame in the message.
 */
int ospr_generate_batch(const holo_frame_desc* h_frames, int n_frames, int precision,
                        void* d_ws, size_t ws_bytes, holo_stream_t s);

/*
 * Host buffers of one batch frame for ospr_generate_batch_host (an engineering extension
 * for callers whose targets arrive from and whose holograms go back to host memory). Each
 * pointer is optional (NULL: no copy); sizes follow the frame's descriptor.
 *   h_target     [H][W] float32, copied into the frame's d_target before its work.
 *   h_holo_bits  [N][H*W/32] uint32, copied from d_holo_bits after the frame.
 *   h_replay     [H][W] float32, copied from d_replay after the frame.
 *   h_err        [3] float64, copied from d_err after the frame.
 */
typedef struct holo_frame_host {
    const float* h_target;
    uint32_t* h_holo_bits;
    float* h_replay;
    double* h_err;
} holo_frame_host;

/*
 * ospr_generate_batch_host - ospr_generate_batch with each frame's host-to-device and
 * device-to-host copies: the targets are copied in on one internal copy-in stream in the
 * frames' launch order, each frame's work waiting for its own target; its results go out
 * on a copy-out stream of the frame's internal stream, the hologram bits
 * as soon as the last row pass has written them (while the frame's replay passes and
 * error still run), the replay and the error once the frame is done. So the copies
 * overlap kernels and hold up neither the end of their frame nor the next frame of the
 * internal stream. Page-locked host buffers make the copies asynchronous (pageable ones
 * are copied synchronously by CUDA). The host buffers
 * must stay valid, and untouched by the caller, until stream `s` passes the call. Frames
 * must not share a d_target (each frame's copy writes it). HOLO_EINVAL for a NULL table
 * or a host output whose device buffer is NULL; other errors as ospr_generate_batch.
 */
int ospr_generate_batch_host(const holo_frame_desc* h_frames, const holo_frame_host* h_io, int n_frames,
                             int precision, void* d_ws, size_t ws_bytes, holo_stream_t s);

/*
 * A CUDA graph of a whole batch: ospr_batch_graph_create runs the batch once on a private
 * stream (to finish every lazy set-up), then captures it into an executable graph, so
 * that one holo_graph_launch replays the whole batch with a single launch. The graph
 * keeps the descriptors' pointers: refill the same buffers between launches. Launches of
 * one graph must not overlap (they share the workspace).
 */
typedef struct holo_graph holo_graph;
int ospr_batch_graph_create(const holo_frame_desc* h_frames, int n_frames, int precision,
                            void* d_ws, size_t ws_bytes, holo_graph** out);
int holo_graph_launch(holo_graph* g, holo_stream_t s);
int holo_graph_destroy(holo_graph* g);

/*
 * ospr_generate_batch_persistent - the batch of ospr_generate_batch (table build if asked,
 * ospr_generate and, with d_err, replay_error for every frame) as ONE persistent kernel
 * launch with a work queue in device memory (an engineering extension, not part of the
 * method). One 512-thread CTA per SM takes items in queue order: a table range, a column
 * IDFT tile, a row tile, a column DFT tile, a finalize range or an error block of some
 * frame. Dependencies between the passes of a frame are completion counters in the
 * workspace: an item waits (thread 0 polling with acquire loads) only for items that come
 * earlier in the queue, so the launch cannot deadlock; every wait is bounded by
 * wait_limit_us microseconds (0: one second). When a wait expires the kernel sets the
 * flag holo_tc_status reports, every CTA stops taking items and the call's results are not
 * to be trusted (holo_check then returns HOLO_ETIMEOUT).
 * Frames are spread over S workspace slots (S = 8, HOLO_BATCH_STREAMS overrides), longest
 * first; each slot's frames run in order and the slots' items are interleaved. The tile
 * variants are fixed at 0 and the chunking (pairs in flight, accumulator groups) is the
 * shape's current tuning, so each frame's bits, replay and error equal those of
 * ospr_generate + replay_error under tuning (0, 0, 0, chunk, groups) of that shape.
 * Supports H, W in {512, 1024, 2048}, float32, frames with d_target and d_replay
 * (HOLO_EUNSUPPORTED / HOLO_EINVAL otherwise). The workspace (caller-owned, 256-byte
 * aligned) holds the slots, the counters, the frame table and the queue; the call writes
 * the table and the queue (a copy ordered on s before the launch). Calls sharing a
 * workspace must not overlap on the GPU, and frames that build their table (build_lut)
 * must not share its buffer with another frame of the batch.
 * ospr_batch_persistent_graph_create captures the counter clear and the launch in a CUDA
 * graph (replayed by holo_graph_launch); the queue stays in d_ws, which the graph reuses.
 */
int ospr_batch_persistent_workspace_size(const holo_frame_desc* h_frames, int n_frames, size_t* bytes);
int ospr_generate_batch_persistent(const holo_frame_desc* h_frames, int n_frames, int wait_limit_us,
                                   void* d_ws, size_t ws_bytes, holo_stream_t s);
int ospr_batch_persistent_graph_create(const holo_frame_desc* h_frames, int n_frames, int wait_limit_us,
                                       void* d_ws, size_t ws_bytes, holo_graph** out);

/* --------------------------------------------------------------------- GS ---- */

/*
 * gs_workspace_size - bytes of device workspace gs_iterate and gs_iterate_fresnel need
 * (the complex field, scalars, error partials and the H + W Fresnel chirp factors).
 */
int gs_workspace_size(int H, int W, int iters, int precision, size_t* bytes);

/*
 * gs_iterate - Gerchberg-Saxton iterations with a phase-quantised hologram (Section 2;
 * random initial phase of Section 3 drawn from the LUT; Section 8: for GS only the
 * prime-length and longer-than-the-largest-dimension rules apply).
 *
 * T_s = T * sqrt(H*W / sum T^2). Start field E (replay plane): d_state_in if given,
 * else T_s * exp(i*phi) with phi = d_init_phase if given, else the LUT phases of
 * sub-frame 0 (draw index start_index + p, same code rules as ospr_generate).
 * Iteration k = 1..iters:
 *   H = IDFT(E); q = floor(levels*arg(H)/(2 pi) + 1/2) mod levels (arg(0) = 0);
 *   h = exp(2 pi i q/levels); R = DFT(h); eps_k = sum (|R| - T_s)^2;
 *   E = T_s * exp(i arg R)  (arg(0) = 0)
 *
 *   levels        hologram phase levels, a power of two in [2, 256] (2 = binary).
 *   d_init_phase  [H][W] float32 radians or NULL.
 *   d_codes, L, lut_levels, seed, start_index: the initial-phase LUT (as ospr_generate).
 *   d_phase_codes [H][W] uint8 output or NULL: q of the last iteration.
 *   d_replay      [H][W] float32 output or NULL: |R|^2 of the last iteration.
 *   d_err         [iters] float64 output or NULL: eps_k.
 *   d_state_in    [H][W][2] float32 (re, im) replay-plane field to resume from, or NULL.
 *   d_state_out   [H][W][2] float32 output or NULL: E after the last iteration.
 *   precision     HOLO_FP32, or HOLO_FP16X2 / HOLO_BF16X2 (the DFT-32 stages of every line
 *                 transform on the tcgen05 tensor cores with split hi/lo operands and float32
 *                 accumulation, as in ospr_generate) for H, W in {1024, 2048}.
 * Errors: HOLO_EINVAL, HOLO_EUNSUPPORTED, HOLO_EWORKSPACE, HOLO_ECUDA.
 */
int gs_iterate(const float* d_target, int H, int W, int iters, int levels,
               const float* d_init_phase,
               const uint8_t* d_codes, int64_t L, int lut_levels, uint64_t seed,
               int64_t start_index, int precision,
               uint8_t* d_phase_codes, float* d_replay, double* d_err,
               const float* d_state_in, float* d_state_out,
               void* d_ws, size_t ws_bytes, holo_stream_t s);

/*
 * gs_iterate_fresnel - gs_iterate under Fresnel propagation (Section 2 names both regimes;
 * the quadratic-phase model and kappa are those of ospr_generate_fresnel): per iteration
 *   H = conj(Q) * IDFT(E); q and h as gs_iterate; R = DFT(h * Q); eps_k and E as gs_iterate,
 * Q(y, x) = exp(i*pi*kappa*((x - W/2)^2 + (y - H/2)^2)). kappa = 0 gives the results of
 * gs_iterate. Float32; every other argument as gs_iterate; HOLO_EINVAL for a kappa that is
 * not finite or above 1e6 in magnitude.
 */
int gs_iterate_fresnel(const float* d_target, int H, int W, int iters, int levels,
                       const float* d_init_phase, const uint8_t* d_codes, int64_t L, int lut_levels,
                       uint64_t seed, int64_t start_index, double kappa, uint8_t* d_phase_codes,
                       float* d_replay, double* d_err, const float* d_state_in, float* d_state_out,
                       void* d_ws, size_t ws_bytes, holo_stream_t s);

/*
 * gs_iterate_batch - gs_iterate for B targets of one shape in the same launches (every
 * pass covers all targets, so small fields fill the GPU together). Target b is
 * d_targets + b*H*W and every per-target input and output advances the same way:
 *   d_targets      [B][H][W] float32.
 *   d_init_phases  [B][H][W] float32 radians or NULL.
 *   d_states_in    [B][H][W][2] float32 or NULL.
 *   d_phase_codes  [B][H][W] uint8 or NULL; d_replay [B][H][W] float32 or NULL;
 *   d_err          [B][iters] float64 or NULL; d_states_out [B][H][W][2] or NULL.
 * With the LUT start, target b draws its initial phases at start_index + b*H*W + p: the
 * targets continue the table like consecutive frames (Fig. 3; Section 8's rule for GS
 * video: every frame gets fresh phases). Each target's results equal those of gs_iterate
 * with start_index + b*H*W, in either precision. 1 <= B <= 65535 and B*H*W <= 2^31; other
 * arguments (the tensor-core precisions included) and errors as gs_iterate.
 * gs_batch_workspace_size gives the workspace of B targets.
 */
int gs_batch_workspace_size(int B, int H, int W, int iters, int precision, size_t* bytes);
int gs_iterate_batch(const float* d_targets, int B, int H, int W, int iters, int levels,
                     const float* d_init_phases, const uint8_t* d_codes, int64_t L, int lut_levels,
                     uint64_t seed, int64_t start_index, int precision, uint8_t* d_phase_codes,
                     float* d_replay, double* d_err, const float* d_states_in, float* d_states_out,
                     void* d_ws, size_t ws_bytes, holo_stream_t s);

/*
 * gs_state_phase - the replay-plane phase of a GS state (Section 2: GS keeps the phase of
 * the replay field and resets its amplitude to the target): d_phase[p] = arg(E_p) in
 * (-pi, pi] with arg(0) = 0, E = d_state (the [H][W][2] float32 (re, im) field that
 * gs_iterate writes to d_state_out). It is the label the warm-start network is trained
 * on (the phase GS reached after its iterations). One elementwise launch on s; d_phase
 * [H][W] float32 is caller-owned. 1 <= H*W <= 2^28, any H and W. Errors: HOLO_EINVAL,
 * HOLO_ECUDA.
 */
int gs_state_phase(const float* d_state, int H, int W, float* d_phase, holo_stream_t s);

/*
 * GS tile variants per shape (an engineering choice, not part of the method): the column
 * passes and the row pass each have variants 0..2 for line lengths 512..2048 (variant 0
 * only for other lengths; other values fall back to 0). Every variant computes the same
 * values up to float32 rounding order. Defaults are the fastest measured on GB300
 * (1024: column 0, row 1; 2048: column 1, row 1). gs_tuning_set with a negative variant
 * restores the defaults of the shape. Host-only calls; HOLO_EINVAL outside -1..2.
 */
int gs_tuning_set(int H, int W, int col_variant, int row_variant);
int gs_tuning_get(int H, int W, int* col_variant, int* row_variant);

/* ------------------------------------------------------- learned warm start ---- */

/*
 * A learned GS starting phase. Not in the paper: an engineering extension whose fallback
 * and judge is the paper's random start (Section 3). A 4-level convolutional
 * encoder-decoder (3x3 convolutions, 32/64/128/128 channels, 2x2 average pooling, nearest
 * 2x upsampling with additive skips, ReLU) maps a target amplitude, area-averaged to
 * 256x256, to two channels (u, v) whose angle is the predicted replay-plane phase. It is
 * trained on (target, phase) pairs produced by gs_iterate with the offset-invariant loss
 * L = mean_b [1 - |sum_p w_p y_p conj(z_p)| / sum_p w_p], y = (u+iv)/|u+iv|, z = exp(i
 * label), w = target^2 (a global phase offset, which GS leaves free, costs nothing).
 * Weights are float32 masters with Adam (beta 0.9/0.999, eps 1e-8); every convolution
 * runs as a bf16 implicit GEMM on the tensor cores with float32 accumulation.
 *
 * The network owns its device memory (parameters, optimizer state and activations for
 * up to max_batch samples; HOLO_ENOMEM if allocation fails) on the device current at
 * creation; calls must run with that device current.
 *   ws_net_create      seeded He-normal initialisation (SplitMix64 + Box-Muller).
 *   ws_train_step      one Adam step on a batch: d_targets [batch][256][256] float32
 *                      amplitudes, d_label_phase [batch][256][256] radians; d_loss
 *                      (nullable) receives the batch loss (float32, device).
 *   ws_forward_backward  the same without the update (gradients readable by ws_get_tensor).
 *   ws_infer           one target d_target [H][W] (square, H a multiple of 256) ->
 *                      d_phase_out [H][W] radians: the 256x256 prediction resampled
 *                      bilinearly on (u, v); feed it to gs_iterate's d_init_phase.
 *   ws_get_tensor / ws_set_tensor  host copies of layer `layer` (0..11): which = 0 weights
 *                      [Cout][3][3][Cin], 1 biases, 2 weight gradients, 3 bias gradients
 *                      (set: 0 and 1 only); count must equal the tensor size.
 *   ws_layer_shape     input channels, output channels and resolution of a layer.
 *   ws_get_activation  host float32 copy of a stored tensor of the last forward/backward
 *                      for `batch` samples: "x0" (input), "a1" "s1" "p1" "a2" "s2" "p2" "a3"
 *                      "s3" "p3" "a4" "b4" "up4" "u5" "up5" "u6" "up6" "u7" (activations),
 *                      "out" (float32 head output, 8 channels), "g_out" "g_u7" "g_up6"
 *                      "g_u6" "g_s1" (gradients); count must equal the tensor size.
 *   ws_save / ws_load  weights and Adam state to / from a binary file.
 */
typedef struct ws_net ws_net;
int ws_net_create(ws_net** out, uint64_t seed, int max_batch);
int ws_net_destroy(ws_net* net);
int ws_net_param_count(const ws_net* net, int64_t* count);
int ws_train_step(ws_net* net, const float* d_targets, const float* d_label_phase, int batch, float lr,
                  float* d_loss, holo_stream_t s);
int ws_forward_backward(ws_net* net, const float* d_targets, const float* d_label_phase, int batch,
                        float* d_loss, holo_stream_t s);
int ws_infer(ws_net* net, const float* d_target, int H, int W, float* d_phase_out, holo_stream_t s);
int ws_get_tensor(const ws_net* net, int layer, int which, float* h_out, int64_t count);
int ws_set_tensor(ws_net* net, int layer, int which, const float* h_in, int64_t count);
int ws_layer_shape(int layer, int* cin, int* cout, int* resolution);
int ws_get_activation(const ws_net* net, const char* name, int batch, float* h_out, int64_t count);
int ws_save(const ws_net* net, const char* path);
int ws_load(ws_net* net, const char* path);

/*
 * ws_phase_resample - the last step of ws_infer on its own: the network's head output
 * d_uv [H][W][channels] float32 (u in channel 0, v in channel 1; channels >= 2 is the
 * pixel stride) is resampled bilinearly to Ho x Wo and d_phase [Ho][Wo] float32 receives
 * atan2(v, u) in (-pi, pi]. Sampling: output (oy, ox) sits at input coordinates
 * sy = (oy + 1/2)*H/Ho - 1/2, sx = (ox + 1/2)*W/Wo - 1/2, clamped to [0, H-1] and [0, W-1];
 * the four neighbours floor(s) and min(floor(s) + 1, size - 1) are weighted by the
 * fractional parts. Any sizes (non-integer scales included) with H*W*channels <= 2^31 and
 * Ho*Wo <= 2^31. One launch on s; caller-owned buffers. Not in the paper: it maps the
 * learned start onto gs_iterate's grid. Errors: HOLO_EINVAL, HOLO_ECUDA.
 *
 * ws_adam_update - the optimizer step ws_train_step applies to every parameter tensor
 * (Kingma and Ba, 2015, Algorithm 1) on caller buffers of n float32 values:
 *   m = beta1*m + (1-beta1)*g;  v = beta2*v + (1-beta2)*g^2;
 *   w -= lr * (m / (1 - beta1^step)) / (sqrt(v / (1 - beta2^step)) + eps)
 * in place on d_w, d_m, d_v; d_g is read. step >= 1 is the update's 1-based count,
 * 0 <= beta1, beta2 < 1, eps >= 0, 1 <= n <= 2^31. One launch on s. Errors: HOLO_EINVAL,
 * HOLO_ECUDA.
 */
int ws_phase_resample(const float* d_uv, int channels, int H, int W, int Ho, int Wo, float* d_phase,
                      holo_stream_t s);
int ws_adam_update(float* d_w, const float* d_g, float* d_m, float* d_v, int64_t n, float lr, float beta1,
                   float beta2, float eps, int step, holo_stream_t s);

/*
 * nn_conv3x3 - the network's convolution kernel on its own (3x3, zero padding 1, stride
 * 1, channels-last bf16 tensors, channels multiples of 8, float32 accumulation). Modes 0
 * and 1 run on the tcgen05 tensor cores (accumulator in tensor memory) when the output
 * width is 32, 64 or 128, the input has at least 32 channels and every tensor is 16-byte
 * aligned, else on the mma.sync kernel;
 * mode | HOLO_CONV_LEGACY forces the mma.sync kernel (for comparisons). Mode 2 always
 * uses the mma.sync kernel.
 *   mode 0 forward: d_out[p][o] = act(sum X(p,k) W[o][k] + bias[o] + residual[p][o]) with
 *          d_in [B][H][W][Cin], d_wmat [Cout][9*Cin] bf16, bias/residual nullable,
 *          outputs bf16 d_out and/or float32 d_out_f32;
 *   mode 1 input gradient: as mode 0 with d_in = dy [B][H][W][Cin] and d_wmat the
 *          transposed weights [Cout][9*Cin] = W^T of the layer, offsets flipped;
 *   mode 2 weight gradient: d_dw [Cout][9*Cin] float32 += sum_p d_dy[p][o] X(p, k) with
 *          d_in = x [B][H][W][Cin], d_dy [B][H][W][Cout].
 */
#define HOLO_CONV_LEGACY 16
int nn_conv3x3(int mode, int B, int H, int W, int Cin, int Cout, const void* d_in, const void* d_wmat,
               const void* d_dy, const float* d_bias, const void* d_residual, int relu, void* d_out,
               float* d_out_f32, float* d_dw, holo_stream_t s);

/*
 * holo_tc_status - the tcgen05 kernels (the convolutions, the DFT-32 stages of the
 * tensor-core precisions) bound every wait on their mbarriers, and the persistent batch
 * kernel every wait on a dependency counter; a wait that expires sets a device flag (the
 * convolution then skips its outputs; results of a DFT stage or of the persistent batch
 * are not to be trusted). Writes whether any flag is set to *fault (0 = never) and clears the flags
 * when `clear` is nonzero. Synchronous (reads device memory).
 */
int holo_tc_status(int* fault, int clear);

/*
 * holo_wait_selftest - exercises the bounded-wait path of the tcgen05 kernels without a
 * fault: one warp waits on an mbarrier that nothing arrives at, gives up after `limit`
 * polls (1 .. 2^24) and sets the same device flag a real expiry sets. Synchronises s.
 * Returns HOLO_ETIMEOUT (the expected result) with the flag set; holo_check then reports
 * HOLO_ETIMEOUT too until holo_tc_status clears the flag. The context stays usable.
 */
int holo_wait_selftest(int limit, holo_stream_t s);

/* ------------------------------------------------------------ replay error ---- */

/*
 * replay_error_workspace_size - bytes of device workspace replay_error needs.
 */
int replay_error_workspace_size(int H, int W, size_t* bytes);

/*
 * replay_error - error of a replay intensity against its target (Section 5.2, Eq. 3),
 * with the intensity-domain, optimal-scale reading:
 *   alpha = sum(I*T^2) / sum(I^2);  mse = sum((alpha*I - T^2)^2) / P;
 *   nmse  = sum((alpha*I - T^2)^2) / sum(T^4)
 * One pass over the pixels: every block of 4096 pixels also forms its squared error at
 * its own scale a_b and the sum of I*(a_b*I - T^2); the last block to finish reduces the
 * blocks and writes alpha, mse and nmse through the exact identity
 *   sum (alpha I - T^2)^2 = sum_b [S1_b + 2 (alpha - a_b) S2_b + (alpha - a_b)^2 sum_b I^2],
 * whose terms do not cancel. Each thread sums its 16 pixels' terms in float32
 * (single-rounding fmaf); sums across threads and blocks are float-float (about 48
 * significant bits) in a fixed order, so results are bit-reproducible; only the three
 * outputs are float64. The workspace holds the block partial sums and a completion
 * counter that the call clears on the stream (cudaMemsetAsync) before its one launch.
 *
 *   d_replay  [H][W] float32 intensity I.   d_target [H][W] float32 amplitude T.
 *   d_mask    [H][W] uint8 or NULL: nonzero pixels are included (P = their count).
 *   H, W      any sizes with 1 <= H*W <= 2^28 (not restricted to powers of two).
 *   d_out     [3] float64 output: alpha, mse, nmse.
 * Errors: HOLO_EINVAL, HOLO_EWORKSPACE, HOLO_ECUDA.
 */
int replay_error(const float* d_replay, const float* d_target, const uint8_t* d_mask,
                 int H, int W, double* d_out, void* d_ws, size_t ws_bytes,
                 holo_stream_t s);

#ifdef __cplusplus
}
#endif

#endif /* HOLO_H */
