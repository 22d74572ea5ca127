// nn_conv_tc05.cu - the 3x3 convolution of the warm-start network (forward and input
// gradient) as an implicit GEMM on the 5th-generation tensor cores: tcgen05.mma with
// bf16 operands staged in shared memory and a float32 accumulator in tensor memory.
//
// GEMM view (as nn_conv.cu): M = pixels, N = output channels (32, 64 or 128), K = 9*Cin
// ordered (tap, channel). One CTA of 128 threads owns 128 consecutive pixels (the 128
// TMEM lanes) and all N columns:
//   * every thread gathers the 64-element K slice of its own pixel (8 x 16-byte cp.async,
//     zero-filled outside the image or past K) and a share of the weight rows, into a
//     4-stage ring of shared-memory tiles in the canonical K-major 128-byte-swizzle layout
//     (row r of a tile at (r/8)*1024 + (r%8)*128, its 16-byte chunk j at chunk j^(r%8));
//   * thread 0 issues four 128xNx16 MMAs per slice and commits them to the slice's
//     mbarrier, which frees the stage for the copy of slice + 4 (copies run two slices
//     ahead, so the MMAs of one slice overlap the next slice's issue);
//   * after the last slice every warp reads its 32 TMEM lanes (tcgen05.ld 32x32b), adds
//     bias and residual, applies the ReLU and stores bf16 (and optionally float32) rows.
// Every mbarrier wait is bounded: on expiry the kernel records the failure in a device
// flag, stops issuing work, drains its copies, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "nn.h"
#include "runtime.h"

namespace holo {
namespace nn {

constexpr int kTcM = 128;        // pixels per CTA = TMEM lanes
constexpr int kTcK = 64;         // K elements per stage: one 128-byte swizzled row
constexpr int kTcStages = 4;
constexpr int kTcThreads = 128;
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ int g_tc05_fault;     // set when a bounded wait expired

template <int N>
struct Tc05Layout {
    static constexpr int kA = kTcM * 128;            // bytes of an A stage
    static constexpr int kB = N * 128;               // bytes of a B stage
    static constexpr int kStage = kA + kB;
    static constexpr int kBar = kTcStages * kStage;  // mbarriers after the stages
    static constexpr int kBytes = kBar + 8 * kTcStages + 1024;   // + alignment slack
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
// true once the phase with the given parity has completed; false if the limit expired
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
           (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

// instruction descriptor of kind::f16: bf16 A and B (K-major), float32 D, M = 128
template <int N>
__host__ __device__ constexpr uint32_t idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(kTcM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

// 32 consecutive float32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

template <int N>
__global__ void __launch_bounds__(kTcThreads) k_conv3x3_tc05(ConvArgs a) {
    using Lay = Tc05Layout<N>;
    extern __shared__ uint8_t smraw[];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fault;
    // stage tiles start on a 1024-byte boundary (swizzle atoms)
    const uint32_t raw = smem_u32(smraw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t bar0 = base + Lay::kBar;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int HW = a.H * a.W;
    const int M = a.B * HW, K = 9 * a.Cin;
    const int m0 = blockIdx.x * kTcM;
    const int nk = (K + kTcK - 1) / kTcK;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "n"(N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) mbar_init(bar0 + 8 * s, 1);
        s_fault = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // this thread's pixel (GEMM row) and its image coordinates
    const int m = m0 + tid;
    const bool mvalid = m < M;
    const int pb = mvalid ? m / HW : 0, prem = mvalid ? m - pb * HW : 0;
    const int py = prem / a.W, px = prem - py * a.W;
    const uint32_t arow = uint32_t(tid >> 3) * 1024u + uint32_t(tid & 7) * 128u;

    auto load_stage = [&](int kc, int s) {
        const uint32_t As = base + uint32_t(s) * Lay::kStage;
        const uint32_t Bs = As + Lay::kA;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int k = kc * kTcK + v * 8;
            const int tap = k / a.Cin, ci = k - tap * a.Cin;
            const int ky = tap / 3, kx = tap - 3 * ky;
            const int yy = a.flip ? py + 1 - ky : py + ky - 1;
            const int xx = a.flip ? px + 1 - kx : px + kx - 1;
            const bool ok = mvalid && k < K && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
            const __nv_bfloat16* src = ok ? a.in + ((size_t(pb) * a.H + yy) * a.W + xx) * a.Cin + ci : a.in;
            cp_async16(As + arow + (uint32_t(v ^ (tid & 7)) << 4), src, ok ? 16u : 0u);
        }
#pragma unroll
        for (int i = 0; i < N / 16; ++i) {
            const int idx = tid + kTcThreads * i;
            const int n = idx >> 3, v = idx & 7;
            const int k = kc * kTcK + v * 8;
            const bool ok = k < K;
            const __nv_bfloat16* src = ok ? a.wmat + size_t(n) * K + k : a.wmat;
            cp_async16(Bs + uint32_t(n >> 3) * 1024u + uint32_t(n & 7) * 128u + (uint32_t(v ^ (n & 7)) << 4), src,
                       ok ? 16u : 0u);
        }
        cp_async_commit();
    };

    // Pipeline: slice kc is consumed from stage kc % 4 while slices kc+1 (copy landing) and
    // kc-1 (MMAs running) hold two more stages; the fourth stage, freed by slice kc-2's MMA
    // commit, receives slice kc+2. Thread 0 is the only waiter on the mbarriers and the
    // block-wide vote that follows makes every branch uniform.
    constexpr uint32_t idesc = idesc_bf16<N>();
    constexpr int kAhead = kTcStages - 2;
    for (int s = 0; s < kAhead; ++s) {
        if (s < nk) load_stage(s, s);
        else cp_async_commit();
    }
    int issued = -1;   // last slice whose MMAs were committed
    int bad = 0;
    for (int kc = 0; kc < nk; ++kc) {
        const int s = kc % kTcStages;
        cp_async_wait<kAhead - 1>();
        // the tensor cores read shared memory through the async proxy
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        int w = 0;
        if (tid == 0 && kc >= 2) {
            const int j = kc - 2;
            w = !mbar_wait(bar0 + 8 * (j % kTcStages), uint32_t((j / kTcStages) & 1));
        }
        if (__syncthreads_or(w)) {
            bad = 1;
            break;
        }
        if (tid == 0) {
            tc_fence_after();
            const uint32_t As = base + uint32_t(s) * Lay::kStage;
            const uint32_t Bs = As + Lay::kA;
#pragma unroll
            for (int kk = 0; kk < kTcK / 16; ++kk)
                mma_bf16(tmem, sw128_desc(As + 32u * kk), sw128_desc(Bs + 32u * kk), idesc, (kc | kk) != 0);
            mma_commit(bar0 + 8 * s);
        }
        issued = kc;
        const int next = kc + kAhead;
        if (next < nk) load_stage(next, next % kTcStages);
        else cp_async_commit();
    }
    // every MMA done (commits complete in order), or on a fault the last one issued
    int w = 0;
    if (tid == 0 && issued >= 0)
        w = !mbar_wait(bar0 + 8 * (issued % kTcStages), uint32_t((issued / kTcStages) & 1));
    cp_async_wait<0>();
    if (__syncthreads_or(w) || bad) s_fault = 1;
    __syncthreads();
    tc_fence_after();
    if (s_fault) {
        if (tid == 0) atomicExch(&g_tc05_fault, 1);
    } else {
        const uint32_t lane_base = uint32_t(32 * warp) << 16;
        const int row = m0 + 32 * warp + lane;
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + lane_base + uint32_t(c0), r);
            if (row < M) {
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]) + (a.bias ? a.bias[c0 + j] : 0.f);
                const size_t o = size_t(row) * N + c0;
                if (a.residual) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint4 rv = *reinterpret_cast<const uint4*>(a.residual + o + 8 * q);
                        const __nv_bfloat162* r2 = reinterpret_cast<const __nv_bfloat162*>(&rv);
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const float2 f = __bfloat1622float2(r2[h]);
                            v[8 * q + 2 * h] += f.x;
                            v[8 * q + 2 * h + 1] += f.y;
                        }
                    }
                }
                if (a.relu) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j], 0.f);
                }
                if (a.out) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint4 w;
                        __nv_bfloat162* w2 = reinterpret_cast<__nv_bfloat162*>(&w);
#pragma unroll
                        for (int h = 0; h < 4; ++h) w2[h] = __floats2bfloat162_rn(v[8 * q + 2 * h], v[8 * q + 2 * h + 1]);
                        *reinterpret_cast<uint4*>(a.out + o + 8 * q) = w;
                    }
                }
                if (a.out_f32) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *reinterpret_cast<float4*>(a.out_f32 + o + 4 * q) =
                            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(N) : "memory");
}

template <int N>
static int launch_tc05(const ConvArgs& a, cudaStream_t st, const char* family) {
    static uint64_t mask = 0;
    constexpr size_t smem = Tc05Layout<N>::kBytes;
    int rc = ensure_smem((const void*)k_conv3x3_tc05<N>, smem, &mask);
    if (rc) return rc;
    const int M = a.B * a.H * a.W;
    Launch ln(family, st);
    k_conv3x3_tc05<N><<<(M + kTcM - 1) / kTcM, kTcThreads, smem, st>>>(a);
    return ln.done("nn_conv tcgen05 launch");
}

bool conv3x3_tc05_supported(const ConvArgs& a) {
    auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    // with fewer than 32 input channels a K slice is mostly padding (K = 9*Cin) and the
    // mma.sync kernel is faster (measured: 8 -> 32 channels at 256^2)
    return a.Cin % 8 == 0 && a.Cin >= 32 && (a.Cout == 32 || a.Cout == 64 || a.Cout == 128) && al16(a.in) &&
           al16(a.wmat) &&
           al16(a.residual) && al16(a.out) && al16(a.out_f32);
}

int conv3x3_tc05(const ConvArgs& a, int mode, cudaStream_t st) {
    const char* family = mode == kConvFwd ? "nn_conv_fwd" : "nn_conv_dgrad";
    switch (a.Cout) {
        case 32: return launch_tc05<32>(a, st, family);
        case 64: return launch_tc05<64>(a, st, family);
        case 128: return launch_tc05<128>(a, st, family);
        default: return fail(HOLO_EUNSUPPORTED, "conv3x3_tc05: N=%d", a.Cout);
    }
}

int conv3x3_tc05_fault(int* out, bool clear) {
    int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc05_fault, sizeof(int));
    if (e != cudaSuccess) return cuda_status(e, "conv3x3_tc05_fault");
    if (clear && v) {
        const int z = 0;
        if ((e = cudaMemcpyToSymbol(g_tc05_fault, &z, sizeof(int))) != cudaSuccess)
            return cuda_status(e, "conv3x3_tc05_fault");
    }
    *out = v;
    return HOLO_OK;
}

}  // namespace nn
}  // namespace holo
