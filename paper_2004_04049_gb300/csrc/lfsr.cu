// lfsr.cu - m-sequence phase codes, the PRNG alternative of Section 7 (an m-sequence
// generator feeding the cos/sin table), for comparison with the LUT of Sections 4-5.
//
// Galois LFSR over GF(2) with the primitive feedback polynomial p(x) = x^31 + x^3 + 1:
// state s_k = s_0 * x^k mod p (bit j = coefficient of x^j), output bit b_k = coefficient of
// x^30 in s_k. Code i (levels = 2^m) packs b_{m i} .. b_{m i + m - 1}, most significant
// first. Each thread produces a run of kLfsrRun consecutive codes: it jumps to its first
// bit by multiplying s_0 with x^(2^j) mod p for the set bits j of the bit position (the 64
// powers are a constant table made on the host), then steps the register m times per code.
#include <mutex>

#include "runtime.h"

namespace holo {

constexpr uint32_t kLfsrLow = (1u << 3) | 1u;   // p(x) without its x^31 term
constexpr uint32_t kLfsrMask = 0x7FFFFFFFu;
constexpr int kLfsrRun = 512;   // codes per thread (a multiple of 16)

__host__ __device__ __forceinline__ uint32_t lfsr_step(uint32_t s) {
    return ((s << 1) & kLfsrMask) ^ ((s >> 30) ? kLfsrLow : 0u);
}

// a * b mod p: shift-and-add over the 31 coefficients of b
__host__ __device__ __forceinline__ uint32_t lfsr_mulmod(uint32_t a, uint32_t b) {
    uint32_t r = 0;
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
    for (int i = 0; i < 31; ++i) {
        r ^= (b & 1u) ? a : 0u;
        b >>= 1;
        a = lfsr_step(a);
    }
    return r;
}

__constant__ uint32_t c_xpow[64];   // x^(2^j) mod p

__device__ __forceinline__ uint32_t lfsr_code(uint32_t& s, int bits) {
    uint32_t c = 0;
    for (int b = 0; b < bits; ++b) {
        c = (c << 1) | (s >> 30);
        s = lfsr_step(s);
    }
    return c;
}

// vec16: the output is 16-byte aligned, so full groups of 16 codes go out as one uint4
// store (byte stores from threads 512 bytes apart would each cost a separate sector write)
__global__ void k_lfsr_codes(uint32_t s0, uint64_t start, int64_t count, int bits, int vec16,
                             uint8_t* __restrict__ codes) {
    pdl_wait();   // a previous kernel may still read the buffer being rewritten
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t c0 = t * kLfsrRun;
    if (c0 >= count) return;
    uint64_t k = uint64_t(bits) * (start + uint64_t(c0));   // first output bit of the run
    uint32_t s = s0;
    for (int j = 0; j < 64 && k; ++j, k >>= 1)
        if (k & 1u) s = lfsr_mulmod(s, c_xpow[j]);
    const int64_t n = count - c0 < kLfsrRun ? count - c0 : kLfsrRun;
    int64_t i = 0;
    if (vec16) {
        for (; i + 16 <= n; i += 16) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t v = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) v |= lfsr_code(s, bits) << (8 * b);
                w[q] = v;
            }
            *reinterpret_cast<uint4*>(codes + c0 + i) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    for (; i < n; ++i) codes[c0 + i] = uint8_t(lfsr_code(s, bits));
}

// fills the power table on the current device once
static int lfsr_tables() {
    static std::mutex mu;
    static bool dev_done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "lfsr: cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(HOLO_EUNSUPPORTED, "lfsr: device %d", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev_done[dev]) return HOLO_OK;
    uint32_t pw[64];
    uint32_t x = 2u;   // the polynomial x
    for (int j = 0; j < 64; ++j) {
        pw[j] = x;
        x = lfsr_mulmod(x, x);
    }
    if ((e = cudaMemcpyToSymbol(c_xpow, pw, sizeof(pw))) != cudaSuccess) return cuda_status(e, "lfsr: table");
    dev_done[dev] = true;
    return HOLO_OK;
}

}  // namespace holo

using namespace holo;

extern "C" int lfsr_build(uint32_t seed_state, int64_t start, int64_t count, int levels, uint8_t* d_codes,
                          holo_stream_t s) {
    clear_error();
    if (seed_state == 0 || seed_state > kLfsrMask)
        return fail(HOLO_EINVAL, "lfsr_build: seed_state %u must be in [1, 2^31 - 1]", seed_state);
    if (count < 1 || count > INT64_C(0x7FFFFFFF) || start < 0 || start > (INT64_C(1) << 56))
        return fail(HOLO_EINVAL, "lfsr_build: start %lld / count %lld out of range", (long long)start,
                    (long long)count);
    if (!is_pow2(levels) || levels < 2 || levels > 256)
        return fail(HOLO_EINVAL, "lfsr_build: levels=%d is not a power of two in [2, 256]", levels);
    if (!d_codes) return fail(HOLO_EINVAL, "lfsr_build: d_codes is NULL");
    int rc = lfsr_tables();
    if (rc) return rc;
    const int64_t threads = (count + kLfsrRun - 1) / kLfsrRun;
    const int block = 128;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    Launch ln("lfsr_build", st);
    const int vec16 = (reinterpret_cast<uintptr_t>(d_codes) & 15) == 0;
    const cudaError_t le = launch_pdl(k_lfsr_codes, dim3(unsigned((threads + block - 1) / block)), dim3(block), 0, st,
                                      seed_state, uint64_t(start), count, log2i(levels), vec16, d_codes);
    return ln.done("lfsr_build launch", le);
}
