// lut.cu - the phase lookup table of Section 4 (a pool of L random phases generated once
// and then drawn sequentially; 8-bit entries per Section 5.2).
#include "phase_source.cuh"

namespace holo {

// entry k = top `bits` bits of SplitMix64 output k; optional (cos, sin) of its phase
__global__ void k_lut_build(uint64_t seed, int64_t L, int bits, int cs_shift,
                            uint8_t* __restrict__ codes, float2* __restrict__ cs,
                            const float2* __restrict__ cs256) {
    pdl_wait();   // a previous kernel may still read the table being rewritten
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < L; k += stride) {
        const uint32_t c = lut_entry(seed, uint64_t(k), bits);
        codes[k] = uint8_t(c);
        if (cs) cs[k] = __ldg(cs256 + (c << cs_shift));
    }
}

}  // namespace holo

using namespace holo;

extern "C" int lut_build(uint64_t seed, int64_t L, int levels, uint8_t* d_codes, float* d_cs,
                         holo_stream_t s) {
    clear_error();
    if (L < 1 || L > INT64_C(0x7FFFFFFF)) return fail(HOLO_EINVAL, "lut_build: L=%lld out of [1, 2^31-1]", (long long)L);
    if (!is_pow2(levels) || levels < 2 || levels > 256)
        return fail(HOLO_EINVAL, "lut_build: levels=%d is not a power of two in [2, 256]", levels);
    if (!d_codes) return fail(HOLO_EINVAL, "lut_build: d_codes is NULL");
    Tables tab;
    int rc = device_tables(&tab);
    if (rc != HOLO_OK) return rc;
    const int bits = log2i(levels);
    const int threads = 256;
    int64_t blocks = (L + threads - 1) / threads;
    if (blocks > 152 * 32) blocks = 152 * 32;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    Launch ln("lut_build", st);
    const cudaError_t le = launch_pdl(k_lut_build, dim3(int(blocks)), dim3(threads), 0, st, seed, L, bits, 8 - bits,
                                      d_codes, reinterpret_cast<float2*>(d_cs), tab.cs256);
    return ln.done("lut_build launch", le);
}
