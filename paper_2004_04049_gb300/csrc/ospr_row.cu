// ospr_row.cu - launchers of the OSPR row pass (row IDFT, binarise, row DFT) for every
// supported row length and tile variant.
#include "ospr_kernels.cuh"

namespace holo {

template <int NR, int V, bool REPLAY, bool FRESNEL>
static int launch_row(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = row_smem_bytes<NR, V>();
    void (*kern)(OsprArgs) = k_ospr_row<NR, V, REPLAY, FRESNEL>;
    int rc = ensure_smem((const void*)kern, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.H / RowCfg<NR, V>::LPR, a.pairs);
    Launch ln("ospr_row", st);
    const cudaError_t le =
        launch_pdl(kern, grid, dim3((NR / RowCfg<NR, V>::R) * RowCfg<NR, V>::LPR), smem, st, a);
    return ln.done("ospr_row launch", le);
}

template <int NR, int V>
static int launch_row_any(const OsprArgs& a, bool replay, cudaStream_t st) {
    if (a.fresnel) return replay ? launch_row<NR, V, true, true>(a, st) : launch_row<NR, V, false, true>(a, st);
    return replay ? launch_row<NR, V, true, false>(a, st) : launch_row<NR, V, false, false>(a, st);
}

int ospr_run_row(const OsprArgs& a, int v, bool replay, cudaStream_t st) {
    switch (a.W) {
        case 64: return launch_row_any<64, 0>(a, replay, st);
        case 128: return launch_row_any<128, 0>(a, replay, st);
        case 256: return launch_row_any<256, 0>(a, replay, st);
        case 512: return v ? launch_row_any<512, 1>(a, replay, st) : launch_row_any<512, 0>(a, replay, st);
        case 1024: return v ? launch_row_any<1024, 1>(a, replay, st) : launch_row_any<1024, 0>(a, replay, st);
        case 2048: return v ? launch_row_any<2048, 1>(a, replay, st) : launch_row_any<2048, 0>(a, replay, st);
        case 4096: return v ? launch_row_any<4096, 1>(a, replay, st) : launch_row_any<4096, 0>(a, replay, st);
        default: return fail(HOLO_EUNSUPPORTED, "row length %d", a.W);
    }
}

}  // namespace holo
