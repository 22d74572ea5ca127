// ospr_col.cu - launchers of the OSPR column passes (build + column IDFT; column DFT +
// accumulate) for every supported column length and tile variant.
#include "ospr_kernels.cuh"

namespace holo {

// looping kernels: one CTA per resident slot (at most one per tile), each over every G-th
// tile; the others: one CTA per tile
template <int NC, int V>
static int launch_col_ifft(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    static int resident[64] = {};
    constexpr size_t smem = col_ifft_smem_bytes<NC, V>();
    constexpr int threads = (NC / ColCfg<NC, V>::R) * ColCfg<NC, V>::LPC;
    int rc = ensure_smem((const void*)k_ospr_col_ifft<NC, V>, smem, &mask);
    if (rc) return rc;
    const int tiles = a.W / ColCfg<NC, V>::LPC;
    dim3 grid(tiles, a.pairs);
    if constexpr (col_ifft_loops<NC, V>()) {
        int slots = 0;
        if ((rc = resident_ctas((const void*)k_ospr_col_ifft<NC, V>, threads, smem, resident, &slots))) return rc;
        grid = dim3(tiles * a.pairs < slots ? tiles * a.pairs : slots);
    }
    Launch ln("ospr_col_ifft", st);
    const cudaError_t le = launch_pdl(k_ospr_col_ifft<NC, V>, grid, dim3(threads), smem, st, a);
    return ln.done("ospr_col_ifft launch", le);
}

template <int NC, int V>
static int launch_col_fft(const OsprArgs& a, cudaStream_t st) {
    static uint64_t mask = 0;
    constexpr size_t smem = col_fft_smem_bytes<NC, V>();
    int rc = ensure_smem((const void*)k_ospr_col_fft<NC, V>, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.W / ColCfg<NC, V>::LPC, a.groups);
    Launch ln("ospr_col_fft", st);
    const cudaError_t le = launch_pdl(k_ospr_col_fft<NC, V>, grid, dim3((NC / ColCfg<NC, V>::R) * ColCfg<NC, V>::LPC), smem, st, a);
    return ln.done("ospr_col_fft launch", le);
}

#define HOLO_COL_VARIANTS(N, v, F) \
    (v == 2 ? F<N, 2>(a, st) : v == 1 ? F<N, 1>(a, st) : F<N, 0>(a, st))
#define HOLO_COL_SWITCH(n, v, F)                                              \
    switch (n) {                                                              \
        case 64: return F<64, 0>(a, st);                                      \
        case 128: return F<128, 0>(a, st);                                    \
        case 256: return F<256, 0>(a, st);                                    \
        case 512: return HOLO_COL_VARIANTS(512, v, F);                        \
        case 1024: return HOLO_COL_VARIANTS(1024, v, F);                      \
        case 2048: return HOLO_COL_VARIANTS(2048, v, F);                      \
        case 4096: return HOLO_COL_VARIANTS(4096, v, F);                      \
        default: return fail(HOLO_EUNSUPPORTED, "column length %d", n);      \
    }

int ospr_run_col_ifft(const OsprArgs& a, int v, cudaStream_t st) { HOLO_COL_SWITCH(a.H, v, launch_col_ifft) }
int ospr_run_col_fft(const OsprArgs& a, int v, cudaStream_t st) { HOLO_COL_SWITCH(a.H, v, launch_col_fft) }

}  // namespace holo
