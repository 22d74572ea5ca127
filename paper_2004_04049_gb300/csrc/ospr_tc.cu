// ospr_tc.cu - launchers of the OSPR passes whose radix-32 DFT stages run on the tensor
// cores (split fp16 or bf16 operands, float32 accumulation), for line lengths 1024 and 2048.
#include "ospr_kernels.cuh"

namespace holo {

template <int NC, int PREC>
static int launch_col_ifft_tc(const OsprArgs& a, cudaStream_t st) {
    constexpr int V = kTcColVariant;
    static uint64_t mask = 0;
    constexpr size_t smem = col_ifft_smem_bytes<NC, V, PREC>();
    int rc = ensure_smem((const void*)k_ospr_col_ifft<NC, V, PREC>, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.W / ColCfg<NC, V>::LPC, a.pairs);
    Launch ln("ospr_col_ifft", st);
    const cudaError_t le = launch_pdl(k_ospr_col_ifft<NC, V, PREC>, grid, dim3((NC / ColCfg<NC, V>::R) * ColCfg<NC, V>::LPC), smem, st, a);
    return ln.done("ospr_col_ifft launch", le);
}

template <int NC, int PREC>
static int launch_col_fft_tc(const OsprArgs& a, cudaStream_t st) {
    constexpr int V = kTcColVariant;
    static uint64_t mask = 0;
    constexpr size_t smem = col_fft_smem_bytes<NC, V, PREC>();
    int rc = ensure_smem((const void*)k_ospr_col_fft<NC, V, PREC>, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.W / ColCfg<NC, V>::LPC, a.groups);
    Launch ln("ospr_col_fft", st);
    const cudaError_t le = launch_pdl(k_ospr_col_fft<NC, V, PREC>, grid, dim3((NC / ColCfg<NC, V>::R) * ColCfg<NC, V>::LPC), smem, st, a);
    return ln.done("ospr_col_fft launch", le);
}

template <int NR, int PREC, bool REPLAY>
static int launch_row_tc(const OsprArgs& a, cudaStream_t st) {
    constexpr int V = kTcRowVariant;
    static uint64_t mask = 0;
    constexpr size_t smem = row_smem_bytes<NR, V, PREC>();
    int rc = ensure_smem((const void*)k_ospr_row<NR, V, REPLAY, PREC>, smem, &mask);
    if (rc) return rc;
    dim3 grid(a.H / RowCfg<NR, V>::LPR, a.pairs);
    Launch ln("ospr_row", st);
    const cudaError_t le = launch_pdl(k_ospr_row<NR, V, REPLAY, PREC>, grid, dim3((NR / RowCfg<NR, V>::R) * RowCfg<NR, V>::LPR), smem, st, a);
    return ln.done("ospr_row launch", le);
}

int ospr_run_col_ifft_tc(const OsprArgs& a, int prec, cudaStream_t st) {
    if (a.H == 1024) return prec == kTcBf16 ? launch_col_ifft_tc<1024, kTcBf16>(a, st) : launch_col_ifft_tc<1024, kTcFp16>(a, st);
    if (a.H == 2048) return prec == kTcBf16 ? launch_col_ifft_tc<2048, kTcBf16>(a, st) : launch_col_ifft_tc<2048, kTcFp16>(a, st);
    return fail(HOLO_EUNSUPPORTED, "tensor-core stages: column length %d", a.H);
}
int ospr_run_col_fft_tc(const OsprArgs& a, int prec, cudaStream_t st) {
    if (a.H == 1024) return prec == kTcBf16 ? launch_col_fft_tc<1024, kTcBf16>(a, st) : launch_col_fft_tc<1024, kTcFp16>(a, st);
    if (a.H == 2048) return prec == kTcBf16 ? launch_col_fft_tc<2048, kTcBf16>(a, st) : launch_col_fft_tc<2048, kTcFp16>(a, st);
    return fail(HOLO_EUNSUPPORTED, "tensor-core stages: column length %d", a.H);
}
int ospr_run_row_tc(const OsprArgs& a, int prec, bool replay, cudaStream_t st) {
    if (a.W == 1024) {
        if (prec == kTcBf16) return replay ? launch_row_tc<1024, kTcBf16, true>(a, st) : launch_row_tc<1024, kTcBf16, false>(a, st);
        return replay ? launch_row_tc<1024, kTcFp16, true>(a, st) : launch_row_tc<1024, kTcFp16, false>(a, st);
    }
    if (a.W == 2048) {
        if (prec == kTcBf16) return replay ? launch_row_tc<2048, kTcBf16, true>(a, st) : launch_row_tc<2048, kTcBf16, false>(a, st);
        return replay ? launch_row_tc<2048, kTcFp16, true>(a, st) : launch_row_tc<2048, kTcFp16, false>(a, st);
    }
    return fail(HOLO_EUNSUPPORTED, "tensor-core stages: row length %d", a.W);
}

}  // namespace holo
