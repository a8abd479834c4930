// Mixed-precision merge products (BF16 slices on tcgen05 tensor cores).
#include "bdc_internal.cuh"

namespace bdc {

size_t gemm_mixed_scratch(long long rows_total, long long cols_total, int kmax, int prec, int slices) {
    (void)rows_total; (void)cols_total; (void)kmax; (void)prec; (void)slices;
    return 256;
}

cudaError_t launch_gemm_mixed(const GemmProb *probs, int nprobs, int mmax_rows, int nmax_cols, int kmax,
                              int prec, int slices, void *scratch, size_t scratch_bytes, cudaStream_t st) {
    (void)probs; (void)nprobs; (void)mmax_rows; (void)nmax_cols; (void)kmax; (void)prec; (void)slices;
    (void)scratch; (void)scratch_bytes; (void)st;
    return cudaErrorNotSupported;
}

}  // namespace bdc
