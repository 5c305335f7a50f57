// Instantiation of the column update pass for up to 2 observed block(s).
#include "k_cols.cuh"

namespace fftenkf {
cudaError_t col_update_nobs2(const ColUpdParams& p, cudaStream_t s) { return col_update_dispatch<2>(p, s); }
}  // namespace fftenkf
