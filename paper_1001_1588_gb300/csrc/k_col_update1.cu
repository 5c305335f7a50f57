// Instantiation of the column update pass for up to 1 observed block(s).
#include "k_cols.cuh"

namespace fftenkf {
cudaError_t col_update_nobs1(const ColUpdParams& p, cudaStream_t s) { return col_update_dispatch<1>(p, s); }
}  // namespace fftenkf
