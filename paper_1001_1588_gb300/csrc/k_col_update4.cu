// Instantiation of the column update pass for up to 4 observed block(s).
#include "k_cols.cuh"

namespace fftenkf {
cudaError_t col_update_nobs4(const ColUpdParams& p, cudaStream_t s) { return col_update_dispatch<4>(p, s); }
}  // namespace fftenkf
