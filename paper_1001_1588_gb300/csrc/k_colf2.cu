// Fused column pass, instantiated for 2 observed block(s).
#include "k_colf.cuh"

namespace fftenkf {
cudaError_t col_fused_nobs2(const ColFusedParams& p, cudaStream_t s) { return col_fused_dispatch<2>(p, s); }
}  // namespace fftenkf
