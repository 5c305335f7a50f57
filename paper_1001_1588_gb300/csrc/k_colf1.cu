// Fused column pass, instantiated for 1 observed block(s).
#include "k_colf.cuh"

namespace fftenkf {
cudaError_t col_fused_nobs1(const ColFusedParams& p, cudaStream_t s) { return col_fused_dispatch<1>(p, s); }
}  // namespace fftenkf
