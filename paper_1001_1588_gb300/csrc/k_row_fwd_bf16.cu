// Forward row pass, BF16 storage.
#include "k_rows.cuh"

namespace fftenkf {
cudaError_t launch_row_fwd_bf16(const RowFwdParams& p, int n_fields, cudaStream_t s) {
  return launch_row_fwd_st<kBF16>(p, n_fields, s);
}
}  // namespace fftenkf
