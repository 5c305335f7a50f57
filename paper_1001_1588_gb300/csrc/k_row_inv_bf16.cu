// Inverse row pass, BF16 storage.
#include "k_rows.cuh"

namespace fftenkf {
cudaError_t launch_row_inv_bf16(const RowInvParams& p, int n_fields, cudaStream_t s) {
  return launch_row_inv_st<kBF16>(p, n_fields, s);
}
}  // namespace fftenkf
