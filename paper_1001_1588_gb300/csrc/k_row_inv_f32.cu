// Inverse row pass, F32 storage.
#include "k_rows.cuh"

namespace fftenkf {
cudaError_t launch_row_inv_f32(const RowInvParams& p, int n_fields, cudaStream_t s) {
  return launch_row_inv_st<kF32>(p, n_fields, s);
}
}  // namespace fftenkf
