// Forward row pass, F32 storage.
#include "k_rows.cuh"

namespace fftenkf {
cudaError_t launch_row_fwd_f32(const RowFwdParams& p, int n_fields, cudaStream_t s) {
  return launch_row_fwd_st<kF32>(p, n_fields, s);
}
}  // namespace fftenkf
