// Storage-independent entry points of the row passes (the row kernels are in
// k_rows.cuh).
#include "k_rows.cuh"

namespace fftenkf {

cudaError_t launch_row_fwd(const RowFwdParams& p, int n_fields, cudaStream_t s) {
  return p.storage == kBF16 ? launch_row_fwd_bf16(p, n_fields, s) : launch_row_fwd_f32(p, n_fields, s);
}

bool row_line_supported(int n) {
  switch (n) {
#define CASE(m) case m: return true;
    FFTENKF_ROW_SIZES(CASE)
#undef CASE
    default: return false;
  }
}

template <int L>
int row_inv_rows_L(int vsel, int ny, int nx, int es) {
  const int V = (vsel & 1) ? plan_V(L, 1) : plan_V(L, 0);
  RowShape s = inv_shape(L, V, ny, nx, es, (vsel & 2) != 0);
  // tensor copies need R >= 2 (16-byte rows of the box)
  return (s.R < 2 || s.smem > 227 * 1024 || s.T * s.R > 512) ? 0 : s.R;
}

int row_inv_rows(int L, int vsel, int ny, int nx, int es) {
  switch (L) {
#define CASE(n) case n: return row_inv_rows_L<n>(vsel, ny, nx, es);
    FFTENKF_ROW_SIZES(CASE)
#undef CASE
    default: return 0;
  }
}

cudaError_t launch_row_inv(const RowInvParams& p, int n_fields, cudaStream_t s) {
  return p.storage == kBF16 ? launch_row_inv_bf16(p, n_fields, s) : launch_row_inv_f32(p, n_fields, s);
}

}  // namespace fftenkf
