// Column-pass launchers: shared-memory sizing and dispatch on the number of
// observed blocks (one translation unit per instantiation, compiled in parallel).
#include "k_cols.cuh"

namespace fftenkf {

size_t col_stats_smem(int ny, int nf, int* lpc) {
  const int V = default_V(ny);
  const int T = ny / V;
  const size_t per = ((size_t)nf * ny + 2 * (size_t)padded_len(ny)) * sizeof(float);
  int want = 256 / T;
  if (want < 1) want = 1;
  const size_t cap = 200 * 1024;
  int n = want;
  while (n > 1 && n * per > cap) n >>= 1;
  if (n * per > 227 * 1024) return 0;
  if (lpc) *lpc = n;
  return n * per;
}

cudaError_t launch_col_stats(const ColStatsParams& p, cudaStream_t s) {
  if (p.n_obs <= 1) return col_stats_nobs1(p, s);
  if (p.n_obs <= 2) return col_stats_nobs2(p, s);
  return col_stats_nobs4(p, s);
}

cudaError_t launch_col_update(const ColUpdParams& p, cudaStream_t s) {
  if (p.n_obs <= 1) return col_update_nobs1(p, s);
  if (p.n_obs <= 2) return col_update_nobs2(p, s);
  return col_update_nobs4(p, s);
}

bool line_supported(int n) {
  switch (n) {
#define CASE(m) case m: return true;
    FFTENKF_COL_SIZES(CASE)
#undef CASE
    default: return false;
  }
}

}  // namespace fftenkf
