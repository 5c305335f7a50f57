// Column-pass launchers: shared-memory sizing and dispatch on the number of
// observed blocks (one translation unit per instantiation, compiled in parallel).
#include "k_cols.cuh"

namespace fftenkf {

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

static size_t padded_bytes(int ny) { return (size_t)((padded_len(ny) + 1) & ~1) * sizeof(float2); }

// per group: accumulators nf*ny floats, exchange line, one prefetch line
size_t col_stats_smem(int ny, int nf, int vsel, int* lpc) {
  const int V = plan_V(ny, vsel);
  const int T = ny / V;
  const size_t per = (size_t)nf * ny * sizeof(float) + padded_bytes(ny) + (size_t)ny * sizeof(float2);
  int n = 256 / T;
  if (n < 1) n = 1;
  while (n > 1 && n * per + 16 > 200 * 1024) n >>= 1;
  if (n * per + 16 > 227 * 1024) return 0;
  if (lpc) *lpc = n;
  return n * per + 16;
}

// per group: one or two stages of n_obs innovation lines, one stage of gain lines, exchange line
size_t col_update_smem(int ny, int n_obs, int vsel, int* lpc, int* n_stages) {
  const int V = plan_V(ny, vsel);
  const int T = ny / V;
  const size_t lines = (size_t)n_obs * ny * sizeof(float2);
  for (int nst = 2; nst >= 1; --nst) {
    const size_t per = (nst + 1) * lines + padded_bytes(ny);
    int n = 256 / T;
    if (n < 1) n = 1;
    while (n > 1 && n * per + 32 > 200 * 1024) n >>= 1;
    if (n * per + 32 <= 227 * 1024) {
      if (lpc) *lpc = n;
      if (n_stages) *n_stages = nst;
      return n * per + 32;
    }
  }
  return 0;
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
