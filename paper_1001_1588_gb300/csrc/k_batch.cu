// Host side of the batched passes: unit counts, costs and shared memory per
// (pass, item, CTA size, schedule), and the launch switch.
#include <cmath>

#include "k_batch.cuh"

namespace fftenkf {

cudaError_t launch_batch_rows(int pass, const BatchParams& p, int bt, size_t smem, int grid, cudaStream_t s);
cudaError_t launch_batch_cols(int pass, const BatchParams& p, int bt, size_t smem, int grid, cudaStream_t s);

bool batch_line_supported(int n) {
  switch (n) {
#define CASE(m) case m: return true;
    FFTENKF_BATCH_SIZES(CASE)
#undef CASE
    default: return false;
  }
}

static int lines_per_cta(int n, int bt, int vsel) {
  const int T = n / plan_V(n, vsel);
  return T >= bt ? 1 : bt / T;
}

int batch_units(int pass, const BatchItem& it, int bt, int vsel) {
  const long long G = (long long)it.ny * it.nx;
  switch (pass) {
    case kBMean: return (int)((G + 8LL * bt - 1) / (8LL * bt));
    case kBRowAnom:
    case kBRowInnov:
    case kBRowInv: {
      const int R = batch_rows_per_tile(it.ny, lines_per_cta(it.L, bt, vsel));
      return it.N * (it.ny / R);
    }
    case kBStats: {
      const int lpc = lines_per_cta(it.ny, bt, vsel);
      return (it.L + 1 + lpc - 1) / lpc;
    }
    case kBGain: return ((it.L + 1 + 31) / 32) * ((it.ny + 31) / 32);
    case kBUpdate: {
      const int lpc = lines_per_cta(it.ny, bt, vsel);
      return (int)(((long long)(it.L + 1) * it.N + lpc - 1) / lpc);
    }
  }
  return 0;
}

double batch_unit_cost(int pass, const BatchItem& it, int bt, int vsel) {
  const double lx = std::log2((double)it.L), ly = std::log2((double)it.ny);
  switch (pass) {
    case kBMean: return 8.0 * bt * it.N;
    case kBRowAnom:
    case kBRowInnov:
    case kBRowInv: {
      const int R = batch_rows_per_tile(it.ny, lines_per_cta(it.L, bt, vsel));
      return (double)R * it.L * (lx + 2.0);
    }
    case kBStats: return (double)lines_per_cta(it.ny, bt, vsel) * it.N * it.ny * (ly + 1.0);
    case kBGain: return 1024.0;
    case kBUpdate: return (double)lines_per_cta(it.ny, bt, vsel) * it.ny * (2.0 * ly + 1.0);
  }
  return 0.0;
}

size_t batch_smem(int pass, const BatchItem& it, int bt, int vsel) {
  switch (pass) {
    case kBRowAnom:
    case kBRowInnov:
    case kBRowInv: {
      const int R = batch_rows_per_tile(it.ny, lines_per_cta(it.L, bt, vsel));
      return (size_t)(R + 1) * row_pitch(it.L) * sizeof(float2);
    }
    case kBStats:
    case kBUpdate: {
      const int PL = (padded_len(it.ny) + 1) & ~1;
      return (size_t)lines_per_cta(it.ny, bt, vsel) * PL * sizeof(float2);
    }
  }
  return 0;
}

cudaError_t launch_batch_pass(int pass, const BatchParams& p, int bt, size_t smem, int grid, cudaStream_t s) {
  if (p.n_units == 0) return cudaSuccess;
  if (pass == kBMean || pass == kBRowAnom || pass == kBRowInnov || pass == kBRowInv)
    return launch_batch_rows(pass, p, bt, smem, grid, s);
  return launch_batch_cols(pass, p, bt, smem, grid, s);
}

}  // namespace fftenkf
