// Batched analyses: many independent single-block, fully observed (H = I)
// FFT EnKF analyses of uneven grid and ensemble sizes, one persistent launch
// per pass over a work list that mixes units of every analysis.
//
// A work unit is (analysis, unit index); each persistent CTA walks the list
// with a static stride (the list is sorted by decreasing cost on the host) and
// dispatches on the unit's line length to the same templated line FFTs as the
// single-analysis passes.  Loads are plain coalesced loads: the batched sizes
// need little shared memory, so several CTAs per SM hide the latency.
#pragma once
#include "common.cuh"

namespace fftenkf {

struct BatchItem {
  int ny, nx, L, N;
  void* ens;                 // [N][ny][nx] storage dtype, updated in place
  const float* data;         // [ny][nx]
  const void* pert;          // [N][ny][nx]
  const double* rhat;        // [ny][nx/2+1]
  float* mean;               // workspace: [ny][nx]
  float2* A;                 // [N][L][ny] anomaly row spectra, then increments
  float2* W;                 // [N][L][ny] innovation row spectra
  float* chat;               // [L+1][ny]
  float* gain;               // [L+1][ny], 1/(ny nx) folded in
  const float2* twL;         // stage-major twiddles of the L-point plan (schedule of the pass)
  const float2* twY;
  const float2* twX;         // exp(-2 pi i k / nx)
  const float2* twL_alt;     // same for the other schedule
  const float2* twY_alt;
};

struct BatchUnit {
  int item, u;
};

struct BatchParams {
  const BatchItem* items;
  const BatchUnit* units;
  int n_units;
  int storage;
  int mode;                  // row_fwd: kAnomaly / kInnovation
  int vsel;                  // line-FFT schedule of this pass
  int* status;
};

// work units of one item in pass `pass` for CTAs of bt threads and schedule vsel,
// their relative cost (for ordering), and the shared memory a unit needs
int batch_units(int pass, const BatchItem& it, int bt, int vsel);
double batch_unit_cost(int pass, const BatchItem& it, int bt, int vsel);
size_t batch_smem(int pass, const BatchItem& it, int bt, int vsel);
bool batch_line_supported(int n);

enum BatchPass { kBMean, kBRowAnom, kBStats, kBGain, kBRowInnov, kBUpdate, kBRowInv, kBPassCount };
cudaError_t launch_batch_pass(int pass, const BatchParams& p, int bt, size_t smem, int grid, cudaStream_t s);

}  // namespace fftenkf
