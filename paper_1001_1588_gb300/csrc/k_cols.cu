// Column-pass launchers: shared-memory sizing and dispatch on the number of
// observed blocks (one translation unit per instantiation, compiled in parallel).
#include <cudaTypedefs.h>

#include <mutex>

#include "k_cols.cuh"
#include "k_colf.cuh"

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

// S [fields][L][ny] viewed as float32 {2 ny, L, fields}; a box is R consecutive k_y of
// box_cols consecutive columns of one field, landing in shared memory as [box_cols][R]
bool encode_increment_map(CUtensorMap* out, const float2* S, int fields, int ny, int L, int R, int box_cols) {
  if (R < 2 || box_cols < 1 || box_cols > 256 || L % box_cols) return false;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!encode) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * ny, (cuuint64_t)L, (cuuint64_t)fields};
  const cuuint64_t strides[2] = {(cuuint64_t)ny * sizeof(float2), (cuuint64_t)L * ny * sizeof(float2)};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * R), (cuuint32_t)box_cols, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  return encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(S), dims, strides, box, estride,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
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
    const size_t per = (nst + 1) * lines + (size_t)col_line_slots(ny) * sizeof(float2);
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

bool col_fused_supported(int ny, int n_obs, int M, int sel) {
  switch (ny) {
#define CASE(n) case n:
    FFTENKF_FUSED_SIZES(CASE)
#undef CASE
      break;
    default:
      return false;
  }
  if (n_obs < 1 || n_obs > 2 || M < n_obs) return false;
  const ColFusedLaunch s = col_fused_launch(ny, sel);
  if (s.lpc < 1) return false;
  const int nf = n_obs * (1 + 2 * (M - n_obs));   // sums / gains per wavenumber
  return (nf + 4) * s.V <= s.cols_per_thread;     // + the member's spectra (two complex halves)
}

cudaError_t launch_col_fused(const ColFusedParams& p, cudaStream_t s) {
  if (!col_fused_supported(p.ny, p.n_obs, p.M, p.vsel)) return cudaErrorNotSupported;
  return p.n_obs == 1 ? col_fused_nobs1(p, s) : col_fused_nobs2(p, s);
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
