// Shared definitions of the analysis kernels: launch parameters, layouts and
// element access for the two storage types.
//
// Spectral intermediates ("row spectra") are stored per field as
// [nx/2][ny] float2: for every packed row-spectrum column c the ny values are
// contiguous, so the column passes read and write whole lines with unit
// stride.  Packed column 0 carries the real DC value of each row in .x and the
// real Nyquist value in .y (both are real for a real row).  The column passes
// treat k_x = 0 and k_x = nx/2 as "virtual columns" 0 and nx/2 that take the
// .x or the .y part of packed column 0, so every wavenumber column k_x in
// [0, nx/2] is one line of length ny.
#pragma once
#include <cuda.h>   // CUtensorMap (type only; maps are encoded through the runtime's driver entry point)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_core.cuh"

namespace fftenkf {

// (hi + lo) / n for an unevaluated sum hi + lo (an error-free accumulation) and an
// integer n: q = hi inv_n, corrected by the remainder hi - q n (exact with an FMA,
// since it is a small multiple of ulp(q)) plus lo.  The result is within one unit of
// the last place of the exact quotient and equals it whenever that quotient is a
// float (n equal members give their own value back).  inv_n = 1/n rounded.
__device__ __forceinline__ float pair_div(float hi, float lo, float n, float inv_n) {
  const float q = hi * inv_n;
  const float r = fmaf(-q, n, hi) + lo;
  return fmaf(r, inv_n, q);
}

constexpr int kMaxBlocks = 16;
constexpr int kMaxObs = 4;

// innovation rows d - u + e with given perturbations, or d - u when the perturbations are drawn in
// frequency space by the column update
enum RowMode { kAnomaly = 0, kInnovation = 1, kInnovationDrawn = 2 };
enum Storage { kF32 = 0, kBF16 = 1 };

// Status bits written by kernels (OR-ed into the plan's device word).
enum DeviceStatusBits { kStatusNonFinite = 1, kStatusTimeout = 2 };

__device__ __forceinline__ float2 load2(const void* base, size_t idx, int storage) {
  // two consecutive elements idx, idx+1 (idx even)
  if (storage == kBF16) {
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(
        reinterpret_cast<const __nv_bfloat16*>(base) + idx);
    return __bfloat1622float2(b);
  }
  return *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(base) + idx);
}

// the same with the storage type fixed at compile time
template <int ST>
__device__ __forceinline__ float2 load2(const void* base, size_t idx) {
  if constexpr (ST == kBF16) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(reinterpret_cast<const __nv_bfloat16*>(base) + idx));
  } else {
    return *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(base) + idx);
  }
}
template <int ST>
__device__ __forceinline__ void store2(void* base, size_t idx, float2 v) {
  if constexpr (ST == kBF16) {
    *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(base) + idx) = __float22bfloat162_rn(v);
  } else {
    *reinterpret_cast<float2*>(reinterpret_cast<float*>(base) + idx) = v;
  }
}

__device__ __forceinline__ void store2(void* base, size_t idx, float2 v, int storage) {
  if (storage == kBF16) {
    *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(base) + idx) =
        __float22bfloat162_rn(v);
  } else {
    *reinterpret_cast<float2*>(reinterpret_cast<float*>(base) + idx) = v;
  }
}

struct RowFwdParams {
  int ny, nx, L, R;       // L = nx/2, R rows per CTA
  int M, N, n_obs, mode, storage;
  int n_tiles;            // ny / R
  int obs[kMaxObs];
  const void* ens;        // [M][N][ny][nx]
  const float* data;      // [n_obs][ny][nx]     (innovation mode)
  const void* pert;       // [N][n_obs][ny][nx]  (innovation mode)
  float2* out;            // row spectra: anomaly field j*N+k, innovation field k*n_obs+i
  const float2* twL;      // exp(-2 pi i e / L), e < L
  const float2* twX;      // exp(-2 pi i k / nx), k <= L
  int* status;
  int vsel;               // line-FFT schedule (plan_V)
  int expire_first_wait;  // test setting: every CTA's first bulk-copy wait gives up at once
  // anomaly mode: 1/sqrt(N), and the tensor-memory columns of the running sums (set by the launcher)
  float inv_sqrt_N;
  int tm_cols, tm_alloc;  // per thread (a multiple of 8), per CTA (a power of two >= 32)
};

struct RowInvParams {
  int ny, nx, L, R, M, N, storage, n_tiles;
  int box_cols;           // columns per tensor copy of the increment spectra (divides L, at most 256)
  // row spectra of the increments, field j*N+k, [field][L][ny]; read through tm_in, the
  // float32 view {2 ny, L, fields} with box {2 R, box_cols, 1} (R rows of box_cols columns)
  alignas(64) CUtensorMap tm_in;
  void* ens;              // [M][N][ny][nx], updated in place
  const float2* twL;
  const float2* twX;
  int* status;
  int vsel;
};

struct ColStatsParams {
  int ny, L, M, N, n_obs, n_un;
  int obs[kMaxObs];
  int un[kMaxBlocks];
  const float2* A;        // anomaly row spectra, field j*N+k
  float* chat;            // [n_obs][L+1][ny] real, then [n_obs*n_un][L+1][ny] float2 (null: not written)
  float scale;            // 1 / ((N-1) * ny * nx)
  // gains in the epilogue (analysis): rhat transposed to [n_obs][L+1][ny]; null = no gains
  const double* rhat_t;
  float* goo;             // [n_obs][L+1][ny]
  float2* gjo;            // [n_obs*n_un][L+1][ny]
  float inv_G;            // 1 / (ny nx)
  const float2* twY;      // stage-major twiddles of the ny-point plan
  int* status;
  int vsel;
  // coupled observed blocks (n_obs <= 2, tables only: rhat_t null): the complex tables start
  // with n_pair = n_obs (n_obs - 1) / 2 observed-pair tables chat^(o1 o0)
  int n_pair;
};

// Gains with coupled observed blocks (n_obs <= 2) from the column statistics' tables, per
// wavenumber: K_r = chat_{r,O} (chat_OO + diag(rhat))^-1 for every block r in role order
// (observed, then unobserved), scaled by 1/(ny nx), into gall [role][n_obs][L+1][ny].
struct CoupledGainParams {
  int ny, L, n_obs, n_un, n_pair;
  const float* chat_t;    // [n_obs][L+1][ny] then complex [n_pair + n_obs n_un][L+1][ny]
  const double* rhat_t;   // [n_obs][L+1][ny]
  float2* gall;
  float inv_G;
  int* status;
};
cudaError_t launch_coupled_gain(const CoupledGainParams& p, cudaStream_t s);

struct ColUpdParams {
  int ny, L, M, N, n_obs, n_un;
  int obs_of_block[kMaxBlocks];   // observed index of block j, or -1
  int un_of_block[kMaxBlocks];    // unobserved index of block j, or -1
  const float2* W;        // innovation row spectra, field k*n_obs+i
  const float* goo;       // [n_obs][L+1][ny]
  const float2* gjo;      // [n_obs*n_un][L+1][ny], table i*n_un+u
  float2* S;              // increment row spectra, field j*N+k
  const float2* twY;
  int* status;
  int n_stages;           // innovation prefetch stages (set by the launcher)
  int vsel;
  int coupled;            // gains of every block j in gall [M][n_obs][L+1][ny] (complex)
  const float2* gall;
  // perturbations drawn here (seeded analysis): what_{k,o} += sqrt(ny nx) sqrt(rhat_o) zhat_{k,o},
  // zhat from Philox4x32-10 per (wavenumber, stream k n_obs + o) under key `seed`
  int drawn;
  unsigned long long seed;
  const double* rhat_t;   // [n_obs][L+1][ny]
  float sqrt_G;
};

// Fused column pass (statistics, gains and update of one wavenumber column per thread group,
// per-column tables in tensor memory): one or two observed blocks, not coupled.  Blocks are
// taken in "role" order, observed first, and transformed two at a time.
struct ColFusedParams {
  int ny, L, M, N, n_obs, n_un;
  int role_block[kMaxBlocks];   // block of role r (r < n_obs: the observed ones)
  const float2* A;        // anomaly row spectra, field j*N+k
  const float2* W;        // innovation row spectra, field k*n_obs+i; null: statistics only
  float2* S;              // increment row spectra, field j*N+k (may alias A)
  const double* rhat_t;   // [n_obs][L+1][ny] (analysis)
  float* chat;            // statistics only: tables in the col_stats layout
  const float4* tw;       // paired compact stage twiddles of the ny-point plan
  float scale;            // 1 / ((N-1) ny nx)
  float inv_G;            // 1 / (ny nx)
  int* status;
  int vsel;               // line-FFT schedule: 0 = wide (V = 16), 1 = narrow (V = 8, twice the threads)
  // perturbations drawn here (seeded analysis; the innovation rows are then d - u): what_{k,i} +=
  // amp_i zhat_{k,i}, zhat from Philox4x32-10 under `seed` (stream k n_obs + i), amp = sqrt(ny nx rhat)
  int drawn;
  unsigned long long seed;
  const float* amp_t;     // [n_obs][L+1][ny]
};
// launch of the fused column pass; cudaErrorNotSupported when the shape is not covered
cudaError_t launch_col_fused(const ColFusedParams& p, cudaStream_t s);
// whether the fused column pass covers (ny, n_obs, blocks) with schedule sel
bool col_fused_supported(int ny, int n_obs, int M, int sel);

struct GainParams {
  int ny, L, n_obs, n_un;
  const float* chat_t;    // stats kernel output (transposed, float), or null
  const double* spec;     // caller spectrum (natural layout, double), or null
  const double* rhat;     // [n_obs][ny][L+1]
  float* goo;
  float2* gjo;
  float scale;            // 1 / (ny*nx): folds the unnormalised inverse transform
  int* status;
};

// host-side launchers (one switch over the line length per pass)
cudaError_t launch_row_fwd(const RowFwdParams& p, int n_fields, cudaStream_t s);
cudaError_t launch_row_inv(const RowInvParams& p, int n_fields, cudaStream_t s);
// rows per item of the inverse row pass for (nx/2, schedule, ny, nx, storage bytes); 0 = unsupported
int row_inv_rows(int L, int vsel, int ny, int nx, int es);
// tensor map of the increment row spectra [fields][L][ny] for the inverse row pass's tile
// loads (R rows x box_cols columns per copy); false if R < 2 or cuTensorMapEncodeTiled rejects it
bool encode_increment_map(CUtensorMap* out, const float2* S, int fields, int ny, int L, int R, int box_cols);
cudaError_t launch_col_stats(const ColStatsParams& p, cudaStream_t s);
cudaError_t launch_col_update(const ColUpdParams& p, cudaStream_t s);
cudaError_t launch_gain(const GainParams& p, cudaStream_t s);
// output order of the complex spectrum tables: complex output q comes from complex
// column-pass table src[q], conjugated where conj[q] is set
struct ChatOutMap {
  int n_auto, n_cplx;
  int src[64];
  int conj[64];
};
ChatOutMap chat_out_map(int n_obs, int n_un, int coupled, const int* obs, const int* un, int M);
cudaError_t launch_chat_out(const float* chat_t, double* out, int ny, int L, const ChatOutMap& map,
                            cudaStream_t s);
// rhat [n][ny][L+1] -> rhat_t [n][L+1][ny]; with amp also amp [n][L+1][ny] = sqrt_G sqrt(rhat) (FP32)
cudaError_t launch_rhat_transpose(const double* rhat, double* rhat_t, int n, int ny, int L, cudaStream_t s,
                                  float* amp = nullptr, float sqrt_G = 0.f);
bool line_supported(int n);       // column line lengths
bool row_line_supported(int n);   // row line lengths (nx/2)
// shared-memory bytes a pass needs (0 = unsupported), for plan-time checks
size_t col_stats_smem(int ny, int nf, int vsel, int* lpc);
size_t col_update_smem(int ny, int n_obs, int vsel, int* lpc, int* n_stages);

// Radial bins of the learned denoiser (device tables, built once per grid) and the scratch of
// its segmented binning.
struct MlpBins {
  int K1, nseg, max_batch;
  const uint32_t* order;     // [K1] entries grouped by bin
  const uint32_t* start;     // [129] bin offsets into order
  const uint32_t* seg_off;   // [nseg + 1] segment offsets into order (each within one bin)
  const uint32_t* bin_seg;   // [129] first segment of every bin
  const float* centre_log;   // [128]
  unsigned* cmax_bits;       // [max_batch] scratch
  float* part;               // [max_batch][nseg] scratch
};

}  // namespace fftenkf
