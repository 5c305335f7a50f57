// Spectral covariance estimate without any device allocation: the same passes
// as fftenkf_estimate_spectrum for one block, with every scratch buffer
// (twiddle tables, status word, row spectra, covariance table)
// carved out of one file-scope __device__ array instead of a workspace.
//
// The array lives in the library's device image, so every GPU that loads the
// library holds kStaticScratchBytes of it until the process exits.  Host code
// cannot use the array's name as a device address; the address is obtained
// once per device with cudaGetSymbolAddress (with that device current) on the
// first call made on that device, and cached.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/fftenkf.h"
#include "common.cuh"

namespace fftenkf {
void set_last_error(const std::string& msg);
}  // namespace fftenkf

using namespace fftenkf;

namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;   // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

size_t rup(size_t x) { return (x + 255) / 256 * 256; }

// stage-major twiddles of the (N, V) line plan, computed on the device (see fft_core.cuh)
__global__ void stage_twiddles_kernel(float2* out, int N, int V) {
  const int count = twiddle_count(N, V);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const long long e = twiddle_exponent(N, V, i);
    double sn, cs;
    sincospi(2.0 * (double)e / (double)N, &sn, &cs);
    out[i] = make_float2((float)cs, (float)-sn);
  }
}

// exp(-2 pi i k / nx), k <= count - 1
__global__ void plain_twiddles_kernel(float2* out, int nx, int count) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)k / (double)nx, &sn, &cs);
    out[k] = make_float2((float)cs, (float)-sn);
  }
}

fftenkf_status sfail(fftenkf_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

// address of this device's copy of the array, set up on the first call on that device
fftenkf_status scratch_address(char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sfail(FFTENKF_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return sfail(FFTENKF_EUNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return sfail(FFTENKF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<char*>(g_scratch_ptr[dev]);
  return FFTENKF_OK;
}

}  // namespace

// the status word sits at offset 0 of the array (see the layout below)
extern "C" fftenkf_status fftenkf_static_last_device_status(void* stream) {
  set_last_error("");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sfail(FFTENKF_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return sfail(FFTENKF_EUNSUPPORTED, "device index out of range");
  e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return sfail(FFTENKF_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    base = static_cast<char*>(g_scratch_ptr[dev]);
  }
  if (!base) return FFTENKF_OK;   // no call on this device yet
  int word = 0;
  e = cudaMemcpy(&word, base, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(base, 0, sizeof(int));
  if (e != cudaSuccess) return sfail(FFTENKF_ECUDA, std::string("status word: ") + cudaGetErrorString(e));
  if (word & kStatusTimeout) return sfail(FFTENKF_ETIMEOUT, "a bounded wait for an asynchronous copy gave up");
  if (word & kStatusNonFinite) return sfail(FFTENKF_ENONFINITE, "non-finite spectral covariance");
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_estimate_spectrum_static(const void* ensemble, int ny, int nx, int n_members,
                                                           int storage, double* spectrum_out, void* stream) {
  set_last_error("");
  if (!ensemble || !spectrum_out) return sfail(FFTENKF_EINVAL, "null argument");
  if (((uintptr_t)ensemble | (uintptr_t)spectrum_out) % 16) return sfail(FFTENKF_EINVAL, "pointers must be 16-byte aligned");
  if (storage != FFTENKF_F32 && storage != FFTENKF_BF16) return sfail(FFTENKF_EINVAL, "unknown storage");
  if (n_members < 2) return sfail(FFTENKF_EUNSUPPORTED, "need at least 2 members (the covariance divides by N-1)");
  if (nx % 2 || nx < 16 || nx > 8192 || !row_line_supported(nx / 2) || ny < 16 || ny > 4096 || !line_supported(ny))
    return sfail(FFTENKF_EUNSUPPORTED, "ny, nx must be 2^a or 3*2^a (16 <= nx <= 8192, 16 <= ny <= 4096)");
  if (col_stats_smem(ny, 1, 0, nullptr) == 0) return sfail(FFTENKF_EUNSUPPORTED, "column statistics do not fit in shared memory");
  const int L = nx / 2;
  const int Vl = plan_V(L, 0), Vy = plan_V(ny, 0);
  const size_t K1 = (size_t)ny * (L + 1);
  size_t off = 0;
  const size_t off_status = off;  off = rup(off + sizeof(int));
  const size_t off_twL = off;     off = rup(off + (size_t)twiddle_count(L, Vl) * sizeof(float2));
  const size_t off_twY = off;     off = rup(off + (size_t)twiddle_count(ny, Vy) * sizeof(float2));
  const size_t off_twX = off;     off = rup(off + (size_t)(L + 1) * sizeof(float2));
  const size_t off_A = off;       off = rup(off + (size_t)n_members * L * ny * sizeof(float2));
  const size_t off_chat = off;    off = rup(off + K1 * sizeof(float));
  if (off > kStaticScratchBytes)
    return sfail(FFTENKF_EUNSUPPORTED, "needs " + std::to_string(off) + " bytes of scratch; the static array holds " +
                                           std::to_string(kStaticScratchBytes) + " (64 MiB)");
  char* base = nullptr;
  fftenkf_status st = scratch_address(&base);
  if (st != FFTENKF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* status = reinterpret_cast<int*>(base + off_status);
  float2* twL = reinterpret_cast<float2*>(base + off_twL);
  float2* twY = reinterpret_cast<float2*>(base + off_twY);
  float2* twX = reinterpret_cast<float2*>(base + off_twX);
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);   // the array keeps the previous call's contents
  if (e == cudaSuccess) {
    stage_twiddles_kernel<<<64, 256, 0, s>>>(twL, L, Vl);
    stage_twiddles_kernel<<<64, 256, 0, s>>>(twY, ny, Vy);
    plain_twiddles_kernel<<<16, 256, 0, s>>>(twX, nx, L + 1);
    e = cudaGetLastError();
  }
  RowFwdParams rp;
  memset(&rp, 0, sizeof(rp));
  rp.ny = ny; rp.nx = nx; rp.L = L; rp.M = 1; rp.N = n_members; rp.n_obs = 1; rp.mode = kAnomaly;
  rp.storage = storage; rp.ens = ensemble;
  rp.out = reinterpret_cast<float2*>(base + off_A);
  rp.twL = twL; rp.twX = twX; rp.status = status; rp.vsel = 0;
  if (e == cudaSuccess) e = launch_row_fwd(rp, n_members, s);
  ColStatsParams cp;
  memset(&cp, 0, sizeof(cp));
  cp.ny = ny; cp.L = L; cp.M = 1; cp.N = n_members; cp.n_obs = 1; cp.n_un = 0; cp.obs[0] = 0;
  cp.A = rp.out;
  cp.chat = reinterpret_cast<float*>(base + off_chat);
  cp.scale = (float)(1.0 / ((double)(n_members - 1) * (double)ny * (double)nx));
  cp.twY = twY; cp.status = status; cp.vsel = 0;
  if (e == cudaSuccess) e = launch_col_stats(cp, s);
  const int block0 = 0;
  if (e == cudaSuccess) e = launch_chat_out(cp.chat, spectrum_out, ny, L, chat_out_map(1, 0, 0, &block0, nullptr, 1), s);
  if (e != cudaSuccess) return sfail(FFTENKF_ECUDA, std::string("estimate_spectrum_static: ") + cudaGetErrorString(e));
  return FFTENKF_OK;
}
