// C ABI of the learned spectral-variance denoiser.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/fftenkf.h"
#include "common.cuh"

namespace fftenkf {
void set_last_error(const std::string& msg);
int mlp_param_count();
int mlp_seg_len();
cudaError_t launch_mlp_bin(const double* chat, const MlpBins& t, int B, float* feat, float* mean, cudaStream_t s);
cudaError_t launch_mlp_finish(const float* out, const float* mean, float* out_log, int* flag, const double* chat_in,
                              double* chat_out, int K1, int ny, int L, float w, cudaStream_t s);
cudaError_t launch_mlp_forward(const float* params, const float* X, int B, float* out, float* acts, cudaStream_t s);
cudaError_t launch_mlp_gradient(const float* params, const float* X, const float* target, int B, float* grads,
                                float* loss, cudaStream_t s);
cudaError_t launch_mlp_adam(float* params, float* m, float* v, const float* g, int step, float lr, cudaStream_t s);
}  // namespace fftenkf

using namespace fftenkf;

namespace {
fftenkf_status mfail(fftenkf_status s, const std::string& m) {
  set_last_error(m);
  return s;
}
fftenkf_status mcuda(cudaError_t e, const char* where) {
  return e == cudaSuccess ? FFTENKF_OK : mfail(FFTENKF_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
constexpr int kNB = 128;
constexpr int kMaxBatch = 64;   // spectra binned per slice of a batch
}  // namespace

struct fftenkf_denoiser_s {
  int ny, nx, L, K1, trained_members;
  float w;                 // bin width in |k| units
  uint32_t* d_order = nullptr;   // entries grouped by radial bin
  uint32_t* d_start = nullptr;   // [129] offsets of the bins in d_order
  uint32_t* d_seg = nullptr;     // segment offsets [nseg + 1] | first segment of every bin [129]
  int nseg = 0;
  float* d_centre_log = nullptr;
  float* d_scratch = nullptr;   // features 256 | mean 1 | out 128 | out_log 128
  unsigned* d_cmax = nullptr;   // [kMaxBatch]
  float* d_part = nullptr;      // [kMaxBatch][nseg]
  int* d_flag = nullptr;
  MlpBins bins() const {
    return MlpBins{K1, nseg, kMaxBatch, d_order, d_start, d_seg, d_seg + nseg + 1, d_centre_log, d_cmax, d_part};
  }
};

extern "C" int fftenkf_mlp_param_count(void) { return mlp_param_count(); }

extern "C" fftenkf_status fftenkf_denoiser_create(fftenkf_denoiser* out, int ny, int nx, int trained_members) {
  set_last_error("");
  if (!out || ny <= 0 || nx <= 0 || nx % 2 || trained_members < 2) return mfail(FFTENKF_EINVAL, "bad arguments");
  *out = nullptr;
  fftenkf_denoiser d = new fftenkf_denoiser_s();
  d->ny = ny;
  d->nx = nx;
  d->L = nx / 2;
  d->K1 = ny * (d->L + 1);
  d->trained_members = trained_members;
  // radial bins decided in FP64: b = min(127, floor(|k| / w)), w = sqrt(ny^2 + nx^2) / 2 / 128
  const double w = std::sqrt((double)ny * ny + (double)nx * nx) / 2.0 / kNB;
  d->w = (float)w;
  std::vector<int> bins(d->K1);
  std::vector<uint32_t> start(kNB + 1, 0);
  for (int ky = 0; ky < ny; ++ky) {
    const double kyv = (ky <= ny / 2) ? ky : ky - ny;
    for (int kx = 0; kx <= d->L; ++kx) {
      const double kabs = std::sqrt(kyv * kyv + (double)kx * kx);
      const double b = std::floor(kabs / w);
      const int bi = (int)(b > kNB - 1 ? kNB - 1 : b);
      bins[ky * (d->L + 1) + kx] = bi;
      start[bi + 1] += 1;
    }
  }
  for (int b = 0; b < kNB; ++b) start[b + 1] += start[b];
  std::vector<uint32_t> order(d->K1), fill(start.begin(), start.end() - 1);
  for (int i = 0; i < d->K1; ++i) order[fill[bins[i]]++] = (uint32_t)i;
  // every bin cut into segments of at most mlp_seg_len() entries
  std::vector<uint32_t> seg(1, 0), bin_seg(kNB + 1, 0);
  const uint32_t sl = (uint32_t)mlp_seg_len();
  for (int b = 0; b < kNB; ++b) {
    bin_seg[b] = (uint32_t)(seg.size() - 1);
    for (uint32_t x = start[b]; x < start[b + 1]; x += sl) seg.push_back(std::min(x + sl, start[b + 1]));
  }
  bin_seg[kNB] = (uint32_t)(seg.size() - 1);
  d->nseg = (int)(seg.size() - 1);
  seg.insert(seg.end(), bin_seg.begin(), bin_seg.end());
  std::vector<float> cl(kNB);
  for (int b = 0; b < kNB; ++b) {
    const double c = (b + 0.5) * w;
    cl[b] = (float)std::log(c > 0.5 ? c : 0.5);
  }
  cudaError_t e = cudaMalloc(&d->d_order, d->K1 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemcpy(d->d_order, order.data(), d->K1 * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&d->d_start, (kNB + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemcpy(d->d_start, start.data(), (kNB + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&d->d_seg, seg.size() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemcpy(d->d_seg, seg.data(), seg.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&d->d_cmax, kMaxBatch * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&d->d_part, (size_t)kMaxBatch * std::max(d->nseg, 1) * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d->d_centre_log, kNB * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(d->d_centre_log, cl.data(), kNB * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&d->d_scratch, (256 + 4 + 2 * kNB) * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d->d_flag, sizeof(int));
  if (e != cudaSuccess) {
    fftenkf_denoiser_destroy(d);
    return mfail(FFTENKF_ENOMEM, "denoiser allocation failed");
  }
  *out = d;
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_denoiser_destroy(fftenkf_denoiser d) {
  if (!d) return FFTENKF_OK;
  if (d->d_order) cudaFree(d->d_order);
  if (d->d_start) cudaFree(d->d_start);
  if (d->d_seg) cudaFree(d->d_seg);
  if (d->d_cmax) cudaFree(d->d_cmax);
  if (d->d_part) cudaFree(d->d_part);
  if (d->d_centre_log) cudaFree(d->d_centre_log);
  if (d->d_scratch) cudaFree(d->d_scratch);
  if (d->d_flag) cudaFree(d->d_flag);
  delete d;
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_denoiser_features(fftenkf_denoiser d, const double* chat, int batch, float* features,
                                                    float* means, void* stream) {
  set_last_error("");
  if (!d || !chat || !features || !means || batch <= 0) return mfail(FFTENKF_EINVAL, "bad arguments");
  return mcuda(launch_mlp_bin(chat, d->bins(), batch, features, means, static_cast<cudaStream_t>(stream)),
               "denoiser_features");
}

extern "C" fftenkf_status fftenkf_mlp_forward(const float* params, const float* features, int batch, float* out,
                                              void* stream) {
  set_last_error("");
  if (!params || !features || !out || batch <= 0) return mfail(FFTENKF_EINVAL, "bad arguments");
  return mcuda(launch_mlp_forward(params, features, batch, out, nullptr, static_cast<cudaStream_t>(stream)),
               "mlp_forward");
}

extern "C" fftenkf_status fftenkf_mlp_gradient(const float* params, const float* features, const float* targets,
                                               int batch, float* grads, float* loss, void* stream) {
  set_last_error("");
  if (!params || !features || !targets || !grads || !loss || batch <= 0) return mfail(FFTENKF_EINVAL, "bad arguments");
  return mcuda(launch_mlp_gradient(params, features, targets, batch, grads, loss, static_cast<cudaStream_t>(stream)),
               "mlp_gradient");
}

extern "C" fftenkf_status fftenkf_mlp_adam(float* params, float* m, float* v, const float* grads, int step, float lr,
                                           void* stream) {
  set_last_error("");
  if (!params || !m || !v || !grads || step < 1 || !(lr > 0.f)) return mfail(FFTENKF_EINVAL, "bad arguments");
  return mcuda(launch_mlp_adam(params, m, v, grads, step, lr, static_cast<cudaStream_t>(stream)), "mlp_adam");
}

extern "C" fftenkf_status fftenkf_denoise_spectrum(fftenkf_denoiser d, const float* params, const double* chat_in,
                                                   double* chat_out, int n_members, int* used_fallback, void* stream) {
  set_last_error("");
  if (!d || !params || !chat_in || !chat_out) return mfail(FFTENKF_EINVAL, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_members != d->trained_members) {   // the network only knows the ensemble size it was trained for
    cudaError_t e = cudaMemcpyAsync(chat_out, chat_in, d->K1 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (used_fallback) *used_fallback = 1;
    return mcuda(e, "denoise_spectrum");
  }
  float* feat = d->d_scratch;
  float* mean = feat + 256;
  float* out = mean + 4;
  float* out_log = out + kNB;
  cudaError_t e = launch_mlp_bin(chat_in, d->bins(), 1, feat, mean, s);
  if (e == cudaSuccess) e = launch_mlp_forward(params, feat, 1, out, nullptr, s);
  if (e == cudaSuccess)
    e = launch_mlp_finish(out, mean, out_log, d->d_flag, chat_in, chat_out, d->K1, d->ny, d->L, d->w, s);
  if (e != cudaSuccess) return mcuda(e, "denoise_spectrum");
  if (used_fallback) {
    e = cudaMemcpyAsync(used_fallback, d->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return mcuda(e, "denoise_spectrum");
  }
  return FFTENKF_OK;
}
