// Learned spectral-variance denoiser: radial binning of log chat, a small MLP
// (256 -> 64 -> 64 -> 64 -> 128, exact GELU, BF16 weights, FP32 accumulation)
// with its backward pass and Adam update, and unbinning back to a
// per-wavenumber spectrum.  Parameters are one flat FP32 vector
// [W1 (64x256, out-major), b1, W2, b2, W3, b3, W4 (128x64), b4]; the forward
// and backward passes use their BF16 rounding (gradients are those of the
// BF16 network and are applied to the FP32 master copy).
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace fftenkf {

constexpr int kBins = 128;
constexpr int kIn = 256, kH = 64, kOut = 128;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH, kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kOut * kH,
              kParams = kOffB4 + kOut;
constexpr int kActs = kIn + 3 * kH + kOut;   // per sample: x | z1 | z2 | z3 | out
constexpr int SB = 8;                        // samples per CTA

// ----------------------------------------------------------------- binning
// chat: [B][ny][L+1] f64 (one real table per sample); feat: [B][256] f32; mean: [B] f32.
// The bins are fixed per grid (FP64 decision, made on the host): bin_order lists the K1
// half-spectrum entries grouped by bin (ascending), bin_start[129] their offsets.  Each bin is
// cut into segments of at most kSegLen entries (seg_off[nseg+1], bin_seg[129] the segments of
// every bin), so that one spectrum spreads over many CTAs:
//   1. mlp_max_kernel: cmax per sample (atomicMax on the bit patterns of non-negative floats,
//      exact and independent of the order);
//   2. mlp_binsum_kernel: one CTA per (segment, sample) sums log(max(c / cmax, 1e-30));
//   3. mlp_binfin_kernel: per bin the segment sums in segment order, mean log + log cmax,
//      the features.
// log(max(c, 1e-30 cmax)) is evaluated as log(max(c/cmax, 1e-30)) + log(cmax) so that the floor
// never underflows; one conversion to float per entry.  No floating-point atomics: the result
// does not depend on the schedule.
constexpr int kSegLen = 2048;

__device__ __forceinline__ float block_sum256(float v, float* red8) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red8[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red8[w];
  return t;   // valid in thread 0
}

// cmax_bits[B] zeroed by the caller; grid (chunks, B)
__global__ void __launch_bounds__(256) mlp_max_kernel(const double* __restrict__ chat, int K1,
                                                      unsigned* __restrict__ cmax_bits) {
  __shared__ float red8[8];
  const double* c = chat + (size_t)blockIdx.y * K1;
  float mx = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K1; i += gridDim.x * blockDim.x) mx = fmaxf(mx, (float)c[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red8[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) m = fmaxf(m, red8[w]);
    if (!(m > 0.f)) m = 0.f;   // +0 (never -0 or NaN): bit patterns then order like the values
    atomicMax(cmax_bits + blockIdx.y, __float_as_uint(m));
  }
}

__device__ __forceinline__ float cmax_of(const unsigned* cmax_bits, int smp) {
  const float m = __uint_as_float(cmax_bits[smp]);
  return m > 0.f ? m : 1.f;
}

// grid (nseg, B): part[smp][seg] = sum over the segment of log(max(c / cmax, 1e-30))
__global__ void __launch_bounds__(256) mlp_binsum_kernel(const double* __restrict__ chat,
                                                         const uint32_t* __restrict__ bin_order,
                                                         const uint32_t* __restrict__ seg_off, int K1, int nseg,
                                                         const unsigned* __restrict__ cmax_bits,
                                                         float* __restrict__ part) {
  __shared__ float red8[8];
  const double* c = chat + (size_t)blockIdx.y * K1;
  const float inv = 1.f / cmax_of(cmax_bits, blockIdx.y);
  const uint32_t i0 = seg_off[blockIdx.x], i1 = seg_off[blockIdx.x + 1];
  float acc = 0.f;
  for (uint32_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc += logf(fmaxf((float)c[bin_order[i]] * inv, 1e-30f));
  const float t = block_sum256(acc, red8);
  if (threadIdx.x == 0) part[(size_t)blockIdx.y * nseg + blockIdx.x] = t;
}

// grid B, kBins threads: per-bin means, their mean mu, features [binned - mu | centre_log]
__global__ void __launch_bounds__(kBins) mlp_binfin_kernel(const float* __restrict__ part, int nseg,
                                                           const uint32_t* __restrict__ bin_seg,
                                                           const uint32_t* __restrict__ bin_start,
                                                           const unsigned* __restrict__ cmax_bits,
                                                           const float* __restrict__ centre_log,
                                                           float* __restrict__ feat, float* __restrict__ mean) {
  __shared__ float red4[kBins / 32];
  const int b = threadIdx.x, smp = blockIdx.x;
  const float lmax = logf(cmax_of(cmax_bits, smp));
  const float* ps = part + (size_t)smp * nseg;
  float acc = 0.f;
  for (uint32_t sg = bin_seg[b]; sg < bin_seg[b + 1]; ++sg) acc += ps[sg];
  const uint32_t n = bin_start[b + 1] - bin_start[b];
  const float v = n ? acc / (float)n + lmax : 0.f;
  float t = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((b & 31) == 0) red4[b >> 5] = t;
  __syncthreads();
  float tot = 0.f;
#pragma unroll
  for (int w = 0; w < kBins / 32; ++w) tot += red4[w];
  const float mu = tot / kBins;
  float* f = feat + (size_t)smp * kIn;
  f[b] = v - mu;
  f[kBins + b] = centre_log[b];
  if (b == 0) mean[smp] = mu;
}

// out_log: [128] learned binned log spectrum (mean already added); chat: [ny][L+1] f64
__global__ void mlp_unbin_kernel(const float* __restrict__ out_log, int ny, int L, float w,
                                 double* __restrict__ chat) {
  const int K1 = ny * (L + 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K1; i += gridDim.x * blockDim.x) {
    const int ky = i / (L + 1), kx = i - ky * (L + 1);
    const int kyv = (ky <= ny / 2) ? ky : ky - ny;
    const float kabs = sqrtf((float)(kyv * kyv + kx * kx));
    const float pos = kabs / w - 0.5f;   // position in units of bins relative to centre 0
    float v;
    if (pos <= 0.f) {
      v = out_log[0];
    } else if (pos >= kBins - 1) {
      v = out_log[kBins - 1];
    } else {
      const int b = (int)pos;
      const float fr = pos - b;
      v = out_log[b] + fr * (out_log[b + 1] - out_log[b]);
    }
    chat[i] = (double)expf(v);
  }
}

// out_log = out + mean (one sample); flag = 1 if any value is non-finite
__global__ void mlp_finish_kernel(const float* __restrict__ out, const float* __restrict__ mean, float* __restrict__ out_log,
                                  int* __restrict__ flag) {
  const int b = threadIdx.x;
  const float v = out[b] + mean[0];
  out_log[b] = v;
  const int bad = __syncthreads_or(!isfinite(v));
  if (b == 0) *flag = bad;
}

// chat_out = flag ? chat_in : chat_out (the plain estimate replaces a non-finite learned one)
__global__ void mlp_select_kernel(const double* __restrict__ chat_in, double* __restrict__ chat_out, int K1,
                                  const int* __restrict__ flag) {
  if (!*flag) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K1; i += gridDim.x * blockDim.x) chat_out[i] = chat_in[i];
}

// ----------------------------------------------------------------- MLP
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

struct MlpSmem {
  __nv_bfloat16 w[kOffB4 + kOut];   // whole parameter vector, BF16 (biases too, converted on use: unused)
  float bias[kH * 3 + kOut];
  float a[SB][kActs];
  float d[SB][kIn];                  // backward: deltas
};

__device__ void load_weights(MlpSmem& s, const float* __restrict__ params) {
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) s.w[i] = __float2bfloat16_rn(params[i]);
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    s.bias[i] = params[kOffB1 + i];
    s.bias[kH + i] = params[kOffB2 + i];
    s.bias[2 * kH + i] = params[kOffB3 + i];
  }
  for (int i = threadIdx.x; i < kOut; i += blockDim.x) s.bias[3 * kH + i] = params[kOffB4 + i];
}

// one dense layer for the CTA's samples: z[s][o] = b[o] + sum_i W[o][i] in[s][i]
__device__ void dense(const MlpSmem& s, int woff, const float* bias, int in_dim, int out_dim, int in_off, int out_off,
                      int nsamp, float (*a)[kActs]) {
  for (int idx = threadIdx.x; idx < nsamp * out_dim; idx += blockDim.x) {
    const int sm = idx / out_dim, o = idx - sm * out_dim;
    const __nv_bfloat16* wr = s.w + woff + o * in_dim;
    const float* x = a[sm] + in_off;
    float acc = bias[o];
    for (int i = 0; i < in_dim; i += 2) {
      const float2 wv = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(wr + i));
      acc = fmaf(wv.x, x[i], acc);
      acc = fmaf(wv.y, x[i + 1], acc);
    }
    a[sm][out_off + o] = acc;
  }
}

__device__ void forward_block(MlpSmem& s, int nsamp) {
  // a[s] = x | z1 | z2 | z3 | out ; hidden activations are gelu(z) computed on the fly
  float (*a)[kActs] = s.a;
  __shared__ float h[SB][kH];
  dense(s, kOffW1, s.bias, kIn, kH, 0, kIn, nsamp, a);
  __syncthreads();
  for (int idx = threadIdx.x; idx < nsamp * kH; idx += blockDim.x) h[idx / kH][idx % kH] = gelu(a[idx / kH][kIn + idx % kH]);
  __syncthreads();
  // layer 2 input is h: copy into d scratch as the dense() input row
  for (int idx = threadIdx.x; idx < nsamp * kH; idx += blockDim.x) s.d[idx / kH][idx % kH] = h[idx / kH][idx % kH];
  __syncthreads();
  for (int idx = threadIdx.x; idx < nsamp * kH; idx += blockDim.x) {
    const int sm = idx / kH, o = idx - sm * kH;
    const __nv_bfloat16* wr = s.w + kOffW2 + o * kH;
    float acc = s.bias[kH + o];
    for (int i = 0; i < kH; ++i) acc = fmaf(__bfloat162float(wr[i]), s.d[sm][i], acc);
    a[sm][kIn + kH + o] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nsamp * kH; idx += blockDim.x) s.d[idx / kH][idx % kH] = gelu(a[idx / kH][kIn + kH + idx % kH]);
  __syncthreads();
  for (int idx = threadIdx.x; idx < nsamp * kH; idx += blockDim.x) {
    const int sm = idx / kH, o = idx - sm * kH;
    const __nv_bfloat16* wr = s.w + kOffW3 + o * kH;
    float acc = s.bias[2 * kH + o];
    for (int i = 0; i < kH; ++i) acc = fmaf(__bfloat162float(wr[i]), s.d[sm][i], acc);
    a[sm][kIn + 2 * kH + o] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nsamp * kH; idx += blockDim.x) s.d[idx / kH][idx % kH] = gelu(a[idx / kH][kIn + 2 * kH + idx % kH]);
  __syncthreads();
  for (int idx = threadIdx.x; idx < nsamp * kOut; idx += blockDim.x) {
    const int sm = idx / kOut, o = idx - sm * kOut;
    const __nv_bfloat16* wr = s.w + kOffW4 + o * kH;
    float acc = s.bias[3 * kH + o];
    for (int i = 0; i < kH; ++i) acc = fmaf(__bfloat162float(wr[i]), s.d[sm][i], acc);
    a[sm][kIn + 3 * kH + o] = acc;
  }
  __syncthreads();
}

// X: [B][256]; out: [B][128]; acts (optional): [B][kActs]
__global__ void __launch_bounds__(256) mlp_fwd_kernel(const float* __restrict__ params, const float* __restrict__ X,
                                                      int B, float* __restrict__ out, float* __restrict__ acts) {
  extern __shared__ __align__(16) unsigned char raw[];
  MlpSmem& s = *reinterpret_cast<MlpSmem*>(raw);
  load_weights(s, params);
  const int s0 = blockIdx.x * SB;
  const int nsamp = min(SB, B - s0);
  for (int idx = threadIdx.x; idx < nsamp * kIn; idx += blockDim.x) s.a[idx / kIn][idx % kIn] = X[(size_t)s0 * kIn + idx];
  __syncthreads();
  forward_block(s, nsamp);
  for (int idx = threadIdx.x; idx < nsamp * kOut; idx += blockDim.x)
    out[(size_t)s0 * kOut + idx] = s.a[idx / kOut][kIn + 3 * kH + idx % kOut];
  if (acts)
    for (int idx = threadIdx.x; idx < nsamp * kActs; idx += blockDim.x)
      acts[(size_t)s0 * kActs + idx] = s.a[idx / kActs][idx % kActs];
}

// Gradient of mean((out - target)^2) over all B x 128 outputs: recomputes the
// forward pass of its samples, then back-propagates; weight gradients summed
// over the CTA's samples and added to grads with one atomic per parameter.
__global__ void __launch_bounds__(256) mlp_bwd_kernel(const float* __restrict__ params, const float* __restrict__ X,
                                                      const float* __restrict__ target, int B, float* __restrict__ grads,
                                                      float* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char raw[];
  MlpSmem& s = *reinterpret_cast<MlpSmem*>(raw);
  __shared__ float dcur[SB][kOut];
  __shared__ float hin[SB][kH];
  __shared__ float lsum[256];
  load_weights(s, params);
  const int s0 = blockIdx.x * SB;
  const int nsamp = min(SB, B - s0);
  for (int idx = threadIdx.x; idx < nsamp * kIn; idx += blockDim.x) s.a[idx / kIn][idx % kIn] = X[(size_t)s0 * kIn + idx];
  __syncthreads();
  forward_block(s, nsamp);
  // output delta and loss
  const float scale = 2.f / ((float)B * kOut);
  float l = 0.f;
  for (int idx = threadIdx.x; idx < nsamp * kOut; idx += blockDim.x) {
    const int sm = idx / kOut, o = idx - sm * kOut;
    const float diff = s.a[sm][kIn + 3 * kH + o] - target[(size_t)(s0 + sm) * kOut + o];
    l += diff * diff;
    dcur[sm][o] = scale * diff;
  }
  lsum[threadIdx.x] = l;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) lsum[threadIdx.x] += lsum[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, lsum[0] / ((float)B * kOut));
  // layers 4..1; input activation of layer l: gelu(z_{l-1}) (layer 1: x)
  int out_dim = kOut;
  for (int layer = 3; layer >= 0; --layer) {
    const int in_dim = (layer == 0) ? kIn : kH;
    const int woff = (layer == 0) ? kOffW1 : (layer == 1) ? kOffW2 : (layer == 2) ? kOffW3 : kOffW4;
    const int boff = (layer == 0) ? kOffB1 : (layer == 1) ? kOffB2 : (layer == 2) ? kOffB3 : kOffB4;
    const int zin = kIn + (layer - 1) * kH;   // z of the previous layer (layer >= 1)
    // input activations
    for (int idx = threadIdx.x; idx < nsamp * in_dim; idx += blockDim.x) {
      const int sm = idx / in_dim, i = idx - sm * in_dim;
      s.d[sm][i] = (layer == 0) ? s.a[sm][i] : gelu(s.a[sm][zin + i]);
    }
    __syncthreads();
    // weight and bias gradients
    for (int idx = threadIdx.x; idx < out_dim * in_dim; idx += blockDim.x) {
      const int o = idx / in_dim, i = idx - o * in_dim;
      float g = 0.f;
      for (int sm = 0; sm < nsamp; ++sm) g = fmaf(dcur[sm][o], s.d[sm][i], g);
      atomicAdd(grads + woff + idx, g);
    }
    for (int o = threadIdx.x; o < out_dim; o += blockDim.x) {
      float g = 0.f;
      for (int sm = 0; sm < nsamp; ++sm) g += dcur[sm][o];
      atomicAdd(grads + boff + o, g);
    }
    if (layer == 0) break;
    // delta of the previous layer
    for (int idx = threadIdx.x; idx < nsamp * in_dim; idx += blockDim.x) {
      const int sm = idx / in_dim, i = idx - sm * in_dim;
      float acc = 0.f;
      for (int o = 0; o < out_dim; ++o) acc = fmaf(__bfloat162float(s.w[woff + o * in_dim + i]), dcur[sm][o], acc);
      hin[sm][i] = acc * gelu_grad(s.a[sm][zin + i]);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nsamp * in_dim; idx += blockDim.x) dcur[idx / in_dim][idx % in_dim] = hin[idx / in_dim][idx % in_dim];
    __syncthreads();
    out_dim = in_dim;
  }
}

__global__ void mlp_adam_kernel(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                                float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ----------------------------------------------------------------- launchers
int mlp_param_count() { return kParams; }
int mlp_acts_per_sample() { return kActs; }

int mlp_seg_len() { return kSegLen; }

// Features of B spectra in slices of at most max_batch samples (the scratch: cmax_bits
// [max_batch], part [max_batch][nseg]).
cudaError_t launch_mlp_bin(const double* chat, const MlpBins& t, int B, float* feat, float* mean, cudaStream_t s) {
  const int chunks = std::max(1, std::min((t.K1 + 4095) / 4096, 1024));
  for (int b0 = 0; b0 < B; b0 += t.max_batch) {
    const int nb = std::min(t.max_batch, B - b0);
    const double* c = chat + (size_t)b0 * t.K1;
    cudaError_t e = cudaMemsetAsync(t.cmax_bits, 0, nb * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    mlp_max_kernel<<<dim3(chunks, nb), 256, 0, s>>>(c, t.K1, t.cmax_bits);
    mlp_binsum_kernel<<<dim3(t.nseg, nb), 256, 0, s>>>(c, t.order, t.seg_off, t.K1, t.nseg, t.cmax_bits, t.part);
    mlp_binfin_kernel<<<nb, kBins, 0, s>>>(t.part, t.nseg, t.bin_seg, t.start, t.cmax_bits, t.centre_log,
                                           feat + (size_t)b0 * kIn, mean + b0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_mlp_unbin(const float* out_log, int ny, int L, float w, double* chat, cudaStream_t s) {
  const int K1 = ny * (L + 1);
  int grid = (K1 + 255) / 256;
  if (grid > 4096) grid = 4096;
  mlp_unbin_kernel<<<grid, 256, 0, s>>>(out_log, ny, L, w, chat);
  return cudaGetLastError();
}

cudaError_t launch_mlp_finish(const float* out, const float* mean, float* out_log, int* flag, const double* chat_in,
                              double* chat_out, int K1, int ny, int L, float w, cudaStream_t s) {
  mlp_finish_kernel<<<1, kBins, 0, s>>>(out, mean, out_log, flag);
  cudaError_t e = launch_mlp_unbin(out_log, ny, L, w, chat_out, s);
  if (e != cudaSuccess) return e;
  int grid = (K1 + 255) / 256;
  if (grid > 4096) grid = 4096;
  mlp_select_kernel<<<grid, 256, 0, s>>>(chat_in, chat_out, K1, flag);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* params, const float* X, int B, float* out, float* acts, cudaStream_t s) {
  const size_t smem = sizeof(MlpSmem);
  cudaError_t e = cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  mlp_fwd_kernel<<<(B + SB - 1) / SB, 256, smem, s>>>(params, X, B, out, acts);
  return cudaGetLastError();
}

cudaError_t launch_mlp_gradient(const float* params, const float* X, const float* target, int B, float* grads,
                                float* loss, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(grads, 0, kParams * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), s);
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(MlpSmem);
  e = cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  mlp_bwd_kernel<<<(B + SB - 1) / SB, 256, smem, s>>>(params, X, target, B, grads, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* params, float* m, float* v, const float* g, int step, float lr, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  mlp_adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(params, m, v, g, kParams, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

}  // namespace fftenkf
