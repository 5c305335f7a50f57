// Gain tables of eq. (spectral-enkf) / eq. (spectral-multi-enkf), computed in
// FP64 per wavenumber, and the transpose of the covariance tables to the
// boundary's [k_y][k_x] layout.
//
//   G^(oo) = chat^(oo) / (chat^(oo) + rhat_o),  G^(jo) = chat^(jo) / (chat^(oo) + rhat_o)
//
// with G = 0 where the denominator is 0.  The tables are stored as float in
// the column passes' [k_x][k_y] layout with 1/(ny nx) folded in (the column
// and row passes use unnormalised transforms).  rhat and a caller-supplied
// spectrum arrive in [k_y][k_x] layout and are transposed through shared
// memory in 32 x 32 tiles so that every global access is coalesced.
#include "common.cuh"

namespace fftenkf {

constexpr int TB = 32;

// 1/x in FP64 for normal x > 0: the hardware's approximate reciprocal refined
// by two steps of the Newton-Raphson iteration for f(y) = 1/y - x
// (e <- 1 - x y, y <- y + y e), each of which doubles the correct bits.
// Subnormal or zero x are handled by the caller.
__device__ __forceinline__ double recip64(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// load a [ny][L+1] double tile (rows ky0.., cols c0..) into s[ky][c]
__device__ __forceinline__ void load_tile(double (*s)[TB + 1], const double* __restrict__ src, int ny, int L1,
                                          int ky0, int c0, int stride_elems, int comp) {
  for (int yy = threadIdx.y; yy < TB; yy += blockDim.y) {
    const int ky = ky0 + yy, c = c0 + threadIdx.x;
    s[yy][threadIdx.x] = (ky < ny && c < L1) ? src[((size_t)ky * L1 + c) * stride_elems + comp] : 0.0;
  }
}

__global__ void __launch_bounds__(256) gain_kernel(const GainParams p) {
  __shared__ double rs[TB][TB + 1];
  __shared__ double ca[TB][TB + 1];
  __shared__ double cre[TB][TB + 1];
  __shared__ double cim[TB][TB + 1];
  const int L1 = p.L + 1;
  const int c0 = blockIdx.x * TB, ky0 = blockIdx.y * TB, i = blockIdx.z;
  const size_t K = (size_t)p.ny * L1;   // doubles per real table (natural layout)
  const size_t tab = (size_t)L1 * p.ny;  // elements per transposed table
  load_tile(rs, p.rhat + i * K, p.ny, L1, ky0, c0, 1, 0);
  if (p.spec) load_tile(ca, p.spec + i * K, p.ny, L1, ky0, c0, 1, 0);
  __syncthreads();
  // thread (x -> ky offset, y -> column offset): coalesced along k_y on output
  const int ky = ky0 + threadIdx.x;
  double inv[TB / 8];
  bool bad = false;
#pragma unroll
  for (int q = 0; q < TB / 8; ++q) {
    const int cl = threadIdx.y + 8 * q;
    const int c = c0 + cl;
    inv[q] = 0.0;
    if (c < L1 && ky < p.ny) {
      const double a = p.spec ? ca[threadIdx.x][cl] : (double)p.chat_t[i * tab + (size_t)c * p.ny + ky];
      bad |= !isfinite(a);
      const double den = a + rs[threadIdx.x][cl];
      inv[q] = (den > 1e-300) ? recip64(den) : ((den != 0.0) ? 1.0 / den : 0.0);
      inv[q] *= (double)p.scale;
      p.goo[i * tab + (size_t)c * p.ny + ky] = (float)(a * inv[q]);
    }
  }
  const double* xspec = p.spec ? p.spec + (size_t)p.n_obs * K : nullptr;
  const float2* xchat = reinterpret_cast<const float2*>(p.chat_t + (size_t)p.n_obs * tab);
  for (int u = 0; u < p.n_un; ++u) {
    const int qt = i * p.n_un + u;
    if (p.spec) {
      __syncthreads();
      load_tile(cre, xspec + (size_t)qt * 2 * K, p.ny, L1, ky0, c0, 2, 0);
      load_tile(cim, xspec + (size_t)qt * 2 * K, p.ny, L1, ky0, c0, 2, 1);
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < TB / 8; ++q) {
      const int cl = threadIdx.y + 8 * q;
      const int c = c0 + cl;
      if (c < L1 && ky < p.ny) {
        double re, im;
        if (p.spec) {
          re = cre[threadIdx.x][cl];
          im = cim[threadIdx.x][cl];
        } else {
          const float2 v = xchat[qt * tab + (size_t)c * p.ny + ky];
          re = v.x;
          im = v.y;
        }
        bad |= !(isfinite(re) && isfinite(im));
        const double sc = inv[q];
        p.gjo[qt * tab + (size_t)c * p.ny + ky] = make_float2((float)(re * sc), (float)(im * sc));
      }
    }
  }
  if (bad) atomicOr(p.status, kStatusNonFinite);
}

cudaError_t launch_gain(const GainParams& p, cudaStream_t s) {
  dim3 grid((p.L + 1 + TB - 1) / TB, (p.ny + TB - 1) / TB, p.n_obs);
  gain_kernel<<<grid, dim3(TB, 8), 0, s>>>(p);
  return cudaGetLastError();
}

// chat_t (float, [table][L+1][ny]) -> out (double, natural [table][ny][L+1], crosses (re,im))
__global__ void __launch_bounds__(256) chat_out_kernel(const float* __restrict__ chat_t, double* __restrict__ out,
                                                       int ny, int L, int n_obs, int n_un) {
  __shared__ float2 tile[TB][TB + 1];
  const int L1 = L + 1;
  const int c0 = blockIdx.x * TB, ky0 = blockIdx.y * TB, q = blockIdx.z;
  const bool is_auto = q < n_obs;
  const size_t tab = (size_t)L1 * ny;
  const size_t K = (size_t)ny * L1;
  for (int cc = threadIdx.y; cc < TB; cc += blockDim.y) {
    const int c = c0 + cc, ky = ky0 + threadIdx.x;
    float2 v = make_float2(0.f, 0.f);
    if (c < L1 && ky < ny) {
      if (is_auto) {
        v.x = chat_t[q * tab + (size_t)c * ny + ky];
      } else {
        v = reinterpret_cast<const float2*>(chat_t + n_obs * tab)[(q - n_obs) * tab + (size_t)c * ny + ky];
      }
    }
    tile[cc][threadIdx.x] = v;
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < TB; yy += blockDim.y) {
    const int ky = ky0 + yy, c = c0 + threadIdx.x;
    if (ky < ny && c < L1) {
      const float2 v = tile[threadIdx.x][yy];
      if (is_auto) {
        out[q * K + (size_t)ky * L1 + c] = v.x;
      } else {
        double* o = out + n_obs * K + (size_t)(q - n_obs) * 2 * K + ((size_t)ky * L1 + c) * 2;
        o[0] = v.x;
        o[1] = v.y;
      }
    }
  }
}

cudaError_t launch_chat_out(const float* chat_t, double* out, int ny, int L, int n_obs, int n_un, cudaStream_t s) {
  dim3 grid((L + 1 + TB - 1) / TB, (ny + TB - 1) / TB, n_obs + n_obs * n_un);
  chat_out_kernel<<<grid, dim3(TB, 8), 0, s>>>(chat_t, out, ny, L, n_obs, n_un);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) rhat_transpose_kernel(const double* __restrict__ in, double* __restrict__ out,
                                                             int ny, int L1) {
  __shared__ double tile[TB][TB + 1];
  const int c0 = blockIdx.x * TB, ky0 = blockIdx.y * TB;
  const size_t K = (size_t)ny * L1;
  const double* src = in + blockIdx.z * K;
  double* dst = out + blockIdx.z * K;
  for (int yy = threadIdx.y; yy < TB; yy += blockDim.y) {
    const int ky = ky0 + yy, c = c0 + threadIdx.x;
    tile[yy][threadIdx.x] = (ky < ny && c < L1) ? src[(size_t)ky * L1 + c] : 0.0;
  }
  __syncthreads();
  for (int cc = threadIdx.y; cc < TB; cc += blockDim.y) {
    const int c = c0 + cc, ky = ky0 + threadIdx.x;
    if (c < L1 && ky < ny) dst[(size_t)c * ny + ky] = tile[threadIdx.x][cc];
  }
}

cudaError_t launch_rhat_transpose(const double* rhat, double* rhat_t, int n, int ny, int L, cudaStream_t s) {
  dim3 grid((L + 1 + TB - 1) / TB, (ny + TB - 1) / TB, n);
  rhat_transpose_kernel<<<grid, dim3(TB, 8), 0, s>>>(rhat, rhat_t, ny, L + 1);
  return cudaGetLastError();
}

}  // namespace fftenkf
