// Column passes: the second half of each 2-D transform, fused with the
// per-wavenumber work of Sec. 2.1.
//
// col_stats (steps 1-2, eq. dii and eq. cov-multi-spectral): a thread group
// owns one wavenumber column k_x and loops over the members; for each member
// it transforms the column of every block's anomaly row spectrum and
// accumulates |ahat^(o)|^2 for observed o and ahat^(j) conj(ahat^(o)) for
// unobserved j in shared memory (each thread only touches the k_y it owns, so
// the accumulation needs no synchronisation).  Member spectra never leave the
// chip; only the covariance tables are written.
//
// col_update (eq. spectral-multi-enkf): a thread group owns (k_x, member k):
// it transforms the innovation columns of every observed block, multiplies by
// the gain tables, sums over observed blocks, applies the inverse column
// transform for every target block and writes the increment's row spectra.
#pragma once
#include "common.cuh"

namespace fftenkf {

template <int NY, int V>
__device__ __forceinline__ void load_col(float2 (&v)[V], const float2* __restrict__ src, int t, int part,
                                         bool active) {
  constexpr int T = NY / V;
#pragma unroll
  for (int m = 0; m < V; ++m) {
    float2 a = active ? src[t + T * m] : make_float2(0.f, 0.f);
    if (part == 1) a = make_float2(a.x, 0.f);
    if (part == 2) a = make_float2(a.y, 0.f);
    v[m] = a;
  }
}

template <int NY, int V, int NOBS>
__global__ void __launch_bounds__(256) col_stats_kernel(const ColStatsParams p) {
  constexpr int T = NY / V;
  extern __shared__ float smf[];
  const int LPC = blockDim.x / T;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int c = blockIdx.x * LPC + g;            // wavenumber column k_x in [0, L]
  const bool active = c <= p.L;
  const int nf = p.n_obs + 2 * p.n_obs * p.n_un;
  float* acc = smf + (size_t)g * ((size_t)nf * NY + 2 * padded_len(NY));
  float2* xacc = reinterpret_cast<float2*>(acc + p.n_obs * NY);
  float2* line = reinterpret_cast<float2*>(acc + (size_t)nf * NY);
  for (int s = t; s < nf * NY; s += T) acc[s] = 0.f;
  const int col = (c == p.L) ? 0 : c;
  const int part = (c == 0) ? 1 : ((c == p.L) ? 2 : 0);
  const size_t fstride = (size_t)p.L * NY;
  for (int k = 0; k < p.N; ++k) {
    float2 ko[NOBS][V];
#pragma unroll
    for (int i = 0; i < NOBS; ++i) {
      if (i < p.n_obs) {
        float2 v[V];
        load_col<NY, V>(v, p.A + ((size_t)p.obs[i] * p.N + k) * fstride + (size_t)col * NY, t, part, active);
        fft_line<NY, V, false>(v, line, t, p.twY);
#pragma unroll
        for (int m = 0; m < V; ++m) {
          ko[i][m] = v[m];
          acc[i * NY + t + T * m] += v[m].x * v[m].x + v[m].y * v[m].y;
        }
      }
    }
    for (int u = 0; u < p.n_un; ++u) {
      float2 v[V];
      load_col<NY, V>(v, p.A + ((size_t)p.un[u] * p.N + k) * fstride + (size_t)col * NY, t, part, active);
      fft_line<NY, V, false>(v, line, t, p.twY);
#pragma unroll
      for (int i = 0; i < NOBS; ++i) {
        if (i < p.n_obs) {
          float2* a = xacc + (size_t)(i * p.n_un + u) * NY + t;
#pragma unroll
          for (int m = 0; m < V; ++m) {
            const float2 cr = cmulc(v[m], ko[i][m]);
            a[T * m].x += cr.x;
            a[T * m].y += cr.y;
          }
        }
      }
    }
  }
  if (!active) return;
  const size_t tab = (size_t)(p.L + 1) * NY;
  bool bad = false;
  for (int i = 0; i < p.n_obs; ++i) {
#pragma unroll
    for (int m = 0; m < V; ++m) {
      const int ky = t + T * m;
      const float val = acc[i * NY + ky] * p.scale;
      bad |= !isfinite(val);
      p.chat[i * tab + (size_t)c * NY + ky] = val;
    }
  }
  float2* xout = reinterpret_cast<float2*>(p.chat + p.n_obs * tab);
  for (int q = 0; q < p.n_obs * p.n_un; ++q) {
#pragma unroll
    for (int m = 0; m < V; ++m) {
      const int ky = t + T * m;
      const float2 a = xacc[(size_t)q * NY + ky];
      const float2 val = make_float2(a.x * p.scale, a.y * p.scale);
      bad |= !(isfinite(val.x) && isfinite(val.y));
      xout[q * tab + (size_t)c * NY + ky] = val;
    }
  }
  if (bad) atomicOr(p.status, kStatusNonFinite);
}

template <int NY, int V, int NOBS>
__global__ void __launch_bounds__(256) col_update_kernel(const ColUpdParams p) {
  constexpr int T = NY / V;
  extern __shared__ float2 sm2[];
  const int LPC = blockDim.x / T;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int item = blockIdx.x * LPC + g;
  const int c = item / p.N;
  const int k = item - c * p.N;
  const bool active = c <= p.L;
  float2* line = sm2 + (size_t)g * padded_len(NY);
  const int col = (c == p.L) ? 0 : c;
  const int part = (c == 0) ? 1 : ((c == p.L) ? 2 : 0);
  const size_t fstride = (size_t)p.L * NY;
  const size_t tab = (size_t)(p.L + 1) * NY;
  const size_t cc = active ? (size_t)c * NY : 0;
  float2 w[NOBS][V];
#pragma unroll
  for (int i = 0; i < NOBS; ++i) {
    if (i < p.n_obs) {
      float2 v[V];
      load_col<NY, V>(v, p.W + ((size_t)k * p.n_obs + i) * fstride + (size_t)col * NY, t, part, active);
      fft_line<NY, V, false>(v, line, t, p.twY);
#pragma unroll
      for (int m = 0; m < V; ++m) w[i][m] = v[m];
    }
  }
  for (int j = 0; j < p.M; ++j) {
    float2 s[V];
    const int io = p.obs_of_block[j];
#pragma unroll
    for (int m = 0; m < V; ++m) s[m] = make_float2(0.f, 0.f);
    if (io >= 0) {
      const float* gp = p.goo + io * tab + cc + t;
#pragma unroll
      for (int i = 0; i < NOBS; ++i) {
        if (i == io) {
#pragma unroll
          for (int m = 0; m < V; ++m) {
            const float gv = active ? __ldg(gp + T * m) : 0.f;
            s[m] = make_float2(gv * w[i][m].x, gv * w[i][m].y);
          }
        }
      }
    } else {
      const int u = p.un_of_block[j];
#pragma unroll
      for (int i = 0; i < NOBS; ++i) {
        if (i < p.n_obs) {
          const float2* gp = p.gjo + (size_t)(i * p.n_un + u) * tab + cc + t;
#pragma unroll
          for (int m = 0; m < V; ++m) {
            const float2 gv = active ? __ldg(gp + T * m) : make_float2(0.f, 0.f);
            s[m] = cadd(s[m], cmul(gv, w[i][m]));
          }
        }
      }
    }
    fft_line<NY, V, true>(s, line, t, p.twY);
    if (active) {
      float2* dst = p.S + ((size_t)j * p.N + k) * fstride + (size_t)col * NY + t;
      if (part == 0) {
#pragma unroll
        for (int m = 0; m < V; ++m) dst[T * m] = s[m];
      } else {
        float* d1 = reinterpret_cast<float*>(dst) + (part == 1 ? 0 : 1);
#pragma unroll
        for (int m = 0; m < V; ++m) d1[2 * T * m] = s[m].x;
      }
    }
  }
}

// ----------------------------------------------------------------- launch templates
template <int NY, int NOBS>
inline cudaError_t col_stats_NY(const ColStatsParams& p, cudaStream_t st) {
  constexpr int V = default_V(NY);
  constexpr int T = NY / V;
  int lpc = 1;
  const int nf = p.n_obs + 2 * p.n_obs * p.n_un;
  const size_t smem = col_stats_smem(NY, nf, &lpc);
  if (smem == 0) return cudaErrorInvalidConfiguration;
  auto kern = col_stats_kernel<NY, V, NOBS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (p.L + 1 + lpc - 1) / lpc;
  kern<<<grid, T * lpc, smem, st>>>(p);
  return cudaGetLastError();
}

template <int NY, int NOBS>
inline cudaError_t col_update_NY(const ColUpdParams& p, cudaStream_t st) {
  constexpr int V = default_V(NY);
  constexpr int T = NY / V;
  int lpc = 256 / T;
  if (lpc < 1) lpc = 1;
  const size_t smem = (size_t)lpc * padded_len(NY) * sizeof(float2);
  auto kern = col_update_kernel<NY, V, NOBS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long items = (long long)(p.L + 1) * p.N;
  const long long grid = (items + lpc - 1) / lpc;
  kern<<<(unsigned)grid, T * lpc, smem, st>>>(p);
  return cudaGetLastError();
}

#define FFTENKF_COL_SIZES(X) \
  X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2048) X(3072) X(4096)

template <int NOBS>
inline cudaError_t col_stats_dispatch(const ColStatsParams& p, cudaStream_t s) {
  switch (p.ny) {
#define CASE(n) case n: return col_stats_NY<n, NOBS>(p, s);
    FFTENKF_COL_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

template <int NOBS>
inline cudaError_t col_update_dispatch(const ColUpdParams& p, cudaStream_t s) {
  switch (p.ny) {
#define CASE(n) case n: return col_update_NY<n, NOBS>(p, s);
    FFTENKF_COL_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}


cudaError_t col_stats_nobs1(const ColStatsParams& p, cudaStream_t s);
cudaError_t col_stats_nobs2(const ColStatsParams& p, cudaStream_t s);
cudaError_t col_stats_nobs4(const ColStatsParams& p, cudaStream_t s);
cudaError_t col_update_nobs1(const ColUpdParams& p, cudaStream_t s);
cudaError_t col_update_nobs2(const ColUpdParams& p, cudaStream_t s);
cudaError_t col_update_nobs4(const ColUpdParams& p, cudaStream_t s);

}  // namespace fftenkf
