// Ensemble mean, forward row pass (real-to-complex) and inverse row pass
// (complex-to-real + add + store).
//
// Forward row pass, one CTA per (field, tile of R rows): every row of nx reals
// is read as nx/2 complex values z[m] = x[2m] + i x[2m+1], transformed by an
// L = nx/2 point FFT, and the spectrum of the real row is recovered from the
// pairs Z[k], Z[L-k] (X[k] = E[k] + W^k O[k], E/O the spectra of even/odd
// samples).  The R transformed rows are staged in shared memory and written
// transposed, R consecutive rows of one column k_x per 16-byte vector store,
// so that the column passes read each wavenumber column as one contiguous line.
// The inverse row pass does the same in reverse and adds the increment to the
// forecast member in the same pass.
#include "common.cuh"

namespace fftenkf {

// ----------------------------------------------------------------- mean
// ubar^(j)(x) = (1/N) sum_k u_k^(j)(x).  The sum is carried as an unevaluated
// pair hi + lo with an error-free two-sum per addition, so the mean is the
// exact sum divided by N and rounded once to float.
__global__ void __launch_bounds__(256) mean_kernel(const MeanParams p) {
  const long long nvec = p.G / 8;
  const long long total = nvec * p.M;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / nvec);
    const long long q = idx - (long long)j * nvec;
    float hi[8], lo[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) hi[e] = lo[e] = 0.f;
    for (int k = 0; k < p.N; ++k) {
      const size_t off = ((size_t)j * p.N + k) * (size_t)p.G + (size_t)q * 8;
      float x[8];
      if (p.storage == kBF16) {
        const uint4 raw = __ldcs(reinterpret_cast<const uint4*>(reinterpret_cast<const __nv_bfloat16*>(p.ens) + off));
        const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float2 f = __bfloat1622float2(b[e]);
          x[2 * e] = f.x;
          x[2 * e + 1] = f.y;
        }
      } else {
        const float4* src = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(p.ens) + off);
        float4 a = __ldcs(src), b = __ldcs(src + 1);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float s = hi[e] + x[e];
        const float bp = s - hi[e];
        const float err = (hi[e] - (s - bp)) + (x[e] - bp);
        hi[e] = s;
        lo[e] += err;
      }
    }
    const float invN = 1.0f / (float)p.N;
    float m[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) m[e] = (hi[e] + lo[e]) * invN;
    float4* dst = reinterpret_cast<float4*>(p.mean + (size_t)j * p.G + (size_t)q * 8);
    dst[0] = make_float4(m[0], m[1], m[2], m[3]);
    dst[1] = make_float4(m[4], m[5], m[6], m[7]);
  }
}

cudaError_t launch_mean(const MeanParams& p, cudaStream_t s) {
  const long long total = (p.G / 8) * p.M;
  long long blocks = (total + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  mean_kernel<<<(int)blocks, 256, 0, s>>>(p);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- rows
template <int L, int V>
__global__ void __launch_bounds__(512) row_fwd_kernel(const RowFwdParams p) {
  constexpr int T = L / V;
  extern __shared__ float2 sm[];
  const int pitch = padded_len(L) + 1;
  const int LPC = blockDim.x / T;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  int b = blockIdx.x;
  const int k = b % p.N;
  b /= p.N;
  const int tile = b % p.n_tiles;
  const int jb = b / p.n_tiles;       // block j (anomaly) or observed index i (innovation)
  const int y0 = tile * p.R;
  const size_t G = (size_t)p.ny * p.nx;
  size_t f;
  const void* u;
  const float* mu = nullptr;
  const float* d = nullptr;
  const void* e = nullptr;
  if (p.mode == kAnomaly) {
    f = (size_t)jb * p.N + k;
    u = (p.storage == kBF16) ? (const void*)((const __nv_bfloat16*)p.ens + f * G)
                             : (const void*)((const float*)p.ens + f * G);
    mu = p.mean + (size_t)jb * G;
  } else {
    f = (size_t)k * p.n_obs + jb;
    const size_t fu = (size_t)p.obs[jb] * p.N + k;
    u = (p.storage == kBF16) ? (const void*)((const __nv_bfloat16*)p.ens + fu * G)
                             : (const void*)((const float*)p.ens + fu * G);
    d = p.data + (size_t)jb * G;
    e = (p.storage == kBF16) ? (const void*)((const __nv_bfloat16*)p.pert + f * G)
                             : (const void*)((const float*)p.pert + f * G);
  }
  for (int r0 = 0; r0 < p.R; r0 += LPC) {
    const int r = r0 + g;
    const size_t rowoff = (size_t)(y0 + r) * p.nx;
    float2 v[V];
#pragma unroll
    for (int m = 0; m < V; ++m) {
      const size_t idx = rowoff + 2 * (size_t)(t + T * m);
      const float2 a = load2(u, idx, p.storage);
      if (p.mode == kAnomaly) {
        const float2 c = *reinterpret_cast<const float2*>(mu + idx);
        v[m] = make_float2(a.x - c.x, a.y - c.y);
      } else {
        const float2 dd = *reinterpret_cast<const float2*>(d + idx);
        const float2 ee = load2(e, idx, p.storage);
        v[m] = make_float2((dd.x + ee.x) - a.x, (dd.y + ee.y) - a.y);
      }
    }
    float2* line = sm + r * pitch;
    fft_line<L, V, false>(v, line, t, p.twL);
#pragma unroll
    for (int m = 0; m < V; ++m) line[pidx(t + T * m)] = v[m];
  }
  __syncthreads();
  // spectrum of the real rows, written transposed: out[c][y0 + r]
  float2* out = p.out + f * (size_t)L * p.ny + y0;
  const int RP = p.R >> 1;
  for (int idx = threadIdx.x; idx < L * RP; idx += blockDim.x) {
    const int rp = idx % RP;
    const int c = idx / RP;
    const float2 w = __ldg(p.twX + c);
    float2 res[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float2* row = sm + (2 * rp + q) * pitch;
      const float2 Z = row[pidx(c)];
      if (c == 0) {
        res[q] = make_float2(Z.x + Z.y, Z.x - Z.y);   // packed: X[0] + i X[L]
      } else {
        const float2 Zc = row[pidx(L - c)];
        const float2 E = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y - Zc.y));
        const float2 O = make_float2(0.5f * (Z.y + Zc.y), -0.5f * (Z.x - Zc.x));
        res[q] = cadd(E, cmul(w, O));
      }
    }
    *reinterpret_cast<float4*>(out + (size_t)c * p.ny + 2 * rp) = make_float4(res[0].x, res[0].y, res[1].x, res[1].y);
  }
}

template <int L, int V>
__global__ void __launch_bounds__(512) row_inv_kernel(const RowInvParams p) {
  constexpr int T = L / V;
  extern __shared__ float2 sm[];
  const int pitch = padded_len(L) + 1;
  const int LPC = blockDim.x / T;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int tile = blockIdx.x % p.n_tiles;
  const size_t f = blockIdx.x / p.n_tiles;         // field j*N + k
  const int y0 = tile * p.R;
  const size_t G = (size_t)p.ny * p.nx;
  const float2* in = p.in + f * (size_t)L * p.ny + y0;
  const int RP = p.R >> 1;
  for (int idx = threadIdx.x; idx < L * RP; idx += blockDim.x) {
    const int rp = idx % RP;
    const int c = idx / RP;
    const float4 v4 = *reinterpret_cast<const float4*>(in + (size_t)c * p.ny + 2 * rp);
    sm[(2 * rp) * pitch + pidx(c)] = make_float2(v4.x, v4.y);
    sm[(2 * rp + 1) * pitch + pidx(c)] = make_float2(v4.z, v4.w);
  }
  __syncthreads();
  void* u = (p.storage == kBF16) ? (void*)((__nv_bfloat16*)p.ens + f * G) : (void*)((float*)p.ens + f * G);
  for (int r0 = 0; r0 < p.R; r0 += LPC) {
    const int r = r0 + g;
    float2* line = sm + r * pitch;
    float2 v[V];
#pragma unroll
    for (int m = 0; m < V; ++m) {
      const int c = t + T * m;
      const float2 X = line[pidx(c)];
      if (c == 0) {
        v[m] = make_float2(X.x + X.y, X.x - X.y);
      } else {
        const float2 Xc = line[pidx(L - c)];
        const float2 A = make_float2(X.x + Xc.x, X.y - Xc.y);
        const float2 B = make_float2(X.x - Xc.x, X.y + Xc.y);
        const float2 Bw = cmulc(B, __ldg(p.twX + c));
        v[m] = make_float2(A.x - Bw.y, A.y + Bw.x);
      }
    }
    __syncthreads();
    fft_line<L, V, true>(v, line, t, p.twL);
    const size_t rowoff = (size_t)(y0 + r) * p.nx;
#pragma unroll
    for (int m = 0; m < V; ++m) {
      const size_t idx = rowoff + 2 * (size_t)(t + T * m);
      const float2 a = load2(u, idx, p.storage);
      store2(u, idx, make_float2(a.x + v[m].x, a.y + v[m].y), p.storage);
    }
  }
}

// ----------------------------------------------------------------- launch
struct RowShape {
  int T, R, LPC;
  size_t smem;
};

static RowShape row_shape(int L, int V, int ny) {
  RowShape s;
  s.T = L / V;
  int pow2 = ny & -ny;                       // largest power of two dividing ny
  int R = 256 / s.T;
  if (R < 8) R = 8;
  if (R > pow2) R = pow2;
  while (R > 2 && (size_t)R * (padded_len(L) + 1) * sizeof(float2) > 160 * 1024) R >>= 1;
  s.R = R;
  int LPC = 512 / s.T;
  if (LPC < 1) LPC = 1;
  if (LPC > R) LPC = R;
  s.LPC = LPC;
  s.smem = (size_t)R * (padded_len(L) + 1) * sizeof(float2);
  return s;
}

template <int L>
static cudaError_t row_fwd_L(RowFwdParams p, int n_fields, cudaStream_t st) {
  constexpr int V = default_V(L);
  RowShape s = row_shape(L, V, p.ny);
  p.R = s.R;
  p.n_tiles = p.ny / s.R;
  auto kern = row_fwd_kernel<L, V>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  if (e != cudaSuccess) return e;
  const long long grid = (long long)n_fields * p.n_tiles;  // = (obs or blocks) * tiles * N
  kern<<<(unsigned)grid, s.T * s.LPC, s.smem, st>>>(p);
  return cudaGetLastError();
}

template <int L>
static cudaError_t row_inv_L(RowInvParams p, int n_fields, cudaStream_t st) {
  constexpr int V = default_V(L);
  RowShape s = row_shape(L, V, p.ny);
  p.R = s.R;
  p.n_tiles = p.ny / s.R;
  auto kern = row_inv_kernel<L, V>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  if (e != cudaSuccess) return e;
  const long long grid = (long long)n_fields * p.n_tiles;
  kern<<<(unsigned)grid, s.T * s.LPC, s.smem, st>>>(p);
  return cudaGetLastError();
}

#define FFTENKF_ROW_SIZES(X) \
  X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2048) X(3072) X(4096)

cudaError_t launch_row_fwd(const RowFwdParams& p, int n_fields, cudaStream_t s) {
  switch (p.L) {
#define CASE(n) case n: return row_fwd_L<n>(p, n_fields, s);
    FFTENKF_ROW_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

bool row_line_supported(int n) {
  switch (n) {
#define CASE(m) case m: return true;
    FFTENKF_ROW_SIZES(CASE)
#undef CASE
    default: return false;
  }
}

cudaError_t launch_row_inv(const RowInvParams& p, int n_fields, cudaStream_t s) {
  switch (p.L) {
#define CASE(n) case n: return row_inv_L<n>(p, n_fields, s);
    FFTENKF_ROW_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fftenkf
