// Ensemble mean and the storage-independent entry points of the row passes
// (the row kernels are in k_rows.cuh).
#include "k_rows.cuh"

namespace fftenkf {

// ----------------------------------------------------------------- mean
// ubar^(j)(x) = (1/N) sum_k u_k^(j)(x).  The sum is carried as an unevaluated
// pair hi + lo with an error-free two-sum per addition, so it is exact; the mean
// is its quotient by N to within one unit in the last place (pair_div), exact
// when that quotient is a float.
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
    // four members' loads in flight before they are summed
    for (int k0 = 0; k0 < p.N; k0 += 4) {
      float x[4][8];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int k = k0 + kk;
        if (k >= p.N) break;
        const size_t off = ((size_t)j * p.N + k) * (size_t)p.G + (size_t)q * 8;
        if (p.storage == kBF16) {
          const uint4 raw = __ldcs(reinterpret_cast<const uint4*>(reinterpret_cast<const __nv_bfloat16*>(p.ens) + off));
          const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float2 f = __bfloat1622float2(b[e]);
            x[kk][2 * e] = f.x;
            x[kk][2 * e + 1] = f.y;
          }
        } else {
          const float4* src = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(p.ens) + off);
          float4 a = __ldcs(src), b = __ldcs(src + 1);
          x[kk][0] = a.x; x[kk][1] = a.y; x[kk][2] = a.z; x[kk][3] = a.w;
          x[kk][4] = b.x; x[kk][5] = b.y; x[kk][6] = b.z; x[kk][7] = b.w;
        }
      }
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        if (k0 + kk >= p.N) break;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float s = hi[e] + x[kk][e];
          const float bp = s - hi[e];
          const float err = (hi[e] - (s - bp)) + (x[kk][e] - bp);
          hi[e] = s;
          lo[e] += err;
        }
      }
    }
    const float Nf = (float)p.N, inv_N = 1.0f / Nf;
    float m[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) m[e] = pair_div(hi[e], lo[e], Nf, inv_N);
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

cudaError_t launch_row_fwd(const RowFwdParams& p, int n_fields, cudaStream_t s) {
  return p.storage == kBF16 ? launch_row_fwd_bf16(p, n_fields, s) : launch_row_fwd_f32(p, n_fields, s);
}

bool row_line_supported(int n) {
  switch (n) {
#define CASE(m) case m: return true;
    FFTENKF_ROW_SIZES(CASE)
#undef CASE
    default: return false;
  }
}

template <int L>
int row_inv_rows_L(int vsel, int ny, int nx, int es) {
  const int V = (vsel & 1) ? plan_V(L, 1) : plan_V(L, 0);
  RowShape s = inv_shape(L, V, ny, nx, es, (vsel & 2) != 0);
  // tensor copies need R >= 2 (16-byte rows of the box)
  return (s.R < 2 || s.smem > 227 * 1024 || s.T * s.R > 512) ? 0 : s.R;
}

int row_inv_rows(int L, int vsel, int ny, int nx, int es) {
  switch (L) {
#define CASE(n) case n: return row_inv_rows_L<n>(vsel, ny, nx, es);
    FFTENKF_ROW_SIZES(CASE)
#undef CASE
    default: return 0;
  }
}

cudaError_t launch_row_inv(const RowInvParams& p, int n_fields, cudaStream_t s) {
  return p.storage == kBF16 ? launch_row_inv_bf16(p, n_fields, s) : launch_row_inv_f32(p, n_fields, s);
}

}  // namespace fftenkf
