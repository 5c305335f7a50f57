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
#include "tma.cuh"

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
// Persistent CTAs walk the tiles (member fastest, so the CTAs working on the
// same rows of different members run together and share the mean or data rows
// through L2).  Each tile of R rows is done in rounds of LPC rows; the
// per-member input rows of the next round (u, and e for innovations) are bulk
// copied into a shared-memory stage while the current round is transformed.
struct RowTile {
  int k, tile, jb;
};

__device__ __forceinline__ RowTile decode_tile(long long q, int N, int n_tiles) {
  RowTile r;
  r.k = (int)(q % N);
  q /= N;
  r.tile = (int)(q % n_tiles);
  r.jb = (int)(q / n_tiles);
  return r;
}

template <int L, int V>
__global__ void __launch_bounds__(512, 1) row_fwd_kernel(const RowFwdParams p) {
  constexpr int T = L / V;
  constexpr int pitch = row_pitch(L);
  extern __shared__ __align__(128) unsigned char smraw[];
  const int LPC = blockDim.x / T;
  const int rounds = p.R / LPC;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int nx = p.nx;
  const size_t G = (size_t)p.ny * nx;
  const int es = (p.storage == kBF16) ? 2 : 4;
  const int n_in = (p.mode == kAnomaly) ? 1 : 2;
  const uint32_t round_bytes = (uint32_t)LPC * nx * es;
  float2* lines = reinterpret_cast<float2*>(smraw);
  unsigned char* stage = smraw + (((size_t)p.R * pitch * sizeof(float2) + 127) & ~(size_t)127);
  uint64_t* bar = reinterpret_cast<uint64_t*>(stage + (size_t)n_in * round_bytes);
  int* flag = reinterpret_cast<int*>(bar + 1);
  const int n_jb = (p.mode == kAnomaly) ? p.M : p.n_obs;
  const long long Q = (long long)n_jb * p.n_tiles * p.N;
  const char* ens = reinterpret_cast<const char*>(p.ens);
  const char* pert = reinterpret_cast<const char*>(p.pert);

  auto issue = [&](long long q, int r) {
    const RowTile w = decode_tile(q, p.N, p.n_tiles);
    const size_t row0 = (size_t)w.tile * p.R + (size_t)r * LPC;
    const size_t fu = (p.mode == kAnomaly) ? (size_t)w.jb * p.N + w.k : (size_t)p.obs[w.jb] * p.N + w.k;
    mbar_arrive_expect_tx(bar, n_in * round_bytes);
    bulk_g2s(stage, ens + (fu * G + row0 * nx) * es, round_bytes, bar);
    if (p.mode == kInnovation) {
      const size_t fe = (size_t)w.k * p.n_obs + w.jb;
      bulk_g2s(stage + round_bytes, pert + (fe * G + row0 * nx) * es, round_bytes, bar);
    }
  };

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  long long q = blockIdx.x;
  if (threadIdx.x == 0 && q < Q) issue(q, 0);
  const int RP = p.R >> 1;
  const int rp = threadIdx.x % RP;
  const int cstep = blockDim.x / RP;
  for (; q < Q; q += gridDim.x) {
    const RowTile w = decode_tile(q, p.N, p.n_tiles);
    const int y0 = w.tile * p.R;
    const size_t f = (p.mode == kAnomaly) ? (size_t)w.jb * p.N + w.k : (size_t)w.k * p.n_obs + w.jb;
    const float* shared_in = (p.mode == kAnomaly) ? p.mean + (size_t)w.jb * G : p.data + (size_t)w.jb * G;
    for (int r = 0; r < rounds; ++r) {
      const int row = r * LPC + g;
      const float* sh = shared_in + (size_t)(y0 + row) * nx;
      float2 sv[V];
#pragma unroll
      for (int m = 0; m < V; ++m) sv[m] = __ldg(reinterpret_cast<const float2*>(sh) + t + T * m);
      if (!cta_wait(bar, phase, p.status, flag)) return;
      phase ^= 1;
      float2 v[V];
      const unsigned char* st_row = stage + (size_t)g * nx * es;
#pragma unroll
      for (int m = 0; m < V; ++m) {
        const size_t idx = 2 * (size_t)(t + T * m);
        const float2 a = load2(st_row, idx, p.storage);
        if (p.mode == kAnomaly) {
          v[m] = make_float2(a.x - sv[m].x, a.y - sv[m].y);
        } else {
          const float2 ee = load2(st_row + round_bytes, idx, p.storage);
          v[m] = make_float2((sv[m].x + ee.x) - a.x, (sv[m].y + ee.y) - a.y);
        }
      }
      __syncthreads();   // stage consumed
      if (threadIdx.x == 0) {
        if (r + 1 < rounds) issue(q, r + 1);
        else if (q + gridDim.x < Q) issue(q + gridDim.x, 0);
      }
      float2* line = lines + row * pitch;
      fft_line<L, V, false>(v, line, t, p.twL);
#pragma unroll
      for (int m = 0; m < V; ++m) line[pidx(t + T * m)] = v[m];
    }
    __syncthreads();
    // spectrum of the real rows, written transposed: out[c][y0 + r]
    float2* out = p.out + f * (size_t)L * p.ny + y0 + 2 * rp;
    const float2* r0 = lines + (2 * rp) * pitch;
    const float2* r1 = r0 + pitch;
    for (int c = threadIdx.x / RP; c < L; c += cstep) {
      float2 res[2];
      const float2 Z0 = r0[pidx(c)], Z1 = r1[pidx(c)];
      if (c == 0) {
        res[0] = make_float2(Z0.x + Z0.y, Z0.x - Z0.y);   // packed: X[0] + i X[L]
        res[1] = make_float2(Z1.x + Z1.y, Z1.x - Z1.y);
      } else {
        const float2 wt = __ldg(p.twX + c);
        const float2 C0 = r0[pidx(L - c)], C1 = r1[pidx(L - c)];
        const float2 E0 = make_float2(0.5f * (Z0.x + C0.x), 0.5f * (Z0.y - C0.y));
        const float2 O0 = make_float2(0.5f * (Z0.y + C0.y), -0.5f * (Z0.x - C0.x));
        const float2 E1 = make_float2(0.5f * (Z1.x + C1.x), 0.5f * (Z1.y - C1.y));
        const float2 O1 = make_float2(0.5f * (Z1.y + C1.y), -0.5f * (Z1.x - C1.x));
        res[0] = cadd(E0, cmul(wt, O0));
        res[1] = cadd(E1, cmul(wt, O1));
      }
      *reinterpret_cast<float4*>(out + (size_t)c * p.ny) = make_float4(res[0].x, res[0].y, res[1].x, res[1].y);
    }
    __syncthreads();
  }
}

template <int L, int V>
__global__ void __launch_bounds__(512, 1) row_inv_kernel(const RowInvParams p) {
  constexpr int T = L / V;
  constexpr int pitch = row_pitch(L);
  extern __shared__ __align__(128) unsigned char smraw[];
  const int LPC = blockDim.x / T;
  const int rounds = p.R / LPC;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int nx = p.nx;
  const size_t G = (size_t)p.ny * nx;
  const int es = (p.storage == kBF16) ? 2 : 4;
  const uint32_t round_bytes = (uint32_t)LPC * nx * es;
  float2* lines = reinterpret_cast<float2*>(smraw);
  unsigned char* stage = smraw + (((size_t)p.R * pitch * sizeof(float2) + 127) & ~(size_t)127);
  uint64_t* bar = reinterpret_cast<uint64_t*>(stage + round_bytes);
  int* flag = reinterpret_cast<int*>(bar + 1);
  const long long Q = (long long)p.M * p.N * p.n_tiles;
  char* ens = reinterpret_cast<char*>(p.ens);

  auto issue = [&](long long q, int r) {      // forecast rows of the next round
    const size_t f = q / p.n_tiles;
    const int tile = (int)(q - (long long)f * p.n_tiles);
    const size_t row0 = (size_t)tile * p.R + (size_t)r * LPC;
    mbar_arrive_expect_tx(bar, round_bytes);
    bulk_g2s(stage, ens + (f * G + row0 * nx) * es, round_bytes, bar);
  };

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  long long q = blockIdx.x;
  if (threadIdx.x == 0 && q < Q) issue(q, 0);
  const int RP = p.R >> 1;
  const int rp = threadIdx.x % RP;
  const int cstep = blockDim.x / RP;
  for (; q < Q; q += gridDim.x) {
    const size_t f = q / p.n_tiles;               // field j*N + k
    const int tile = (int)(q - (long long)f * p.n_tiles);
    const int y0 = tile * p.R;
    {
      const float2* in = p.in + f * (size_t)L * p.ny + y0 + 2 * rp;
      float2* s0 = lines + (2 * rp) * pitch;
      float2* s1 = s0 + pitch;
      // 8 loads in flight per thread before their values are staged
      const int c0 = threadIdx.x / RP;
      const int nper = (L + cstep - 1) / cstep;
      for (int i0 = 0; i0 < nper; i0 += 8) {
        float4 v4[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = c0 + (i0 + u) * cstep;
          if (i0 + u < nper && c < L) v4[u] = __ldcs(reinterpret_cast<const float4*>(in + (size_t)c * p.ny));
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = c0 + (i0 + u) * cstep;
          if (i0 + u < nper && c < L) {
            s0[pidx(c)] = make_float2(v4[u].x, v4[u].y);
            s1[pidx(c)] = make_float2(v4[u].z, v4[u].w);
          }
        }
      }
    }
    __syncthreads();
    for (int r = 0; r < rounds; ++r) {
      const int row = r * LPC + g;
      float2* line = lines + row * pitch;
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
      if (!cta_wait(bar, phase, p.status, flag)) return;
      phase ^= 1;
      const unsigned char* st_row = stage + (size_t)g * nx * es;
      float2 a[V];
#pragma unroll
      for (int m = 0; m < V; ++m) a[m] = load2(st_row, 2 * (size_t)(t + T * m), p.storage);
      __syncthreads();   // stage consumed
      if (threadIdx.x == 0) {
        if (r + 1 < rounds) issue(q, r + 1);
        else if (q + gridDim.x < Q) issue(q + gridDim.x, 0);
      }
      char* urow = ens + (f * G + (size_t)(y0 + row) * nx) * es;
#pragma unroll
      for (int m = 0; m < V; ++m)
        store2(urow, 2 * (size_t)(t + T * m), make_float2(a[m].x + v[m].x, a[m].y + v[m].y), p.storage);
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------- launch
int sm_count();

struct RowShape {
  int T, R, LPC;
  size_t smem;
};

// rows per tile R (a power of two dividing ny), rows per round LPC, and the
// shared memory: R staged rows plus one round of n_in input rows
static RowShape row_shape(int L, int V, int ny, int nx, int es, int n_in, bool half) {
  RowShape s;
  s.T = L / V;
  const int pow2 = ny & -ny;
  int R = 256 / s.T;
  if (R < 8) R = 8;
  if (R > pow2) R = pow2;
  if (half && R > 2) R >>= 1;
  for (;;) {
    int LPC = 512 / s.T;
    if (LPC < 1) LPC = 1;
    if (LPC > R) LPC = R;
    const size_t lines = ((size_t)R * row_pitch(L) * sizeof(float2) + 127) & ~(size_t)127;
    const size_t smem = lines + (size_t)n_in * LPC * nx * es + 16;
    if (smem <= 220 * 1024 || R <= 2) {
      s.R = R;
      s.LPC = LPC;
      s.smem = smem;
      return s;
    }
    R >>= 1;
  }
}

template <int L, int V>
static cudaError_t row_fwd_LV(RowFwdParams p, int n_fields, cudaStream_t st) {
  const int es = p.storage == kBF16 ? 2 : 4;
  RowShape s = row_shape(L, V, p.ny, p.nx, es, p.mode == kAnomaly ? 1 : 2, (p.vsel & 2) != 0);
  if (s.smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  p.R = s.R;
  p.n_tiles = p.ny / s.R;
  auto kern = row_fwd_kernel<L, V>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, s.T * s.LPC, s.smem);
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)n_fields * p.n_tiles;
  const long long cap = (long long)sm_count() * per_sm;
  if (grid > cap) grid = cap;
  kern<<<(unsigned)grid, s.T * s.LPC, s.smem, st>>>(p);
  return cudaGetLastError();
}

template <int L, int V>
static cudaError_t row_inv_LV(RowInvParams p, int n_fields, cudaStream_t st) {
  const int es = p.storage == kBF16 ? 2 : 4;
  RowShape s = row_shape(L, V, p.ny, p.nx, es, 1, (p.vsel & 2) != 0);
  if (s.smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  p.R = s.R;
  p.n_tiles = p.ny / s.R;
  auto kern = row_inv_kernel<L, V>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, s.T * s.LPC, s.smem);
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)n_fields * p.n_tiles;
  const long long cap = (long long)sm_count() * per_sm;
  if (grid > cap) grid = cap;
  kern<<<(unsigned)grid, s.T * s.LPC, s.smem, st>>>(p);
  return cudaGetLastError();
}

template <int L>
static cudaError_t row_fwd_L(const RowFwdParams& p, int n_fields, cudaStream_t st) {
  if (p.vsel & 1) return row_fwd_LV<L, plan_V(L, 1)>(p, n_fields, st);
  return row_fwd_LV<L, plan_V(L, 0)>(p, n_fields, st);
}

template <int L>
static cudaError_t row_inv_L(const RowInvParams& p, int n_fields, cudaStream_t st) {
  if (p.vsel & 1) return row_inv_LV<L, plan_V(L, 1)>(p, n_fields, st);
  return row_inv_LV<L, plan_V(L, 0)>(p, n_fields, st);
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
