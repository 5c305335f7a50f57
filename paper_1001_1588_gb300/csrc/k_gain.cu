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
#include <cstring>

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
                                                       int ny, int L, const ChatOutMap map) {
  __shared__ float2 tile[TB][TB + 1];
  const int L1 = L + 1;
  const int c0 = blockIdx.x * TB, ky0 = blockIdx.y * TB, q = blockIdx.z;
  const bool is_auto = q < map.n_auto;
  const size_t tab = (size_t)L1 * ny;
  const size_t K = (size_t)ny * L1;
  int src = 0, cj = 0;
  if (!is_auto) {
#pragma unroll 1
    for (int i = 0; i < 64; ++i)   // constant indices keep the map in the parameter bank
      if (i == q - map.n_auto) {
        src = map.src[i];
        cj = map.conj[i];
      }
  }
  for (int cc = threadIdx.y; cc < TB; cc += blockDim.y) {
    const int c = c0 + cc, ky = ky0 + threadIdx.x;
    float2 v = make_float2(0.f, 0.f);
    if (c < L1 && ky < ny) {
      if (is_auto) {
        v.x = chat_t[q * tab + (size_t)c * ny + ky];
      } else {
        v = reinterpret_cast<const float2*>(chat_t + map.n_auto * tab)[src * tab + (size_t)c * ny + ky];
        if (cj) v.y = -v.y;
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
        double* o = out + map.n_auto * K + (size_t)(q - map.n_auto) * 2 * K + ((size_t)ky * L1 + c) * 2;
        o[0] = v.x;
        o[1] = v.y;
      }
    }
  }
}

// Output tables: the auto table of every observed block, then for every observed o (ascending)
// the cross tables chat^(jo) of every block j != o (ascending; unobserved j only unless coupled).
// Column-pass tables: autos, then (coupled) the observed pair chat^(o1 o0), then chat^(u o_i) at
// n_pair + i n_un + u.
ChatOutMap chat_out_map(int n_obs, int n_un, int coupled, const int* obs, const int* un, int M) {
  ChatOutMap m;
  memset(&m, 0, sizeof(m));
  m.n_auto = n_obs;
  const int n_pair = coupled ? n_obs * (n_obs - 1) / 2 : 0;
  for (int i = 0; i < n_obs; ++i) {
    for (int j = 0; j < M; ++j) {
      if (j == obs[i]) continue;
      int u = -1, oi = -1;
      for (int a = 0; a < n_un; ++a)
        if (un[a] == j) u = a;
      for (int a = 0; a < n_obs; ++a)
        if (obs[a] == j) oi = a;
      if (u >= 0) {
        m.src[m.n_cplx] = n_pair + i * n_un + u;
        m.conj[m.n_cplx] = 0;
        ++m.n_cplx;
      } else if (coupled && oi >= 0) {   // n_obs = 2: chat^(o1 o0) stored, chat^(o0 o1) its conjugate
        m.src[m.n_cplx] = 0;
        m.conj[m.n_cplx] = (oi == 0) ? 1 : 0;
        ++m.n_cplx;
      }
    }
  }
  return m;
}

cudaError_t launch_chat_out(const float* chat_t, double* out, int ny, int L, const ChatOutMap& map, cudaStream_t s) {
  dim3 grid((L + 1 + TB - 1) / TB, (ny + TB - 1) / TB, map.n_auto + map.n_cplx);
  chat_out_kernel<<<grid, dim3(TB, 8), 0, s>>>(chat_t, out, ny, L, map);
  return cudaGetLastError();
}

// rhat [n][ny][L1] -> rhat_t [n][L1][ny]; with amp non-null also amp [n][L1][ny] = sqrt_G sqrt(rhat) in
// FP32, the amplitude of the perturbations drawn in frequency space
__global__ void __launch_bounds__(256) rhat_transpose_kernel(const double* __restrict__ in, double* __restrict__ out,
                                                             int ny, int L1, float* __restrict__ amp, float sqrt_G) {
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
    if (c < L1 && ky < ny) {
      const double r = tile[threadIdx.x][cc];
      dst[(size_t)c * ny + ky] = r;
      if (amp) amp[blockIdx.z * K + (size_t)c * ny + ky] = sqrt_G * sqrtf((float)r);
    }
  }
}

cudaError_t launch_rhat_transpose(const double* rhat, double* rhat_t, int n, int ny, int L, cudaStream_t s,
                                  float* amp, float sqrt_G) {
  dim3 grid((L + 1 + TB - 1) / TB, (ny + TB - 1) / TB, n);
  rhat_transpose_kernel<<<grid, dim3(TB, 8), 0, s>>>(rhat, rhat_t, ny, L + 1, amp, sqrt_G);
  return cudaGetLastError();
}

// One thread per wavenumber (column-major index at = k_x ny + k_y).  The bracket
// A = chat_OO + diag(rhat) is inverted in FP64: A^-1 when det A > 1e-6 a11 a22, the
// pseudo-inverse A / tr(A)^2 of a rank-1 bracket otherwise, 0 where tr(A) = 0; it is
// scaled by 1/(ny nx) and rounded to float, and K_r = chat_{r,O} A^-1 is formed in FP32.
__global__ void __launch_bounds__(256) coupled_gain_kernel(const CoupledGainParams p) {
  const size_t tab = (size_t)(p.L + 1) * p.ny;
  const float2* cx = reinterpret_cast<const float2*>(p.chat_t + p.n_obs * tab);
  bool bad = false;
  for (size_t at = blockIdx.x * (size_t)blockDim.x + threadIdx.x; at < tab; at += (size_t)gridDim.x * blockDim.x) {
    const float a0 = p.chat_t[at];
    const float a1 = (p.n_obs == 2) ? p.chat_t[tab + at] : 0.f;
    const float2 b10 = (p.n_obs == 2) ? cx[at] : make_float2(0.f, 0.f);   // chat^(o1 o0)
    float s00 = 0.f, s11 = 0.f;
    float2 s01 = make_float2(0.f, 0.f);
    const double g = (double)p.inv_G;
    if (p.n_obs == 1) {
      const double a = (double)a0 + p.rhat_t[at];
      s00 = (a != 0.0) ? (float)(g / a) : 0.f;
    } else {
      const double a = (double)a0 + p.rhat_t[at], d = (double)a1 + p.rhat_t[tab + at];
      const double br = b10.x, bi = b10.y;
      const double det = a * d - (br * br + bi * bi);
      const double tr = a + d;
      double f = 0.0, q00 = 0.0, q11 = 0.0, q01r = 0.0, q01i = 0.0;   // A^-1 = f [[q00, q01], [conj q01, q11]]
      if (det > 1e-6 * a * d) {
        f = g / det;
        q00 = d; q11 = a; q01r = -br; q01i = bi;      // [[d, -conj b10], [-b10, a]] / det
      } else if (tr > 0.0) {
        f = g / (tr * tr);
        q00 = a; q11 = d; q01r = br; q01i = -bi;      // [[a, conj b10], [b10, d]] / tr^2
      }
      s00 = (float)(f * q00);
      s11 = (float)(f * q11);
      s01 = make_float2((float)(f * q01r), (float)(f * q01i));
    }
    const float2 s10 = make_float2(s01.x, -s01.y);
    bad |= !(isfinite(s00) && isfinite(s11) && isfinite(s01.x) && isfinite(s01.y));
    // rows chat_{r,O}: observed o0 (a0, conj b10); observed o1 (b10, a1); unobserved u (x_0u, x_1u)
    for (int r = 0; r < p.n_obs + p.n_un; ++r) {
      float2 c0, c1 = make_float2(0.f, 0.f);
      if (r == 0) {
        c0 = make_float2(a0, 0.f);
        c1 = make_float2(b10.x, -b10.y);
      } else if (r == 1 && p.n_obs == 2) {
        c0 = b10;
        c1 = make_float2(a1, 0.f);
      } else {
        const int u = r - p.n_obs;
        c0 = cx[(size_t)(p.n_pair + u) * tab + at];
        if (p.n_obs == 2) c1 = cx[(size_t)(p.n_pair + p.n_un + u) * tab + at];
      }
      // K_{r,0} = c0 A^-1[0][0] + c1 A^-1[1][0], K_{r,1} = c0 A^-1[0][1] + c1 A^-1[1][1]
      const float2 k0 = cadd(cscale(c0, s00), cmul(c1, s10));
      p.gall[(size_t)r * p.n_obs * tab + at] = (p.n_obs == 2) ? k0 : cscale(c0, s00);
      if (p.n_obs == 2) p.gall[((size_t)r * 2 + 1) * tab + at] = cadd(cmul(c0, s01), cscale(c1, s11));
    }
  }
  if (bad) atomicOr(p.status, kStatusNonFinite);
}

cudaError_t launch_coupled_gain(const CoupledGainParams& p, cudaStream_t s) {
  const size_t tab = (size_t)(p.L + 1) * p.ny;
  long long blocks = (long long)((tab + 255) / 256);
  if (blocks > 152LL * 8) blocks = 152LL * 8;
  coupled_gain_kernel<<<(unsigned)blocks, 256, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace fftenkf
