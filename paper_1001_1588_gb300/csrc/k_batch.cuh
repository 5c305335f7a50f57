// Device bodies of the batched passes (one work unit each), shared by the
// per-pass translation units k_batch_*.cu.
#pragma once
#include "batch.cuh"

namespace fftenkf {

#define FFTENKF_BATCH_SIZES(X) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024)

__device__ __forceinline__ const float2* sel_tw(const float2* a, const float2* b, int vsel) { return vsel ? b : a; }

// rows per row-pass tile: one round of lpc concurrent rows, at least 8, at most the
// largest power of two dividing ny (host and device agree through this function)
__host__ __device__ __forceinline__ int batch_rows_per_tile(int ny, int lpc) {
  int R = lpc < 8 ? 8 : lpc;
  const int pow2 = ny & -ny;
  return R > pow2 ? pow2 : R;
}

// ----------------------------------------------------------------- mean
__device__ __forceinline__ void batch_mean_unit(const BatchItem& it, int u, int storage) {
  const size_t G = (size_t)it.ny * it.nx;
  const size_t q = ((size_t)u * blockDim.x + threadIdx.x) * 8;
  if (q >= G) return;
  float hi[8], lo[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) hi[e] = lo[e] = 0.f;
  for (int k = 0; k < it.N; ++k) {
    const size_t off = (size_t)k * G + q;
    float x[8];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      const float2 a = load2(it.ens, off + e, storage);
      x[e] = a.x;
      x[e + 1] = a.y;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float s = hi[e] + x[e];
      const float bp = s - hi[e];
      lo[e] += (hi[e] - (s - bp)) + (x[e] - bp);
      hi[e] = s;
    }
  }
  const float Nf = (float)it.N, inv_N = 1.0f / Nf;
  float4* dst = reinterpret_cast<float4*>(it.mean + q);
  dst[0] = make_float4(pair_div(hi[0], lo[0], Nf, inv_N), pair_div(hi[1], lo[1], Nf, inv_N), pair_div(hi[2], lo[2], Nf, inv_N),
                       pair_div(hi[3], lo[3], Nf, inv_N));
  dst[1] = make_float4(pair_div(hi[4], lo[4], Nf, inv_N), pair_div(hi[5], lo[5], Nf, inv_N), pair_div(hi[6], lo[6], Nf, inv_N),
                       pair_div(hi[7], lo[7], Nf, inv_N));
}

// ----------------------------------------------------------------- row passes
template <int L, int V>
__device__ void batch_row_fwd_unit(const BatchItem& it, int u, int mode, int storage, int vsel, float2* sm) {
  constexpr int T = L / V;
  constexpr int pitch = row_pitch(L);
  const int LPC = blockDim.x / T;
  const int g = threadIdx.x / T, t = threadIdx.x - g * T;
  const int R = batch_rows_per_tile(it.ny, LPC);
  const int n_tiles = it.ny / R;
  const int k = u / n_tiles, tile = u - k * n_tiles;
  const int y0 = tile * R;
  const size_t G = (size_t)it.ny * it.nx;
  const float2* tw = sel_tw(it.twL, it.twL_alt, vsel);
  const int es = storage == kBF16 ? 2 : 4;
  const char* ub = reinterpret_cast<const char*>(it.ens) + (size_t)k * G * es;
  const char* eb = reinterpret_cast<const char*>(it.pert) + (size_t)k * G * es;
  for (int r0 = 0; r0 < R; r0 += LPC) {
    const int row = r0 + g;
    const bool act = row < R;
    float2 v[V];
    const size_t rowoff = (size_t)(y0 + (act ? row : 0)) * it.nx;
#pragma unroll
    for (int m = 0; m < V; ++m) {
      const size_t idx = rowoff + 2 * (size_t)(t + T * m);
      const float2 a = act ? load2(ub, idx, storage) : make_float2(0.f, 0.f);
      if (mode == kAnomaly) {
        const float2 c = act ? *reinterpret_cast<const float2*>(it.mean + idx) : make_float2(0.f, 0.f);
        v[m] = make_float2(a.x - c.x, a.y - c.y);
      } else {
        const float2 dd = act ? *reinterpret_cast<const float2*>(it.data + idx) : make_float2(0.f, 0.f);
        const float2 ee = act ? load2(eb, idx, storage) : make_float2(0.f, 0.f);
        v[m] = make_float2((dd.x - a.x) + ee.x, (dd.y - a.y) + ee.y);   // d - u first: exact for close d, u
      }
    }
    float2* line = sm + (act ? row : R) * pitch;     // idle groups use a spare line
    fft_line<L, V, false>(v, line, t, tw);
    if (act) {
#pragma unroll
      for (int m = 0; m < V; ++m) line[pidx(t + T * m)] = v[m];
    }
  }
  __syncthreads();
  float2* out = ((mode == kAnomaly) ? it.A : it.W) + (size_t)k * L * it.ny + y0;
  const int RP = R >> 1;
  for (int idx = threadIdx.x; idx < L * RP; idx += blockDim.x) {
    const int rp = idx % RP, c = idx / RP;
    float2 res[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float2* row = sm + (2 * rp + q) * pitch;
      const float2 Z = row[pidx(c)];
      if (c == 0) {
        res[q] = make_float2(Z.x + Z.y, Z.x - Z.y);
      } else {
        const float2 Zc = row[pidx(L - c)];
        const float2 E = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y - Zc.y));
        const float2 O = make_float2(0.5f * (Z.y + Zc.y), -0.5f * (Z.x - Zc.x));
        res[q] = cadd(E, cmul(__ldg(it.twX + c), O));
      }
    }
    *reinterpret_cast<float4*>(out + (size_t)c * it.ny + 2 * rp) = make_float4(res[0].x, res[0].y, res[1].x, res[1].y);
  }
  __syncthreads();
}

template <int L, int V>
__device__ void batch_row_inv_unit(const BatchItem& it, int u, int storage, int vsel, float2* sm) {
  constexpr int T = L / V;
  constexpr int pitch = row_pitch(L);
  const int LPC = blockDim.x / T;
  const int g = threadIdx.x / T, t = threadIdx.x - g * T;
  const int R = batch_rows_per_tile(it.ny, LPC);
  const int n_tiles = it.ny / R;
  const int k = u / n_tiles, tile = u - k * n_tiles;
  const int y0 = tile * R;
  const size_t G = (size_t)it.ny * it.nx;
  const float2* tw = sel_tw(it.twL, it.twL_alt, vsel);
  const float2* in = it.A + (size_t)k * L * it.ny + y0;
  const int RP = R >> 1;
  for (int idx = threadIdx.x; idx < L * RP; idx += blockDim.x) {
    const int rp = idx % RP, c = idx / RP;
    const float4 v4 = *reinterpret_cast<const float4*>(in + (size_t)c * it.ny + 2 * rp);
    sm[(2 * rp) * pitch + pidx(c)] = make_float2(v4.x, v4.y);
    sm[(2 * rp + 1) * pitch + pidx(c)] = make_float2(v4.z, v4.w);
  }
  __syncthreads();
  char* ub = reinterpret_cast<char*>(it.ens) + (size_t)k * G * (storage == kBF16 ? 2 : 4);
  for (int r0 = 0; r0 < R; r0 += LPC) {
    const int row = r0 + g;
    const bool act = row < R;
    float2* line = sm + (act ? row : R) * pitch;
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
        const float2 Bw = cmulc(B, __ldg(it.twX + c));
        v[m] = make_float2(A.x - Bw.y, A.y + Bw.x);
      }
    }
    __syncthreads();
    fft_line<L, V, true>(v, line, t, tw);
    if (act) {
      const size_t rowoff = (size_t)(y0 + row) * it.nx;
#pragma unroll
      for (int m = 0; m < V; ++m) {
        const size_t idx = rowoff + 2 * (size_t)(t + T * m);
        const float2 a = load2(ub, idx, storage);
        store2(ub, idx, make_float2(a.x + v[m].x, a.y + v[m].y), storage);
      }
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------- column passes
template <int NY, int V>
__device__ void batch_col_stats_unit(const BatchItem& it, int u, int vsel, float2* sm, int* status) {
  constexpr int T = NY / V;
  constexpr int PL = (padded_len(NY) + 1) & ~1;
  const int LPC = blockDim.x / T;
  const int g = threadIdx.x / T, t = threadIdx.x - g * T;
  const int c = u * LPC + g;
  const bool act = c <= it.L;
  const int col = (c == it.L) ? 0 : c;
  const int part = (c == 0) ? 1 : ((c == it.L) ? 2 : 0);
  const float2* tw = sel_tw(it.twY, it.twY_alt, vsel);
  float2* line = sm + (size_t)g * PL;
  float acc[V];
#pragma unroll
  for (int m = 0; m < V; ++m) acc[m] = 0.f;
  for (int k = 0; k < it.N; ++k) {
    const float2* src = it.A + ((size_t)k * it.L + col) * NY;
    float2 v[V];
#pragma unroll
    for (int m = 0; m < V; ++m) {
      float2 a = act ? src[t + T * m] : make_float2(0.f, 0.f);
      if (part == 1) a.y = 0.f;
      if (part == 2) a = make_float2(a.y, 0.f);
      v[m] = a;
    }
    fft_line<NY, V, false>(v, line, t, tw);
#pragma unroll
    for (int m = 0; m < V; ++m) acc[m] += v[m].x * v[m].x + v[m].y * v[m].y;
  }
  if (act) {
    const float scale = 1.0f / ((float)(it.N - 1) * (float)it.ny * (float)it.nx);
    bool bad = false;
#pragma unroll
    for (int m = 0; m < V; ++m) {
      const float val = acc[m] * scale;
      bad |= !isfinite(val);
      it.chat[(size_t)c * NY + t + T * m] = val;
    }
    if (bad) atomicOr(status, kStatusNonFinite);
  }
}

template <int NY, int V>
__device__ void batch_col_update_unit(const BatchItem& it, int u, int vsel, float2* sm) {
  constexpr int T = NY / V;
  constexpr int PL = (padded_len(NY) + 1) & ~1;
  const int LPC = blockDim.x / T;
  const int g = threadIdx.x / T, t = threadIdx.x - g * T;
  const int item = u * LPC + g;
  const int c = item / it.N, k = item - (item / it.N) * it.N;
  const bool act = c <= it.L;
  const int col = (c == it.L) ? 0 : c;
  const int part = (c == 0) ? 1 : ((c == it.L) ? 2 : 0);
  const float2* tw = sel_tw(it.twY, it.twY_alt, vsel);
  float2* line = sm + (size_t)g * PL;
  const float2* src = it.W + ((size_t)k * it.L + col) * NY;
  float2 v[V];
#pragma unroll
  for (int m = 0; m < V; ++m) {
    float2 a = act ? src[t + T * m] : make_float2(0.f, 0.f);
    if (part == 1) a.y = 0.f;
    if (part == 2) a = make_float2(a.y, 0.f);
    v[m] = a;
  }
  fft_line<NY, V, false>(v, line, t, tw);
  const float* gp = it.gain + (size_t)(act ? c : 0) * NY + t;
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const float gv = act ? __ldg(gp + T * m) : 0.f;
    v[m] = make_float2(gv * v[m].x, gv * v[m].y);
  }
  fft_line<NY, V, true>(v, line, t, tw);
  if (act) {
    float2* dst = it.A + ((size_t)k * it.L + col) * NY + t;
    if (part == 0) {
#pragma unroll
      for (int m = 0; m < V; ++m) dst[T * m] = v[m];
    } else {
      float* d1 = reinterpret_cast<float*>(dst) + (part == 1 ? 0 : 1);
#pragma unroll
      for (int m = 0; m < V; ++m) d1[2 * T * m] = v[m].x;
    }
  }
}

}  // namespace fftenkf
