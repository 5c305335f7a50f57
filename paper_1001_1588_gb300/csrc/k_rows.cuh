// Forward row pass (real-to-complex) and inverse row pass (complex-to-real +
// add + store): kernels and launch templates, instantiated per storage type in
// k_row_{fwd,inv}_{bf16,f32}.cu.
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
//
// The anomaly rows take the first member as pivot (row_anom_kernel): the sample
// covariance of eq. (dii) is unchanged when one field is subtracted from every
// member, and d_k = u_k - u_0 is exact in FP32 for BF16 members (and for FP32
// members within a factor two of each other, as under a large common mean), so
// the transforms see anomaly-sized values and no mean pass is needed.  Field
// j*N+k (k >= 1) receives the row spectra of d_k; field j*N+0 receives those of
// (1/sqrt N) sum_k d_k = sqrt(N) (ubar - u_0), whose products the column
// statistics subtract: sum_k D_k D'_k* - N Dbar Dbar'* = sum_k A_k A'_k* with
// D = F d, Dbar = F(ubar - u_0), A_k = F(u_k - ubar).
#pragma once
#include <cmath>

#include "common.cuh"
#include "tma.cuh"
#include "tmem.cuh"

namespace fftenkf {

int sm_count();

#define FFTENKF_ROW_SIZES(X) \
  X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2048) X(3072) X(4096)

// ----------------------------------------------------------------- rows
// Persistent CTAs walk the tiles.  Each tile of R rows is done in rounds of LPC
// rows; the per-member input rows of the next round (u, and e for innovations)
// are bulk copied into a shared-memory stage while the current round is
// transformed.
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

// Spectrum of the R real rows staged in `lines` (their L-point transforms), written transposed:
// out[c][y0 + r] of the field at fout.  Columns c and L - c come from the same pair Z[c], Z[L-c]:
// with E = (Z[c] + conj Z[L-c]) / 2 and O = -i (Z[c] - conj Z[L-c]) / 2, X[c] = E + W^c O and
// X[L-c] = conj(E - W^c O); column 0 holds X[0] + i X[L] (packed).  Every thread of the CTA calls it.
template <int L>
__device__ __forceinline__ void row_twist_store(const float2* lines, float2* fout, int R, int ny, int y0,
                                                const float2* __restrict__ twX) {
  constexpr int pitch = row_pitch(L);
  const int RP = R >> 1;
  const int rp = threadIdx.x % RP;
  const int cstep = blockDim.x / RP;
  float2* out = fout + y0 + 2 * rp;
  const float2* r0 = lines + (2 * rp) * pitch;
  const float2* r1 = r0 + pitch;
  for (int c = threadIdx.x / RP; c <= L / 2; c += cstep) {
    const float2 Z0 = r0[pidx(c)], Z1 = r1[pidx(c)];
    if (c == 0) {
      *reinterpret_cast<float4*>(out) = make_float4(Z0.x + Z0.y, Z0.x - Z0.y, Z1.x + Z1.y, Z1.x - Z1.y);
      continue;
    }
    const float2 C0 = r0[pidx(L - c)], C1 = r1[pidx(L - c)];
    float2 wt = __ldg(twX + c);
    wt = make_float2(0.5f * wt.x, 0.5f * wt.y);
    float2 lo[2], hi[2];
    const float2 Zs[2] = {Z0, Z1}, Cs[2] = {C0, C1};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float2 E2 = make_float2(Zs[h].x + Cs[h].x, Zs[h].y - Cs[h].y);   // 2 E
      const float2 O2 = make_float2(Zs[h].y + Cs[h].y, Cs[h].x - Zs[h].x);   // 2 O
      const float2 P = cmul(wt, O2);                                          // W^c O
      lo[h] = make_float2(fmaf(0.5f, E2.x, P.x), fmaf(0.5f, E2.y, P.y));
      hi[h] = make_float2(fmaf(0.5f, E2.x, -P.x), fmaf(-0.5f, E2.y, P.y));
    }
    *reinterpret_cast<float4*>(out + (size_t)c * ny) = make_float4(lo[0].x, lo[0].y, lo[1].x, lo[1].y);
    if (c != L - c)
      *reinterpret_cast<float4*>(out + (size_t)(L - c) * ny) = make_float4(hi[0].x, hi[0].y, hi[1].x, hi[1].y);
  }
}

// Innovation rows: work items (member k fastest, tile, observed block), so that the CTAs
// working on the same rows of different members run together and share the data rows
// through L2.
template <int L, int V, int ST, int MODE>
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
  constexpr int es = (ST == kBF16) ? 2 : 4;
  constexpr int n_in = (MODE == kInnovation) ? 2 : 1;   // u, and e when the perturbations are given
  const uint32_t round_bytes = (uint32_t)LPC * nx * es;
  float2* lines = reinterpret_cast<float2*>(smraw);
  unsigned char* stage = smraw + (((size_t)p.R * pitch * sizeof(float2) + 127) & ~(size_t)127);
  uint64_t* bar = reinterpret_cast<uint64_t*>(stage + (size_t)n_in * round_bytes);
  int* flag = reinterpret_cast<int*>(bar + 1);
  static_assert(MODE != kAnomaly, "anomaly rows: row_anom_kernel");
  const long long Q = (long long)p.n_obs * p.n_tiles * p.N;
  const char* ens = reinterpret_cast<const char*>(p.ens);
  const char* pert = reinterpret_cast<const char*>(p.pert);

  auto issue = [&](long long q, int r) {
    const RowTile w = decode_tile(q, p.N, p.n_tiles);
    const size_t row0 = (size_t)w.tile * p.R + (size_t)r * LPC;
    int blk = w.jb;                 // the jb-th observed block
#pragma unroll
    for (int i = 0; i < kMaxObs; ++i)   // constant indices: the parameter array stays in the constant bank
      if (i == w.jb) blk = p.obs[i];
    const size_t fu = (size_t)blk * p.N + w.k;
    mbar_arrive_expect_tx(bar, n_in * round_bytes);
    bulk_g2s(stage, ens + (fu * G + row0 * nx) * es, round_bytes, bar);
    if constexpr (MODE == kInnovation) {
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
  bool expire = p.expire_first_wait != 0;   // test setting: the CTA's first wait gives up
  for (; q < Q; q += gridDim.x) {
    const RowTile w = decode_tile(q, p.N, p.n_tiles);
    const int y0 = w.tile * p.R;
    const size_t f = (size_t)w.k * p.n_obs + w.jb;
    const float* shared_in = p.data + (size_t)w.jb * G;
    for (int r = 0; r < rounds; ++r) {
      const int row = r * LPC + g;
      const float* sh = shared_in + (size_t)(y0 + row) * nx;
      float2 sv[V];
#pragma unroll
      for (int m = 0; m < V; ++m) sv[m] = __ldg(reinterpret_cast<const float2*>(sh) + t + T * m);
      if (!cta_wait(bar, phase, p.status, flag, expire)) return;
      expire = false;
      phase ^= 1;
      float2 v[V];
      const unsigned char* st_row = stage + (size_t)g * nx * es;
#pragma unroll
      for (int m = 0; m < V; ++m) {
        const size_t idx = 2 * (size_t)(t + T * m);
        const float2 a = load2<ST>(st_row, idx);
        if constexpr (MODE == kInnovation) {
          const float2 ee = load2<ST>(st_row + round_bytes, idx);
          // w = (d - u) + e: d - u first, exact when d and u are close (large common mean)
          v[m] = make_float2((sv[m].x - a.x) + ee.x, (sv[m].y - a.y) + ee.y);
        } else {
          v[m] = make_float2(sv[m].x - a.x, sv[m].y - a.y);
        }
      }
      __syncthreads();   // stage consumed
      if (threadIdx.x == 0) {
        if (r + 1 < rounds) issue(q, r + 1);
        else if (q + gridDim.x < Q) issue(q + gridDim.x, 0);
      }
      float2* line = lines + row * pitch;
      fft_line<L, V, false>(v, line, t, p.twL, line_bar<T>(g));
#pragma unroll
      for (int m = 0; m < V; ++m) line[pidx(t + T * m)] = v[m];
    }
    __syncthreads();
    row_twist_store<L>(lines, p.out + f * (size_t)L * p.ny, p.R, p.ny, y0, p.twX);
    __syncthreads();
  }
}

// Anomaly rows with the first member as pivot.  A work item is R rows of one block j; the CTA
// takes its members k = 1..N-1 in turn (rounds of LPC rows each, the next round's rows bulk
// copied while the current one is transformed), transforms d_k = u_k - u_0 into field j*N+k, and
// keeps the running sum of the d_k of its rows: thread (g, t) the 2V values of each round, in
// tm_cols tensor-memory columns of its lane -- or, for CTAs that are not whole warps (short
// rows; tm_alloc == 0), in a shared-memory slot of tm_cols floats.  A last step transforms that
// sum times 1/sqrt(N) into field j*N+0.  The pivot rows are read from global memory (L1/L2)
// next to every round.
template <int L, int V, int ST>
__global__ void __launch_bounds__(512, 1) row_anom_kernel(const RowFwdParams p) {
  constexpr int T = L / V;
  constexpr int pitch = row_pitch(L);
  static_assert((2 * V) % 8 == 0, "tensor-memory runs of 8 columns");
  extern __shared__ __align__(128) unsigned char smraw[];
  const int LPC = blockDim.x / T;
  const int rounds = p.R / LPC;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int nx = p.nx, N = p.N;
  const size_t G = (size_t)p.ny * nx;
  constexpr int es = (ST == kBF16) ? 2 : 4;
  const uint32_t round_bytes = (uint32_t)LPC * nx * es;
  float2* lines = reinterpret_cast<float2*>(smraw);
  unsigned char* stage = smraw + (((size_t)p.R * pitch * sizeof(float2) + 127) & ~(size_t)127);
  uint64_t* bar = reinterpret_cast<uint64_t*>(stage + round_bytes);
  int* flag = reinterpret_cast<int*>(bar + 1);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(flag + 1);
  const bool in_tm = p.tm_alloc != 0;
  float* ssum = reinterpret_cast<float*>(tslot + 1) + (size_t)threadIdx.x * p.tm_cols;   // !in_tm
  const long long Q = (long long)p.M * p.n_tiles;   // item q: block q / n_tiles, tile q mod n_tiles
  const int steps = (N - 1) * rounds;              // copy unit s of an item: member 1 + s / rounds, round s mod rounds
  const char* ens = reinterpret_cast<const char*>(p.ens);

  auto issue = [&](long long q, int s) {
    const int jb = (int)(q / p.n_tiles);
    const int tile = (int)(q - (long long)jb * p.n_tiles);
    const int k = 1 + s / rounds, r = s - (s / rounds) * rounds;
    const size_t row0 = (size_t)tile * p.R + (size_t)r * LPC;
    mbar_arrive_expect_tx(bar, round_bytes);
    bulk_g2s(stage, ens + (((size_t)jb * N + k) * G + row0 * nx) * es, round_bytes, bar);
  };

  if (in_tm && (threadIdx.x >> 5) == 0) tm_alloc(tslot, (uint32_t)p.tm_alloc);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  if (in_tm) tm_fence_before_sync();
  __syncthreads();
  if (in_tm) tm_fence_after_sync();
  const uint32_t ta = in_tm ? tm_addr(*tslot, (threadIdx.x >> 7) * p.tm_cols) : 0u;
  auto sum_load = [&](int r, float* acc) {
    if (in_tm) {
      tm_wait_st();   // this thread's earlier stores
      tm_ld<2 * V>(ta + (uint32_t)(r * 2 * V), acc);
    } else {
#pragma unroll
      for (int i = 0; i < 2 * V; ++i) acc[i] = ssum[r * 2 * V + i];
    }
  };
  auto sum_store = [&](int r, const float* acc) {
    if (in_tm) {
      tm_st<2 * V>(ta + (uint32_t)(r * 2 * V), acc);
    } else {
#pragma unroll
      for (int i = 0; i < 2 * V; ++i) ssum[r * 2 * V + i] = acc[i];
    }
  };

  uint32_t phase = 0;
  long long q = blockIdx.x;
  if (threadIdx.x == 0 && q < Q) issue(q, 0);
  bool expire = p.expire_first_wait != 0;   // test setting: the CTA's first wait gives up
  bool alive = true;
  for (; q < Q && alive; q += gridDim.x) {
    const int jb = (int)(q / p.n_tiles);
    const int y0 = (int)(q - (long long)jb * p.n_tiles) * p.R;
    const char* piv = ens + (size_t)jb * N * G * es;   // member 0 of block j
    for (int k = 1; k <= N && alive; ++k) {   // k == N: the scaled sum, written as member 0
      for (int r = 0; r < rounds; ++r) {
        const int row = r * LPC + g;
        float2 v[V];
        if (k < N) {
          float2 sv[V];
          const char* prow = piv + (size_t)(y0 + row) * nx * es;
#pragma unroll
          for (int m = 0; m < V; ++m) sv[m] = load2<ST>(prow, 2 * (size_t)(t + T * m));
          if (!cta_wait(bar, phase, p.status, flag, expire)) {
            alive = false;
            break;
          }
          expire = false;
          phase ^= 1;
          const unsigned char* st_row = stage + (size_t)g * nx * es;
#pragma unroll
          for (int m = 0; m < V; ++m) {
            const float2 a = load2<ST>(st_row, 2 * (size_t)(t + T * m));
            v[m] = make_float2(a.x - sv[m].x, a.y - sv[m].y);
          }
          __syncthreads();   // stage consumed
          if (threadIdx.x == 0) {
            const int s = (k - 1) * rounds + r + 1;
            if (s < steps) issue(q, s);
            else if (q + gridDim.x < Q) issue(q + gridDim.x, 0);
          }
          float acc[2 * V];
          if (k == 1) {
#pragma unroll
            for (int m = 0; m < V; ++m) {
              acc[2 * m] = v[m].x;
              acc[2 * m + 1] = v[m].y;
            }
          } else {
            sum_load(r, acc);   // the sums stored for the previous member
#pragma unroll
            for (int m = 0; m < V; ++m) {
              acc[2 * m] += v[m].x;
              acc[2 * m + 1] += v[m].y;
            }
          }
          sum_store(r, acc);
        } else {
          float acc[2 * V];
          sum_load(r, acc);
#pragma unroll
          for (int m = 0; m < V; ++m) v[m] = make_float2(acc[2 * m] * p.inv_sqrt_N, acc[2 * m + 1] * p.inv_sqrt_N);
        }
        float2* line = lines + row * pitch;
        fft_line<L, V, false>(v, line, t, p.twL, line_bar<T>(g));
#pragma unroll
        for (int m = 0; m < V; ++m) line[pidx(t + T * m)] = v[m];
      }
      if (!alive) break;
      __syncthreads();
      const size_t f = (size_t)jb * N + (k < N ? k : 0);
      row_twist_store<L>(lines, p.out + f * (size_t)L * p.ny, p.R, p.ny, y0, p.twX);
      __syncthreads();
    }
  }
  if (in_tm) {
    tm_wait_st();
    tm_fence_before_sync();
  }
  __syncthreads();
  if (in_tm && (threadIdx.x >> 5) == 0) tm_dealloc(*tslot, (uint32_t)p.tm_alloc);
}

// Inverse row pass.  A work item is R rows of one field (R = the rows the CTA
// transforms at once); its increment spectra (R consecutive k_y of every column of
// the column-major row spectra) arrive as a tile [L][R] by tensor copies while the
// previous item is transformed, and its forecast rows by one bulk copy into a
// stage.  The inverse real-FFT twist runs cooperatively over the tile, a pair of
// columns c, L - c per step, and stages each row in its padded line buffer, which
// then serves as that row's FFT exchange buffer.
template <int L, int V, int ST>
__global__ void __launch_bounds__(512, 1) row_inv_kernel(const __grid_constant__ RowInvParams p) {
  constexpr int T = L / V;
  constexpr int pitch = row_pitch(L);
  extern __shared__ __align__(128) unsigned char smraw[];
  const int R = p.R;                 // a power of two
  const int rs = __ffs(R) - 1;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int nx = p.nx;
  const size_t G = (size_t)p.ny * nx;
  constexpr int es = (ST == kBF16) ? 2 : 4;
  const uint32_t tile_bytes = (uint32_t)L * R * sizeof(float2);
  const uint32_t item_bytes = (uint32_t)R * nx * es;
  float2* tile = reinterpret_cast<float2*>(smraw);
  float2* lines = reinterpret_cast<float2*>(smraw + ((tile_bytes + 127) & ~127u));
  unsigned char* stage = reinterpret_cast<unsigned char*>(lines) + (((size_t)R * pitch * sizeof(float2) + 127) & ~(size_t)127);
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage + item_bytes);   // [0] tile, [1] forecast rows
  int* flag = reinterpret_cast<int*>(bars + 2);
  const long long Q = (long long)p.M * p.N * p.n_tiles;   // item q = field q / n_tiles, tile q mod n_tiles
  char* ens = reinterpret_cast<char*>(p.ens);

  auto issue_tile = [&](long long q) {   // R k_y of every column of item q's field -> tile [L][R]
    const int f = (int)(q / p.n_tiles);
    const int y0 = (int)(q - (long long)f * p.n_tiles) * R;
    mbar_arrive_expect_tx(&bars[0], tile_bytes);
    for (int cb = 0; cb < L; cb += p.box_cols) tensor_load_3d(tile + (size_t)cb * R, &p.tm_in, 2 * y0, cb, f, &bars[0]);
  };
  auto issue_rows = [&](long long q) {
    const size_t f = q / p.n_tiles;
    const size_t row0 = (size_t)(q - (long long)f * p.n_tiles) * R;
    mbar_arrive_expect_tx(&bars[1], item_bytes);
    bulk_g2s(stage, ens + (f * G + row0 * nx) * es, item_bytes, &bars[1]);
  };

  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t tph = 0, rph = 0;
  long long q = blockIdx.x;
  if (threadIdx.x == 0 && q < Q) {
    issue_tile(q);
    issue_rows(q);
  }
  for (; q < Q; q += gridDim.x) {
    const size_t f = q / p.n_tiles;
    const int y0 = (int)(q - (long long)f * p.n_tiles) * R;
    if (!cta_wait(&bars[0], tph, p.status, flag)) {
      if (threadIdx.x == 0) mbar_wait_bounded(&bars[1], rph);   // forecast copy may be landing
      return;
    }
    tph ^= 1;
    // inverse twist: from X[c], X[L-c] of a row, z[c] = A + i B conj(W^c) and
    // z[L-c] = conj(A - i B conj(W^c)), A = X[c] + conj X[L-c], B = X[c] - conj X[L-c]
    for (int i = threadIdx.x; i < (L / 2 + 1) * R; i += blockDim.x) {
      const int c = i >> rs, r = i & (R - 1);
      float2* line = lines + (size_t)r * pitch;
      const float2 X = tile[c * R + r];
      if (c == 0) {   // packed X[0] + i X[L]
        line[pidx(0)] = make_float2(X.x + X.y, X.x - X.y);
        continue;
      }
      const float2 Xm = tile[(L - c) * R + r];
      const float2 A = make_float2(X.x + Xm.x, X.y - Xm.y);
      const float2 B = make_float2(X.x - Xm.x, X.y + Xm.y);
      const float2 Bw = cmulc(B, __ldg(p.twX + c));
      line[pidx(c)] = make_float2(A.x - Bw.y, A.y + Bw.x);
      if (c != L - c) line[pidx(L - c)] = make_float2(A.x + Bw.y, Bw.x - A.y);
    }
    __syncthreads();   // tile consumed, rows staged
    if (threadIdx.x == 0 && q + gridDim.x < Q) issue_tile(q + gridDim.x);
    float2* line = lines + (size_t)g * pitch;
    float2 v[V];
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = line[pidx(t + T * m)];
    line_sync<T>(line_bar<T>(g));   // the row is read before the FFT reuses its buffer
    fft_line<L, V, true, false>(v, line, t, p.twL, line_bar<T>(g));   // the buffer is next written after the waits below
    if (!cta_wait(&bars[1], rph, p.status, flag)) {
      if (threadIdx.x == 0) mbar_wait_bounded(&bars[0], tph);   // next tile may be landing
      return;
    }
    rph ^= 1;
    const unsigned char* st_row = stage + (size_t)g * nx * es;
    float2 a[V];
#pragma unroll
    for (int m = 0; m < V; ++m) a[m] = load2<ST>(st_row, 2 * (size_t)(t + T * m));
    __syncthreads();   // stage consumed
    if (threadIdx.x == 0 && q + gridDim.x < Q) issue_rows(q + gridDim.x);
    char* urow = ens + (f * G + (size_t)(y0 + g) * nx) * es;
#pragma unroll
    for (int m = 0; m < V; ++m)
      store2<ST>(urow, 2 * (size_t)(t + T * m), make_float2(a[m].x + v[m].x, a[m].y + v[m].y));
  }
}

// ----------------------------------------------------------------- launch

struct RowShape {
  int T, R, LPC;
  size_t smem;
};

// rows per tile R (a power of two dividing ny), rows per round LPC, and the
// shared memory: R staged rows plus one round of n_in input rows.  The half
// schedule halves both, so that two CTAs of half the threads share an SM.
inline RowShape row_shape(int L, int V, int ny, int nx, int es, int n_in, bool half) {
  RowShape s;
  s.T = L / V;
  const int pow2 = ny & -ny;
  int R = 256 / s.T;
  if (R < 8) R = 8;
  if (R > pow2) R = pow2;
  if (half && R > 2) R >>= 1;
  for (;;) {
    int LPC = (half ? 256 : 512) / s.T;
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

// Anomaly rows: the row shape of row_shape, with R halved (down to one round) until the running
// sums fit the tensor memory: rounds x 2V columns per thread, threads 128 apart sharing a lane.
template <int L, int V, int ST>
cudaError_t row_anom_LV(RowFwdParams p, cudaStream_t st) {
  constexpr int es = ST == kBF16 ? 2 : 4;
  RowShape s = row_shape(L, V, p.ny, p.nx, es, 1, (p.vsel & 2) != 0);
  const int threads = s.T * s.LPC;
  const int share = (threads + 127) / 128;
  const bool in_tm = threads % 32 == 0;   // tensor-memory loads and stores take whole warps
  int alloc = 0;
  for (;;) {
    p.tm_cols = (s.R / s.LPC) * 2 * V;
    alloc = 32;
    while (alloc < share * p.tm_cols) alloc <<= 1;
    if (!in_tm || alloc <= 512 || s.R <= s.LPC) break;
    s.R >>= 1;
  }
  s.smem = (((size_t)s.R * row_pitch(L) * sizeof(float2) + 127) & ~(size_t)127) + (size_t)s.LPC * p.nx * es + 16;
  if (!in_tm) s.smem += (size_t)threads * p.tm_cols * sizeof(float);
  if ((in_tm && alloc > 512) || s.smem > 227 * 1024 || s.R < 2) return cudaErrorInvalidConfiguration;
  p.tm_alloc = in_tm ? alloc : 0;
  p.R = s.R;
  p.n_tiles = p.ny / s.R;
  p.inv_sqrt_N = (float)(1.0 / std::sqrt((double)p.N));
  auto kern = row_anom_kernel<L, V, ST>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, s.smem);
  if (in_tm && per_sm > 512 / alloc) per_sm = 512 / alloc;   // co-resident CTAs never wait for tensor memory
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)p.M * p.n_tiles;
  const long long cap = (long long)sm_count() * per_sm;
  if (grid > cap) grid = cap;
  kern<<<(unsigned)grid, threads, s.smem, st>>>(p);
  return cudaGetLastError();
}

template <int L, int V, int ST, int MODE>
cudaError_t row_fwd_LV(RowFwdParams p, int n_fields, cudaStream_t st) {
  constexpr int es = ST == kBF16 ? 2 : 4;
  RowShape s = row_shape(L, V, p.ny, p.nx, es, MODE == kInnovation ? 2 : 1, (p.vsel & 2) != 0);
  if (s.smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  p.R = s.R;
  p.n_tiles = p.ny / s.R;
  auto kern = row_fwd_kernel<L, V, ST, MODE>;
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

// rows per item of the inverse pass: the rows one CTA of at most 512 threads transforms at
// once (a power of two dividing ny), halved while the tile, the row buffers and the stage
// exceed 220 KB, and once more for the half schedule
inline RowShape inv_shape(int L, int V, int ny, int nx, int es, bool half) {
  RowShape s;
  s.T = L / V;
  const int pow2 = ny & -ny;
  int R = 512 / s.T;
  if (R < 1) R = 1;
  if (R > pow2) R = pow2;
  if (R > 128) R = 128;   // a tensor copy's box rows (2 R floats) are at most 256
  auto smem = [&](int r) {
    return (((size_t)L * r * sizeof(float2) + 127) & ~(size_t)127) +
           (((size_t)r * row_pitch(L) * sizeof(float2) + 127) & ~(size_t)127) + (size_t)r * nx * es + 32;
  };
  while (R > 2 && smem(R) > 220 * 1024) R >>= 1;
  if (half && R > 2) R >>= 1;
  s.R = R;
  s.LPC = R;
  s.smem = smem(R);
  return s;
}

template <int L, int V, int ST>
cudaError_t row_inv_LV(RowInvParams p, int n_fields, cudaStream_t st) {
  constexpr int es = ST == kBF16 ? 2 : 4;
  RowShape s = inv_shape(L, V, p.ny, p.nx, es, (p.vsel & 2) != 0);
  if (s.R != p.R || s.smem > 227 * 1024 || s.T * s.R > 512) return cudaErrorInvalidConfiguration;
  p.n_tiles = p.ny / s.R;
  auto kern = row_inv_kernel<L, V, ST>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, s.T * s.R, s.smem);
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)n_fields * p.n_tiles;
  const long long cap = (long long)sm_count() * per_sm;
  if (grid > cap) grid = cap;
  kern<<<(unsigned)grid, s.T * s.R, s.smem, st>>>(p);
  return cudaGetLastError();
}

template <int L, int ST>
cudaError_t row_fwd_L(const RowFwdParams& p, int n_fields, cudaStream_t st) {
  if (p.mode == kAnomaly) {
    if (p.vsel & 1) return row_anom_LV<L, plan_V(L, 1), ST>(p, st);
    return row_anom_LV<L, plan_V(L, 0), ST>(p, st);
  }
  if (p.mode == kInnovationDrawn) {
    if (p.vsel & 1) return row_fwd_LV<L, plan_V(L, 1), ST, kInnovationDrawn>(p, n_fields, st);
    return row_fwd_LV<L, plan_V(L, 0), ST, kInnovationDrawn>(p, n_fields, st);
  }
  if (p.vsel & 1) return row_fwd_LV<L, plan_V(L, 1), ST, kInnovation>(p, n_fields, st);
  return row_fwd_LV<L, plan_V(L, 0), ST, kInnovation>(p, n_fields, st);
}

template <int L, int ST>
cudaError_t row_inv_L(const RowInvParams& p, int n_fields, cudaStream_t st) {
  if (p.vsel & 1) return row_inv_LV<L, plan_V(L, 1), ST>(p, n_fields, st);
  return row_inv_LV<L, plan_V(L, 0), ST>(p, n_fields, st);
}

// the launchers of one storage type (one translation unit each)
template <int ST>
cudaError_t launch_row_fwd_st(const RowFwdParams& p, int n_fields, cudaStream_t s) {
  switch (p.L) {
#define CASE(n) case n: return row_fwd_L<n, ST>(p, n_fields, s);
    FFTENKF_ROW_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

template <int ST>
cudaError_t launch_row_inv_st(const RowInvParams& p, int n_fields, cudaStream_t s) {
  switch (p.L) {
#define CASE(n) case n: return row_inv_L<n, ST>(p, n_fields, s);
    FFTENKF_ROW_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_row_fwd_bf16(const RowFwdParams& p, int n_fields, cudaStream_t s);
cudaError_t launch_row_fwd_f32(const RowFwdParams& p, int n_fields, cudaStream_t s);
cudaError_t launch_row_inv_bf16(const RowInvParams& p, int n_fields, cudaStream_t s);
cudaError_t launch_row_inv_f32(const RowInvParams& p, int n_fields, cudaStream_t s);

}  // namespace fftenkf
