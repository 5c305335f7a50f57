// Fused column pass: the second half of the 2-D transforms, the spectral
// covariance, the gains and the update of eq. (dii), (cov-multi-spectral) and
// (spectral-multi-enkf), one wavenumber column k_x per thread group.
//
// For its column a group
//   1. transforms the column of every member's anomaly row spectrum and
//      accumulates chat^(oo) = sum_k |ahat^(o)|^2 and chat^(jo) =
//      sum_k ahat^(j) conj(ahat^(o)) (eq. dii, eq. cov-multi-spectral);
//   2. turns the sums into the gains G^(oo) = chat^(oo) / (chat^(oo) + rhat_o)
//      and G^(jo) = chat^(jo) / (chat^(oo) + rhat_o) (eq. spectral-multi-enkf),
//      or writes the covariance tables when only the spectrum is estimated;
//   3. for every member transforms the innovation columns, forms
//      S^(j) = sum_o G^(jo) what_o for every block and applies the inverse
//      column transform, writing the increment's row spectra.
// The per-wavenumber sums and gains of the column (10 floats per wavenumber for
// 4 blocks, 2 observed: 160 KB at 4096 rows) live in tensor memory, each thread
// keeping those of the wavenumbers it transforms; nothing of them goes through
// shared memory or HBM.  Blocks are taken in role order (observed first) two at
// a time, and each pair of lines is transformed at once in paired FP32
// (fft_pair.cuh); the observed pair (or the observed block and its partner) is
// transformed first, so the cross terms of every later pair find it in
// tensor memory.  Lines arrive by bulk copies into two stage slots, one unit (two
// lines) ahead; once a unit's lines are read, its slot is the second exchange
// buffer of that unit's transforms, which alternate between it and the group's
// exchange buffer and so take one barrier per exchange.  Every group has its own
// slots, barriers and column sequence, so the groups of a CTA never wait for one
// another.
#pragma once
#include "common.cuh"
#include "fft_pair.cuh"
#include "perturb.cuh"
#include "tma.cuh"
#include "tmem.cuh"

namespace fftenkf {

template <int NY, int V>
struct ColFusedShape {
  static constexpr int T = NY / V;
  static constexpr int PL = (pair_padded_len(NY, V) + 7) & ~7;           // 16-byte exchange slots
  static constexpr size_t stage_bytes = (size_t)2 * NY * sizeof(float2);   // one unit: two lines
  // a stage slot also serves as the second exchange buffer once its unit is read
  static constexpr size_t slot_bytes =
      ((stage_bytes > (size_t)PL * 16 ? stage_bytes : (size_t)PL * 16) + 127) & ~(size_t)127;
  static constexpr size_t group_bytes = ((2 * slot_bytes + (size_t)PL * 16 + 32) + 127) & ~(size_t)127;
};

// tensor-memory columns of one thread when a CTA of `threads` threads shares the 128 lanes x
// 512 columns (threads 128 apart share a lane), a multiple of 8
__host__ __device__ constexpr int fused_cols_per_thread(int threads) {
  return (512 / ((threads + 127) / 128)) & ~7;
}

// the two lines of a unit as pairs; part 1 / 2: the real DC (.x) or Nyquist (.y) column
template <int NY, int V>
__device__ __forceinline__ void read_pair(cp (&v)[V], const float2* __restrict__ l0, const float2* __restrict__ l1,
                                          bool has1, int t, int part) {
  constexpr int T = NY / V;
  const float2 z = make_float2(0.f, 0.f);
  if (part == 0) {
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = cp_of(l0[t + T * m], has1 ? l1[t + T * m] : z);
  } else if (part == 1) {
#pragma unroll
    for (int m = 0; m < V; ++m)
      v[m] = cp_of(make_float2(l0[t + T * m].x, 0.f), make_float2(has1 ? l1[t + T * m].x : 0.f, 0.f));
  } else {
#pragma unroll
    for (int m = 0; m < V; ++m)
      v[m] = cp_of(make_float2(l0[t + T * m].y, 0.f), make_float2(has1 ? l1[t + T * m].y : 0.f, 0.f));
  }
}

template <int H>
__device__ __forceinline__ float2 half_of(const cp& v) {
  return H == 0 ? make_float2(v.re.x, v.im.x) : make_float2(v.re.y, v.im.y);
}
template <int H>
__device__ __forceinline__ void set_half(cp& v, float2 x) {
  if (H == 0) {
    v.re.x = x.x;
    v.im.x = x.y;
  } else {
    v.re.y = x.x;
    v.im.y = x.y;
  }
}

// Both halves of a pair, (re, im) interleaved per wavenumber, into the tensor-memory
// columns at at: half h at at + 2 V h.
template <int V>
__device__ __forceinline__ void store_halves(const cp (&v)[V], uint32_t at) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int m0 = 0; m0 < V; m0 += 8) {
      float a[16];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float2 x = h ? half_of<1>(v[m0 + q]) : half_of<0>(v[m0 + q]);
        a[2 * q] = x.x;
        a[2 * q + 1] = x.y;
      }
      tm_st16(at + 2 * V * h + 2 * m0, a);
    }
  }
}

// Statistics of one transformed pair (roles 2pp, 2pp+1) into the tensor-memory sums at ta:
// auto sums of observed role i at columns [i V, i V + V), cross sums of unobserved u with
// observed i at XB + (u n_obs + i) 2V, interleaved (re, im) per wavenumber.  The observed
// spectra of the member (half i of its first pair) are at KB + 2 V i.  sg = -1 subtracts the
// products (the pivot sum in the place of member 0), +1 adds them.
template <int V, int NOBS>
__device__ __forceinline__ void fused_accumulate(const cp (&v)[V], int pp, int M, int n_obs, uint32_t ta, int KB,
                                                 float sg) {
  const int XB = n_obs * V;
  tm_wait_st();   // the sums (and the member's spectra) stored by earlier units
  if (2 * pp + 1 < n_obs) {   // both roles observed: their auto sums are adjacent, one load
    float a[2 * V];
    tm_ld<2 * V>(ta + 2 * pp * V, a);
#pragma unroll
    for (int m = 0; m < V; ++m) {
      const float2 x0 = half_of<0>(v[m]), x1 = half_of<1>(v[m]);
      a[m] = fmaf(sg * x0.x, x0.x, fmaf(sg * x0.y, x0.y, a[m]));
      a[V + m] = fmaf(sg * x1.x, x1.x, fmaf(sg * x1.y, x1.y, a[V + m]));
    }
    tm_st<2 * V>(ta + 2 * pp * V, a);
    return;
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = 2 * pp + h;
    if (r >= M) continue;
    if (r < n_obs) {
      float a[V];
      tm_ld<V>(ta + r * V, a);
#pragma unroll
      for (int m = 0; m < V; ++m) {
        const float2 x = h ? half_of<1>(v[m]) : half_of<0>(v[m]);
        a[m] = fmaf(sg * x.x, x.x, fmaf(sg * x.y, x.y, a[m]));
      }
      tm_st<V>(ta + r * V, a);
    } else {
      const int u = r - n_obs;
#pragma unroll
      for (int i = 0; i < NOBS; ++i) {
        if (i >= n_obs) continue;
        const uint32_t at = ta + XB + (u * n_obs + i) * 2 * V;
        float a[2 * V], o[2 * V];
        tm_ld2<2 * V, 2 * V>(at, a, ta + KB + 2 * V * i, o);
#pragma unroll
        for (int m = 0; m < V; ++m) {   // += sg x conj(o)
          float2 x = h ? half_of<1>(v[m]) : half_of<0>(v[m]);
          x = make_float2(sg * x.x, sg * x.y);
          a[2 * m] = fmaf(x.x, o[2 * m], fmaf(x.y, o[2 * m + 1], a[2 * m]));
          a[2 * m + 1] = fmaf(x.y, o[2 * m], fmaf(-x.x, o[2 * m + 1], a[2 * m + 1]));
        }
        tm_st<2 * V>(at, a);
      }
    }
  }
}

// Sums -> gains in place (analysis), or -> covariance tables in global memory (statistics
// only), for the wavenumbers (t + T m, column c) of this thread.  The denominator
// chat^(oo) + rhat is formed in FP64 and rounded once; the quotients are FP32, or FP64 where
// the rounded denominator is below FLT_MIN (0 where it is exactly 0, as in the oracle).  With
// the pivot form chat^(oo) can come out a few rounding errors below 0 where the ensemble has
// no variance above FFT round-off; with rhat = 0 such a wavenumber keeps the gain 1 of
// chat / chat.  Returns false if a sum is not finite.
template <int NY, int V, int NOBS>
__device__ __forceinline__ bool fused_gains(const ColFusedParams& p, uint32_t ta, int c, int t) {
  constexpr int T = NY / V;
  const int XB = p.n_obs * V;
  const size_t tab = (size_t)(p.L + 1) * NY;
  const bool stats_only = (p.W == nullptr);
  float2* xout = stats_only ? reinterpret_cast<float2*>(p.chat + p.n_obs * tab) : nullptr;
  bool ok = true;
  tm_wait_st();
#pragma unroll 1
  for (int i = 0; i < NOBS; ++i) {
    if (i >= p.n_obs) break;
    float a[V];
    tm_ld<V>(ta + i * V, a);
    float val[V], inv[V];
    double rr[V];
    unsigned tiny = 0;
#pragma unroll
    for (int m = 0; m < V; ++m) {
      val[m] = a[m] * p.scale;
      ok &= isfinite(val[m]);
    }
    if (stats_only) {
#pragma unroll
      for (int m = 0; m < V; ++m) p.chat[i * tab + (size_t)c * NY + t + T * m] = val[m];
    } else {
#pragma unroll
      for (int m = 0; m < V; ++m) rr[m] = __ldg(p.rhat_t + i * tab + (size_t)c * NY + t + T * m);
#pragma unroll
      for (int m = 0; m < V; ++m) {
        const double den = (double)val[m] + rr[m];
        const float denf = (float)den;
        if (denf >= 1.17549435e-38f) {
          inv[m] = __fdividef(p.inv_G, denf);
          a[m] = val[m] * inv[m];
        } else {
          tiny |= 1u << m;
          const double rd = (den != 0.0) ? (double)p.inv_G / den : 0.0;
          inv[m] = 0.f;
          a[m] = (float)((double)val[m] * rd);
        }
      }
      tm_st<V>(ta + i * V, a);
    }
#pragma unroll 1
    for (int u = 0; u < p.n_un; ++u) {
      float x[2 * V];
      const uint32_t at = ta + XB + (u * p.n_obs + i) * 2 * V;
      tm_ld<2 * V>(at, x);
#pragma unroll
      for (int m = 0; m < V; ++m) {
        const float xr = x[2 * m] * p.scale, xi = x[2 * m + 1] * p.scale;
        ok &= isfinite(xr) && isfinite(xi);
        if (stats_only) {
          xout[(size_t)(i * p.n_un + u) * tab + (size_t)c * NY + t + T * m] = make_float2(xr, xi);
        } else if (tiny & (1u << m)) {
          const double den = (double)val[m] + rr[m];
          const double rd = (den != 0.0) ? (double)p.inv_G / den : 0.0;
          x[2 * m] = (float)((double)xr * rd);
          x[2 * m + 1] = (float)((double)xi * rd);
        } else {
          x[2 * m] = xr * inv[m];
          x[2 * m + 1] = xi * inv[m];
        }
      }
      if (!stats_only) tm_st<2 * V>(at, x);
    }
  }
  return ok;
}

// S for the target pair (roles 2tp, 2tp+1) of one member from its innovation spectra, held
// in tensor memory at KB (half i: observed block i)
template <int V, int NOBS>
__device__ __forceinline__ void fused_targets(cp (&s)[V], int tp, int M, int n_obs, uint32_t ta, int KB) {
  const int XB = n_obs * V;
  tm_wait_st();   // the member's innovation spectra
#pragma unroll
  for (int m = 0; m < V; ++m) s[m] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = 2 * tp + h;
    if (r >= M) continue;
    if (r < n_obs) {   // an observed block: its own innovation times G^(oo)
      float gv[V], x[2 * V];
      tm_ld2<V, 2 * V>(ta + r * V, gv, ta + KB + 2 * V * r, x);
#pragma unroll
      for (int m = 0; m < V; ++m) {
        const float2 y = make_float2(gv[m] * x[2 * m], gv[m] * x[2 * m + 1]);
        if (h) set_half<1>(s[m], y); else set_half<0>(s[m], y);
      }
    } else {           // an unobserved block: sum over observed i of G^(ji) what_i, into s
      const int u = r - n_obs;
#pragma unroll
      for (int i = 0; i < NOBS; ++i) {
        if (i >= n_obs) continue;
        float gx[2 * V], x[2 * V];
        tm_ld2<2 * V, 2 * V>(ta + XB + (u * n_obs + i) * 2 * V, gx, ta + KB + 2 * V * i, x);
#pragma unroll
        for (int m = 0; m < V; ++m) {
          float2 acc = h ? half_of<1>(s[m]) : half_of<0>(s[m]);
          acc.x = fmaf(gx[2 * m], x[2 * m], fmaf(-gx[2 * m + 1], x[2 * m + 1], acc.x));
          acc.y = fmaf(gx[2 * m], x[2 * m + 1], fmaf(gx[2 * m + 1], x[2 * m], acc.y));
          if (h) set_half<1>(s[m], acc); else set_half<0>(s[m], acc);
        }
      }
    }
  }
}

// Perturbations drawn in frequency space added to the innovation spectra of member k (seeded
// analysis): half i of w gets amp_i(k_y, c) zhat_{k,i}(k_y, c), zhat from Philox4x32-10 counters and
// Box-Muller (perturb.cuh), on the same counter layout as the separate column update.
template <int NY, int V, int NOBS>
__device__ __forceinline__ void fused_add_drawn(cp (&w)[V], const ColFusedParams& p, int k, int c, int t) {
  constexpr int T = NY / V;
  const size_t tab = (size_t)(p.L + 1) * NY;
#pragma unroll
  for (int i = 0; i < NOBS; ++i) {
    if (i >= p.n_obs) continue;
    const int stream = k * p.n_obs + i;
    const float* amp = p.amp_t + (size_t)i * tab + (size_t)c * NY + t;
    if (c != 0 && c != p.L) {
      // one generator call serves k_y (words 0, 1) and k_y + ny/2 (words 2, 3): slots m and m + V/2
      const float h = 0.70710678118654752f;
#pragma unroll
      for (int m = 0; m < V / 2; ++m) {
        const uint4 w4 = philox4x32_10(make_uint4((uint32_t)(t + T * m), (uint32_t)c, (uint32_t)stream, 0u),
                                       (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
        const float2 zl = box_muller(w4.x, w4.y), zh = box_muller(w4.z, w4.w);
        const float al = h * __ldg(amp + T * m), ah = h * __ldg(amp + T * (m + V / 2));
        float2 a = i ? half_of<1>(w[m]) : half_of<0>(w[m]);
        float2 b = i ? half_of<1>(w[m + V / 2]) : half_of<0>(w[m + V / 2]);
        a = make_float2(fmaf(al, zl.x, a.x), fmaf(al, zl.y, a.y));
        b = make_float2(fmaf(ah, zh.x, b.x), fmaf(ah, zh.y, b.y));
        if (i) { set_half<1>(w[m], a); set_half<1>(w[m + V / 2], b); }
        else { set_half<0>(w[m], a); set_half<0>(w[m + V / 2], b); }
      }
    } else {
#pragma unroll
      for (int m = 0; m < V; ++m) {
        const float am = __ldg(amp + T * m);
        const float2 z = white_edge(p.seed, stream, t + T * m, c, NY);
        float2 a = i ? half_of<1>(w[m]) : half_of<0>(w[m]);
        a = make_float2(fmaf(am, z.x, a.x), fmaf(am, z.y, a.y));
        if (i) set_half<1>(w[m], a); else set_half<0>(w[m], a);
      }
    }
  }
}

// DRAWN: perturbations drawn here (seeded analysis); a separate instantiation, so that the analysis
// with given perturbations carries none of the generator's code
template <int NY, int V, int NOBS, bool DRAWN>
__global__ void __launch_bounds__(V <= 8 ? 512 : 256, 1) col_fused_kernel(const __grid_constant__ ColFusedParams p) {
  using Sh = ColFusedShape<NY, V>;
  constexpr int T = Sh::T;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int LPC = blockDim.x / T;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int bid = (T == 32) ? -1 : 1 + g;
  unsigned char* gb = smraw + (size_t)g * Sh::group_bytes;
  // [2 stage slots][2 lines][NY] (slots of slot_bytes)
  auto slot = [&](int b) { return gb + (size_t)b * Sh::slot_bytes; };
  float4* xbuf = reinterpret_cast<float4*>(gb + 2 * Sh::slot_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gb + 2 * Sh::slot_bytes + (size_t)Sh::PL * 16);
  int* gflag = reinterpret_cast<int*>(bars + 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smraw + (size_t)LPC * Sh::group_bytes);

  if ((threadIdx.x >> 5) == 0) tm_alloc(tslot, 512);
  if (t == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  tm_fence_before_sync();
  __syncthreads();
  tm_fence_after_sync();
  const uint32_t ta = tm_addr(*tslot, (threadIdx.x >> 7) * fused_cols_per_thread(blockDim.x));

  const int M = p.M, N = p.N;
  const int P = (M + 1) / 2;                       // role pairs
  const int units_stats = N * P;
  const int units = units_stats + (p.W ? N : 0);   // + one innovation pair per member
  const int ncol = p.L + 1;
  const size_t fstride = (size_t)p.L * NY;
  const int col_step = gridDim.x * LPC;
  const int nf_cols = p.n_obs * V * (1 + 2 * p.n_un);
  const int KB = nf_cols;   // the member's observed (statistics) or innovation (update) spectra

  // issue side (thread t == 0 of the group): the next (column, unit) to copy
  int ic = blockIdx.x * LPC + g, iu = 0, issued = 0, consumed = 0;
  uint32_t ph0 = 0, ph1 = 0;
  auto issue_next = [&]() {
    if (ic >= ncol) return;
    const int b = issued & 1;
    const int col = (ic == p.L) ? 0 : ic;
    const float2* src0;
    const float2* src1 = nullptr;
    if (iu < units_stats) {
      const int k = iu / P, pp = iu - (iu / P) * P;
      src0 = p.A + ((size_t)p.role_block[2 * pp] * N + k) * fstride + (size_t)col * NY;
      if (2 * pp + 1 < M) src1 = p.A + ((size_t)p.role_block[2 * pp + 1] * N + k) * fstride + (size_t)col * NY;
    } else {
      const int k = iu - units_stats;
      src0 = p.W + ((size_t)k * p.n_obs) * fstride + (size_t)col * NY;
      if (p.n_obs == 2) src1 = p.W + ((size_t)k * p.n_obs + 1) * fstride + (size_t)col * NY;
    }
    float2* dst = reinterpret_cast<float2*>(slot(b));
    mbar_arrive_expect_tx(&bars[b], (uint32_t)((src1 ? 2 : 1) * NY * sizeof(float2)));
    bulk_g2s(dst, src0, NY * sizeof(float2), &bars[b]);
    if (src1) bulk_g2s(dst + NY, src1, NY * sizeof(float2), &bars[b]);
    ++issued;
    if (++iu == units) {
      iu = 0;
      ic += col_step;
    }
  };
  if (t == 0) {
    issue_next();
    issue_next();
  }

  bool alive = true;
  bool bad = false;
  for (int c = blockIdx.x * LPC + g; c < ncol && alive; c += col_step) {
    const int part = (c == 0) ? 1 : ((c == p.L) ? 2 : 0);
    const int col = (c == p.L) ? 0 : c;
    {   // zero the column's sums
      float z[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) z[q] = 0.f;
      for (int q = 0; q < nf_cols; q += 8) tm_st8(ta + q, z);
    }
    for (int u = 0; u < units; ++u) {
      const int b = consumed & 1;
      // the group waits for the unit's copies (thread 0 polls, bounded; the verdict is shared)
      if (t == 0) {
        bool ok = mbar_wait_bounded(&bars[b], b ? ph1 : ph0);
        if (!ok) {
          atomicOr(p.status, kStatusTimeout);
          mbar_wait_bounded(&bars[b], b ? ph1 : ph0);   // let the copies land before leaving
          if (issued - consumed > 1) mbar_wait_bounded(&bars[b ^ 1], b ? ph0 : ph1);
        }
        *gflag = ok ? 1 : 0;
      }
      line_sync<T>(bid);
      if (!*gflag) {
        alive = false;
        break;
      }
      if (b) ph1 ^= 1; else ph0 ^= 1;
      // every thread of the group has left the previous unit (its reads of the other slot,
      // as a stage and as an exchange buffer): that slot takes the next unit's copy
      if (t == 0 && consumed > 0) issue_next();
      const bool stats = u < units_stats;
      const int pp = stats ? u % P : 0;
      const bool has1 = stats ? (2 * pp + 1 < M) : (p.n_obs == 2);
      cp v[V];
      const float2* l0 = reinterpret_cast<const float2*>(slot(b));
      read_pair<NY, V>(v, l0, l0 + NY, has1, t, part);
      ++consumed;
      // the unit's slot, read, is the second exchange buffer: its first write follows the first
      // exchange's barrier, which every thread reaches after read_pair
      float4* xb2 = reinterpret_cast<float4*>(slot(b));
      if (stats) {
        fft_pair2<NY, V, false>(v, xbuf, xb2, t, p.tw, bid);
        if (pp == 0) store_halves<V>(v, ta + KB);
        fused_accumulate<V, NOBS>(v, pp, M, p.n_obs, ta, KB, u < P ? -1.f : 1.f);   // units of member 0 first
        if (u == units_stats - 1) bad |= !fused_gains<NY, V, NOBS>(p, ta, c, t);
      } else {
        const int k = u - units_stats;
        fft_pair2<NY, V, false>(v, xbuf, xb2, t, p.tw, bid);   // what
        if constexpr (DRAWN) fused_add_drawn<NY, V, NOBS>(v, p, k, c, t);
        store_halves<V>(v, ta + KB);
#pragma unroll 1
        for (int tp = 0; tp < P; ++tp) {
          cp s[V];
          fused_targets<V, NOBS>(s, tp, M, p.n_obs, ta, KB);
          fft_pair2<NY, V, true>(s, xbuf, xb2, t, p.tw, bid);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = 2 * tp + h;
            if (r >= M) continue;
            float2* dst = p.S + ((size_t)p.role_block[r] * N + k) * fstride + (size_t)col * NY + t;
            if (part == 0) {
#pragma unroll
              for (int m = 0; m < V; ++m) dst[T * m] = h ? half_of<1>(s[m]) : half_of<0>(s[m]);
            } else {
              float* d1 = reinterpret_cast<float*>(dst) + (part == 1 ? 0 : 1);
#pragma unroll
              for (int m = 0; m < V; ++m) d1[2 * T * m] = h ? s[m].re.y : s[m].re.x;
            }
          }
        }
      }
    }
  }
  if (bad) atomicOr(p.status, kStatusNonFinite);
  tm_wait_st();
  tm_fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tm_dealloc(*tslot, 512);
}

}  // namespace fftenkf

namespace fftenkf {

int sm_count();

// launch shape of the fused pass for ny and schedule sel (V = plan_V(ny, sel); the narrow
// schedule, V = 8, runs twice the threads per column at half the registers): groups per CTA
// (<= 256 or 512 threads, shared memory), dynamic shared memory, tensor-memory columns per
// thread; lpc = 0: unsupported
struct ColFusedLaunch {
  int V, T, lpc;
  size_t smem;
  int cols_per_thread;
};
inline ColFusedLaunch col_fused_launch(int ny, int sel) {
  ColFusedLaunch s{};
  s.V = plan_V(ny, sel);
  s.T = ny / s.V;
  const int max_threads = s.V <= 8 ? 512 : 256;
  if (s.T < 32 || s.T % 32 || s.T > max_threads) return s;
  const size_t pl = (size_t)((pair_padded_len(ny, s.V) + 7) & ~7);
  const size_t stage = (size_t)2 * ny * sizeof(float2);
  const size_t slot = ((stage > pl * 16 ? stage : pl * 16) + 127) & ~(size_t)127;   // as ColFusedShape
  const size_t group = ((2 * slot + pl * 16 + 32) + 127) & ~(size_t)127;
  int lpc = max_threads / s.T;
  while (lpc > 0 && (size_t)lpc * group + 16 > (size_t)227 * 1024) --lpc;
  s.lpc = lpc;
  s.smem = (size_t)lpc * group + 16;
  s.cols_per_thread = fused_cols_per_thread(s.T * lpc);
  return s;
}

template <int NY, int NOBS, int SEL>
inline cudaError_t col_fused_NYS(const ColFusedParams& p, cudaStream_t st) {
  constexpr int V = plan_V(NY, SEL);
  const ColFusedLaunch s = col_fused_launch(NY, SEL);
  if (s.lpc < 1 || s.V != V) return cudaErrorNotSupported;
  auto kern = p.drawn ? col_fused_kernel<NY, V, NOBS, true> : col_fused_kernel<NY, V, NOBS, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  if (e != cudaSuccess) return e;
  const int groups = (p.L + 1 + s.lpc - 1) / s.lpc;
  int grid = sm_count();
  if (grid > groups) grid = groups;
  kern<<<grid, s.T * s.lpc, s.smem, st>>>(p);
  return cudaGetLastError();
}

template <int NY, int NOBS>
inline cudaError_t col_fused_NY(const ColFusedParams& p, cudaStream_t st) {
  return p.vsel ? col_fused_NYS<NY, NOBS, 1>(p, st) : col_fused_NYS<NY, NOBS, 0>(p, st);
}

#define FFTENKF_FUSED_SIZES(X) X(512) X(1024) X(2048) X(4096)

template <int NOBS>
inline cudaError_t col_fused_dispatch(const ColFusedParams& p, cudaStream_t s) {
  switch (p.ny) {
#define CASE(n) case n: return col_fused_NY<n, NOBS>(p, s);
    FFTENKF_FUSED_SIZES(CASE)
#undef CASE
    default: return cudaErrorNotSupported;
  }
}

cudaError_t col_fused_nobs1(const ColFusedParams& p, cudaStream_t s);
cudaError_t col_fused_nobs2(const ColFusedParams& p, cudaStream_t s);

}  // namespace fftenkf
