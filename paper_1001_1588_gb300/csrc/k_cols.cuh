// Column passes: the second half of each 2-D transform, fused with the
// per-wavenumber work of Sec. 2.1.  Both are persistent kernels whose input
// lines (one wavenumber column k_x of a field's row spectra, ny contiguous
// complex values) arrive in shared memory by bulk asynchronous copies issued
// one step ahead, so HBM latency overlaps the transforms.
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
#include "perturb.cuh"
#include "tma.cuh"

namespace fftenkf {

// Gains of one wavenumber whose denominator chat^(oo) + rhat is below FLT_MIN (both
// vanish, or rhat = 0 and chat a few rounding errors below 0): the quotients in FP64, 0
// where the denominator is exactly 0.  Kept out of line so
// that the common FP32 path carries none of its instructions.  xa: the first cross
// accumulator of this wavenumber (stride ny between tables).  Returns false if a
// cross spectrum is not finite.
static __device__ __noinline__ bool gains_fp64(float* goo, float2* gjo, float2* xout, const float2* xa, size_t xstride,
                                        int i, int n_un, size_t at, size_t tab, double den, float val, float inv_G,
                                        float scale) {
  bool ok = true;
  const double rd = (den != 0.0) ? (double)inv_G / den : 0.0;
  goo[i * tab + at] = (float)((double)val * rd);
  for (int u = 0; u < n_un; ++u) {
    const float2 a = xa[(size_t)(i * n_un + u) * xstride];
    const float2 x = make_float2(a.x * scale, a.y * scale);
    ok &= isfinite(x.x) && isfinite(x.y);
    if (xout) xout[(i * n_un + u) * tab + at] = x;
    gjo[(i * n_un + u) * tab + at] = make_float2((float)((double)x.x * rd), (float)((double)x.y * rd));
  }
  return ok;
}

// A column line into the canonical registers.  part 1 / 2: the real DC column (.x of the
// packed column 0) or the real Nyquist column (.y); the branch is taken once per line.
template <int NY, int V>
__device__ __forceinline__ void read_line(float2 (&v)[V], const float2* __restrict__ src, int t, int part) {
  constexpr int T = NY / V;
  if (part == 0) {
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = src[t + T * m];
  } else if (part == 1) {
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = make_float2(src[t + T * m].x, 0.f);
  } else {
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = make_float2(src[t + T * m].y, 0.f);
  }
}

// ----------------------------------------------------------------- col_stats
// smem: acc [LPC][nf][NY] f32 | xbuf [LPC][padded(NY)] f2 | stage [LPC][NY] f2 | bar | flag
template <int NY, int V, int NOBS>
__global__ void __launch_bounds__((NY / V > 256) ? 512 : 256, 1) col_stats_kernel(const ColStatsParams p) {
  constexpr int T = NY / V;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int LPC = blockDim.x / T;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int nf = p.n_obs + 2 * p.n_pair + 2 * p.n_obs * p.n_un;
  float* acc_all = reinterpret_cast<float*>(smraw);
  float* acc = acc_all + (size_t)g * nf * NY;
  float2* xacc = reinterpret_cast<float2*>(acc + p.n_obs * NY);
  float2* xbuf_all = reinterpret_cast<float2*>(acc_all + (size_t)LPC * nf * NY);
  constexpr int PL = (padded_len(NY) + 1) & ~1;
  float2* line = xbuf_all + (size_t)g * PL;
  float2* stage_all = xbuf_all + (size_t)LPC * PL;
  float2* stage = stage_all + (size_t)g * NY;
  uint64_t* bar = reinterpret_cast<uint64_t*>(stage_all + (size_t)LPC * NY);
  int* flag = reinterpret_cast<int*>(bar + 1);
  const int M = p.M;
  const int lines_per_col = p.N * M;
  const size_t fstride = (size_t)p.L * NY;
  const int ncol = p.L + 1;
  const int col_step = gridDim.x * LPC;

  // global line l of column group starting at cb: member k = l / M, block slot b = l % M
  auto issue = [&](int cb, int l) {
    const int k = l / M, b = l - (l / M) * M;
    const int blk = (b < p.n_obs) ? p.obs[b] : p.un[b - p.n_obs];
    int nvalid = 0;
    for (int gg = 0; gg < LPC; ++gg) nvalid += (cb + gg < ncol);
    mbar_arrive_expect_tx(bar, (uint32_t)(nvalid * NY * sizeof(float2)));
    for (int gg = 0; gg < LPC; ++gg) {
      const int c = cb + gg;
      if (c >= ncol) break;
      const int col = (c == p.L) ? 0 : c;
      bulk_g2s(stage_all + (size_t)gg * NY, p.A + ((size_t)blk * p.N + k) * fstride + (size_t)col * NY,
               NY * sizeof(float2), bar);
    }
  };

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  int cb = blockIdx.x * LPC;
  if (threadIdx.x == 0 && cb < ncol) issue(cb, 0);
  for (; cb < ncol; cb += col_step) {
    const int c = cb + g;
    const bool active = c < ncol;
    const int part = (c == 0) ? 1 : ((c == p.L) ? 2 : 0);
    for (int s = t; s < nf * NY; s += T) acc[s] = 0.f;
    float2 ko[NOBS][V];
#pragma unroll
    for (int i = 0; i < NOBS; ++i)
#pragma unroll
      for (int m = 0; m < V; ++m) ko[i][m] = make_float2(0.f, 0.f);
    for (int l = 0; l < lines_per_col; ++l) {
      const int b = l % M;
      const float sg = (l < M) ? -1.f : 1.f;   // member 0's place holds the pivot sum: its products are subtracted
      if (!cta_wait(bar, phase, p.status, flag)) return;
      phase ^= 1;
      float2 v[V];
      read_line<NY, V>(v, stage, t, part);
      __syncthreads();                                   // stage consumed
      if (threadIdx.x == 0) {
        if (l + 1 < lines_per_col) issue(cb, l + 1);
        else if (cb + col_step < ncol) issue(cb + col_step, 0);
      }
      // no trailing barrier: the buffer is next written after the next line's CTA-wide waits
      fft_line<NY, V, false, false>(v, line, t, p.twY, line_bar<T>(g));
      if (b < p.n_obs) {
#pragma unroll
        for (int i = 0; i < NOBS; ++i) {
          if (i == b) {
#pragma unroll
            for (int m = 0; m < V; ++m) {
              ko[i][m] = v[m];
              float& a = acc[i * NY + t + T * m];
              a = fmaf(sg * v[m].x, v[m].x, fmaf(sg * v[m].y, v[m].y, a));
            }
            if (NOBS >= 2 && i == 1 && p.n_pair) {   // coupled: observed pair chat^(o1 o0) += v conj(ko_0)
              float2* a = xacc + t;
#pragma unroll
              for (int m = 0; m < V; ++m) {
                const float2 w = make_float2(sg * v[m].x, sg * v[m].y);
                float2 o = a[T * m];
                o.x = fmaf(w.x, ko[0][m].x, fmaf(w.y, ko[0][m].y, o.x));
                o.y = fmaf(w.y, ko[0][m].x, fmaf(-w.x, ko[0][m].y, o.y));
                a[T * m] = o;
              }
            }
          }
        }
      } else {
        const int u = b - p.n_obs;
#pragma unroll
        for (int i = 0; i < NOBS; ++i) {
          if (i < p.n_obs) {
            float2* a = xacc + (size_t)(p.n_pair + i * p.n_un + u) * NY + t;
#pragma unroll
            for (int m = 0; m < V; ++m) {
              // o += sg v conj(ko), as two fused multiply-adds per component
              const float2 w = make_float2(sg * v[m].x, sg * v[m].y);
              float2 o = a[T * m];
              o.x = fmaf(w.x, ko[i][m].x, fmaf(w.y, ko[i][m].y, o.x));
              o.y = fmaf(w.y, ko[i][m].x, fmaf(-w.x, ko[i][m].y, o.y));
              a[T * m] = o;
            }
          }
        }
      }
    }
    if (active) {
      const size_t tab = (size_t)(p.L + 1) * NY;
      bool bad = false;
      float2* xout = p.chat ? reinterpret_cast<float2*>(p.chat + p.n_obs * tab) : nullptr;
      // rhat values are requested E at a time before any of their tables is stored, so the
      // epilogue waits for one memory latency per E values rather than one per value
      constexpr int E = (V % 8 == 0) ? 8 : ((V % 4 == 0) ? 4 : V);
      if (p.n_pair && p.chat) {   // coupled: the observed pair chat^(o1 o0), first complex table
#pragma unroll
        for (int m = 0; m < V; ++m) {
          const int ky = t + T * m;
          const float2 a = xacc[ky];
          const float2 x = make_float2(a.x * p.scale, a.y * p.scale);
          bad |= !(isfinite(x.x) && isfinite(x.y));
          xout[(size_t)c * NY + ky] = x;
        }
      }
#pragma unroll 1
      for (int i = 0; i < p.n_obs; ++i) {
#pragma unroll 1
        for (int m0 = 0; m0 < V; m0 += E) {
          double rr[E];
          if (p.rhat_t) {
#pragma unroll
            for (int e = 0; e < E; ++e) rr[e] = __ldg(p.rhat_t + i * tab + (size_t)c * NY + t + T * (m0 + e));
          }
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int ky = t + T * (m0 + e);
            const size_t at = (size_t)c * NY + ky;
            const float val = acc[i * NY + ky] * p.scale;
            bad |= !isfinite(val);
            if (p.chat) p.chat[i * tab + at] = val;
            if (p.rhat_t) {
              // eq. (spectral-multi-enkf): G = chat / (chat^(oo) + rhat).  The sum is formed in
              // FP64 (where chat << rhat it keeps chat's digits), then rounded once; the
              // quotients are FP32; a sum below FLT_MIN takes the FP64 path (gains_fp64).
              const double den = (double)val + rr[e];
              const float denf = (float)den;
              const float inv = __fdividef(p.inv_G, denf);
              const bool tiny = !(denf >= 1.17549435e-38f);
              if (tiny) {
                bad |= !gains_fp64(p.goo, p.gjo, xout, xacc + ky, NY, i, p.n_un, at, tab, den, val, p.inv_G, p.scale);
              } else {
                p.goo[i * tab + at] = val * inv;
                for (int u = 0; u < p.n_un; ++u) {
                  const float2 a = xacc[(size_t)(i * p.n_un + u) * NY + ky];
                  const float2 x = make_float2(a.x * p.scale, a.y * p.scale);
                  bad |= !(isfinite(x.x) && isfinite(x.y));
                  if (xout) xout[(i * p.n_un + u) * tab + at] = x;
                  p.gjo[(i * p.n_un + u) * tab + at] = make_float2(x.x * inv, x.y * inv);
                }
              }
            } else if (xout) {
              for (int u = 0; u < p.n_un; ++u) {
                const int q = p.n_pair + i * p.n_un + u;
                const float2 a = xacc[(size_t)q * NY + ky];
                const float2 x = make_float2(a.x * p.scale, a.y * p.scale);
                bad |= !(isfinite(x.x) && isfinite(x.y));
                xout[q * tab + at] = x;
              }
            }
          }
        }
      }
      if (bad) atomicOr(p.status, kStatusNonFinite);
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------- col_update
// Two bulk-copy pipelines: innovation lines one item ahead (two stages, or one
// when shared memory is short) and gain lines one target block ahead (one
// stage, read into registers before the next copy is issued).
// smem: wst [nst][LPC][n_obs][NY] f2 | gst [LPC][n_obs][NY] f2 | xbuf [LPC][PL] f2 | bars[3] | flag
// DRAWN: the perturbations are drawn here (seeded analysis); a separate instantiation, so that the
// analysis with given perturbations carries none of the generator's code
template <int NY, int V, int NOBS, bool DRAWN>
__global__ void __launch_bounds__((NY / V > 256) ? 512 : 256, 1) col_update_kernel(const ColUpdParams p) {
  constexpr int T = NY / V;
  constexpr int PL = col_line_slots(NY);
  extern __shared__ __align__(128) unsigned char smraw[];
  const int LPC = blockDim.x / T;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int nst = p.n_stages;
  const size_t stage_elems = (size_t)LPC * p.n_obs * NY;
  float2* wst = reinterpret_cast<float2*>(smraw);
  float2* gst = wst + nst * stage_elems;
  float2* xbuf = gst + stage_elems + (size_t)g * PL;
  uint64_t* bars = reinterpret_cast<uint64_t*>(gst + stage_elems + (size_t)LPC * PL);
  uint64_t* gbar = bars + 2;
  int* flag = reinterpret_cast<int*>(bars + 3);
  const long long n_items = (long long)(p.L + 1) * p.N;
  const long long step = (long long)gridDim.x * LPC;
  const size_t fstride = (size_t)p.L * NY;
  const size_t tab = (size_t)(p.L + 1) * NY;

  auto issue_w = [&](long long base, int s) {
    int nvalid = 0;
    for (int gg = 0; gg < LPC; ++gg) nvalid += (base + gg < n_items);
    mbar_arrive_expect_tx(&bars[s], (uint32_t)(nvalid * p.n_obs * NY * sizeof(float2)));
    for (int gg = 0; gg < LPC; ++gg) {
      const long long item = base + gg;
      if (item >= n_items) break;
      const int c = (int)(item / p.N), k = (int)(item - (long long)c * p.N);
      const int col = (c == p.L) ? 0 : c;
      for (int i = 0; i < p.n_obs; ++i)
        bulk_g2s(wst + s * stage_elems + ((size_t)gg * p.n_obs + i) * NY,
                 p.W + ((size_t)k * p.n_obs + i) * fstride + (size_t)col * NY, NY * sizeof(float2), &bars[s]);
    }
  };
  // gain lines of target block j for every group's item: observed j -> one float line,
  // unobserved j -> n_obs complex lines
  auto issue_g = [&](long long base, int j) {
    const int io = p.coupled ? -1 : p.obs_of_block[j];   // coupled: n_obs complex gains for every block
    const uint32_t line_bytes = (io >= 0) ? NY * sizeof(float) : NY * sizeof(float2);
    const int nl = (io >= 0) ? 1 : p.n_obs;
    int nvalid = 0;
    for (int gg = 0; gg < LPC; ++gg) nvalid += (base + gg < n_items);
    mbar_arrive_expect_tx(gbar, (uint32_t)(nvalid * nl) * line_bytes);
    for (int gg = 0; gg < LPC; ++gg) {
      const long long item = base + gg;
      if (item >= n_items) break;
      const int c = (int)(item / p.N);
      float2* dst = gst + (size_t)gg * p.n_obs * NY;
      if (io >= 0) {
        bulk_g2s(dst, p.goo + io * tab + (size_t)c * NY, line_bytes, gbar);
      } else if (p.coupled) {   // gall [role][n_obs]: observed blocks first, then unobserved
        const int role = (p.obs_of_block[j] >= 0) ? p.obs_of_block[j] : p.n_obs + p.un_of_block[j];
        for (int i = 0; i < p.n_obs; ++i)
          bulk_g2s(dst + (size_t)i * NY, p.gall + (size_t)(role * p.n_obs + i) * tab + (size_t)c * NY, line_bytes, gbar);
      } else {
        const int u = p.un_of_block[j];
        for (int i = 0; i < p.n_obs; ++i)
          bulk_g2s(dst + (size_t)i * NY, p.gjo + (size_t)(i * p.n_un + u) * tab + (size_t)c * NY, line_bytes, gbar);
      }
    }
  };

  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(gbar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t wph0 = 0, wph1 = 0, gph = 0;
  long long base = (long long)blockIdx.x * LPC;
  if (threadIdx.x == 0 && base < n_items) {
    issue_w(base, 0);
    issue_g(base, 0);
  }
  for (int it = 0; base < n_items; base += step, ++it) {
    const int s = (nst == 2) ? (it & 1) : 0;
    if (!cta_wait(&bars[s], s ? wph1 : wph0, p.status, flag)) {
      if (threadIdx.x == 0) {   // other copies may still be landing: let them finish
        mbar_wait_bounded(&bars[s ^ 1], s ? wph0 : wph1);
        mbar_wait_bounded(gbar, gph);
      }
      return;
    }
    if (s) wph1 ^= 1; else wph0 ^= 1;
    if (nst == 2 && threadIdx.x == 0 && base + step < n_items) issue_w(base + step, s ^ 1);
    const long long item = base + g;
    const bool active = item < n_items;
    const int c = active ? (int)(item / p.N) : 0;
    const int k = active ? (int)(item - (long long)c * p.N) : 0;
    const int col = (c == p.L) ? 0 : c;
    const int part = (c == 0) ? 1 : ((c == p.L) ? 2 : 0);
    float2* w = wst + s * stage_elems + (size_t)g * p.n_obs * NY;
    const float2* gl = gst + (size_t)g * p.n_obs * NY;
    // forward column transforms of the innovations, kept in registers
    float2 wv[NOBS][V];
#pragma unroll
    for (int i = 0; i < NOBS; ++i) {
      if (i < p.n_obs) {
        read_line<NY, V>(wv[i], w + (size_t)i * NY, t, part);
        if (i + 1 < p.n_obs)   // the next innovation's transform reuses xbuf at once
          fft_line<NY, V, false>(wv[i], xbuf, t, p.twY, line_bar<T>(g));
        else                   // the gain wait below synchronises the CTA first
          fft_line<NY, V, false, false>(wv[i], xbuf, t, p.twY, line_bar<T>(g));
        if constexpr (DRAWN) {   // what += sqrt(ny nx) sqrt(rhat) zhat: the perturbation e_{k,i} in frequency space
          const double* rh = p.rhat_t + (size_t)i * tab + (size_t)c * NY + t;
          const int stream = k * p.n_obs + i;
          if (c != 0 && c != p.L) {
            // interior column: one generator call per k_y < ny/2 serves k_y (words 0, 1) and
            // k_y + ny/2 (words 2, 3), the slots m and m + V/2 of this thread
            const float h = 0.70710678118654752f;
#pragma unroll
            for (int m = 0; m < V / 2; ++m) {
              const uint4 w4 = philox4x32_10(make_uint4((uint32_t)(t + T * m), (uint32_t)c, (uint32_t)stream, 0u),
                                             (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
              const float2 zl = box_muller(w4.x, w4.y), zh = box_muller(w4.z, w4.w);
              const float al = h * p.sqrt_G * sqrtf((float)__ldg(rh + T * m));
              const float ah = h * p.sqrt_G * sqrtf((float)__ldg(rh + T * (m + V / 2)));
              wv[i][m] = make_float2(fmaf(al, zl.x, wv[i][m].x), fmaf(al, zl.y, wv[i][m].y));
              wv[i][m + V / 2] = make_float2(fmaf(ah, zh.x, wv[i][m + V / 2].x), fmaf(ah, zh.y, wv[i][m + V / 2].y));
            }
          } else {
#pragma unroll
            for (int m = 0; m < V; ++m) {
              const float a = p.sqrt_G * sqrtf((float)__ldg(rh + T * m));
              const float2 z = white_edge(p.seed, stream, t + T * m, c, NY);
              wv[i][m] = make_float2(fmaf(a, z.x, wv[i][m].x), fmaf(a, z.y, wv[i][m].y));
            }
          }
        }
      } else {
#pragma unroll
        for (int m = 0; m < V; ++m) wv[i][m] = make_float2(0.f, 0.f);
      }
    }
    for (int j = 0; j < p.M; ++j) {
      if (!cta_wait(gbar, gph, p.status, flag)) {
        if (threadIdx.x == 0) {
          mbar_wait_bounded(&bars[0], wph0);
          mbar_wait_bounded(&bars[1], wph1);
        }
        return;
      }
      gph ^= 1;
      float2 sv[V];
      const int io = p.coupled ? -1 : p.obs_of_block[j];
#pragma unroll
      for (int m = 0; m < V; ++m) sv[m] = make_float2(0.f, 0.f);
      if (io >= 0) {
        const float* gp = reinterpret_cast<const float*>(gl) + t;
#pragma unroll
        for (int i = 0; i < NOBS; ++i) {
          if (i == io) {
#pragma unroll
            for (int m = 0; m < V; ++m) {
              const float gv = gp[T * m];
              sv[m] = make_float2(gv * wv[i][m].x, gv * wv[i][m].y);
            }
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < NOBS; ++i) {
          if (i < p.n_obs) {
            const float2* gp = gl + (size_t)i * NY + t;
#pragma unroll
            for (int m = 0; m < V; ++m) {   // sv += G w, as two fused multiply-adds per component
              const float2 gv = gp[T * m];
              sv[m].x = fmaf(gv.x, wv[i][m].x, fmaf(-gv.y, wv[i][m].y, sv[m].x));
              sv[m].y = fmaf(gv.x, wv[i][m].y, fmaf(gv.y, wv[i][m].x, sv[m].y));
            }
          }
        }
      }
      __syncthreads();   // gain stage consumed
      if (threadIdx.x == 0) {
        if (j + 1 < p.M) issue_g(base, j + 1);
        else if (base + step < n_items) issue_g(base + step, 0);
      }
      fft_line<NY, V, true, false>(sv, xbuf, t, p.twY, line_bar<T>(g));   // next use follows a CTA-wide wait
      if (active) {
        float2* dst = p.S + ((size_t)j * p.N + k) * fstride + (size_t)col * NY + t;
        if (part == 0) {
#pragma unroll
          for (int m = 0; m < V; ++m) dst[T * m] = sv[m];
        } else {
          float* d1 = reinterpret_cast<float*>(dst) + (part == 1 ? 0 : 1);
#pragma unroll
          for (int m = 0; m < V; ++m) d1[2 * T * m] = sv[m].x;
        }
      }
    }
    __syncthreads();
    if (nst == 1 && threadIdx.x == 0 && base + step < n_items) issue_w(base + step, 0);
  }
}

// ----------------------------------------------------------------- launch templates
int sm_count();

template <int NY, int V, int NOBS>
inline cudaError_t col_stats_NYV(const ColStatsParams& p, cudaStream_t st) {
  constexpr int T = NY / V;
  int lpc = 1;
  const int nf = p.n_obs + 2 * p.n_pair + 2 * p.n_obs * p.n_un;
  const size_t smem = col_stats_smem(NY, nf, p.vsel, &lpc);
  if (smem == 0) return cudaErrorInvalidConfiguration;
  auto kern = col_stats_kernel<NY, V, NOBS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T * lpc, smem);
  if (per_sm < 1) per_sm = 1;
  const int groups = (p.L + 1 + lpc - 1) / lpc;
  int grid = sm_count() * per_sm;
  if (grid > groups) grid = groups;
  kern<<<grid, T * lpc, smem, st>>>(p);
  return cudaGetLastError();
}

size_t col_update_smem(int ny, int n_obs, int* lpc, int* n_stages);

template <int NY, int V, int NOBS>
inline cudaError_t col_update_NYV(const ColUpdParams& p, cudaStream_t st) {
  constexpr int T = NY / V;
  int lpc = 1, nst = 2;
  const size_t smem = col_update_smem(NY, p.n_obs, p.vsel, &lpc, &nst);
  if (smem == 0) return cudaErrorInvalidConfiguration;
  ColUpdParams q = p;
  q.n_stages = nst;
  auto kern = p.drawn ? col_update_kernel<NY, V, NOBS, true> : col_update_kernel<NY, V, NOBS, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T * lpc, smem);
  if (per_sm < 1) per_sm = 1;
  const long long items = (long long)(p.L + 1) * p.N;
  const long long groups = (items + lpc - 1) / lpc;
  long long grid = (long long)sm_count() * per_sm;
  if (grid > groups) grid = groups;
  kern<<<(unsigned)grid, T * lpc, smem, st>>>(q);
  return cudaGetLastError();
}

template <int NY, int NOBS>
inline cudaError_t col_stats_NY(const ColStatsParams& p, cudaStream_t st) {
  if (p.vsel) return col_stats_NYV<NY, plan_V(NY, 1), NOBS>(p, st);
  return col_stats_NYV<NY, plan_V(NY, 0), NOBS>(p, st);
}

template <int NY, int NOBS>
inline cudaError_t col_update_NY(const ColUpdParams& p, cudaStream_t st) {
  if (p.vsel) return col_update_NYV<NY, plan_V(NY, 1), NOBS>(p, st);
  return col_update_NYV<NY, plan_V(NY, 0), NOBS>(p, st);
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
