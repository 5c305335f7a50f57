// Line FFTs of two lines at once in paired FP32 arithmetic.
//
// Blackwell issues add/sub/mul/fma on two packed FP32 values (f32x2) at the
// issue cost of one scalar instruction.  A thread that transforms two lines a
// and b with the same plan holds each element as a "pair" {re = (a.re, b.re),
// im = (a.im, b.im)}: every butterfly add and multiply then becomes one
// paired instruction for both lines, multiplication by +-i is a renaming of
// re and im, and an exchange through shared memory moves both lines' element
// as one 16-byte access.  The schedule (canonical distribution: thread t owns
// elements t + T m, radix plan, Stockham stages, stage-major twiddle tables)
// is the one of fft_core.cuh; the paired twiddle table holds each entry w of
// fft_core.cuh's compact table as the broadcast pairs (w.re, w.re, w.im, w.im).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_core.cuh"

namespace fftenkf {

// ------------------------------------------------------------------ paired scalars
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) {
  unsigned long long A, B, D;
  __builtin_memcpy(&A, &a, 8);
  __builtin_memcpy(&B, &b, 8);
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(D) : "l"(A), "l"(B));
  float2 d;
  __builtin_memcpy(&d, &D, 8);
  return d;
}
__device__ __forceinline__ float2 p_bc(float s) { return make_float2(s, s); }

// one element of two lines
struct cp {
  float2 re, im;
};
__device__ __forceinline__ cp cp_add(cp a, cp b) { return {p_add(a.re, b.re), p_add(a.im, b.im)}; }
__device__ __forceinline__ cp cp_sub(cp a, cp b) { return {p_sub(a.re, b.re), p_sub(a.im, b.im)}; }
// a + s d and a - s d with s = -i (forward) or +i (INV)
template <bool INV>
__device__ __forceinline__ cp cp_add_rot(cp a, cp d) {
  return INV ? cp{p_sub(a.re, d.im), p_add(a.im, d.re)} : cp{p_add(a.re, d.im), p_sub(a.im, d.re)};
}
template <bool INV>
__device__ __forceinline__ cp cp_sub_rot(cp a, cp d) {
  return INV ? cp{p_add(a.re, d.im), p_sub(a.im, d.re)} : cp{p_sub(a.re, d.im), p_add(a.im, d.re)};
}
// s d, s = -i (forward) or +i (INV): the negation costs one paired op
template <bool INV>
__device__ __forceinline__ cp cp_rot(cp d) {
  const float2 z = make_float2(0.f, 0.f);
  return INV ? cp{p_sub(z, d.im), d.re} : cp{d.im, p_sub(z, d.re)};
}
// 16-byte shared-memory form {a.re, b.re, a.im, b.im}
__device__ __forceinline__ float4 cp_pack(cp a) { return make_float4(a.re.x, a.re.y, a.im.x, a.im.y); }
__device__ __forceinline__ cp cp_unpack(float4 v) { return {make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
// the pair of two separate complex values
__device__ __forceinline__ cp cp_of(float2 a, float2 b) { return {make_float2(a.x, b.x), make_float2(a.y, b.y)}; }
__device__ __forceinline__ float2 cp_a(cp v) { return make_float2(v.re.x, v.im.x); }
__device__ __forceinline__ float2 cp_b(cp v) { return make_float2(v.re.y, v.im.y); }

// ------------------------------------------------------------------ small DFTs
template <int R, bool INV> struct PDft;

template <bool INV> struct PDft<2, INV> {
  static __device__ __forceinline__ void run(cp* a) {
    const cp t = a[0];
    a[0] = cp_add(t, a[1]);
    a[1] = cp_sub(t, a[1]);
  }
};

template <bool INV> struct PDft<3, INV> {
  static __device__ __forceinline__ void run(cp* a) {
    const float2 h = p_bc(0.86602540378443864676f);   // sin(2 pi / 3)
    const float2 half = p_bc(0.5f);
    const cp s = cp_add(a[1], a[2]);
    const cp df = cp_sub(a[1], a[2]);
    const cp d = {p_mul(df.re, h), p_mul(df.im, h)};
    const cp m = {p_sub(a[0].re, p_mul(half, s.re)), p_sub(a[0].im, p_mul(half, s.im))};
    a[0] = cp_add(a[0], s);
    a[1] = cp_add_rot<INV>(m, d);
    a[2] = cp_sub_rot<INV>(m, d);
  }
};

template <bool INV> struct PDft<4, INV> {
  static __device__ __forceinline__ void run(cp* a) {
    const cp t0 = cp_add(a[0], a[2]), t1 = cp_sub(a[0], a[2]);
    const cp t2 = cp_add(a[1], a[3]), d = cp_sub(a[1], a[3]);
    a[0] = cp_add(t0, t2);
    a[2] = cp_sub(t0, t2);
    a[1] = cp_add_rot<INV>(t1, d);
    a[3] = cp_sub_rot<INV>(t1, d);
  }
};

// multiply by exp(-+ 2 pi i e / 8), e = 1 or 3 (e = 2 is a rotation)
template <int E, bool INV>
__device__ __forceinline__ cp pw8(cp v) {
  const float2 c = p_bc(0.70710678118654752440f);
  if (E == 1) {
    return INV ? cp{p_mul(c, p_sub(v.re, v.im)), p_mul(c, p_add(v.re, v.im))}
               : cp{p_mul(c, p_add(v.re, v.im)), p_mul(c, p_sub(v.im, v.re))};
  }
  // E == 3
  const float2 nc = p_bc(-0.70710678118654752440f);
  return INV ? cp{p_mul(nc, p_add(v.re, v.im)), p_mul(c, p_sub(v.re, v.im))}
             : cp{p_mul(c, p_sub(v.im, v.re)), p_mul(nc, p_add(v.re, v.im))};
}

template <bool INV> struct PDft<8, INV> {
  static __device__ __forceinline__ void run(cp* a) {
    cp e[4] = {a[0], a[2], a[4], a[6]};
    cp o[4] = {a[1], a[3], a[5], a[7]};
    PDft<4, INV>::run(e);
    PDft<4, INV>::run(o);
    o[1] = pw8<1, INV>(o[1]);
    o[3] = pw8<3, INV>(o[3]);
    a[0] = cp_add(e[0], o[0]);
    a[4] = cp_sub(e[0], o[0]);
    a[1] = cp_add(e[1], o[1]);
    a[5] = cp_sub(e[1], o[1]);
    a[2] = cp_add_rot<INV>(e[2], o[2]);   // o[2] times exp(-+ 2 pi i 2/8) = -+i
    a[6] = cp_sub_rot<INV>(e[2], o[2]);
    a[3] = cp_add(e[3], o[3]);
    a[7] = cp_sub(e[3], o[3]);
  }
};

// multiply by exp(-+ 2 pi i e / 16) for odd e in {1, 3, 9}
template <int E, bool INV>
__device__ __forceinline__ cp pw16(cp v) {
  constexpr float c1 = 0.92387953251128675613f;  // cos(pi/8)
  constexpr float s1 = 0.38268343236508977173f;  // sin(pi/8)
  constexpr float cr = (E == 1) ? c1 : (E == 3) ? s1 : -c1;
  constexpr float si = (E == 1) ? s1 : (E == 3) ? c1 : -s1;
  // forward: (cr re + si im, cr im - si re); inverse: (cr re - si im, cr im + si re)
  const float2 C = p_bc(cr), S = p_bc(INV ? -si : si), NS = p_bc(INV ? si : -si);
  return {p_fma(v.re, C, p_mul(v.im, S)), p_fma(v.im, C, p_mul(v.re, NS))};
}

template <bool INV> struct PDft<16, INV> {
  // 16 = 4 x 4: inner DFT4 over a[4 n1 + n2], twiddle W16^(n2 k1), outer DFT4 over n2
  static __device__ __forceinline__ void run(cp* a) {
    cp y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      cp t[4] = {a[n2], a[4 + n2], a[8 + n2], a[12 + n2]};
      PDft<4, INV>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = t[k1];
    }
    y[1][1] = pw16<1, INV>(y[1][1]);
    y[1][2] = pw8<1, INV>(y[1][2]);
    y[1][3] = pw16<3, INV>(y[1][3]);
    y[2][1] = pw8<1, INV>(y[2][1]);
    y[2][2] = cp_rot<INV>(y[2][2]);
    y[2][3] = pw8<3, INV>(y[2][3]);
    y[3][1] = pw16<3, INV>(y[3][1]);
    y[3][2] = pw8<3, INV>(y[3][2]);
    y[3][3] = pw16<9, INV>(y[3][3]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      cp t[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      PDft<4, INV>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = t[k2];
    }
  }
};

// ------------------------------------------------------------------ exchange layout
// 16-byte slots; one spare slot per 2^sh keeps the stride-R writes of the first
// stage (the only strided ones) on distinct bank quads: sh = 4 when the first
// radix is 16, else 3.
__host__ __device__ constexpr int pair_pad_shift(int N, int V) { return radix_at(N, V, 0) == 16 ? 4 : 3; }
__host__ __device__ constexpr int pair_padded_len(int N, int V) { return N + (N >> pair_pad_shift(N, V)); }
template <int SH>
__device__ __forceinline__ int ppidx(int i) { return i + (i >> SH); }

// ------------------------------------------------------------------ stages
// The twiddle powers w^r of one butterfly as broadcast pairs (wr[r], wi[r]), from the
// paired table (entries (w.re, w.re, w.im, w.im) in the order of fft_core.cuh's compact
// table: stored powers 1, 2, 4, 8, the others formed by products), conjugated for INV.
template <int R, bool INV>
__device__ __forceinline__ void pair_twiddle_powers(float2 (&wr)[R], float2 (&wi)[R], const float4* __restrict__ tws,
                                                    int NS) {
#pragma unroll
  for (int q = 0; q < tw_npow(R); ++q) {
    const float4 x = __ldg(tws + q * NS);
    wr[tw_pow(q)] = make_float2(x.x, x.y);
    wi[tw_pow(q)] = INV ? make_float2(-x.z, -x.w) : make_float2(x.z, x.w);
  }
#pragma unroll
  for (int r = 3; r < R; ++r) {
    if ((r & (r - 1)) == 0) continue;
    const int hi = r >= 8 ? 8 : (r >= 4 ? 4 : 2);
    const int lo = r - hi;
    wr[r] = p_sub(p_mul(wr[hi], wr[lo]), p_mul(wi[hi], wi[lo]));
    wi[r] = p_fma(wr[hi], wi[lo], p_mul(wi[hi], wr[lo]));
  }
}
// a w for a broadcast factor (wr, wi) (already conjugated for the inverse)
__device__ __forceinline__ cp cp_mulw(cp a, float2 wr, float2 wi) {
  return {p_sub(p_mul(a.re, wr), p_mul(a.im, wi)), p_fma(a.re, wi, p_mul(a.im, wr))};
}

// As Stage in fft_core.cuh, for two lines.
template <int N, int V, int S, int NS, bool INV, bool TRAIL>
struct PStage {
  static __device__ __forceinline__ void run(cp (&v)[V], float4* sm, int t, const float4* __restrict__ tw, int bid) {
    constexpr int R = radix_at(N, V, S);
    constexpr int T = N / V;
    constexpr int B = V / R;
    constexpr int SH = pair_pad_shift(N, V);
    constexpr bool LAST = (S == num_stages(N, V) - 1);
#pragma unroll
    for (int b = 0; b < B; ++b) {
      cp a[R];
#pragma unroll
      for (int r = 0; r < R; ++r) a[r] = v[b + r * B];
      const int j = t + T * b;
      if (NS > 1) {
        float2 wr[R], wi[R];
        pair_twiddle_powers<R, INV>(wr, wi, tw + twiddle_offset(N, V, S) + (j % NS), NS);
#pragma unroll
        for (int r = 1; r < R; ++r) a[r] = cp_mulw(a[r], wr[r], wi[r]);
      }
      PDft<R, INV>::run(a);
      if (LAST) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[b + r * B] = a[r];
      } else {
        const int p = (j / NS) * NS * R + (j % NS);
#pragma unroll
        for (int r = 0; r < R; ++r) sm[ppidx<SH>(p + r * NS)] = cp_pack(a[r]);
      }
    }
    if constexpr (!LAST) {
      line_sync<T>(bid);
#pragma unroll
      for (int m = 0; m < V; ++m) v[m] = cp_unpack(sm[ppidx<SH>(t + T * m)]);
      if constexpr (TRAIL || S + 2 < num_stages(N, V)) line_sync<T>(bid);
      PStage<N, V, S + 1, NS * R, INV, TRAIL>::run(v, sm, t, tw, bid);
    }
  }
};

// As PStage, with the exchanges alternating between two buffers (even exchanges in sa, odd
// ones in sb), so that no barrier separates one exchange's reads from the next one's writes:
// a thread writes sb only after the barrier of the previous exchange, which every thread
// reaches after its last read of sb, and likewise for sa.  With an odd number of exchanges the
// last one is followed by a barrier, so that the next transform may start again in sa.
template <int N, int V, int S, int NS, bool INV>
struct PStage2 {
  static __device__ __forceinline__ void run(cp (&v)[V], float4* sa, float4* sb, int t, const float4* __restrict__ tw,
                                             int bid) {
    constexpr int R = radix_at(N, V, S);
    constexpr int T = N / V;
    constexpr int B = V / R;
    constexpr int SH = pair_pad_shift(N, V);
    constexpr bool LAST = (S == num_stages(N, V) - 1);
    float4* sm = (S % 2 == 0) ? sa : sb;
#pragma unroll
    for (int b = 0; b < B; ++b) {
      cp a[R];
#pragma unroll
      for (int r = 0; r < R; ++r) a[r] = v[b + r * B];
      const int j = t + T * b;
      if (NS > 1) {
        float2 wr[R], wi[R];
        pair_twiddle_powers<R, INV>(wr, wi, tw + twiddle_offset(N, V, S) + (j % NS), NS);
#pragma unroll
        for (int r = 1; r < R; ++r) a[r] = cp_mulw(a[r], wr[r], wi[r]);
      }
      PDft<R, INV>::run(a);
      if (LAST) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[b + r * B] = a[r];
      } else {
        const int p = (j / NS) * NS * R + (j % NS);
#pragma unroll
        for (int r = 0; r < R; ++r) sm[ppidx<SH>(p + r * NS)] = cp_pack(a[r]);
      }
    }
    if constexpr (!LAST) {
      line_sync<T>(bid);
#pragma unroll
      for (int m = 0; m < V; ++m) v[m] = cp_unpack(sm[ppidx<SH>(t + T * m)]);
      if constexpr (S + 2 == num_stages(N, V) && (num_stages(N, V) - 1) % 2 == 1) line_sync<T>(bid);
      PStage2<N, V, S + 1, NS * R, INV>::run(v, sa, sb, t, tw, bid);
    }
  }
};

// Unnormalised DFT of two lines at once, sign -1 (forward) or +1 (INV); the
// calling conventions (bid, TRAIL, canonical distribution) are those of
// fft_line.  sm: the pair's buffer of pair_padded_len(N, V) 16-byte slots.
template <int N, int V, bool INV, bool TRAIL = true>
__device__ __forceinline__ void fft_pair(cp (&v)[V], float4* sm, int t, const float4* __restrict__ tw, int bid = 0) {
  static_assert(N % V == 0, "V must divide N");
  static_assert(num_stages(N, V) > 0, "no radix plan");
  PStage<N, V, 0, 1, INV, TRAIL>::run(v, sm, t, tw, bid);
}

// Two-buffer form (PStage2): each exchange takes one barrier.  Every thread of the line (bid)
// calls it; sa and sb hold pair_padded_len(N, V) slots each; on return both may be written
// again by the next transform's exchanges (which start in sa), but not by anything else
// before a barrier of the line.
template <int N, int V, bool INV>
__device__ __forceinline__ void fft_pair2(cp (&v)[V], float4* sa, float4* sb, int t, const float4* __restrict__ tw,
                                          int bid = 0) {
  static_assert(N % V == 0, "V must divide N");
  static_assert(num_stages(N, V) > 0, "no radix plan");
  PStage2<N, V, 0, 1, INV>::run(v, sa, sb, t, tw, bid);
}

}  // namespace fftenkf
