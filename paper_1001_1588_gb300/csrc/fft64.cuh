// Two-stage line FFTs with a radix-64 first stage, for lines of N = 64 S
// points (S = 16, 32, 64: N = 1024, 2048, 4096).
//
// A line is transformed by T = N/64 threads that hold 64 values each in the
// canonical distribution of fft_core.cuh (thread t owns elements t + T m).
// Stage 0 is a radix-64 butterfly on a thread's own values (an 8 x 8
// two-factor DFT in registers, no table twiddles), stage 1 a radix-S
// butterfly after the twiddles W_N^(j r).  Between them the line goes once
// through shared memory, so every element passes shared memory twice (one
// store, one load) instead of four times with three radix-16 stages: on this
// hardware the shared-memory/L1 data path, not the FP32 pipe, bounds line
// FFTs.  A 2048-point line is one warp (its exchange needs only __syncwarp),
// a 4096-point line two warps (a named barrier of 64 threads), a 1024-point
// line half a warp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "fft_core.cuh"

namespace fftenkf {

// ------------------------------------------------------------------ compile-time constants
// sin and cos of 2 pi e / R in double precision from their Taylor series on the
// argument reduced to [-pi, pi] (30 terms: truncation below 1e-18), for the
// twiddle constants of the in-register butterflies.
__host__ __device__ constexpr double cx_angle(int e, int R) {
  const double pi = 3.14159265358979323846264338327950288;
  double a = 2.0 * pi * (double)(e % R) / (double)R;
  return a > pi ? a - 2.0 * pi : a;
}
__host__ __device__ constexpr double cx_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double cx_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// v times exp(-2 pi i E / R) (forward) or exp(+2 pi i E / R) (INV), E known at compile time
template <int E, int R, bool INV>
__device__ __forceinline__ float2 twc(float2 v) {
  constexpr int e = E % R;
  if constexpr (e == 0) {
    return v;
  } else if constexpr (4 * e == R) {
    return rot90<INV>(v);
  } else if constexpr (2 * e == R) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (4 * e == 3 * R) {
    return rot90<!INV>(v);
  } else if constexpr ((8 * e) % R == 0 && (8 * e) / R < 4) {   // pi/4 or 3 pi/4
    return w8<(8 * e) / R, INV>(v);
  } else if constexpr ((8 * e) % R == 0) {                         // 5 pi/4 or 7 pi/4: the negated ones
    const float2 u = w8<(8 * e) / R - 4, INV>(v);
    return make_float2(-u.x, -u.y);
  } else {
    constexpr float c = (float)cx_cos(cx_angle(e, R));
    constexpr float s = (float)cx_sin(cx_angle(e, R));
    // forward: v (c - i s); inverse: v (c + i s)
    return INV ? make_float2(fmaf(c, v.x, -s * v.y), fmaf(c, v.y, s * v.x))
               : make_float2(fmaf(c, v.x, s * v.y), fmaf(c, v.y, -s * v.x));
  }
}

// R = R1 R2 point DFT in registers: inner R1-point DFTs over a[R2 n1 + n2],
// twiddles W_R^(n2 k1), outer R2-point DFTs over n2; result X[k1 + R1 k2] in a[k1 + R1 k2].
template <int R1, int R2, bool INV>
struct DftRR {
  static __device__ __forceinline__ void run(float2* a) {
    constexpr int R = R1 * R2;
    float2 y[R];   // y[R2 k1 + n2]
    static_for<0, R2>([&](auto n2c) {
      constexpr int n2 = decltype(n2c)::value;
      float2 t[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) t[n1] = a[R2 * n1 + n2];
      Dft<R1, INV>::run(t);
      static_for<0, R1>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        y[R2 * k1 + n2] = twc<n2 * k1, R, INV>(t[k1]);
      });
    });
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      float2 t[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) t[n2] = y[R2 * k1 + n2];
      Dft<R2, INV>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) a[k1 + R1 * k2] = t[k2];
    }
  }
};

template <int R, bool INV> struct DftBig;
template <bool INV> struct DftBig<16, INV> {
  static __device__ __forceinline__ void run(float2* a) { Dft<16, INV>::run(a); }
};
template <bool INV> struct DftBig<32, INV> {
  static __device__ __forceinline__ void run(float2* a) { DftRR<8, 4, INV>::run(a); }
};
template <bool INV> struct DftBig<64, INV> {
  static __device__ __forceinline__ void run(float2* a) { DftRR<8, 8, INV>::run(a); }
};

// ------------------------------------------------------------------ layout
// exchange buffer slots: one spare 8-byte slot per 64 keeps the stage-0 writes (stride 64) on
// distinct banks within a half-warp
__host__ __device__ constexpr int line64_slots(int N) { return N + N / 64; }
__device__ __forceinline__ int p64(int i) { return i + (i >> 6); }
// stage-1 twiddle table: entry (r - 1) 64 + j = W_N^(j r), j < 64, 0 < r < N/64
__host__ __device__ constexpr int tw64_count(int N) { return (N / 64 - 1) * 64; }

template <int T>
__device__ __forceinline__ void sync64(int bid) {
  if constexpr (T <= 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(bid), "n"(T) : "memory");
  }
}

// Unnormalised DFT of one line of N = 64 S points (sign -1, or +1 with INV) by the
// T = S threads that call it with the same sm and bid (bid: a named barrier id
// reserved for this line when T > 32; lines of at most 32 threads synchronise their
// warp, whose other lanes, if any, must call it too).  v: canonical values in and
// out.  tw: the stage-1 table of N (exp(-2 pi i e/N) values).  With TRAIL = false
// the call returns while other threads of the line may still read sm.
template <int N, bool INV, bool TRAIL = true>
__device__ __forceinline__ void fft64_line(float2 (&v)[64], float2* sm, int t, const float2* __restrict__ tw,
                                           int bid = 1) {
  constexpr int T = N / 64;
  constexpr int S = N / 64;
  constexpr int B = 64 / S;
  static_assert(S == 16 || S == 32 || S == 64, "N must be 1024, 2048 or 4096");
  DftBig<64, INV>::run(v);
#pragma unroll
  for (int r = 0; r < 64; ++r) sm[p64(t * 64 + r)] = v[r];
  sync64<T>(bid);
#pragma unroll
  for (int m = 0; m < 64; ++m) v[m] = sm[p64(t + T * m)];
  if constexpr (TRAIL) sync64<T>(bid);
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = t + T * b;
    float2 a[S];
#pragma unroll
    for (int r = 0; r < S; ++r) a[r] = v[b + r * B];
#pragma unroll
    for (int r = 1; r < S; ++r) {
      float2 w = __ldg(tw + (r - 1) * 64 + j);
      if (INV) w.y = -w.y;
      a[r] = cmul(a[r], w);
    }
    DftBig<S, INV>::run(a);
#pragma unroll
    for (int r = 0; r < S; ++r) v[b + r * B] = a[r];
  }
}

}  // namespace fftenkf
