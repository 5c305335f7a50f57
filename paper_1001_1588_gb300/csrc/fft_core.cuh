// Register/shared-memory FFT of one line, the building block of every pass.
//
// A line of N complex values (N = 2^a or 3*2^a) is transformed by T = N/V
// threads.  Data is held in the "canonical" distribution: thread t owns
// elements t + T*m in register slot m (m < V), both on input and on output,
// so a line is loaded from and stored to global memory with unit-stride,
// fully coalesced warp accesses, and a forward transform's output can feed an
// inverse transform without any exchange.  Between radix stages the values go
// through a padded shared-memory line buffer (Stockham self-sorting order), so
// no bit reversal is needed.  Radices are 16, 8, 4, 2 and 3; the plan is fixed
// at compile time from (N, V).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fftenkf {

// ------------------------------------------------------------------ complex
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward sign) or +i (inverse sign)
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ------------------------------------------------------------------ plan
__host__ __device__ constexpr int pick_radix(int rem, int V) {
  return (rem % 16 == 0 && V % 16 == 0) ? 16
       : (rem % 8 == 0 && V % 8 == 0)   ? 8
       : (rem % 4 == 0 && V % 4 == 0)   ? 4
       : (rem % 2 == 0 && V % 2 == 0)   ? 2
       : (rem % 3 == 0 && V % 3 == 0)   ? 3
                                        : 0;
}
__host__ __device__ constexpr int radix_at(int N, int V, int s) {
  int rem = N;
  for (int i = 0; i < s; ++i) rem /= pick_radix(rem, V);
  return rem == 1 ? 1 : pick_radix(rem, V);
}
__host__ __device__ constexpr int num_stages(int N, int V) {
  int rem = N, s = 0;
  while (rem > 1) {
    int r = pick_radix(rem, V);
    if (r == 0) return -1;
    rem /= r;
    ++s;
  }
  return s;
}
// default values per thread: 16 for powers of two, 24 (or N) for 3*2^a
__host__ __device__ constexpr int default_V(int N) {
  return (N % 3 == 0) ? (N >= 24 ? 24 : N) : (N >= 16 ? 16 : N);
}
// values per thread of schedule `sel`: 0 = wide (radix 16 / 8-3), 1 = narrow (radix 8 / 4-3):
// twice the threads per line, one more exchange
__host__ __device__ constexpr int plan_V(int N, int sel) {
  return sel == 0 ? default_V(N) : ((N % 3 == 0) ? (N >= 12 ? 12 : N) : (N >= 8 ? 8 : N));
}
// padded shared-memory index: one spare slot per 16 keeps stride-R writes
// of the Stockham stages on distinct 8-byte banks
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int N) { return N + N / 16; }
// slots of a column pass's line buffer: a padded line rounded up to 16 slots (128 bytes)
__host__ __device__ constexpr int col_line_slots(int N) { return (padded_len(N) + 15) & ~15; }
// pitch of the staged rows of the row passes: a padded line rounded to 2 (mod 8) slots, so
// that reading two rows x four columns per half-warp hits 16 distinct 8-byte banks
__host__ __device__ constexpr int row_pitch(int N) { return padded_len(N) + ((10 - padded_len(N) % 8) % 8); }

// ------------------------------------------------------------------ small DFTs
// Forward kernels use exp(-2 pi i / R); INV uses exp(+2 pi i / R).
template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<2, INV> {
  static __device__ __forceinline__ void run(float2* a) {
    float2 t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  }
};

template <bool INV> struct Dft<3, INV> {
  static __device__ __forceinline__ void run(float2* a) {
    const float h = 0.86602540378443864676f;  // sin(2 pi / 3)
    float2 s = cadd(a[1], a[2]);
    float2 d = cscale(csub(a[1], a[2]), h);
    float2 m = make_float2(a[0].x - 0.5f * s.x, a[0].y - 0.5f * s.y);
    a[0] = cadd(a[0], s);
    float2 rd = rot90<INV>(d);       // -i d (forward)
    a[1] = cadd(m, rd);
    a[2] = csub(m, rd);
  }
};

template <bool INV> struct Dft<4, INV> {
  static __device__ __forceinline__ void run(float2* a) {
    float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
    float2 t2 = cadd(a[1], a[3]), t3 = rot90<INV>(csub(a[1], a[3]));
    a[0] = cadd(t0, t2);
    a[2] = csub(t0, t2);
    a[1] = cadd(t1, t3);
    a[3] = csub(t1, t3);
  }
};

// multiply by exp(-+ 2 pi i e / 8) for e = 1, 2, 3
template <int E, bool INV>
__device__ __forceinline__ float2 w8(float2 v) {
  const float c = 0.70710678118654752440f;
  if (E == 0) return v;
  if (E == 2) return rot90<INV>(v);
  if (E == 1) return INV ? make_float2(c * (v.x - v.y), c * (v.x + v.y))
                         : make_float2(c * (v.x + v.y), c * (v.y - v.x));
  // E == 3
  return INV ? make_float2(-c * (v.x + v.y), c * (v.x - v.y))
             : make_float2(c * (v.y - v.x), -c * (v.x + v.y));
}

template <bool INV> struct Dft<8, INV> {
  static __device__ __forceinline__ void run(float2* a) {
    float2 e[4] = {a[0], a[2], a[4], a[6]};
    float2 o[4] = {a[1], a[3], a[5], a[7]};
    Dft<4, INV>::run(e);
    Dft<4, INV>::run(o);
    o[1] = w8<1, INV>(o[1]);
    o[2] = w8<2, INV>(o[2]);
    o[3] = w8<3, INV>(o[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k] = cadd(e[k], o[k]);
      a[k + 4] = csub(e[k], o[k]);
    }
  }
};

// multiply by exp(-+ 2 pi i e / 16)
template <int E, bool INV>
__device__ __forceinline__ float2 w16(float2 v) {
  const float c1 = 0.92387953251128675613f;  // cos(pi/8)
  const float s1 = 0.38268343236508977173f;  // sin(pi/8)
  if (E == 0) return v;
  if (E % 2 == 0) return w8<E / 2, INV>(v);
  // angle = 2 pi E / 16; (cr, si) = (cos, sin)
  const float cr = (E == 1) ? c1 : (E == 3) ? s1 : (E == 9) ? -c1 : 0.f;
  const float si = (E == 1) ? s1 : (E == 3) ? c1 : (E == 9) ? -s1 : 0.f;
  // forward multiplies by (cr - i si), inverse by (cr + i si)
  return INV ? make_float2(cr * v.x - si * v.y, cr * v.y + si * v.x)
             : make_float2(cr * v.x + si * v.y, cr * v.y - si * v.x);
}

template <bool INV> struct Dft<16, INV> {
  // 16 = 4 x 4: inner DFT4 over a[4 n1 + n2], twiddle W16^(n2 k1), outer DFT4 over n2
  static __device__ __forceinline__ void run(float2* a) {
    float2 y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      float2 t[4] = {a[n2], a[4 + n2], a[8 + n2], a[12 + n2]};
      Dft<4, INV>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = t[k1];
    }
    y[1][1] = w16<1, INV>(y[1][1]);
    y[1][2] = w16<2, INV>(y[1][2]);
    y[1][3] = w16<3, INV>(y[1][3]);
    y[2][1] = w16<2, INV>(y[2][1]);
    y[2][2] = w16<4, INV>(y[2][2]);
    y[2][3] = w16<6, INV>(y[2][3]);
    y[3][1] = w16<3, INV>(y[3][1]);
    y[3][2] = w16<6, INV>(y[3][2]);
    y[3][3] = w16<9, INV>(y[3][3]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 t[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      Dft<4, INV>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = t[k2];
    }
  }
};

// Twiddle tables.  Butterfly j of a stage with NS > 1 multiplies its input r by w^r,
// w = W_N^((j mod NS) N/(NS R)).  The table stores only the powers w^p for p in
// {1, 2, 4, 8} below R (w and w^2 for radix 3), as rows of NS entries (the threads of a
// warp, consecutive j, read consecutive entries); the butterfly forms the other powers
// by at most three complex products (w^3 = w^2 w, w^5 = w^4 w, ..., w^15 = w^8 w^7).
// A 4096-point plan then needs 1088 entries (8.5 KB) instead of 4080, which stay in L1
// when a pass gives most of the SM's on-chip memory to shared memory.  Stages are
// concatenated in order; twiddle_offset(N, V, s) is where stage s starts.
__host__ __device__ constexpr int tw_npow(int R) { return R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : R == 3 ? 2 : 1; }
__host__ __device__ constexpr int tw_pow(int q) { return 1 << q; }   // the q-th stored power
__host__ __device__ constexpr int stage_ns(int N, int V, int s) {
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= radix_at(N, V, i);
  return ns;
}
__host__ __device__ constexpr int twiddle_offset(int N, int V, int s) {
  int off = 0;
  for (int i = 1; i < s; ++i) off += tw_npow(radix_at(N, V, i)) * stage_ns(N, V, i);
  return off;
}
__host__ __device__ constexpr int twiddle_count(int N, int V) { return twiddle_offset(N, V, num_stages(N, V)); }
// exponent e (of W_N^e = exp(-2 pi i e / N)) of table entry i, 0 <= i < twiddle_count(N, V)
__host__ __device__ constexpr long long twiddle_exponent(int N, int V, int i) {
  const int S = num_stages(N, V);
  int s = 1;
  while (s + 1 < S && twiddle_offset(N, V, s + 1) <= i) ++s;
  const int NS = stage_ns(N, V, s), R = radix_at(N, V, s);
  const int local = i - twiddle_offset(N, V, s);
  const int q = local / NS, jm = local - q * NS;
  return ((long long)jm * tw_pow(q) * (N / (NS * R))) % N;
}

// w^r for r = 1..R-1 of one butterfly from the stored powers (tws: this butterfly's
// first entry; rows NS apart); conjugated for the inverse transform
template <int R, bool INV>
__device__ __forceinline__ void twiddle_powers(float2 (&w)[R], const float2* __restrict__ tws, int NS) {
#pragma unroll
  for (int q = 0; q < tw_npow(R); ++q) {
    float2 x = __ldg(tws + q * NS);
    if (INV) x.y = -x.y;
    w[tw_pow(q)] = x;
  }
#pragma unroll
  for (int r = 3; r < R; ++r) {
    if ((r & (r - 1)) == 0) continue;          // stored
    const int hi = r >= 8 ? 8 : (r >= 4 ? 4 : 2);   // largest stored power below r
    w[r] = cmul(w[hi], w[r - hi]);
  }
}

// Barrier over the threads that transform one line: the whole CTA (bid 0) or
// named barrier bid over the line's T threads, when each line owns whole warps
// and the CTA holds several lines, so that lines progress independently.
// bid < 0: the line is one warp, which synchronises alone.
template <int T>
__device__ __forceinline__ void line_sync(int bid) {
  if (bid == 0) {
    __syncthreads();
  } else if (bid < 0) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(bid), "n"(T) : "memory");
  }
}
// barrier id of line group g for line_sync: 1 + g when lines of T threads own whole warps
// (at most 8 lines per CTA of up to 512 threads), else 0 (the CTA barrier)
template <int T>
__device__ __forceinline__ int line_bar(int g) {
  return (T % 32 == 0 && T >= 64) ? 1 + g : 0;
}

// ------------------------------------------------------------------ stages
// Stage S of the Stockham transform; NS = product of the radices before it.
// Butterfly j reads x[j + r N/R], multiplies by W_N^((j mod NS) r N/(NS R)),
// applies the R-point DFT and writes x[(j/NS) NS R + (j mod NS) + r NS].
// Thread t owns butterflies j = t + T b (b < V/R), whose inputs are its
// canonical slots b + r V/R; the last stage's outputs land in canonical slots.
template <int N, int V, int S, int NS, bool INV, bool TRAIL>
struct Stage {
  static __device__ __forceinline__ void run(float2 (&v)[V], float2* sm, int t, const float2* __restrict__ tw, int bid) {
    constexpr int R = radix_at(N, V, S);
    constexpr int T = N / V;
    constexpr int B = V / R;
    constexpr bool LAST = (S == num_stages(N, V) - 1);
#pragma unroll
    for (int b = 0; b < B; ++b) {
      float2 a[R];
#pragma unroll
      for (int r = 0; r < R; ++r) a[r] = v[b + r * B];
      const int j = t + T * b;
      if (NS > 1) {
        float2 w[R];
        twiddle_powers<R, INV>(w, tw + twiddle_offset(N, V, S) + (j % NS), NS);
#pragma unroll
        for (int r = 1; r < R; ++r) a[r] = cmul(a[r], w[r]);
      }
      Dft<R, INV>::run(a);
      if (LAST) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[b + r * B] = a[r];
      } else {
        const int p = (j / NS) * NS * R + (j % NS);
#pragma unroll
        for (int r = 0; r < R; ++r) sm[pidx(p + r * NS)] = a[r];
      }
    }
    if constexpr (!LAST) {
      line_sync<T>(bid);
#pragma unroll
      for (int m = 0; m < V; ++m) v[m] = sm[pidx(t + T * m)];
      // the buffer is written again by the next stage, or (after the last exchange) by the caller;
      // without TRAIL the caller synchronises before it reuses the buffer
      if constexpr (TRAIL || S + 2 < num_stages(N, V)) line_sync<T>(bid);
      Stage<N, V, S + 1, NS * R, INV, TRAIL>::run(v, sm, t, tw, bid);
    }
  }
};

// Unnormalised line DFT, sign -1 (forward) or +1 (INV).  Every thread of the
// CTA (bid 0) or of the line (bid = line_bar(g)) must call it: it synchronises
// with line_sync(bid) when the plan has >1 stage.  With TRAIL = false it returns
// while other threads of the line may still read sm: the caller must pass a
// barrier of those threads before anything writes sm again.
// tw: the stage-major twiddle table of (N, V) described above (exp(-2 pi i e/N)
// values).  sm: this line's padded buffer.
template <int N, int V, bool INV, bool TRAIL = true>
__device__ __forceinline__ void fft_line(float2 (&v)[V], float2* sm, int t, const float2* __restrict__ tw, int bid = 0) {
  static_assert(N % V == 0, "V must divide N");
  static_assert(num_stages(N, V) > 0, "no radix plan");
  Stage<N, V, 0, 1, INV, TRAIL>::run(v, sm, t, tw, bid);
}

}  // namespace fftenkf
