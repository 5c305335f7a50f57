// Perturbations drawn by the method in frequency space (the seeded analysis):
// the unitary DFT of white N(0, 1) noise generated directly on the half
// spectrum from counter-based Philox4x32-10 words and Box-Muller pairs, scaled by
// sqrt(rhat) (eq. enkf: e_k ~ N(0, R), R = F* diag(rhat) F).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fftenkf {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of two 32 x 32 -> 64-bit
// products mixed with the other counter words and the key, the key advanced by the Weyl
// increments after every round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// One normal pair from two generator words: u = (w / 2^8 + 1/2) 2^-24 (single precision) and
// Box-Muller, sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b).  With the hardware approximations of
// log, sin and cos: -2 ln u_a is clamped at 0 (the approximation's absolute error, 2^-21 near
// u_a = 1, could make it negative), and cos 2 pi u_b = -cos t, sin 2 pi u_b = -sin t with
// t = 2 pi (u_b - 1/2) in [-pi, pi), where the approximations' absolute error is about 2^-21.
__device__ __forceinline__ float2 box_muller(uint32_t wa, uint32_t wb) {
  const float ua = ((float)(wa >> 8) + 0.5f) * 5.9604644775390625e-8f;
  const float ub = ((float)(wb >> 8) + 0.5f) * 5.9604644775390625e-8f;
  const float r = sqrtf(fmaxf(-2.f * __logf(ua), 0.f));
  float sn, cs;
  __sincosf(6.28318530717958647692f * (ub - 0.5f), &sn, &cs);
  return make_float2(-r * cs, -r * sn);
}

// zhat(k_y, k_x) of one stream in the columns k_x = 0 and L (Hermitian in k_y): counter
// (min(k_y, ny - k_y), k_x, stream, 0), words 0, 1; real N(0, 1) at the self-conjugate k_y,
// (n1 + i n2) / sqrt(2) otherwise, conjugated for k_y > ny/2.
__device__ __forceinline__ float2 white_edge(unsigned long long seed, int stream, int ky, int kx, int ny) {
  const int m = (ny - ky) % ny;
  const int kyc = ky < m ? ky : m;
  const uint4 w = philox4x32_10(make_uint4((uint32_t)kyc, (uint32_t)kx, (uint32_t)stream, 0u), (uint32_t)seed,
                                (uint32_t)(seed >> 32));
  const float2 n = box_muller(w.x, w.y);
  if (ky == 0 || 2 * ky == ny) return make_float2(n.x, 0.f);
  const float h = 0.70710678118654752f;
  return make_float2(n.x * h, (2 * ky > ny) ? -(n.y * h) : n.y * h);
}


}  // namespace fftenkf
