// Morphing transform around the FFT EnKF (Sec. 2.2, eq. morphing-transform and eq. inverse-morphing).
// The registration mappings T_k are inputs; these kernels compute
//   forward:   r_k^(j) = u_k^(j) o (I + T_k)^-1 - u_ref^(j)
//   reference: mean over the members of the extended state (T^a, r^a)
//   inverse:   u_k^(j),a = (u_ref^(j) + r_k^(j),a) o (I + T_k^a)
// on a periodic ny x nx grid with unit spacing.  f o (I + T) at node p is f(p + T(p)) with f
// interpolated bilinearly between nodes; (I + T)^-1(p) is the fixed point q = p - T(q), reached by
// n_iter steps from q = p.  Every point is kept as its node plus an FP32 offset d, so the
// interpolation weights carry the precision of the displacement, not of the grid coordinate.
//
// Layouts (row-major, x fastest): members u [M][K][ny][nx]; reference u_ref [M][ny][nx]; extended
// ensemble ext [M+2][K][ny][nx] = (T_x, T_y, r^(1), ..., r^(M)), the analysis layout with T_x, T_y and
// r^(1) as the observed blocks.  Gathers are local (|T| of a few cells), so L1 and L2 serve them.

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "../../include/fftenkf.h"

namespace fftenkf {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int kThreads = 256;
constexpr float kMaxOffset = 4194304.f;  // 2^22 cells: offsets are clamped to this for indexing
constexpr int kMaxIter = 1024;

fftenkf_status mfail(fftenkf_status s, const std::string& msg) {
  fftenkf::set_last_error(msg);
  return s;
}

// Bilinear stencil of node (y, x) displaced by (dy, dx) on the periodic grid.  Indexes always lie in
// the grid; a non-finite offset gives non-finite weights, so it shows in the output.  Plane offsets
// are 32-bit (ny * nx < 2^31).
struct Stencil {
  int r0, r1, x0, x1;   // row offsets y * nx and columns
  float wy, wx;
};

__device__ __forceinline__ void axis(int p, float d, int n, int& i0, int& i1, float& w) {
  const float dc = fminf(fmaxf(d, -kMaxOffset), kMaxOffset);
  const float f = floorf(dc);
  w = isfinite(d) ? dc - f : d - d;
  int i = p + (int)f;
  if ((unsigned)i >= (unsigned)n) {   // off the grid: wrap (rare for offsets of a few cells)
    i %= n;
    if (i < 0) i += n;
  }
  i0 = i;
  i1 = (i + 1 == n) ? 0 : i + 1;
}

__device__ __forceinline__ Stencil stencil(int y, int x, float dy, float dx, int ny, int nx) {
  Stencil s;
  int y0, y1;
  axis(y, dy, ny, y0, y1, s.wy);
  axis(x, dx, nx, s.x0, s.x1, s.wx);
  s.r0 = y0 * nx;
  s.r1 = y1 * nx;
  return s;
}

__device__ __forceinline__ float interp(const float* __restrict__ f, const Stencil& s) {
  const float f00 = __ldg(f + s.r0 + s.x0), f01 = __ldg(f + s.r0 + s.x1);
  const float f10 = __ldg(f + s.r1 + s.x0), f11 = __ldg(f + s.r1 + s.x1);
  return (1.f - s.wy) * ((1.f - s.wx) * f00 + s.wx * f01) + s.wy * ((1.f - s.wx) * f10 + s.wx * f11);
}

// grid (x: nodes of one plane, grid-stride; y: member k).  ext blocks 0, 1 (T) are read, blocks 2..
// (r) written.  The iteration stops after the first step that moves the point by at most tol cells
// in each component (tol = 0: once an iterate repeats exactly, which gives the result of all n_iter
// steps), else after n_iter steps.
__global__ void __launch_bounds__(kThreads, 4) morph_forward_kernel(const float* __restrict__ u,
                                                                 const float* __restrict__ u_ref,
                                                                 float* __restrict__ ext, int M, int K, int ny,
                                                                 int nx, int n_iter, float tol) {
  const int plane = ny * nx;
  const int k = blockIdx.y;
  const float* tx = ext + (size_t)k * plane;
  const float* ty = ext + ((size_t)K + k) * plane;
  for (int p = blockIdx.x * kThreads + threadIdx.x; p < plane; p += gridDim.x * kThreads) {
    const int y = p / nx, x = p - y * nx;
    float dy = 0.f, dx = 0.f;   // q_0 = p
    for (int it = 0; it < n_iter; ++it) {
      const Stencil s = stencil(y, x, dy, dx, ny, nx);
      const float ndx = -interp(tx, s);
      const float ndy = -interp(ty, s);
      const bool same = (fabsf(ndx - dx) <= tol) && (fabsf(ndy - dy) <= tol);
      dx = ndx;
      dy = ndy;
      if (same) break;
    }
    const Stencil s = stencil(y, x, dy, dx, ny, nx);
    for (int j = 0; j < M; ++j) {
      const float v = interp(u + ((size_t)j * K + k) * plane, s);
      ext[((size_t)(2 + j) * K + k) * plane + p] = v - __ldg(u_ref + (size_t)j * plane + p);
    }
  }
}

// ext_ref [C][ny][nx] = member mean of ext [C][K][ny][nx], summed in member order.
__global__ void __launch_bounds__(kThreads) morph_reference_kernel(const float* __restrict__ ext,
                                                                   float* __restrict__ ext_ref, int C, int K,
                                                                   size_t plane) {
  const size_t total = (size_t)C * plane;
  const float inv = 1.f / (float)K;
  for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < total; i += (size_t)gridDim.x * kThreads) {
    const size_t c = i / plane, p = i - c * plane;
    const float* e = ext + c * K * plane + p;
    float acc = 0.f;
    for (int k = 0; k < K; ++k) acc += __ldg(e + (size_t)k * plane);
    ext_ref[i] = acc * inv;
  }
}

// grid (x: nodes of one plane, grid-stride; y: member k): u_out[j][k](p) = (u_ref[j] + r[j][k]) at
// p + T_k(p).
__global__ void __launch_bounds__(kThreads, 8) morph_inverse_kernel(const float* __restrict__ ext,
                                                                 const float* __restrict__ u_ref,
                                                                 float* __restrict__ u_out, int M, int K, int ny,
                                                                 int nx) {
  const int plane = ny * nx;
  const int k = blockIdx.y;
  const float* tx = ext + (size_t)k * plane;
  const float* ty = ext + ((size_t)K + k) * plane;
  for (int p = blockIdx.x * kThreads + threadIdx.x; p < plane; p += gridDim.x * kThreads) {
    const int y = p / nx, x = p - y * nx;
    const Stencil s = stencil(y, x, __ldg(ty + p), __ldg(tx + p), ny, nx);
#pragma unroll 1   // 31 registers: 8 CTAs (2048 threads) per SM keep more gathers in flight
    for (int j = 0; j < M; ++j) {
      const float* g = u_ref + (size_t)j * plane;
      const float* r = ext + ((size_t)(2 + j) * K + k) * plane;
      const float f00 = __ldg(g + s.r0 + s.x0) + __ldg(r + s.r0 + s.x0);
      const float f01 = __ldg(g + s.r0 + s.x1) + __ldg(r + s.r0 + s.x1);
      const float f10 = __ldg(g + s.r1 + s.x0) + __ldg(r + s.r1 + s.x0);
      const float f11 = __ldg(g + s.r1 + s.x1) + __ldg(r + s.r1 + s.x1);
      u_out[((size_t)j * K + k) * plane + p] =
          (1.f - s.wy) * ((1.f - s.wx) * f00 + s.wx * f01) + s.wy * ((1.f - s.wx) * f10 + s.wx * f11);
    }
  }
}

// Launch shape of the per-member kernels: member k on grid.y and floor(resident / K) CTAs per member,
// so that every CTA is resident at once (one wave, no tail of a few CTAs each looping over its whole
// share of the plane).  resident = the SM count x the CTAs of 256 threads that fit on one SM, as the
// occupancy calculator gives them for the kernel (4 for the forward at 64 registers, 8 for the inverse
// at 32 on a 152-SM GB300).
template <typename K>
int resident_ctas(K kernel) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return sms * per_sm;
}
dim3 member_grid(int plane, int K, int resident) {
  int gx = resident / K;
  const int need = (plane + kThreads - 1) / kThreads;
  if (gx > need) gx = need;
  if (gx < 1) gx = 1;
  return dim3(gx, K);
}

int grid_for(size_t units, int resident) {
  const size_t g = (units + kThreads - 1) / kThreads;
  return (int)(g < (size_t)resident ? (g ? g : 1) : (size_t)resident);
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
  return pa < pb + nb && pb < pa + na;
}

fftenkf_status check_dims(const char* who, int M, int K, int ny, int nx) {
  if (M < 1 || K < 1 || ny < 1 || nx < 1)
    return mfail(FFTENKF_EINVAL, std::string(who) + ": n_blocks, n_members, ny, nx must be >= 1");
  if (K > 65535) return mfail(FFTENKF_EUNSUPPORTED, std::string(who) + ": n_members must be at most 65535");
  if ((long long)ny * nx > (1LL << 31) - (1LL << 20))
    return mfail(FFTENKF_EUNSUPPORTED, std::string(who) + ": ny * nx must be at most 2^31 - 2^20");
  return FFTENKF_OK;
}

bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3) == 0; }

fftenkf_status finish(const char* who) {
  const cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return mfail(FFTENKF_ECUDA, std::string(who) + ": launch failed: " + cudaGetErrorString(ce));
  return FFTENKF_OK;
}

}  // namespace

extern "C" fftenkf_status fftenkf_morph_forward(const float* u, const float* u_ref, float* ext, int n_blocks,
                                                int n_members, int ny, int nx, int n_iter, float tol,
                                                void* stream) {
  const char* who = "fftenkf_morph_forward";
  fftenkf_status st = check_dims(who, n_blocks, n_members, ny, nx);
  if (st != FFTENKF_OK) return st;
  if (!u || !u_ref || !ext || !aligned4(u) || !aligned4(u_ref) || !aligned4(ext))
    return mfail(FFTENKF_EINVAL, std::string(who) + ": null or misaligned pointer");
  if (n_iter < 0 || n_iter > kMaxIter) return mfail(FFTENKF_EINVAL, std::string(who) + ": n_iter must be in [0, 1024]");
  if (!(tol >= 0.f) || !std::isfinite(tol)) return mfail(FFTENKF_EINVAL, std::string(who) + ": tol must be finite and >= 0");
  const size_t plane = (size_t)ny * nx * sizeof(float);
  const size_t r_bytes = (size_t)n_blocks * n_members * plane;
  const float* r = ext + (size_t)2 * n_members * ny * nx;
  if (overlaps(r, r_bytes, u, r_bytes) || overlaps(r, r_bytes, u_ref, (size_t)n_blocks * plane) ||
      overlaps(r, r_bytes, ext, (size_t)2 * n_members * plane))
    return mfail(FFTENKF_EINVAL, std::string(who) + ": the residual blocks of ext overlap an input");
  morph_forward_kernel<<<member_grid(ny * nx, n_members, resident_ctas(morph_forward_kernel)), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      u, u_ref, ext, n_blocks, n_members, ny, nx, n_iter, tol);
  return finish(who);
}

extern "C" fftenkf_status fftenkf_morph_reference(const float* ext, float* ext_ref, int n_channels, int n_members,
                                                  int ny, int nx, void* stream) {
  const char* who = "fftenkf_morph_reference";
  fftenkf_status st = check_dims(who, n_channels, n_members, ny, nx);
  if (st != FFTENKF_OK) return st;
  if (!ext || !ext_ref || !aligned4(ext) || !aligned4(ext_ref))
    return mfail(FFTENKF_EINVAL, std::string(who) + ": null or misaligned pointer");
  const size_t plane = (size_t)ny * nx;
  if (overlaps(ext, (size_t)n_channels * n_members * plane * sizeof(float), ext_ref,
               (size_t)n_channels * plane * sizeof(float)))
    return mfail(FFTENKF_EINVAL, std::string(who) + ": ext_ref overlaps ext");
  morph_reference_kernel<<<grid_for((size_t)n_channels * plane, resident_ctas(morph_reference_kernel)), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      ext, ext_ref, n_channels, n_members, plane);
  return finish(who);
}

extern "C" fftenkf_status fftenkf_morph_inverse(const float* ext, const float* u_ref, float* u_out, int n_blocks,
                                                int n_members, int ny, int nx, void* stream) {
  const char* who = "fftenkf_morph_inverse";
  fftenkf_status st = check_dims(who, n_blocks, n_members, ny, nx);
  if (st != FFTENKF_OK) return st;
  if (!ext || !u_ref || !u_out || !aligned4(ext) || !aligned4(u_ref) || !aligned4(u_out))
    return mfail(FFTENKF_EINVAL, std::string(who) + ": null or misaligned pointer");
  const size_t plane = (size_t)ny * nx * sizeof(float);
  const size_t out_bytes = (size_t)n_blocks * n_members * plane;
  if (overlaps(u_out, out_bytes, ext, (size_t)(n_blocks + 2) * n_members * plane) ||
      overlaps(u_out, out_bytes, u_ref, (size_t)n_blocks * plane))
    return mfail(FFTENKF_EINVAL, std::string(who) + ": u_out overlaps an input");
  morph_inverse_kernel<<<member_grid(ny * nx, n_members, resident_ctas(morph_inverse_kernel)), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      ext, u_ref, u_out, n_blocks, n_members, ny, nx);
  return finish(who);
}
